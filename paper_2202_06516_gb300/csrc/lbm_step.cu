// Fused multiphase LBM time step (Eq. 1-4, 7, 12-14 of arXiv:2202.06516), one launch per step.
//
// Stored state between steps, per fluid node z:
//   rho(z, t)                      density of the current (post-streaming) populations
//   h_q(z) = f*_q(z, t-1) - w_q rho(z, t)
// i.e. the post-collision populations of the previous step as deviations from the rest-state
// equilibrium w_q rho at the node's current density. Deviations are O(rho |u|) and O(f - f_eq),
// so FP32 keeps their relative precision in both phases although the liquid is ~145 times
// denser than the gas; the density itself is stored once per node.
//
// One CTA owns a TX x TY tile and stages, in shared memory:
//   rho, flags   tile + 7    (loaded)
//   wetting layers           first layer on tile + 6, second on tile + 5 (Eq. 14, recomputed
//                            from fluid densities, so no separate boundary kernel runs)
//   mu           tile + 3    (Eq. 12: k^2 psi'(rho) - kappa lap(rho) at fluid nodes, mu_w on the
//                            wetting layers; fourth-order stencils reach 2 nodes)
//   g*           tile + 1    (post-collision deviations from w_q rho(t), collision of Eq. 1 with
//                            force Eq. 7 and exact-difference forcing Eq. 13)
// and writes, for the tile only, rho(t+1) = sum_q f*_q(x - e_q) (pull streaming of Eq. 4 with
// half-way bounce-back on links into the solid) and the new deviations h. Collisions on the
// one-node ring are recomputed by the neighbouring CTAs; that redundancy buys a single pass over
// the populations per step (36 B read + 36 B written + 8 B of density per node in FP32).
#include "lbm_step_body.cuh"

namespace lbm {
namespace {

using namespace stepdev;

// the interpolated bounce-back kernels exist for the default variants only (32 x 16 tiles,
// 5 CTAs per SM in FP32, unconstrained in FP64)
template <typename T, int TX, int TY, int MINB>
constexpr bool has_ibb() {
    return TX == 32 && TY == 16 && MINB == (sizeof(T) == 4 ? 5 : 1);
}

template <typename T, int TX, int TY, int MINB>
cudaError_t configure_one() {
    using L = Layout<T, TX, TY>;
    cudaError_t e = cudaFuncSetAttribute(k_step<T, TX, TY, 256, false, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step<T, TX, TY, 256, true, MINB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
    if constexpr (has_ibb<T, TX, TY, MINB>()) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_step<T, TX, TY, 256, false, MINB, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_step<T, TX, TY, 256, true, MINB, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
    }
    return e;
}

template <typename T, int TX, int TY, int MINB>
cudaError_t launch_one(lbm_ctx* c, const StepArgs<T>& a, bool macro) {
    using L = Layout<T, TX, TY>;
    dim3 grid((c->nx + TX - 1) / TX, (c->ny + TY - 1) / TY);
    const T rho_mid = (T)(0.5 * (c->rho_g + c->rho_l));
    if (c->ibb) {
        if constexpr (has_ibb<T, TX, TY, MINB>()) {
            if (macro)
                k_step<T, TX, TY, 256, true, MINB, true><<<grid, 256, L::bytes, c->stream>>>(a, rho_mid);
            else
                k_step<T, TX, TY, 256, false, MINB, true><<<grid, 256, L::bytes, c->stream>>>(a,
                                                                                         rho_mid);
            return cudaGetLastError();
        }
        return cudaErrorInvalidValue;
    }
    if (macro)
        k_step<T, TX, TY, 256, true, MINB><<<grid, 256, L::bytes, c->stream>>>(a, rho_mid);
    else
        k_step<T, TX, TY, 256, false, MINB><<<grid, 256, L::bytes, c->stream>>>(a, rho_mid);
    return cudaGetLastError();
}

template <typename T>
StepArgs<T> make_args(lbm_ctx* c, int src) {
    StepArgs<T> a{};
    a.h_in = (const T*)c->h[src];
    a.h_out = (T*)c->h[src ^ 1];
    for (int q = 0; q < 9; ++q) {
        a.hq_in[q] = a.h_in + (size_t)q * c->plane;
        a.hq_out[q] = a.h_out + (size_t)q * c->plane;
    }
    a.rho_in = (const T*)c->rho[src];
    a.rho_out = (T*)c->rho[src ^ 1];
    a.flags = c->flags;
    a.muw = (const T*)c->muw;
    a.dlt = (const T*)c->dlt;
    a.vx = (T*)c->vel;
    a.vy = c->vel ? (T*)c->vel + c->plane : nullptr;
    a.nx = c->nx;
    a.ny = c->ny;
    a.P = c->P;
    a.plane = (int)c->plane;
    a.k2 = (T)c->p.k2;
    a.kappa = (T)c->p.kappa;
    a.gx = (T)c->p.gx;
    a.gy = (T)c->p.gy;
    a.gbx = (T)(-c->p.g_rho_ref * c->p.gx);
    a.gby = (T)(-c->p.g_rho_ref * c->p.gy);
    a.s_e = (T)c->p.s_e;
    a.s_eps = (T)c->p.s_eps;
    a.s_q = (T)c->p.s_q;
    a.s_v = (T)(1.0 / c->p.tau);
    a.inv_tau = (T)(1.0 / c->p.tau);
    a.bgk = c->p.collision == LBM_BGK;
    a.eos = c->eosc.eos;
    a.RT = (T)c->eosc.RT;
    a.aal = (T)c->eosc.aal;
    a.b = (T)c->eosc.b;
    return a;
}

}  // namespace

// Supported step-kernel variants: tile (TX, TY) and the minimum resident CTAs per SM the
// compiler is asked to fit (register budget); min_blocks 0 = no constraint.
#define LBM_STEP_VARIANTS(X)                                     \
    X(float, 32, 8, 1) X(float, 32, 8, 6) X(float, 32, 16, 1)    \
    X(float, 32, 16, 5) X(float, 32, 16, 6) X(float, 64, 16, 1)  \
    X(float, 32, 32, 1) X(double, 32, 8, 1) X(double, 32, 16, 1)

static int minb_of(lbm_ctx* c) { return c->min_blocks > 0 ? c->min_blocks : 1; }

size_t step_smem_bytes(int tx, int ty, size_t esz, int min_blocks) {
    const int mb = min_blocks > 0 ? min_blocks : 1;
#define X(T, A, B, M) \
    if (esz == sizeof(T) && tx == A && ty == B && mb == M) return Layout<T, A, B>::bytes;
    LBM_STEP_VARIANTS(X)
#undef X
    return 0;
}

bool step_has_ibb(size_t esz, int tx, int ty, int min_blocks) {
    return tx == 32 && ty == 16 && min_blocks == (esz == 4 ? 5 : 0);
}

void step_variants(size_t esz, std::vector<StepVariant>* out) {
    out->clear();
#define X(T, A, B, M) \
    if (esz == sizeof(T)) out->push_back(StepVariant{A, B, M == 1 ? 0 : M});
    LBM_STEP_VARIANTS(X)
#undef X
}

cudaError_t step_configure(lbm_ctx* c) {
#define X(T, A, B, M) \
    if (c->esz == sizeof(T) && c->tile_x == A && c->tile_y == B && minb_of(c) == M) \
        return configure_one<T, A, B, M>();
    LBM_STEP_VARIANTS(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_step(lbm_ctx* c, int src, bool macro) {
    if (c->esz == 4) {
        const StepArgs<float> a = make_args<float>(c, src);
#define X(T, A, B, M)                                                                 \
    if constexpr (sizeof(T) == 4)                                                     \
        if (c->tile_x == A && c->tile_y == B && minb_of(c) == M)                      \
            return launch_one<float, A, B, M>(c, a, macro);
        LBM_STEP_VARIANTS(X)
#undef X
    } else {
        const StepArgs<double> a = make_args<double>(c, src);
#define X(T, A, B, M)                                                                 \
    if constexpr (sizeof(T) == 8)                                                     \
        if (c->tile_x == A && c->tile_y == B && minb_of(c) == M)                      \
            return launch_one<double, A, B, M>(c, a, macro);
        LBM_STEP_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
