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
#include <math.h>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

// Bulk chemical potential psi'(rho) at k = 1: Eq. 11 without the gradient term (PR), or the CS
// counterpart from Eq. 9 with the ideal-gas antiderivative. The FP32 path uses the hardware
// logarithm and approximate division (relative error ~1e-6 on psi', far below the FP32 noise
// of the force); the FP64 path keeps correctly rounded operations.
template <typename T>
__device__ __forceinline__ T psi_prime(T rho, const StepArgs<T>& a);

template <>
__device__ __forceinline__ float psi_prime<float>(float rho, const StepArgs<float>& a) {
    if (a.eos == LBM_EOS_PR) {
        const float br = a.b * rho;
        const float s2 = 1.41421356f;
        const float inv = __fdividef(1.0f, 1.0f - br);
        const float t13 = a.RT * (__logf(rho * inv) + inv);
        const float t2 = a.aal * __fdividef(1.0f, 2.0f * s2 * a.b) *
                         __logf(__fdividef(s2 - 1.0f + br, s2 + 1.0f - br));
        const float t4 = __fdividef(a.aal * rho, 1.0f + 2.0f * br - br * br);
        return t13 - t2 - t4;
    }
    const float n = a.b * rho * 0.25f;
    const float om = 1.0f - n;
    return a.RT * (__logf(rho) + __fdividef(8.0f * n - 9.0f * n * n + 3.0f * n * n * n,
                                            om * om * om)) -
           2.0f * a.aal * rho;
}

template <>
__device__ __forceinline__ double psi_prime<double>(double rho, const StepArgs<double>& a) {
    if (a.eos == LBM_EOS_PR) {
        const double br = a.b * rho;
        const double s2 = 1.4142135623730951;
        const double t1 = a.RT * log(rho / (1.0 - br));
        const double t2 = a.aal / (2.0 * s2 * a.b) * log((s2 - 1.0 + br) / (s2 + 1.0 - br));
        const double t3 = a.RT / (1.0 - br);
        const double t4 = a.aal * rho / (1.0 + 2.0 * br - br * br);
        return t1 - t2 + t3 - t4;
    }
    const double n = a.b * rho * 0.25;
    const double om = 1.0 - n;
    return a.RT * (log(rho) + (8.0 * n - 9.0 * n * n + 3.0 * n * n * n) / (om * om * om)) -
           2.0 * a.aal * rho;
}

// Collision in deviation variables g_q = f_q - w_q rho, then exact-difference forcing.
// MRT: Lallemand-Luo moments (rho, e, eps, jx, qx, jy, qy, pxx, pxy); the equilibrium moments of
// Eq. 2 minus those of w_q rho are (0, 3 rho u^2, -3 rho u^2, jx, -jx, jy, -jy,
// rho (ux^2 - uy^2), rho ux uy). Relaxed moments are mapped back with M^-1 = M^T diag(1/|M_k|^2).
// Forcing (Eq. 13): F_q = f_eq(rho, u + F/rho) - f_eq(rho, u)
//                       = w_q [3 e.F + 4.5 (e.F)(e.s) - 1.5 F.s],  s = 2u + F/rho.
template <typename T>
__device__ __forceinline__ void collide(T g[9], T rho, T Fx, T Fy, const StepArgs<T>& a,
                                        T& ux, T& uy) {
    const T inv_rho = (T)1 / rho;
    const T jx = g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
    const T jy = g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
    ux = jx * inv_rho;
    uy = jy * inv_rho;
    const T uu = ux * ux + uy * uy;
    if (a.bgk) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const T eu = (T)qx(q) * ux + (T)qy(q) * uy;
            const T geq = rho * qw<T>(q) * ((T)3 * eu + (T)4.5 * eu * eu - (T)1.5 * uu);
            g[q] -= (g[q] - geq) * a.inv_tau;
        }
    } else {
        const T axis = g[1] + g[2] + g[3] + g[4];
        const T diag = g[5] + g[6] + g[7] + g[8];
        const T m1 = (T)-4 * g[0] - axis + (T)2 * diag;
        const T m2 = (T)4 * g[0] - (T)2 * axis + diag;
        const T m4 = (T)-2 * g[1] + (T)2 * g[3] + g[5] - g[6] - g[7] + g[8];
        const T m6 = (T)-2 * g[2] + (T)2 * g[4] + g[5] + g[6] - g[7] - g[8];
        const T m7 = g[1] - g[2] + g[3] - g[4];
        const T m8 = g[5] - g[6] + g[7] - g[8];
        const T a1 = a.s_e * (m1 - (T)3 * rho * uu) * ((T)1 / (T)36);
        const T a2 = a.s_eps * (m2 + (T)3 * rho * uu) * ((T)1 / (T)36);
        const T a4 = a.s_q * (m4 + jx) * ((T)1 / (T)12);
        const T a6 = a.s_q * (m6 + jy) * ((T)1 / (T)12);
        const T a7 = a.s_v * (m7 - rho * (ux * ux - uy * uy)) * (T)0.25;
        const T a8 = a.s_v * (m8 - rho * ux * uy) * (T)0.25;
        const T c_ax = -a1 - (T)2 * a2;
        const T c_dg = (T)2 * a1 + a2;
        g[0] -= (T)-4 * a1 + (T)4 * a2;
        g[1] -= c_ax - (T)2 * a4 + a7;
        g[2] -= c_ax - (T)2 * a6 - a7;
        g[3] -= c_ax + (T)2 * a4 + a7;
        g[4] -= c_ax + (T)2 * a6 - a7;
        g[5] -= c_dg + a4 + a6 + a8;
        g[6] -= c_dg - a4 + a6 - a8;
        g[7] -= c_dg - a4 - a6 + a8;
        g[8] -= c_dg + a4 - a6 - a8;
    }
    const T sx = (T)2 * ux + Fx * inv_rho, sy = (T)2 * uy + Fy * inv_rho;
    const T Fs = Fx * sx + Fy * sy;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const T eF = (T)qx(q) * Fx + (T)qy(q) * Fy;
        const T es = (T)qx(q) * sx + (T)qy(q) * sy;
        g[q] += qw<T>(q) * ((T)3 * eF + (T)4.5 * eF * es - (T)1.5 * Fs);
    }
}

template <typename T, int TX, int TY>
struct Layout {
    static constexpr int RW = TX + 16, RH = TY + 14;  // rho / flags: x0-8.., y0-7..
    static constexpr int MW = TX + 6, MH = TY + 6;    // mu: x0-3.., y0-3..
    static constexpr int CW = TX + 2, CH = TY + 2;    // g*: x0-1.., y0-1..
    static constexpr size_t bytes =
        sizeof(T) * ((size_t)RW * RH + (size_t)MW * MH + 9 * (size_t)CW * CH) + (size_t)RW * RH;
};

// four consecutive elements, global (aligned to 4 elements) to shared
__device__ __forceinline__ void load4(const float* g, float* s) {
    *reinterpret_cast<float4*>(s) = __ldg(reinterpret_cast<const float4*>(g));
}
__device__ __forceinline__ void load4(const double* g, double* s) {
    *reinterpret_cast<double2*>(s) = __ldg(reinterpret_cast<const double2*>(g));
    *reinterpret_cast<double2*>(s + 2) = __ldg(reinterpret_cast<const double2*>(g + 2));
}

template <typename T, int RW>
__device__ __forceinline__ T mu_fluid(const T* s_rho, int o, const StepArgs<T>& a) {
    const T c0 = s_rho[o];
    const T lapx = -s_rho[o + 2] + (T)16 * s_rho[o + 1] - (T)30 * c0 + (T)16 * s_rho[o - 1] -
                   s_rho[o - 2];
    const T lapy = -s_rho[o + 2 * RW] + (T)16 * s_rho[o + RW] - (T)30 * c0 +
                   (T)16 * s_rho[o - RW] - s_rho[o - 2 * RW];
    return a.k2 * psi_prime<T>(c0, a) - a.kappa * (lapx + lapy) * ((T)1 / (T)12);
}

// MIXED: the tile and its halo contain non-fluid nodes (walls, the disc, the domain edge), so
// wetting layers are rebuilt and every neighbour access checks the node class. Interior tiles
// take the branch-free path (the choice is uniform per CTA).
template <typename T, int TX, int TY, int NT, bool MACRO, bool MIXED>
__device__ __forceinline__ void step_body(const StepArgs<T>& a, const T rho_mid, T* s_rho,
                                          T* s_mu, T* s_g, const uint8_t* s_flag, int x0,
                                          int y0) {
    using L = Layout<T, TX, TY>;
    constexpr int RW = L::RW, RH = L::RH, MW = L::MW, MH = L::MH, CW = L::CW, CH = L::CH;
    const int tid = threadIdx.x;
    (void)RH;
    (void)rho_mid;

    if (MIXED) {
        // (2) first wetting layer (Eq. 14, switch on fluid neighbours)
        for (int idx = tid; idx < (RW - 2) * (RH - 2); idx += NT) {
            const int ly = 1 + idx / (RW - 2), lx = 1 + idx % (RW - 2);
            const int o = ly * RW + lx;
            if (s_flag[o] != kLayer1) continue;
            T num = 0, den = 0;
#pragma unroll
            for (int q = 1; q < 9; ++q) {
                const int on = o + qy(q) * RW + qx(q);
                if (s_flag[on] == kFluid) {
                    num += qw<T>(q) * s_rho[on];
                    den += qw<T>(q);
                }
            }
            s_rho[o] = den > (T)0 ? num / den : rho_mid;
        }
        __syncthreads();
        // (3) second wetting layer (switch on first-layer neighbours)
        for (int idx = tid; idx < (RW - 4) * (RH - 4); idx += NT) {
            const int ly = 2 + idx / (RW - 4), lx = 2 + idx % (RW - 4);
            const int o = ly * RW + lx;
            if (s_flag[o] != kLayer2) continue;
            T num = 0, den = 0;
#pragma unroll
            for (int q = 1; q < 9; ++q) {
                const int on = o + qy(q) * RW + qx(q);
                if (s_flag[on] == kLayer1) {
                    num += qw<T>(q) * s_rho[on];
                    den += qw<T>(q);
                }
            }
            s_rho[o] = den > (T)0 ? num / den : rho_mid;
        }
        __syncthreads();
    }

    // (4) chemical potential on tile + 3 (Eq. 12)
    for (int idx = tid; idx < MW * MH; idx += NT) {
        const int my = idx / MW, mx = idx - my * MW;
        const int o = (my + 4) * RW + (mx + 5);
        T mu;
        if (!MIXED) {
            mu = mu_fluid<T, RW>(s_rho, o, a);
        } else {
            const uint8_t f = s_flag[o];
            if (f == kFluid)
                mu = mu_fluid<T, RW>(s_rho, o, a);
            else if (f == kLayer1 || f == kLayer2)
                mu = a.muw[lidx(a.P, x0 - 3 + mx, y0 - 3 + my)];
            else
                mu = (T)0;
        }
        s_mu[idx] = mu;
    }
    __syncthreads();

    // (5) force and collision on tile + 1
    const T c12 = (T)1 / (T)12;
    for (int idx = tid; idx < CW * CH; idx += NT) {
        const int cy = idx / CW, cx = idx - cy * CW;
        const int o = (cy + 6) * RW + (cx + 7);
        if (MIXED && s_flag[o] != kFluid) continue;
        const int om = (cy + 2) * MW + (cx + 2);
        const int gx = x0 - 1 + cx, gy = y0 - 1 + cy;
        const int self = lidx(a.P, gx, gy);
        const T rho = s_rho[o];
        const T dmux = ((T)8 * (s_mu[om + 1] - s_mu[om - 1]) - (s_mu[om + 2] - s_mu[om - 2])) * c12;
        const T dmuy =
            ((T)8 * (s_mu[om + MW] - s_mu[om - MW]) - (s_mu[om + 2 * MW] - s_mu[om - 2 * MW])) * c12;
        const T drx = ((T)8 * (s_rho[o + 1] - s_rho[o - 1]) - (s_rho[o + 2] - s_rho[o - 2])) * c12;
        const T dry =
            ((T)8 * (s_rho[o + RW] - s_rho[o - RW]) - (s_rho[o + 2 * RW] - s_rho[o - 2 * RW])) * c12;
        const T Fx = -rho * dmux + drx * ((T)1 / (T)3) + rho * a.gx;
        const T Fy = -rho * dmuy + dry * ((T)1 / (T)3) + rho * a.gy;
        // pull the populations of time t (Eq. 4) with half-way bounce-back
        T g[9];
        g[0] = __ldg(a.h_in + self);
#pragma unroll
        for (int q = 1; q < 9; ++q) {
            const int os = o - qy(q) * RW - qx(q);
            if (!MIXED || s_flag[os] == kFluid) {
                const int src = self - qy(q) * a.P - qx(q);
                g[q] = __ldg(a.h_in + (size_t)q * a.plane + src) + qw<T>(q) * (s_rho[os] - rho);
            } else {
                g[q] = __ldg(a.h_in + (size_t)qopp(q) * a.plane + self);
            }
        }
        T ux, uy;
        collide<T>(g, rho, Fx, Fy, a, ux, uy);
        if (MACRO) {
            if (cx >= 1 && cx <= TX && cy >= 1 && cy <= TY && gx < a.nx && gy < a.ny) {
                a.vx[self] = ux + (T)0.5 * Fx / rho;
                a.vy[self] = uy + (T)0.5 * Fy / rho;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 9; ++q) s_g[q * CW * CH + idx] = g[q];
        }
    }
    if (MACRO) return;
    __syncthreads();

    // (6) streaming into the tile: new density and deviations (and their periodic images)
    for (int idx = tid; idx < TX * TY; idx += NT) {
        const int ty = idx / TX, tx = idx - ty * TX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (MIXED && (gx >= a.nx || gy >= a.ny)) continue;
        const int o = (ty + 7) * RW + (tx + 8);
        if (MIXED && s_flag[o] != kFluid) continue;
        const int oc = (ty + 1) * CW + (tx + 1);
        const T r0 = s_rho[o];
        T A = 0, B = 0;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int os = o - qy(q) * RW - qx(q);
            if (!MIXED || q == 0 || s_flag[os] == kFluid) {
                B += s_g[q * CW * CH + oc - qy(q) * CW - qx(q)];
                A += qw<T>(q) * s_rho[os];
            } else {
                B += s_g[qopp(q) * CW * CH + oc];
                A += qw<T>(q) * r0;
            }
        }
        const T r1 = A + B;
        const int self = lidx(a.P, gx, gy);
        const bool lo = gx < kPadX, hi = gx >= a.nx - kPadX;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const T v = s_g[q * CW * CH + oc] + qw<T>(q) * (r0 - r1);
            T* hq = a.h_out + (size_t)q * a.plane;
            hq[self] = v;
            if (lo) hq[self + a.nx] = v;
            if (hi) hq[self - a.nx] = v;
        }
        a.rho_out[self] = r1;
        if (lo) a.rho_out[self + a.nx] = r1;
        if (hi) a.rho_out[self - a.nx] = r1;
    }
}

template <typename T, int TX, int TY, int NT, bool MACRO, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_step(const StepArgs<T> a, const T rho_mid) {
    using L = Layout<T, TX, TY>;
    constexpr int RW = L::RW, RH = L::RH, MW = L::MW, MH = L::MH, CW = L::CW, CH = L::CH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s_rho = reinterpret_cast<T*>(smem_raw);
    T* s_mu = s_rho + RW * RH;
    T* s_g = s_mu + MW * MH;
    uint8_t* s_flag = reinterpret_cast<uint8_t*>(s_g + 9 * CW * CH);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

    // (1) density and flags on x0-8 .. x0+TX+7, y0-7 .. y0+TY+6, four nodes per access; the
    // pads supply periodic images and wall rows, positions past the padded plane read as solid
    constexpr int NV = RW / 4;
    int any = 0;
    for (int v = threadIdx.x; v < NV * RH; v += NT) {
        const int r = v / NV, c4 = v - r * NV;
        const int gy = y0 - 7 + r, gx = x0 - 8 + 4 * c4;
        T* sr = s_rho + r * RW + 4 * c4;
        uint32_t fl = 0x03030303u;
        if (gy >= -kPadY && gy < a.ny + kPadY && gx < a.nx + kPadX) {
            const int e = lidx(a.P, gx, gy);
            load4(a.rho_in + e, sr);
            fl = __ldg(reinterpret_cast<const unsigned int*>(a.flags + e));
        } else {
            sr[0] = sr[1] = sr[2] = sr[3] = (T)0;
        }
        *reinterpret_cast<uint32_t*>(s_flag + r * RW + 4 * c4) = fl;
        any |= fl != 0u;
    }
    if (__syncthreads_or(any))
        step_body<T, TX, TY, NT, MACRO, true>(a, rho_mid, s_rho, s_mu, s_g, s_flag, x0, y0);
    else
        step_body<T, TX, TY, NT, MACRO, false>(a, rho_mid, s_rho, s_mu, s_g, s_flag, x0, y0);
}

template <typename T, int TX, int TY, int MINB>
cudaError_t configure_one() {
    using L = Layout<T, TX, TY>;
    cudaError_t e = cudaFuncSetAttribute(k_step<T, TX, TY, 256, false, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_step<T, TX, TY, 256, true, MINB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
}

template <typename T, int TX, int TY, int MINB>
cudaError_t launch_one(lbm_ctx* c, const StepArgs<T>& a, bool macro) {
    using L = Layout<T, TX, TY>;
    dim3 grid((c->nx + TX - 1) / TX, (c->ny + TY - 1) / TY);
    const T rho_mid = (T)(0.5 * (c->rho_g + c->rho_l));
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
    a.rho_in = (const T*)c->rho[src];
    a.rho_out = (T*)c->rho[src ^ 1];
    a.flags = c->flags;
    a.muw = (const T*)c->muw;
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
    if (sizeof(T) == 4 && c->tile_x == A && c->tile_y == B && minb_of(c) == M) \
        return launch_one<float, A, B, M>(c, a, macro);
        LBM_STEP_VARIANTS(X)
#undef X
    } else {
        const StepArgs<double> a = make_args<double>(c, src);
#define X(T, A, B, M)                                                                 \
    if (sizeof(T) == 8 && c->tile_x == A && c->tile_y == B && minb_of(c) == M) \
        return launch_one<double, A, B, M>(c, a, macro);
        LBM_STEP_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
