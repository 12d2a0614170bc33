// C ABI of liblbm.so: context management, host-side coexistence solver and the orchestration of
// the device kernels (geometry, fused step, reductions, measurement). Declarations and contracts
// are in include/lbm.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "lbm_internal.cuh"
#include "lbm_trace.h"

namespace lbm {
size_t meas_partial_bytes(int nblocks);
}

namespace {

thread_local std::string g_last_error;

lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg) {
    if (c)
        c->err = msg;
    else
        g_last_error = msg;
    return s;
}

#define LBM_CUDA(ctx, expr)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail((ctx), LBM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------------------------------------
// Host equation of state (Eq. 10-11 for PR; CS with the ideal-gas antiderivative of Eq. 9) and
// the Maxwell construction. The coexistence is found by parametrising both stable branches by
// the chemical potential: for mu0 between the spinodal values, the gas and liquid densities with
// mu(rho) = mu0 are unique, and G(mu0) = p(rho_l) - p(rho_g) increases monotonically
// (dG/dmu0 = rho_l - rho_g by Gibbs-Duhem); its root is the equal-area coexistence.
// ---------------------------------------------------------------------------------------------
struct HostEos {
    int eos;
    double a, b, R, T, al;
    double rho_max() const { return eos == LBM_EOS_PR ? 1.0 / b : 4.0 / b; }
    double p(double r) const {
        if (eos == LBM_EOS_PR) {
            const double x = b * r;
            return r * R * T / (1.0 - x) - a * al * r * r / (1.0 + 2.0 * x - x * x);
        }
        const double n = 0.25 * b * r, m = 1.0 - n;
        return r * R * T * (1.0 + n + n * n - n * n * n) / (m * m * m) - a * r * r;
    }
    double mu(double r) const {
        if (eos == LBM_EOS_PR) {
            const double x = b * r, s = sqrt(2.0);
            return R * T * (log(r) - log(1.0 - x)) + R * T / (1.0 - x) -
                   a * al / (2.0 * s * b) * (log(s - 1.0 + x) - log(s + 1.0 - x)) -
                   a * al * r / (1.0 + 2.0 * x - x * x);
        }
        const double n = 0.25 * b * r, m = 1.0 - n;
        return R * T * (log(r) + n * (8.0 - 9.0 * n + 3.0 * n * n) / (m * m * m)) - 2.0 * a * r;
    }
};

bool make_eos(int eos, double Tr, HostEos* e) {
    e->eos = eos;
    if (eos == LBM_EOS_PR) {
        e->a = 2.0 / 49.0;
        e->b = 2.0 / 21.0;
        e->R = 1.0;
        const double Tc = 0.0778 / 0.45724 * e->a / (e->b * e->R);
        e->T = Tr * Tc;
        const double w = 0.344;
        const double m = 0.37464 + 1.54226 * w - 0.26992 * w * w;
        const double s = 1.0 + m * (1.0 - sqrt(Tr));
        e->al = s * s;
        return true;
    }
    if (eos == LBM_EOS_CS) {
        e->a = 1.0;
        e->b = 4.0;
        e->R = 1.0;
        e->T = Tr * 0.3773 * e->a / (e->b * e->R);
        e->al = 1.0;
        return true;
    }
    return false;
}

// density on a monotone branch [lo, hi] of mu with mu(rho) = target (bisection in log rho)
double branch_root(const HostEos& e, double lo, double hi, double target) {
    double l = log(lo), h = log(hi);
    for (int it = 0; it < 400 && h - l > 1e-16 * fabs(h); ++it) {
        const double m = 0.5 * (l + h);
        if (e.mu(exp(m)) < target)
            l = m;
        else
            h = m;
    }
    return exp(0.5 * (l + h));
}

bool coexistence(const HostEos& e, double out[4]) {
    // spinodals: local maximum of p (gas side) and local minimum (liquid side), located on a
    // logarithmic grid and refined by ternary search
    const int N = 4000;
    const double rmax = e.rho_max() * 0.9999;
    const double lo = rmax * 1e-7;
    std::vector<double> rr(N + 1), pp(N + 1);
    for (int k = 0; k <= N; ++k) {
        rr[k] = lo * pow(rmax / lo, (double)k / N);
        pp[k] = e.p(rr[k]);
    }
    int kmax = -1, kmin = -1;
    for (int k = 1; k < N; ++k) {
        if (kmax < 0 && pp[k] >= pp[k - 1] && pp[k] > pp[k + 1]) kmax = k;
        if (kmax >= 0 && k > kmax && pp[k] <= pp[k - 1] && pp[k] < pp[k + 1]) {
            kmin = k;
            break;
        }
    }
    if (kmax < 0 || kmin < 0) return false;
    auto refine = [&](int k, bool maximum) {
        double a = rr[k - 1], b = rr[k + 1];
        for (int it = 0; it < 200; ++it) {
            const double m1 = a + (b - a) / 3.0, m2 = b - (b - a) / 3.0;
            const bool left = maximum ? (e.p(m1) > e.p(m2)) : (e.p(m1) < e.p(m2));
            if (left)
                b = m2;
            else
                a = m1;
        }
        return 0.5 * (a + b);
    };
    const double rs1 = refine(kmax, true), rs2 = refine(kmin, false);
    double mlo = e.mu(rs2), mhi = e.mu(rs1);
    if (!(mlo < mhi)) return false;
    double rg = 0, rl = 0;
    for (int it = 0; it < 200; ++it) {
        const double m0 = 0.5 * (mlo + mhi);
        rg = branch_root(e, lo * 1e-30 > 0 ? lo * 1e-30 : 1e-300, rs1, m0);
        rl = branch_root(e, rs2, rmax, m0);
        if (e.p(rl) - e.p(rg) > 0)
            mhi = m0;
        else
            mlo = m0;
        if (mhi - mlo <= 1e-17 * fabs(mhi)) break;
    }
    const double m0 = 0.5 * (mlo + mhi);
    rg = branch_root(e, 1e-300, rs1, m0);
    rl = branch_root(e, rs2, rmax, m0);
    out[0] = rg;
    out[1] = rl;
    out[2] = 0.5 * (e.p(rg) + e.p(rl));
    out[3] = m0;
    return true;
}

bool half_integral(double v) { return fabs(2.0 * v - nearbyint(2.0 * v)) < 1e-9; }

void destroy_graphs(lbm_ctx* c) {
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < lbm::kGraphSizes; ++k) {
            if (c->graph[p][k]) cudaGraphExecDestroy(c->graph[p][k]);
            c->graph[p][k] = nullptr;
        }
    c->graphs_ready = false;
}

void free_all(lbm_ctx* c) {
    destroy_graphs(c);
    for (int k = 0; k < 2; ++k) {
        cudaFree(c->h[k]);
        cudaFree(c->rho[k]);
        c->h[k] = c->rho[k] = nullptr;
    }
    cudaFree(c->muw);
    cudaFree(c->flags);
    cudaFree(c->linkmask);
    cudaFree(c->dlt);
    c->dlt = nullptr;
    cudaFree(c->red_partials);
    cudaFree(c->red_out);
    cudaFree(c->meas_partials);
    cudaFree(c->meas_out);
    cudaFree(c->vel);
    cudaFree(c->stage);
    c->stage = nullptr;
    c->muw = c->vel = c->meas_partials = nullptr;
    c->flags = c->linkmask = nullptr;
    c->red_partials = nullptr;
    c->red_out = nullptr;
    c->meas_out = nullptr;
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    c->stream = nullptr;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

// Capture the step graphs of every size for both starting buffers, once per variant and
// geometry: a later lbm_step of any length then runs as a few graph launches (largest first) and
// at most one single launch, with no capture inside it. On any capture failure the context falls
// back to single launches for good.
lbm_status capture_graphs(lbm_ctx* c) {
    if (c->graph_failed || c->graphs_ready) return LBM_OK;
    for (int start = 0; start < 2; ++start)
        for (int k = 0; k < lbm::kGraphSizes; ++k) {
            const int n = lbm::kGraphChunk >> k;
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) !=
                cudaSuccess) {
                cudaGetLastError();
                c->graph_failed = true;
                destroy_graphs(c);
                return LBM_OK;
            }
            int cur = start;
            cudaError_t le = cudaSuccess;
            for (int s = 0; s < n; ++s) {
                cudaError_t e = lbm::launch_step(c, cur, false);
                if (e != cudaSuccess && le == cudaSuccess) le = e;
                cur ^= 1;
            }
            cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
            cudaError_t ie = cudaErrorUnknown;
            if (le == cudaSuccess && ee == cudaSuccess && g)
                ie = cudaGraphInstantiate(&c->graph[start][k], g, 0);
            // move the one-time device upload here, out of the first lbm_step that uses it
            if (ie == cudaSuccess) ie = cudaGraphUpload(c->graph[start][k], c->stream);
            if (g) cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                cudaGetLastError();
                c->graph[start][k] = nullptr;
                c->graph_failed = true;
                destroy_graphs(c);
                return LBM_OK;
            }
        }
    c->graphs_ready = true;
    return LBM_OK;
}

}  // namespace

namespace lbm {
// message for lbm_last_error(NULL) from entry points outside this file
void set_global_error(const std::string& msg) { g_last_error = msg; }
}  // namespace lbm

extern "C" {

lbm_status lbm_coexistence(int32_t eos, double Tr, double out[4]) {
    HostEos e;
    if (!out) return fail(nullptr, LBM_ERR_ARG, "lbm_coexistence: out is NULL");
    if (!make_eos(eos, Tr, &e)) return fail(nullptr, LBM_ERR_ARG, "lbm_coexistence: unknown EOS");
    if (!(Tr > 0.0 && Tr < 1.0) || !coexistence(e, out))
        return fail(nullptr, LBM_ERR_ARG, "lbm_coexistence: no coexistence at this temperature");
    return LBM_OK;
}

lbm_status lbm_eos_eval(int32_t eos, double Tr, double rho, double out[2]) {
    HostEos e;
    if (!out) return fail(nullptr, LBM_ERR_ARG, "lbm_eos_eval: out is NULL");
    if (!make_eos(eos, Tr, &e)) return fail(nullptr, LBM_ERR_ARG, "lbm_eos_eval: unknown EOS");
    if (!(Tr > 0.0 && Tr < 1.0))
        return fail(nullptr, LBM_ERR_ARG, "lbm_eos_eval: Tr must lie in (0, 1)");
    if (!(rho > 0.0 && rho < e.rho_max()))
        return fail(nullptr, LBM_ERR_ARG, "lbm_eos_eval: rho outside (0, rho_max)");
    out[0] = e.p(rho);
    out[1] = e.mu(rho);
    return LBM_OK;
}

lbm_status lbm_create(const lbm_params* p, lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "lbm_create: out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, LBM_ERR_ARG, "lbm_create: params is NULL");
    if (p->nx < 8 || p->ny < 8 || p->nx > (1 << 20) || p->ny > (1 << 20))
        return fail(nullptr, LBM_ERR_ARG, "lbm_create: nx and ny must lie in [8, 2^20]");
    if (p->precision != LBM_FP32 && p->precision != LBM_FP64)
        return fail(nullptr, LBM_ERR_ARG, "lbm_create: precision must be LBM_FP32 or LBM_FP64");
    if (p->collision != LBM_MRT && p->collision != LBM_BGK)
        return fail(nullptr, LBM_ERR_ARG, "lbm_create: collision must be LBM_MRT or LBM_BGK");
    if (!(p->tau > 0.5) || !(p->k2 > 0) || !(p->kappa >= 0))
        return fail(nullptr, LBM_ERR_ARG, "lbm_create: need tau > 1/2, k2 > 0, kappa >= 0");
    HostEos he;
    if (!make_eos(p->eos, p->Tr, &he)) return fail(nullptr, LBM_ERR_ARG, "lbm_create: unknown EOS");
    double co[4];
    if (!(p->Tr > 0 && p->Tr < 1) || !coexistence(he, co))
        return fail(nullptr, LBM_ERR_ARG, "lbm_create: no coexistence at this Tr");
    const bool tile_auto = p->tile_x == LBM_TILE_AUTO;
    const bool tile_default = tile_auto || (!p->tile_x && !p->tile_y && !p->min_blocks);
    const int tx = tile_default || !p->tile_x ? 32 : p->tile_x;
    const int ty = tile_default || !p->tile_y ? 16 : p->tile_y;
    const size_t esz = p->precision == LBM_FP32 ? 4 : 8;
    // default variant: FP32 32x16 fitted to 5 CTAs per SM (measured fastest on GB300)
    const int min_blocks = tile_default ? (esz == 4 ? 5 : 0) : p->min_blocks;
    if (lbm::step_smem_bytes(tx, ty, esz, min_blocks) == 0)
        return fail(nullptr, LBM_ERR_ARG,
                    "lbm_create: unsupported (tile, min_blocks) variant for this precision");
    {
        const long long P = (p->nx + 2 * lbm::kPadX + 31) / 32 * 32;
        if (9 * P * (p->ny + 2 * lbm::kPadY + 1) >= (1LL << 31))
            return fail(nullptr, LBM_ERR_ARG, "lbm_create: lattice too large (plane >= 2^31 nodes)");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, LBM_ERR_CUDA, "lbm_create: no CUDA device");
    }
    if (p->device < 0 || p->device >= ndev)
        return fail(nullptr, LBM_ERR_ARG, "lbm_create: device ordinal out of range");

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_create: out of host memory");
    DeviceGuard dg(p->device);
    c->p = *p;
    c->device = p->device;
    c->nx = p->nx;
    c->ny = p->ny;
    c->P = (p->nx + 2 * lbm::kPadX + 31) / 32 * 32;
    // one slack row past the last pad row: the step kernel's 4-wide halo loads may start up to
    // 3 columns before the end of a padded row
    c->plane = (size_t)(c->ny + 2 * lbm::kPadY + 1) * c->P;
    c->esz = esz;
    c->tile_x = tx;
    c->tile_y = ty;
    c->min_blocks = min_blocks;
    c->autotune_pending = tile_auto;
    c->eosc.eos = p->eos;
    c->eosc.RT = he.R * he.T;
    c->eosc.aal = he.a * he.al;
    c->eosc.b = he.b;
    c->T = he.T;
    c->rho_g = p->rho_g > 0 ? p->rho_g : co[0];
    c->rho_l = p->rho_l > 0 ? p->rho_l : co[1];
    c->p_sat = co[2];
    c->mu_sat = co[3];
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    c->red_blocks = 2 * sms;

    auto cleanup = [&](const std::string& msg) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return fail(nullptr, LBM_ERR_CUDA, msg);
    };
    cudaError_t e = cudaSuccess;
    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cleanup(std::string("stream: ") + cudaGetErrorString(e));
        c->own_stream = true;
    }
    const size_t hbytes = 9 * c->plane * esz;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&c->h[k], hbytes);
        if (e == cudaSuccess) e = cudaMalloc(&c->rho[k], c->plane * esz);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->muw, c->plane * esz);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->flags, c->plane);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->linkmask, c->plane);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->red_partials, sizeof(double) * 8 * c->red_blocks);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->red_out, sizeof(lbm::ReduceOut));
    if (e == cudaSuccess) e = cudaMalloc(&c->meas_partials, lbm::meas_partial_bytes(c->red_blocks));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->meas_out, 2 * sizeof(lbm_angle));
    if (e == cudaSuccess) e = lbm::step_configure(c);
    if (e != cudaSuccess) return cleanup(std::string("lbm_create: ") + cudaGetErrorString(e));
    *out = c;
    return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx* c, const lbm_geometry* g) {
    lbm::NvtxRange nvtx_("lbm_set_geometry");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_set_geometry: ctx is NULL");
    if (!g) return fail(c, LBM_ERR_ARG, "lbm_set_geometry: geometry is NULL");
    if (g->has_circle && (!half_integral(g->cx) || !half_integral(g->cy) || !half_integral(g->R) ||
                          !(g->R > 0)))
        return fail(c, LBM_ERR_ARG, "lbm_set_geometry: circle centre and radius must be positive "
                                    "multiples of 1/2");
    if (g->stripes && !(g->stripe_arc > 0))
        return fail(c, LBM_ERR_ARG, "lbm_set_geometry: stripe_arc must be positive");
    if (!g->rho0 && !(g->drop_W > 0))
        return fail(c, LBM_ERR_ARG, "lbm_set_geometry: drop_W must be positive");
    if (g->boundary != LBM_BB_HALFWAY && g->boundary != LBM_BB_INTERP)
        return fail(c, LBM_ERR_ARG, "lbm_set_geometry: boundary must be LBM_BB_HALFWAY or "
                                    "LBM_BB_INTERP");
    DeviceGuard dg(c->device);
    // the walls (classes, wetting layers, wall potentials, links) depend on these fields only;
    // the drop and rho0 set the initial state
    const lbm_geometry& o = c->geom;
    const bool same_walls = c->has_geometry && o.has_circle == g->has_circle &&
                            o.stripes == g->stripes && o.cx == g->cx && o.cy == g->cy &&
                            o.R == g->R && o.mu_circle == g->mu_circle &&
                            o.stripe_arc == g->stripe_arc && o.mu_stripe_b == g->mu_stripe_b &&
                            o.mu_bottom == g->mu_bottom && o.mu_top == g->mu_top &&
                            o.concave == g->concave && o.boundary == g->boundary;
    lbm::GeomArgs a{};
    a.nx = c->nx;
    a.ny = c->ny;
    a.P = c->P;
    a.plane = (int)c->plane;
    a.has_circle = g->has_circle;
    a.stripes = g->stripes;
    a.concave = g->has_circle && g->concave;
    a.cx2 = llround(2.0 * g->cx);
    a.cy2 = llround(2.0 * g->cy);
    a.r2 = llround(2.0 * g->R);
    a.cx = g->cx;
    a.cy = g->cy;
    a.R = g->R;
    a.stripe_arc = g->stripe_arc;
    a.mu_circle = g->mu_circle;
    a.mu_stripe_b = g->mu_stripe_b;
    a.mu_bottom = g->mu_bottom;
    a.mu_top = g->mu_top;
    if (!same_walls) {
        c->has_geometry = false;  // until the new walls are complete
        LBM_CUDA(c, cudaMemsetAsync(c->flags, lbm::kSolid, c->plane, c->stream));
        LBM_CUDA(c, cudaMemsetAsync(c->muw, 0, c->plane * c->esz, c->stream));
        LBM_CUDA(c, cudaMemsetAsync(c->linkmask, 0, c->plane, c->stream));
        LBM_CUDA(c, lbm::launch_geometry(c, a));
    }
    // captured step graphs stay valid across geometries (the kernels read the same buffers);
    // they hold the boundary scheme and the variant, so a change of either drops them
    const bool ibb = g->boundary == LBM_BB_INTERP;
    if (ibb != c->ibb) destroy_graphs(c);
    c->ibb = ibb;
    if (c->ibb && !same_walls) {
        if (!c->dlt) {
            destroy_graphs(c);
            LBM_CUDA(c, cudaMalloc(&c->dlt, 8 * c->plane * c->esz));
        }
        LBM_CUDA(c, lbm::launch_link_fractions(c, a));
        // the interpolated scheme is compiled for the default tile variant only
        if (!lbm::step_has_ibb(c->esz, c->tile_x, c->tile_y, c->min_blocks)) {
            destroy_graphs(c);
            c->tile_x = 32;
            c->tile_y = 16;
            c->min_blocks = c->esz == 4 ? 5 : 0;
            LBM_CUDA(c, lbm::step_configure(c));
        }
    }
    if (g->rho0) {
        const size_t nb = sizeof(double) * (size_t)c->nx * c->ny;
        if (!c->stage) LBM_CUDA(c, cudaMalloc((void**)&c->stage, nb));
        cudaError_t e = cudaMemcpyAsync(c->stage, g->rho0, nb, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = lbm::launch_init_state(c, *g, c->stage);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
            return fail(c, LBM_ERR_CUDA, std::string("lbm_set_geometry: ") + cudaGetErrorString(e));
    } else {
        LBM_CUDA(c, lbm::launch_init_state(c, *g, nullptr));
    }
    c->geom = *g;
    c->geom.rho0 = nullptr;
    c->sub.circle = g->has_circle ? 1 : 0;
    c->sub.concave = g->has_circle && g->concave ? 1 : 0;
    c->sub.cx = g->cx;
    c->sub.cy = g->cy;
    // the wall surface: half a link beyond the solid nodes (both boundary schemes)
    c->sub.Rs = g->R + 0.5;
    c->cur = 0;
    c->steps = 0;
    c->has_geometry = true;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int64_t nsteps) {
    lbm::NvtxRange nvtx_("lbm_step");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_step: ctx is NULL");
    if (nsteps < 0) return fail(c, LBM_ERR_ARG, "lbm_step: nsteps < 0");
    if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "lbm_step: call lbm_set_geometry first");
    DeviceGuard dg(c->device);
    if (c->autotune_pending && nsteps > 0) {
        c->autotune_pending = false;
        const lbm_status st = lbm_autotune(c, lbm::kAutotuneTrial, nullptr, 0, nullptr);
        if (st != LBM_OK) return st;
    }
    int64_t left = nsteps;
    if (c->ibb && c->steps == 0 && left > 0) {
        // the initial populations are f = w rho0 themselves (the stored state encodes them for
        // half-way pulls): nothing has come back from a wall yet, so the first step pulls
        // without interpolation
        c->ibb = false;
        const cudaError_t e = lbm::launch_step(c, c->cur, false);
        c->ibb = true;
        LBM_CUDA(c, e);
        c->cur ^= 1;
        --left;
    }
    if (left >= 2 && !c->graphs_ready && !c->graph_failed) capture_graphs(c);
    for (int k = 0; c->graphs_ready && k < lbm::kGraphSizes; ++k) {
        const int n = lbm::kGraphChunk >> k;
        while (left >= n) {
            LBM_CUDA(c, cudaGraphLaunch(c->graph[c->cur][k], c->stream));
            left -= n;  // even chunk: parity of c->cur unchanged
        }
    }
    for (; left > 0; --left) {
        LBM_CUDA(c, lbm::launch_step(c, c->cur, false));
        c->cur ^= 1;
    }
    c->steps += nsteps;
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx* c, int32_t trial_steps, lbm_tune_entry* entries,
                        int32_t max_entries, int32_t* n_out) {
    lbm::NvtxRange nvtx_("lbm_autotune");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_autotune: ctx is NULL");
    if (trial_steps < 1) return fail(c, LBM_ERR_ARG, "lbm_autotune: trial_steps < 1");
    if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "lbm_autotune: call lbm_set_geometry first");
    DeviceGuard dg(c->device);
    std::vector<lbm::StepVariant> vs;
    lbm::step_variants(c->esz, &vs);
    if (c->ibb) {  // interpolated bounce-back: only the variants compiled with it
        std::vector<lbm::StepVariant> keep_ibb;
        for (const auto& v : vs)
            if (lbm::step_has_ibb(c->esz, v.tile_x, v.tile_y, v.min_blocks)) keep_ibb.push_back(v);
        vs.swap(keep_ibb);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LBM_CUDA(c, cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        LBM_CUDA(c, ce);
    }
    const lbm::StepVariant keep{c->tile_x, c->tile_y, c->min_blocks};
    int best = -1;
    double best_us = 0;
    cudaError_t err = cudaSuccess;
    for (size_t i = 0; i < vs.size() && err == cudaSuccess; ++i) {
        c->tile_x = vs[i].tile_x;
        c->tile_y = vs[i].tile_y;
        c->min_blocks = vs[i].min_blocks;
        err = lbm::step_configure(c);
        // every launch reads buffer cur and writes buffer cur ^ 1: the state does not advance
        for (int w = 0; w < 2 && err == cudaSuccess; ++w) err = lbm::launch_step(c, c->cur, false);
        if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
        for (int s = 0; s < trial_steps && err == cudaSuccess; ++s)
            err = lbm::launch_step(c, c->cur, false);
        if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) break;
        const double us = 1e3 * (double)ms / trial_steps;
        if (entries && (int32_t)i < max_entries)
            entries[i] = lbm_tune_entry{vs[i].tile_x, vs[i].tile_y, vs[i].min_blocks, us};
        if (best < 0 || us < best_us) {
            best = (int)i;
            best_us = us;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const lbm::StepVariant pick = (err == cudaSuccess && best >= 0) ? vs[best] : keep;
    c->tile_x = pick.tile_x;
    c->tile_y = pick.tile_y;
    c->min_blocks = pick.min_blocks;
    LBM_CUDA(c, err);
    LBM_CUDA(c, lbm::step_configure(c));
    // the captured graphs hold the previous variant
    destroy_graphs(c);
    if (n_out) *n_out = (int32_t)vs.size();
    return LBM_OK;
}

lbm_status lbm_measure_contact_angle(lbm_ctx* c, lbm_angle out[2]) {
    lbm::NvtxRange nvtx_("lbm_measure_contact_angle");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_measure_contact_angle: ctx is NULL");
    if (!out) return fail(c, LBM_ERR_ARG, "lbm_measure_contact_angle: out is NULL");
    if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "lbm_measure_contact_angle: no geometry");
    DeviceGuard dg(c->device);
    LBM_CUDA(c, lbm::launch_measure(c));
    LBM_CUDA(c, cudaMemcpyAsync(out, c->meas_out, 2 * sizeof(lbm_angle), cudaMemcpyDeviceToHost,
                                c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (out[0].status != LBM_OK || out[1].status != LBM_OK)
        return fail(c, LBM_ERR_NO_CONTACT, "lbm_measure_contact_angle: a side has no contact");
    return LBM_OK;
}

lbm_status lbm_mass(lbm_ctx* c, double out[4]) {
    lbm::NvtxRange nvtx_("lbm_mass");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_mass: ctx is NULL");
    if (!out) return fail(c, LBM_ERR_ARG, "lbm_mass: out is NULL");
    if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "lbm_mass: no geometry");
    DeviceGuard dg(c->device);
    lbm::ReduceOut r{};
    LBM_CUDA(c, lbm::launch_reduce(c));
    LBM_CUDA(c, cudaMemcpyAsync(&r, c->red_out, sizeof r, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    out[0] = r.mass;
    out[1] = r.n_liquid;
    out[2] = r.sx;
    out[3] = r.sy;
    if (r.bad > 0) return fail(c, LBM_ERR_UNSTABLE, "lbm_mass: non-finite or non-positive density");
    return LBM_OK;
}

lbm_status lbm_read_fields(lbm_ctx* c, uint32_t which, double* rho, double* ux, double* uy,
                           size_t n) {
    lbm::NvtxRange nvtx_("lbm_read_fields");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_read_fields: ctx is NULL");
    if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "lbm_read_fields: no geometry");
    const size_t N = (size_t)c->nx * c->ny;
    if (n != N) return fail(c, LBM_ERR_ARG, "lbm_read_fields: n must equal nx * ny");
    if (((which & LBM_FIELD_RHO) && !rho) || ((which & LBM_FIELD_VEL) && (!ux || !uy)))
        return fail(c, LBM_ERR_ARG, "lbm_read_fields: NULL buffer for a requested field");
    DeviceGuard dg(c->device);
    const bool dev = (which & LBM_FIELD_DEVICE_DST) != 0;
    if (!dev && !c->stage) LBM_CUDA(c, cudaMalloc((void**)&c->stage, sizeof(double) * N));
    double* tmp = dev ? nullptr : c->stage;
    auto emit = [&](const void* src, double* dst) -> cudaError_t {
        double* target = dev ? dst : tmp;
        cudaError_t e = lbm::launch_to_double(c, src, target, 0);
        if (e == cudaSuccess && !dev)
            e = cudaMemcpyAsync(dst, tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && !dev) e = cudaStreamSynchronize(c->stream);
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (which & LBM_FIELD_RHO) e = emit(c->rho[c->cur], rho);
    if (e == cudaSuccess && (which & LBM_FIELD_VEL)) {
        if (!c->vel) e = cudaMalloc(&c->vel, 2 * c->plane * c->esz);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->vel, 0, 2 * c->plane * c->esz, c->stream);
        if (e == cudaSuccess) e = lbm::launch_step(c, c->cur, true);
        if (e == cudaSuccess) e = emit(c->vel, ux);
        if (e == cudaSuccess) e = emit((const char*)c->vel + c->plane * c->esz, uy);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return fail(c, LBM_ERR_CUDA, std::string("lbm_read_fields: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_read_geometry(lbm_ctx* c, uint8_t* flags, double* mu_w, int64_t* links,
                             int64_t cap, int64_t* n_links) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_read_geometry: ctx is NULL");
    if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "lbm_read_geometry: no geometry");
    DeviceGuard dg(c->device);
    const int nx = c->nx, rows = c->ny + 4;
    const size_t o_ext = (size_t)lbm::lidx(c->P, 0, -2), o_dom = (size_t)lbm::lidx(c->P, 0, 0);
    if (flags)
        LBM_CUDA(c, cudaMemcpy2DAsync(flags, nx, c->flags + o_ext, c->P, nx, rows,
                                      cudaMemcpyDeviceToHost, c->stream));
    std::vector<unsigned char> mw;
    if (mu_w) {
        mw.resize((size_t)rows * nx * c->esz);
        LBM_CUDA(c, cudaMemcpy2DAsync(mw.data(), nx * c->esz, (const char*)c->muw + o_ext * c->esz,
                                      c->P * c->esz, nx * c->esz, rows, cudaMemcpyDeviceToHost,
                                      c->stream));
    }
    std::vector<uint8_t> lm;
    if (links || n_links) {
        lm.resize((size_t)c->ny * nx);
        LBM_CUDA(c, cudaMemcpy2DAsync(lm.data(), nx, c->linkmask + o_dom, c->P, nx, c->ny,
                                      cudaMemcpyDeviceToHost, c->stream));
    }
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (mu_w)
        for (size_t k = 0; k < (size_t)rows * nx; ++k)
            mu_w[k] = c->esz == 4 ? (double)((const float*)mw.data())[k] : ((const double*)mw.data())[k];
    if (links || n_links) {
        int64_t k = 0;
        for (size_t n = 0; n < lm.size(); ++n)
            for (int q = 1; q < 9; ++q)
                if (lm[n] & (1u << (q - 1))) {
                    if (links && k < cap) links[k] = (int64_t)n * 9 + q;
                    ++k;
                }
        if (n_links) *n_links = k;
    }
    return LBM_OK;
}

lbm_status lbm_read_candidates(lbm_ctx* c, int64_t* ids, double* pxyd, int64_t cap, int64_t* n) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_read_candidates: ctx is NULL");
    if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "lbm_read_candidates: no geometry");
    DeviceGuard dg(c->device);
    const size_t N4 = (size_t)c->nx * c->ny * 4;
    uint8_t* d_mark = nullptr;
    double* d_p = nullptr;
    LBM_CUDA(c, cudaMalloc((void**)&d_mark, N4));
    cudaError_t e = cudaMalloc((void**)&d_p, N4 * 3 * sizeof(double));
    std::vector<uint8_t> mark(N4);
    std::vector<double> pts(N4 * 3);
    if (e == cudaSuccess) e = lbm::launch_candidates(c, d_mark, d_p);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mark.data(), d_mark, N4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pts.data(), d_p, N4 * 3 * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_mark);
    cudaFree(d_p);
    if (e != cudaSuccess)
        return fail(c, LBM_ERR_CUDA, std::string("lbm_read_candidates: ") + cudaGetErrorString(e));
    int64_t k = 0;
    for (size_t m = 0; m < N4; ++m) {
        if (!mark[m]) continue;
        if (k < cap) {
            if (ids) ids[k] = (int64_t)m;
            if (pxyd)
                for (int t = 0; t < 3; ++t) pxyd[3 * k + t] = pts[3 * m + t];
        }
        ++k;
    }
    if (n) *n = k;
    return LBM_OK;
}

lbm_status lbm_get_info(lbm_ctx* c, lbm_info* out) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_get_info: ctx is NULL");
    if (!out) return fail(c, LBM_ERR_ARG, "lbm_get_info: out is NULL");
    out->rho_g = c->rho_g;
    out->rho_l = c->rho_l;
    out->p_sat = c->p_sat;
    out->mu_sat = c->mu_sat;
    out->T = c->T;
    out->steps = c->steps;
    out->n_fluid = c->n_fluid;
    out->tile_x = c->tile_x;
    out->tile_y = c->tile_y;
    out->precision = c->p.precision;
    out->min_blocks = c->min_blocks;
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------------
// Checkpoint of the dynamic state: a fixed header, then the current population planes and the
// current density plane exactly as stored on the device (padded layout, FP32 or FP64).
// ---------------------------------------------------------------------------------------------
namespace {
constexpr uint64_t kStateMagic = 0x314b43504d424c00ull;  // "\0LBMPCK1" little-endian
constexpr int32_t kStateVersion = 1;
struct StateHeader {
    uint64_t magic;
    int32_t version, nx, ny, esz;
    int64_t steps;
    uint64_t plane;    // elements per padded plane
    uint64_t payload;  // bytes after the header: 10 planes
};
size_t state_payload(const lbm_ctx* c) { return 10 * c->plane * c->esz; }
}  // namespace

size_t lbm_state_bytes(const lbm_ctx* c) {
    return c ? sizeof(StateHeader) + state_payload(c) : 0;
}

lbm_status lbm_save_state(lbm_ctx* c, void* host, size_t bytes) {
    lbm::NvtxRange nvtx_("lbm_save_state");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_save_state: ctx is NULL");
    if (!host) return fail(c, LBM_ERR_ARG, "lbm_save_state: buffer is NULL");
    if (!c->has_geometry) return fail(c, LBM_ERR_STATE, "lbm_save_state: no geometry");
    if (bytes != lbm_state_bytes(c))
        return fail(c, LBM_ERR_ARG, "lbm_save_state: bytes must equal lbm_state_bytes(ctx) = " +
                                        std::to_string(lbm_state_bytes(c)));
    DeviceGuard dg(c->device);
    StateHeader h{kStateMagic, kStateVersion, c->nx, c->ny, (int32_t)c->esz, c->steps,
                  (uint64_t)c->plane, (uint64_t)state_payload(c)};
    memcpy(host, &h, sizeof h);
    uint8_t* dst = static_cast<uint8_t*>(host) + sizeof h;
    const size_t hb = 9 * c->plane * c->esz;
    LBM_CUDA(c, cudaMemcpyAsync(dst, c->h[c->cur], hb, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync(dst + hb, c->rho[c->cur], c->plane * c->esz,
                                cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_ctx* c, const void* host, size_t bytes) {
    lbm::NvtxRange nvtx_("lbm_load_state");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_load_state: ctx is NULL");
    if (!host) return fail(c, LBM_ERR_ARG, "lbm_load_state: buffer is NULL");
    if (!c->has_geometry)
        return fail(c, LBM_ERR_STATE, "lbm_load_state: call lbm_set_geometry (the checkpoint's "
                                      "geometry) first");
    if (bytes < sizeof(StateHeader))
        return fail(c, LBM_ERR_ARG, "lbm_load_state: buffer shorter than the header");
    StateHeader h;
    memcpy(&h, host, sizeof h);
    if (h.magic != kStateMagic || h.version != kStateVersion)
        return fail(c, LBM_ERR_ARG, "lbm_load_state: not a checkpoint of this library version");
    if (h.nx != c->nx || h.ny != c->ny || h.esz != (int32_t)c->esz || h.plane != c->plane ||
        h.payload != state_payload(c) || bytes != lbm_state_bytes(c) || h.steps < 0)
        return fail(c, LBM_ERR_ARG, "lbm_load_state: checkpoint of another lattice size or "
                                    "precision, or wrong buffer size");
    DeviceGuard dg(c->device);
    const uint8_t* src = static_cast<const uint8_t*>(host) + sizeof h;
    const size_t hb = 9 * c->plane * c->esz;
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));  // nothing in flight reads the buffers
    LBM_CUDA(c, cudaMemcpyAsync(c->h[c->cur], src, hb, cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync(c->rho[c->cur], src + hb, c->plane * c->esz,
                                cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->steps = h.steps;
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_ctx* c) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "lbm_synchronize: ctx is NULL");
    DeviceGuard dg(c->device);
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    {
        DeviceGuard dg(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        free_all(c);
    }
    delete c;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : g_last_error.c_str(); }

}  // extern "C"
