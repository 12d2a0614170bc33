// Batched sweep: many independent lattices of uneven size advanced together (the parameter
// sweeps over drop radius, cylinder curvature and wettability of Sec. 4.1-4.2).
//
// Every instance is an ordinary lbm_ctx (its own planes, geometry and measurement scratch, all
// on the batch's stream). A device tile table lists (instance, tile) pairs of the instances still
// running; one kernel launch per time step walks the table and advances each tile one step with
// the same device code as the single-lattice kernel. Its grid is either one CTA per tile of all
// instances (CTAs past the current table length exit at once) or persistent (one CTA per
// resident slot, looping over the table); the autotuner times both, and one CTA per tile is the
// default (measured faster: the hardware scheduler interleaves CTAs in different stages of
// their tiles, while a persistent CTA serialises its tiles' four barriers). A CUDA graph holds
// `check_every` such launches. After each graph the FP64 residual sum |rho(t) - rho(t - check)| /
// sum rho of every running instance is computed (one block per instance, fixed order), converged
// instances leave the table, and the graph is replayed on the shorter table without recapture
// (the kernels read the table length from device memory).
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "lbm_step_body.cuh"
#include "lbm_trace.h"

namespace lbm {
void set_global_error(const std::string& msg);
}

struct lbm_batch {
    int n = 0;
    cudaStream_t stream = nullptr;
    std::vector<lbm_ctx*> inst;
    std::vector<int> cur;         // buffer parity of each instance
    std::vector<int64_t> steps;   // steps taken by each instance
    std::vector<int> running;     // 1 while the instance is in the tile table
    std::vector<int> has_geom;
    void* d_desc = nullptr;       // BatchInst[n]
    int2* d_tiles = nullptr;      // (instance, tile index)
    int* d_ntiles = nullptr;
    int* d_active = nullptr;      // running instance ids (residual kernel)
    double* d_res = nullptr;      // per instance: residual sum, mass
    float* snap = nullptr;        // one density snapshot plane per instance
    std::vector<size_t> snap_off;
    int max_tiles = 0;
    int grid = 0;                 // resident slots (persistent grid)
    bool persistent = false;      // grid mode: resident slots, or one CTA per tile
    int variant = 0;              // index into the compiled tile variants
    int tx = 32, ty = 16;         // its tile shape
    bool autotune_pending = false;
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0;
    int graph_parity = -1;
    lbm::StepArgs<float> model{};
    std::string err;
};

namespace lbm {
namespace {

using namespace stepdev;

constexpr int NTB = 256;

// Compiled tile variants of the persistent kernel: tile (TX, TY) and the CTAs per SM its
// register budget is fitted to. Variant 1 (32 x 16, 5 CTAs/SM) is the default; the autotuner
// times all of them on the batch's own tile table.
#define LBM_BATCH_VARIANTS(X) X(32, 8, 5) X(32, 16, 5) X(64, 16, 3) X(32, 32, 3)
constexpr int kBatchDefaultVariant = 1;

struct BatchInst {
    float* h[2];
    float* rho[2];
    const uint8_t* flags;
    const float* muw;
    float* snap;
    int nx, ny, P, plane;
    float rho_mid;
};

template <int TX, int TY, int MINB>
__global__ void __launch_bounds__(NTB, MINB)
    k_batch_step(const StepArgs<float> model, const BatchInst* inst, const int2* tiles,
                 const int* n_tiles, int parity) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nt = *n_tiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 e = tiles[t];
        const BatchInst& I = inst[e.x];
        StepArgs<float> a = model;
        a.h_in = I.h[parity];
        a.h_out = I.h[parity ^ 1];
        a.rho_in = I.rho[parity];
        a.rho_out = I.rho[parity ^ 1];
        a.flags = I.flags;
        a.muw = I.muw;
        a.nx = I.nx;
        a.ny = I.ny;
        a.P = I.P;
        a.plane = I.plane;
        const int tiles_x = (I.nx + TX - 1) / TX;
        const int ty = e.y / tiles_x, tx = e.y - ty * tiles_x;
        step_tile<float, TX, TY, NTB, false, false>(a, I.rho_mid, smem_raw, tx * TX, ty * TY);
        __syncthreads();  // the next tile reuses shared memory
    }
}

// One block per running instance: sum |rho - snapshot| and sum rho over fluid nodes in a fixed
// order, then refresh the snapshot. res[2 i] = sum |drho|, res[2 i + 1] = sum rho.
__global__ void k_batch_residual(const BatchInst* inst, const int* active, int parity, double* res,
                                 int refresh) {
    const int id = active[blockIdx.x];
    const BatchInst& I = inst[id];
    const float* rho = I.rho[parity];
    double dsum = 0, msum = 0;
    const int n = I.nx * I.ny;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int j = k / I.nx, i = k - j * I.nx;
        const int o = lidx(I.P, i, j);
        if (I.flags[o] != kFluid) continue;
        const float r = rho[o];
        dsum += fabs((double)r - (double)I.snap[o]);
        msum += (double)r;
        if (refresh) I.snap[o] = r;
    }
    __shared__ double s[2][NTB / 32];
    for (int o = 16; o > 0; o >>= 1) {
        dsum += __shfl_down_sync(0xffffffffu, dsum, o);
        msum += __shfl_down_sync(0xffffffffu, msum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s[0][threadIdx.x >> 5] = dsum;
        s[1][threadIdx.x >> 5] = msum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s[0][w];
            b += s[1][w];
        }
        res[2 * id] = a;
        res[2 * id + 1] = b;
    }
}

lbm_status bfail(lbm_batch* b, lbm_status st, const std::string& msg) {
    if (b)
        b->err = msg;
    else
        set_global_error(msg);
    return st;
}

#define BCUDA(b, expr)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail((b), LBM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int tiles_of(const lbm_ctx* c, int tx, int ty) {
    return ((c->nx + tx - 1) / tx) * ((c->ny + ty - 1) / ty);
}
int tiles_of(const lbm_batch* b, const lbm_ctx* c) { return tiles_of(c, b->tx, b->ty); }

int num_variants() {
    int n = 0;
#define X(A, B, M) ++n;
    LBM_BATCH_VARIANTS(X)
#undef X
    return n;
}

// select variant v: shared-memory attribute, tile shape and the persistent grid (resident CTAs
// per SM x SMs)
cudaError_t configure_variant(lbm_batch* b, int v) {
    int i = 0, per_sm = 0, sms = 0, dev = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define X(A, B, M)                                                                           \
    if (v == i++) {                                                                          \
        const int bytes = (int)Layout<float, A, B>::bytes;                                   \
        e = cudaFuncSetAttribute(k_batch_step<A, B, M>,                                      \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);        \
        if (e == cudaSuccess)                                                                \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step<A, B, M>, \
                                                              NTB, bytes);                   \
        b->tx = A;                                                                           \
        b->ty = B;                                                                           \
    }
    LBM_BATCH_VARIANTS(X)
#undef X
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    b->variant = v;
    b->grid = (per_sm > 0 ? per_sm : 1) * sms;
    return cudaSuccess;
}

void variant_shape(int v, int* tx, int* ty, int* minb) {
    int i = 0;
#define X(A, B, M)  \
    if (v == i++) { \
        *tx = A;    \
        *ty = B;    \
        *minb = M;  \
    }
    LBM_BATCH_VARIANTS(X)
#undef X
}

lbm_status upload_desc(lbm_batch* b) {
    std::vector<BatchInst> d(b->n);
    for (int i = 0; i < b->n; ++i) {
        lbm_ctx* c = b->inst[i];
        BatchInst& I = d[i];
        I.h[0] = (float*)c->h[0];
        I.h[1] = (float*)c->h[1];
        I.rho[0] = (float*)c->rho[0];
        I.rho[1] = (float*)c->rho[1];
        I.flags = c->flags;
        I.muw = (const float*)c->muw;
        I.snap = b->snap + b->snap_off[i];
        I.nx = c->nx;
        I.ny = c->ny;
        I.P = c->P;
        I.plane = (int)c->plane;
        I.rho_mid = (float)(0.5 * (c->rho_g + c->rho_l));
    }
    BCUDA(b, cudaMemcpyAsync(b->d_desc, d.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice,
                             b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

// tile table of the running instances that share parity p; returns the number of tiles
lbm_status upload_tiles(lbm_batch* b, int p, int* ntiles, std::vector<int>* act) {
    std::vector<int2> t;
    act->clear();
    for (int i = 0; i < b->n; ++i) {
        if (!b->running[i] || b->cur[i] != p) continue;
        act->push_back(i);
        const int k = tiles_of(b, b->inst[i]);
        for (int q = 0; q < k; ++q) t.push_back(make_int2(i, q));
    }
    *ntiles = (int)t.size();
    if (!t.empty())
        BCUDA(b, cudaMemcpyAsync(b->d_tiles, t.data(), sizeof(int2) * t.size(),
                                 cudaMemcpyHostToDevice, b->stream));
    BCUDA(b, cudaMemcpyAsync(b->d_ntiles, ntiles, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    if (!act->empty())
        BCUDA(b, cudaMemcpyAsync(b->d_active, act->data(), sizeof(int) * act->size(),
                                 cudaMemcpyHostToDevice, b->stream));
    // the pageable sources must stay valid until the copies ran
    BCUDA(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

cudaError_t launch_batch_step(lbm_batch* b, int parity) {
    int i = 0;
    int grid = b->grid;
    if (!b->persistent) {  // one CTA per tile of every instance; CTAs past the table exit at once
        long long all = 0;
        for (const lbm_ctx* c : b->inst) all += tiles_of(b, c);
        grid = (int)std::max<long long>(1, all);
    }
#define X(A, B, M)                                                                           \
    if (b->variant == i++) {                                                                 \
        k_batch_step<A, B, M><<<grid, NTB, Layout<float, A, B>::bytes, b->stream>>>(         \
            b->model, (const BatchInst*)b->d_desc, b->d_tiles, b->d_ntiles, parity);         \
        return cudaGetLastError();                                                           \
    }
    LBM_BATCH_VARIANTS(X)
#undef X
    return cudaErrorInvalidValue;
}

lbm_status capture(lbm_batch* b, int chunk, int parity) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return LBM_OK;  // plain launches
    }
    cudaError_t le = cudaSuccess;
    for (int s = 0; s < chunk; ++s) {
        cudaError_t e = launch_batch_step(b, parity ^ (s & 1));
        if (e != cudaSuccess && le == cudaSuccess) le = e;
    }
    cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess || ee != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return LBM_OK;
    }
    if (cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) {
        cudaGetLastError();
        b->graph = nullptr;
    }
    cudaGraphDestroy(g);
    b->graph_chunk = chunk;
    b->graph_parity = parity;
    return LBM_OK;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

lbm_status lbm_batch_create(const lbm_params* model, int32_t n, const int32_t* nx,
                            const int32_t* ny, lbm_batch** out) {
    if (!out) return bfail(nullptr, LBM_ERR_ARG, "lbm_batch_create: out is NULL");
    *out = nullptr;
    if (!model || !nx || !ny || n <= 0)
        return bfail(nullptr, LBM_ERR_ARG, "lbm_batch_create: need model, n > 0, nx[], ny[]");
    if (model->precision != LBM_FP32)
        return bfail(nullptr, LBM_ERR_ARG, "lbm_batch_create: batches run in LBM_FP32");
    lbm_batch* b = new lbm_batch();
    b->n = n;
    auto cleanup = [&](lbm_status st, const std::string& msg) {
        for (lbm_ctx* c : b->inst) lbm_destroy(c);
        if (b->graph) cudaGraphExecDestroy(b->graph);
        cudaFree(b->d_desc);
        cudaFree(b->d_tiles);
        cudaFree(b->d_ntiles);
        cudaFree(b->d_active);
        cudaFree(b->d_res);
        cudaFree(b->snap);
        if (b->stream) cudaStreamDestroy(b->stream);
        delete b;
        return bfail(nullptr, st, msg);
    };
    int dev = model->device;
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bfail(nullptr, LBM_ERR_CUDA, "lbm_batch_create: cannot select the device");
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(LBM_ERR_CUDA, "lbm_batch_create: stream");
    size_t snap_total = 0;
    for (int i = 0; i < n; ++i) {
        lbm_params p = *model;
        p.nx = nx[i];
        p.ny = ny[i];
        p.tile_x = 32;
        p.tile_y = 16;
        p.min_blocks = 5;
        p.stream = b->stream;
        lbm_ctx* c = nullptr;
        lbm_status st = lbm_create(&p, &c);
        if (st != LBM_OK)
            return cleanup(st, std::string("lbm_batch_create: instance ") + std::to_string(i) +
                                   ": " + lbm_last_error(nullptr));
        b->inst.push_back(c);
        b->snap_off.push_back(snap_total);
        snap_total += c->plane;
        int most = 0;
        for (int v = 0; v < num_variants(); ++v) {
            int vx = 0, vy = 0, vm = 0;
            variant_shape(v, &vx, &vy, &vm);
            most = std::max(most, tiles_of(c, vx, vy));
        }
        b->max_tiles += most;
    }
    b->cur.assign(n, 0);
    b->steps.assign(n, 0);
    b->running.assign(n, 0);
    b->has_geom.assign(n, 0);
    e = cudaMalloc(&b->d_desc, sizeof(BatchInst) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_tiles, sizeof(int2) * b->max_tiles);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_ntiles, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_active, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_res, sizeof(double) * 2 * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->snap, sizeof(float) * snap_total);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->snap, 0, sizeof(float) * snap_total, b->stream);
    if (e == cudaSuccess) e = configure_variant(b, kBatchDefaultVariant);
    if (e != cudaSuccess)
        return cleanup(LBM_ERR_CUDA, std::string("lbm_batch_create: ") + cudaGetErrorString(e));
    b->autotune_pending = model->tile_x == LBM_TILE_AUTO;
    // model part of the step arguments (per-instance fields are filled in the kernel)
    lbm_ctx* c0 = b->inst[0];
    StepArgs<float>& a = b->model;
    a.k2 = (float)c0->p.k2;
    a.kappa = (float)c0->p.kappa;
    a.gx = (float)c0->p.gx;
    a.gy = (float)c0->p.gy;
    a.gbx = (float)(-c0->p.g_rho_ref * c0->p.gx);
    a.gby = (float)(-c0->p.g_rho_ref * c0->p.gy);
    a.s_e = (float)c0->p.s_e;
    a.s_eps = (float)c0->p.s_eps;
    a.s_q = (float)c0->p.s_q;
    a.s_v = (float)(1.0 / c0->p.tau);
    a.inv_tau = (float)(1.0 / c0->p.tau);
    a.bgk = c0->p.collision == LBM_BGK;
    a.eos = c0->eosc.eos;
    a.RT = (float)c0->eosc.RT;
    a.aal = (float)c0->eosc.aal;
    a.b = (float)c0->eosc.b;
    lbm_status st = upload_desc(b);
    if (st != LBM_OK) return cleanup(st, b->err);
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_set_geometry(lbm_batch* b, int32_t i, const lbm_geometry* g) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "lbm_batch_set_geometry: batch is NULL");
    if (i < 0 || i >= b->n) return bfail(b, LBM_ERR_ARG, "lbm_batch_set_geometry: bad index");
    if (g && g->boundary != LBM_BB_HALFWAY)
        return bfail(b, LBM_ERR_ARG, "lbm_batch_set_geometry: batches use half-way bounce-back");
    lbm_status st = lbm_set_geometry(b->inst[i], g);
    if (st != LBM_OK) return bfail(b, st, lbm_last_error(b->inst[i]));
    b->cur[i] = 0;
    b->steps[i] = 0;
    b->has_geom[i] = 1;
    b->running[i] = 0;
    return LBM_OK;
}

lbm_status lbm_batch_run(lbm_batch* b, int64_t max_steps, int32_t check_every, double tol,
                         double angle_tol, int64_t* steps_out, int32_t* converged_out,
                         double* residual_out) {
    lbm::NvtxRange nvtx_("lbm_batch_run");
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "lbm_batch_run: batch is NULL");
    if (max_steps < 0 || check_every < 2 || (check_every & 1))
        return bfail(b, LBM_ERR_ARG, "lbm_batch_run: need max_steps >= 0 and an even check_every >= 2");
    BCUDA(b, cudaSetDevice(b->inst[0]->device));
    if (b->autotune_pending) {
        bool any = false;
        for (int i = 0; i < b->n; ++i) any = any || b->has_geom[i];
        if (any) {
            b->autotune_pending = false;
            const lbm_status ts = lbm_batch_autotune(b, kAutotuneTrial, nullptr, 0, nullptr);
            if (ts != LBM_OK) return ts;
        }
    }
    std::vector<int> conv(b->n, 0);
    std::vector<double> resid(b->n, -1.0);
    std::vector<double> last_theta(2 * b->n, -1.0);
    std::vector<int> stable(b->n, 0);
    // every instance with geometry starts at parity 0 (set_geometry) or where it stopped
    for (int i = 0; i < b->n; ++i) b->running[i] = b->has_geom[i];
    std::vector<int> act;
    int ntiles = 0;
    int64_t done = 0;
    // the running set must share one parity; group by the parity of the first running instance
    int parity = -1;
    for (int i = 0; i < b->n; ++i)
        if (b->running[i]) {
            if (parity < 0) parity = b->cur[i];
            if (b->cur[i] != parity) b->running[i] = 0;  // run them in a later call
        }
    if (parity < 0) parity = 0;
    lbm_status st = upload_tiles(b, parity, &ntiles, &act);
    if (st != LBM_OK) return st;
    if (!act.empty()) {
        k_batch_residual<<<(int)act.size(), NTB, 0, b->stream>>>((const BatchInst*)b->d_desc,
                                                                 b->d_active, parity, b->d_res, 1);
        BCUDA(b, cudaGetLastError());
    }
    while (done < max_steps && !act.empty()) {
        const int chunk = (int)std::min<int64_t>(check_every, max_steps - done);
        if (chunk == check_every) {
            if (!b->graph || b->graph_chunk != chunk || b->graph_parity != parity)
                capture(b, chunk, parity);
            if (b->graph) {
                BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
            } else {
                for (int s = 0; s < chunk; ++s) BCUDA(b, launch_batch_step(b, parity ^ (s & 1)));
            }
        } else {
            for (int s = 0; s < chunk; ++s) BCUDA(b, launch_batch_step(b, parity ^ (s & 1)));
        }
        parity ^= (chunk & 1);
        done += chunk;
        for (int i : act) {
            b->steps[i] += chunk;
            b->cur[i] = parity;
        }
        k_batch_residual<<<(int)act.size(), NTB, 0, b->stream>>>((const BatchInst*)b->d_desc,
                                                                 b->d_active, parity, b->d_res, 1);
        BCUDA(b, cudaGetLastError());
        std::vector<double> res(2 * b->n);
        BCUDA(b, cudaMemcpyAsync(res.data(), b->d_res, sizeof(double) * 2 * b->n,
                                 cudaMemcpyDeviceToHost, b->stream));
        BCUDA(b, cudaStreamSynchronize(b->stream));
        bool changed = false;
        for (int i : act) {
            const double r = res[2 * i + 1] > 0 ? res[2 * i] / res[2 * i + 1] : 0.0;
            resid[i] = r;
            if (!(res[2 * i + 1] > 0) || !std::isfinite(res[2 * i + 1])) {
                b->running[i] = 0;  // unstable: stop it, report not converged
                changed = true;
                continue;
            }
            bool done_i = r < tol;
            if (!done_i && angle_tol > 0) {
                // angle stationarity: both sides measured and within angle_tol of the previous
                // check, twice in a row
                lbm_ctx* c = b->inst[i];
                c->cur = b->cur[i];
                lbm_angle ang[2];
                const lbm_status ms = lbm_measure_contact_angle(c, ang);
                if (ms == LBM_OK) {
                    const bool still = last_theta[2 * i] >= 0 &&
                                       fabs(ang[0].theta_deg - last_theta[2 * i]) <= angle_tol &&
                                       fabs(ang[1].theta_deg - last_theta[2 * i + 1]) <= angle_tol;
                    stable[i] = still ? stable[i] + 1 : 0;
                    last_theta[2 * i] = ang[0].theta_deg;
                    last_theta[2 * i + 1] = ang[1].theta_deg;
                    done_i = stable[i] >= 2;
                } else if (ms == LBM_ERR_NO_CONTACT) {
                    stable[i] = 0;
                    last_theta[2 * i] = last_theta[2 * i + 1] = -1.0;
                } else {
                    return bfail(b, ms, lbm_last_error(c));
                }
            }
            if (done_i) {
                conv[i] = 1;
                b->running[i] = 0;
                changed = true;
            }
        }
        if (changed) {
            st = upload_tiles(b, parity, &ntiles, &act);
            if (st != LBM_OK) return st;
        }
    }
    BCUDA(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i) {
        b->inst[i]->cur = b->cur[i];
        b->inst[i]->steps = b->steps[i];
        if (steps_out) steps_out[i] = b->steps[i];
        if (converged_out) converged_out[i] = conv[i];
        if (residual_out) residual_out[i] = resid[i];
    }
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int32_t trial_steps, lbm_tune_entry* entries,
                              int32_t max_entries, int32_t* n_out) {
    lbm::NvtxRange nvtx_("lbm_batch_autotune");
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "lbm_batch_autotune: batch is NULL");
    if (trial_steps < 1) return bfail(b, LBM_ERR_ARG, "lbm_batch_autotune: trial_steps < 1");
    BCUDA(b, cudaSetDevice(b->inst[0]->device));
    // the instances with geometry that share the parity of the first one
    int parity = -1;
    for (int i = 0; i < b->n; ++i)
        if (b->has_geom[i] && parity < 0) parity = b->cur[i];
    if (parity < 0) return bfail(b, LBM_ERR_STATE, "lbm_batch_autotune: no instance has geometry");
    const std::vector<int> keep_running = b->running;
    for (int i = 0; i < b->n; ++i) b->running[i] = b->has_geom[i] && b->cur[i] == parity;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    const int keep = b->variant;
    const bool keep_persistent = b->persistent;
    int best = -1;
    double best_us = 0;
    lbm_status st = LBM_OK;
    std::vector<int> act;
    // trial k: tile variant k / 2, grid one CTA per tile (k even) or persistent (k odd)
    for (int k2 = 0; k2 < 2 * num_variants() && err == cudaSuccess && st == LBM_OK; ++k2) {
        const int v = k2 / 2;
        b->persistent = (k2 & 1) != 0;
        err = configure_variant(b, v);
        if (err != cudaSuccess) break;
        int ntiles = 0;
        st = upload_tiles(b, parity, &ntiles, &act);
        if (st != LBM_OK) break;
        // every launch reads buffer `parity` and writes the other one: nothing advances
        for (int w = 0; w < 2 && err == cudaSuccess; ++w) err = launch_batch_step(b, parity);
        if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
        for (int k = 0; k < trial_steps && err == cudaSuccess; ++k)
            err = launch_batch_step(b, parity);
        if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) break;
        const double us = 1e3 * (double)ms / trial_steps;
        int vx = 0, vy = 0, vm = 0;
        variant_shape(v, &vx, &vy, &vm);
        if (entries && k2 < max_entries)
            entries[k2] = lbm_tune_entry{vx, vy, vm, us, b->persistent ? 1 : 0};
        if (best < 0 || us < best_us) {
            best = k2;
            best_us = us;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->running = keep_running;
    const bool ok = err == cudaSuccess && st == LBM_OK && best >= 0;
    b->persistent = ok ? (best & 1) != 0 : keep_persistent;
    const cudaError_t ce = configure_variant(b, ok ? best / 2 : keep);
    if (st != LBM_OK) return st;
    BCUDA(b, err);
    BCUDA(b, ce);
    // the captured graph was built for the previous tile table
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_chunk = 0;
    b->graph_parity = -1;
    if (n_out) *n_out = 2 * num_variants();
    return LBM_OK;
}

lbm_status lbm_batch_measure(lbm_batch* b, lbm_angle* out) {
    lbm::NvtxRange nvtx_("lbm_batch_measure");
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "lbm_batch_measure: batch is NULL");
    if (!out) return bfail(b, LBM_ERR_ARG, "lbm_batch_measure: out is NULL");
    lbm_status worst = LBM_OK;
    for (int i = 0; i < b->n; ++i) {
        if (!b->has_geom[i]) {
            out[2 * i].status = out[2 * i + 1].status = LBM_ERR_STATE;
            continue;
        }
        b->inst[i]->cur = b->cur[i];
        lbm_status st = lbm_measure_contact_angle(b->inst[i], &out[2 * i]);
        if (st == LBM_ERR_NO_CONTACT) {
            worst = LBM_ERR_NO_CONTACT;
        } else if (st != LBM_OK) {
            return bfail(b, st, lbm_last_error(b->inst[i]));
        }
    }
    return worst;
}

lbm_status lbm_batch_instance(lbm_batch* b, int32_t i, lbm_ctx** ctx) {
    if (!b || !ctx) return bfail(b, LBM_ERR_ARG, "lbm_batch_instance: NULL argument");
    if (i < 0 || i >= b->n) return bfail(b, LBM_ERR_ARG, "lbm_batch_instance: bad index");
    b->inst[i]->cur = b->cur[i];
    b->inst[i]->steps = b->steps[i];
    *ctx = b->inst[i];
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) {
    return b ? b->err.c_str() : lbm_last_error(nullptr);
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (lbm_ctx* c : b->inst) lbm_destroy(c);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->d_desc);
    cudaFree(b->d_tiles);
    cudaFree(b->d_ntiles);
    cudaFree(b->d_active);
    cudaFree(b->d_res);
    cudaFree(b->snap);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
