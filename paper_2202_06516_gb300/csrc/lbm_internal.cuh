// Internal declarations of the GB300 multiphase LBM library: context layout, kernel argument
// blocks and launcher entry points shared by the translation units of liblbm.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

// D2Q9 direction order: rest, E, N, W, S, NE, NW, SW, SE (e_q and weights w_q of Eq. 1-2).
__host__ __device__ constexpr int qx(int q) {
    return q == 1 || q == 5 || q == 8 ? 1 : (q == 3 || q == 6 || q == 7 ? -1 : 0);
}
__host__ __device__ constexpr int qy(int q) {
    return q == 2 || q == 5 || q == 6 ? 1 : (q == 4 || q == 7 || q == 8 ? -1 : 0);
}
__host__ __device__ constexpr int qopp(int q) {
    return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 3) % 4) + 5);
}
template <typename T>
__host__ __device__ constexpr T qw(int q) {
    return q == 0 ? T(4) / T(9) : (q <= 4 ? T(1) / T(9) : T(1) / T(36));
}

constexpr uint8_t kFluid = 0, kLayer1 = 1, kLayer2 = 2, kSolid = 3;

// Device layout shared by every plane (populations, density, flags, wall chemical potential):
// node (x, j) of the fluid domain lives at (j + kPadY) * P + kPadX + x. Columns -kPadX..-1 and
// nx..nx+kPadX-1 hold copies of the periodic images (x + nx, x - nx); rows -2, -1, ny, ny+1 are
// the solid wall rows, and the remaining pad rows are inner solid. With the pads in place the
// step kernel reads any node within 8 columns and 7 rows of the domain without wrapping. Every
// plane ends with one more (slack) row.
constexpr int kPadX = 8, kPadY = 8;
__host__ __device__ __forceinline__ int lidx(int P, int x, int j) {
    return (j + kPadY) * P + kPadX + x;
}

// Equation-of-state constants in the form the kernels evaluate psi'(rho) in.
struct EosConst {
    int eos;      // LBM_EOS_PR / LBM_EOS_CS
    double RT;    // R * T
    double aal;   // a * alpha(T) (PR) or a (CS)
    double b;
};

// Arguments of the fused step kernel (one time step, Eq. 1-4, 7, 12-14).
template <typename T>
struct StepArgs {
    const T* h_in;     // 9 planes, post-collision deviations f*_q - w_q rho (see step .cu)
    T* h_out;
    const T* hq_in[9]; // the same planes one pointer each (single-lattice kernel)
    T* hq_out[9];
    const T* rho_in;   // rho(t)
    T* rho_out;        // rho(t+1)
    const uint8_t* flags;
    const T* muw;      // wall chemical potential on the wetting layers
    const T* dlt;      // interpolated bounce-back: link fraction of direction q at plane q - 1
    T* vx;             // optional velocity output (macroscopic mode)
    T* vy;
    int nx, ny, P;
    int plane;         // elements per plane: (ny + 2 kPadY + 1) * P
    T k2, kappa, gx, gy;
    T gbx, gby;        // -g_rho_ref * g: constant part of the body force
    T s_e, s_eps, s_q, s_v, inv_tau;
    int bgk;
    int eos;
    T RT, aal, b;
};

struct GeomArgs {
    int nx, ny, P, plane;
    int has_circle, stripes, concave;
    long long cx2, cy2, r2;  // doubled-integer circle
    double cx, cy, R, stripe_arc;
    double mu_circle, mu_stripe_b, mu_bottom, mu_top;
};

// Device result block of the reductions: sums over fluid nodes.
struct ReduceOut {
    double mass, n_liquid, sx, sy, bad, pad0, pad1, pad2;
};

struct Substrate {
    int circle;       // 1: circle (cx, cy, Rs), 0: flat bottom wall at y = -1/2
    int concave;      // circle only: 1 = the fluid lies inside the circle
    double cx, cy, Rs;
};

}  // namespace lbm

struct lbm_ctx {
    lbm_params p;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nx = 0, ny = 0, P = 0;
    size_t plane = 0;  // elements per padded plane
    size_t esz = 4;
    void* h[2] = {nullptr, nullptr};
    void* rho[2] = {nullptr, nullptr};
    void* muw = nullptr;
    uint8_t* flags = nullptr;
    uint8_t* linkmask = nullptr;   // per node, bit q-1 set when fluid x has a solid x + e_q
    void* dlt = nullptr;           // 8 planes of link fractions (interpolated bounce-back)
    bool ibb = false;
    int cur = 0;
    bool has_geometry = false;
    int64_t steps = 0;
    int64_t n_fluid = 0;
    lbm::EosConst eosc{};
    double rho_g = 0, rho_l = 0, p_sat = 0, mu_sat = 0, T = 0;
    lbm_geometry geom{};
    lbm::Substrate sub{};
    // reduction / measurement scratch
    double* red_partials = nullptr;
    lbm::ReduceOut* red_out = nullptr;
    void* meas_partials = nullptr;
    lbm_angle* meas_out = nullptr;
    int red_blocks = 0;
    // velocity scratch for lbm_read_fields
    void* vel = nullptr;
    // nx * ny doubles staging host transfers (initial density in, fields out), kept between calls
    double* stage = nullptr;
    // graphs of kGraphChunk >> k steps (k = 0 .. kGraphSizes - 1) starting from buffer 0 / 1
    cudaGraphExec_t graph[2][6] = {};
    bool graphs_ready = false;
    bool graph_failed = false;
    int tile_x = 32, tile_y = 16, min_blocks = 0;
    bool autotune_pending = false;  // LBM_TILE_AUTO: tune at the first lbm_step
    std::string err;
};

namespace lbm {

constexpr int kGraphChunk = 64;   // steps in the largest captured graph
constexpr int kGraphSizes = 6;    // graphs of 64, 32, 16, 8, 4, 2 steps (even: parity preserved)
constexpr int kRedThreads = 256;
constexpr int kAutotuneTrial = 20;  // timed launches per variant when LBM_TILE_AUTO tunes

// launchers (return the CUDA error of the launch)
cudaError_t launch_geometry(lbm_ctx* c, const GeomArgs& g);
cudaError_t launch_link_fractions(lbm_ctx* c, const GeomArgs& g);
cudaError_t launch_init_state(lbm_ctx* c, const lbm_geometry& g, const double* d_rho0);
cudaError_t launch_step(lbm_ctx* c, int src, bool macro);
size_t step_smem_bytes(int tile_x, int tile_y, size_t esz, int min_blocks);
struct StepVariant {
    int tile_x, tile_y, min_blocks;
};
// the compiled step-kernel variants for element size esz (4: FP32, 8: FP64)
void step_variants(size_t esz, std::vector<StepVariant>* out);
bool step_has_ibb(size_t esz, int tile_x, int tile_y, int min_blocks);
cudaError_t step_configure(lbm_ctx* c);
cudaError_t launch_reduce(lbm_ctx* c);
cudaError_t launch_measure(lbm_ctx* c);
cudaError_t launch_candidates(lbm_ctx* c, uint8_t* d_mark, double* d_pxyd);
cudaError_t launch_to_double(lbm_ctx* c, const void* src, double* dst, int src_is_rho_plane);
cudaError_t launch_fill_pads(lbm_ctx* c, void* plane, size_t esz);

}  // namespace lbm
