// lbm_mass_noalloc: the density sums of lbm_mass for a caller-owned density field, with every
// scratch byte in a fixed device array that the library image carries, so the call allocates
// nothing. Meant for callers that may not allocate device memory at the point of the call (a
// framework that owns all device memory through its own pool, code that must not trigger the
// implicit synchronisation of cudaMalloc/cudaFree, or a host process that has budgeted every
// byte of the GPU). The paper has no counterpart; it is a deployment convenience.
//
// Scratch: one row of 8 doubles per lattice row (per-row partial sums), at most
// LBM_NOALLOC_MAX_ROWS rows (256 KiB). Every GPU that loads the library holds this array until
// the process exits. Each call overwrites the rows it uses before reading them, so nothing needs
// clearing between calls; two calls that overlap on the GPU (different streams, or different
// host threads) share the array and race.
#include <mutex>
#include <string>

#include "lbm_internal.cuh"

namespace lbm {
void set_global_error(const std::string& msg);
}

namespace {

constexpr int kRowThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_row_partials[LBM_NOALLOC_MAX_ROWS * 8];

std::mutex g_mu;
double* g_scratch[kMaxDevices] = {nullptr};

// One block per lattice row: FP64 sums of density, liquid count, liquid x, liquid y and the
// count of non-finite or non-positive densities over the row's fluid nodes.
__global__ void k_row_sums(const float* rho, const uint8_t* flags, int nx, int pitch,
                           double rho_m, double* rows) {
    const int j = blockIdx.x;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const size_t o = (size_t)j * pitch + i;
        if (flags[o] != 0) continue;
        const double r = (double)rho[o];
        acc[0] += r;
        if (!(r > 0.0) || !isfinite(r)) acc[4] += 1.0;
        if (r > rho_m) {
            acc[1] += 1.0;
            acc[2] += (double)i;
            acc[3] += (double)j;
        }
    }
    __shared__ double s[kRowThreads / 32][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0;
        for (int w = 0; w < kRowThreads / 32; ++w) v += s[w][threadIdx.x];
        rows[(size_t)j * 8 + threadIdx.x] = v;
    }
}

// Adds the row partials in row order and writes mass, n_liquid, centroid x, centroid y, n_bad.
__global__ void k_rows_final(const double* rows, int ny, double* out) {
    if (threadIdx.x != 0) return;
    double v[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < ny; ++j)
        for (int k = 0; k < 5; ++k) v[k] += rows[(size_t)j * 8 + k];
    out[0] = v[0];
    out[1] = v[1];
    out[2] = v[1] > 0 ? v[2] / v[1] : 0.0;
    out[3] = v[1] > 0 ? v[3] / v[1] : 0.0;
    out[4] = v[4];
}

lbm_status fail(lbm_status st, const std::string& msg) {
    lbm::set_global_error(msg);
    return st;
}

}  // namespace

extern "C" lbm_status lbm_mass_noalloc(const float* rho, const uint8_t* flags, int32_t nx,
                                       int32_t ny, int32_t pitch, double rho_m, double* out,
                                       void* stream) {
    if (!rho || !flags || !out) return fail(LBM_ERR_ARG, "lbm_mass_noalloc: NULL pointer");
    if (nx <= 0 || ny <= 0 || pitch < nx)
        return fail(LBM_ERR_ARG, "lbm_mass_noalloc: need nx > 0, ny > 0 and pitch >= nx");
    if (ny > LBM_NOALLOC_MAX_ROWS)
        return fail(LBM_ERR_ARG, "lbm_mass_noalloc: ny = " + std::to_string(ny) +
                                     " exceeds LBM_NOALLOC_MAX_ROWS = " +
                                     std::to_string(LBM_NOALLOC_MAX_ROWS) +
                                     " (the fixed scratch holds one entry per row)");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(LBM_ERR_CUDA, std::string("lbm_mass_noalloc: no usable current device: ") +
                                      cudaGetErrorString(e));
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch[dev]) {
            // The array's name in host code is only a host-side handle; the kernels need the
            // device address, taken once per device with that device current.
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_row_partials);
            if (e != cudaSuccess || !p)
                return fail(LBM_ERR_CUDA, std::string("lbm_mass_noalloc: cudaGetSymbolAddress: ") +
                                              cudaGetErrorString(e));
            g_scratch[dev] = (double*)p;
        }
        scratch = g_scratch[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    k_row_sums<<<ny, kRowThreads, 0, s>>>(rho, flags, nx, pitch, rho_m, scratch);
    k_rows_final<<<1, 32, 0, s>>>(scratch, ny, out);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(LBM_ERR_CUDA, std::string("lbm_mass_noalloc: launch: ") + cudaGetErrorString(e));
    return LBM_OK;
}
