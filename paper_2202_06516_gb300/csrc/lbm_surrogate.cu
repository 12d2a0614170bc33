// Learned warm start: a convolutional U-Net that maps (solid mask, wall-wetting map, drop-volume
// plane) on an H x W lattice to a near-equilibrium density field, trained on equilibrated fields
// the solver generates. The paper has no such component; it shortens the plain relaxation from a
// flat-cap start (Sec. 4, Eq. 16) that the solver otherwise performs.
//
// Network (levels l = 1..4, channels c_l = base * 2^(l-1)):
//   encoder   conv3x3 + leaky ReLU (slope 0.1) twice per level, 2x2 average pooling between
//   decoder   2x upsampling folded into the next conv3x3 (nearest), the skip concatenation folded
//             into the following conv3x3 (two-source im2col), conv3x3 + leaky ReLU twice per level
//   head      1x1 conv to one channel, sigmoid: phi = (rho - rho_g) / (rho_l - rho_g)
// Activations BF16 NHWC, weights FP32 masters with BF16 copies, all contractions on the tcgen05
// tensor cores with FP32 accumulation in tensor memory (sg_tc.cuh), as implicit GEMMs whose
// operands are the 3 x 3 neighbourhoods of the activations: the forward convolution, the
// weight gradient (pixels as K; an im2col buffer only when the resolution is not a power of two)
// and the data gradient (output gradients around each source pixel). Where the shapes allow,
// the operands arrive as tensor-map (TMA) boxes built once per network (make_tensor_maps): the
// tap's offset moves the box, the image border is zero-filled, upsampling layers order their
// rows or K even/odd or read every second pixel; the 32/64-channel levels stage one window per
// slice or tile and take the nine taps from it; elsewhere the loaders gather with cp.async.
// Loss: masked mean squared error on phi. Optimiser: Adam.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lbm_internal.cuh"
#include "lbm_trace.h"
#include "sg_gemm.cuh"
#include "sg_tc.cuh"

#include <atomic>
#include <mutex>

namespace lbm {
void set_global_error(const std::string& msg);
}

using bf16 = __nv_bfloat16;

namespace lbm {
namespace sg {
namespace {

constexpr int kT = 256;
constexpr int kReluBlocks = 1024;  // blocks of the fused leaky-ReLU adjoint / bias-sum pass

int blocks_for(long long n) {
    long long b = (n + kT - 1) / kT;
    return (int)(b > 65535LL * 8 ? 65535LL * 8 : (b < 1 ? 1 : b));
}

// Pixel index p -> (n, y, x) of a batch of H x W images (NHWC); P2: H and W are powers of two
// and the split is done with shifts and masks.
struct PixDims {
    int H, W, lh, lw;  // lh, lw: log2 H, log2 W when P2
};

template <bool P2>
__device__ __forceinline__ void pix_split(int p, const PixDims& d, int& n, int& y, int& x) {
    if (P2) {
        x = p & (d.W - 1);
        y = (p >> d.lw) & (d.H - 1);
        n = p >> (d.lw + d.lh);
    } else {
        x = p % d.W;
        const int q = p / d.W;
        y = q % d.H;
        n = q / d.H;
    }
}

// im2col of a 3x3, pad-1 convolution whose input channels are [source 1 | source 2]:
// col[p][(ky*3+kx)*C + c] = x(n, y+ky-1, x+kx-1, c). Source 1 may be stored at half resolution
// (up1 = 1: nearest 2x upsampling on the fly). Eight channels per thread (16-byte accesses); the
// number of 8-channel groups C / 8 = 2^lc8, so thread t writes the 16 bytes at col + 8 t.
template <bool P2>
__global__ void k_im2col(const bf16* x1, int C1, int up1, const bf16* x2, int C2, PixDims d,
                         int P, int lc8, bf16* col) {
    const int C8 = 1 << lc8;
    const long long total = (long long)P * 9 * C8;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c8 = (int)(t & (C8 - 1));
        const int tq = (int)(t >> lc8);  // p * 9 + tap
        const int p = tq / 9, tap = tq - p * 9;
        int n, yy, xx;
        pix_split<P2>(p, d, n, yy, xx);
        const int sy = yy + tap / 3 - 1, sx = xx + tap % 3 - 1;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (sy >= 0 && sy < d.H && sx >= 0 && sx < d.W) {
            const int c = c8 * 8;
            if (c < C1) {
                const int h1 = up1 ? d.H / 2 : d.H, w1 = up1 ? d.W / 2 : d.W;
                const int ty = up1 ? sy >> 1 : sy, tx = up1 ? sx >> 1 : sx;
                v = *reinterpret_cast<const uint4*>(x1 + (((size_t)n * h1 + ty) * w1 + tx) * C1 + c);
            } else {
                v = *reinterpret_cast<const uint4*>(x2 + (((size_t)n * d.H + sy) * d.W + sx) * C2 +
                                                    (c - C1));
            }
        }
        *reinterpret_cast<uint4*>(col + (size_t)t * 8) = v;
    }
}

__global__ void k_avgpool(const bf16* x, bf16* y, int B, int H, int W, int C) {
    const int h = H / 2, w = W / 2;
    const long long total = (long long)B * h * w * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % C);
        const long long q = t / C;
        const int X = (int)(q % w), Y = (int)((q / w) % h), n = (int)(q / ((long long)w * h));
        const size_t b = (((size_t)n * H + 2 * Y) * W + 2 * X) * C + c;
        const float s = __bfloat162float(x[b]) + __bfloat162float(x[b + C]) +
                        __bfloat162float(x[b + (size_t)W * C]) +
                        __bfloat162float(x[b + (size_t)W * C + C]);
        y[t] = __float2bfloat16_rn(0.25f * s);
    }
}

// The leaky-ReLU adjoint of one convolution's output fused with what feeds it and what reads
// it: g = (dy + dyp / 4) * (y > 0 ? 1 : 0.1), stored as BF16 for the gradient GEMMs, where dyp
// (POOL) is the gradient of the 2 x 2 average pool taken of this output, whose adjoint gives a
// quarter to each of the four source pixels (added after the other consumers' contributions,
// as a separate pass would); and the per-block column sums of the stored g (the bias gradient's
// partials). Thread t always covers the eight channels 8 t mod C (8 x threads per block is a
// multiple of C), so each block adds its threads' sums per channel in thread order into
// part[c][block] (deterministic). H, W: the output resolution (even when POOL).
template <bool POOL>
__global__ void k_relu_bias(const float* dy, const float* dyp, const bf16* y, bf16* g,
                            long long n8, int C, int H, int W, float* part) {
    __shared__ float sred[kT * 8];
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n8;
         t += (long long)gridDim.x * blockDim.x) {
        const uint4 yv = reinterpret_cast<const uint4*>(y)[t];
        const float4 a = reinterpret_cast<const float4*>(dy)[2 * t];
        const float4 b = reinterpret_cast<const float4*>(dy)[2 * t + 1];
        float d[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        if (POOL) {
            const long long e = 8 * t, p = e / C;
            const int c = (int)(e - p * C);
            const long long q = p / W, n = q / H;
            const int xx = (int)(p - q * W), yy = (int)(q - n * H);
            const float4* src = reinterpret_cast<const float4*>(
                dyp + (((n * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C + c));
            const float4 pa = src[0], pb = src[1];
            const float pv[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) d[j] += 0.25f * pv[j];
        }
        const __nv_bfloat162* yh = reinterpret_cast<const __nv_bfloat162*>(&yv);
        uint4 out;
        __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&out);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 yf = __bfloat1622float2(yh[i]);
            const float g0 = yf.x > 0.f ? d[2 * i] : 0.1f * d[2 * i];
            const float g1 = yf.y > 0.f ? d[2 * i + 1] : 0.1f * d[2 * i + 1];
            oh[i] = __floats2bfloat162_rn(g0, g1);
            const float2 r = __bfloat1622float2(oh[i]);
            acc[2 * i] += r.x;
            acc[2 * i + 1] += r.y;
        }
        reinterpret_cast<uint4*>(g)[t] = out;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) sred[threadIdx.x * 8 + j] = acc[j];
    __syncthreads();
    // channel c: the threads c / 8 + k C / 8 (k = 0, 1, ...), slot c % 8
    const int groups = C / 8, reps = blockDim.x / groups;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < reps; ++k) s += sred[(c / 8 + k * groups) * 8 + (c & 7)];
        part[(size_t)c * gridDim.x + blockIdx.x] = s;
    }
}

// out[c] = sum over b of the partials of column c: part[b * C + c], or part[c * nb + b] when
// transposed; one block per column, a fixed-shape tree in shared memory (deterministic)
__global__ void k_colsum_final(const float* part, int nb, int C, float* out, int transposed = 0) {
    __shared__ float sm[kT];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        s += transposed ? part[(size_t)c * nb + b] : part[(size_t)b * C + c];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sm[0];
}

// head: phi = sigmoid(sum_c x[p][c] w[c] + b); with targets, also the loss terms and the
// gradient: dz = 2 m (phi - t) phi (1 - phi) / n_mask, dx[p][c] = dz w[c]; per-block partial sums
// of loss, dz * x[p][c] (weight gradient) and dz (bias gradient) for a deterministic reduction.
template <int C>
__global__ void k_head(const bf16* x, const float* w, const float* bptr, float* phi, long long P,
                       const float* target, const uint8_t* mask, float inv_n, float* dx,
                       float* part /* per block: C + 2 */) {
    __shared__ float sw[C];
    __shared__ float red[kT / 32][C + 2];
    for (int c = threadIdx.x; c < C; c += blockDim.x) sw[c] = w[c];
    __syncthreads();
    const float b = *bptr;
    float acc[C + 2];
#pragma unroll
    for (int c = 0; c < C + 2; ++c) acc[c] = 0.f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        float z = b;
        float xv[C];
        // the pixel's C channels as 16-byte vectors (C is a multiple of 8)
#pragma unroll
        for (int v = 0; v < C / 8; ++v) {
            const uint4 raw = reinterpret_cast<const uint4*>(x + p * C)[v];
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 f2 = __bfloat1622float2(h[i]);
                xv[8 * v + 2 * i] = f2.x;
                xv[8 * v + 2 * i + 1] = f2.y;
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) z += xv[c] * sw[c];
        const float f = 1.f / (1.f + __expf(-z));
        phi[p] = f;
        if (target) {
            const float m = mask[p] ? 1.f : 0.f;
            const float e = f - target[p];
            const float dz = 2.f * m * e * f * (1.f - f) * inv_n;
            acc[C] += m * e * e * inv_n;
            acc[C + 1] += dz;
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] += dz * xv[c];
#pragma unroll
            for (int c = 0; c < C; c += 4)
                reinterpret_cast<float4*>(dx + p * C)[c / 4] =
                    make_float4(dz * sw[c], dz * sw[c + 1], dz * sw[c + 2], dz * sw[c + 3]);
        }
    }
    if (!target) return;
#pragma unroll
    for (int c = 0; c < C + 2; ++c) {
        float v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C + 2; c += blockDim.x) {
        float s = 0.f;
        for (int q = 0; q < kT / 32; ++q) s += red[q][c];
        part[(size_t)blockIdx.x * (C + 2) + c] = s;
    }
}

// Offsets and shapes of the convolution weights in the parameter vector, for the kernels that
// keep the BF16 copies (the forward/weight-gradient layout w[co][tap][ci] and the data-gradient
// layout wd[ci][tap][co]).
struct ConvTable {
    int n;
    long long off[24];
    int cout[24], cin[24];
};

// BF16 copies of parameter t with FP32 value x: wb[t], and for a convolution weight also its
// data-gradient position wd[off + (ci 9 + tap) cout + co]
__device__ __forceinline__ void store_bf16_copies(long long t, float x, bf16* wb, bf16* wd,
                                                  const ConvTable& tab) {
    const bf16 h = __float2bfloat16_rn(x);
    wb[t] = h;
    for (int k = 0; k < tab.n; ++k) {
        const long long loc = t - tab.off[k];
        const long long len = (long long)tab.cout[k] * 9 * tab.cin[k];
        if (loc >= 0 && loc < len) {
            const int cin = tab.cin[k], cout = tab.cout[k];
            const int co = (int)(loc / (9 * cin)), rem = (int)(loc - (long long)co * 9 * cin);
            const int tap = rem / cin, ci = rem - tap * cin;
            wd[tab.off[k] + ((long long)ci * 9 + tap) * cout + co] = h;
            return;
        }
    }
}

// Adam with bias correction (c1, c2 = 1 / (1 - beta^t)), followed by the BF16 copies of the
// updated parameter
__global__ void k_adam(float* w, const float* g, float* m, float* v, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2, bf16* wb, bf16* wd,
                       const ConvTable tab) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const float gi = g[t];
        const float mi = b1 * m[t] + (1.f - b1) * gi;
        const float vi = b2 * v[t] + (1.f - b2) * gi * gi;
        m[t] = mi;
        v[t] = vi;
        const float wi = w[t] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        w[t] = wi;
        store_bf16_copies(t, wi, wb, wd, tab);
    }
}

// the BF16 copies of every parameter (after the FP32 masters were set)
__global__ void k_bf16_copies(const float* w, long long n, bf16* wb, bf16* wd,
                              const ConvTable tab) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        store_bf16_copies(t, w[t], wb, wd, tab);
}


struct Conv {
    int src1, C1, up1;  // source tensor index, channels, stored at half resolution
    int src2, C2;       // second source (-1: none)
    int Cout, out;      // output tensor index
    int H, W;           // output resolution
    size_t w_off, b_off;  // offsets into the parameter vector
    // tensor maps of the TMA-fed forward (f) and data-gradient (d) GEMMs: A source 1, A source
    // 2 (concatenation), B; f_ks, d_ks: the K elements per stage of those maps (64 or 32), 0
    // when the shapes do not allow it and the loaders gather with cp.async
    int f_ks = 0, d_ks = 0;
    CUtensorMap fmap[3] = {}, dmap[3] = {};
    // weight gradient (w): A sources 1 and 2 and the output gradient, boxes of 32 channels x 64
    // pixels; w_tma false: gathered with cp.async
    bool w_tma = false;
    CUtensorMap wmap[3] = {};
    // weight gradient from one staged input window per slice (k_gemm_wwin): C_in / 32 when it
    // applies (1 or 2), else 0; maps: sources 1 and 2 (32 channels x 72 pixels x 3 rows), dY
    int ww_cb = 0;
    CUtensorMap wwmap[3] = {};
    // forward (fw) and data gradient (dw) from one staged window per tile of 128 pixels of one
    // row (k_gemm_fwin): 32-channel blocks of the window operand (1 where it applies, else 0)
    // and the N tile; maps: source 1 (dY for dw) as boxes of 32 channels x 136 pixels x 3 rows,
    // source 2 likewise, and the weights as 32 x N-tile blocks
    int fw_cb = 0, fw_bn = 0, dw_cb = 0, dw_bn = 0;
    CUtensorMap fwmap[3] = {}, dwmap[3] = {};
};

struct Tensor {
    int H, W, C;
    bf16* y = nullptr;   // activation
    float* dy = nullptr; // gradient
};

}  // namespace
}  // namespace sg
}  // namespace lbm

using namespace lbm::sg;

struct lbm_surrogate {
    int H = 0, W = 0, base = 0, maxB = 0, device = 0;
    cudaStream_t stream = nullptr;
    std::vector<Tensor> t;      // 0: input (8 channels)
    std::vector<Conv> convs;
    std::vector<std::pair<int, int>> pools;  // (from, to)
    int head_in = -1;
    size_t head_w = 0, head_b = 0;
    size_t nparams = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    bf16* wb = nullptr;
    bf16* wbd = nullptr;        // per convolution [C_in][tap][C_out] (data-gradient operand)
    bf16 *col = nullptr, *gmask = nullptr;
    size_t col_elems = 0, act_elems = 0;
    float* part = nullptr;  // reduction partials
    float* phi = nullptr;   // head output
    float* hpart = nullptr;
    float* bpart = nullptr;   // per-block column sums of the bias gradients
    float* splitk = nullptr;  // split-K partials of the weight gradient
    size_t splitk_elems = 0;
    int part_blocks = 256;
    ConvTable tab{};  // convolution weight shapes for the BF16 copies
    long long adam_t = 0;
    std::string err;
};

extern "C" void lbm_surrogate_destroy(lbm_surrogate* s);

namespace {

lbm_status sfail(lbm_surrogate* s, lbm_status st, const std::string& msg) {
    if (s)
        s->err = msg;
    else
        lbm::set_global_error(msg);
    return st;
}

#define SCUDA(s, expr)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return sfail((s), LBM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Latched timeout flag of the tensor-core GEMM: mapped host memory that the kernels write on
// a wait that ran out; reported (and cleared) by the next host call that checks it.
struct TcFlag {
    volatile int* host = nullptr;
    int* dev = nullptr;
};

TcFlag& tc_flag() {
    static std::mutex mu;
    static TcFlag f;
    std::lock_guard<std::mutex> lk(mu);
    if (!f.host) {
        int* h = nullptr;
        if (cudaHostAlloc((void**)&h, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            return f;
        }
        *h = 0;
        int* d = nullptr;
        if (cudaHostGetDevicePointer((void**)&d, h, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(h);
            return f;
        }
        f.host = h;
        f.dev = d;
    }
    return f;
}

// true (and the flag cleared) if a tensor-core GEMM launched earlier gave up waiting
bool tc_timed_out() {
    TcFlag& f = tc_flag();
    if (!f.host) return false;
    const bool t = *f.host != 0;
    *f.host = 0;
    return t;
}

template <int BN, int STAGES, bool AMN, bool BMN, bool GA, bool GD, bool GAM, int TMA = 0>
cudaError_t launch_tc(cudaStream_t st, const GemmArgs& a, int splits,
                      const CUtensorMap* maps = nullptr) {
    using TS = lbm::sgtc::TcShape<BN, STAGES, BMN, lbm::sgtc::slice_k(TMA)>;
    // the shared-memory opt-in is per device: one bit per device ordinal that has it (setting it
    // twice from racing host threads is harmless)
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(lbm::sgtc::k_gemm_tc<BN, STAGES, AMN, BMN, GA, GD, GAM, TMA>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, TS::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    int* flag = tc_flag().dev;
    if (!flag) return cudaErrorMemoryAllocation;
    dim3 grid((a.N + BN - 1) / BN, (a.M + lbm::sgtc::BM - 1) / lbm::sgtc::BM, splits);
    static const CUtensorMap none[3] = {};
    const CUtensorMap* m = maps ? maps : none;
    lbm::sgtc::k_gemm_tc<BN, STAGES, AMN, BMN, GA, GD, GAM, TMA>
        <<<grid, lbm::sgtc::TC_THREADS, TS::SMEM_BYTES, st>>>(a, flag, m[0], m[1], m[2]);
    return cudaGetLastError();
}

// C = A B on the tcgen05 tensor cores, each operand K-major or MN-major (AMN, BMN). The N tile
// is the compiled width that covers N with the fewest computed columns (ties: fewer tiles);
// wide tiles keep two stages so that two CTAs share an SM and one's epilogue overlaps the
// other's MMAs. GA / GAM: A (K-major / MN-major) is the implicit im2col of a.conv; GD: A is the
// gathered data-gradient operand a.dg.
int pick_bn(int N) {
    static const int widths[] = {32, 64, 80, 128, 144, 192, 256};
    int best = 256, best_cols = 1 << 30, best_tiles = 1 << 30;
    for (int w : widths) {
        const int tiles = (N + w - 1) / w, cols = tiles * w;
        if (cols < best_cols || (cols == best_cols && tiles < best_tiles)) {
            best = w;
            best_cols = cols;
            best_tiles = tiles;
        }
    }
    return best;
}

template <bool AMN, bool BMN, bool GA = false, bool GD = false, bool GAM = false>
cudaError_t gemm_tc(cudaStream_t st, const GemmArgs& a, int splits = 1) {
    switch (pick_bn(a.N)) {
        case 32: return launch_tc<32, 3, AMN, BMN, GA, GD, GAM>(st, a, splits);
        case 64: return launch_tc<64, 3, AMN, BMN, GA, GD, GAM>(st, a, splits);
        case 80: return launch_tc<80, 4, AMN, BMN, GA, GD, GAM>(st, a, splits);
        case 128: return launch_tc<128, 3, AMN, BMN, GA, GD, GAM>(st, a, splits);
        case 144: return launch_tc<144, 2, AMN, BMN, GA, GD, GAM>(st, a, splits);
        case 192: return launch_tc<192, 2, AMN, BMN, GA, GD, GAM>(st, a, splits);
        default: return launch_tc<256, 2, AMN, BMN, GA, GD, GAM>(st, a, splits);
    }
}

// cuTensorMapEncodeTiled from the driver (null if the driver does not provide it)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Map of an NHWC BF16 tensor [N][H][W][C] (C innermost), box ks channels x bw x bh pixels x 1
// image, ks = 64 with 128-byte or ks = 32 with 64-byte swizzle (the K-major layouts the MMAs
// read), out-of-range elements zero.
bool map_nhwc(CUtensorMap* m, const void* base, int C, int W, int H, int N, int bw, int bh,
              int ks, int step = 1) {
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dim[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t stride[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2,
                                  (cuuint64_t)H * W * C * 2};
    // step 2: every second pixel in x and y (the box spans 2 bw x 2 bh pixels, loads bw x bh)
    const cuuint32_t box[4] = {(cuuint32_t)ks, (cuuint32_t)(bw * step), (cuuint32_t)(bh * step), 1};
    const cuuint32_t es[4] = {1, (cuuint32_t)step, (cuuint32_t)step, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dim, stride, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE,
               ks == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Map of a row-major BF16 matrix [rows][K], box ks (K) x box_rows, swizzled as in map_nhwc.
bool map_rows(CUtensorMap* m, const void* base, int K, int rows, int box_rows, int ks) {
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t stride[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)ks, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dim, stride, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE,
               ks == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The TMA-fed gathering GEMM (GA or GD with tensor maps, see Conv::fmap / dmap), ks elements
// of K per stage: N tiles of 32, 64, 128 or 256 columns; few stages, so that several CTAs share
// an SM (each CTA's load latency overlaps the others' MMAs and epilogues).
template <bool GA, bool GD>
cudaError_t gemm_tc_tma(cudaStream_t st, const GemmArgs& a, int splits, const CUtensorMap* maps,
                        int ks) {
    const int bn = pick_bn(a.N);
    if (ks == 64) switch (bn) {
            case 32: return launch_tc<32, 3, false, false, GA, GD, false, 64>(st, a, splits, maps);
            case 64: return launch_tc<64, 3, false, false, GA, GD, false, 64>(st, a, splits, maps);
            case 128: return launch_tc<128, 3, false, false, GA, GD, false, 64>(st, a, splits, maps);
            case 256: return launch_tc<256, 2, false, false, GA, GD, false, 64>(st, a, splits, maps);
            default: break;
        }
    if (ks == 32) switch (bn) {
            case 32: return launch_tc<32, 4, false, false, GA, GD, false, 32>(st, a, splits, maps);
            case 64: return launch_tc<64, 4, false, false, GA, GD, false, 32>(st, a, splits, maps);
            case 128: return launch_tc<128, 6, false, false, GA, GD, false, 32>(st, a, splits, maps);
            case 256: return launch_tc<256, 4, false, false, GA, GD, false, 32>(st, a, splits, maps);
            default: break;
        }
    return cudaErrorInvalidValue;
}

// The gathering GEMMs (GA: forward convolution, GD: data gradient) with fewer output tiles than
// about three quarters of the SMs (the coarse levels): K is cut into up to 2 x 152 / tiles ranges
// of whole 64-wide slices, at least four each, whose FP32 partials k_splitk_finish sums in a
// fixed order before applying the GEMM's own epilogue (bias, leaky ReLU, BF16 or accumulated
// FP32 stores). Otherwise one launch as usual.
template <bool GA, bool GD>
cudaError_t gemm_tc_split(cudaStream_t st, const GemmArgs& a, float* scratch,
                          size_t scratch_elems, const CUtensorMap* maps = nullptr, int ks = 0) {
    const int bn = pick_bn(a.N);
    const long long tiles =
        (long long)((a.N + bn - 1) / bn) * ((a.M + lbm::sgtc::BM - 1) / lbm::sgtc::BM);
    const int nkt = (a.K + lbm::sgtc::BK - 1) / lbm::sgtc::BK;
    long long splits = 1;
    if (tiles < 114 && a.N % 4 == 0 && !a.tout && !a.kchunk && !a.rperm)
        splits = std::min<long long>(2 * 152 / tiles, nkt / 4);
    while (splits > 1 && (size_t)splits * a.M * a.N > scratch_elems) --splits;
    if (splits <= 1)
        return ks ? gemm_tc_tma<GA, GD>(st, a, 1, maps, ks) : gemm_tc<false, false, GA, GD>(st, a);
    const int chunk = (int)((nkt + splits - 1) / splits) * lbm::sgtc::BK;
    const int nsp = (a.K + chunk - 1) / chunk;
    GemmArgs p = a;
    p.Cf = scratch;
    p.Cb = nullptr;
    p.Cf2 = nullptr;
    p.ldc = a.N;
    p.ldc2 = 0;
    p.nsplit = 0;
    p.bias = nullptr;
    p.relu = 0;
    p.accumulate = 0;
    p.kchunk = chunk;
    p.split_stride = (long long)a.M * a.N;
    cudaError_t e = ks ? gemm_tc_tma<GA, GD>(st, p, nsp, maps, ks)
                       : gemm_tc<false, false, GA, GD>(st, p, nsp);
    if (e != cudaSuccess) return e;
    k_splitk_finish<<<blocks_for((long long)a.M * a.N / 4), kT, 0, st>>>(
        scratch, nsp, a.M, a.N, a.bias, a.relu, a.Cb, a.Cf, a.ldc, a.Cf2, a.ldc2, a.nsplit,
        a.accumulate);
    return cudaGetLastError();
}

// AK / BK: operand stored K-major (else MN-major)
template <bool AK, bool BK>
cudaError_t gemm(cudaStream_t st, const GemmArgs& a) {
    return gemm_tc<!AK, !BK>(st, a);
}

// Weight-gradient GEMM dW[co][k] = sum_p dY[p][co] col[p][k] (K = pixels, both operands
// MN-major): few output tiles and a very long K, so K is split over up to 128 CTA slices whose
// FP32 partials are summed in a fixed order. gather: computed transposed, dW^T = col^T dY with
// the im2col columns gathered by the loader as the 128-row operand (each thread decodes its tap
// and channel once) and stored transposed; else from the im2col buffer a.B.
// The TMA-fed weight gradient (gathered and transposed, maps: Conv::wmap): N tiles of 32, 64,
// 128 or 256 columns, few stages as in gemm_tc_tma.
cudaError_t gemm_wgrad_tma(cudaStream_t st, const GemmArgs& a, int splits, const CUtensorMap* maps) {
    switch (pick_bn(a.N)) {
        case 32: return launch_tc<32, 3, true, true, false, false, true, 1>(st, a, splits, maps);
        case 64: return launch_tc<64, 3, true, true, false, false, true, 1>(st, a, splits, maps);
        case 128: return launch_tc<128, 3, true, true, false, false, true, 1>(st, a, splits, maps);
        case 256: return launch_tc<256, 2, true, true, false, false, true, 1>(st, a, splits, maps);
        default: return cudaErrorInvalidValue;
    }
}

// Launch of k_gemm_wwin over `splits` K ranges (one CTA each).
template <int BN, int CB>
cudaError_t launch_wwin(cudaStream_t st, const GemmArgs& a, int splits, const CUtensorMap* maps) {
    constexpr int STAGES = 4;
    constexpr int STAGE = CB * 4 * 72 * 64 + BN * 128;
    constexpr int RAW = 1024 + STAGES * STAGE + 8 * (2 * STAGES + 1) + 16;
    constexpr int CTAS = 512 / (int)lbm::sgtc::tmem_pow2(3 * CB * BN);
    constexpr int MINB = 233472 / (CTAS + 1) + 1;
    constexpr int SMEM = RAW > MINB ? RAW : MINB;
    auto* kern = lbm::sgtc::k_gemm_wwin<BN, CB, STAGES>;
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    int* flag = tc_flag().dev;
    if (!flag) return cudaErrorMemoryAllocation;
    kern<<<splits, lbm::sgtc::TC_THREADS, SMEM, st>>>(a, flag, maps[0], maps[1], maps[2]);
    return cudaGetLastError();
}

// Launch of k_gemm_fwin: one CTA per tile of 128 pixels x BN columns.
template <int BN, int CB, bool GD>
cudaError_t launch_fwin(cudaStream_t st, const GemmArgs& a, const CUtensorMap* maps) {
    // 512-byte alignment slack (the 64-byte swizzle repeats every 512 bytes): 45,088 bytes at
    // BN = 32, five CTAs per SM
    constexpr int SMEM = 512 + CB * 3 * 136 * 64 + 9 * CB * BN * 64 + 32;
    auto* kern = lbm::sgtc::k_gemm_fwin<BN, CB, GD>;
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    int* flag = tc_flag().dev;
    if (!flag) return cudaErrorMemoryAllocation;
    dim3 grid(a.N / BN, a.M / lbm::sgtc::BM);
    kern<<<grid, lbm::sgtc::TC_THREADS, SMEM, st>>>(a, flag, maps[0], maps[1], maps[2]);
    return cudaGetLastError();
}

// The window-fed forward (GD false) or data gradient of a convolution that qualifies (see
// Conv::fw_cb / dw_cb): a.M a multiple of 128, a.N of bn.
template <bool GD>
cudaError_t gemm_fwin(cudaStream_t st, const GemmArgs& a, int cb, int bn, const CUtensorMap* maps) {
    if (a.M % lbm::sgtc::BM || a.N % bn) return cudaErrorInvalidValue;
    if (cb == 1 && bn == 32) return launch_fwin<32, 1, GD>(st, a, maps);
    if (cb == 1 && bn == 64) return launch_fwin<64, 1, GD>(st, a, maps);
    return cudaErrorInvalidValue;
}

// The weight gradient through k_gemm_wwin (a: the transposed, gathered form of gemm_wgrad):
// K ranges of at least 16 slices, at most two per SM, their partials summed in order.
cudaError_t gemm_wgrad_window(cudaStream_t st, GemmArgs a, float* scratch, size_t scratch_elems,
                              float* out, int cb, const CUtensorMap* maps) {
    const long long stride = (long long)a.N * a.ldc;
    const int slices = a.K / 64;
    int splits = std::max(1, std::min(304, slices / 16));
    while (splits > 1 && (size_t)splits * stride > scratch_elems) splits /= 2;
    const int chunk = (slices + splits - 1) / splits * 64;
    splits = (a.K + chunk - 1) / chunk;
    a.kchunk = chunk;
    a.split_stride = splits > 1 ? stride : 0;
    a.Cf = splits > 1 ? scratch : out;
    cudaError_t e = cudaErrorInvalidValue;
    if (a.N == 32 && cb == 1) e = launch_wwin<32, 1>(st, a, splits, maps);
    if (a.N == 32 && cb == 2) e = launch_wwin<32, 2>(st, a, splits, maps);
    if (a.N == 64 && cb == 1) e = launch_wwin<64, 1>(st, a, splits, maps);
    if (a.N == 64 && cb == 2) e = launch_wwin<64, 2>(st, a, splits, maps);
    if (e != cudaSuccess || splits == 1) return e;
    if (stride % 4 == 0 && ((uintptr_t)out & 15) == 0)
        k_splitk_sum4<<<(unsigned)((stride / 4 + 31) / 32), 256, 0, st>>>(scratch, splits, stride,
                                                                          stride, out);
    else
        k_splitk_sum<<<blocks_for(stride), kT, 0, st>>>(scratch, splits, stride, stride, out);
    return cudaGetLastError();
}

cudaError_t gemm_wgrad(cudaStream_t st, GemmArgs a, float* scratch, size_t scratch_elems,
                       float* out, bool gather, const CUtensorMap* maps = nullptr,
                       int ww_cb = 0, const CUtensorMap* wwmaps = nullptr) {
    if (gather) {
        // rows: the 9 C_in im2col columns; columns: C_out; a.ldc (= 9 C_in) stays the row
        // length of dW, written at dW[n * ldc + m]
        GemmArgs t = a;
        t.M = a.N;
        t.N = a.M;
        t.B = a.A;
        t.ldb = a.lda;
        t.tout = 1;
        a = t;
        if (ww_cb) return gemm_wgrad_window(st, a, scratch, scratch_elems, out, ww_cb, wwmaps);
    }
    // enough K slices for every SM to hold as many CTAs as fit (three of the narrow tiles, two
    // of the wide ones): each CTA keeps only two K-slices of gathers in flight
    const int bn = pick_bn(a.N);
    const int tiles = ((a.N + bn - 1) / bn) * ((a.M + lbm::sgtc::BM - 1) / lbm::sgtc::BM);
    const int occ = bn <= 64 && !maps ? 3 : 2;
    int splits = std::max(1, std::min(128, occ * 152 / std::max(1, tiles)));
    const long long stride = gather ? (long long)a.N * a.ldc : (long long)a.M * a.ldc;
    while (splits > 1 && (size_t)splits * stride > scratch_elems) splits /= 2;
    if (splits == 1) {
        a.Cf = out;
        return maps     ? gemm_wgrad_tma(st, a, 1, maps)
               : gather ? gemm_tc<true, true, false, false, true>(st, a)
                        : gemm_tc<true, true>(st, a);
    }
    int chunk = (a.K + splits - 1) / splits;
    chunk = (chunk + lbm::sgtc::BK - 1) / lbm::sgtc::BK * lbm::sgtc::BK;
    splits = (a.K + chunk - 1) / chunk;
    a.Cf = scratch;
    a.kchunk = chunk;
    a.split_stride = stride;
    cudaError_t e = maps     ? gemm_wgrad_tma(st, a, splits, maps)
                    : gather ? gemm_tc<true, true, false, false, true>(st, a, splits)
                             : gemm_tc<true, true>(st, a, splits);
    if (e != cudaSuccess) return e;
    if (stride % 4 == 0 && ((uintptr_t)out & 15) == 0)
        k_splitk_sum4<<<(unsigned)((stride / 4 + 31) / 32), 256, 0, st>>>(scratch, splits, stride,
                                                                          stride, out);
    else
        k_splitk_sum<<<blocks_for(stride), kT, 0, st>>>(scratch, splits, stride, stride, out);
    return cudaGetLastError();
}

// BF16 copies of the weights (after the FP32 masters changed): W for the forward pass and the
// weight gradient, the rearranged copy for the data gradient
cudaError_t refresh_bf16_weights(lbm_surrogate* s) {
    k_bf16_copies<<<blocks_for((long long)s->nparams), kT, 0, s->stream>>>(
        s->w, (long long)s->nparams, s->wb, s->wbd, s->tab);
    return cudaGetLastError();
}

int ilog2_exact(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return (1 << l) == v ? l : -1;
}

PixDims pix_dims(int H, int W) { return PixDims{H, W, ilog2_exact(H), ilog2_exact(W)}; }

// im2col of convolution c (channel groups of 8, a power of two, checked at creation)
cudaError_t launch_im2col(lbm_surrogate* s, const Conv& c, int B) {
    const bf16* x1 = s->t[c.src1].y;
    const bf16* x2 = c.src2 >= 0 ? s->t[c.src2].y : nullptr;
    const PixDims d = pix_dims(c.H, c.W);
    const int P = B * c.H * c.W;
    const int lc8 = ilog2_exact((c.C1 + c.C2) / 8);
    const long long total = (long long)P * 9 * ((c.C1 + c.C2) / 8);
    if (d.lh >= 0 && d.lw >= 0)
        k_im2col<true><<<blocks_for(total), kT, 0, s->stream>>>(x1, c.C1, c.up1, x2, c.C2, d, P,
                                                                lc8, s->col);
    else
        k_im2col<false><<<blocks_for(total), kT, 0, s->stream>>>(x1, c.C1, c.up1, x2, c.C2, d, P,
                                                                 lc8, s->col);
    return cudaGetLastError();
}

int add_tensor(lbm_surrogate* s, int H, int W, int C) {
    Tensor x;
    x.H = H;
    x.W = W;
    x.C = C;
    s->t.push_back(x);
    return (int)s->t.size() - 1;
}

int add_conv(lbm_surrogate* s, int src1, int up1, int src2, int Cout) {
    Conv c;
    c.src1 = src1;
    c.C1 = s->t[src1].C;
    c.up1 = up1;
    c.src2 = src2;
    c.C2 = src2 >= 0 ? s->t[src2].C : 0;
    c.H = up1 ? s->t[src1].H * 2 : s->t[src1].H;
    c.W = up1 ? s->t[src1].W * 2 : s->t[src1].W;
    c.Cout = Cout;
    c.out = add_tensor(s, c.H, c.W, Cout);
    c.w_off = s->nparams;
    s->nparams += (size_t)Cout * 9 * (c.C1 + c.C2);
    c.b_off = s->nparams;
    s->nparams += Cout;
    s->convs.push_back(c);
    return c.out;
}

void build(lbm_surrogate* s) {
    const int b = s->base;
    int x = add_tensor(s, s->H, s->W, 8);
    int s1 = add_conv(s, add_conv(s, x, 0, -1, b), 0, -1, b);
    int p1 = add_tensor(s, s->H / 2, s->W / 2, b);
    s->pools.push_back({s1, p1});
    int s2 = add_conv(s, add_conv(s, p1, 0, -1, 2 * b), 0, -1, 2 * b);
    int p2 = add_tensor(s, s->H / 4, s->W / 4, 2 * b);
    s->pools.push_back({s2, p2});
    int s3 = add_conv(s, add_conv(s, p2, 0, -1, 4 * b), 0, -1, 4 * b);
    int p3 = add_tensor(s, s->H / 8, s->W / 8, 4 * b);
    s->pools.push_back({s3, p3});
    int bt = add_conv(s, add_conv(s, p3, 0, -1, 8 * b), 0, -1, 8 * b);
    int u3 = add_conv(s, bt, 1, -1, 4 * b);
    int d3 = add_conv(s, add_conv(s, u3, 0, s3, 4 * b), 0, -1, 4 * b);
    int u2 = add_conv(s, d3, 1, -1, 2 * b);
    int d2 = add_conv(s, add_conv(s, u2, 0, s2, 2 * b), 0, -1, 2 * b);
    int u1 = add_conv(s, d2, 1, -1, b);
    int d1 = add_conv(s, add_conv(s, u1, 0, s1, b), 0, -1, b);
    s->head_in = d1;
    s->head_w = s->nparams;
    s->nparams += b;
    s->head_b = s->nparams;
    s->nparams += 1;
}

lbm_status forward(lbm_surrogate* s, const bf16* x, int B) {
    s->t[0].y = const_cast<bf16*>(x);
    // convolutions run in production order; a pool runs right after the conv that feeds it
    for (const Conv& c : s->convs) {
        const Tensor& a = s->t[c.src1];
        if (a.y == nullptr) return sfail(s, LBM_ERR_STATE, "surrogate: missing activation");
        const int Cin = c.C1 + c.C2;
        const long long P = (long long)B * c.H * c.W;
        // implicit GEMM: the 3 x 3 neighbourhoods are gathered from the activations by the
        // tensor-core kernel's loader (no im2col buffer)
        GemmArgs g{};
        g.conv.x1 = a.y;
        g.conv.x2 = c.src2 >= 0 ? s->t[c.src2].y : nullptr;
        g.conv.C1 = c.C1;
        g.conv.C2 = c.C2;
        g.conv.up1 = c.up1;
        g.conv.H = c.H;
        g.conv.W = c.W;
        g.conv.lc = ilog2_exact(Cin);
        g.B = s->wb + c.w_off;
        g.M = (int)P;
        g.N = c.Cout;
        g.K = 9 * Cin;
        g.ldb = 9 * Cin;
        g.Cb = s->t[c.out].y;
        g.ldc = c.Cout;
        g.bias = s->w + c.b_off;
        g.relu = 1;
        if (c.up1 && c.f_ks) g.rperm = std::min(c.W, 128) / 2;
        if (c.fw_cb)
            SCUDA(s, gemm_fwin<false>(s->stream, g, c.fw_cb, c.fw_bn, c.fwmap));
        else
            SCUDA(s, (gemm_tc_split<true, false>(s->stream, g, s->splitk, s->splitk_elems, c.fmap,
                                                  c.f_ks)));
        // a pool whose source is this conv's output runs right after it
        for (const auto& pl : s->pools)
            if (pl.first == c.out) {
                const Tensor& src = s->t[pl.first];
                k_avgpool<<<blocks_for((long long)B * src.H * src.W * src.C / 4), kT, 0,
                            s->stream>>>(src.y, s->t[pl.second].y, B, src.H, src.W, src.C);
            }
    }
    return LBM_OK;
}

// Tensor maps for the forward and data-gradient GEMMs whose A operand the copy engine can fetch
// as boxes: no upsampled source, channel counts multiples of 64 (one K-slice of 64 = one tap of
// one source) or else of 32 (slices of 32), the 128 rows of a tile a whole block of pixels of
// one image, and N tiles of 32, 64, 128 or 256 columns. The network input (its pointer changes
// per call) never qualifies.
void make_tensor_maps(lbm_surrogate* s) {
    auto tma_width = [](int bn) { return bn == 32 || bn == 64 || bn == 128 || bn == 256; };
    auto slice = [](int a, int b) { return a % 64 == 0 && b % 64 == 0 ? 64
                                         : a % 32 == 0 && b % 32 == 0 ? 32 : 0; };
    for (Conv& c : s->convs) {
        const int W = c.W, H = c.H;
        if (c.up1 && c.src1 != 0) {
            // forward of an upsampling convolution: tile rows in runs of even, then odd output
            // columns, each run a box of half a tile row of source pixels
            const int fk = slice(c.C1, c.C2);
            if ((W % 128 == 0 || 128 % W == 0) && (H * W) % 128 == 0 && W >= 16 && fk &&
                c.C2 == 0 && tma_width(pick_bn(c.Cout)) &&
                map_nhwc(&c.fmap[0], s->t[c.src1].y, c.C1, W / 2, H / 2, s->maxB,
                         std::min(W, 128) / 2, 1, fk) &&
                map_rows(&c.fmap[2], s->wb + c.w_off, 9 * c.C1, c.Cout, pick_bn(c.Cout), fk))
                c.f_ks = fk;
            // data gradient of an upsampling convolution: rows are source pixels (half
            // resolution), the output gradient read every second pixel; B wraps every 9 Cout
            const int Ws = W / 2, Hs = H / 2, cin = c.C1 + c.C2, dk = slice(c.Cout, 0);
            if ((Ws % 128 == 0 || 128 % Ws == 0) && (Hs * Ws) % 128 == 0 && dk &&
                (9 * c.Cout) % dk == 0 && tma_width(pick_bn(cin))) {
                const int bw = std::min(Ws, 128), bh = 128 / bw;
                if (map_nhwc(&c.dmap[0], s->gmask, c.Cout, W, H, s->maxB, bw, bh, dk, 2) &&
                    map_rows(&c.dmap[2], s->wbd + c.w_off, 9 * c.Cout, cin, pick_bn(cin), dk))
                    c.d_ks = dk;
            }
            // weight gradient: 32 source pixels x 32 channels per box, and 32 output-gradient
            // pixels taken every second one
            if (W % 64 == 0 && c.C2 == 0 && c.C1 % 32 == 0 && c.Cout % 32 == 0 &&
                tma_width(pick_bn(c.Cout)))
                c.w_tma = map_nhwc(&c.wmap[0], s->t[c.src1].y, c.C1, Ws, Hs, s->maxB, 32, 1, 32) &&
                          map_nhwc(&c.wmap[2], s->gmask, c.Cout, W, H, s->maxB, 32, 1, 32, 2);
            continue;
        }
        if (!((W % 128 == 0 || 128 % W == 0) && (H * W) % 128 == 0) || c.src1 == 0)
            continue;
        const int bw = std::min(W, 128), bh = 128 / bw, cin = c.C1 + c.C2;
        const int fk = slice(c.C1, c.C2), dk = slice(c.Cout, 0);
        if (fk && tma_width(pick_bn(c.Cout)) &&
            map_nhwc(&c.fmap[0], s->t[c.src1].y, c.C1, W, H, s->maxB, bw, bh, fk) &&
            (c.src2 < 0 || map_nhwc(&c.fmap[1], s->t[c.src2].y, c.C2, W, H, s->maxB, bw, bh, fk)) &&
            map_rows(&c.fmap[2], s->wb + c.w_off, 9 * cin, c.Cout, pick_bn(c.Cout), fk))
            c.f_ks = fk;
        // window-fed forward and data gradient: 128-pixel row segments, a window operand of 32
        // channels (the input for the forward, dY for the data gradient) and 32 or 64 output
        // columns (at most 64 KB of shared memory, five or three CTAs per SM). With 64 window
        // channels (90 KB and two CTAs per SM, each loading, multiplying and storing in turn,
        // or one CTA per SM at N = 64) the pipelined TMA path is faster, so those keep it.
        if (W % 128 == 0 && (long long)s->maxB * H * W / 128 <= 65535) {
            if (cin == 32 && c.C2 == 0 && (c.Cout == 32 || c.Cout == 64) &&
                map_nhwc(&c.fwmap[0], s->t[c.src1].y, c.C1, W, H, s->maxB, 136, 3, 32) &&
                map_rows(&c.fwmap[2], s->wb + c.w_off, 9 * cin, c.Cout, c.Cout, 32)) {
                c.fw_cb = 1;
                c.fw_bn = c.Cout;
            }
            if (c.Cout == 32 && c.C1 % 32 == 0 && c.C2 % 32 == 0 && (cin == 32 || cin == 64) &&
                map_nhwc(&c.dwmap[0], s->gmask, c.Cout, W, H, s->maxB, 136, 3, 32) &&
                map_rows(&c.dwmap[2], s->wbd + c.w_off, 9 * c.Cout, cin, cin, 32)) {
                c.dw_cb = 1;
                c.dw_bn = cin;
            }
        }
        if (W % 64 == 0 && c.C1 % 32 == 0 && c.C2 % 32 == 0 && (cin == 32 || cin == 64) &&
            (c.Cout == 32 || c.Cout == 64)) {
            const int wc = cin / 32;
            if (map_nhwc(&c.wwmap[0], s->t[c.src1].y, c.C1, W, H, s->maxB, 72, 3, 32) &&
                (c.src2 < 0 ||
                 map_nhwc(&c.wwmap[1], s->t[c.src2].y, c.C2, W, H, s->maxB, 72, 3, 32)) &&
                map_nhwc(&c.wwmap[2], s->gmask, c.Cout, W, H, s->maxB, 64, 1, 32))
                c.ww_cb = wc;
        }
        if (W % 64 == 0 || 64 % W == 0) {
            const int ww = std::min(W, 64), wh = 64 / ww;
            c.w_tma = c.C1 % 32 == 0 && c.C2 % 32 == 0 && c.Cout % 32 == 0 &&
                      tma_width(pick_bn(c.Cout)) &&
                      map_nhwc(&c.wmap[0], s->t[c.src1].y, c.C1, W, H, s->maxB, ww, wh, 32) &&
                      (c.src2 < 0 ||
                       map_nhwc(&c.wmap[1], s->t[c.src2].y, c.C2, W, H, s->maxB, ww, wh, 32)) &&
                      map_nhwc(&c.wmap[2], s->gmask, c.Cout, W, H, s->maxB, ww, wh, 32);
        }
        if (dk && tma_width(pick_bn(cin)) &&
            map_nhwc(&c.dmap[0], s->gmask, c.Cout, W, H, s->maxB, bw, bh, dk) &&
            map_rows(&c.dmap[2], s->wbd + c.w_off, 9 * c.Cout, cin, pick_bn(cin), dk))
            c.d_ks = dk;
    }
}

}  // namespace

extern "C" {

lbm_status lbm_surrogate_create(int32_t H, int32_t W, int32_t base, int32_t max_batch,
                                int32_t device, lbm_surrogate** out) {
    if (!out) return sfail(nullptr, LBM_ERR_ARG, "lbm_surrogate_create: out is NULL");
    *out = nullptr;
    if (H <= 0 || W <= 0 || H % 8 || W % 8 || (base != 8 && base != 16 && base != 32) ||
        max_batch <= 0)
        return sfail(nullptr, LBM_ERR_ARG,
                     "lbm_surrogate_create: H, W multiples of 8, base 8, 16 or 32, batch > 0");
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return sfail(nullptr, LBM_ERR_CUDA, "lbm_surrogate_create: cannot select the device");
    }
    lbm_surrogate* s = new lbm_surrogate();
    s->H = H;
    s->W = W;
    s->base = base;
    s->maxB = max_batch;
    s->device = device;
    build(s);
    s->tab.n = std::min<int>(24, (int)s->convs.size());  // 17 convolutions
    for (int k = 0; k < s->tab.n; ++k) {
        s->tab.off[k] = (long long)s->convs[k].w_off;
        s->tab.cout[k] = s->convs[k].Cout;
        s->tab.cin[k] = s->convs[k].C1 + s->convs[k].C2;
    }
    auto cleanup = [&](const char* e) {
        lbm_surrogate_destroy(s);
        return sfail(nullptr, LBM_ERR_CUDA, std::string("lbm_surrogate_create: ") + e);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(cudaGetErrorString(e));
    size_t colmax = 0;
    for (const Conv& c : s->convs)
        colmax = std::max(colmax, (size_t)max_batch * c.H * c.W * 9 * (c.C1 + c.C2));
    s->col_elems = colmax;
    for (size_t k = 1; k < s->t.size() && e == cudaSuccess; ++k) {
        Tensor& x = s->t[k];
        const size_t n = (size_t)max_batch * x.H * x.W * x.C;
        e = cudaMalloc((void**)&x.y, n * sizeof(bf16));
        if (e == cudaSuccess) e = cudaMalloc((void**)&x.dy, n * sizeof(float));
        s->act_elems = std::max(s->act_elems, n);
    }
    const size_t np = s->nparams;
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->w, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->g, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->m, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->v, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->wb, np * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->wbd, np * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->col, colmax * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->gmask, s->act_elems * sizeof(bf16));
    if (e == cudaSuccess)
        e = cudaMalloc((void**)&s->part, (size_t)s->part_blocks * 8 * base * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->phi, (size_t)max_batch * H * W * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc((void**)&s->hpart, (size_t)s->part_blocks * (base + 2) * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc((void**)&s->bpart, (size_t)kReluBlocks * 8 * base * sizeof(float));
    size_t wmax = 0;
    for (const Conv& c : s->convs) wmax = std::max(wmax, (size_t)c.Cout * 9 * (c.C1 + c.C2));
    s->splitk_elems = std::min<size_t>(wmax * 128, (size_t)64 << 20);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->splitk, s->splitk_elems * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(s->w, 0, np * sizeof(float), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->m, 0, np * sizeof(float), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->v, 0, np * sizeof(float), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->wb, 0, np * sizeof(bf16), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->wbd, 0, np * sizeof(bf16), s->stream);
    if (e != cudaSuccess) return cleanup(cudaGetErrorString(e));
    make_tensor_maps(s);
    *out = s;
    return LBM_OK;
}

int64_t lbm_surrogate_num_params(const lbm_surrogate* s) { return s ? (int64_t)s->nparams : 0; }

lbm_status lbm_surrogate_set_weights(lbm_surrogate* s, const float* host, int64_t n) {
    if (!s || !host || n != (int64_t)s->nparams)
        return sfail(s, LBM_ERR_ARG, "lbm_surrogate_set_weights: need num_params floats");
    SCUDA(s, cudaSetDevice(s->device));
    SCUDA(s, cudaMemcpyAsync(s->w, host, n * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    SCUDA(s, refresh_bf16_weights(s));
    SCUDA(s, cudaMemsetAsync(s->m, 0, n * sizeof(float), s->stream));
    SCUDA(s, cudaMemsetAsync(s->v, 0, n * sizeof(float), s->stream));
    s->adam_t = 0;
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

lbm_status lbm_surrogate_get_weights(lbm_surrogate* s, float* host, int64_t n, int32_t grads) {
    if (!s || !host || n != (int64_t)s->nparams)
        return sfail(s, LBM_ERR_ARG, "lbm_surrogate_get_weights: need num_params floats");
    SCUDA(s, cudaSetDevice(s->device));
    SCUDA(s, cudaMemcpyAsync(host, grads ? s->g : s->w, n * sizeof(float), cudaMemcpyDeviceToHost,
                             s->stream));
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

lbm_status lbm_surrogate_forward(lbm_surrogate* s, const void* x, int32_t B, float* phi_out) {
    lbm::NvtxRange nvtx_("lbm_surrogate_forward");
    if (!s || !x || !phi_out || B <= 0 || B > s->maxB)
        return sfail(s, LBM_ERR_ARG, "lbm_surrogate_forward: bad arguments");
    SCUDA(s, cudaSetDevice(s->device));
    lbm_status st = forward(s, (const bf16*)x, B);
    if (st != LBM_OK) return st;
    const long long P = (long long)B * s->H * s->W;
    const int nb = std::min(s->part_blocks, blocks_for(P));
    if (s->base == 32)
        k_head<32><<<nb, kT, 0, s->stream>>>(s->t[s->head_in].y, s->w + s->head_w,
                                             s->w + s->head_b, phi_out, P, nullptr, nullptr, 0.f,
                                             nullptr, nullptr);
    else if (s->base == 8)
        k_head<8><<<nb, kT, 0, s->stream>>>(s->t[s->head_in].y, s->w + s->head_w,
                                            s->w + s->head_b, phi_out, P, nullptr, nullptr, 0.f,
                                            nullptr, nullptr);
    else if (s->base == 16)
        k_head<16><<<nb, kT, 0, s->stream>>>(s->t[s->head_in].y, s->w + s->head_w,
                                             s->w + s->head_b, phi_out, P, nullptr, nullptr, 0.f,
                                             nullptr, nullptr);
    else
        return sfail(s, LBM_ERR_ARG, "lbm_surrogate_forward: base must be 8, 16 or 32");
    SCUDA(s, cudaGetLastError());
    SCUDA(s, cudaStreamSynchronize(s->stream));
    if (tc_timed_out())
        return sfail(s, LBM_ERR_TIMEOUT, "lbm_surrogate_forward: a tensor-core wait timed out");
    return LBM_OK;
}

// Gradients of the masked MSE into s->g; with lr > 0 also an Adam update. *loss gets the loss.
lbm_status lbm_surrogate_train_step(lbm_surrogate* s, const void* xin, const float* target,
                                    const uint8_t* mask, int32_t B, float lr, double* loss) {
    lbm::NvtxRange nvtx_("lbm_surrogate_train_step");
    if (!s || !xin || !target || !mask || B <= 0 || B > s->maxB)
        return sfail(s, LBM_ERR_ARG, "lbm_surrogate_train_step: bad arguments");
    SCUDA(s, cudaSetDevice(s->device));
    lbm_status st = forward(s, (const bf16*)xin, B);
    if (st != LBM_OK) return st;
    const long long P = (long long)B * s->H * s->W;
    std::vector<uint8_t> hm;
    // zero all activation gradients (they accumulate from several consumers)
    for (size_t k = 1; k < s->t.size(); ++k) {
        const Tensor& x = s->t[k];
        SCUDA(s, cudaMemsetAsync(x.dy, 0, (size_t)B * x.H * x.W * x.C * sizeof(float), s->stream));
    }
    SCUDA(s, cudaMemsetAsync(s->g, 0, s->nparams * sizeof(float), s->stream));
    float inv_n = 1.f / (float)P;
    {
        // number of loss pixels: the mask (B*H*W bytes) is counted on the host once per step
        hm.resize((size_t)P);
        SCUDA(s, cudaMemcpyAsync(hm.data(), mask, (size_t)P, cudaMemcpyDeviceToHost, s->stream));
        SCUDA(s, cudaStreamSynchronize(s->stream));
        long long cnt = 0;
        for (uint8_t b : hm) cnt += b != 0;
        inv_n = cnt > 0 ? 1.f / (float)cnt : 0.f;
    }
    const int C = s->base;
    const int nb = std::min(s->part_blocks, blocks_for(P));
    Tensor& hin = s->t[s->head_in];
    if (C == 32)
        k_head<32><<<nb, kT, 0, s->stream>>>(hin.y, s->w + s->head_w, s->w + s->head_b, s->phi, P,
                                             target, mask, inv_n, hin.dy, s->hpart);
    else if (C == 16)
        k_head<16><<<nb, kT, 0, s->stream>>>(hin.y, s->w + s->head_w, s->w + s->head_b, s->phi, P,
                                             target, mask, inv_n, hin.dy, s->hpart);
    else if (C == 8)
        k_head<8><<<nb, kT, 0, s->stream>>>(hin.y, s->w + s->head_w, s->w + s->head_b, s->phi, P,
                                            target, mask, inv_n, hin.dy, s->hpart);
    else
        return sfail(s, LBM_ERR_ARG, "lbm_surrogate_train_step: base must be 8, 16 or 32");
    SCUDA(s, cudaGetLastError());
    // head gradients: sum the per-block partials (C weights, loss, bias)
    k_colsum_final<<<C + 2, kT, 0, s->stream>>>(s->hpart, nb, C + 2, s->part);
    SCUDA(s, cudaMemcpyAsync(s->g + s->head_w, s->part, C * sizeof(float),
                             cudaMemcpyDeviceToDevice, s->stream));
    SCUDA(s, cudaMemcpyAsync(s->g + s->head_b, s->part + C + 1, sizeof(float),
                             cudaMemcpyDeviceToDevice, s->stream));
    float hl = 0.f;
    SCUDA(s, cudaMemcpyAsync(&hl, s->part + C, sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    // backward through the convolutions (reverse order), pools interleaved
    for (int ci = (int)s->convs.size() - 1; ci >= 0; --ci) {
        const Conv& c = s->convs[ci];
        // gradient arriving at this conv's output also includes the pool path (already added,
        // pools run before: a pool's output gradient is complete once every later conv is done)
        const float* dyp = nullptr;
        for (const auto& pl : s->pools)
            if (pl.first == c.out) dyp = s->t[pl.second].dy;
        Tensor& o = s->t[c.out];
        const int Cin = c.C1 + c.C2;
        const long long Pc = (long long)B * c.H * c.W;
        const long long n_out = Pc * c.Cout;
        // leaky-ReLU adjoint (with the pool's), BF16 copy and the bias gradient's partial sums
        const int rb = (int)std::min<long long>(kReluBlocks, (n_out / 8 + kT - 1) / kT);
        if (dyp)
            k_relu_bias<true><<<rb, kT, 0, s->stream>>>(o.dy, dyp, o.y, s->gmask, n_out / 8,
                                                        c.Cout, c.H, c.W, s->bpart);
        else
            k_relu_bias<false><<<rb, kT, 0, s->stream>>>(o.dy, nullptr, o.y, s->gmask, n_out / 8,
                                                         c.Cout, c.H, c.W, s->bpart);
        k_colsum_final<<<c.Cout, kT, 0, s->stream>>>(s->bpart, rb, c.Cout, s->g + c.b_off, 1);
        // weight gradient: dW[co][k] = sum_p g[p][co] col[p][k], the im2col columns gathered by
        // the GEMM's loader when the resolution allows (powers of two), else from a buffer
        GemmArgs gw{};
        gw.conv.x1 = s->t[c.src1].y;
        gw.conv.x2 = c.src2 >= 0 ? s->t[c.src2].y : nullptr;
        gw.conv.C1 = c.C1;
        gw.conv.C2 = c.C2;
        gw.conv.up1 = c.up1;
        gw.conv.H = c.H;
        gw.conv.W = c.W;
        gw.conv.lc = ilog2_exact(Cin);
        gw.conv.lh = ilog2_exact(c.H);
        gw.conv.lw = ilog2_exact(c.W);
        const bool gather = gw.conv.lh >= 0 && gw.conv.lw >= 0;
        if (!gather) SCUDA(s, launch_im2col(s, c, B));
        gw.A = s->gmask;
        gw.B = s->col;
        gw.M = c.Cout;
        gw.N = 9 * Cin;
        gw.K = (int)Pc;
        gw.lda = c.Cout;
        gw.ldb = 9 * Cin;
        gw.ldc = 9 * Cin;
        SCUDA(s, gemm_wgrad(s->stream, gw, s->splitk, s->splitk_elems, s->g + c.w_off, gather,
                            gather && c.w_tma ? c.wmap : nullptr, gather ? c.ww_cb : 0, c.wwmap));
        // data gradient (not needed for the input tensor)
        if (c.src1 == 0) continue;
        // implicit GEMM over the source pixels: dX_src[q][ci] += sum over (sub-pixel, tap, co)
        // of dY gathered around q times the rearranged weights (no column buffer)
        if (c.up1 && c.C2 > 0) return sfail(s, LBM_ERR_STATE, "surrogate: upsampled cat source");
        GemmArgs gd{};
        gd.dg.dy = s->gmask;
        gd.dg.H = c.H;
        gd.dg.W = c.W;
        gd.dg.lco = ilog2_exact(c.Cout);
        gd.dg.up1 = c.up1;
        gd.B = s->wbd + c.w_off;
        gd.ldb = 9 * c.Cout;
        gd.kperiod = c.up1 ? 9 * c.Cout : 0;
        gd.M = (int)((long long)B * (c.H >> c.up1) * (c.W >> c.up1));
        gd.N = Cin;
        gd.K = (c.up1 ? 36 : 9) * c.Cout;
        gd.Cf = s->t[c.src1].dy;
        gd.ldc = c.C1;
        gd.accumulate = 1;
        if (c.C2 > 0) {
            gd.Cf2 = s->t[c.src2].dy;
            gd.ldc2 = c.C2;
            gd.nsplit = c.C1;
        }
        if (c.dw_cb)
            SCUDA(s, gemm_fwin<true>(s->stream, gd, c.dw_cb, c.dw_bn, c.dwmap));
        else
            SCUDA(s, (gemm_tc_split<false, true>(s->stream, gd, s->splitk, s->splitk_elems,
                                                  c.dmap, c.d_ks)));
    }
    if (lr > 0.f) {
        ++s->adam_t;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f / (1.f - powf(b1, (float)s->adam_t));
        const float c2 = 1.f / (1.f - powf(b2, (float)s->adam_t));
        k_adam<<<blocks_for((long long)s->nparams), kT, 0, s->stream>>>(
            s->w, s->g, s->m, s->v, (long long)s->nparams, lr, b1, b2, 1e-8f, c1, c2, s->wb, s->wbd,
            s->tab);
    }
    SCUDA(s, cudaGetLastError());
    SCUDA(s, cudaStreamSynchronize(s->stream));
    if (tc_timed_out())
        return sfail(s, LBM_ERR_TIMEOUT, "lbm_surrogate_train_step: a tensor-core wait timed out");
    if (loss) *loss = hl;
    return LBM_OK;
}

lbm_status lbm_surrogate_phi(lbm_surrogate* s, float* host_phi, int32_t B) {
    if (!s || !host_phi || B <= 0 || B > s->maxB)
        return sfail(s, LBM_ERR_ARG, "lbm_surrogate_phi: bad arguments");
    SCUDA(s, cudaMemcpyAsync(host_phi, s->phi, (size_t)B * s->H * s->W * sizeof(float),
                             cudaMemcpyDeviceToHost, s->stream));
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

// C = A * B with BF16 operands (device), FP32 output; a_kmajor / b_kmajor select the storage
// of A (M x K) and B (K x N): K-major A[m*lda + k], B[n*ldb + k]; MN-major A[k*lda + m],
// B[k*ldb + n].
lbm_status lbm_sg_gemm(const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                       int32_t a_kmajor, int32_t b_kmajor, int32_t lda, int32_t ldb, float* C,
                       int32_t ldc, void* stream) {
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0)
        return sfail(nullptr, LBM_ERR_ARG, "lbm_sg_gemm: bad arguments");
    if ((a_kmajor && (K % 8 || lda % 8)) || (!a_kmajor && (M % 8 || lda % 8)) ||
        (b_kmajor && (K % 8 || ldb % 8)) || (!b_kmajor && (N % 8 || ldb % 8)))
        return sfail(nullptr, LBM_ERR_ARG, "lbm_sg_gemm: alignment (multiples of 8) violated");
    if (tc_timed_out())
        return sfail(nullptr, LBM_ERR_TIMEOUT, "lbm_sg_gemm: an earlier tensor-core wait timed out");
    GemmArgs g{};
    g.A = (const bf16*)A;
    g.B = (const bf16*)B;
    g.M = M;
    g.N = N;
    g.K = K;
    g.lda = lda;
    g.ldb = ldb;
    g.Cf = C;
    g.ldc = ldc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (a_kmajor && b_kmajor)
        e = gemm<true, true>(st, g);
    else if (a_kmajor)
        e = gemm<true, false>(st, g);
    else if (b_kmajor)
        e = gemm<false, true>(st, g);
    else
        e = gemm<false, false>(st, g);
    if (e != cudaSuccess)
        return sfail(nullptr, LBM_ERR_CUDA, std::string("lbm_sg_gemm: ") + cudaGetErrorString(e));
    return LBM_OK;
}

// Host-side fault injection: latch the timeout flag exactly as a device wait that ran out
// would, so that callers can exercise their LBM_ERR_TIMEOUT path without stalling a GPU.
lbm_status lbm_sg_inject_timeout(void) {
    TcFlag& f = tc_flag();
    if (!f.host)
        return sfail(nullptr, LBM_ERR_CUDA,
                     "lbm_sg_inject_timeout: the mapped timeout flag could not be allocated");
    *f.host = 1;
    return LBM_OK;
}

void lbm_surrogate_destroy(lbm_surrogate* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (size_t k = 1; k < s->t.size(); ++k) {
        cudaFree(s->t[k].y);
        cudaFree(s->t[k].dy);
    }
    cudaFree(s->w);
    cudaFree(s->g);
    cudaFree(s->m);
    cudaFree(s->v);
    cudaFree(s->wb);
    cudaFree(s->wbd);
    cudaFree(s->col);
    cudaFree(s->gmask);
    cudaFree(s->part);
    cudaFree(s->phi);
    cudaFree(s->hpart);
    cudaFree(s->splitk);
    cudaFree(s->bpart);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char* lbm_surrogate_last_error(const lbm_surrogate* s) {
    return s ? s->err.c_str() : lbm_last_error(nullptr);
}

}  // extern "C"
