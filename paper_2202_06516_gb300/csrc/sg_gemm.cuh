// Argument block and shared helpers of the surrogate's GEMMs (the tensor-core kernel itself is
// in sg_tc.cuh): C[M x N] = A B with either operand stored K-major or MN-major. Requirements:
// K-major operands have K % 8 == 0 and 16-byte aligned rows; MN-major operands have M (resp. N)
// % 8 == 0; a split-K chunk is a multiple of the kernel's K slice. Out-of-range rows and columns
// are zero-filled on load and masked on store. Epilogue: optional bias[n], leaky ReLU (slope
// 0.1), FP32 or BF16 output, optional accumulation into FP32.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace lbm {
namespace sg {

// A operand gathered straight from NHWC activations (implicit im2col of a 3 x 3, pad-1
// convolution): A[p][(ky * 3 + kx) * C + c] = x(n, y + ky - 1, x + kx - 1, c) for output pixel
// p = (n, y, x), with channels [source 1 | source 2]; source 1 may be stored at half resolution
// (nearest 2x upsampling). C = C1 + C2 = 2^lc; C1 and C2 multiples of 8.
struct ConvGather {
    const __nv_bfloat16* x1;
    const __nv_bfloat16* x2;  // nullptr when C2 = 0
    int C1, C2, up1;
    int H, W;                 // output (full) resolution
    int lc;
    int lh, lw;               // log2 H, log2 W (the pixel-major gather needs powers of two)
};

// A operand of the data gradient gathered from the output gradient dY (NHWC, full resolution
// H x W, Cout = 2^lco channels): rows are pixels q of the source (full resolution, or half
// resolution when up1) and A[q][((s * 9) + tap) * Cout + co] = dY(f q + s - off(tap))[co], with
// off(tap) = (tap / 3 - 1, tap % 3 - 1), f = 2 and the 2 x 2 sub-pixel s = (sy, sx) when up1
// (the nearest upsampling's adjoint sums them), f = 1 and s = 0 otherwise; 0 outside the image.
struct DgradGather {
    const __nv_bfloat16* dy;
    int H, W;      // output resolution of the convolution
    int lco;       // log2 Cout
    int up1;
};

struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int M, N, K;
    int lda, ldb;      // element stride between consecutive rows of the stored matrix
    float* Cf;         // FP32 output (or nullptr)
    __nv_bfloat16* Cb; // BF16 output (or nullptr)
    int ldc;
    const float* bias; // per column n (or nullptr)
    int relu;          // apply the leaky ReLU max(v, 0.1 v)
    int accumulate;    // FP32 output: C += result
    int kchunk;        // split-K: blockIdx.z covers K range [z kchunk, (z + 1) kchunk); its FP32
                       // result goes to Cf + z * split_stride (0: no split)
    long long split_stride;
    ConvGather conv;   // used instead of A (or B) by the gathering (implicit-convolution) kernel
    DgradGather dg;    // used instead of A by the data-gradient kernel
    int kperiod;       // K-major B read at column k % kperiod (0: no wrap)
    float* Cf2;        // FP32 output columns n >= nsplit go to Cf2[m * ldc2 + n - nsplit]
    int ldc2, nsplit;
    int tout;          // FP32 output stored transposed: Cf[n * ldc + m] (no bias / ReLU)
    int rperm;         // h > 0: the rows of a tile come in runs of 2 h pixels, each run's even
                       // columns first, then its odd columns (row_pixel); 0: in pixel order
};

// pixel offset within its tile of tile row r (see GemmArgs::rperm)
__host__ __device__ __forceinline__ int row_pixel(int r, int h) {
    if (h == 0) return r;
    const int w2 = 2 * h, i = r / w2, j = r - i * w2;
    return i * w2 + (j < h ? 2 * j : 2 * (j - h) + 1);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
    const int n = pred ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)),
                 "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

}  // namespace sg
}  // namespace lbm

namespace lbm {
namespace sg {
// sum of the split-K partials in split order (deterministic): out[i] = sum_z part[z * stride + i]
__global__ void k_splitk_sum(const float* part, int splits, long long stride, long long n,
                             float* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * stride + i];
        out[i] = s;
    }
}

// the same sum for four consecutive outputs at a time (n and stride multiples of 4), the splits
// spread over the eight warps of a 256-thread block: warp w adds splits w, w + 8, ... in order
// for the 32 float4 outputs of the block, then the eight warp sums are added in warp order
// (deterministic: the grouping does not depend on the launch).
__global__ void k_splitk_sum4(const float* part, int splits, long long stride, long long n,
                              float* out) {
    __shared__ float4 sm[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long i = blockIdx.x * 32LL + lane, n4 = n / 4;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n4)
        for (int z = w; z < splits; z += 8) {
            const float4 v = reinterpret_cast<const float4*>(part + (size_t)z * stride)[i];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
    sm[w][lane] = s;
    __syncthreads();
    if (w == 0 && i < n4) {
        float4 t = sm[0][lane];
        for (int k = 1; k < 8; ++k) {
            t.x += sm[k][lane].x;
            t.y += sm[k][lane].y;
            t.z += sm[k][lane].z;
            t.w += sm[k][lane].w;
        }
        reinterpret_cast<float4*>(out)[i] = t;
    }
}

// Finish a split-K GEMM whose FP32 partials part[z][m][n] (row length N, splits stride M N)
// were written by the K-ranges z = 0 .. splits - 1: the sum in order z = 0, 1, ..., then the
// epilogue of the unsplit GEMM (bias, leaky ReLU, BF16 store to Cb, or FP32 store / accumulation
// to Cf, columns n >= nsplit to Cf2). Four consecutive columns per thread (N % 4 == 0).
__global__ void k_splitk_finish(const float* part, int splits, int M, int N, const float* bias,
                                int relu, __nv_bfloat16* Cb, float* Cf, int ldc, float* Cf2,
                                int ldc2, int nsplit, int accumulate) {
    const long long stride = (long long)M * N, n4 = stride / 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        const long long e = 4 * i;
        const int m = (int)(e / N), n = (int)(e - (long long)m * N);
        float4 x = reinterpret_cast<const float4*>(part + e)[0];
        for (int z = 1; z < splits; ++z) {
            const float4 y = reinterpret_cast<const float4*>(part + (size_t)z * stride + e)[0];
            x.x += y.x;
            x.y += y.y;
            x.z += y.z;
            x.w += y.w;
        }
        if (bias) {
            x.x += bias[n];
            x.y += bias[n + 1];
            x.z += bias[n + 2];
            x.w += bias[n + 3];
        }
        if (relu) {
            x.x = fmaxf(x.x, 0.1f * x.x);
            x.y = fmaxf(x.y, 0.1f * x.y);
            x.z = fmaxf(x.z, 0.1f * x.z);
            x.w = fmaxf(x.w, 0.1f * x.w);
        }
        if (Cb) {
            __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(Cb + (size_t)m * ldc + n);
            o[0] = __floats2bfloat162_rn(x.x, x.y);
            o[1] = __floats2bfloat162_rn(x.z, x.w);
            continue;
        }
        float* o = (Cf2 && n >= nsplit) ? Cf2 + (size_t)m * ldc2 + (n - nsplit)
                                        : Cf + (size_t)m * ldc + n;
        if (accumulate) {
            x.x += o[0];
            x.y += o[1];
            x.z += o[2];
            x.w += o[3];
        }
        o[0] = x.x;
        o[1] = x.y;
        o[2] = x.z;
        o[3] = x.w;
    }
}
}  // namespace sg
}  // namespace lbm
