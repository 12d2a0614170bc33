// BF16 tensor-core GEMM (mma.sync m16n8k16, FP32 accumulation) for the surrogate network:
// C[M x N] = A[M x K] * B[K x N] with either operand stored K-major or MN-major, so the forward
// pass (Xcol * W^T), the data gradient (dY * W) and the weight gradient (dY^T * Xcol) all run in
// one kernel without transposed copies. Tiles of 128 x 128 x 32 per CTA (8 warps of 64 x 32),
// two-stage cp.async pipeline, fragments via ldmatrix (.trans for MN-major operands).
// Requirements: K-major operands have K % 8 == 0 and 16-byte aligned rows; MN-major operands
// have M (resp. N) % 8 == 0; a split-K chunk is a multiple of GBK. Out-of-range rows and columns are zero-filled on load and masked on
// store. Epilogue: optional bias[n], leaky ReLU (slope 0.1), FP32 or BF16 output, optional
// accumulation into FP32.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace lbm {
namespace sg {

constexpr int GBM = 128, GBN = 128, GBK = 32, GTHREADS = 256;

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
};

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

__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                        const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                          const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// shared tiles with 8 elements of padding per row (ldmatrix rows land in distinct banks)
template <bool KMAJ, int ROWS>
struct TileShape {
    // K-major: ROWS x GBK stored [row][k]; MN-major: GBK x ROWS stored [k][row]
    static constexpr int R = KMAJ ? ROWS : GBK;
    static constexpr int C = KMAJ ? GBK + 8 : ROWS + 8;
    static constexpr int elems = R * C;
};

template <bool KMAJ, int ROWS>
__device__ __forceinline__ void load_tile(__nv_bfloat16* s, const __nv_bfloat16* g, int ld,
                                          int row0, int nrows, int k0, int K) {
    using S = TileShape<KMAJ, ROWS>;
    if (KMAJ) {
        // ROWS rows x (GBK / 8) chunks of 8 elements
        constexpr int CH = GBK / 8;
        for (int c = threadIdx.x; c < ROWS * CH; c += GTHREADS) {
            const int r = c / CH, kc = (c % CH) * 8;
            const bool ok = (row0 + r < nrows) && (k0 + kc < K);
            const __nv_bfloat16* src = ok ? g + (size_t)(row0 + r) * ld + k0 + kc : g;
            cp_async16(s + r * S::C + kc, src, ok);
        }
    } else {
        // GBK rows (k) x (ROWS / 8) chunks along the M/N direction
        constexpr int CH = ROWS / 8;
        for (int c = threadIdx.x; c < GBK * CH; c += GTHREADS) {
            const int kr = c / CH, rc = (c % CH) * 8;
            const bool ok = (k0 + kr < K) && (row0 + rc < nrows);
            const __nv_bfloat16* src = ok ? g + (size_t)(k0 + kr) * ld + row0 + rc : g;
            cp_async16(s + kr * S::C + rc, src, ok);
        }
    }
}

// A fragment (16 rows x 16 k) at (m, kk) of the stage tile
template <bool KMAJ>
__device__ __forceinline__ void frag_a(uint32_t* a, const __nv_bfloat16* s, int m, int kk,
                                       int lane) {
    using S = TileShape<KMAJ, GBM>;
    if (KMAJ) {
        const int r = m + (lane & 15), c = kk + (lane >> 4) * 8;
        ldsm_x4(a[0], a[1], a[2], a[3], s + r * S::C + c);
    } else {
        const int j = lane >> 3;
        const int k = kk + (lane & 7) + (j >> 1) * 8, mm = m + (j & 1) * 8;
        ldsm_x4_t(a[0], a[1], a[2], a[3], s + k * S::C + mm);
    }
}

// two B fragments (16 k x 8 n each) for columns n .. n+15 of the stage tile
template <bool KMAJ>
__device__ __forceinline__ void frag_b2(uint32_t* b, const __nv_bfloat16* s, int n, int kk,
                                        int lane) {
    using S = TileShape<KMAJ, GBN>;
    const int j = lane >> 3;
    if (KMAJ) {
        const int nn = n + (lane & 7) + (j >> 1) * 8, k = kk + (j & 1) * 8;
        ldsm_x4(b[0], b[1], b[2], b[3], s + nn * S::C + k);
    } else {
        const int k = kk + (lane & 7) + (j & 1) * 8, nn = n + (j >> 1) * 8;
        ldsm_x4_t(b[0], b[1], b[2], b[3], s + k * S::C + nn);
    }
}

template <bool AK, bool BK>
__global__ void __launch_bounds__(GTHREADS) k_gemm_bf16(const GemmArgs g) {
    using SA = TileShape<AK, GBM>;
    using SB = TileShape<BK, GBN>;
    __shared__ __align__(128) __nv_bfloat16 sA[2][SA::elems];
    __shared__ __align__(128) __nv_bfloat16 sB[2][SB::elems];
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;  // 2 x 4 warps of 64 x 32
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    // K range of this CTA (the whole K without split-K); loads stay masked by the full K
    const int kb = g.kchunk ? blockIdx.z * g.kchunk : 0;
    const int ke = g.kchunk ? min(g.K, kb + g.kchunk) : g.K;
    const int nk = ke > kb ? (ke - kb + GBK - 1) / GBK : 0;
    if (nk > 0) {
        load_tile<AK, GBM>(sA[0], g.A, g.lda, m0, g.M, kb, ke);
        load_tile<BK, GBN>(sB[0], g.B, g.ldb, n0, g.N, kb, ke);
    }
    cp_async_commit();
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) {
            load_tile<AK, GBM>(sA[st ^ 1], g.A, g.lda, m0, g.M, kb + (kt + 1) * GBK, ke);
            load_tile<BK, GBN>(sB[st ^ 1], g.B, g.ldb, n0, g.N, kb + (kt + 1) * GBK, ke);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t a[4][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) frag_a<AK>(a[i], sA[st], wm + i * 16, kk, lane);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint32_t t[4];
                frag_b2<BK>(t, sB[st], wn + j * 16, kk, lane);
                b[2 * j][0] = t[0];
                b[2 * j][1] = t[1];
                b[2 * j + 1][0] = t[2];
                b[2 * j + 1][1] = t[3];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    cp_async_wait<0>();
    // epilogue: accumulator (i, j, e) holds row wm + 16 i + lane/4 (+8 for e >= 2), column
    // wn + 8 j + 2 (lane % 4) + (e & 1)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + i * 16 + (lane >> 2) + (e >> 1) * 8;
                const int n = n0 + wn + j * 8 + (lane & 3) * 2 + (e & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = acc[i][j][e];
                if (g.bias) v += g.bias[n];
                if (g.relu) v = fmaxf(v, 0.1f * v);
                const size_t o = (size_t)m * g.ldc + n +
                                 (g.kchunk ? (size_t)blockIdx.z * g.split_stride : 0);
                if (g.Cf) {
                    if (g.accumulate)
                        g.Cf[o] += v;
                    else
                        g.Cf[o] = v;
                } else {
                    g.Cb[o] = __float2bfloat16_rn(v);
                }
            }
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
}  // namespace sg
}  // namespace lbm
