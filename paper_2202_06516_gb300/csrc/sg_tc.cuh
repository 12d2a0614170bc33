// BF16 GEMM on the 5th-generation tensor cores (tcgen05, accumulators in tensor memory) for the
// surrogate network: C[M x N] = sum_k A(m, k) B(n, k), each operand K-major (A[m][k], B[n][k])
// or MN-major (A[k][m], B[k][n]): the forward convolution Xcol W^T and, with a transposed
// weight copy, the data gradient dY W (both K-major), and the weight gradient dY^T Xcol (both
// MN-major, K = pixels).
//
// One CTA of 128 threads computes a 128 x BN tile. Its K-slices reach shared memory either as
// cp.async gathers by all threads (TMA = 0), in the 128-byte-swizzled K-major layout the tensor
// core reads (8-row atoms of 1 KB; the 16-byte chunk c of row r stored at chunk c ^ (r % 8)), or
// as tensor-map (TMA) boxes issued by thread 0 (TMA = 64 / 32: K-major slices of 64 or 32
// elements, 128- or 64-byte swizzle; TMA = 1: the weight gradient's MN-major blocks), STAGES
// slices in flight. Thread 0 issues the 128 x BN x 16 MMAs of each slice (kind::f16, BF16 in,
// FP32 accumulate into BN tensor-memory columns) and commits them to the slice's mbarrier,
// which frees the slice for the next load. The epilogue reads the accumulator lanes back with
// tcgen05.ld (warp w owns rows 32 w .. 32 w + 31), adds the bias, applies the leaky ReLU and
// stores FP32 or BF16. k_gemm_wwin computes the weight gradient of the 32/64-channel levels from
// one staged input window per slice, and k_gemm_fwin the forward convolution or data gradient of
// a layer whose window operand has 32 channels from one staged window per 128-pixel tile (the
// nine taps as operands shifted by whole rows inside the window).
//
// Every wait on an mbarrier is polled by one thread with an iteration limit; on expiry the
// CTA sets *err, waits (bounded) for the MMAs it issued, frees its tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "sg_gemm.cuh"

namespace lbm {
namespace sgtc {

constexpr int BM = 128, BK = 64, TC_THREADS = 128;
constexpr long long kWaitLimit = 1ll << 22;

__host__ __device__ constexpr int tmem_cols(int bn) {
    return bn <= 32 ? 32 : bn <= 64 ? 64 : bn <= 128 ? 128 : 256;
}

// elements of K per stage of a kernel variant: 64, or 32 for the 64-byte-swizzled K-major TMA
// variant (TMA = 32); the launch sizes shared memory with the same rule as the kernel
__host__ __device__ constexpr int slice_k(int tma) { return tma == 64 || tma == 32 ? tma : BK; }

// KS: elements of K per stage (slice_k of the variant)
template <int BN, int STAGES, bool BMN = false, int KS = BK>
struct TcShape {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "MMA N of kind::f16 at M = 128");
    static constexpr int A_BYTES = BM * KS * 2;  // 16 KB (8 KB when KS = 32)
    // MN-major slices are whole 64-element swizzle atoms wide along M or N
    static constexpr int B_BYTES = BMN ? (BN + 63) / 64 * 64 * KS * 2 : BN * KS * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    // 1 KB alignment slack for the swizzle atoms, then the stages, mbarriers and the TMEM slot
    static constexpr int RAW_BYTES = 1024 + STAGES * STAGE_BYTES + 8 * (2 * STAGES + 1) + 16;
    // at least enough shared memory that the CTAs resident on one SM never ask for more than
    // the 512 tensor-memory columns together (an allocation beyond them would wait)
    static constexpr int TMEM_CTAS = 512 / tmem_cols(BN);
    static constexpr int MIN_BYTES = 233472 / (TMEM_CTAS + 1) + 1;
    static constexpr int SMEM_BYTES = RAW_BYTES > MIN_BYTES ? RAW_BYTES : MIN_BYTES;
};

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1 KB apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// the same for 64-byte rows (32 elements of K), 64-byte swizzle, 8-row groups 512 B apart
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// shared-memory descriptor: MN-major operand, 64-byte swizzle; atoms of 32 (M or N) x 8 (K)
// elements, the 8-row K-groups of one 32-wide block 512 B apart (stride offset), blocks of 64 K
// rows 4 KB apart along M or N (leading offset)
__device__ __forceinline__ uint64_t desc_sw64_mn(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(4096 >> 4) << 16) |
           ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// shared-memory descriptor: MN-major operand, 128-byte swizzle; atoms of 64 (M or N) x 8 (K)
// elements, the 8 K-groups of one 64-wide block 1 KB apart (stride offset), blocks 8 KB apart
// along M or N (leading offset)
__device__ __forceinline__ uint64_t desc_sw128_mn(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(8192 >> 4) << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, each K-major (0) or
// MN-major (1: the operand's transpose bit), M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn = 0, int b_mn = 0) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

// poll one phase of an mbarrier; false when the iteration limit ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
        : "memory");
}

// the mbarrier expects `bytes` more transaction bytes (one arrival)
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// tiled tensor copies global -> shared, completion counted on an mbarrier; coordinates are
// innermost first, out-of-range elements are zero-filled
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// 32 consecutive FP32 accumulator columns of the warp's 32 lanes (one row per thread)
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// 16 consecutive FP32 accumulator columns of the warp's 32 lanes
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// one K-slice of ROWS x 64 elements of a K-major operand into the swizzled layout; rows past
// nrows and k past ke are zero-filled
template <int ROWS>
__device__ __forceinline__ void load_slice(uint8_t* s, const __nv_bfloat16* g, int ld, int row0,
                                           int nrows, int k0, int ke, int kperiod = 0) {
    constexpr int CHUNKS = ROWS * (BK / 8);
#pragma unroll 4
    for (int i = threadIdx.x; i < CHUNKS; i += TC_THREADS) {
        const int r = i >> 3, c = i & 7;
        const bool ok = (row0 + r < nrows) && (k0 + c * 8 < ke);
        const int kc = kperiod ? (k0 + c * 8) % kperiod : k0 + c * 8;
        const __nv_bfloat16* src = ok ? g + (size_t)(row0 + r) * ld + kc : g;
        uint8_t* dst = s + (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4);
        sg::cp_async16(dst, src, ok);
    }
}

// one K-slice of 64 (K) x ROWS (M or N) elements of an MN-major operand (row k of the stored
// matrix holds consecutive M or N indices) into the swizzled MN-major layout: element (mn, k) in
// block mn / 64, K-group k / 8 (1 KB apart), row k % 8, 16-byte chunk ((mn % 64) / 8) ^ (k % 8);
// positions past nrows or ke are zero-filled
template <int ROWS>
__device__ __forceinline__ void load_slice_mn(uint8_t* s, const __nv_bfloat16* g, int ld,
                                              int row0, int nrows, int k0, int ke) {
    constexpr int CPR = ROWS / 8;  // 16-byte chunks per stored row (ROWS % 8 == 0)
    constexpr int CHUNKS = BK * CPR;
#pragma unroll 4
    for (int i = threadIdx.x; i < CHUNKS; i += TC_THREADS) {
        const int k = i / CPR, c = i - k * CPR;
        const bool ok = (row0 + c * 8 < nrows) && (k0 + k < ke);
        const __nv_bfloat16* src = ok ? g + (size_t)(k0 + k) * ld + row0 + c * 8 : g;
        uint8_t* dst = s + (c >> 3) * (BK / 8 * 1024) + (k >> 3) * 1024 + (k & 7) * 128 +
                       (((c & 7) ^ (k & 7)) << 4);
        sg::cp_async16(dst, src, ok);
    }
}

// One K-slice of 128 rows (output pixels m0 ..) x 64 (K) of the gathered convolution operand
// (see sg::ConvGather), in the K-major swizzled layout of load_slice. Thread t always fills the
// 16-byte chunk column t % 8 of rows t / 8 + 16 j (j = 0..7), whose pixel coordinates it keeps
// in yx[j] (y | x << 16) and nn[j] (image index, -1 past M).
__device__ __forceinline__ void load_slice_conv(uint8_t* s, const sg::ConvGather& cv,
                                                const int* yx, const int* nn, int k0, int ke) {
    const int c = threadIdx.x & 7;
    const int k = k0 + c * 8;
    const bool kok = k < ke;
    const int tap = k >> cv.lc, ci = k & ((1 << cv.lc) - 1);
    const int dy = tap / 3 - 1, dx = tap - (tap / 3) * 3 - 1;
    const int h1 = cv.H >> cv.up1, w1 = cv.W >> cv.up1;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int r = (threadIdx.x >> 3) + 16 * j;
        const int y = (yx[j] & 0xFFFF) + dy, x = (yx[j] >> 16) + dx, n = nn[j];
        const bool ok = kok && n >= 0 && y >= 0 && y < cv.H && x >= 0 && x < cv.W;
        const __nv_bfloat16* src = cv.x1;
        if (ok) {
            if (ci < cv.C1)
                src = cv.x1 + ((((size_t)n * h1 + (y >> cv.up1)) * w1 + (x >> cv.up1)) * cv.C1 + ci);
            else
                src = cv.x2 + ((((size_t)n * cv.H + y) * cv.W + x) * cv.C2 + (ci - cv.C1));
        }
        uint8_t* dst = s + (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4);
        sg::cp_async16(dst, src, ok);
    }
}

// One K-slice of 128 source pixels x 64 (K) of the data-gradient operand (see
// sg::DgradGather) in the K-major swizzled layout; rows as in load_slice_conv (yx, nn).
__device__ __forceinline__ void load_slice_dgrad(uint8_t* s, const sg::DgradGather& dg,
                                                 const int* yx, const int* nn, int k0, int ke) {
    const int c = threadIdx.x & 7;
    const int k = k0 + c * 8;
    const bool kok = k < ke;
    const int co = k & ((1 << dg.lco) - 1), t = k >> dg.lco;  // t = s * 9 + tap
    const int sub = t / 9, tap = t - sub * 9;
    const int dy = tap / 3 - 1, dx = tap - (tap / 3) * 3 - 1;
    const int oy = (sub >> 1) - dy, ox = (sub & 1) - dx;  // sub = 0 unless up1
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int r = (threadIdx.x >> 3) + 16 * j;
        const int y = ((yx[j] & 0xFFFF) << dg.up1) + oy, x = ((yx[j] >> 16) << dg.up1) + ox;
        const int n = nn[j];
        const bool ok = kok && n >= 0 && y >= 0 && y < dg.H && x >= 0 && x < dg.W;
        const __nv_bfloat16* src =
            ok ? dg.dy + ((((size_t)n * dg.H + y) * dg.W + x) << dg.lco) + co : dg.dy;
        uint8_t* dst = s + (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4);
        sg::cp_async16(dst, src, ok);
    }
}

// One K-slice of 64 pixels (K) x 128 im2col columns (M: (tap, channel) of the gathered
// convolution operand) in the MN-major swizzled layout, as the A operand of the transposed
// weight gradient. Thread t always fills the 16-byte column chunk t % 16 (columns
// m0 + 8 (t % 16) ..), whose tap and channel it decodes once (tc, cc: ci | tap << 16, -1 past
// M); its pixels are k0 + t / 16 + 8 j (j = 0..7). H and W are powers of two.
__device__ __forceinline__ void load_slice_mn_conv_a(uint8_t* s, const sg::ConvGather& cv,
                                                     int tc, int k0, int ke) {
    const int c = threadIdx.x & 15;
    const int ci = tc & 0xFFFF, tap = tc >> 16;
    const int dy = tap / 3 - 1, dx = tap - (tap / 3) * 3 - 1;
    const int h1 = cv.H >> cv.up1, w1 = cv.W >> cv.up1;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = (threadIdx.x >> 4) + 8 * j;
        const int p = k0 + k;
        const int y = ((p >> cv.lw) & (cv.H - 1)) + dy, x = (p & (cv.W - 1)) + dx;
        const int n = p >> (cv.lw + cv.lh);
        const bool ok = tc >= 0 && p < ke && y >= 0 && y < cv.H && x >= 0 && x < cv.W;
        const __nv_bfloat16* src = cv.x1;
        if (ok) {
            if (ci < cv.C1)
                src = cv.x1 + ((((size_t)n * h1 + (y >> cv.up1)) * w1 + (x >> cv.up1)) * cv.C1 + ci);
            else
                src = cv.x2 + ((((size_t)n * cv.H + y) * cv.W + x) * cv.C2 + (ci - cv.C1));
        }
        uint8_t* dst = s + (c >> 3) * (BK / 8 * 1024) + (k >> 3) * 1024 + (k & 7) * 128 +
                       (((c & 7) ^ (k & 7)) << 4);
        sg::cp_async16(dst, src, ok);
    }
}

// Epilogue of one 128 x BN output tile whose FP32 accumulator sits in tensor-memory columns
// tacc .. tacc + BN - 1 (zero: no K slices, the result is 0). Warp `warp` (0 .. 3) reads
// accumulator lanes 32 warp .. 32 warp + 31 (rows m0 + 32 warp ..) and passes them through its
// own 32 x 32 staging block ep (rows 144 B apart), so that stores write whole row segments:
// 16-byte vectors when the output allows (no accumulation or split, aligned rows), else one
// column per lane; bias, leaky ReLU, BF16 or FP32 (accumulated, split at nsplit, or transposed)
// as the arguments say. zoff: the split-K partial's offset.
template <int BN>
__device__ __forceinline__ void epilogue_tile(const sg::GemmArgs& g, uint32_t tacc, float* ep,
                                              int warp, int lane, int m0, int n0, bool zero,
                                              size_t zoff) {
    // FP32 outputs may accumulate and may be split at column nsplit into two tensors; the
    // vector path then takes a 32-column chunk that lies on one side of the split
    const bool vec = !g.kchunk &&
                     (g.Cb ? (!g.accumulate && g.ldc % 8 == 0 && ((uintptr_t)g.Cb & 15) == 0)
                           : (g.ldc % 4 == 0 && ((uintptr_t)g.Cf & 15) == 0 &&
                              (!g.Cf2 || (g.ldc2 % 4 == 0 && g.nsplit % 4 == 0 &&
                                          ((uintptr_t)g.Cf2 & 15) == 0))));
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        if (n0 + c0 >= g.N) break;
        const int w = BN - c0 >= 32 ? 32 : 16;
        float v[32];
        const uint32_t ta = tacc + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        if (zero) {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = 0.f;
        } else if (w == 32) {
            tc_ld32(ta, v);
        } else {
            tc_ld16(ta, v);
        }
        if (g.tout) {
            // transposed FP32 store: for each column, the warp's 32 rows are consecutive
            const int m = m0 + warp * 32 + lane;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int n = n0 + c0 + j;
                if (j >= w || n >= g.N || m >= g.M) continue;
                float* o = g.Cf + (size_t)n * g.ldc + m + zoff;
                *o = g.accumulate ? *o + v[j] : v[j];
            }
            continue;
        }
#pragma unroll
        for (int j = 0; j < 32; j += 4)
            if (j < w)
                *reinterpret_cast<float4*>(ep + lane * 36 + j) =
                    make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        __syncwarp();
        const bool one_side = !g.Cf2 || n0 + c0 + 32 <= g.nsplit || n0 + c0 >= g.nsplit;
        if (vec && w == 32 && n0 + c0 + 32 <= g.N && one_side) {
            if (g.Cb) {
                // lane: row it * 8 + lane / 4, columns 8 (lane % 4) .. + 7
                const int cc = 8 * (lane & 3), n = n0 + c0 + cc;
                float bn[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) bn[j] = g.bias ? g.bias[n + j] : 0.f;
#pragma unroll
                for (int it = 0; it < 4; ++it) {
                    const int r = it * 8 + (lane >> 2);
                    const int m = m0 + sg::row_pixel(warp * 32 + r, g.rperm);
                    if (m >= g.M) continue;
                    const float4 x0 = *reinterpret_cast<const float4*>(ep + r * 36 + cc);
                    const float4 x1 = *reinterpret_cast<const float4*>(ep + r * 36 + cc + 4);
                    float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                    uint4 o;
                    __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
                    for (int j = 0; j < 8; j += 2) {
                        float a0 = x[j] + bn[j], a1 = x[j + 1] + bn[j + 1];
                        if (g.relu) {
                            a0 = fmaxf(a0, 0.1f * a0);
                            a1 = fmaxf(a1, 0.1f * a1);
                        }
                        oh[j / 2] = __floats2bfloat162_rn(a0, a1);
                    }
                    *reinterpret_cast<uint4*>(g.Cb + (size_t)m * g.ldc + n) = o;
                }
            } else {
                // lane: row it * 4 + lane / 8, columns 4 (lane % 8) .. + 3
                const int cc = 4 * (lane & 7), n = n0 + c0 + cc;
                float bn[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) bn[j] = g.bias ? g.bias[n + j] : 0.f;
                // destination of row it * 4 + lane / 8; with accumulation all eight old
                // values are loaded before the first store, so their latencies overlap
                auto dst_of = [&](int it) {
                    const int m = m0 + sg::row_pixel(warp * 32 + it * 4 + (lane >> 3), g.rperm);
                    return (g.Cf2 && n >= g.nsplit)
                               ? reinterpret_cast<float4*>(g.Cf2 + (size_t)m * g.ldc2 +
                                                           (n - g.nsplit))
                               : reinterpret_cast<float4*>(g.Cf + (size_t)m * g.ldc + n);
                };
                float4 old[8];
                if (g.accumulate) {
#pragma unroll
                    for (int it = 0; it < 8; ++it) {
                        const int m = m0 + sg::row_pixel(warp * 32 + it * 4 + (lane >> 3), g.rperm);
                        old[it] = m < g.M ? *dst_of(it) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int r = it * 4 + (lane >> 3);
                    const int m = m0 + sg::row_pixel(warp * 32 + r, g.rperm);
                    if (m >= g.M) continue;
                    float4 x = *reinterpret_cast<const float4*>(ep + r * 36 + cc);
                    x.x += bn[0];
                    x.y += bn[1];
                    x.z += bn[2];
                    x.w += bn[3];
                    if (g.relu) {
                        x.x = fmaxf(x.x, 0.1f * x.x);
                        x.y = fmaxf(x.y, 0.1f * x.y);
                        x.z = fmaxf(x.z, 0.1f * x.z);
                        x.w = fmaxf(x.w, 0.1f * x.w);
                    }
                    if (g.accumulate) {
                        x.x += old[it].x;
                        x.y += old[it].y;
                        x.z += old[it].z;
                        x.w += old[it].w;
                    }
                    *dst_of(it) = x;
                }
            }
        } else {
            const int n = n0 + c0 + lane;
            const bool col_ok = lane < w && n < g.N;
            const float bn = (col_ok && g.bias) ? g.bias[n] : 0.f;
#pragma unroll 4
            for (int r = 0; r < 32; ++r) {
                const int m = m0 + sg::row_pixel(warp * 32 + r, g.rperm);
                if (!col_ok || m >= g.M) continue;
                float x = ep[r * 36 + lane] + bn;
                if (g.relu) x = fmaxf(x, 0.1f * x);
                float* cf = g.Cf;
                size_t o = (size_t)m * g.ldc + n + zoff;
                if (g.Cf2 && n >= g.nsplit) {
                    cf = g.Cf2;
                    o = (size_t)m * g.ldc2 + (n - g.nsplit);
                }
                if (cf) {
                    if (g.accumulate)
                        cf[o] += x;
                    else
                        cf[o] = x;
                } else {
                    g.Cb[o] = __float2bfloat16_rn(x);
                }
            }
        }
        __syncwarp();
    }
}

// GA: A is the gathered convolution operand (K-major, rows = output pixels); GD: A is the
// gathered data-gradient operand; GAM: A is the gathered convolution operand MN-major (K =
// pixels, M = im2col columns).
// TMA (64 or 32; with GA or GD, both operands K-major): thread 0 alone feeds the stages with
// tiled tensor copies of TMA elements of K per stage (128- or 64-byte swizzled rows): A as one
// box of TMA channels x the tile's 128 pixels (a block of whole rows, or 128 pixels of one row)
// of the activation (GA; the tap's offset applied to the box origin, x1 or x2 by channel) or of
// the output gradient (GD, the offset negated), out-of-image pixels zero-filled by the copy
// itself; B as a TMA x BN box of the weight matrix. Stage s completes on full[s] (transaction
// bytes), is released by the MMAs' commit to empty[s], and STAGES slices are in flight.
// TMA = 1 (with GAM, both operands MN-major): the same feeding for the weight gradient, 64
// pixels of K per stage in 64-byte-swizzled MN-major blocks of 32: A as four boxes of 32
// channels x the 64 pixels (a block of whole rows or 64 pixels of one row), each at its tap's
// offset; B as BN / 32 boxes of 32 output-gradient channels x the same pixels.
template <int BN, int STAGES, bool AMN = false, bool BMN = false, bool GA = false, bool GD = false,
          bool GAM = false, int TMA = 0>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const sg::GemmArgs g, int* err, const __grid_constant__ CUtensorMap tmA1,
              const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB) {
    static_assert(!TMA || ((GA || GD) && !AMN && !BMN && (TMA == 64 || TMA == 32)) ||
                      (GAM && AMN && BMN && TMA == 1 && BN % 32 == 0),
                  "TMA feeds the K-major gathers (64 or 32) or the weight gradient (1)");
    constexpr int KS = slice_k(TMA);
    using S = TcShape<BN, STAGES, BMN, KS>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    // 1 KB-aligned base of the stages (the swizzle pattern follows shared-memory address bits)
    const uint32_t raw = su32(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * S::STAGE_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = g.kchunk ? blockIdx.z * g.kchunk : 0;
    const int ke = g.kchunk ? min(g.K, kb + g.kchunk) : g.K;
    const int nk = ke > kb ? (ke - kb + KS - 1) / KS : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         su32(tmem_slot)),
                     "r"(tmem_cols(BN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s <= 2 * STAGES; ++s) mbar_init(su32(bars + s), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_ok = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t IDESC = idesc_bf16(BM, BN, AMN ? 1 : 0, BMN ? 1 : 0);

    auto stage_a = [&](int s) { return base + s * S::STAGE_BYTES; };
    auto stage_b = [&](int s) { return base + s * S::STAGE_BYTES + S::A_BYTES; };
    // GA / GD: pixel coordinates of the thread's eight A rows, fixed for all K-slices (rows are
    // output pixels, or source pixels at the source's resolution)
    int yx[8], nn[8];
    if (GA || GD) {
        const int RH = GA ? g.conv.H : g.dg.H >> g.dg.up1, RWd = GA ? g.conv.W : g.dg.W >> g.dg.up1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int p = m0 + (tid >> 3) + 16 * j;
            const int x = p % RWd, q = p / RWd, y = q % RH;
            yx[j] = y | (x << 16);
            nn[j] = p < g.M ? q / RH : -1;
        }
    }
    // GAM: tap and channel of the thread's A column chunk
    int tcol = -1;
    if (GAM) {
        const int col = m0 + 8 * (tid & 15);
        if (col < g.M) {
            const int tap = col >> g.conv.lc;
            tcol = (col & ((1 << g.conv.lc) - 1)) | (tap << 16);
        }
    }
    auto load = [&](int s, int k0) {
        if (GAM)
            load_slice_mn_conv_a(stage_a(s), g.conv, tcol, k0, ke);
        else if (GA)
            load_slice_conv(stage_a(s), g.conv, yx, nn, k0, ke);
        else if (GD)
            load_slice_dgrad(stage_a(s), g.dg, yx, nn, k0, ke);
        else if (AMN)
            load_slice_mn<BM>(stage_a(s), g.A, g.lda, m0, g.M, k0, ke);
        else
            load_slice<BM>(stage_a(s), g.A, g.lda, m0, g.M, k0, ke);
        if (BMN)
            load_slice_mn<BN>(stage_b(s), g.B, g.ldb, n0, g.N, k0, ke);
        else
            load_slice<BN>(stage_b(s), g.B, g.ldb, n0, g.N, k0, ke, g.kperiod);
    };

    bool ok = true;
    if constexpr (TMA) {
        // tile origin: n, y0, x0 of the first of the 128 pixels (a tbh x tbw block); the data
        // gradient of an upsampling convolution has its rows at the source's half resolution
        const int TH = GA || GAM ? g.conv.H : g.dg.H >> g.dg.up1;
        const int TW = GA || GAM ? g.conv.W : g.dg.W >> g.dg.up1;
        const int img = m0 / (TH * TW), rem = m0 - img * (TH * TW);
        const int y0 = rem / TW, x0 = rem - (rem / TW) * TW;
        const int lk = GA || GAM ? g.conv.lc : g.dg.lco;
        auto issue = [&](int st, int k0) {
            const uint32_t full = su32(bars + st);
            if constexpr (GAM) {
                // K = pixels k0 .. k0 + 63: image, row and column of the first
                mbar_expect_tx(full, (uint32_t)(BM * 64 * 2 + BN * 64 * 2));
                const int pn = k0 / (TH * TW), pr = k0 - pn * (TH * TW);
                const int py = pr / TW, px = pr - (pr / TW) * TW;
                if (g.conv.up1) {
                    // upsampling convolution: the slice's 64 pixels (one row segment) in the
                    // order even columns, odd columns (K is summed over, the same order for A
                    // and B); each half reads a run of 32 consecutive source pixels and every
                    // second output-gradient pixel
#pragma unroll
                    for (int b = 0; b < BM / 32; ++b) {
                        const int col = m0 + 32 * b, tap = col >> lk, ci = col & ((1 << lk) - 1);
                        const int dy = tap / 3 - 1, dx = tap - (tap / 3) * 3 - 1;
                        const int sy = (py + dy) >= 0 ? (py + dy) >> 1 : -1;
                        const uint32_t dst = su32(stage_a(st)) + 4096 * b;
                        tma_load_4d(dst, &tmA1, full, ci, (px >> 1) + (dx < 0 ? -1 : 0), sy, pn);
                        tma_load_4d(dst + 2048, &tmA1, full, ci, (px >> 1) + (dx > 0 ? 1 : 0), sy,
                                    pn);
                    }
#pragma unroll
                    for (int b = 0; b < BN / 32; ++b) {
                        const uint32_t dst = su32(stage_b(st)) + 4096 * b;
                        tma_load_4d(dst, &tmB, full, n0 + 32 * b, px, py, pn);
                        tma_load_4d(dst + 2048, &tmB, full, n0 + 32 * b, px + 1, py, pn);
                    }
                    return;
                }
#pragma unroll
                for (int b = 0; b < BM / 32; ++b) {
                    const int col = m0 + 32 * b, tap = col >> lk, ci = col & ((1 << lk) - 1);
                    const int dy = tap / 3 - 1, dx = tap - (tap / 3) * 3 - 1;
                    if (ci < g.conv.C1)
                        tma_load_4d(su32(stage_a(st)) + 4096 * b, &tmA1, full, ci, px + dx,
                                    py + dy, pn);
                    else
                        tma_load_4d(su32(stage_a(st)) + 4096 * b, &tmA2, full, ci - g.conv.C1,
                                    px + dx, py + dy, pn);
                }
#pragma unroll
                for (int b = 0; b < BN / 32; ++b)
                    tma_load_4d(su32(stage_b(st)) + 4096 * b, &tmB, full, n0 + 32 * b, px, py, pn);
                return;
            }
            mbar_expect_tx(full, (uint32_t)(S::A_BYTES + S::B_BYTES));
            const int tap = k0 >> lk, ch = k0 & ((1 << lk) - 1);
            const int dy = tap / 3 - 1, dx = tap - (tap / 3) * 3 - 1;
            if (GA && g.conv.up1) {
                // upsampling layer: the tile's rows come as runs of even, then odd output
                // columns (rperm = half a tile row); each run reads consecutive source pixels of
                // the half-resolution source row floor((y + dy) / 2)
                const int h = g.rperm, tbh = BM / (2 * h);
                for (int i = 0; i < tbh; ++i) {
                    const int yo = y0 + i + dy, sy = yo >= 0 ? yo >> 1 : -1;
                    const uint32_t row = su32(stage_a(st)) + (uint32_t)(i * 2 * h * KS * 2);
                    tma_load_4d(row, &tmA1, full, ch, (x0 >> 1) + (dx < 0 ? -1 : 0), sy, img);
                    tma_load_4d(row + (uint32_t)(h * KS * 2), &tmA1, full, ch,
                                (x0 >> 1) + (dx > 0 ? 1 : 0), sy, img);
                }
            } else if (GA) {
                if (ch < g.conv.C1)
                    tma_load_4d(su32(stage_a(st)), &tmA1, full, ch, x0 + dx, y0 + dy, img);
                else
                    tma_load_4d(su32(stage_a(st)), &tmA2, full, ch - g.conv.C1, x0 + dx, y0 + dy,
                                img);
            } else if (g.dg.up1) {
                // K = (sub-pixel s, tap, channel): the output gradient at (2 y + sy - dy,
                // 2 x + sx - dx), every second pixel in both directions (a strided box)
                const int sub = tap / 9, t9 = tap - sub * 9;
                const int uy = t9 / 3 - 1, ux = t9 - (t9 / 3) * 3 - 1;
                tma_load_4d(su32(stage_a(st)), &tmA1, full, ch, 2 * x0 + (sub & 1) - ux,
                            2 * y0 + (sub >> 1) - uy, img);
            } else {
                tma_load_4d(su32(stage_a(st)), &tmA1, full, ch, x0 - dx, y0 - dy, img);
            }
            tma_load_2d(su32(stage_b(st)), &tmB, full, g.kperiod ? k0 % g.kperiod : k0, n0);
        };
        if (tid == 0) {
            int issued = 0, done_mma = 0;
            bool good = true;
            for (; issued < STAGES && issued < nk; ++issued) issue(issued, kb + issued * KS);
            for (int kt = 0; kt < nk; ++kt) {
                const int st = kt % STAGES;
                if (!mbar_wait(su32(bars + st), (kt / STAGES) & 1)) {
                    good = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = su32(stage_a(st)), b0 = su32(stage_b(st));
#pragma unroll
                for (int j = 0; j < KS / 16; ++j) {
                    // K = 16 per MMA: 32 bytes along a K-major row, or two 512-byte K-groups of
                    // an MN-major 64-byte-swizzled block
                    const uint64_t ad = GAM         ? desc_sw64_mn(a0 + 1024 * j)
                                        : KS == 64 ? desc_sw128(a0 + 32 * j)
                                                   : desc_sw64(a0 + 32 * j);
                    const uint64_t bd = GAM         ? desc_sw64_mn(b0 + 1024 * j)
                                        : KS == 64 ? desc_sw128(b0 + 32 * j)
                                                   : desc_sw64(b0 + 32 * j);
                    tc_mma(tmem, ad, bd, IDESC, (kt > 0 || j > 0) ? 1u : 0u);
                }
                tc_commit(su32(bars + STAGES + st));
                done_mma = kt + 1;
                // refill the stage that slice kt - 1 used once its MMAs have read it
                if (kt >= 1 && issued < nk) {
                    const int sp = (kt - 1) % STAGES;
                    if (!mbar_wait(su32(bars + STAGES + sp), ((kt - 1) / STAGES) & 1)) {
                        good = false;
                        break;
                    }
                    issue(sp, kb + issued * KS);
                    ++issued;
                }
            }
            if (!good) {
                // let the copies still in flight land before the CTA may leave (bounded)
                for (int j = done_mma; j < issued; ++j)
                    mbar_wait(su32(bars + j % STAGES), (j / STAGES) & 1);
            }
            if (nk > 0) {
                tc_commit(su32(bars + 2 * STAGES));
                if (!mbar_wait(su32(bars + 2 * STAGES), 0)) good = false;
            }
            if (!good) s_ok = 0;
        }
        __syncthreads();
        ok = s_ok;
    } else {
#pragma unroll 1
    for (int p = 0; p < STAGES - 1; ++p) {
        if (p < nk) load(p, kb + p * BK);
        sg::cp_async_commit();
    }
#pragma unroll 1
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % STAGES;
        sg::cp_async_wait<STAGES - 2>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = su32(stage_a(s)), b0 = su32(stage_b(s));
#pragma unroll
            for (int j = 0; j < BK / 16; ++j) {
                // K = 16 per MMA: 32 bytes along a K-major swizzle row, two 1 KB K-groups of an
                // MN-major block
                const uint64_t ad = AMN ? desc_sw128_mn(a0 + 2048 * j) : desc_sw128(a0 + 32 * j);
                const uint64_t bd = BMN ? desc_sw128_mn(b0 + 2048 * j) : desc_sw128(b0 + 32 * j);
                tc_mma(tmem, ad, bd, IDESC, (kt > 0 || j > 0) ? 1u : 0u);
            }
            tc_commit(su32(bars + s));
        }
        const int nxt = kt + STAGES - 1;
        if (nxt < nk && kt >= 1) {
            // the slice being refilled was read by the MMAs of k-tile kt - 1
            if (tid == 0 && !mbar_wait(su32(bars + (kt - 1) % STAGES), ((kt - 1) / STAGES) & 1))
                s_ok = 0;
            __syncthreads();
            if (!s_ok) {
                ok = false;
                break;
            }
        }
        if (nxt < nk) load(nxt % STAGES, kb + nxt * BK);
        sg::cp_async_commit();
    }
    sg::cp_async_wait<0>();
    // completion of every MMA issued (the last commit tracks all earlier ones)
    if (nk > 0) {
        if (tid == 0) {
            tc_commit(su32(bars + 2 * STAGES));
            if (!mbar_wait(su32(bars + 2 * STAGES), 0)) s_ok = 0;
        }
        __syncthreads();
        ok = ok && s_ok;
    }
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        tc_fence_after();
        // the staging blocks lie in the now idle stage buffers
        epilogue_tile<BN>(g, tmem, reinterpret_cast<float*>(base) + warp * (32 * 36), warp, lane,
                          m0, n0, nk == 0, g.kchunk ? (size_t)blockIdx.z * g.split_stride : 0);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(tmem_cols(BN))
                     : "memory");
    }
}

// shared-memory descriptor of an MN-major, 64-byte-swizzled operand whose 32-wide blocks are
// lbo bytes apart (K-groups of 8 rows 512 B apart); the start may lie on any 64-byte row, the
// swizzle follows the absolute shared-memory address
__device__ __forceinline__ uint64_t desc_sw64_mn_lbo(uint32_t saddr, uint32_t lbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

__host__ __device__ constexpr uint32_t tmem_pow2(int cols) {
    return cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
}

// Weight gradient of a 3 x 3 convolution with C_in = 32 CB input channels from one staged input
// window per K slice: dW^T[(tap, ci)][co] = sum over pixels p of x(p + off(tap))[ci] dY(p)[co]
// (K = pixels of one image row segment, 64 per slice; each CTA one split-K range, grid = splits).
// Per slice thread 0 loads with TMA, for each 32-channel block, the input rows y - 1 .. y + 1 of
// pixels x - 4 .. x + 67 (64-byte-swizzled rows of 32 channels: the MN-major layout with K =
// pixels), and the 32-channel blocks of dY for the 64 pixels. The nine taps are then MN-major A
// operands that start a whole number of rows into that window (dx) with the three dy rows as their
// first three 32-wide M blocks (4,608 B apart; the fourth block reads a row that is not loaded and
// its outputs are dropped): accumulator tile (block cb, dx) in tensor-memory columns
// (3 cb + dx + 1) BN. Every input element is read once per slice instead of once per tap. The
// epilogue writes the split's FP32 partial transposed, dW^T row tap C_in + ci.
template <int BN, int CB, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_wwin(const sg::GemmArgs g, int* err, const __grid_constant__ CUtensorMap tmX1,
                const __grid_constant__ CUtensorMap tmX2, const __grid_constant__ CUtensorMap tmDY) {
    static_assert(BN % 32 == 0 && 3 * CB * BN <= 512, "accumulators must fit tensor memory");
    constexpr int T = 3 * CB, WROW = 72, WIN = 4 * WROW * 64;
    constexpr int A_B = CB * WIN, B_B = BN * 128, STAGE = A_B + B_B;
    constexpr uint32_t TX = (uint32_t)(CB * 3 * WROW * 64 + B_B);
    constexpr uint32_t COLS = tmem_pow2(T * BN);
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kb = blockIdx.x * g.kchunk, ke = min(g.K, kb + g.kchunk);
    const int nk = ke > kb ? (ke - kb) / 64 : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         su32(tmem_slot)),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i <= 2 * STAGES; ++i) mbar_init(su32(bars + i), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_ok = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t IDESC = idesc_bf16(BM, BN, 1, 1);
    const int H = g.conv.H, W = g.conv.W;
    auto win = [&](int st, int cb) { return su32(base + st * STAGE + cb * WIN); };
    auto dyb = [&](int st) { return su32(base + st * STAGE + A_B); };
    auto issue = [&](int st, int k0) {
        const uint32_t full = su32(bars + st);
        mbar_expect_tx(full, TX);
        const int pn = k0 / (H * W), pr = k0 - pn * (H * W);
        const int py = pr / W, px = pr - (pr / W) * W;
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            const int ci = 32 * cb;
            if (ci < g.conv.C1)
                tma_load_4d(win(st, cb), &tmX1, full, ci, px - 4, py - 1, pn);
            else
                tma_load_4d(win(st, cb), &tmX2, full, ci - g.conv.C1, px - 4, py - 1, pn);
        }
#pragma unroll
        for (int b = 0; b < BN / 32; ++b) tma_load_4d(dyb(st) + 4096 * b, &tmDY, full, 32 * b, px, py, pn);
    };
    if (tid == 0) {
        int issued = 0, done_mma = 0;
        bool good = true;
        for (; issued < STAGES && issued < nk; ++issued) issue(issued, kb + issued * 64);
        for (int kt = 0; kt < nk; ++kt) {
            const int st = kt % STAGES;
            if (!mbar_wait(su32(bars + st), (kt / STAGES) & 1)) {
                good = false;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const int cb = t / 3, dxi = t - 3 * (t / 3);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint64_t ad =
                        desc_sw64_mn_lbo(win(st, cb) + (uint32_t)((3 + dxi) * 64 + 1024 * j), WROW * 64);
                    const uint64_t bd = desc_sw64_mn(dyb(st) + 1024 * j);
                    tc_mma(tmem + (uint32_t)(t * BN), ad, bd, IDESC, (kt > 0 || j > 0) ? 1u : 0u);
                }
            }
            tc_commit(su32(bars + STAGES + st));
            done_mma = kt + 1;
            if (kt >= 1 && issued < nk) {
                const int sp = (kt - 1) % STAGES;
                if (!mbar_wait(su32(bars + STAGES + sp), ((kt - 1) / STAGES) & 1)) {
                    good = false;
                    break;
                }
                issue(sp, kb + issued * 64);
                ++issued;
            }
        }
        if (!good)
            for (int j = done_mma; j < issued; ++j) mbar_wait(su32(bars + j % STAGES), (j / STAGES) & 1);
        if (nk > 0) {
            tc_commit(su32(bars + 2 * STAGES));
            if (!mbar_wait(su32(bars + 2 * STAGES), 0)) good = false;
        }
        if (!good) s_ok = 0;
    }
    __syncthreads();
    if (!s_ok) {
        if (tid == 0) atomicExch(err, 1);
    } else if (warp < 3) {
        // warp w holds M block w: dy = w - 1, lane = channel within the block
        tc_fence_after();
        const size_t zoff = (size_t)blockIdx.x * g.split_stride;
        const int cin = 32 * CB;
#pragma unroll 1
        for (int t = 0; t < T; ++t) {
            const int cb = t / 3, dxi = t - 3 * (t / 3);
            const int m = (warp * 3 + dxi) * cin + 32 * cb + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                float v[32];
                if (nk == 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0.f;
                } else {
                    tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * BN + c0), v);
                }
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < g.N) g.Cf[(size_t)(c0 + j) * g.ldc + m + zoff] = v[j];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(COLS)
                     : "memory");
    }
}

// Forward convolution (GA) or data gradient (GD) of a 3 x 3 convolution for a tile of 128
// output pixels of one image row, from one staged window: with C = 32 CB channels of the operand
// (the input for GA, concatenated sources by channel; the output gradient for GD), thread 0
// loads with TMA, per 32-channel block, the rows y - 1 .. y + 1 of pixels x - 4 .. x + 131
// (K-major rows of 32 channels, 64-byte swizzle) and the tile's 32 x BN weight blocks of all
// nine taps (output columns BN blockIdx.x ..), all on one mbarrier. Each tap (dy, dx) is then a K-major A operand that starts whole rows into
// the window (GA: row dy + 1, column 4 + dx; GD: the offsets negated), two 16-deep MMAs per
// (tap, block) into one accumulator. Every operand element is read once per tile instead of once
// per tap. The epilogue is the GEMM's own (bias and leaky ReLU with BF16 output, or the
// accumulating, possibly split FP32 output of the data gradient).
template <int BN, int CB, bool GD>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_fwin(const sg::GemmArgs g, int* err, const __grid_constant__ CUtensorMap tmA1,
                const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB) {
    static_assert((BN == 32 || BN == 64) && (CB == 1 || CB == 2), "32 or 64 columns and channels");
    constexpr int WROW = 136, WINB = 3 * WROW * 64;  // one 32-channel block of the window
    constexpr int A_B = CB * WINB, BSUB = BN * 64, B_B = 9 * CB * BSUB;
    constexpr uint32_t TX = (uint32_t)(A_B + B_B);
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    // 512-byte-aligned base: the 64-byte swizzle repeats every 512 bytes of shared memory
    uint8_t* base = smem_raw + ((512u - (raw & 511u)) & 511u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + A_B + B_B);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         su32(tmem_slot)),
                     "r"(tmem_cols(BN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(su32(bars), 1);
        mbar_init(su32(bars + 1), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_ok = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t IDESC = idesc_bf16(BM, BN, 0, 0);
    const int H = GD ? g.dg.H : g.conv.H, W = GD ? g.dg.W : g.conv.W;
    const int img = m0 / (H * W), rem = m0 - img * (H * W);
    const int y0 = rem / W, x0 = rem - (rem / W) * W;
    const uint32_t A = su32(base), B = su32(base + A_B);
    if (tid == 0) {
        bool good = true;
        const uint32_t full = su32(bars);
        mbar_expect_tx(full, TX);
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
            const int ci = 32 * cb;
            if (GD || ci < g.conv.C1)
                tma_load_4d(A + cb * WINB, &tmA1, full, ci, x0 - 4, y0 - 1, img);
            else
                tma_load_4d(A + cb * WINB, &tmA2, full, ci - g.conv.C1, x0 - 4, y0 - 1, img);
        }
        for (int t = 0; t < 9; ++t)
#pragma unroll
            for (int cb = 0; cb < CB; ++cb)
                tma_load_2d(B + (t * CB + cb) * BSUB, &tmB, full, (t * CB + cb) * 32, n0);
        if (!mbar_wait(full, 0)) {
            good = false;
            mbar_wait(full, 0);  // let the copies in flight land before the CTA may leave (bounded)
        }
        if (good) {
            tc_fence_after();
            for (int t = 0; t < 9; ++t) {
                const int dy = t / 3 - 1, dx = t - (t / 3) * 3 - 1;
                const int wr = GD ? 1 - dy : 1 + dy, wc = GD ? 4 - dx : 4 + dx;
#pragma unroll
                for (int cb = 0; cb < CB; ++cb)
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const uint32_t a = A + cb * WINB + (uint32_t)((wr * WROW + wc) * 64 + 32 * j);
                        const uint32_t b = B + (t * CB + cb) * BSUB + 32 * j;
                        tc_mma(tmem, desc_sw64(a), desc_sw64(b), IDESC,
                               (t > 0 || cb > 0 || j > 0) ? 1u : 0u);
                    }
            }
            tc_commit(su32(bars + 1));
            if (!mbar_wait(su32(bars + 1), 0)) good = false;
        }
        if (!good) s_ok = 0;
    }
    __syncthreads();
    if (!s_ok) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        tc_fence_after();
        // the staging blocks lie in the window, no longer read
        epilogue_tile<BN>(g, tmem, reinterpret_cast<float*>(base) + warp * (32 * 36), warp, lane,
                          m0, n0, false, 0);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(tmem_cols(BN))
                     : "memory");
    }
}

}  // namespace sgtc
}  // namespace lbm
