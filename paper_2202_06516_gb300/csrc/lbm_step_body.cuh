// Device code of the fused multiphase LBM time step, shared by the single-lattice kernel
// (lbm_step.cu) and the batched multi-lattice kernel (lbm_batch.cu). See lbm_step.cu for the
// storage scheme and the stage structure.
#pragma once

#include <math.h>

#include "lbm_internal.cuh"

namespace lbm {
namespace stepdev {

// Explicitly rounded operations: the FP32 step is written with them so that its rounding does not
// depend on where the compiler fuses a multiply into an add (which can differ between the kernels
// that inline it), and the single-lattice and batched kernels stay bit-identical.
__device__ __forceinline__ float add_rn(float x, float y) { return __fadd_rn(x, y); }
__device__ __forceinline__ float sub_rn(float x, float y) { return __fsub_rn(x, y); }
__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ float fma_rn(float x, float y, float z) { return __fmaf_rn(x, y, z); }
__device__ __forceinline__ double add_rn(double x, double y) { return __dadd_rn(x, y); }
__device__ __forceinline__ double sub_rn(double x, double y) { return __dsub_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }
__device__ __forceinline__ double fma_rn(double x, double y, double z) { return __fma_rn(x, y, z); }

// Bulk chemical potential psi'(rho) at k = 1: Eq. 11 without the gradient term (PR), or the CS
// counterpart from Eq. 9 with the ideal-gas antiderivative. The FP32 path uses the hardware
// logarithm and approximate division (relative error ~1e-6 on psi', far below the FP32 noise
// of the force); the FP64 path keeps correctly rounded operations.
template <typename T>
__device__ __forceinline__ T psi_prime(T rho, const StepArgs<T>& a);

template <>
__device__ __forceinline__ float psi_prime<float>(float rho, const StepArgs<float>& a) {
    if (a.eos == LBM_EOS_PR) {
        // with d1 = 1 - b rho, d2 = sqrt2 + 1 - b rho, n2 = sqrt2 - 1 + b rho the three
        // divisions of Eq. 11 share one reciprocal, since 1 + 2 b rho - (b rho)^2 = d2 n2
        const float s2 = 1.41421356f;
        const float br = mul_rn(a.b, rho);
        const float d1 = sub_rn(1.0f, br), d2 = sub_rn(s2 + 1.0f, br), n2 = add_rn(s2 - 1.0f, br);
        const float dn = mul_rn(d2, n2);
        const float r = __fdividef(1.0f, mul_rn(d1, dn));
        const float inv_d1 = mul_rn(dn, r);  // 1 / d1
        const float inv_dn = mul_rn(d1, r);  // 1 / (d2 n2)
        const float t13 = mul_rn(a.RT, add_rn(__logf(mul_rn(rho, inv_d1)), inv_d1));
        const float c2 = mul_rn(a.aal, __fdividef(1.0f, mul_rn(2.0f * s2, a.b)));
        const float t2 = mul_rn(c2, __logf(mul_rn(mul_rn(n2, n2), inv_dn)));
        const float t4 = mul_rn(mul_rn(a.aal, rho), inv_dn);
        return sub_rn(sub_rn(t13, t2), t4);
    }
    const float n = mul_rn(mul_rn(a.b, rho), 0.25f);
    const float om = sub_rn(1.0f, n);
    const float num = mul_rn(n, fma_rn(fma_rn(3.0f, n, -9.0f), n, 8.0f));  // 8n - 9n^2 + 3n^3
    return fma_rn(a.RT, add_rn(__logf(rho), __fdividef(num, mul_rn(mul_rn(om, om), om))),
                  mul_rn(-2.0f * a.aal, rho));
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

// correctly rounded reciprocal (hardware approximation plus refinement in FP32)
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }


// Collision in deviation variables g_q = f_q - w_q rho with exact-difference forcing (Eq. 13).
// MRT: Lallemand-Luo moments (rho, e, eps, jx, qx, jy, qy, pxx, pxy); the equilibrium moments of
// Eq. 2 minus those of w_q rho are (0, 3 rho u^2, -3 rho u^2, jx, -jx, jy, -jy,
// rho (ux^2 - uy^2), rho ux uy). The forcing term F_q = f_eq(rho, u') - f_eq(rho, u) with
// u' = u + F / rho has the moments (0, 3 rho (u'^2 - u^2), -3 rho (u'^2 - u^2), Fx, -Fx, Fy, -Fy,
// rho (u'x^2 - u'y^2 - ux^2 + uy^2), rho (u'x u'y - ux uy)); it is added in moment space, so a
// single back-transform M^-1 = M^T diag(1/|M_k|^2) applies relaxation and forcing together.
// BGK: g - (g - g_eq) / tau + F_q evaluated per direction.
template <typename T>
__device__ __forceinline__ void collide(T g[9], T rho, T Fx, T Fy, const StepArgs<T>& a,
                                        T& ux, T& uy) {
    const T inv_rho = recip(rho);
    // sums and differences of opposite (axis) and mirrored (diagonal) pairs
    const T s13 = add_rn(g[1], g[3]), s24 = add_rn(g[2], g[4]);
    const T d13 = sub_rn(g[1], g[3]), d24 = sub_rn(g[2], g[4]);
    const T s57 = add_rn(g[5], g[7]), s68 = add_rn(g[6], g[8]);
    const T e57 = sub_rn(g[5], g[7]), e86 = sub_rn(g[8], g[6]);
    const T jx = add_rn(d13, add_rn(e57, e86));
    const T jy = add_rn(d24, sub_rn(e57, e86));
    ux = mul_rn(jx, inv_rho);
    uy = mul_rn(jy, inv_rho);
    const T uxx = mul_rn(ux, ux), uyy = mul_rn(uy, uy), uxy = mul_rn(ux, uy);
    const T uu = add_rn(uxx, uyy);
    if (a.bgk) {
        const T sx = (T)2 * ux + Fx * inv_rho, sy = (T)2 * uy + Fy * inv_rho;
        const T Fs = Fx * sx + Fy * sy;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const T eu = (T)qx(q) * ux + (T)qy(q) * uy;
            const T geq = rho * qw<T>(q) * ((T)3 * eu + (T)4.5 * eu * eu - (T)1.5 * uu);
            const T eF = (T)qx(q) * Fx + (T)qy(q) * Fy;
            const T es = (T)qx(q) * sx + (T)qy(q) * sy;
            g[q] += -(g[q] - geq) * a.inv_tau +
                    qw<T>(q) * ((T)3 * eF + (T)4.5 * eF * es - (T)1.5 * Fs);
        }
        return;
    }
    // forced velocity and the moment increments of the forcing term
    const T vx = fma_rn(Fx, inv_rho, ux), vy = fma_rn(Fy, inv_rho, uy);
    const T vxx = mul_rn(vx, vx), vyy = mul_rn(vy, vy), vxy = mul_rn(vx, vy);
    const T r3 = mul_rn((T)3, rho);
    const T pu = sub_rn(uxx, uyy);
    const T dE = mul_rn(r3, sub_rn(add_rn(vxx, vyy), uu));
    const T dP = mul_rn(rho, sub_rn(sub_rn(vxx, vyy), pu));
    const T dQ = mul_rn(rho, sub_rn(vxy, uxy));
    // non-conserved moments (Lallemand-Luo order)
    const T axis = add_rn(s13, s24), diag = add_rn(s57, s68);
    const T m1 = fma_rn((T)-4, g[0], fma_rn((T)2, diag, -axis));  // e
    const T m2 = fma_rn((T)4, g[0], fma_rn((T)-2, axis, diag));   // eps
    const T m4 = fma_rn((T)-3, d13, jx);                          // qx
    const T m6 = fma_rn((T)-3, d24, jy);                          // qy
    const T m7 = sub_rn(s13, s24);                                // pxx
    const T m8 = sub_rn(s57, s68);                                // pxy
    // a_k = (S_k (m_k - m_eq,k) - dM_k) / |M_k|^2
    const T ruu3 = mul_rn(r3, uu);
    const T a1 = mul_rn(fma_rn(a.s_e, sub_rn(m1, ruu3), -dE), (T)1 / (T)36);
    const T a2 = mul_rn(fma_rn(a.s_eps, add_rn(m2, ruu3), dE), (T)1 / (T)36);
    const T a3 = mul_rn(Fx, (T)-1 / (T)6);
    const T a5 = mul_rn(Fy, (T)-1 / (T)6);
    const T a4 = mul_rn(fma_rn(a.s_q, add_rn(m4, jx), Fx), (T)1 / (T)12);
    const T a6 = mul_rn(fma_rn(a.s_q, add_rn(m6, jy), Fy), (T)1 / (T)12);
    const T a7 = mul_rn(fma_rn(a.s_v, fma_rn(-rho, pu, m7), -dP), (T)0.25);
    const T a8 = mul_rn(fma_rn(a.s_v, fma_rn(-rho, uxy, m8), -dQ), (T)0.25);
    // back-transform M^-1 a, grouped by pairs: g_q -= sum_k M_kq a_k
    const T c_ax = fma_rn((T)-2, a2, -a1);
    const T c_dg = fma_rn((T)2, a1, a2);
    g[0] = fma_rn((T)4, sub_rn(a1, a2), g[0]);
    const T S13 = add_rn(c_ax, a7), D13 = fma_rn((T)-2, a4, a3);
    const T S24 = sub_rn(c_ax, a7), D24 = fma_rn((T)-2, a6, a5);
    g[1] = sub_rn(g[1], add_rn(S13, D13));
    g[3] = sub_rn(g[3], sub_rn(S13, D13));
    g[2] = sub_rn(g[2], add_rn(S24, D24));
    g[4] = sub_rn(g[4], sub_rn(S24, D24));
    const T p34 = add_rn(a3, a4), p56 = add_rn(a5, a6);
    const T S57 = add_rn(c_dg, a8), S68 = sub_rn(c_dg, a8);
    const T D57 = add_rn(p34, p56), D68 = sub_rn(p56, p34);
    g[5] = sub_rn(g[5], add_rn(S57, D57));
    g[7] = sub_rn(g[7], sub_rn(S57, D57));
    g[6] = sub_rn(g[6], add_rn(S68, D68));
    g[8] = sub_rn(g[8], sub_rn(S68, D68));
}

template <typename T, int TX, int TY>
struct Layout {
    static constexpr int RW = TX + 16, RH = TY + 14;  // rho / flags: x0-8.., y0-7..
    static constexpr int MW = TX + 6, MH = TY + 6;    // mu: x0-3.., y0-3..
    static constexpr int CW = TX + 2, CH = TY + 2;    // g*: x0-1.., y0-1..
    // g* holds 9 planes plus one for sum_q w_q rho(x - e_q, t) (the rest-state part of the
    // next density, formed where the neighbour densities are already in registers)
    static constexpr size_t bytes =
        sizeof(T) * ((size_t)RW * RH + (size_t)MW * MH + 10 * (size_t)CW * CH) + (size_t)RW * RH;
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
    // 12 x the fourth-order Laplacian: 16 (sum of axis neighbours at 1) - 60 c0 - (sum at 2)
    const T s1 = add_rn(add_rn(s_rho[o + 1], s_rho[o - 1]), add_rn(s_rho[o + RW], s_rho[o - RW]));
    const T s2 = add_rn(add_rn(s_rho[o + 2], s_rho[o - 2]),
                        add_rn(s_rho[o + 2 * RW], s_rho[o - 2 * RW]));
    const T lap12 = fma_rn((T)16, s1, fma_rn((T)-60, c0, -s2));
    return fma_rn(a.k2, psi_prime<T>(c0, a), mul_rn(mul_rn(a.kappa, (T)-1 / (T)12), lap12));
}

// Interpolated bounce-back of population q at fluid node x whose source x - e_q is solid, as a
// deviation from w_q rho(x). out = h_qbar(x) is the deviation of the population that left x
// toward the wall (what half-way bounce-back returns). With the wall at the link fraction D:
//   D < 1/2: 2D f*_qbar(x) + (1 - 2D) f*_qbar(x + e_q)   (the half-way value if x + e_q is not
//            fluid), i.e. 2D out + (1 - 2D) (h_qbar(x + e_q) + w_q (rho(x + e_q) - rho(x)));
//   D >= 1/2: f*_qbar(x) / 2D + (1 - 1/2D) f*_q(x), i.e. out / 2D + (1 - 1/2D) h_q(x).
// The caller adds out minus the returned value to the rest population (mass correction).
template <typename T, int RW, bool PP>
__device__ __forceinline__ T ibb_return(const StepArgs<T>& a, int q, unsigned us, int o, T rho,
                                        T out, const T* s_rho, const uint8_t* s_flag) {
    const T D = a.dlt[(unsigned)(q - 1) * (unsigned)a.plane + us];
    const T D2 = add_rn(D, D);
    if (D < (T)0.5) {
        const int ob = o + qy(q) * RW + qx(q);
        if (s_flag[ob] != kFluid) return out;
        const unsigned ub = us + (unsigned)(qy(q) * a.P + qx(q));
        const T hbh = PP ? __ldg(a.hq_in[qopp(q)] + ub)
                         : __ldg(a.h_in + (unsigned)qopp(q) * (unsigned)a.plane + ub);
        const T behind = fma_rn(qw<T>(q), sub_rn(s_rho[ob], rho), hbh);
        return fma_rn(D2, out, mul_rn(sub_rn((T)1, D2), behind));
    }
    const T hq = PP ? __ldg(a.hq_in[q] + us) : __ldg(a.h_in + (unsigned)q * (unsigned)a.plane + us);
    const T c = recip(D2);
    return fma_rn(c, out, mul_rn(sub_rn((T)1, c), hq));  // exactly out at D = 1/2
}

// (6) of the step: new density rho(t+1) = sum_q f*_q(x - e_q) (half-way bounce-back where the
// source is not fluid) and the stored deviations f*_q(x) - w_q rho(t+1)(x). EDGE: the tile lies
// within kPadX of an x edge and also writes the periodic images into the pads. PP: the planes
// are addressed through the per-plane pointers of StepArgs (single-lattice kernel), else as
// h_out + q * plane (batched kernel).
template <typename T, int TX, int TY, int NT, bool MIXED, bool EDGE, bool PP>
__device__ __forceinline__ void stream_out(const StepArgs<T>& a, const T* s_rho, const T* s_g,
                                           const uint8_t* s_flag, int x0, int y0) {
    using L = Layout<T, TX, TY>;
    constexpr int RW = L::RW, CW = L::CW, CH = L::CH;
    const unsigned upl = (unsigned)a.plane;
    for (int idx = threadIdx.x; idx < TX * TY; idx += NT) {
        const int ty = idx / TX, tx = idx - ty * TX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (MIXED && (gx >= a.nx || gy >= a.ny)) continue;
        const int o = (ty + 7) * RW + (tx + 8);
        if (MIXED && s_flag[o] != kFluid) continue;
        const int oc = (ty + 1) * CW + (tx + 1);
        const T r0 = s_rho[o];
        T B = s_g[oc];
#pragma unroll
        for (int q = 1; q < 9; ++q) {
            const int os = o - qy(q) * RW - qx(q);
            if (!MIXED || s_flag[os] == kFluid)
                B = add_rn(B, s_g[q * CW * CH + oc - qy(q) * CW - qx(q)]);
            else
                B = add_rn(B, s_g[qopp(q) * CW * CH + oc]);
        }
        const T r1 = add_rn(s_g[9 * CW * CH + oc], B);
        const unsigned us = (unsigned)lidx(a.P, gx, gy);
        const T dr = sub_rn(r0, r1);
        T v[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] = fma_rn(qw<T>(q), dr, s_g[q * CW * CH + oc]);
        if (EDGE) {
            const bool lo = gx < kPadX, hi = gx >= a.nx - kPadX;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                T* ob = (PP ? a.hq_out[q] : a.h_out + (unsigned)q * upl) + us;
                ob[0] = v[q];
                if (lo) ob[a.nx] = v[q];
                if (hi) ob[-a.nx] = v[q];
            }
            a.rho_out[us] = r1;
            if (lo) a.rho_out[us + a.nx] = r1;
            if (hi) a.rho_out[us - a.nx] = r1;
        } else {
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                if (PP)
                    a.hq_out[q][us] = v[q];
                else
                    a.h_out[us + (unsigned)q * upl] = v[q];
            }
            a.rho_out[us] = r1;
        }
    }
}

// MIXED: the tile and its halo contain non-fluid nodes (walls, the disc, the domain edge), so
// wetting layers are rebuilt and every neighbour access checks the node class. Interior tiles
// take the branch-free path (the choice is uniform per CTA). IBB: interpolated, mass-corrected
// bounce-back on cut links (a separate kernel, so the default one carries none of its code).
template <typename T, int TX, int TY, int NT, bool MACRO, bool MIXED, bool PP, bool IBB = false>
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
                    num = fma_rn(qw<T>(q), s_rho[on], num);
                    den = add_rn(den, qw<T>(q));
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
                    num = fma_rn(qw<T>(q), s_rho[on], num);
                    den = add_rn(den, qw<T>(q));
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
    // PP = false: 32-bit element offsets of plane q and of the pulled source of direction q
    // (the same for every thread, so they live in uniform registers)
    const unsigned upl = (unsigned)a.plane, uP = (unsigned)a.P;
#define QPL(q) ((unsigned)(q) * upl)
#define QSRC(q) ((unsigned)(q) * upl - (unsigned)(qy(q) * (int)uP + qx(q)))
    for (int idx = tid; idx < CW * CH; idx += NT) {
        const int cy = idx / CW, cx = idx - cy * CW;
        const int o = (cy + 6) * RW + (cx + 7);
        if (MIXED && s_flag[o] != kFluid) continue;
        const int om = (cy + 2) * MW + (cx + 2);
        const int gx = x0 - 1 + cx, gy = y0 - 1 + cy;
        const int self = lidx(a.P, gx, gy);
        const T rho = s_rho[o];
        // Eq. 7: F = -rho grad(mu) + c_s^2 grad(rho) + rho g with fourth-order differences;
        // G = 12 x the derivative: 8 (f(+1) - f(-1)) - (f(+2) - f(-2))
        const T Gmx = fma_rn((T)8, sub_rn(s_mu[om + 1], s_mu[om - 1]),
                             sub_rn(s_mu[om - 2], s_mu[om + 2]));
        const T Gmy = fma_rn((T)8, sub_rn(s_mu[om + MW], s_mu[om - MW]),
                             sub_rn(s_mu[om - 2 * MW], s_mu[om + 2 * MW]));
        const T Grx = fma_rn((T)8, sub_rn(s_rho[o + 1], s_rho[o - 1]),
                             sub_rn(s_rho[o - 2], s_rho[o + 2]));
        const T Gry = fma_rn((T)8, sub_rn(s_rho[o + RW], s_rho[o - RW]),
                             sub_rn(s_rho[o - 2 * RW], s_rho[o + 2 * RW]));
        const T Fx = fma_rn(rho, fma_rn(Gmx, (T)-1 / (T)12, a.gx), fma_rn(Grx, (T)1 / (T)36, a.gbx));
        const T Fy = fma_rn(rho, fma_rn(Gmy, (T)-1 / (T)12, a.gy), fma_rn(Gry, (T)1 / (T)36, a.gby));
        // pull the populations of time t (Eq. 4) with half-way bounce-back
        const unsigned us = (unsigned)self;
        const T* hb = a.h_in + us;
        // PP: rows of the sources with e_q,y = 0, +1, -1
        const unsigned r0 = us, rdn = us - uP, rup = us + uP;
        T g[9];
        g[0] = PP ? __ldg(a.hq_in[0] + r0) : __ldg(hb);
        T A = mul_rn(qw<T>(0), rho);  // sum_q w_q rho(x - e_q); bounce-back sources take rho(x)
        T dm = (T)0;                  // interpolated bounce-back: mass returned to the rest population
#pragma unroll
        for (int q = 1; q < 9; ++q) {
            const int os = o - qy(q) * RW - qx(q);
            if (!MIXED || s_flag[os] == kFluid) {
                const T rs = s_rho[os];
                const T h = PP ? __ldg(a.hq_in[q] + (int)((qy(q) > 0 ? rdn : qy(q) < 0 ? rup : r0) -
                                                          qx(q)))
                               : __ldg(hb + (int)QSRC(q));
                g[q] = fma_rn(qw<T>(q), sub_rn(rs, rho), h);
                A = fma_rn(qw<T>(q), rs, A);
            } else {
                const T out = PP ? __ldg(a.hq_in[qopp(q)] + r0) : __ldg(hb + (int)QPL(qopp(q)));
                g[q] = out;
                if (MIXED && IBB) {
                    g[q] = ibb_return<T, RW, PP>(a, q, us, o, rho, out, s_rho, s_flag);
                    dm = add_rn(dm, sub_rn(out, g[q]));
                }
                A = fma_rn(qw<T>(q), rho, A);
            }
        }
        if (MIXED && IBB) g[0] = add_rn(g[0], dm);
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
            s_g[9 * CW * CH + idx] = A;
        }
    }
    if (MACRO) return;
    __syncthreads();

    // (6) streaming into the tile: new density and deviations; tiles within kPadX of the x
    // edges also refresh the periodic images in the pads (a CTA-uniform branch)
    if (x0 < kPadX || x0 + TX > a.nx - kPadX)
        stream_out<T, TX, TY, NT, MIXED, true, PP>(a, s_rho, s_g, s_flag, x0, y0);
    else
        stream_out<T, TX, TY, NT, MIXED, false, PP>(a, s_rho, s_g, s_flag, x0, y0);
#undef QPL
#undef QSRC
}

// (1) density and flags on x0-8 .. x0+TX+7, y0-7 .. y0+TY+6, four nodes per access; the pads
// supply periodic images and wall rows, positions past the padded plane read as solid. Returns,
// in the thread's bits: 1 if it saw a non-fluid node, 2 if it saw a fluid node of the tile.
template <typename T, int TX, int TY, int NT>
__device__ __forceinline__ int stage_load(const StepArgs<T>& a, T* s_rho, uint8_t* s_flag, int x0,
                                          int y0) {
    using L = Layout<T, TX, TY>;
    constexpr int RW = L::RW, RH = L::RH;
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
        any |= fl != 0u ? 1 : 0;
        // a zero byte (fluid) among the four, inside the tile proper
        const bool inside = r >= 7 && r < 7 + TY && c4 >= 2 && c4 < 2 + TX / 4;
        if (inside && ((fl - 0x01010101u) & ~fl & 0x80808080u)) any |= 2;
    }
    return any;
}

// One time step of one TX x TY tile with origin (x0, y0); smem holds Layout<T, TX, TY>::bytes.
template <typename T, int TX, int TY, int NT, bool MACRO, bool PP, bool IBB = false>
__device__ __forceinline__ void step_tile(const StepArgs<T>& a, const T rho_mid,
                                          unsigned char* smem, int x0, int y0) {
    using L = Layout<T, TX, TY>;
    constexpr int RW = L::RW, RH = L::RH, MW = L::MW, MH = L::MH, CW = L::CW, CH = L::CH;
    T* s_rho = reinterpret_cast<T*>(smem);
    T* s_mu = s_rho + RW * RH;
    T* s_g = s_mu + MW * MH;
    uint8_t* s_flag = reinterpret_cast<uint8_t*>(s_g + 10 * CW * CH);
    const int any = stage_load<T, TX, TY, NT>(a, s_rho, s_flag, x0, y0);
    const int mixed = __syncthreads_or(any & 1);
    // a tile without fluid nodes (inside the disc or the wall rows) has nothing to write
    // (an all-fluid staged region certainly holds fluid nodes: one barrier less for those)
    if (mixed && !__syncthreads_or(any & 2)) return;
    if (mixed)
        step_body<T, TX, TY, NT, MACRO, true, PP, IBB>(a, rho_mid, s_rho, s_mu, s_g, s_flag, x0,
                                                       y0);
    else
        step_body<T, TX, TY, NT, MACRO, false, PP>(a, rho_mid, s_rho, s_mu, s_g, s_flag, x0, y0);
}

template <typename T, int TX, int TY, int NT, bool MACRO, int MINB, bool IBB = false>
__global__ void __launch_bounds__(NT, MINB) k_step(const StepArgs<T> a, const T rho_mid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    step_tile<T, TX, TY, NT, MACRO, true, IBB>(a, rho_mid, smem_raw, blockIdx.x * TX,
                                               blockIdx.y * TY);
}

}  // namespace stepdev
}  // namespace lbm
