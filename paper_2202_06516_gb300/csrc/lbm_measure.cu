// FP64 reductions and the on-device contact-angle measurement (Sec. 3.2, Eq. 15, Fig. 1-2).
//
// Reductions (mass, liquid-node count and centroid) are two-pass and deterministic: every block
// writes FP64 partial sums to scratch, one block adds them in a fixed order.
//
// Measurement: every thread scans nodes for liquid/gas links (one end rho > rho_m, the other not)
// in the four undirected link directions, places the Eq. 15 point on the link, measures its
// distance d to the substrate and keeps, per side, the links nearest to d = 1 and d = 2 within
// the band 0.5 <= d <= 2.5 (ordered by |d - target|, then link id). Blocks reduce with warp
// shuffles into per-block partials; a final single-block kernel picks the winners and builds the
// line, the contact point and the angle. The point and distance arithmetic uses explicitly
// rounded FP64 operations (no contraction), so the candidate set and the chosen links are
// reproducible bit for bit by any IEEE implementation that evaluates the same operations.
#include <math.h>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

struct Best {
    double key;
    long long id;
    double px, py, d;
};

__device__ __forceinline__ bool better(double k1, long long i1, double k2, long long i2) {
    return k1 < k2 || (k1 == k2 && i1 < i2);
}

__device__ __forceinline__ void shfl_best(Best& b, int o) {
    Best c;
    c.key = __shfl_down_sync(0xffffffffu, b.key, o);
    c.id = __shfl_down_sync(0xffffffffu, b.id, o);
    c.px = __shfl_down_sync(0xffffffffu, b.px, o);
    c.py = __shfl_down_sync(0xffffffffu, b.py, o);
    c.d = __shfl_down_sync(0xffffffffu, b.d, o);
    if (better(c.key, c.id, b.key, b.id)) b = c;
}

// link slots: the four undirected D2Q9 link directions (1,0), (0,1), (1,1), (-1,1)
__device__ __forceinline__ int slot_x(int sl) { return sl == 1 ? 0 : (sl == 3 ? -1 : 1); }
__device__ __forceinline__ int slot_y(int sl) { return sl == 0 ? 0 : 1; }

template <typename T>
__global__ void k_reduce(const T* rho, const uint8_t* flags, int nx, int ny, int P, double rho_m,
                         double* partials) {
    double acc[5] = {0, 0, 0, 0, 0};  // mass, n_liquid, sx, sy, bad
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < (long long)nx * ny;
         n += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(n / nx), i = (int)(n % nx);
        if (flags[lidx(P, i, j)] != kFluid) continue;
        const double r = (double)rho[lidx(P, i, j)];
        acc[0] += r;
        if (!(r > 0.0) || !isfinite(r)) acc[4] += 1.0;
        if (r > rho_m) {
            acc[1] += 1.0;
            acc[2] += (double)i;
            acc[3] += (double)j;
        }
    }
    __shared__ double s[kRedThreads / 32][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0;
        for (int w = 0; w < kRedThreads / 32; ++w) v += s[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 8 + threadIdx.x] = v;
    }
}

__global__ void k_reduce_final(const double* partials, int nblocks, ReduceOut* out) {
    __shared__ double s[5];
    if (threadIdx.x < 5) {
        double v = 0;
        for (int b = 0; b < nblocks; ++b) v += partials[(size_t)b * 8 + threadIdx.x];
        s[threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        out->mass = s[0];
        out->n_liquid = s[1];
        out->sx = s[1] > 0 ? s[2] / s[1] : 0.0;
        out->sy = s[1] > 0 ? s[3] / s[1] : 0.0;
        out->bad = s[4];
    }
}

// Eq. 15 point of the link from node (i, j) along slot sl, if it joins liquid and gas.
template <typename T>
__device__ __forceinline__ bool link_point(const T* rho, const uint8_t* flags, int nx, int ny,
                                           int P, double rho_m, int i, int j, int sl, double& px,
                                           double& py) {
    const int ti = i + slot_x(sl), tj = j + slot_y(sl);
    if (tj >= ny) return false;
    const int wi = ti < 0 ? ti + nx : (ti >= nx ? ti - nx : ti);
    if (flags[lidx(P, wi, tj)] != kFluid) return false;
    const double ra = (double)rho[lidx(P, i, j)], rb = (double)rho[lidx(P, wi, tj)];
    const bool la = ra > rho_m, lb = rb > rho_m;
    if (la == lb) return false;
    double xg, yg, rg, rl, ex, ey;
    if (la) {
        xg = ti; yg = tj; rg = rb; rl = ra; ex = -slot_x(sl); ey = -slot_y(sl);
    } else {
        xg = i; yg = j; rg = ra; rl = rb; ex = slot_x(sl); ey = slot_y(sl);
    }
    const double fr = __ddiv_rn(__dsub_rn(rho_m, rg), __dsub_rn(rl, rg));
    px = __dadd_rn(xg, __dmul_rn(fr, ex));
    py = __dadd_rn(yg, __dmul_rn(fr, ey));
    return true;
}

// distance from the wall surface into the fluid
__device__ __forceinline__ double substrate_dist(const Substrate& s, double px, double py) {
    if (s.circle) {
        const double dx = __dsub_rn(px, s.cx), dy = __dsub_rn(py, s.cy);
        const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        return s.concave ? __dsub_rn(s.Rs, r) : __dsub_rn(r, s.Rs);
    }
    return __dsub_rn(py, -0.5);
}

template <typename T>
__global__ void k_meas_cand(const T* rho, const uint8_t* flags, int nx, int ny, int P,
                            double rho_m, Substrate sub, const ReduceOut* red, Best* partials) {
    const double qxc = red->sx, qyc = red->sy;
    Best b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] = Best{INFINITY, 0x7fffffffffffffffLL, 0, 0, 0};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < (long long)nx * ny;
         n += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(n / nx), i = (int)(n % nx);
        if (flags[lidx(P, i, j)] != kFluid) continue;
        for (int sl = 0; sl < 4; ++sl) {
            double px, py;
            if (!link_point<T>(rho, flags, nx, ny, P, rho_m, i, j, sl, px, py)) continue;
            const double d = substrate_dist(sub, px, py);
            if (!(d >= 0.5 && d <= 2.5)) continue;
            int side;
            if (sub.circle) {
                const double ax = __dsub_rn(qxc, sub.cx), ay = __dsub_rn(qyc, sub.cy);
                const double bx = __dsub_rn(px, sub.cx), by = __dsub_rn(py, sub.cy);
                const double cr = __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx));
                // the wall normal into the fluid at the centroid is (ax, ay) on the convex
                // circle and -(ax, ay) on the concave one
                side = (sub.concave ? cr < 0.0 : cr > 0.0) ? 0 : 1;
            } else {
                side = px < qxc ? 0 : 1;
            }
            const long long id = n * 4 + sl;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const double key = fabs(__dsub_rn(d, (double)(t + 1)));
                Best& bb = b[side * 2 + t];
                if (better(key, id, bb.key, bb.id)) bb = Best{key, id, px, py, d};
            }
        }
    }
    __shared__ Best s[kRedThreads / 32][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        for (int o = 16; o > 0; o >>= 1) shfl_best(b[k], o);
        if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5][k] = b[k];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        Best r = s[0][threadIdx.x];
        for (int w = 1; w < kRedThreads / 32; ++w)
            if (better(s[w][threadIdx.x].key, s[w][threadIdx.x].id, r.key, r.id)) r = s[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 4 + threadIdx.x] = r;
    }
}

// Contact point, tangent and angle for one side (Fig. 1, Fig. 2).
__device__ void finish_side(const Best& b1, const Best& b2, const Substrate& sub, int side,
                            lbm_angle* o) {
    o->status = LBM_OK;
    if (!(b1.key < INFINITY) || !(b2.key < INFINITY) || b1.id == b2.id) {
        o->status = LBM_ERR_NO_CONTACT;
        return;
    }
    o->p1_x = b1.px; o->p1_y = b1.py; o->d1 = b1.d; o->link1 = b1.id;
    o->p2_x = b2.px; o->p2_y = b2.py; o->d2 = b2.d; o->link2 = b2.id;
    double vx = b2.px - b1.px, vy = b2.py - b1.py;
    const double vl = sqrt(vx * vx + vy * vy);
    vx /= vl;
    vy /= vl;
    double Cx, Cy, tx, ty;
    if (sub.circle) {
        const double wx = b1.px - sub.cx, wy = b1.py - sub.cy;
        const double wv = wx * vx + wy * vy;
        const double disc = wv * wv - (wx * wx + wy * wy - sub.Rs * sub.Rs);
        if (disc < 0) {
            o->status = LBM_ERR_NO_CONTACT;
            return;
        }
        const double sq = sqrt(disc);
        const double s1 = -wv - sq, s2 = -wv + sq;
        const double sc = fabs(s1) < fabs(s2) ? s1 : s2;
        Cx = b1.px + sc * vx;
        Cy = b1.py + sc * vy;
        double nxr = Cx - sub.cx, nyr = Cy - sub.cy;
        const double nl = sqrt(nxr * nxr + nyr * nyr);
        nxr /= nl;
        nyr /= nl;
        if (sub.concave) {  // wall normal into the fluid points to the centre
            nxr = -nxr;
            nyr = -nyr;
        }
        // tangent toward the liquid: clockwise on the left side, counter-clockwise on the right
        if (side == 0) {
            tx = nyr;
            ty = -nxr;
        } else {
            tx = -nyr;
            ty = nxr;
        }
    } else {
        if (vy == 0) {
            o->status = LBM_ERR_NO_CONTACT;
            return;
        }
        const double sc = (-0.5 - b1.py) / vy;
        Cx = b1.px + sc * vx;
        Cy = -0.5;
        tx = side == 0 ? 1.0 : -1.0;
        ty = 0.0;
    }
    const double ct = fmin(1.0, fmax(-1.0, tx * vx + ty * vy));
    o->theta_deg = acos(ct) * (180.0 / M_PI);
    o->alpha_deg = acos(fmin(1.0, fabs(tx))) * (180.0 / M_PI);
    o->beta_deg = !sub.circle ? o->theta_deg
                  : (sub.concave ? o->theta_deg - o->alpha_deg : o->theta_deg + o->alpha_deg);
    o->contact_x = Cx;
    o->contact_y = Cy;
}

__global__ void k_meas_final(const Best* partials, int nblocks, Substrate sub, lbm_angle* out) {
    __shared__ Best s[kRedThreads / 32][4];
    Best b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] = Best{INFINITY, 0x7fffffffffffffffLL, 0, 0, 0};
    for (int blk = threadIdx.x; blk < nblocks; blk += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const Best& c = partials[(size_t)blk * 4 + k];
            if (better(c.key, c.id, b[k].key, b[k].id)) b[k] = c;
        }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        for (int o = 16; o > 0; o >>= 1) shfl_best(b[k], o);
        if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5][k] = b[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Best w[4];
        for (int k = 0; k < 4; ++k) {
            w[k] = s[0][k];
            for (int v = 1; v < kRedThreads / 32; ++v)
                if (better(s[v][k].key, s[v][k].id, w[k].key, w[k].id)) w[k] = s[v][k];
        }
        for (int side = 0; side < 2; ++side) {
            lbm_angle o{};
            finish_side(w[side * 2], w[side * 2 + 1], sub, side, &o);
            out[side] = o;
        }
    }
}

// dense per-(node, slot) candidate marks and points, for parity checks
template <typename T>
__global__ void k_cand_dense(const T* rho, const uint8_t* flags, int nx, int ny, int P,
                             double rho_m, Substrate sub, uint8_t* mark, double* pxyd) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < (long long)nx * ny;
         n += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(n / nx), i = (int)(n % nx);
        const bool fl = flags[lidx(P, i, j)] == kFluid;
        for (int sl = 0; sl < 4; ++sl) {
            double px = 0, py = 0;
            const bool ok = fl && link_point<T>(rho, flags, nx, ny, P, rho_m, i, j, sl, px, py);
            mark[n * 4 + sl] = ok ? 1 : 0;
            if (ok) {
                pxyd[(n * 4 + sl) * 3 + 0] = px;
                pxyd[(n * 4 + sl) * 3 + 1] = py;
                pxyd[(n * 4 + sl) * 3 + 2] = substrate_dist(sub, px, py);
            }
        }
    }
}

template <typename T>
__global__ void k_to_double(const T* src, const uint8_t* flags, int nx, int ny, int P,
                            double* dst) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < (long long)nx * ny;
         n += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(n / nx), i = (int)(n % nx);
        dst[n] = flags[lidx(P, i, j)] == kFluid ? (double)src[lidx(P, i, j)] : 0.0;
    }
}

}  // namespace

cudaError_t launch_reduce(lbm_ctx* c) {
    const double rho_m = 0.5 * (c->rho_g + c->rho_l);
    if (c->esz == 4)
        k_reduce<float><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            (const float*)c->rho[c->cur], c->flags, c->nx, c->ny, c->P, rho_m, c->red_partials);
    else
        k_reduce<double><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            (const double*)c->rho[c->cur], c->flags, c->nx, c->ny, c->P, rho_m, c->red_partials);
    k_reduce_final<<<1, 32, 0, c->stream>>>(c->red_partials, c->red_blocks, c->red_out);
    return cudaGetLastError();
}

cudaError_t launch_measure(lbm_ctx* c) {
    cudaError_t e = launch_reduce(c);
    if (e != cudaSuccess) return e;
    const double rho_m = 0.5 * (c->rho_g + c->rho_l);
    Best* part = (Best*)c->meas_partials;
    if (c->esz == 4)
        k_meas_cand<float><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            (const float*)c->rho[c->cur], c->flags, c->nx, c->ny, c->P, rho_m, c->sub, c->red_out,
            part);
    else
        k_meas_cand<double><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            (const double*)c->rho[c->cur], c->flags, c->nx, c->ny, c->P, rho_m, c->sub, c->red_out,
            part);
    k_meas_final<<<1, kRedThreads, 0, c->stream>>>(part, c->red_blocks, c->sub, c->meas_out);
    return cudaGetLastError();
}

size_t meas_partial_bytes(int nblocks) { return sizeof(Best) * 4 * (size_t)nblocks; }

cudaError_t launch_candidates(lbm_ctx* c, uint8_t* d_mark, double* d_pxyd) {
    const double rho_m = 0.5 * (c->rho_g + c->rho_l);
    if (c->esz == 4)
        k_cand_dense<float><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            (const float*)c->rho[c->cur], c->flags, c->nx, c->ny, c->P, rho_m, c->sub, d_mark,
            d_pxyd);
    else
        k_cand_dense<double><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            (const double*)c->rho[c->cur], c->flags, c->nx, c->ny, c->P, rho_m, c->sub, d_mark,
            d_pxyd);
    return cudaGetLastError();
}

cudaError_t launch_to_double(lbm_ctx* c, const void* src, double* dst, int) {
    if (c->esz == 4)
        k_to_double<float><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            (const float*)src, c->flags, c->nx, c->ny, c->P, dst);
    else
        k_to_double<double><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            (const double*)src, c->flags, c->nx, c->ny, c->P, dst);
    return cudaGetLastError();
}

}  // namespace lbm
