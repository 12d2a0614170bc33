// Geometry and initial-state kernels (Sec. 3.1, Fig. 1, Fig. 9, Eq. 16).
//
// Classification is integer-exact: a node is solid when it lies in a wall row or in the circle's
// solid (inside the closed disc, or outside it for a concave cavity), tested in doubled-integer
// coordinates. Wetting layers follow Sec. 3.1: layer 1 is
// a solid node with a fluid node among its 8 neighbours, layer 2 a remaining solid node with a
// layer-1 node among its 8 neighbours. Both passes update flags in place: layer 1 only reads the
// fluid/solid distinction, which it never changes, and layer 2 only reads "is layer 1", which it
// never changes.
#include <math.h>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int wrap(int i, int nx) {
    i %= nx;
    return i < 0 ? i + nx : i;
}

// node in the circle's solid: the closed disc (convex) or its complement (concave)
__device__ __forceinline__ bool in_circle_solid(const GeomArgs& g, int i, int j) {
    if (!g.has_circle) return false;
    const long long dx = 2LL * i - g.cx2, dy = 2LL * j - g.cy2;
    const bool in_disc = dx * dx + dy * dy <= g.r2 * g.r2;
    return g.concave ? !in_disc : in_disc;
}

// Classification on the canonical nodes (0 <= x < nx, -2 <= j < ny + 2); the remaining pad rows
// stay inner solid (memset by the caller) and the pad columns are filled afterwards.
__global__ void k_classify(uint8_t* flags, GeomArgs g) {
    const int rows = g.ny + 4;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)rows * g.nx;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / g.nx), i = (int)(e % g.nx);
        const int j = r - 2;
        const bool solid = j < 0 || j >= g.ny || in_circle_solid(g, i, j);
        flags[lidx(g.P, i, j)] = solid ? kSolid : kFluid;
    }
}

// match: class of neighbour that promotes (fluid for layer 1, layer 1 for layer 2)
__global__ void k_layer(uint8_t* flags, GeomArgs g, uint8_t match, uint8_t promote) {
    const int rows = g.ny + 4;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)rows * g.nx;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / g.nx), i = (int)(e % g.nx);
        const int j = r - 2;
        if (flags[lidx(g.P, i, j)] != kSolid) continue;
        bool hit = false;
#pragma unroll
        for (int q = 1; q < 9; ++q) {
            const int rr = r + qy(q);
            if (rr < 0 || rr >= rows) continue;
            hit |= flags[lidx(g.P, wrap(i + qx(q), g.nx), j + qy(q))] == match;
        }
        if (hit) flags[lidx(g.P, i, j)] = promote;
    }
}

template <typename T>
__global__ void k_muw(const uint8_t* flags, T* muw, GeomArgs g) {
    const int rows = g.ny + 4;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)rows * g.nx;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / g.nx), i = (int)(e % g.nx);
        const int j = r - 2;
        const uint8_t f = flags[lidx(g.P, i, j)];
        double mu = 0.0;
        if (f == kLayer1 || f == kLayer2) {
            if (in_circle_solid(g, i, j)) {
                mu = g.mu_circle;
                if (g.stripes) {
                    const double phi = atan2((double)j - g.cy, (double)i - g.cx);
                    const double s = g.R * (phi - 0.5 * M_PI);
                    const long long k = (long long)floor(s / g.stripe_arc);
                    mu = (k % 2 == 0) ? g.mu_circle : g.mu_stripe_b;
                }
            } else {
                mu = j < 0 ? g.mu_bottom : g.mu_top;
            }
        }
        muw[lidx(g.P, i, j)] = (T)mu;
    }
}

// bit (q-1) set when fluid node x has a solid node at x + e_q; counts fluid nodes
__global__ void k_linkmask(const uint8_t* flags, uint8_t* mask, unsigned long long* n_fluid,
                           GeomArgs g) {
    unsigned long long local = 0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < (long long)g.ny * g.nx;
         n += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(n / g.nx), i = (int)(n % g.nx);
        uint8_t m = 0;
        if (flags[lidx(g.P, i, j)] == kFluid) {
            ++local;
#pragma unroll
            for (int q = 1; q < 9; ++q)
                if (flags[lidx(g.P, wrap(i + qx(q), g.nx), j + qy(q))] != kFluid)
                    m |= (uint8_t)(1u << (q - 1));
        }
        mask[lidx(g.P, i, j)] = m;
    }
    // integer atomics: exact and order-independent
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(n_fluid, local);
}

// Fraction of the link from fluid node (i, j) along e_d at which it first enters the analytic
// solid: the disc of radius R + 1/2 (its outside for a cavity; the wall surface the half-way
// scheme approximates) or the half-planes y <= -1/2 and y >= ny - 1/2; 1/2 where the link does
// not cross the wall surface within its length; at least 1/10. Every operation is a separately
// rounded IEEE double operation.
__device__ double link_fraction(const GeomArgs& g, int i, int j, int d) {
    const double vx = qx(d), vy = qy(d);
    double best = 2.0;
    if (vy < 0) {
        const double s = __ddiv_rn(__dadd_rn((double)j, 0.5), -vy);
        if (s >= 0 && s <= 1 && s < best) best = s;
    } else if (vy > 0) {
        const double s = __ddiv_rn(__dsub_rn(__dsub_rn((double)g.ny, 0.5), (double)j), vy);
        if (s >= 0 && s <= 1 && s < best) best = s;
    }
    if (g.has_circle) {
        const double px = __dsub_rn((double)i, g.cx), py = __dsub_rn((double)j, g.cy);
        const double a = __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy));
        const double b = __dadd_rn(__dmul_rn(px, vx), __dmul_rn(py, vy));
        const double Rw = __dadd_rn(g.R, 0.5);
        const double cc = __dsub_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)),
                                    __dmul_rn(Rw, Rw));
        const double disc = __dsub_rn(__dmul_rn(b, b), __dmul_rn(a, cc));
        if (disc >= 0) {
            const double sq = __dsqrt_rn(disc);
            double s = g.concave ? __ddiv_rn(__dadd_rn(-b, sq), a) : __ddiv_rn(__dsub_rn(-b, sq), a);
            // a crossing behind the node (moving away from the disc) does not count; a node on
            // the circle itself starts in the wall
            if (s > -1e-12 && s <= 1) {
                if (s < 0) s = 0;
                if (s < best) best = s;
            }
        }
    }
    best = best <= 1.0 ? best : 0.5;
    // a wall closer than a tenth of the link is taken at a tenth (Delta -> 0 copies the returned
    // population from the node behind alone, which is unstable next to a cavity wall)
    return best < 0.1 ? 0.1 : best;
}

// dlt[(q - 1) * plane + x] = link fraction toward the solid source x - e_q of population q
template <typename T>
__global__ void k_link_fractions(const uint8_t* flags, T* dlt, GeomArgs g) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < (long long)g.ny * g.nx;
         n += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(n / g.nx), i = (int)(n % g.nx);
        const int o = lidx(g.P, i, j);
        const bool fluid = flags[o] == kFluid;
#pragma unroll 1
        for (int q = 1; q < 9; ++q) {
            double v = 0.5;
            if (fluid && flags[lidx(g.P, wrap(i - qx(q), g.nx), j - qy(q))] != kFluid)
                v = link_fraction(g, i, j, qopp(q));
            dlt[(size_t)(q - 1) * g.plane + o] = (T)v;
        }
    }
}

// Eq. 16 drop (or a given density) at fluid nodes; zero elsewhere
template <typename T>
__global__ void k_init_rho(const uint8_t* flags, T* rho, T* rho_other, const double* rho0,
                           GeomArgs g, double rg, double rl, double x0, double y0, double r0,
                           double W) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < (long long)g.ny * g.nx;
         n += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(n / g.nx), i = (int)(n % g.nx);
        const int o = lidx(g.P, i, j);
        double v = 0.0;
        if (flags[o] == kFluid) {
            if (rho0) {
                v = rho0[n];
            } else {
                const double dx = i - x0, dy = j - y0;
                const double r = sqrt(dx * dx + dy * dy);
                v = 0.5 * (rg + rl) + 0.5 * (rg - rl) * tanh(2.0 * (r - r0) / W);
            }
        }
        rho[o] = (T)v;
        rho_other[o] = (T)0;
    }
}

// Stored populations are post-collision deviations h_q(z) = f*_q(z) - w_q rho(z). Starting from
// f(x, 0) = w_q rho0(x) means f*_q(z, -1) = w_q rho0(z + e_q) when z + e_q is fluid (it streams
// there) and w_q rho0(z) when it is solid (it bounces back to z).
template <typename T>
__global__ void k_init_h(const uint8_t* flags, const T* rho, T* h, GeomArgs g) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < (long long)g.ny * g.nx;
         n += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(n / g.nx), i = (int)(n % g.nx);
        const int o = lidx(g.P, i, j);
        const bool fluid = flags[o] == kFluid;
        const T r0 = rho[o];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            T v = (T)0;
            if (fluid && q > 0) {
                const int t = lidx(g.P, wrap(i + qx(q), g.nx), j + qy(q));
                if (flags[t] == kFluid) v = qw<T>(q) * (rho[t] - r0);
            }
            h[(size_t)q * g.plane + o] = v;
        }
    }
}

// Periodic images: columns -kPadX..-1 copy nx-kPadX..nx-1 and nx..nx+kPadX-1 copy 0..kPadX-1,
// on every row of the padded plane.
template <typename T>
__global__ void k_fill_pads(T* a, int nx, int P, int rows) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * 2 * kPadX;
         e += gridDim.x * blockDim.x) {
        const int r = e / (2 * kPadX), k = e % (2 * kPadX);
        const int j = r - kPadY;
        const int x = k < kPadX ? k - kPadX : nx + (k - kPadX);
        const int src = k < kPadX ? x + nx : x - nx;
        a[lidx(P, x, j)] = a[lidx(P, src, j)];
    }
}

int grid_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b > 152LL * 16) b = 152LL * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_geometry(lbm_ctx* c, const GeomArgs& g) {
    const long long next = (long long)(c->ny + 4) * c->nx;
    const long long nf = (long long)c->ny * c->nx;
    k_classify<<<grid_for(next), kThreads, 0, c->stream>>>(c->flags, g);
    k_layer<<<grid_for(next), kThreads, 0, c->stream>>>(c->flags, g, kFluid, kLayer1);
    k_layer<<<grid_for(next), kThreads, 0, c->stream>>>(c->flags, g, kLayer1, kLayer2);
    if (c->esz == 4)
        k_muw<float><<<grid_for(next), kThreads, 0, c->stream>>>(c->flags, (float*)c->muw, g);
    else
        k_muw<double><<<grid_for(next), kThreads, 0, c->stream>>>(c->flags, (double*)c->muw, g);
    const int rows = c->ny + 2 * kPadY;
    k_fill_pads<uint8_t><<<grid_for(rows * 2 * kPadX), kThreads, 0, c->stream>>>(c->flags, c->nx,
                                                                                  c->P, rows);
    if (c->esz == 4)
        k_fill_pads<float><<<grid_for(rows * 2 * kPadX), kThreads, 0, c->stream>>>(
            (float*)c->muw, c->nx, c->P, rows);
    else
        k_fill_pads<double><<<grid_for(rows * 2 * kPadX), kThreads, 0, c->stream>>>(
            (double*)c->muw, c->nx, c->P, rows);
    unsigned long long* d_nf = (unsigned long long*)c->red_out;  // scratch, overwritten later
    cudaError_t e = cudaMemsetAsync(d_nf, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    k_linkmask<<<grid_for(nf), kThreads, 0, c->stream>>>(c->flags, c->linkmask, d_nf, g);
    unsigned long long nfl = 0;
    e = cudaMemcpyAsync(&nfl, d_nf, sizeof nfl, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(c->stream);
    c->n_fluid = (int64_t)nfl;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_link_fractions(lbm_ctx* c, const GeomArgs& g) {
    const long long nf = (long long)c->ny * c->nx;
    if (c->esz == 4)
        k_link_fractions<float><<<grid_for(nf), kThreads, 0, c->stream>>>(c->flags, (float*)c->dlt, g);
    else
        k_link_fractions<double><<<grid_for(nf), kThreads, 0, c->stream>>>(c->flags, (double*)c->dlt,
                                                                           g);
    cudaError_t e = cudaGetLastError();
    for (int q = 0; q < 8 && e == cudaSuccess; ++q)
        e = launch_fill_pads(c, (char*)c->dlt + (size_t)q * c->plane * c->esz, c->esz);
    return e;
}

cudaError_t launch_init_state(lbm_ctx* c, const lbm_geometry& geo, const double* d_rho0) {
    GeomArgs g{};
    g.nx = c->nx;
    g.ny = c->ny;
    g.P = c->P;
    g.plane = (int)c->plane;
    const long long nf = (long long)c->ny * c->nx;
    // both buffers start at zero (pads and solid nodes included)
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMemsetAsync(c->h[k], 0, 9 * c->plane * c->esz, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->rho[k], 0, c->plane * c->esz, c->stream);
    }
    if (e != cudaSuccess) return e;
    if (c->esz == 4) {
        k_init_rho<float><<<grid_for(nf), kThreads, 0, c->stream>>>(
            c->flags, (float*)c->rho[0], (float*)c->rho[1], d_rho0, g, c->rho_g, c->rho_l,
            geo.drop_x, geo.drop_y, geo.drop_r, geo.drop_W);
        k_init_h<float><<<grid_for(nf), kThreads, 0, c->stream>>>(c->flags, (const float*)c->rho[0],
                                                                 (float*)c->h[0], g);
    } else {
        k_init_rho<double><<<grid_for(nf), kThreads, 0, c->stream>>>(
            c->flags, (double*)c->rho[0], (double*)c->rho[1], d_rho0, g, c->rho_g, c->rho_l,
            geo.drop_x, geo.drop_y, geo.drop_r, geo.drop_W);
        k_init_h<double><<<grid_for(nf), kThreads, 0, c->stream>>>(
            c->flags, (const double*)c->rho[0], (double*)c->h[0], g);
    }
    e = launch_fill_pads(c, c->rho[0], c->esz);
    for (int q = 0; q < 9 && e == cudaSuccess; ++q)
        e = launch_fill_pads(c, (char*)c->h[0] + (size_t)q * c->plane * c->esz, c->esz);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_fill_pads(lbm_ctx* c, void* plane, size_t esz) {
    const int rows = c->ny + 2 * kPadY;
    const int n = rows * 2 * kPadX;
    if (esz == 4)
        k_fill_pads<float><<<grid_for(n), kThreads, 0, c->stream>>>((float*)plane, c->nx, c->P, rows);
    else if (esz == 8)
        k_fill_pads<double><<<grid_for(n), kThreads, 0, c->stream>>>((double*)plane, c->nx, c->P, rows);
    else
        k_fill_pads<uint8_t><<<grid_for(n), kThreads, 0, c->stream>>>((uint8_t*)plane, c->nx, c->P,
                                                                      rows);
    return cudaGetLastError();
}

}  // namespace lbm
