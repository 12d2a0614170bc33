/*
 * FP64 CPU oracle for the chemical-potential multiphase lattice Boltzmann method with a curved
 * wetting solid and geometric contact-angle measurement (Liu, Yao, Li, Wen, arXiv:2202.06516).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, literal restatement of the method that the
 * CUDA path is checked against. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may build or call it. It shares no code, header, table or constant generator with the CUDA
 * library; the two are written independently from the paper.
 *
 * Layout (deliberately unlike the GPU): populations are array-of-structs f[node*9 + i] in FP64,
 * the step is split into separate full-lattice passes in the order of the paper
 * (density -> solid layers -> chemical potential -> force -> collision -> streaming).
 *
 * Lattice: fluid-domain nodes (i, j), 0 <= i < nx (periodic), 0 <= j < ny. Rows j = -2, -1 and
 * j = ny, ny+1 are solid wall rows (the two wetting layers the fourth-order stencil reaches).
 * Extended node index: (j + 2) * nx + i.
 *
 * Parity status per function (what pins it lives in tests/):
 *   orc_eos_eval, orc_maxwell        pinned (Gibbs-Duhem, equal-area rule, closed forms)
 *   orc_create (geometry)            pinned (brute-force classification on small cases)
 *   orc_step                         pinned (mass to round-off, EDM moments, BGK==MRT, flat
 *                                    interface coexistence, Laplace's law)
 *   orc_measure                      pinned (synthetic analytic caps of known angle)
 *   orc_cap_angle                    pinned (closed-form circle-circle angle)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------------ */
/* D2Q9 velocity set (Sec. 2.1, Eq. 1-2): rest, 4 axis, 4 diagonal; weights 4/9, 1/9, 1/36.     */
/* ------------------------------------------------------------------------------------------ */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPPOSITE[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* Lallemand-Luo moment matrix (cited for the MRT form of Eq. 1); rows are
 * (rho, e, eps, jx, qx, jy, qy, pxx, pxy), matching the zero pattern of S in Sec. 2.1. */
static const double MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

enum { ORC_FLUID = 0, ORC_LAYER1 = 1, ORC_LAYER2 = 2, ORC_SOLID = 3 };
enum { ORC_EOS_PR = 0, ORC_EOS_CS = 1 };
enum { ORC_MRT = 0, ORC_BGK = 1 };

typedef struct {
    int32_t nx, ny;
    int32_t eos;       /* ORC_EOS_PR (Eq. 10-11) or ORC_EOS_CS */
    int32_t collision; /* ORC_MRT (Eq. 1) or ORC_BGK (Eq. 3) */
    double Tr;         /* reduced temperature T/Tc */
    double k2;         /* k^2 of Eq. 12 */
    double kappa;      /* kappa-hat of Eq. 12 */
    double tau;        /* s_v = 1/tau; BGK relaxation time */
    double s_e, s_eps, s_q;
    double gx, gy;     /* body acceleration; force (rho - g_rho_ref) g */
    double g_rho_ref;  /* reference density of the body force (0: full weight) */
    double rho_g, rho_l; /* coexistence densities (<= 0: Maxwell construction) */
    int32_t has_circle;
    double cx, cy, R;  /* circle centre and radius, multiples of 1/2 */
    double mu_circle;  /* wall chemical potential on the circle */
    int32_t stripes;   /* 1: circle alternates mu_circle / mu_stripe_b by arc length */
    double stripe_arc, mu_stripe_b;
    double mu_bottom, mu_top; /* wall chemical potential on the flat wall rows */
    double drop_x, drop_y, drop_r, drop_W; /* Eq. 16 initial drop */
    int32_t nthreads;  /* OpenMP threads (<= 0: runtime default) */
    int32_t concave;   /* 1: the circle is a cavity, solid outside it (Fig. 2b) */
    int32_t interp_bb; /* 1: interpolated bounce-back on the analytic walls, mass-corrected */
} orc_cfg;

typedef struct {
    int32_t status; /* 0 ok, 1 no candidate points on this side, 2 line misses the substrate */
    double theta, alpha, beta; /* degrees */
    double cx, cy;             /* three-phase contact point */
    double p1x, p1y, p2x, p2y; /* interface points ~1 and ~2 lattice units from the substrate */
    double d1, d2;
    int64_t link1, link2;      /* node index (j*nx+i) * 4 + link slot */
} orc_angle;

typedef struct {
    orc_cfg c;
    int nx, ny, nrow; /* nrow = ny + 4 */
    double a, b, R, T, alpha; /* EOS constants */
    double rho_g, rho_l, p_sat, mu_sat;
    uint8_t *flag; /* extended */
    double *muw;   /* extended, wall chemical potential at layer nodes */
    double *f, *fpost; /* fluid-domain AoS */
    double *rho, *mu;  /* extended */
    double *fx, *fy;   /* fluid-domain force */
    double *ux, *uy;   /* fluid-domain physical velocity u + F/(2 rho) */
    long long steps;
} orc_sim;

/* ------------------------------------------------------------------------------------------ */
/* Equations of state                                                                          */
/* ------------------------------------------------------------------------------------------ */

/* Constants for an EOS at reduced temperature Tr. PR (Eq. 10): a = 2/49, b = 2/21, R = 1,
 * acentric factor 0.344 (Sec. 2.2); Tc = 0.0778 a / (0.45724 b R) from the standard PR critical
 * constants. CS: a = 1, b = 4, R = 1, Tc = 0.3773 a / (b R). */
static void eos_constants(int eos, double Tr, double *a, double *b, double *R, double *T,
                          double *alpha) {
    if (eos == ORC_EOS_PR) {
        *a = 2.0 / 49.0;
        *b = 2.0 / 21.0;
        *R = 1.0;
        double Tc = 0.0778 * (*a) / (0.45724 * (*b) * (*R));
        *T = Tr * Tc;
        double om = 0.344;
        double kap = 0.37464 + 1.54226 * om - 0.26992 * om * om;
        double s = 1.0 + kap * (1.0 - sqrt(Tr));
        *alpha = s * s;
    } else {
        *a = 1.0;
        *b = 4.0;
        *R = 1.0;
        double Tc = 0.3773 * (*a) / ((*b) * (*R));
        *T = Tr * Tc;
        *alpha = 1.0;
    }
}

/* Bulk chemical potential psi'(rho), pressure p0(rho), free-energy density psi(rho) and
 * dp0/drho. PR: psi' is Eq. 11 without the gradient term; p0 is Eq. 10; psi = rho psi' - p0
 * (Eq. 8). CS: p0 = rho R T (1+n+n^2-n^3)/(1-n)^3 - a rho^2 with n = b rho / 4; psi' follows
 * from Eq. 9 with the ideal-gas antiderivative R T ln(rho) and no further constant. */
static void eos_point(int eos, double a, double b, double R, double T, double al, double rho,
                      double *mu0, double *p0, double *psi, double *dp) {
    double m, p, d;
    if (eos == ORC_EOS_PR) {
        double br = b * rho;
        double D = 1.0 + 2.0 * br - br * br;
        double s2 = sqrt(2.0);
        m = R * T * log(rho / (1.0 - br)) -
            a * al / (2.0 * s2 * b) * log((s2 - 1.0 + br) / (s2 + 1.0 - br)) +
            R * T / (1.0 - br) - a * al * rho / D;
        p = rho * R * T / (1.0 - br) - a * al * rho * rho / D;
        double Dp = 2.0 * b - 2.0 * b * br;
        d = R * T / ((1.0 - br) * (1.0 - br)) - a * al * rho * (2.0 * D - rho * Dp) / (D * D);
    } else {
        double n = b * rho / 4.0;
        double om = 1.0 - n;
        m = R * T * (log(rho) + (8.0 * n - 9.0 * n * n + 3.0 * n * n * n) / (om * om * om)) -
            2.0 * a * rho;
        p = rho * R * T * (1.0 + n + n * n - n * n * n) / (om * om * om) - a * rho * rho;
        /* d/drho of rho R T Z(n), Z = (1+n+n^2-n^3)/(1-n)^3; dZ/dn = (4+4n-2n^2)/(1-n)^4 */
        double Z = (1.0 + n + n * n - n * n * n) / (om * om * om);
        double dZ = (4.0 + 4.0 * n - 2.0 * n * n) / (om * om * om * om);
        d = R * T * (Z + n * dZ) - 2.0 * a * rho;
    }
    if (mu0) *mu0 = m;
    if (p0) *p0 = p;
    if (psi) *psi = rho * m - p;
    if (dp) *dp = d;
}

void orc_eos_eval(int eos, double Tr, double rho, double out[4]) {
    double a, b, R, T, al;
    eos_constants(eos, Tr, &a, &b, &R, &T, &al);
    eos_point(eos, a, b, R, T, al, rho, &out[0], &out[1], &out[2], &out[3]);
}

void orc_eos_constants(int eos, double Tr, double out[5]) {
    eos_constants(eos, Tr, &out[0], &out[1], &out[2], &out[3], &out[4]);
}

/* Bisection for the zero of dp0/drho (spinodal) or of p0 - target on [lo, hi]. */
static double bisect_dp(int eos, double a, double b, double R, double T, double al, double lo,
                        double hi) {
    double dlo;
    eos_point(eos, a, b, R, T, al, lo, 0, 0, 0, &dlo);
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi), dm;
        eos_point(eos, a, b, R, T, al, mid, 0, 0, 0, &dm);
        if ((dm > 0) == (dlo > 0)) {
            lo = mid;
            dlo = dm;
        } else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

static double bisect_p(int eos, double a, double b, double R, double T, double al, double lo,
                       double hi, double target) {
    double plo;
    eos_point(eos, a, b, R, T, al, lo, 0, &plo, 0, 0);
    for (int it = 0; it < 300; ++it) {
        double mid = 0.5 * (lo + hi), pm;
        eos_point(eos, a, b, R, T, al, mid, 0, &pm, 0, 0);
        if ((pm - target > 0) == (plo - target > 0)) {
            lo = mid;
            plo = pm;
        } else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Maxwell equal-area construction (Sec. 4, under Eq. 16): the pressure p_sat at which the gas
 * and liquid roots of p0(rho) = p_sat have equal chemical potential. Bisection on p between the
 * spinodal pressures; mu_l - mu_g decreases monotonically in p because dmu = dp / rho.
 * Returns 0 on success, -1 above the critical temperature. out: rho_g, rho_l, p_sat, mu_sat. */
int orc_maxwell(int eos, double Tr, double out[4]) {
    double a, b, R, T, al;
    eos_constants(eos, Tr, &a, &b, &R, &T, &al);
    double rmax = (eos == ORC_EOS_PR) ? 1.0 / b : 4.0 / b;
    /* scan for the spinodals: dp/drho changes + -> - at rs1 and - -> + at rs2 */
    int n = 20000;
    double prev_r = rmax * 1e-6, prev_d;
    eos_point(eos, a, b, R, T, al, prev_r, 0, 0, 0, &prev_d);
    double rs1 = -1, rs2 = -1;
    for (int k = 1; k <= n; ++k) {
        double r = rmax * (1e-6 + (0.999 - 1e-6) * k / n), d;
        eos_point(eos, a, b, R, T, al, r, 0, 0, 0, &d);
        if (rs1 < 0 && prev_d > 0 && d <= 0) rs1 = bisect_dp(eos, a, b, R, T, al, prev_r, r);
        if (rs1 > 0 && rs2 < 0 && prev_d <= 0 && d > 0) {
            rs2 = bisect_dp(eos, a, b, R, T, al, prev_r, r);
            break;
        }
        prev_r = r;
        prev_d = d;
    }
    if (rs1 < 0 || rs2 < 0) return -1;
    double phi, plo;
    eos_point(eos, a, b, R, T, al, rs1, 0, &phi, 0, 0);
    eos_point(eos, a, b, R, T, al, rs2, 0, &plo, 0, 0);
    if (plo < 0) plo = 0;
    double rg = 0, rl = 0;
    for (int it = 0; it < 200; ++it) {
        double p = 0.5 * (plo + phi);
        if (p <= 0) p = 1e-300;
        rg = bisect_p(eos, a, b, R, T, al, 1e-300, rs1, p);
        rl = bisect_p(eos, a, b, R, T, al, rs2, rmax * 0.999999, p);
        double mg, ml;
        eos_point(eos, a, b, R, T, al, rg, &mg, 0, 0, 0);
        eos_point(eos, a, b, R, T, al, rl, &ml, 0, 0, 0);
        if (ml - mg > 0)
            plo = p;
        else
            phi = p;
    }
    double p = 0.5 * (plo + phi);
    rg = bisect_p(eos, a, b, R, T, al, 1e-300, rs1, p);
    rl = bisect_p(eos, a, b, R, T, al, rs2, rmax * 0.999999, p);
    out[0] = rg;
    out[1] = rl;
    out[2] = p;
    eos_point(eos, a, b, R, T, al, rg, &out[3], 0, 0, 0);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Geometry (Sec. 3.1, Fig. 1): node classification, wetting layers, wall chemical potential.  */
/* ------------------------------------------------------------------------------------------ */

static inline int wrapx(int i, int nx) { return ((i % nx) + nx) % nx; }

/* Node in the circle's solid, exact in doubled-integer coordinates: inside the closed disc for a
 * convex substrate, outside it for a concave one (a circular cavity, Fig. 2b). */
static int in_disc(const orc_cfg *c, int i, int j) {
    if (!c->has_circle) return 0;
    long long cx2 = llround(2.0 * c->cx), cy2 = llround(2.0 * c->cy), r2 = llround(2.0 * c->R);
    long long dx = 2LL * i - cx2, dy = 2LL * j - cy2;
    int inside = dx * dx + dy * dy <= r2 * r2;
    return c->concave ? !inside : inside;
}

/* Solid test: wall rows, or the circle's solid. */
static int is_solid_node(const orc_cfg *c, int i, int j) {
    if (j < 0 || j >= c->ny) return 1;
    return in_disc(c, i, j);
}

/* Wall chemical potential of a wetting-layer node: the circle's (uniform or alternating stripes
 * of arc length stripe_arc, counted counter-clockwise from the apex) if the node lies in the
 * circle's solid (the disc, or its outside for a cavity), else the flat wall row's (bottom
 * below the domain, top above it). */
static double wall_mu(const orc_cfg *c, int i, int j) {
    if (in_disc(c, i, j)) {
        if (!c->stripes) return c->mu_circle;
        double phi = atan2((double)j - c->cy, (double)i - c->cx);
        double s = c->R * (phi - 0.5 * M_PI);
        long long k = (long long)floor(s / c->stripe_arc);
        return (k % 2 == 0) ? c->mu_circle : c->mu_stripe_b;
    }
    return (j < 0) ? c->mu_bottom : c->mu_top;
}

/* Fraction Delta in [0, 1] of the link from fluid node (i, j) along direction e_d (whose end
 * node is solid) at which the segment first enters the analytic solid: the disc of radius
 * R + 1/2 (or, for a cavity, the outside of that circle), the wall surface the half-way scheme
 * approximates and the measurement uses, and the half-planes y <= -1/2 and y >= ny - 1/2 of
 * the flat walls (Delta = 1/2). A link that does not cross the wall surface within its length
 * (a fluid node already inside the R + 1/2 circle, or a solid end node not yet beyond it) keeps
 * the half-way value 1/2. Delta is at least 1/10. */
static double link_fraction(const orc_cfg *c, int i, int j, int d) {
    double vx = CX[d], vy = CY[d];
    double best = 2.0;
    if (vy < 0) {
        double s = (j + 0.5) / (-vy);
        if (s >= 0 && s <= 1 && s < best) best = s;
    } else if (vy > 0) {
        double s = ((c->ny - 0.5) - j) / vy;
        if (s >= 0 && s <= 1 && s < best) best = s;
    }
    if (c->has_circle) {
        double px = i - c->cx, py = j - c->cy;
        double a = vx * vx + vy * vy, b = px * vx + py * vy;
        double Rw = c->R + 0.5;
        double cc = px * px + py * py - Rw * Rw;
        double disc = b * b - a * cc;
        if (disc >= 0) {
            double sq = sqrt(disc);
            /* entering the disc: first root; leaving the cavity: second root */
            double s = c->concave ? (-b + sq) / a : (-b - sq) / a;
            /* a crossing behind the node does not count; a node on the circle itself starts
             * in the wall */
            if (s > -1e-12 && s <= 1) {
                if (s < 0) s = 0;
                if (s < best) best = s;
            }
        }
    }
    best = best <= 1.0 ? best : 0.5;
    /* a wall closer than a tenth of the link is taken at a tenth: as Delta -> 0 the returned
     * population is copied from the node behind alone, which drove the gas next to a cavity
     * wall through zero density */
    return best < 0.1 ? 0.1 : best;
}

double orc_link_fraction(const orc_cfg *c, int i, int j, int d) { return link_fraction(c, i, j, d); }

static void build_geometry(orc_sim *s) {
    const orc_cfg *c = &s->c;
    int nx = s->nx, nrow = s->nrow;
    uint8_t *sol = (uint8_t *)calloc((size_t)nx * nrow, 1);
    for (int r = 0; r < nrow; ++r)
        for (int i = 0; i < nx; ++i) sol[r * nx + i] = (uint8_t)is_solid_node(c, i, r - 2);
    for (size_t e = 0; e < (size_t)nx * nrow; ++e) s->flag[e] = sol[e] ? ORC_SOLID : ORC_FLUID;
    /* layer 1: solid with a fluid node among its 8 neighbours */
    for (int r = 0; r < nrow; ++r)
        for (int i = 0; i < nx; ++i) {
            if (!sol[r * nx + i]) continue;
            for (int q = 1; q < 9; ++q) {
                int rr = r + CY[q];
                if (rr < 0 || rr >= nrow) continue;
                if (!sol[rr * nx + wrapx(i + CX[q], nx)]) {
                    s->flag[r * nx + i] = ORC_LAYER1;
                    break;
                }
            }
        }
    /* layer 2: solid, not layer 1, with a layer-1 node among its 8 neighbours */
    for (int r = 0; r < nrow; ++r)
        for (int i = 0; i < nx; ++i) {
            if (s->flag[r * nx + i] != ORC_SOLID) continue;
            for (int q = 1; q < 9; ++q) {
                int rr = r + CY[q];
                if (rr < 0 || rr >= nrow) continue;
                if (s->flag[rr * nx + wrapx(i + CX[q], nx)] == ORC_LAYER1) {
                    s->flag[r * nx + i] = ORC_LAYER2;
                    break;
                }
            }
        }
    for (int r = 0; r < nrow; ++r)
        for (int i = 0; i < nx; ++i) {
            uint8_t fl = s->flag[r * nx + i];
            s->muw[r * nx + i] = (fl == ORC_LAYER1 || fl == ORC_LAYER2) ? wall_mu(c, i, r - 2) : 0.0;
        }
    free(sol);
}

/* ------------------------------------------------------------------------------------------ */
/* Creation and initial state (Eq. 16, f = f_eq(rho, 0))                                       */
/* ------------------------------------------------------------------------------------------ */

static void set_threads(const orc_sim *s) {
#ifdef _OPENMP
    if (s->c.nthreads > 0) omp_set_num_threads(s->c.nthreads);
#else
    (void)s;
#endif
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* rho0: optional fluid-domain initial density (ny*nx); otherwise the Eq. 16 drop. */
orc_sim *orc_create(const orc_cfg *cfg, const double *rho0) {
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->c = *cfg;
    s->nx = cfg->nx;
    s->ny = cfg->ny;
    s->nrow = cfg->ny + 4;
    eos_constants(cfg->eos, cfg->Tr, &s->a, &s->b, &s->R, &s->T, &s->alpha);
    double mx[4];
    if (orc_maxwell(cfg->eos, cfg->Tr, mx) != 0) {
        free(s);
        return NULL;
    }
    s->rho_g = cfg->rho_g > 0 ? cfg->rho_g : mx[0];
    s->rho_l = cfg->rho_l > 0 ? cfg->rho_l : mx[1];
    s->p_sat = mx[2];
    s->mu_sat = mx[3];
    size_t ne = (size_t)s->nx * s->nrow, nf = (size_t)s->nx * s->ny;
    s->flag = (uint8_t *)calloc(ne, 1);
    s->muw = (double *)calloc(ne, sizeof(double));
    s->rho = (double *)calloc(ne, sizeof(double));
    s->mu = (double *)calloc(ne, sizeof(double));
    s->f = (double *)calloc(nf * 9, sizeof(double));
    s->fpost = (double *)calloc(nf * 9, sizeof(double));
    s->fx = (double *)calloc(nf, sizeof(double));
    s->fy = (double *)calloc(nf, sizeof(double));
    s->ux = (double *)calloc(nf, sizeof(double));
    s->uy = (double *)calloc(nf, sizeof(double));
    build_geometry(s);
    for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
            size_t n = (size_t)j * s->nx + i;
            if (s->flag[(j + 2) * s->nx + i] != ORC_FLUID) continue;
            double r0;
            if (rho0)
                r0 = rho0[n];
            else {
                double dx = i - cfg->drop_x, dy = j - cfg->drop_y;
                double r = sqrt(dx * dx + dy * dy);
                r0 = 0.5 * (s->rho_g + s->rho_l) +
                     0.5 * (s->rho_g - s->rho_l) * tanh(2.0 * (r - cfg->drop_r) / cfg->drop_W);
            }
            s->rho[(j + 2) * s->nx + i] = r0;
            for (int q = 0; q < 9; ++q) s->f[n * 9 + q] = WT[q] * r0;
        }
    return s;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free(s->flag);
    free(s->muw);
    free(s->rho);
    free(s->mu);
    free(s->f);
    free(s->fpost);
    free(s->fx);
    free(s->fy);
    free(s->ux);
    free(s->uy);
    free(s);
}

/* ------------------------------------------------------------------------------------------ */
/* One time step, in the paper's order                                                         */
/* ------------------------------------------------------------------------------------------ */

static void feq(double rho, double ux, double uy, double out[9]) {
    double uu = ux * ux + uy * uy;
    for (int q = 0; q < 9; ++q) {
        double eu = CX[q] * ux + CY[q] * uy;
        out[q] = rho * WT[q] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Eq. 14: density of a wetting-layer node as the weighted mean over neighbours selected by the
 * switching function (fluid neighbours for layer 1, layer-1 neighbours for layer 2). */
static void solid_layer(orc_sim *s, int layer, int src) {
    int nx = s->nx, nrow = s->nrow;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nrow; ++r)
        for (int i = 0; i < nx; ++i) {
            size_t e = (size_t)r * nx + i;
            if (s->flag[e] != layer) continue;
            double num = 0, den = 0;
            for (int q = 1; q < 9; ++q) {
                int rr = r + CY[q];
                if (rr < 0 || rr >= nrow) continue;
                size_t en = (size_t)rr * nx + wrapx(i + CX[q], nx);
                if (s->flag[en] == src) {
                    num += WT[q] * s->rho[en];
                    den += WT[q];
                }
            }
            s->rho[e] = den > 0 ? num / den : 0.5 * (s->rho_g + s->rho_l);
            s->mu[e] = s->muw[e];
        }
}

void orc_step(orc_sim *s, int nsteps) {
    set_threads(s);
    const orc_cfg *c = &s->c;
    int nx = s->nx, ny = s->ny;
    double S[9];
    S[0] = 0;
    S[1] = c->s_e;
    S[2] = c->s_eps;
    S[3] = 0;
    S[4] = c->s_q;
    S[5] = 0;
    S[6] = c->s_q;
    S[7] = 1.0 / c->tau;
    S[8] = 1.0 / c->tau;
    double norm[9];
    for (int k = 0; k < 9; ++k) {
        norm[k] = 0;
        for (int q = 0; q < 9; ++q) norm[k] += MM[k][q] * MM[k][q];
    }
    for (int step = 0; step < nsteps; ++step) {
        /* (1) density at fluid nodes (Eq. 1: rho = sum f) */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t e = (size_t)(j + 2) * nx + i, n = (size_t)j * nx + i;
                if (s->flag[e] != ORC_FLUID) continue;
                double r = 0;
                for (int q = 0; q < 9; ++q) r += s->f[n * 9 + q];
                s->rho[e] = r;
            }
        /* (2) wetting layers, first then second (Eq. 14) */
        solid_layer(s, ORC_LAYER1, ORC_FLUID);
        solid_layer(s, ORC_LAYER2, ORC_LAYER1);
        /* (3) chemical potential at fluid nodes (Eq. 12, fourth-order Laplacian) */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t e = (size_t)(j + 2) * nx + i;
                if (s->flag[e] != ORC_FLUID) continue;
                const double *rr = s->rho;
                double c0 = rr[e];
                double xm1 = rr[(size_t)(j + 2) * nx + wrapx(i - 1, nx)];
                double xm2 = rr[(size_t)(j + 2) * nx + wrapx(i - 2, nx)];
                double xp1 = rr[(size_t)(j + 2) * nx + wrapx(i + 1, nx)];
                double xp2 = rr[(size_t)(j + 2) * nx + wrapx(i + 2, nx)];
                double ym1 = rr[(size_t)(j + 1) * nx + i], ym2 = rr[(size_t)(j)*nx + i];
                double yp1 = rr[(size_t)(j + 3) * nx + i], yp2 = rr[(size_t)(j + 4) * nx + i];
                double lap = (-xp2 + 16.0 * xp1 - 30.0 * c0 + 16.0 * xm1 - xm2) / 12.0 +
                             (-yp2 + 16.0 * yp1 - 30.0 * c0 + 16.0 * ym1 - ym2) / 12.0;
                double m0;
                eos_point(c->eos, s->a, s->b, s->R, s->T, s->alpha, c0, &m0, 0, 0, 0);
                s->mu[e] = c->k2 * m0 - c->kappa * lap;
            }
        /* (4)+(5) force (Eq. 7 plus rho g), collision (Eq. 1 or 3) with exact-difference
         * forcing (Eq. 13) */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t e = (size_t)(j + 2) * nx + i, n = (size_t)j * nx + i;
                if (s->flag[e] != ORC_FLUID) continue;
                size_t exm1 = (size_t)(j + 2) * nx + wrapx(i - 1, nx);
                size_t exm2 = (size_t)(j + 2) * nx + wrapx(i - 2, nx);
                size_t exp1 = (size_t)(j + 2) * nx + wrapx(i + 1, nx);
                size_t exp2 = (size_t)(j + 2) * nx + wrapx(i + 2, nx);
                size_t eym1 = (size_t)(j + 1) * nx + i, eym2 = (size_t)j * nx + i;
                size_t eyp1 = (size_t)(j + 3) * nx + i, eyp2 = (size_t)(j + 4) * nx + i;
                const double *R_ = s->rho, *M_ = s->mu;
                double dmux = (8.0 * (M_[exp1] - M_[exm1]) - (M_[exp2] - M_[exm2])) / 12.0;
                double dmuy = (8.0 * (M_[eyp1] - M_[eym1]) - (M_[eyp2] - M_[eym2])) / 12.0;
                double drx = (8.0 * (R_[exp1] - R_[exm1]) - (R_[exp2] - R_[exm2])) / 12.0;
                double dry = (8.0 * (R_[eyp1] - R_[eym1]) - (R_[eyp2] - R_[eym2])) / 12.0;
                double rho = R_[e];
                double Fx = -rho * dmux + drx / 3.0 + (rho - c->g_rho_ref) * c->gx;
                double Fy = -rho * dmuy + dry / 3.0 + (rho - c->g_rho_ref) * c->gy;
                const double *fn = &s->f[n * 9];
                double jx = 0, jy = 0;
                for (int q = 0; q < 9; ++q) {
                    jx += CX[q] * fn[q];
                    jy += CY[q] * fn[q];
                }
                double ux = jx / rho, uy = jy / rho;
                double fe[9], fe2[9], out[9];
                feq(rho, ux, uy, fe);
                feq(rho, ux + Fx / rho, uy + Fy / rho, fe2);
                if (c->collision == ORC_BGK) {
                    for (int q = 0; q < 9; ++q) out[q] = fn[q] - (fn[q] - fe[q]) / c->tau;
                } else {
                    double dm[9];
                    for (int k = 0; k < 9; ++k) {
                        double m = 0, meq = 0;
                        for (int q = 0; q < 9; ++q) {
                            m += MM[k][q] * fn[q];
                            meq += MM[k][q] * fe[q];
                        }
                        dm[k] = S[k] * (m - meq);
                    }
                    for (int q = 0; q < 9; ++q) {
                        double corr = 0;
                        for (int k = 0; k < 9; ++k) corr += MM[k][q] * dm[k] / norm[k];
                        out[q] = fn[q] - corr;
                    }
                }
                for (int q = 0; q < 9; ++q) s->fpost[n * 9 + q] = out[q] + (fe2[q] - fe[q]);
                s->fx[n] = Fx;
                s->fy[n] = Fy;
                s->ux[n] = ux + 0.5 * Fx / rho;
                s->uy[n] = uy + 0.5 * Fy / rho;
            }
        /* (6) streaming (Eq. 4); a population whose source is solid comes back from the wall:
         * half-way bounce-back returns the population that left toward it; the interpolated
         * scheme places the wall at the link fraction Delta (linear interpolation between the
         * node and its fluid neighbour behind it for Delta < 1/2, between the two opposite
         * populations of the node for Delta >= 1/2) and adds the difference between what left
         * and what returns to the rest population, so that no mass is gained or lost. */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t e = (size_t)(j + 2) * nx + i, n = (size_t)j * nx + i;
                if (s->flag[e] != ORC_FLUID) continue;
                for (int q = 0; q < 9; ++q) {
                    /* pull: population q arriving at (i, j) left (i - cx, j - cy) */
                    int si = wrapx(i - CX[q], nx), sj = j - CY[q];
                    size_t es = (size_t)(sj + 2) * nx + si;
                    if (s->flag[es] == ORC_FLUID) {
                        s->f[n * 9 + q] = s->fpost[((size_t)sj * nx + si) * 9 + q];
                        continue;
                    }
                    int qb = OPPOSITE[q];
                    double out = s->fpost[n * 9 + qb]; /* left (i, j) toward the wall */
                    double back = out;
                    if (c->interp_bb) {
                        double D = link_fraction(c, i, j, qb);
                        if (D < 0.5) {
                            int bi = wrapx(i + CX[q], nx), bj = j + CY[q];
                            size_t eb = (size_t)(bj + 2) * nx + bi;
                            if (s->flag[eb] == ORC_FLUID)
                                back = 2.0 * D * out +
                                       (1.0 - 2.0 * D) * s->fpost[((size_t)bj * nx + bi) * 9 + qb];
                        } else {
                            back = out / (2.0 * D) + (1.0 - 1.0 / (2.0 * D)) * s->fpost[n * 9 + q];
                        }
                        s->f[n * 9 + 0] += out - back;
                    }
                    s->f[n * 9 + q] = back;
                }
            }
        s->steps++;
    }
    /* refresh the density of the returned state */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t e = (size_t)(j + 2) * nx + i, n = (size_t)j * nx + i;
            if (s->flag[e] != ORC_FLUID) continue;
            double r = 0;
            for (int q = 0; q < 9; ++q) r += s->f[n * 9 + q];
            s->rho[e] = r;
        }
}

/* ------------------------------------------------------------------------------------------ */
/* Accessors                                                                                   */
/* ------------------------------------------------------------------------------------------ */

void orc_info(const orc_sim *s, double out[8]) {
    out[0] = s->rho_g;
    out[1] = s->rho_l;
    out[2] = s->p_sat;
    out[3] = s->mu_sat;
    out[4] = s->T;
    out[5] = s->alpha;
    out[6] = (double)s->steps;
    out[7] = 0;
}

/* fluid-domain density (0 at solid nodes) */
void orc_get_rho(const orc_sim *s, double *out) {
    for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
            size_t e = (size_t)(j + 2) * s->nx + i;
            out[(size_t)j * s->nx + i] = s->flag[e] == ORC_FLUID ? s->rho[e] : 0.0;
        }
}

/* extended arrays (rows -2 .. ny+1): density incl. wetting layers, chemical potential, flags,
 * wall chemical potential */
void orc_get_ext(const orc_sim *s, double *rho, double *mu, uint8_t *flag, double *muw) {
    size_t ne = (size_t)s->nx * s->nrow;
    if (rho) memcpy(rho, s->rho, ne * sizeof(double));
    if (mu) memcpy(mu, s->mu, ne * sizeof(double));
    if (flag) memcpy(flag, s->flag, ne);
    if (muw) memcpy(muw, s->muw, ne * sizeof(double));
}

void orc_get_f(const orc_sim *s, double *f) { memcpy(f, s->f, (size_t)s->nx * s->ny * 9 * sizeof(double)); }
void orc_set_f(orc_sim *s, const double *f) { memcpy(s->f, f, (size_t)s->nx * s->ny * 9 * sizeof(double)); }

/* physical velocity v = u + F / (2 rho) and force of the last step (Sec. 2.2 below Eq. 13) */
void orc_get_uv(const orc_sim *s, double *ux, double *uy, double *fx, double *fy) {
    size_t nf = (size_t)s->nx * s->ny;
    if (ux) memcpy(ux, s->ux, nf * sizeof(double));
    if (uy) memcpy(uy, s->uy, nf * sizeof(double));
    if (fx) memcpy(fx, s->fx, nf * sizeof(double));
    if (fy) memcpy(fy, s->fy, nf * sizeof(double));
}

/* total mass over fluid nodes, summed in node order */
double orc_mass(const orc_sim *s) {
    double m = 0;
    for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
            size_t e = (size_t)(j + 2) * s->nx + i, n = (size_t)j * s->nx + i;
            if (s->flag[e] != ORC_FLUID) continue;
            for (int q = 0; q < 9; ++q) m += s->f[n * 9 + q];
        }
    return m;
}

/* boundary links: (fluid node n = j*nx+i, direction q) with the node at x + e_q solid, in
 * (n, q) order. Returns the count; writes at most cap codes n*9+q. */
long long orc_links(const orc_sim *s, int64_t *out, long long cap) {
    long long k = 0;
    for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
            if (s->flag[(size_t)(j + 2) * s->nx + i] != ORC_FLUID) continue;
            for (int q = 1; q < 9; ++q) {
                int si = wrapx(i + CX[q], s->nx), sj = j + CY[q];
                if (s->flag[(size_t)(sj + 2) * s->nx + si] != ORC_FLUID) {
                    if (k < cap) out[k] = ((int64_t)j * s->nx + i) * 9 + q;
                    ++k;
                }
            }
        }
    return k;
}

/* ------------------------------------------------------------------------------------------ */
/* Contact-angle measurement (Sec. 3.2, Eq. 15, Fig. 1 and Fig. 2)                             */
/* ------------------------------------------------------------------------------------------ */

/* link slots: the four undirected D2Q9 link directions +x, +y, +x+y, -x+y */
static const int LX[4] = {1, 0, 1, -1};
static const int LY[4] = {0, 1, 1, 1};

typedef struct {
    double px, py, d;
    int64_t id;
    int side;
} cand_t;

/* Radius of the circular wall surface: half a link beyond the solid nodes (both boundary
 * schemes place the wall there). */
static double wall_radius(const orc_cfg *c) { return c->R + 0.5; }

/* Substrate distance of point (px, py), measured from the wall into the fluid: to the circle of
 * radius R + 1/2 (R with interpolated bounce-back) (the wall lies half a link between the last fluid and the first solid node;
 * outward for a convex disc, inward for a concave cavity) or to the bottom wall plane y = -1/2.
 * Evaluated with separate rounded operations (the library is built without contraction) so that
 * both implementations reach the same bits. */
static double substrate_dist(const orc_cfg *c, double px, double py) {
    if (c->has_circle) {
        double dx = px - c->cx, dy = py - c->cy;
        double r2 = dx * dx + dy * dy;
        return c->concave ? wall_radius(c) - sqrt(r2) : sqrt(r2) - wall_radius(c);
    }
    return py - (-0.5);
}

/* Liquid/gas links of a density field (fluid domain, ny*nx; a node is liquid when rho > rho_m)
 * and their Eq. 15 intersection points. Returns the number found. */
static long long collect_links(const orc_cfg *c, const uint8_t *flag, const double *rho,
                               double rho_m, cand_t *out, long long cap) {
    int nx = c->nx, ny = c->ny;
    long long k = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (flag[(size_t)(j + 2) * nx + i] != ORC_FLUID) continue;
            for (int sl = 0; sl < 4; ++sl) {
                int ti = i + LX[sl], tj = j + LY[sl];
                if (tj >= ny) continue;
                int wi = wrapx(ti, nx);
                if (flag[(size_t)(tj + 2) * nx + wi] != ORC_FLUID) continue;
                double ra = rho[(size_t)j * nx + i], rb = rho[(size_t)tj * nx + wi];
                int la = ra > rho_m, lb = rb > rho_m;
                if (la == lb) continue;
                /* gas node xg, liquid node xl, e = xl - xg (unwrapped coordinates) */
                double xg, yg, rg, rl, ex, ey;
                if (la) {
                    xg = ti; yg = tj; rg = rb; rl = ra; ex = -LX[sl]; ey = -LY[sl];
                } else {
                    xg = i; yg = j; rg = ra; rl = rb; ex = LX[sl]; ey = LY[sl];
                }
                double fr = (rho_m - rg) / (rl - rg);
                double px = xg + fr * ex, py = yg + fr * ey;
                if (k < cap) {
                    out[k].px = px;
                    out[k].py = py;
                    out[k].d = substrate_dist(c, px, py);
                    out[k].id = ((int64_t)j * nx + i) * 4 + sl;
                    out[k].side = -1;
                }
                ++k;
            }
        }
    return k;
}

static void make_flags(const orc_cfg *c, uint8_t *flag) {
    orc_sim tmp;
    memset(&tmp, 0, sizeof tmp);
    tmp.c = *c;
    tmp.nx = c->nx;
    tmp.ny = c->ny;
    tmp.nrow = c->ny + 4;
    tmp.flag = flag;
    tmp.muw = (double *)calloc((size_t)c->nx * (c->ny + 4), sizeof(double));
    build_geometry(&tmp);
    free(tmp.muw);
}

/* Measure the left (out[0]) and right (out[1]) contact angles on a fluid-domain density field.
 * rho_m is the mean of the coexistence densities (Sec. 3.2). centroid_out (optional) receives
 * the liquid-node centroid used to split the sides. */
void orc_measure(const orc_cfg *c, const double *rho, double rho_m, orc_angle out[2],
                 double *centroid_out) {
    int nx = c->nx, ny = c->ny;
    uint8_t *flag = (uint8_t *)calloc((size_t)nx * (ny + 4), 1);
    make_flags(c, flag);
    /* liquid centroid: mean position of fluid nodes with rho > rho_m, node order */
    double sx = 0, sy = 0, cnt = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (flag[(size_t)(j + 2) * nx + i] != ORC_FLUID) continue;
            if (rho[(size_t)j * nx + i] > rho_m) {
                sx += i;
                sy += j;
                cnt += 1;
            }
        }
    double qx = cnt > 0 ? sx / cnt : 0, qy = cnt > 0 ? sy / cnt : 0;
    if (centroid_out) {
        centroid_out[0] = qx;
        centroid_out[1] = qy;
    }
    long long cap = 4LL * nx * ny;
    cand_t *cd = (cand_t *)malloc(sizeof(cand_t) * (size_t)(cap > 0 ? cap : 1));
    long long n = collect_links(c, flag, rho, rho_m, cd, cap);
    /* best candidates per side for targets 1 and 2 within the band 0.5 <= d <= 2.5 */
    long long best[2][2] = {{-1, -1}, {-1, -1}};
    for (long long k = 0; k < n; ++k) {
        double d = cd[k].d;
        if (!(d >= 0.5 && d <= 2.5)) continue;
        int side;
        if (c->has_circle) {
            double ax = qx - c->cx, ay = qy - c->cy;
            double bx = cd[k].px - c->cx, by = cd[k].py - c->cy;
            double cr = ax * by - ay * bx;
            /* left = counter-clockwise from the wall normal into the fluid at the centroid:
             * (ax, ay) on a convex circle, -(ax, ay) in a concave cavity */
            side = (c->concave ? cr < 0 : cr > 0) ? 0 : 1;
        } else
            side = cd[k].px < qx ? 0 : 1;
        cd[k].side = side;
        for (int t = 0; t < 2; ++t) {
            double key = fabs(d - (t + 1.0));
            long long b = best[side][t];
            if (b < 0) {
                best[side][t] = k;
                continue;
            }
            double kb = fabs(cd[b].d - (t + 1.0));
            if (key < kb || (key == kb && cd[k].id < cd[b].id)) best[side][t] = k;
        }
    }
    for (int side = 0; side < 2; ++side) {
        orc_angle *o = &out[side];
        memset(o, 0, sizeof *o);
        long long b1 = best[side][0], b2 = best[side][1];
        if (b1 < 0 || b2 < 0 || b1 == b2) {
            o->status = 1;
            continue;
        }
        o->p1x = cd[b1].px; o->p1y = cd[b1].py; o->d1 = cd[b1].d; o->link1 = cd[b1].id;
        o->p2x = cd[b2].px; o->p2y = cd[b2].py; o->d2 = cd[b2].d; o->link2 = cd[b2].id;
        double vx = o->p2x - o->p1x, vy = o->p2y - o->p1y;
        double vl = sqrt(vx * vx + vy * vy);
        vx /= vl;
        vy /= vl;
        double Cx, Cy, tx, ty;
        if (c->has_circle) {
            double Rs = wall_radius(c);
            double wx = o->p1x - c->cx, wy = o->p1y - c->cy;
            double wv = wx * vx + wy * vy;
            double disc = wv * wv - (wx * wx + wy * wy - Rs * Rs);
            if (disc < 0) {
                o->status = 2;
                continue;
            }
            double sq = sqrt(disc);
            double s1 = -wv - sq, s2 = -wv + sq;
            double sc = fabs(s1) < fabs(s2) ? s1 : s2;
            Cx = o->p1x + sc * vx;
            Cy = o->p1y + sc * vy;
            double nxr = Cx - c->cx, nyr = Cy - c->cy, nl = sqrt(nxr * nxr + nyr * nyr);
            nxr /= nl;
            nyr /= nl;
            if (c->concave) { /* normal into the fluid points to the centre */
                nxr = -nxr;
                nyr = -nyr;
            }
            /* tangent pointing into the liquid: clockwise on the left side, counter-clockwise
             * on the right side */
            if (side == 0) {
                tx = nyr;
                ty = -nxr;
            } else {
                tx = -nyr;
                ty = nxr;
            }
        } else {
            if (vy == 0) {
                o->status = 2;
                continue;
            }
            double sc = (-0.5 - o->p1y) / vy;
            Cx = o->p1x + sc * vx;
            Cy = -0.5;
            tx = side == 0 ? 1.0 : -1.0;
            ty = 0.0;
        }
        double ct = tx * vx + ty * vy;
        if (ct > 1) ct = 1;
        if (ct < -1) ct = -1;
        o->theta = acos(ct) * 180.0 / M_PI;
        double ca = fabs(tx);
        if (ca > 1) ca = 1;
        o->alpha = acos(ca) * 180.0 / M_PI;
        /* Fig. 2: beta = theta + alpha on a convex, theta - alpha on a concave substrate */
        o->beta = !c->has_circle ? o->theta
                  : (c->concave ? o->theta - o->alpha : o->theta + o->alpha);
        o->cx = Cx;
        o->cy = Cy;
        o->status = 0;
    }
    free(cd);
    free(flag);
}

/* Candidate list for parity checks: all liquid/gas links (id, px, py, d) in node order.
 * Returns the count; writes at most cap entries. */
long long orc_candidates(const orc_cfg *c, const double *rho, double rho_m, int64_t *ids,
                         double *pxy_d, long long cap) {
    uint8_t *flag = (uint8_t *)calloc((size_t)c->nx * (c->ny + 4), 1);
    make_flags(c, flag);
    long long big = 4LL * c->nx * c->ny;
    cand_t *cd = (cand_t *)malloc(sizeof(cand_t) * (size_t)(big > 0 ? big : 1));
    long long n = collect_links(c, flag, rho, rho_m, cd, big);
    for (long long k = 0; k < n && k < cap; ++k) {
        ids[k] = cd[k].id;
        pxy_d[3 * k] = cd[k].px;
        pxy_d[3 * k + 1] = cd[k].py;
        pxy_d[3 * k + 2] = cd[k].d;
    }
    free(cd);
    free(flag);
    return n;
}

/* Spherical-cap method (Sec. 4.1): fit a circle to the drop's interface points farther than
 * dmin from the substrate (algebraic least squares), intersect it with the substrate to get the
 * base length L and the height H above the base chord, then R0 = (4H^2 + L^2) / (8H),
 * tan(beta) = L / (2 (R0 - H)), alpha = asin(L / (2 Rs)) on a circle (0 on a flat wall) and
 * theta = beta - alpha on a convex, beta + alpha on a concave substrate (Fig. 2; H is measured
 * from the chord along the wall normal into the fluid). out: theta, beta, alpha, L, H, R0, fitted
 * centre x, y, fitted radius. Returns 0, or -1 if the fit or the intersection fails. */
int orc_cap_angle(const orc_cfg *c, const double *rho, double rho_m, double dmin, double out[9]) {
    uint8_t *flag = (uint8_t *)calloc((size_t)c->nx * (c->ny + 4), 1);
    make_flags(c, flag);
    long long big = 4LL * c->nx * c->ny;
    cand_t *cd = (cand_t *)malloc(sizeof(cand_t) * (size_t)(big > 0 ? big : 1));
    long long n = collect_links(c, flag, rho, rho_m, cd, big);
    /* normal equations for x^2 + y^2 + D x + E y + F = 0 */
    double A[3][3] = {{0}}, bv[3] = {0};
    long long used = 0;
    for (long long k = 0; k < n; ++k) {
        if (cd[k].d < dmin) continue;
        double x = cd[k].px, y = cd[k].py, z = -(x * x + y * y);
        double v[3] = {x, y, 1.0};
        for (int r = 0; r < 3; ++r) {
            for (int q = 0; q < 3; ++q) A[r][q] += v[r] * v[q];
            bv[r] += v[r] * z;
        }
        ++used;
    }
    free(cd);
    free(flag);
    if (used < 3) return -1;
    /* Gaussian elimination with partial pivoting */
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col) {
            for (int q = 0; q < 3; ++q) {
                double t = A[col][q];
                A[col][q] = A[piv][q];
                A[piv][q] = t;
            }
            double t = bv[col];
            bv[col] = bv[piv];
            bv[piv] = t;
        }
        if (A[col][col] == 0) return -1;
        for (int r = col + 1; r < 3; ++r) {
            double fct = A[r][col] / A[col][col];
            for (int q = col; q < 3; ++q) A[r][q] -= fct * A[col][q];
            bv[r] -= fct * bv[col];
        }
    }
    double sol[3];
    for (int r = 2; r >= 0; --r) {
        double acc = bv[r];
        for (int q = r + 1; q < 3; ++q) acc -= A[r][q] * sol[q];
        sol[r] = acc / A[r][r];
    }
    double qx = -0.5 * sol[0], qy = -0.5 * sol[1];
    double rr = sqrt(qx * qx + qy * qy - sol[2]);
    /* base chord: intersections of the fitted drop circle with the substrate */
    double c1x, c1y, c2x, c2y, alpha;
    if (c->has_circle) {
        double Rs = wall_radius(c);
        double dx = qx - c->cx, dy = qy - c->cy, D = sqrt(dx * dx + dy * dy);
        if (D >= Rs + rr || D <= fabs(Rs - rr)) return -1;
        double aa = (Rs * Rs - rr * rr + D * D) / (2.0 * D);
        double hh = sqrt(Rs * Rs - aa * aa);
        double mx = c->cx + aa * dx / D, my = c->cy + aa * dy / D;
        c1x = mx + hh * dy / D;
        c1y = my - hh * dx / D;
        c2x = mx - hh * dy / D;
        c2y = my + hh * dx / D;
    } else {
        double yw = -0.5, dy = yw - qy;
        if (fabs(dy) >= rr) return -1;
        double hw = sqrt(rr * rr - dy * dy);
        c1x = qx - hw;
        c1y = yw;
        c2x = qx + hw;
        c2y = yw;
    }
    double L = sqrt((c2x - c1x) * (c2x - c1x) + (c2y - c1y) * (c2y - c1y));
    /* chord midpoint and unit normal pointing away from the substrate */
    double mx = 0.5 * (c1x + c2x), my = 0.5 * (c1y + c2y);
    double nx_, ny_;
    if (c->has_circle) {
        nx_ = mx - c->cx;
        ny_ = my - c->cy;
        double nl = sqrt(nx_ * nx_ + ny_ * ny_);
        nx_ /= nl;
        ny_ /= nl;
        if (c->concave) {
            nx_ = -nx_;
            ny_ = -ny_;
        }
        alpha = asin(L / (2.0 * wall_radius(c)));
    } else {
        nx_ = 0;
        ny_ = 1;
        alpha = 0;
    }
    double H = rr + ((qx - mx) * nx_ + (qy - my) * ny_);
    double R0 = (4.0 * H * H + L * L) / (8.0 * H);
    double beta = atan2(L, 2.0 * (R0 - H));
    out[0] = (c->has_circle && c->concave ? beta + alpha : beta - alpha) * 180.0 / M_PI;
    out[1] = beta * 180.0 / M_PI;
    out[2] = alpha * 180.0 / M_PI;
    out[3] = L;
    out[4] = H;
    out[5] = R0;
    out[6] = qx;
    out[7] = qy;
    out[8] = rr;
    return 0;
}
