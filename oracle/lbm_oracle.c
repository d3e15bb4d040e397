/*
 * FP64 CPU oracle for the EOS-based multiphase lattice Boltzmann step of
 * He, Qin, Chen & Wen, "Numerical simulation of pulmonary airway reopening by
 * the EOS-based multiphase lattice Boltzmann method" (arXiv 2103.08301).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline /
 * reference leg of the benchmark load this library. The CUDA product path
 * shares no code with it (no headers, tables or helpers) and never calls it.
 *
 * It is deliberately plain: double precision throughout, two population
 * arrays, and one pass per algorithmic step, each pass storing its result in
 * its own array, in the order the method defines the step:
 *
 *   1. moments        rho = sum f_i, j = sum f_i e_i, u = j / rho      (Sec. 2.1)
 *   2. ghost density  rho extended by two nodes beyond the fluid       (Sec. 2.2)
 *   3. EOS potential  phi = k^2 p0(rho) - rho/3                        (Eqs. 2.12, 2.14, 2.17)
 *   4. Laplacian      L = lap(rho)                                     (Eq. 2.17)
 *   5. force          F = -grad(phi) + kappa rho grad(L) + G           (Eq. 2.17)
 *   6. collision      BGK with u_eq = u + tau F / rho                  (Eq. 2.2, Sec. 2.1)
 *   7. pressure cols  non-equilibrium extrapolation at rho_b           (Sec. 2.2)
 *   8. streaming      f_i(x + e_i) = f*_i(x), half-way bounce-back     (Eq. 2.1, Sec. 2.2)
 *                     at wall rows and at the nodes of an optional solid mask
 *   9. diagnostics    mass, wall shear, wall pressure (Eq. 2.4)        (Sec. 3, Fig. 3)
 *
 * Where the paper is silent or garbled, the reading taken is written next to
 * the code that implements it.
 *
 * Population layout: f[i * nx * ny + y * nx + x], i = 0..8 (structure of arrays).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

/* D2Q9 lattice. The paper does not name the velocity set; its relaxation
 * matrix S (Sec. 2.1, Eq. 2.1) has nine entries, i.e. D2Q9. */
static const int ex[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ey[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double wq[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int opp[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

typedef struct {
    int32_t nx, ny;
    int32_t walls;  /* 1: rows 0 and ny-1 are solid no-slip walls; 0: periodic in y */
    int32_t bc_x;   /* 1: pressure columns at x = 0 (inlet) and x = nx-1 (outlet); 0: periodic */
    double a, b, R, T;      /* Carnahan-Starling parameters and absolute temperature */
    double k, kappa;        /* proportional coefficient (Eq. 2.13) and kappa of Eq. 2.17 */
    double tau;             /* relaxation time */
    double wet;             /* wall ghost-density offset; 0 = neutral wetting */
    /* Pressure columns. The inlet (outlet) carries the mesh pressure p_in (p_out);
     * its density is the EOS root at that pressure on the branch of the phase
     * found at the interior neighbour x_f: rho_b = rho_b_gas + theta (rho_b_liq -
     * rho_b_gas), theta = clamp((rho_f - ph_g) / (ph_l - ph_g), 0, 1) with
     * ph_g, ph_l the coexistence densities (theta = 0 when ph_l <= ph_g). */
    double rho_in_g, rho_in_l, rho_out_g, rho_out_l;
    double ph_g, ph_l;
    double gx, gy;          /* uniform body-force density added to F */
    /* Equation of state: 0 Carnahan-Starling, 1 Peng-Robinson (Eq. 2.18) with
     * aalpha = a alpha(T). */
    int32_t eos_kind;
    int32_t collision;      /* 0 BGK; 1 MRT (Eq. 2.1) with the rates below */
    double aalpha;
    /* MRT relaxation rates of the moments e, epsilon, j, q and the two stress
     * moments (Lallemand-Luo basis; the density is conserved). The forcing
     * shifts the equilibrium velocity by F / (s_j rho), so the relaxed
     * momentum gains F per step; s_j = 1/tau with every rate 1/tau is BGK. */
    double s_e, s_eps, s_j, s_q, s_nu;
    /* Optional per-node solid mask (nx*ny bytes, 1 = solid), the general wall
     * geometry of the library's lbm_init; NULL: only the rows that 'walls'
     * makes solid. With a mask, stencil reads of solid points take the ghost
     * densities of mask_ghost() below. */
    const uint8_t *mask;
} orc_params;

typedef struct {
    double mass;   /* sum of rho over the non-solid nodes of the state that was read */
    double J;      /* sum over columns of bottom + top wall shear stress of that state */
    double tw_min, tw_max; /* extrema of wall shear over both walls */
    double pw_min, pw_max; /* extrema of wall pressure over both walls */
    double Jp;     /* sum over columns of bottom + top wall pressure of that state */
} orc_diag;

/* ------------------------------------------------------------------------- */
/* Carnahan-Starling equation of state.                                       */
/* The paper's verification uses Peng-Robinson (Eq. 2.18); the workloads this */
/* oracle serves use Carnahan-Starling, p0 = rho R T Z(eta) - a rho^2 with    */
/* eta = b rho / 4 and Z = (1 + eta + eta^2 - eta^3) / (1 - eta)^3.           */
/* ------------------------------------------------------------------------- */

double orc_cs_p0(double a, double b, double R, double T, double rho)
{
    double eta = 0.25 * b * rho;
    double om = 1.0 - eta;
    double Z = (1.0 + eta + eta * eta - eta * eta * eta) / (om * om * om);
    return rho * R * T * Z - a * rho * rho;
}

/* d(eta Z)/d eta = (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4) / (1 - eta)^4 */
static double cs_g1(double eta)
{
    double om = 1.0 - eta;
    double e2 = eta * eta;
    return (1.0 + 4.0 * eta + 4.0 * e2 - 4.0 * e2 * eta + e2 * e2) / (om * om * om * om);
}

/* d^2(eta Z)/d eta^2 = (8 + 20 eta - 4 eta^2) / (1 - eta)^5 */
static double cs_g2(double eta)
{
    double om = 1.0 - eta;
    return (8.0 + 20.0 * eta - 4.0 * eta * eta) / (om * om * om * om * om);
}

double orc_cs_dp0(double a, double b, double R, double T, double rho)
{
    return R * T * cs_g1(0.25 * b * rho) - 2.0 * a * rho;
}

/* Chemical potential mu = psi'(rho) of the Carnahan-Starling free-energy
 * density psi = rho R T (ln rho - 1) + rho R T (4 eta - 3 eta^2)/(1 - eta)^2
 * - a rho^2, which satisfies p0 = rho psi' - psi (Eq. 2.5). */
double orc_cs_mu(double a, double b, double R, double T, double rho)
{
    double eta = 0.25 * b * rho;
    double om = 1.0 - eta;
    double ex_mu = (8.0 * eta - 9.0 * eta * eta + 3.0 * eta * eta * eta) / (om * om * om);
    return R * T * (log(rho) + ex_mu) - 2.0 * a * rho;
}

/* Critical point: dp0/drho = d^2p0/drho^2 = 0. Eliminating T gives
 * g1(eta) - eta g2(eta) = 0, solved by bisection; then R Tc = 8 a / (b g2). */
int orc_cs_critical(double a, double b, double R, double *Tc, double *rhoc)
{
    double lo = 1e-3, hi = 0.5;
    if (!(a > 0.0 && b > 0.0 && R > 0.0)) return 1;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        double h = cs_g1(mid) - mid * cs_g2(mid);
        if (h > 0.0) lo = mid; else hi = mid;
        if (hi - lo <= 0.0) break;
    }
    double eta = 0.5 * (lo + hi);
    *rhoc = 4.0 * eta / b;
    *Tc = 8.0 * a / (b * R * cs_g2(eta));
    return 0;
}

/* Bisection for the root of dp0/drho on [lo, hi] where its sign changes. */
static double dp0_root(double a, double b, double R, double T, double lo, double hi)
{
    double slo = orc_cs_dp0(a, b, R, T, lo);
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        double s = orc_cs_dp0(a, b, R, T, mid);
        if ((s > 0.0) == (slo > 0.0)) { lo = mid; slo = s; } else hi = mid;
        if (!(mid > lo || mid < hi)) break;
    }
    return 0.5 * (lo + hi);
}

/* Root of p0(rho) = p on [lo, hi], where p0 is increasing. */
static double p0_root(double a, double b, double R, double T, double p, double lo, double hi)
{
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_cs_p0(a, b, R, T, mid) < p) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Spinodal densities (roots of dp0/drho) below Tc. */
static int spinodals(double a, double b, double R, double T, double *s1, double *s2)
{
    double Tc, rhoc;
    orc_cs_critical(a, b, R, &Tc, &rhoc);
    if (!(T < Tc)) return 1;
    double rmax = 4.0 / b * (1.0 - 1e-9);
    *s1 = dp0_root(a, b, R, T, 1e-14, rhoc);
    *s2 = dp0_root(a, b, R, T, rhoc, rmax);
    return 0;
}

/* Maxwell equal-area construction: rho_g < rho_l with equal pressure and equal
 * chemical potential (the coexistence the paper checks its model against,
 * Sec. 2.1 "Verification"). Solved as a bisection on the saturation pressure. */
int orc_maxwell(double a, double b, double R, double T, double *rho_g, double *rho_l, double *p_sat)
{
    double s1, s2;
    if (spinodals(a, b, R, T, &s1, &s2)) return 1;
    double rmax = 4.0 / b * (1.0 - 1e-12);
    double plo = orc_cs_p0(a, b, R, T, s2);
    double phi = orc_cs_p0(a, b, R, T, s1);
    if (plo < 0.0) plo = 0.0;
    /* Delta mu(p) = mu(gas root) - mu(liquid root) changes sign across (plo, phi). */
    double lo = plo, hi = phi;
    for (int it = 0; it < 300; ++it) {
        double p = 0.5 * (lo + hi);
        if (p <= lo || p >= hi) break;
        double rg = p0_root(a, b, R, T, p, 1e-300, s1);
        double rl = p0_root(a, b, R, T, p, s2, rmax);
        double dmu = orc_cs_mu(a, b, R, T, rg) - orc_cs_mu(a, b, R, T, rl);
        /* At high p the gas root sits near its spinodal, where its chemical
         * potential exceeds the liquid's: dmu > 0 means p is above p_sat. */
        if (dmu > 0.0) hi = p; else lo = p;
    }
    double p = 0.5 * (lo + hi);
    *p_sat = p;
    *rho_g = p0_root(a, b, R, T, p, 1e-300, s1);
    *rho_l = p0_root(a, b, R, T, p, s2, rmax);
    return 0;
}

/* Density on the liquid branch whose EOS pressure is p0_target (below Tc). */
int orc_liquid_root(double a, double b, double R, double T, double p0_target, double *rho)
{
    double s1, s2;
    if (spinodals(a, b, R, T, &s1, &s2)) return 1;
    double rmax = 4.0 / b * (1.0 - 1e-12);
    if (!(p0_target > orc_cs_p0(a, b, R, T, s2))) return 1;
    *rho = p0_root(a, b, R, T, p0_target, s2, rmax);
    return 0;
}

/* Density on the gas branch whose EOS pressure is p0_target. Below Tc the gas
 * branch ends at the first spinodal; at or above Tc the EOS is monotone. */
int orc_gas_root(double a, double b, double R, double T, double p0_target, double *rho)
{
    double s1, s2, hi;
    if (spinodals(a, b, R, T, &s1, &s2) == 0) hi = s1;
    else hi = 4.0 / b * (1.0 - 1e-12);
    if (!(p0_target > 0.0) || !(p0_target < orc_cs_p0(a, b, R, T, hi))) return 1;
    *rho = p0_root(a, b, R, T, p0_target, 1e-300, hi);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Equation of state, either kind.                                            */
/* Peng-Robinson (Eq. 2.18): p0 = rho R T / (1 - b rho)                       */
/*     - a alpha rho^2 / (1 + 2 b rho - b^2 rho^2),                          */
/* alpha(T) = [1 + (0.37464 + 1.54226 w - 0.26992 w^2)(1 - sqrt(T/Tc))]^2,   */
/* the standard form of the temperature function the paper prints garbled.   */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t kind;           /* 0 Carnahan-Starling, 1 Peng-Robinson */
    double a, b, R, T;
    double aalpha;          /* PR: a alpha(T) */
} orc_eos;

double orc_pr_alpha(double omega, double T_over_Tc)
{
    double m = 0.37464 + 1.54226 * omega - 0.26992 * omega * omega;
    double t = 1.0 + m * (1.0 - sqrt(T_over_Tc));
    return t * t;
}

static double pr_den(double b, double rho) { return 1.0 + 2.0 * b * rho - b * b * rho * rho; }

double orc_eos_p0(const orc_eos *e, double rho)
{
    if (e->kind == 0) return orc_cs_p0(e->a, e->b, e->R, e->T, rho);
    return rho * e->R * e->T / (1.0 - e->b * rho) - e->aalpha * rho * rho / pr_den(e->b, rho);
}

double orc_eos_dp0(const orc_eos *e, double rho)
{
    if (e->kind == 0) return orc_cs_dp0(e->a, e->b, e->R, e->T, rho);
    double om = 1.0 - e->b * rho, D = pr_den(e->b, rho);
    return e->R * e->T / (om * om) - 2.0 * e->aalpha * rho * (1.0 + e->b * rho) / (D * D);
}

/* PR chemical potential mu = f + p0/rho with the specific free energy
 * f = int p0/rho^2 drho = R T ln(rho / (1 - b rho))
 *     - a alpha / (2 sqrt2 b) ln((sqrt2 - 1 + b rho) / (sqrt2 + 1 - b rho)),
 * so that d mu / d rho = p0' / rho (Gibbs-Duhem). */
double orc_eos_mu(const orc_eos *e, double rho)
{
    if (e->kind == 0) return orc_cs_mu(e->a, e->b, e->R, e->T, rho);
    const double r2 = sqrt(2.0), x = e->b * rho;
    double f = e->R * e->T * log(rho / (1.0 - x))
               - e->aalpha / (2.0 * r2 * e->b) * log((r2 - 1.0 + x) / (r2 + 1.0 - x));
    return f + orc_eos_p0(e, rho) / rho;
}

/* PR critical point (alpha = 1 at Tc). With x = b rho and A = a / (b R T),
 * p0' = 0 gives A = D^2 / (2 x (1 + x)(1 - x)^2) and p0'' = 0 gives
 * 2 / (1 - x)^3 = A d/dx[2 x (1 + x) / D^2]; x_c solves both (bisection). */
static double pr_crit_h(double x)
{
    double D = 1.0 + 2.0 * x - x * x, dD = 2.0 - 2.0 * x;
    double g = 2.0 * x * (1.0 + x), dg = 2.0 + 4.0 * x;
    double A = D * D / (g * (1.0 - x) * (1.0 - x));
    double dq = (dg * D - 2.0 * g * dD) / (D * D * D);  /* d/dx (g / D^2) */
    return 2.0 / ((1.0 - x) * (1.0 - x) * (1.0 - x)) - A * dq;
}

int orc_eos_critical(int kind, double a, double b, double R, double *Tc, double *rhoc)
{
    if (kind == 0) return orc_cs_critical(a, b, R, Tc, rhoc);
    if (!(a > 0.0 && b > 0.0 && R > 0.0)) return 1;
    double lo = 0.05, hi = 0.6;
    double hlo = pr_crit_h(lo);
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double h = pr_crit_h(mid);
        if ((h > 0.0) == (hlo > 0.0)) { lo = mid; hlo = h; } else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    double D = 1.0 + 2.0 * x - x * x;
    double A = D * D / (2.0 * x * (1.0 + x) * (1.0 - x) * (1.0 - x));
    *rhoc = x / b;
    *Tc = a / (b * R * A);
    return 0;
}

static double eos_rmax(const orc_eos *e) { return (e->kind == 0 ? 4.0 : 1.0) / e->b; }

/* Bisection for the root of dp0/drho on [lo, hi] where its sign changes. */
static double eos_dp0_root(const orc_eos *e, double lo, double hi)
{
    double slo = orc_eos_dp0(e, lo);
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double sm = orc_eos_dp0(e, mid);
        if ((sm > 0.0) == (slo > 0.0)) { lo = mid; slo = sm; } else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Root of p0(rho) = p on [lo, hi], where p0 is increasing. */
static double eos_p0_root(const orc_eos *e, double p, double lo, double hi)
{
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_eos_p0(e, mid) < p) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static int eos_spinodals(const orc_eos *e, double *s1, double *s2)
{
    double Tc, rhoc;
    if (orc_eos_critical(e->kind, e->a, e->b, e->R, &Tc, &rhoc)) return 1;
    if (!(e->T < Tc)) return 1;
    *s1 = eos_dp0_root(e, 1e-14, rhoc);
    *s2 = eos_dp0_root(e, rhoc, eos_rmax(e) * (1.0 - 1e-9));
    return 0;
}

/* Maxwell equal-area construction for either EOS (bisection on p_sat, as for
 * Carnahan-Starling below). */
int orc_eos_maxwell(const orc_eos *e, double *rho_g, double *rho_l, double *p_sat)
{
    double s1, s2;
    if (eos_spinodals(e, &s1, &s2)) return 1;
    double rmax = eos_rmax(e) * (1.0 - 1e-12);
    double lo = orc_eos_p0(e, s2), hi = orc_eos_p0(e, s1);
    if (lo < 0.0) lo = 0.0;
    for (int it = 0; it < 300; ++it) {
        double p = 0.5 * (lo + hi);
        if (p <= lo || p >= hi) break;
        double rg = eos_p0_root(e, p, 1e-300, s1);
        double rl = eos_p0_root(e, p, s2, rmax);
        if (orc_eos_mu(e, rg) - orc_eos_mu(e, rl) > 0.0) hi = p; else lo = p;
    }
    double p = 0.5 * (lo + hi);
    *p_sat = p;
    *rho_g = eos_p0_root(e, p, 1e-300, s1);
    *rho_l = eos_p0_root(e, p, s2, rmax);
    return 0;
}

int orc_eos_liquid_root(const orc_eos *e, double p0_target, double *rho)
{
    double s1, s2;
    if (eos_spinodals(e, &s1, &s2)) return 1;
    if (!(p0_target > orc_eos_p0(e, s2))) return 1;
    *rho = eos_p0_root(e, p0_target, s2, eos_rmax(e) * (1.0 - 1e-12));
    return 0;
}

int orc_eos_gas_root(const orc_eos *e, double p0_target, double *rho)
{
    double s1, s2, hi;
    if (eos_spinodals(e, &s1, &s2) == 0) hi = s1;
    else hi = eos_rmax(e) * (1.0 - 1e-12);
    if (!(p0_target > 0.0) || !(p0_target < orc_eos_p0(e, hi))) return 1;
    *rho = eos_p0_root(e, p0_target, 1e-300, hi);
    return 0;
}

/* Density of a pressure column on one branch (liquid = 0 gas, 1 liquid) at
 * EOS pressure p0_target. Reading: a pressure beyond the branch's end (above
 * the gas spinodal pressure, below the liquid one) holds the column at that
 * branch's spinodal density, *saturated = 1. Above Tc the gas branch is the
 * whole (monotone) EOS. Returns 1 if p0_target <= 0 on the gas branch or if
 * there is no liquid branch. */
int orc_eos_column_density(const orc_eos *e, int liquid, double p0_target, double *rho, int *saturated)
{
    double s1, s2;
    *saturated = 0;
    if (!liquid) {
        if (!(p0_target > 0.0)) return 1;
        if (eos_spinodals(e, &s1, &s2) == 0 && !(p0_target < orc_eos_p0(e, s1))) {
            *rho = s1;
            *saturated = 1;
            return 0;
        }
        return orc_eos_gas_root(e, p0_target, rho);
    }
    if (eos_spinodals(e, &s1, &s2)) return 1;
    if (!(p0_target > orc_eos_p0(e, s2))) {
        *rho = s2;
        *saturated = 1;
        return 0;
    }
    return orc_eos_liquid_root(e, p0_target, rho);
}

/* ------------------------------------------------------------------------- */
/* Lattice operators                                                          */
/* ------------------------------------------------------------------------- */

/* MRT moments (Lallemand & Luo 2000, the basis the paper cites for Eq. 2.1),
 * rows in the order (rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy) over the
 * velocities above. The rows are orthogonal, so M^-1 = M^T diag(1/|row|^2). */
static const double Mrt[Q][Q] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

/* Moments m = M f of nine populations (for the pins). */
void orc_mrt_moments(const double *f, double *m)
{
    for (int k = 0; k < Q; ++k) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += Mrt[k][i] * f[i];
        m[k] = s;
    }
}

/* MRT relaxation of Eq. 2.1: f* = f - M^-1 S M (f - f_eq), with
 * S = diag(0, s_e, s_eps, s_j, s_q, s_j, s_q, s_nu, s_nu). */
static void mrt_relax(const orc_params *p, const double *f, const double *feq, double *fs)
{
    const double rate[Q] = {0.0, p->s_e, p->s_eps, p->s_j, p->s_q, p->s_j, p->s_q, p->s_nu, p->s_nu};
    double d[Q], m[Q];
    for (int i = 0; i < Q; ++i) d[i] = f[i] - feq[i];
    orc_mrt_moments(d, m);
    for (int k = 0; k < Q; ++k) {
        double norm = 0.0;
        for (int i = 0; i < Q; ++i) norm += Mrt[k][i] * Mrt[k][i];
        m[k] *= rate[k] / norm;
    }
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += Mrt[k][i] * m[k];
        fs[i] = f[i] - s;
    }
}

/* Equilibrium, Eq. 2.2: f_i = rho w_i [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2]. */
void orc_feq(double rho, double ux, double uy, double *feq)
{
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < Q; ++i) {
        double eu = ex[i] * ux + ey[i] * uy;
        feq[i] = rho * wq[i] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Discrete gradient and Laplacian (the paper gives none; isotropic D2Q9 forms):
 *   grad psi(x) = 3 sum_i w_i e_i psi(x + e_i)
 *   lap  psi(x) = 6 sum_i w_i [psi(x + e_i) - psi(x)]
 * Both are written over an extended array E of row stride sx, evaluated at
 * the element index c. */
static void grad_ext(const double *E, long sx, long c, double *gx, double *gy)
{
    double sxv = 0.0, syv = 0.0;
    for (int i = 1; i < Q; ++i) {
        double v = E[c + ey[i] * sx + ex[i]];
        sxv += wq[i] * ex[i] * v;
        syv += wq[i] * ey[i] * v;
    }
    *gx = 3.0 * sxv;
    *gy = 3.0 * syv;
}

static double lap_ext(const double *E, long sx, long c)
{
    double s = 0.0;
    for (int i = 1; i < Q; ++i) s += wq[i] * (E[c + ey[i] * sx + ex[i]] - E[c]);
    return 6.0 * s;
}

static long pmod(long a, long n) { long r = a % n; return r < 0 ? r + n : r; }

/* Periodic versions on an nx x ny field, for the operator pins. */
void orc_grad_periodic(int nx, int ny, const double *psi, double *gx, double *gy)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double sxv = 0.0, syv = 0.0;
            for (int i = 1; i < Q; ++i) {
                double v = psi[pmod(y + ey[i], ny) * nx + pmod(x + ex[i], nx)];
                sxv += wq[i] * ex[i] * v;
                syv += wq[i] * ey[i] * v;
            }
            gx[y * nx + x] = 3.0 * sxv;
            gy[y * nx + x] = 3.0 * syv;
        }
}

void orc_lap_periodic(int nx, int ny, const double *psi, double *out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double c = psi[y * nx + x], s = 0.0;
            for (int i = 1; i < Q; ++i)
                s += wq[i] * (psi[pmod(y + ey[i], ny) * nx + pmod(x + ex[i], nx)] - c);
            out[y * nx + x] = 6.0 * s;
        }
}

/* ------------------------------------------------------------------------- */
/* Geometry (Sec. 2.2: straight rigid channel, walls top and bottom, pressure  */
/* driven ends) and the ghost-density rule for stencils that leave the fluid. */
/* ------------------------------------------------------------------------- */

static int is_solid_row(const orc_params *p, int y)
{
    return p->walls && (y == 0 || y == p->ny - 1);
}

static int is_pressure_col(const orc_params *p, int x)
{
    return p->bc_x && (x == 0 || x == p->nx - 1);
}

/* Solid lattice node: a wall row, or a node the mask marks. */
static int is_solid(const orc_params *p, int x, int y)
{
    return is_solid_row(p, y) || (p->mask && p->mask[(long)y * p->nx + x]);
}

/* Maps an integer point onto the lattice (periodic axes wrap, x beyond a
 * pressure column clamps to the column); returns 0 for rows outside a walled
 * lattice, which count as solid. */
static int map_point(const orc_params *p, int *x, int *y)
{
    if (p->bc_x) { if (*x < 0) *x = 0; if (*x > p->nx - 1) *x = p->nx - 1; }
    else *x = (int)pmod(*x, p->nx);
    if (p->walls) { if (*y < 0 || *y > p->ny - 1) return 0; }
    else *y = (int)pmod(*y, p->ny);
    return 1;
}

static int fluid_point(const orc_params *p, int x, int y)
{
    return map_point(p, &x, &y) && !is_solid(p, x, y);
}

/* Ghost density of a solid point (x, y) for the stencils of nearby fluid
 * nodes, with a mask (the paper gives no rule for general geometry; this is
 * the mirror rule of flat walls, generalised):
 *   - along the four axis directions n, the depth d of the first fluid point
 *     x + d n, d <= 2; the directions of least depth each give one mirror
 *     source: x + (2d - 1) n (the point as deep in front of the wall as x is
 *     behind it) if it is fluid, else x + d n;
 *   - no axis direction within depth 2: the four diagonals, likewise;
 *   - none either: the fluid points at knight offsets (1, 2), (2, 1), ...;
 *   - ghost = mean of the sources' densities + the wetting offset 'wet'.
 * A flat wall reduces to the channel rule: depth 1 mirrors the first fluid
 * row, depth 2 the second. Points with no fluid point within Chebyshev
 * distance 2 feed no fluid node's stencil and read 0. */
static double mask_ghost(const orc_params *p, const double *rho, int x, int y)
{
    static const int axis[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    static const int diag[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    static const int knight[8][2] = {{1, 2}, {2, 1}, {-1, 2}, {-2, 1}, {-1, -2}, {-2, -1}, {1, -2}, {2, -1}};
    double sum = 0.0;
    int n = 0;
    for (int set = 0; set < 2 && n == 0; ++set) {
        const int (*dir)[2] = set == 0 ? axis : diag;
        for (int d = 1; d <= 2 && n == 0; ++d)
            for (int k = 0; k < 4; ++k) {
                int dx = dir[k][0], dy = dir[k][1];
                if (!fluid_point(p, x + d * dx, y + d * dy)) continue;
                if (d == 2 && fluid_point(p, x + dx, y + dy)) continue;
                int sx = x + (2 * d - 1) * dx, sy = y + (2 * d - 1) * dy;
                if (!fluid_point(p, sx, sy)) { sx = x + d * dx; sy = y + d * dy; }
                map_point(p, &sx, &sy);
                sum += rho[(long)sy * p->nx + sx];
                n += 1;
            }
    }
    if (n == 0)
        for (int k = 0; k < 8; ++k) {
            int sx = x + knight[k][0], sy = y + knight[k][1];
            if (!fluid_point(p, sx, sy)) continue;
            map_point(p, &sx, &sy);
            sum += rho[(long)sy * p->nx + sx];
            n += 1;
        }
    if (n == 0) return 0.0;
    return sum / n + p->wet;
}

/* Density of a pressure column at a row whose interior neighbour has density
 * rho_f (see orc_params). */
static double column_density(const orc_params *p, int outlet, double rho_f)
{
    double g = outlet ? p->rho_out_g : p->rho_in_g;
    double l = outlet ? p->rho_out_l : p->rho_in_l;
    double th = 0.0;
    if (p->ph_l > p->ph_g) {
        th = (rho_f - p->ph_g) / (p->ph_l - p->ph_g);
        if (th < 0.0) th = 0.0;
        if (th > 1.0) th = 1.0;
    }
    return g + th * (l - g);
}

/* Density seen by a stencil at lattice point (x, y), which may lie up to two
 * nodes outside the fluid:
 *   - periodic axes wrap;
 *   - walls: a solid row at depth d behind the half-way wall plane takes the
 *     density of the fluid row at depth d in front of it (mirror image), plus
 *     the wetting offset 'wet' (0 gives zero normal gradient: neutral wetting);
 *   - pressure columns carry their boundary density, and points beyond them
 *     take the column's value (clamp). */
static double rho_ghost(const orc_params *p, const double *rho, int x, int y)
{
    int nx = p->nx, ny = p->ny;
    double add = 0.0;
    if (p->mask) {
        int mx = x, my = y;
        if (map_point(p, &mx, &my) && !is_solid(p, mx, my)) return rho[(long)my * nx + mx];
        return mask_ghost(p, rho, x, y);
    }
    if (p->walls) {
        if (y <= 0) { y = 1 - y; add = p->wet; }
        else if (y >= ny - 1) { y = 2 * ny - 3 - y; add = p->wet; }
    } else {
        y = (int)pmod(y, ny);
    }
    if (p->bc_x) {
        if (x < 0) x = 0;           /* the column's own density (set from its */
        if (x > nx - 1) x = nx - 1; /* neighbour's phase) extends beyond it   */
    } else {
        x = (int)pmod(x, nx);
    }
    return rho[(long)y * nx + x] + add;
}

/* Working arrays of one evaluation of the macroscopic fields and the force. */
typedef struct {
    double *rho, *ux, *uy;     /* nx*ny: moments (pressure columns: rho_b, u of x_f) */
    double *Fx, *Fy;           /* nx*ny: total force (non-solid, non-pressure nodes) */
    double *E;                 /* (nx+4)*(ny+4): ghost-extended density */
    double *P;                 /* (nx+4)*(ny+4): phi = k^2 p0 - rho/3 */
    double *L;                 /* (nx+4)*(ny+4): lap(rho), valid one node beyond fluid */
} orc_work;

static int work_alloc(orc_work *w, int nx, int ny)
{
    long n = (long)nx * ny, ne = (long)(nx + 4) * (ny + 4);
    w->rho = calloc(n, sizeof(double));
    w->ux = calloc(n, sizeof(double));
    w->uy = calloc(n, sizeof(double));
    w->Fx = calloc(n, sizeof(double));
    w->Fy = calloc(n, sizeof(double));
    w->E = calloc(ne, sizeof(double));
    w->P = calloc(ne, sizeof(double));
    w->L = calloc(ne, sizeof(double));
    return !(w->rho && w->ux && w->uy && w->Fx && w->Fy && w->E && w->P && w->L);
}

static void work_free(orc_work *w)
{
    free(w->rho); free(w->ux); free(w->uy); free(w->Fx); free(w->Fy);
    free(w->E); free(w->P); free(w->L);
}

/* Passes 1-5 of the step on state f: moments, ghost density, EOS potential,
 * Laplacian and force. */
static void fields_and_force(const orc_params *p, const double *f, orc_work *w)
{
    const int nx = p->nx, ny = p->ny;
    const long n = (long)nx * ny, sx = nx + 4;
    const double k2 = p->k * p->k;
    const orc_eos eos = {p->eos_kind, p->a, p->b, p->R, p->T, p->aalpha};

    /* 1. Moments at every non-solid node (Sec. 2.1). */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            if (is_solid(p, x, y)) { w->rho[c] = 0.0; w->ux[c] = w->uy[c] = 0.0; continue; }
            double r = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < Q; ++i) {
                double fi = f[i * n + c];
                r += fi;
                jx += fi * ex[i];
                jy += fi * ey[i];
            }
            w->rho[c] = r;
            w->ux[c] = jx / r;
            w->uy[c] = jy / r;
        }

    /* Pressure columns: boundary density from the neighbour's phase. */
    if (p->bc_x) {
        for (int y = 0; y < ny; ++y) {
            if (is_solid_row(p, y)) continue;
            w->rho[(long)y * nx] = column_density(p, 0, w->rho[(long)y * nx + 1]);
            w->rho[(long)y * nx + nx - 1] = column_density(p, 1, w->rho[(long)y * nx + nx - 2]);
        }
    }

    /* 2.-3. Ghost-extended density and the EOS potential of Eq. 2.17 read as
     *       F = -grad(k^2 p0 - rho/3) + kappa rho grad(lap rho): k^2 p0 is the
     *       mesh-space EOS of Eq. 2.14 and rho/3 = c_s^2 rho the ideal part P0. */
#pragma omp parallel for schedule(static)
    for (int ye = 0; ye < ny + 4; ++ye)
        for (int xe = 0; xe < nx + 4; ++xe) {
            long c = (long)ye * sx + xe;
            double r = rho_ghost(p, w->rho, xe - 2, ye - 2);
            w->E[c] = r;
            w->P[c] = k2 * orc_eos_p0(&eos, r) - r / 3.0;
        }

    /* 4. Laplacian of the density, on the fluid and one node beyond it. */
#pragma omp parallel for schedule(static)
    for (int ye = 1; ye < ny + 3; ++ye)
        for (int xe = 1; xe < nx + 3; ++xe) {
            long c = (long)ye * sx + xe;
            w->L[c] = lap_ext(w->E, sx, c);
        }

    /* 5. Force at fluid nodes (Eq. 2.17 with the reading above), plus G. */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            long ce = (long)(y + 2) * sx + (x + 2);
            if (is_solid(p, x, y) || is_pressure_col(p, x)) { w->Fx[c] = w->Fy[c] = 0.0; continue; }
            double gpx, gpy, glx, gly;
            grad_ext(w->P, sx, ce, &gpx, &gpy);
            grad_ext(w->L, sx, ce, &glx, &gly);
            double r = w->rho[c];
            w->Fx[c] = -gpx + p->kappa * r * glx + p->gx;
            w->Fy[c] = -gpy + p->kappa * r * gly + p->gy;
        }

    /* Pressure columns carry rho_b; their velocity is that of the interior
     * neighbour x_f, v_f = u_f + F_f / (2 rho_f). */
    if (p->bc_x) {
        for (int y = 0; y < ny; ++y) {
            if (is_solid_row(p, y)) continue;
            for (int side = 0; side < 2; ++side) {
                int xb = side ? nx - 1 : 0, xf = side ? nx - 2 : 1;
                long cb = (long)y * nx + xb, cf = (long)y * nx + xf;
                double rf = w->rho[cf];
                w->ux[cb] = w->ux[cf] + w->Fx[cf] / (2.0 * rf);
                w->uy[cb] = w->uy[cf] + w->Fy[cf] / (2.0 * rf);
            }
        }
    }
}

/* Wall shear (reading: second-order one-sided estimate through v = 0 on the
 * half-way wall plane, v1 and v2 at distances 1/2 and 3/2) and wall pressure
 * (diagonal of the pressure tensor, Eq. 2.4, mesh space: k^2 p0 - kappa rho
 * lap rho - kappa/2 |grad rho|^2), both at the first fluid row of each wall.
 * tw and pw have 2*nx entries: bottom wall then top wall. Pressure columns
 * and channels without walls give zeros. */
static void wall_fields(const orc_params *p, const orc_work *w, double *tw, double *pw)
{
    const int nx = p->nx, ny = p->ny;
    const long sx = nx + 4;
    const double nu = (p->tau - 0.5) / 3.0, k2 = p->k * p->k;
    const orc_eos eos = {p->eos_kind, p->a, p->b, p->R, p->T, p->aalpha};
    for (int side = 0; side < 2; ++side)
        for (int x = 0; x < nx; ++x) {
            tw[side * nx + x] = 0.0;
            pw[side * nx + x] = 0.0;
            if (!p->walls || is_pressure_col(p, x)) continue;
            int y1 = side ? ny - 2 : 1, y2 = side ? ny - 3 : 2;
            if (is_solid(p, x, y1) || is_solid(p, x, y2)) continue; /* wall column covered by an obstacle */
            long c1 = (long)y1 * nx + x, c2 = (long)y2 * nx + x;
            double r1 = w->rho[c1], r2 = w->rho[c2];
            double v1 = w->ux[c1] + w->Fx[c1] / (2.0 * r1);
            double v2 = w->ux[c2] + w->Fx[c2] / (2.0 * r2);
            tw[side * nx + x] = r1 * nu * (9.0 * v1 - v2) / 3.0;
            long ce = (long)(y1 + 2) * sx + (x + 2);
            double grx, gry;
            grad_ext(w->E, sx, ce, &grx, &gry);
            pw[side * nx + x] = k2 * orc_eos_p0(&eos, r1)
                                - p->kappa * r1 * w->L[ce]
                                - 0.5 * p->kappa * (grx * grx + gry * gry);
        }
}

static void diag_of(const orc_params *p, const orc_work *w, orc_diag *d)
{
    const int nx = p->nx, ny = p->ny;
    /* Mass: compensated (Kahan-Babuska) sum over non-solid nodes. */
    double s = 0.0, comp = 0.0;
    for (int y = 0; y < ny; ++y) {
        if (is_solid_row(p, y)) continue;
        for (int x = 0; x < nx; ++x) {
            if (is_solid(p, x, y)) continue;
            double v = w->rho[(long)y * nx + x];
            double t = s + v;
            if (fabs(s) >= fabs(v)) comp += (s - t) + v; else comp += (v - t) + s;
            s = t;
        }
    }
    d->mass = s + comp;
    d->J = 0.0;
    d->Jp = 0.0;
    d->tw_min = d->pw_min = INFINITY;
    d->tw_max = d->pw_max = -INFINITY;
    if (!p->walls) { d->tw_min = d->tw_max = d->pw_min = d->pw_max = 0.0; return; }
    double *tw = malloc(2 * (size_t)nx * sizeof(double));
    double *pw = malloc(2 * (size_t)nx * sizeof(double));
    wall_fields(p, w, tw, pw);
    for (int side = 0; side < 2; ++side)
        for (int x = 0; x < nx; ++x) {
            if (is_pressure_col(p, x)) continue;
            int y1 = side ? ny - 2 : 1, y2 = side ? ny - 3 : 2;
            if (is_solid(p, x, y1) || is_solid(p, x, y2)) continue;
            double t = tw[side * nx + x], q = pw[side * nx + x];
            d->J += t;
            d->Jp += q;
            if (t < d->tw_min) d->tw_min = t;
            if (t > d->tw_max) d->tw_max = t;
            if (q < d->pw_min) d->pw_min = q;
            if (q > d->pw_max) d->pw_max = q;
        }
    free(tw);
    free(pw);
}

/* ------------------------------------------------------------------------- */
/* Public oracle entry points                                                 */
/* ------------------------------------------------------------------------- */

/* f = f_eq(rho0, 0) at every node (solid rows included, so both population
 * arrays start identical everywhere). */
void orc_init(const orc_params *p, const double *rho0, double *f)
{
    const long n = (long)p->nx * p->ny;
    double feq[Q];
    for (long c = 0; c < n; ++c) {
        orc_feq(rho0[c], 0.0, 0.0, feq);
        for (int i = 0; i < Q; ++i) f[i * n + c] = feq[i];
    }
}

/* One time step: fin (post-streaming state n) -> fout (state n+1).
 * Slots that no population reaches keep their value from fin. If d is not
 * NULL it receives the diagnostics of state n. Returns 0, or 1 on allocation
 * failure. */
int orc_step(const orc_params *p, const double *fin, double *fout, orc_diag *d)
{
    const int nx = p->nx, ny = p->ny;
    const long n = (long)nx * ny;
    orc_work w;
    if (work_alloc(&w, nx, ny)) { work_free(&w); return 1; }
    double *fs = malloc((size_t)Q * n * sizeof(double)); /* post-collision f* */
    if (!fs) { work_free(&w); return 1; }

    fields_and_force(p, fin, &w);
    if (d) diag_of(p, &w, d);

    /* 6. Collision with the velocity-shift force (Sec. 2.1): BGK,
     *    u_eq = u + tau F / rho,  f* = f - (f - f_eq(rho, u_eq)) / tau;
     *    or MRT (Eq. 2.1), u_eq = u + F / (s_j rho),
     *    f* = f - M^-1 S M (f - f_eq(rho, u_eq)). */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            if (is_solid(p, x, y) || is_pressure_col(p, x)) continue;
            double r = w.rho[c];
            /* velocity shift: tau F / rho for BGK, F / (s_j rho) for MRT */
            const double shift = p->collision ? 1.0 / p->s_j : p->tau;
            double uex = w.ux[c] + shift * w.Fx[c] / r;
            double uey = w.uy[c] + shift * w.Fy[c] / r;
            double feq[Q];
            orc_feq(r, uex, uey, feq);
            if (p->collision) {
                double fl[Q], fo[Q];
                for (int i = 0; i < Q; ++i) fl[i] = fin[i * n + c];
                mrt_relax(p, fl, feq, fo);
                for (int i = 0; i < Q; ++i) fs[i * n + c] = fo[i];
            } else {
                for (int i = 0; i < Q; ++i) {
                    double fi = fin[i * n + c];
                    fs[i * n + c] = fi - (fi - feq[i]) / p->tau;
                }
            }
        }

    /* 7. Pressure columns (Sec. 2.2 "extrapolated" ends, driven here by a
     *    pressure difference): non-equilibrium extrapolation from the interior
     *    neighbour x_f at the imposed density rho_b,
     *    f*_i(x_b) = f_eq_i(rho_b, v_f) + (1 - 1/tau) (f_i(x_f) - f_eq_i(rho_f, v_f)). */
    if (p->bc_x) {
        for (int y = 0; y < ny; ++y) {
            if (is_solid_row(p, y)) continue;
            for (int side = 0; side < 2; ++side) {
                int xb = side ? nx - 1 : 0, xf = side ? nx - 2 : 1;
                long cb = (long)y * nx + xb, cf = (long)y * nx + xf;
                double vx = w.ux[cb], vy = w.uy[cb]; /* = v_f, set in fields_and_force */
                double fb[Q], ff[Q];
                orc_feq(w.rho[cb], vx, vy, fb);
                orc_feq(w.rho[cf], vx, vy, ff);
                for (int i = 0; i < Q; ++i)
                    fs[i * n + cb] = fb[i] + (1.0 - 1.0 / p->tau) * (fin[i * n + cf] - ff[i]);
            }
        }
    }

    /* 8. Streaming (Eq. 2.1 left-hand side) with half-way bounce-back: a
     *    population whose target is a solid row returns to its own node in
     *    the opposite direction. Populations leaving through a pressure
     *    column's outer edge are dropped. */
    memcpy(fout, fin, (size_t)Q * n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < Q; ++i)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = (long)y * nx + x;
                if (is_solid(p, x, y)) continue;
                int tx = x + ex[i], ty = y + ey[i];
                if (p->walls && (ty == 0 || ty == ny - 1)) {
                    fout[opp[i] * n + c] = fs[i * n + c];
                    continue;
                }
                if (!p->walls) ty = (int)pmod(ty, ny);
                if (p->bc_x) { if (tx < 0 || tx >= nx) continue; }
                else tx = (int)pmod(tx, nx);
                if (p->mask && p->mask[(long)ty * nx + tx]) {
                    /* half-way bounce-back at an obstacle's link */
                    fout[opp[i] * n + c] = fs[i * n + c];
                    continue;
                }
                fout[i * n + (long)ty * nx + tx] = fs[i * n + c];
            }

    free(fs);
    work_free(&w);
    return 0;
}

/* Runs nsteps steps in place on f (scratch: one more population array).
 * acc (may be NULL) receives: mass of the last state read, J summed over the
 * states read (steps 0..nsteps-1), extrema over all of them. */
int orc_run(const orc_params *p, double *f, long nsteps, orc_diag *acc)
{
    const long n = (long)p->nx * p->ny;
    double *g = malloc((size_t)Q * n * sizeof(double));
    if (!g) return 1;
    orc_diag tot = {0.0, 0.0, INFINITY, -INFINITY, INFINITY, -INFINITY, 0.0};
    double *a = f, *b = g;
    for (long s = 0; s < nsteps; ++s) {
        orc_diag d;
        if (orc_step(p, a, b, &d)) { free(g); return 1; }
        tot.mass = d.mass;
        tot.J += d.J;
        tot.Jp += d.Jp;
        if (d.tw_min < tot.tw_min) tot.tw_min = d.tw_min;
        if (d.tw_max > tot.tw_max) tot.tw_max = d.tw_max;
        if (d.pw_min < tot.pw_min) tot.pw_min = d.pw_min;
        if (d.pw_max > tot.pw_max) tot.pw_max = d.pw_max;
        double *t = a; a = b; b = t;
    }
    if (a != f) memcpy(f, a, (size_t)Q * n * sizeof(double));
    free(g);
    if (acc) *acc = tot;
    return 0;
}

/* Macroscopic fields of state f: rho, v = u + F/(2 rho) (Sec. 2.1), wall shear
 * and wall pressure (2*nx each: bottom then top). Any output may be NULL.
 * Solid nodes report zeros. */
int orc_fields(const orc_params *p, const double *f, double *rho, double *vx, double *vy,
               double *tw, double *pw)
{
    const int nx = p->nx, ny = p->ny;
    const long n = (long)nx * ny;
    orc_work w;
    if (work_alloc(&w, nx, ny)) { work_free(&w); return 1; }
    fields_and_force(p, f, &w);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            double r = w.rho[c], X = 0.0, Y = 0.0;
            if (is_solid(p, x, y)) r = 0.0;
            else if (is_pressure_col(p, x)) { X = w.ux[c]; Y = w.uy[c]; }
            else { X = w.ux[c] + w.Fx[c] / (2.0 * r); Y = w.uy[c] + w.Fy[c] / (2.0 * r); }
            if (rho) rho[c] = r;
            if (vx) vx[c] = X;
            if (vy) vy[c] = Y;
        }
    if (tw || pw) {
        double *t = malloc(2 * (size_t)nx * sizeof(double));
        double *q = malloc(2 * (size_t)nx * sizeof(double));
        wall_fields(p, &w, t, q);
        if (tw) memcpy(tw, t, 2 * (size_t)nx * sizeof(double));
        if (pw) memcpy(pw, q, 2 * (size_t)nx * sizeof(double));
        free(t);
        free(q);
    }
    (void)n;
    work_free(&w);
    return 0;
}

/* Force field alone (for pins): Fx, Fy of state f (zero at solid and pressure nodes). */
int orc_force(const orc_params *p, const double *f, double *Fx, double *Fy)
{
    const long n = (long)p->nx * p->ny;
    orc_work w;
    if (work_alloc(&w, p->nx, p->ny)) { work_free(&w); return 1; }
    fields_and_force(p, f, &w);
    memcpy(Fx, w.Fx, n * sizeof(double));
    memcpy(Fy, w.Fy, n * sizeof(double));
    work_free(&w);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops (n >= 1); for timing the oracle on one core. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
