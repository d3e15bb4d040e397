// Host-side FP64 helpers of the solver: thermodynamics of the Carnahan-Starling
// and Peng-Robinson equations of state (critical point, Maxwell coexistence,
// branch densities for a given pressure), the initial density profiles of the
// airway channel and the static droplet, and the liquid-plug analysis. No GPU
// is needed for anything in this file.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {

// Carnahan-Starling pressure p0(rho) = rho R T Z(eta) - a rho^2, eta = b rho/4.
static double cs_pressure(const Thermo &t, double rho)
{
    double eta = 0.25 * t.b * rho, om = 1.0 - eta;
    return rho * t.R * t.T * (1.0 + eta * (1.0 + eta * (1.0 - eta))) / (om * om * om) - t.a * rho * rho;
}

// (eta Z)' and (eta Z)'' with respect to eta.
static double g1(double e)
{
    double om = 1.0 - e;
    return (1.0 + e * (4.0 + e * (4.0 + e * (-4.0 + e)))) / (om * om * om * om);
}
static double g2(double e)
{
    double om = 1.0 - e, om2 = om * om;
    return (8.0 + e * (20.0 - 4.0 * e)) / (om2 * om2 * om);
}
static double g3(double e)
{
    double om = 1.0 - e, om3 = om * om * om;
    return (60.0 + e * (72.0 - 12.0 * e)) / (om3 * om3);
}

// Peng-Robinson pieces: x = b rho, D = 1 + 2x - x^2.
static double pr_D(double x) { return 1.0 + x * (2.0 - x); }

double eos_pressure(const Thermo &t, double rho)
{
    if (t.kind == 0) return cs_pressure(t, rho);
    const double x = t.b * rho;
    return rho * t.R * t.T / (1.0 - x) - t.aalpha * rho * rho / pr_D(x);
}

double eos_dpressure(const Thermo &t, double rho)
{
    if (t.kind == 0) return t.R * t.T * g1(0.25 * t.b * rho) - 2.0 * t.a * rho;
    const double x = t.b * rho, om = 1.0 - x, D = pr_D(x);
    return t.R * t.T / (om * om) - 2.0 * t.aalpha * rho * (1.0 + x) / (D * D);
}

// Chemical potential mu = psi'(rho) (free energy density psi with p0 = rho psi' - psi).
static double eos_mu(const Thermo &t, double rho)
{
    if (t.kind == 0) {
        double eta = 0.25 * t.b * rho, om = 1.0 - eta;
        return t.R * t.T * (std::log(rho) + eta * (8.0 + eta * (-9.0 + 3.0 * eta)) / (om * om * om))
               - 2.0 * t.a * rho;
    }
    // PR: specific free energy int p0/rho^2 drho plus p0/rho
    const double x = t.b * rho, s2 = std::sqrt(2.0);
    const double fe = t.R * t.T * std::log(rho / (1.0 - x))
                      + t.aalpha / (2.0 * s2 * t.b) * std::log((1.0 + s2 - x) / (s2 - 1.0 + x));
    return fe + eos_pressure(t, rho) / rho;
}

// Critical packing fraction: h(eta) = g1 - eta g2 = 0, with h' = -eta g3 (since g1' = g2).
static double critical_eta()
{
    double e = 0.13;
    for (int it = 0; it < 60; ++it) {
        double h = g1(e) - e * g2(e);
        double d = -e * g3(e);
        double step = h / d;
        e -= step;
        if (std::fabs(step) < 1e-17) break;
    }
    return e;
}

// PR: along dp0/drho = 0 the reduced attraction A = a / (b R T) is
// D^2 / (2 x (1 + x)(1 - x)^2); the critical point is its minimum over x
// (below Tc two spinodals share one A). Golden-section search.
static double pr_A(double x)
{
    const double D = pr_D(x), om = 1.0 - x;
    return D * D / (2.0 * x * (1.0 + x) * om * om);
}

void eos_critical(int kind, double a, double b, double R, double *Tc, double *rhoc)
{
    if (kind == 0) {
        double e = critical_eta();
        *rhoc = 4.0 * e / b;
        *Tc = 8.0 * a / (b * R * g2(e));
        return;
    }
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    double lo = 0.05, hi = 0.6;
    double c = hi - gr * (hi - lo), d = lo + gr * (hi - lo);
    for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
        if (pr_A(c) < pr_A(d)) hi = d; else lo = c;
        c = hi - gr * (hi - lo);
        d = lo + gr * (hi - lo);
    }
    const double x = 0.5 * (lo + hi);
    *rhoc = x / b;
    *Tc = a / (b * R * pr_A(x));
}

double pr_alpha(double omega, double T_over_Tc)
{
    const double m = 0.37464 + omega * (1.54226 - 0.26992 * omega);
    const double s = 1.0 + m * (1.0 - std::sqrt(T_over_Tc));
    return s * s;
}

static double rho_max(const Thermo &t) { return (t.kind == 0 ? 4.0 : 1.0) / t.b * (1.0 - 1e-12); }

// Safeguarded Newton for p0(rho) = p on a bracket [lo, hi] where p0 increases.
static double solve_branch(const Thermo &t, double p, double lo, double hi)
{
    double r = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double f = eos_pressure(t, r) - p;
        if (f > 0.0) hi = r; else lo = r;
        double d = eos_dpressure(t, r);
        double rn = (d > 0.0) ? r - f / d : 0.5 * (lo + hi);
        if (!(rn > lo && rn < hi)) rn = 0.5 * (lo + hi);
        if (std::fabs(rn - r) <= 1e-16 * r) { r = rn; break; }
        r = rn;
    }
    return r;
}

// Root of dp0/drho between lo and hi (sign change), by bisection on the sign.
static double spinodal(const Thermo &t, double lo, double hi)
{
    bool slo = eos_dpressure(t, lo) > 0.0;
    for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (lo + hi);
        if ((eos_dpressure(t, m) > 0.0) == slo) lo = m; else hi = m;
    }
    return 0.5 * (lo + hi);
}

// Spinodals s1 < s2 below Tc; nonzero at or above Tc.
static int spinodals(const Thermo &t, double *s1, double *s2)
{
    double Tc, rhoc;
    eos_critical(t.kind, t.a, t.b, t.R, &Tc, &rhoc);
    if (!(t.T < Tc)) return 1;
    *s1 = spinodal(t, 1e-12, rhoc);
    *s2 = spinodal(t, rhoc, rho_max(t));
    return 0;
}

int maxwell(const Thermo &t, double *rho_g, double *rho_l, double *p_sat)
{
    double s1, s2;
    if (spinodals(t, &s1, &s2)) return 1;
    const double rmax = rho_max(t);
    double plo = std::fmax(eos_pressure(t, s2), 0.0), phi = eos_pressure(t, s1);
    // Newton in pressure on dmu(p) = mu(rho_g(p)) - mu(rho_l(p)); by Gibbs-Duhem
    // d dmu / dp = 1/rho_g - 1/rho_l. Bracket kept to stay on both branches.
    double lo = plo, hi = phi, p = 0.5 * (plo + phi), rg = 0, rl = 0;
    for (int it = 0; it < 200; ++it) {
        rg = solve_branch(t, p, 1e-300, s1);
        rl = solve_branch(t, p, s2, rmax);
        double dmu = eos_mu(t, rg) - eos_mu(t, rl);
        if (dmu > 0.0) hi = p; else lo = p;
        double pn = p - dmu / (1.0 / rg - 1.0 / rl);
        if (!(pn > lo && pn < hi)) pn = 0.5 * (lo + hi);
        if (std::fabs(pn - p) <= 1e-17 * p) { p = pn; break; }
        p = pn;
    }
    *p_sat = p;
    *rho_g = solve_branch(t, p, 1e-300, s1);
    *rho_l = solve_branch(t, p, s2, rmax);
    return 0;
}

int gas_density(const Thermo &t, double p, double *rho, bool *saturated)
{
    if (saturated) *saturated = false;
    if (!(p > 0.0)) return 1;
    double s1, s2;
    if (spinodals(t, &s1, &s2)) {  // monotone EOS
        const double hi = rho_max(t);
        if (!(p < eos_pressure(t, hi))) return 1;
        *rho = solve_branch(t, p, 1e-300, hi);
        return 0;
    }
    if (!(p < eos_pressure(t, s1))) {  // beyond the gas branch's end
        *rho = s1;
        if (saturated) *saturated = true;
        return 0;
    }
    *rho = solve_branch(t, p, 1e-300, s1);
    return 0;
}

int liquid_density(const Thermo &t, double p, double *rho, bool *saturated)
{
    if (saturated) *saturated = false;
    double s1, s2;
    if (spinodals(t, &s1, &s2)) return 1;
    if (!(p > eos_pressure(t, s2))) {  // below the liquid branch's end
        *rho = s2;
        if (saturated) *saturated = true;
        return 0;
    }
    *rho = solve_branch(t, p, s2, rho_max(t));
    return 0;
}

int thermo_of(const lbm_eos &e, Thermo *t, double *Tc)
{
    if (!(e.a > 0) || !(e.b > 0) || !(e.R > 0) || !(e.T_over_Tc > 0)) return 1;
    if (e.kind != 0 && e.kind != 1) return 1;
    double tc, rc;
    eos_critical(e.kind, e.a, e.b, e.R, &tc, &rc);
    *t = Thermo{e.a, e.b, e.R, e.T_over_Tc * tc, e.kind, e.kind == 1 ? e.a * pr_alpha(e.omega, e.T_over_Tc) : 0.0};
    if (Tc) *Tc = tc;
    return 0;
}

int channel_thermo(const lbm_eos &e, const lbm_drive &d, bool bc_x, ChannelThermo *out)
{
    ChannelThermo c;
    if (thermo_of(e, &c.th, &c.Tc)) return 1;
    c.T = c.th.T;
    const bool coexist = maxwell(c.th, &c.rho_g, &c.rho_l, &c.p_sat) == 0;
    if (!coexist) c.rho_g = c.rho_l = c.p_sat = 0.0;
    if (bc_x) {
        const double k2 = e.k * e.k;
        double pref = d.p_ref;
        if (std::isnan(pref)) {
            if (!coexist) return 1;
            pref = k2 * c.p_sat;
        }
        const double pin = (pref + 0.5 * d.dp) / k2, pout = (pref - 0.5 * d.dp) / k2;
        if (gas_density(c.th, pin, &c.rho_in, &c.sat[0]) || gas_density(c.th, pout, &c.rho_out, &c.sat[2]))
            return 1;
        if (coexist) {
            if (liquid_density(c.th, pin, &c.rho_in_l, &c.sat[1]) ||
                liquid_density(c.th, pout, &c.rho_out_l, &c.sat[3]))
                return 1;
        } else {
            c.rho_in_l = c.rho_in;
            c.rho_out_l = c.rho_out;
            c.sat[1] = c.sat[0];
            c.sat[3] = c.sat[2];
        }
    }
    *out = c;
    return 0;
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based hash.
static inline uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double node_noise(uint64_t seed, uint64_t node, double amp)
{
    double u = (double)(splitmix64(seed ^ node) >> 11) * (1.0 / 9007199254740992.0);
    return amp * (2.0 * u - 1.0);
}

} // namespace lbm

extern "C" {

lbm_status lbm_coexistence(const lbm_eos *eos, double *Tc, double *rho_g, double *rho_l,
                           double *p_sat)
{
    lbm::Thermo t{};
    double tc;
    if (!eos || lbm::thermo_of(*eos, &t, &tc)) return LBM_ERR_ARG;
    double g, l, p;
    if (lbm::maxwell(t, &g, &l, &p)) return LBM_ERR_PARAM;
    if (Tc) *Tc = tc;
    if (rho_g) *rho_g = g;
    if (rho_l) *rho_l = l;
    if (p_sat) *p_sat = p;
    return LBM_OK;
}

lbm_status lbm_airway_rho0(int32_t nx, int32_t ny, double film, double plug_x, double plug_len,
                           double rho_l, double rho_g, double width, double noise_amp,
                           uint64_t seed, double *out)
{
    if (nx <= 0 || ny <= 0 || !out || !(width > 0)) return LBM_ERR_ARG;
    for (int32_t y = 0; y < ny; ++y)
        for (int32_t x = 0; x < nx; ++x) {
            double d_wall = std::fmin(y - 0.5, (ny - 1.5) - y);
            double s_film = 0.5 * (1.0 - std::tanh(2.0 * (d_wall - film) / width));
            double s_plug = 0.5 * (std::tanh(2.0 * (x - plug_x) / width)
                                   - std::tanh(2.0 * (x - plug_x - plug_len) / width));
            double s = std::fmax(s_film, s_plug);
            uint64_t node = (uint64_t)y * (uint64_t)nx + (uint64_t)x;
            double v = rho_g + (rho_l - rho_g) * s;
            if (noise_amp != 0.0) v += lbm::node_noise(seed, node, noise_amp);
            out[node] = v;
        }
    return LBM_OK;
}

lbm_status lbm_airway_rho0_tangent(int32_t nx, int32_t ny, double film, double plug_x, double plug_len,
                                   double rho_l, double rho_g, double width, double *d_film, double *d_plug)
{
    if (nx <= 0 || ny <= 0 || !(width > 0)) return LBM_ERR_ARG;
    for (int32_t y = 0; y < ny; ++y)
        for (int32_t x = 0; x < nx; ++x) {
            double d_wall = std::fmin(y - 0.5, (ny - 1.5) - y);
            double af = 2.0 * (d_wall - film) / width;
            double a0 = 2.0 * (x - plug_x) / width, a1 = 2.0 * (x - plug_x - plug_len) / width;
            double s_film = 0.5 * (1.0 - std::tanh(af));
            double s_plug = 0.5 * (std::tanh(a0) - std::tanh(a1));
            // d/dh of 0.5 (1 - tanh(2 (d - h) / W)) = sech^2(.) / W; likewise for L
            double cf = std::cosh(af), cp = std::cosh(a1);
            double df = 0.0, dl = 0.0;
            if (s_film >= s_plug) df = 1.0 / (width * cf * cf);
            else dl = 1.0 / (width * cp * cp);
            size_t node = (size_t)y * nx + x;
            if (d_film) d_film[node] = (rho_l - rho_g) * df;
            if (d_plug) d_plug[node] = (rho_l - rho_g) * dl;
        }
    return LBM_OK;
}

lbm_status lbm_disk_rho0(int32_t nx, int32_t ny, double cx, double cy, double r0, double rho_l,
                         double rho_g, double width, double noise_amp, uint64_t seed, double *out)
{
    if (nx <= 0 || ny <= 0 || !out || !(width > 0)) return LBM_ERR_ARG;
    for (int32_t y = 0; y < ny; ++y)
        for (int32_t x = 0; x < nx; ++x) {
            double r = std::sqrt((x - cx) * (x - cx) + (y - cy) * (y - cy));
            double s = 0.5 * (1.0 - std::tanh(2.0 * (r - r0) / width));
            uint64_t node = (uint64_t)y * (uint64_t)nx + (uint64_t)x;
            double v = rho_g + (rho_l - rho_g) * s;
            if (noise_amp != 0.0) v += lbm::node_noise(seed, node, noise_amp);
            out[node] = v;
        }
    return LBM_OK;
}

} // extern "C"

extern "C" lbm_status lbm_plug_analysis(int32_t nx, int32_t ny, const double *rho, double rho_mid,
                                        lbm_plug_state *out)
{
    if (nx <= 0 || ny < 4 || !rho || !out || !std::isfinite(rho_mid)) return LBM_ERR_ARG;
    const int y0 = 1, y1 = ny - 2;  // fluid rows
    auto liquid = [&](int x, int y) { return rho[(size_t)y * nx + x] > rho_mid; };

    // plug ends on the centre row: the longest run of liquid nodes
    const int yc = ny / 2;
    int best_a = -1, best_b = -1;
    for (int x = 0; x < nx;) {
        if (!liquid(x, yc)) { ++x; continue; }
        int e = x;
        while (e + 1 < nx && liquid(e + 1, yc)) ++e;
        if (e - x > best_b - best_a) { best_a = x; best_b = e; }
        x = e + 1;
    }
    out->x_rear = out->x_front = NAN;
    if (best_a >= 0) {
        const double *r = rho + (size_t)yc * nx;
        // crossing of rho_mid between the outer gas node and the liquid end node
        out->x_rear = best_a > 0 ? (best_a - 1) + (rho_mid - r[best_a - 1]) / (r[best_a] - r[best_a - 1])
                                 : (double)best_a;
        out->x_front = best_b < nx - 1 ? best_b + (r[best_b] - rho_mid) / (r[best_b] - r[best_b + 1])
                                       : (double)best_b;
    }

    // intact: some column liquid on every fluid row
    out->intact = 0;
    for (int x = 0; x < nx && !out->intact; ++x) {
        bool full = true;
        for (int y = y0; y <= y1 && full; ++y) full = liquid(x, y);
        if (full) out->intact = 1;
    }

    // 4-connected liquid components (iterative flood fill), classified by wall contact
    std::vector<int32_t> label((size_t)nx * ny, -1);
    std::vector<int32_t> stack;
    out->n_droplets = 0;
    out->droplet_mass = 0.0;
    out->wall_liquid_mass = 0.0;
    int32_t next = 0;
    for (int y = y0; y <= y1; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t c0 = (size_t)y * nx + x;
            if (label[c0] >= 0 || !liquid(x, y)) continue;
            bool wall = false;
            double m = 0.0;
            stack.clear();
            stack.push_back((int32_t)c0);
            label[c0] = next;
            while (!stack.empty()) {
                const size_t c = (size_t)stack.back();
                stack.pop_back();
                const int cx = (int)(c % nx), cy = (int)(c / nx);
                m += rho[c];
                if (cy == y0 || cy == y1) wall = true;
                const int nbx[4] = {cx - 1, cx + 1, cx, cx}, nby[4] = {cy, cy, cy - 1, cy + 1};
                for (int k = 0; k < 4; ++k) {
                    if (nbx[k] < 0 || nbx[k] >= nx || nby[k] < y0 || nby[k] > y1) continue;
                    const size_t d = (size_t)nby[k] * nx + nbx[k];
                    if (label[d] < 0 && liquid(nbx[k], nby[k])) {
                        label[d] = next;
                        stack.push_back((int32_t)d);
                    }
                }
            }
            ++next;
            if (wall) out->wall_liquid_mass += m;
            else {
                out->n_droplets += 1;
                out->droplet_mass += m;
            }
        }
    return LBM_OK;
}
