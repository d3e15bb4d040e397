// Discrete adjoint of the fused step (FP64) with checkpoint-and-recompute.
//
// Objectives (Sec. 3, Figs. 10-12: time-integrated wall loads) over the states
// n = 0 .. N-1 that N steps read:
//   J_tau = sum_n sum_x (tau_w,bottom + tau_w,top),
//   J_p   = sum_n sum_x (p_w,bottom + p_w,top),
// at interior columns, tau_w = rho_1 nu (9 v_1 - v_2) / 3 and
// p_w = k^2 p0(rho_1) - kappa rho_1 lap(rho) - (kappa/2)|grad rho|^2 (Eq. 2.4).
// The adjoint recursion is lambda^N = 0,
//   lambda^n = (d f^{n+1} / d f^n)^T lambda^{n+1} + (d J_n / d f^n)^T,
// the exact transpose of the linearised step that lbm_step takes: moments,
// ghost densities, EOS potential, Laplacian, force (Eq. 2.17), velocity-shift
// BGK or MRT collision, pressure columns, bounce-back streaming. Where the pressure
// column's phase weight is clamped its derivative is taken as zero (the
// derivative almost everywhere). Gradients:
//   dJ/drho0(x) = sum_i w_i lambda^0_i(x)          (f^0 = f_eq(rho0, 0)),
//   dJ/d(dp)    through the column densities, d rho_root / d p = 1 / (k^2 p0'),
//   dJ/dG       = sum_n sum_x Fbar(x)              (body force in F).
//
// One reverse step is seven gather-only kernels (no atomics, so results do
// not depend on scheduling); the forward states of each block of K steps are
// recomputed from a checkpoint by the FP64 forward context and kept in HBM.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace {

using lbm::ex_;
using lbm::ey_;
using lbm::opp_;

__device__ __forceinline__ double wq(int i) { return lbm::w_<double>(i); }

struct AdjGeo {
    int nx, ny, walls, bc_x;
    int fp;                       // plane pitch of a stored state: rows of nine planes, f[(y * 9 + i) * fp + x]
    int eos_kind;                 // 0 Carnahan-Starling, 1 Peng-Robinson
    double RT, a, b4, k2, kappa, tau, nu, wet, gx, gy;
    double bpr, aalpha;           // PR: b and a alpha(T)
    double g_in, l_in, g_out, l_out, ph_g, inv_dph;  // inv_dph = 0: single phase, no blend
    double w_tau, w_p;
    // collision: BGK (mrt = 0) or MRT with rates over the squared row norms of
    // the moment basis (mrate[k] = s_k / |M_k|^2); the equilibrium velocity is
    // u + ushift F / rho with ushift = tau (BGK) or 1 / s_j (MRT)
    int mrt;
    double ushift, mrate[9];
};

// Lallemand-Luo moment basis (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy)
// over the D2Q9 velocities.
__device__ __constant__ const int Mrow[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},      {-4, -1, -1, -1, -1, 2, 2, 2, 2}, {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},   {0, -2, 0, 2, 0, 1, -1, -1, 1},   {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},   {0, 1, -1, 1, -1, 0, 0, 0, 0},    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

// v -> K v with K = M^-1 S M = M^T diag(s_k / |M_k|^2) M. K is symmetric, so
// the same map transposes the MRT relaxation f* = f - K (f - f_eq).
__device__ __forceinline__ void mrt_apply(const AdjGeo &g, const double (&v)[9], double (&out)[9])
{
    double m[9];
    for (int k = 0; k < 9; ++k) {
        double t = 0.0;
        for (int i = 0; i < 9; ++i) t += Mrow[k][i] * v[i];
        m[k] = t * g.mrate[k];
    }
    for (int i = 0; i < 9; ++i) {
        double t = 0.0;
        for (int k = 0; k < 9; ++k) t += Mrow[k][i] * m[k];
        out[i] = t;
    }
}

__device__ __forceinline__ bool solid_row(const AdjGeo &g, int y) { return g.walls && (y == 0 || y == g.ny - 1); }
__device__ __forceinline__ bool pcol(const AdjGeo &g, int x) { return g.bc_x && (x == 0 || x == g.nx - 1); }
__device__ __forceinline__ int pmod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// EOS p0 and dp0/drho: Carnahan-Starling (eta = b rho / 4) or Peng-Robinson
// (x = b rho, D = 1 + 2x - x^2).
__device__ __forceinline__ double cs_p0(const AdjGeo &g, double r)
{
    if (g.eos_kind == 1) {
        const double x = g.bpr * r;
        return r * g.RT / (1.0 - x) - g.aalpha * r * r / (1.0 + x * (2.0 - x));
    }
    const double eta = g.b4 * r, om = 1.0 - eta;
    return r * g.RT * (1.0 + eta * (1.0 + eta * (1.0 - eta))) / (om * om * om) - g.a * r * r;
}
__device__ __forceinline__ double cs_dp0(const AdjGeo &g, double r)
{
    if (g.eos_kind == 1) {
        const double x = g.bpr * r, om = 1.0 - x, D = 1.0 + x * (2.0 - x);
        return g.RT / (om * om) - 2.0 * g.aalpha * r * (1.0 + x) / (D * D);
    }
    const double eta = g.b4 * r, om = 1.0 - eta, om2 = om * om;
    return g.RT * (1.0 + eta * (4.0 + eta * (4.0 + eta * (-4.0 + eta)))) / (om2 * om2) - 2.0 * g.a * r;
}
__device__ __forceinline__ double phi_of(const AdjGeo &g, double r) { return g.k2 * cs_p0(g, r) - r / 3.0; }

__device__ __forceinline__ int map_y(const AdjGeo &g, int y)
{
    if (g.walls) return y <= 0 ? 1 - y : (y >= g.ny - 1 ? 2 * g.ny - 3 - y : y);
    return pmod(y, g.ny);
}
__device__ __forceinline__ int map_x(const AdjGeo &g, int x)
{
    if (g.bc_x) return x < 0 ? 0 : (x > g.nx - 1 ? g.nx - 1 : x);
    return pmod(x, g.nx);
}
// Density seen by a stencil at (x, y), up to two nodes outside the lattice:
// mirror images behind walls (plus the wetting offset), clamp beyond pressure
// columns, wrap on periodic axes.
__device__ __forceinline__ double ghost_rho(const AdjGeo &g, const double *rho, int x, int y)
{
    const bool beyond = g.walls && (y <= 0 || y >= g.ny - 1);
    return rho[map_y(g, y) * g.nx + map_x(g, x)] + (beyond ? g.wet : 0.0);
}

// Ring-1 (fluid plus one node) and ring-2 extended grids.
__device__ __forceinline__ int ri1(const AdjGeo &g, int x, int y) { return (y + 1) * (g.nx + 2) + (x + 1); }
__device__ __forceinline__ bool in_r1(const AdjGeo &g, int x, int y)
{
    return x >= -1 && x <= g.nx && y >= -1 && y <= g.ny;
}
__device__ __forceinline__ bool in_lat(const AdjGeo &g, int x, int y)
{
    return x >= 0 && x < g.nx && y >= 0 && y < g.ny;
}

// Phase weight of a pressure column whose neighbour has density rf, and its
// derivative (zero where clamped).
__device__ __forceinline__ double col_theta(const AdjGeo &g, double rf, double &dth)
{
    dth = 0.0;
    if (!(g.inv_dph > 0.0)) return 0.0;
    double th = (rf - g.ph_g) * g.inv_dph;
    if (th < 0.0) return 0.0;
    if (th > 1.0) return 1.0;
    if (th > 0.0 && th < 1.0) dth = g.inv_dph;
    return th;
}

// ---- forward recompute of the fields of one state ---------------------------

// S: the stored state's type (double, or float for an FP32 forward; widened here)
template <typename S>
__global__ void adj_moments(AdjGeo g, const S *__restrict__ f, double *rho, double *jx, double *jy)
{
    const int n = g.nx * g.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int x = c % g.nx, y = c / g.nx;
    if (solid_row(g, y)) { rho[c] = jx[c] = jy[c] = 0.0; return; }
    const S *fr = f + (size_t)y * 9 * g.fp;  // row y of the state
    if (pcol(g, x)) {
        const int xf = x == 0 ? 1 : g.nx - 2;
        double rf = 0.0;
        for (int i = 0; i < 9; ++i) rf += (double)fr[i * g.fp + xf];
        double dth;
        const double th = col_theta(g, rf, dth);
        const double gg = x == 0 ? g.g_in : g.g_out, ll = x == 0 ? g.l_in : g.l_out;
        rho[c] = gg + th * (ll - gg);
        jx[c] = jy[c] = 0.0;
        return;
    }
    double r = 0.0, X = 0.0, Y = 0.0;
    for (int i = 0; i < 9; ++i) {
        const double fi = (double)fr[i * g.fp + x];
        r += fi;
        X += ex_(i) * fi;
        Y += ey_(i) * fi;
    }
    rho[c] = r;
    jx[c] = X;
    jy[c] = Y;
}

// lap(rho) = 6 sum_i w_i (rho(x + e_i) - rho(x)) on the ring-1 grid.
__global__ void adj_lap(AdjGeo g, const double *__restrict__ rho, double *L1)
{
    const int w = g.nx + 2, m = w * (g.ny + 2);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int x = t % w - 1, y = t / w - 1;
    const double e0 = ghost_rho(g, rho, x, y);
    double s = 0.0;
    for (int i = 1; i < 9; ++i) s += 6.0 * wq(i) * (ghost_rho(g, rho, x + ex_(i), y + ey_(i)) - e0);
    L1[t] = s;
}

// F = -grad phi + kappa rho grad L + G at fluid nodes (grad = 3 sum_i w_i e_i).
__global__ void adj_force(AdjGeo g, const double *__restrict__ rho, const double *__restrict__ L1, double *Fx,
                          double *Fy)
{
    const int n = g.nx * g.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int x = c % g.nx, y = c / g.nx;
    if (solid_row(g, y) || pcol(g, x)) { Fx[c] = Fy[c] = 0.0; return; }
    double gpx = 0, gpy = 0, glx = 0, gly = 0;
    for (int i = 1; i < 9; ++i) {
        const int qx = x + ex_(i), qy = y + ey_(i);
        const double p = phi_of(g, ghost_rho(g, rho, qx, qy)), l = L1[ri1(g, qx, qy)];
        gpx += 3.0 * wq(i) * ex_(i) * p;
        gpy += 3.0 * wq(i) * ey_(i) * p;
        glx += 3.0 * wq(i) * ex_(i) * l;
        gly += 3.0 * wq(i) * ey_(i) * l;
    }
    Fx[c] = -gpx + g.kappa * rho[c] * glx + g.gx;
    Fy[c] = -gpy + g.kappa * rho[c] * gly + g.gy;
}

__device__ __forceinline__ void grad_rho(const AdjGeo &g, const double *rho, int x, int y, double &gx, double &gy)
{
    gx = gy = 0.0;
    for (int i = 1; i < 9; ++i) {
        const double e = ghost_rho(g, rho, x + ex_(i), y + ey_(i));
        gx += 3.0 * wq(i) * ex_(i) * e;
        gy += 3.0 * wq(i) * ey_(i) * e;
    }
}

// Wall shear and wall pressure per (side, column): 2 nx entries each.
__global__ void adj_wall_terms(AdjGeo g, const double *__restrict__ rho, const double *__restrict__ jx,
                               const double *__restrict__ Fx, const double *__restrict__ L1, double *tw,
                               double *pw)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * g.nx) return;
    const int side = t / g.nx, x = t % g.nx;
    tw[t] = pw[t] = 0.0;
    if (!g.walls || pcol(g, x)) return;
    const int y1 = side ? g.ny - 2 : 1, y2 = side ? g.ny - 3 : 2;
    const int c1 = y1 * g.nx + x, c2 = y2 * g.nx + x;
    const double r1 = rho[c1], r2 = rho[c2];
    const double m1 = jx[c1] + 0.5 * Fx[c1], v2 = (jx[c2] + 0.5 * Fx[c2]) / r2;
    tw[t] = g.nu * (9.0 * m1 - r1 * v2) / 3.0;
    double grx, gry;
    grad_rho(g, rho, x, y1, grx, gry);
    pw[t] = g.k2 * cs_p0(g, r1) - g.kappa * r1 * L1[ri1(g, x, y1)] - 0.5 * g.kappa * (grx * grx + gry * gry);
}

// ---- reverse step ---------------------------------------------------------

// Local part of the reverse step at every lattice node: reverse streaming,
// reverse collision, the pressure column fed by this node, and the wall
// objective terms of this node. Outputs Fbar (A), jbar, the local rho-bar (R;
// a column's own entry is written by its interior neighbour), the objective
// sources of Lbar and Ebar (Ls, Cx, Cy) and (1 - 1/tau) f*-bar into lam_out.
__global__ void adj_local(AdjGeo g, const double *__restrict__ lam_in,
                          const double *__restrict__ rho, const double *__restrict__ jx,
                          const double *__restrict__ jy, const double *__restrict__ Fx,
                          const double *__restrict__ Fy, const double *__restrict__ L1, double *lam_out,
                          double *Ax, double *Ay, double *Jbx, double *Jby, double *R, double *Ls, double *Cx,
                          double *Cy)
{
    const int n = g.nx * g.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int x = c % g.nx, y = c / g.nx;
    Ls[c] = Cx[c] = Cy[c] = 0.0;
    Ax[c] = Ay[c] = Jbx[c] = Jby[c] = 0.0;
    if (solid_row(g, y) || pcol(g, x)) {
        if (solid_row(g, y)) R[c] = 0.0;
        for (int i = 0; i < 9; ++i) lam_out[i * n + c] = 0.0;
        return;
    }
    const double omt = 1.0 - 1.0 / g.tau;
    const double r = rho[c], jX = jx[c], jY = jy[c], FX = Fx[c], FY = Fy[c];

    // reverse streaming: f*_i(x) went to x + e_i, or back to x as opp(i)
    double gb[9];
    for (int i = 0; i < 9; ++i) {
        int tx = x + ex_(i), ty = y + ey_(i);
        if (g.walls && (ty == 0 || ty == g.ny - 1)) { gb[i] = lam_in[opp_(i) * n + c]; continue; }
        if (!g.walls) ty = pmod(ty, g.ny);
        if (!g.bc_x) tx = pmod(tx, g.nx);
        gb[i] = lam_in[i * n + ty * g.nx + tx];
    }

    // collision f* = f - K (f - f_eq(rho, u_eq)), u_eq = (j + ushift F) / rho,
    // K = I / tau (BGK) or M^-1 S M (MRT): f-bar = g - K g, f_eq-bar = K g
    double lam[9], kg[9];
    if (g.mrt) {
        mrt_apply(g, gb, kg);
    } else {
        for (int i = 0; i < 9; ++i) kg[i] = gb[i] / g.tau;
    }
    const double uex = (jX + g.ushift * FX) / r, uey = (jY + g.ushift * FY) / r;
    const double usq = uex * uex + uey * uey;
    double rb = 0.0, ubx = 0.0, uby = 0.0;
    for (int i = 0; i < 9; ++i) {
        lam[i] = gb[i] - kg[i];
        const double eb = kg[i];
        const double eu = ex_(i) * uex + ey_(i) * uey;
        rb += eb * wq(i) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
        ubx += eb * wq(i) * r * (3.0 * ex_(i) + 9.0 * eu * ex_(i) - 3.0 * uex);
        uby += eb * wq(i) * r * (3.0 * ey_(i) + 9.0 * eu * ey_(i) - 3.0 * uey);
    }
    double jbx = ubx / r, jby = uby / r;
    double ax = g.ushift * ubx / r, ay = g.ushift * uby / r;
    rb -= (ubx * uex + uby * uey) / r;

    // wall objective terms (interior columns; a row may serve both walls on
    // very low channels)
    if (g.walls) {
        for (int side = 0; side < 2; ++side) {
            const int y1 = side ? g.ny - 2 : 1, y2 = side ? g.ny - 3 : 2;
            if (y == y1) {
                const int c2 = y2 * g.nx + x;
                const double v2 = (jx[c2] + 0.5 * Fx[c2]) / rho[c2];
                jbx += g.w_tau * 3.0 * g.nu;
                ax += g.w_tau * 1.5 * g.nu;
                rb += -g.w_tau * g.nu / 3.0 * v2;
                rb += g.w_p * (g.k2 * cs_dp0(g, r) - g.kappa * L1[ri1(g, x, y)]);
                Ls[c] += -g.w_p * g.kappa * r;
                double grx, gry;
                grad_rho(g, rho, x, y, grx, gry);
                Cx[c] += -g.w_p * g.kappa * grx;
                Cy[c] += -g.w_p * g.kappa * gry;
            }
            if (y == y2) {
                const double r1v = rho[y1 * g.nx + x];
                const double v2 = (jX + 0.5 * FX) / r;
                jbx += -g.w_tau * g.nu / 3.0 * r1v / r;
                ax += -g.w_tau * g.nu / 6.0 * r1v / r;
                rb += g.w_tau * g.nu / 3.0 * r1v * v2 / r;
            }
        }
    }

    // pressure column fed by this node:
    // f*_i(x_b) = f_eq_i(rho_b, v_f) + (1 - 1/tau)(f_i(x_f) - f_eq_i(rho_f, v_f)),
    // v_f = (j_f + F_f / 2) / rho_f
    if (g.bc_x && (x == 1 || x == g.nx - 2)) {
        const int xb = x == 1 ? 0 : g.nx - 1, cb = y * g.nx + xb;
        double gc[9];
        for (int i = 0; i < 9; ++i) {
            int tx = xb + ex_(i), ty = y + ey_(i);
            gc[i] = 0.0;
            if (g.walls && (ty == 0 || ty == g.ny - 1)) continue;  // into the column's own (unread) slots
            if (!g.walls) ty = pmod(ty, g.ny);
            if (tx < 0 || tx >= g.nx) continue;                      // leaves the lattice
            gc[i] = lam_in[i * n + ty * g.nx + tx];
        }
        const double rbv = rho[cb];
        const double vx = (jX + 0.5 * FX) / r, vy = (jY + 0.5 * FY) / r;
        const double vsq = vx * vx + vy * vy;
        double rbb = 0.0, vbx = 0.0, vby = 0.0;
        for (int i = 0; i < 9; ++i) {
            const double ev = ex_(i) * vx + ey_(i) * vy;
            const double q = wq(i) * (1.0 + 3.0 * ev + 4.5 * ev * ev - 1.5 * vsq);
            lam[i] += omt * gc[i];
            rbb += gc[i] * q;
            rb -= omt * gc[i] * q;
            const double s = gc[i] * (rbv - omt * r) * wq(i);
            vbx += s * (3.0 * ex_(i) + 9.0 * ev * ex_(i) - 3.0 * vx);
            vby += s * (3.0 * ey_(i) + 9.0 * ev * ey_(i) - 3.0 * vy);
        }
        R[cb] = rbb;
        jbx += vbx / r;
        jby += vby / r;
        ax += 0.5 * vbx / r;
        ay += 0.5 * vby / r;
        rb -= (vbx * vx + vby * vy) / r;
    }

    // F = ... + kappa rho grad L: the rho factor
    double glx = 0.0, gly = 0.0;
    for (int i = 1; i < 9; ++i) {
        const double l = L1[ri1(g, x + ex_(i), y + ey_(i))];
        glx += 3.0 * wq(i) * ex_(i) * l;
        gly += 3.0 * wq(i) * ey_(i) * l;
    }
    rb += g.kappa * (ax * glx + ay * gly);

    for (int i = 0; i < 9; ++i) lam_out[i * n + c] = lam[i];
    Ax[c] = ax;
    Ay[c] = ay;
    Jbx[c] = jbx;
    Jby[c] = jby;
    R[c] = rb;
}

// Lbar and phibar on the ring-1 grid: transposed gradients of the force.
__global__ void adj_lbar(AdjGeo g, const double *__restrict__ rho, const double *__restrict__ Ax,
                         const double *__restrict__ Ay, const double *__restrict__ Ls, double *Lb1, double *Pb1)
{
    const int w = g.nx + 2, m = w * (g.ny + 2);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int x = t % w - 1, y = t / w - 1;
    double lb = in_lat(g, x, y) ? Ls[y * g.nx + x] : 0.0, pb = 0.0;
    for (int i = 1; i < 9; ++i) {
        const int qx = x - ex_(i), qy = y - ey_(i);
        if (!in_lat(g, qx, qy)) continue;
        const int q = qy * g.nx + qx;
        const double s = 3.0 * wq(i) * (ex_(i) * Ax[q] + ey_(i) * Ay[q]);
        lb += g.kappa * rho[q] * s;
        pb -= s;
    }
    Lb1[t] = lb;
    Pb1[t] = pb;
}

// Ebar (adjoint of the ghost-extended density) on the ring-2 grid.
__global__ void adj_ebar(AdjGeo g, const double *__restrict__ rho, const double *__restrict__ Lb1,
                         const double *__restrict__ Pb1, const double *__restrict__ Cx,
                         const double *__restrict__ Cy, double *Eb2)
{
    const int w = g.nx + 4, m = w * (g.ny + 4);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int x = t % w - 2, y = t / w - 2;
    double eb = 0.0;
    if (in_r1(g, x, y)) {
        const double e = ghost_rho(g, rho, x, y);
        eb += Pb1[ri1(g, x, y)] * (g.k2 * cs_dp0(g, e) - 1.0 / 3.0);
        eb -= 6.0 * (1.0 - wq(0)) * Lb1[ri1(g, x, y)];
    }
    for (int i = 1; i < 9; ++i) {
        const int qx = x - ex_(i), qy = y - ey_(i);
        if (in_lat(g, qx, qy)) {
            const int q = qy * g.nx + qx;
            eb += 3.0 * wq(i) * (ex_(i) * Cx[q] + ey_(i) * Cy[q]);
        }
        if (in_r1(g, qx, qy)) eb += 6.0 * wq(i) * Lb1[ri1(g, qx, qy)];
    }
    Eb2[t] = eb;
}

// Sum of Ebar over the extended points whose ghost density is node (x, y).
__device__ double gather_pre(const AdjGeo &g, const double *Eb2, int x, int y)
{
    int px[8], py[8], nxp = 0, nyp = 0;
    if (g.bc_x) {
        px[nxp++] = x;
        if (x == 0) { px[nxp++] = -1; px[nxp++] = -2; }
        if (x == g.nx - 1) { px[nxp++] = g.nx; px[nxp++] = g.nx + 1; }
    } else {
        for (int k = -3; k <= 3; ++k) {
            const int v = x + k * g.nx;
            if (v >= -2 && v <= g.nx + 1 && nxp < 8) px[nxp++] = v;
        }
    }
    if (g.walls) {
        const int cand[3] = {y, 1 - y, 2 * g.ny - 3 - y};
        for (int k = 0; k < 3; ++k) {
            const int v = cand[k];
            if (v < -2 || v > g.ny + 1 || map_y(g, v) != y) continue;
            bool dup = false;
            for (int j = 0; j < nyp; ++j) dup |= py[j] == v;
            if (!dup) py[nyp++] = v;
        }
    } else {
        for (int k = -3; k <= 3; ++k) {
            const int v = y + k * g.ny;
            if (v >= -2 && v <= g.ny + 1 && nyp < 8) py[nyp++] = v;
        }
    }
    double s = 0.0;
    for (int b = 0; b < nyp; ++b)
        for (int a = 0; a < nxp; ++a) s += Eb2[(py[b] + 2) * (g.nx + 4) + (px[a] + 2)];
    return s;
}

// Final gather: lambda^n_i(x) = (1 - 1/tau) f*-bar + rhobar + jbar . e_i.
// Interior neighbours of pressure columns also take the column's rho-bar
// through the phase weight and record the column-density sensitivities.
__global__ void adj_final(AdjGeo g, const double *__restrict__ rho, const double *__restrict__ R,
                          const double *__restrict__ Jbx, const double *__restrict__ Jby,
                          const double *__restrict__ Eb2, double *lam_out, double *colp)
{
    const int n = g.nx * g.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int x = c % g.nx, y = c / g.nx;
    if (solid_row(g, y) || pcol(g, x)) return;  // adj_local zeroed these
    double rb = R[c] + gather_pre(g, Eb2, x, y);
    if (g.bc_x && (x == 1 || x == g.nx - 2)) {
        const int side = x == 1 ? 0 : 1, xb = side ? g.nx - 1 : 0;
        const double rbb = R[y * g.nx + xb] + gather_pre(g, Eb2, xb, y);
        double dth;
        const double th = col_theta(g, rho[c], dth);
        const double gg = side ? g.g_out : g.g_in, ll = side ? g.l_out : g.l_in;
        rb += rbb * dth * (ll - gg);
        colp[(side * g.ny + y) * 2 + 0] = rbb * (1.0 - th);
        colp[(side * g.ny + y) * 2 + 1] = rbb * th;
    }
    const double bx = Jbx[c], by = Jby[c];
    for (int i = 0; i < 9; ++i) lam_out[i * n + c] += rb + bx * ex_(i) + by * ey_(i);
}

// One-block deterministic sums: acc[slot + k] += sum over the k-th series.
constexpr int RED_THREADS = 512;
__global__ void adj_reduce(const double *__restrict__ a, long long stride_a, long long len, int nseries,
                           double *acc)
{
    __shared__ double sh[RED_THREADS];
    for (int k = 0; k < nseries; ++k) {
        double s = 0.0;
        for (long long i = threadIdx.x; i < len; i += RED_THREADS) s += a[k * stride_a + i];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int h = RED_THREADS / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) acc[k] += sh[0];
        __syncthreads();
    }
}

// colp holds (side, row, {gas, liquid}) pairs; sums into acc[0..3] as
// (gas_in, liq_in, gas_out, liq_out).
__global__ void adj_reduce_col(const double *__restrict__ colp, int ny, double *acc)
{
    __shared__ double sh[RED_THREADS];
    for (int k = 0; k < 4; ++k) {
        const int side = k / 2, br = k % 2;
        double s = 0.0;
        for (int y = threadIdx.x; y < ny; y += RED_THREADS) s += colp[(side * ny + y) * 2 + br];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int h = RED_THREADS / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) acc[k] += sh[0];
        __syncthreads();
    }
}

// the resting equilibrium of rho0, in the state layout (padding columns stay as set)
template <typename S>
__global__ void adj_init_f(AdjGeo g, const double *__restrict__ rho0, S *f)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.nx * g.ny) return;
    const int x = c % g.nx, y = c / g.nx;
    for (int i = 0; i < 9; ++i) f[((size_t)y * 9 + i) * g.fp + x] = (S)(wq(i) * rho0[c]);
}

__global__ void adj_grad_rho0(const double *__restrict__ lam, int n, double *g)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += wq(i) * lam[i * n + c];
    g[c] = s;
}

constexpr int TPB = 256;
inline unsigned blocks(long long m) { return (unsigned)((m + TPB - 1) / TPB); }

} // namespace

struct lbm_adjoint {
    lbm_grid grid{};
    lbm_eos eos{};
    lbm_drive drive{};
    double tau = 1, wet = 0;
    int64_t nsteps = 0, K = 0, nblocks = 0;
    cudaStream_t stream = nullptr;
    lbm_ctx *ctx = nullptr;
    bool have_drive = false, forward_done = false;
    lbm_collision coll{};  // BGK unless set
    AdjGeo geo{};
    double dgin = 0, dlin = 0, dgout = 0, dlout = 0;  // d rho_column / d dp
    // device buffers
    double *ckpt = nullptr, *blk = nullptr, *lam0 = nullptr, *lam1 = nullptr;
    double *rho = nullptr, *jx = nullptr, *jy = nullptr, *Fx = nullptr, *Fy = nullptr, *L1 = nullptr;
    double *Ax = nullptr, *Ay = nullptr, *Jbx = nullptr, *Jby = nullptr, *R = nullptr, *Ls = nullptr;
    double *Cx = nullptr, *Cy = nullptr, *Lb1 = nullptr, *Pb1 = nullptr, *Eb2 = nullptr;
    double *tw = nullptr, *pw = nullptr, *colp = nullptr, *acc = nullptr, *rho0 = nullptr;
    std::vector<void *> allocs;
    std::string err;
};

namespace {

lbm_status adj_fail(lbm_adjoint *a, cudaError_t e, const char *what)
{
    a->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define ACK(expr, what)                              \
    do {                                             \
        cudaError_t e_ = (expr);                     \
        if (e_ != cudaSuccess) return adj_fail(a, e_, what); \
    } while (0)

lbm_status adj_alloc(lbm_adjoint *a, double **p, size_t count)
{
    void *q = nullptr;
    ACK(cudaMalloc(&q, count * sizeof(double)), "adjoint allocation");
    a->allocs.push_back(q);
    *p = (double *)q;
    return LBM_OK;
}

size_t npop(const lbm_adjoint *a) { return (size_t)9 * a->grid.nx * a->grid.ny; }
// one stored state in the forward context's own layout (plane pitch pitch_of(nx))
size_t spop(const lbm_adjoint *a) { return (size_t)9 * lbm::pitch_of(a->grid.nx) * a->grid.ny; }
// bytes of one stored state (the forward precision), and state k of an array of them
size_t sbytes(const lbm_adjoint *a) { return spop(a) * (a->grid.precision == 32 ? 4 : 8); }
void *state_at(double *base, size_t k, size_t bytes) { return (char *)base + k * bytes; }

lbm_status adj_fields(lbm_adjoint *a, const void *f)
{
    const AdjGeo &g = a->geo;
    const long long n = (long long)g.nx * g.ny, m1 = (long long)(g.nx + 2) * (g.ny + 2);
    if (a->grid.precision == 32)
        adj_moments<float><<<blocks(n), TPB, 0, a->stream>>>(g, (const float *)f, a->rho, a->jx, a->jy);
    else
        adj_moments<double><<<blocks(n), TPB, 0, a->stream>>>(g, (const double *)f, a->rho, a->jx, a->jy);
    adj_lap<<<blocks(m1), TPB, 0, a->stream>>>(g, a->rho, a->L1);
    adj_force<<<blocks(n), TPB, 0, a->stream>>>(g, a->rho, a->L1, a->Fx, a->Fy);
    ACK(cudaGetLastError(), "adjoint field kernels");
    return LBM_OK;
}

lbm_status adj_objective(lbm_adjoint *a, const void *f)
{
    lbm_status s = adj_fields(a, f);
    if (s != LBM_OK) return s;
    const AdjGeo &g = a->geo;
    adj_wall_terms<<<blocks(2LL * g.nx), TPB, 0, a->stream>>>(g, a->rho, a->jx, a->Fx, a->L1, a->tw, a->pw);
    // tw and pw are adjacent: two series of 2 nx
    adj_reduce<<<1, RED_THREADS, 0, a->stream>>>(a->tw, 2LL * g.nx, 2LL * g.nx, 2, a->acc);
    ACK(cudaGetLastError(), "adjoint objective kernels");
    return LBM_OK;
}

lbm_status adj_reverse_step(lbm_adjoint *a, const void *f, const double *lam_in, double *lam_out)
{
    lbm_status s = adj_fields(a, f);
    if (s != LBM_OK) return s;
    const AdjGeo &g = a->geo;
    const long long n = (long long)g.nx * g.ny, m1 = (long long)(g.nx + 2) * (g.ny + 2),
                    m2 = (long long)(g.nx + 4) * (g.ny + 4);
    adj_local<<<blocks(n), TPB, 0, a->stream>>>(g, lam_in, a->rho, a->jx, a->jy, a->Fx, a->Fy, a->L1, lam_out,
                                                a->Ax, a->Ay, a->Jbx, a->Jby, a->R, a->Ls, a->Cx, a->Cy);
    adj_lbar<<<blocks(m1), TPB, 0, a->stream>>>(g, a->rho, a->Ax, a->Ay, a->Ls, a->Lb1, a->Pb1);
    adj_ebar<<<blocks(m2), TPB, 0, a->stream>>>(g, a->rho, a->Lb1, a->Pb1, a->Cx, a->Cy, a->Eb2);
    ACK(cudaMemsetAsync(a->colp, 0, 4 * (size_t)g.ny * sizeof(double), a->stream), "adjoint memset");
    adj_final<<<blocks(n), TPB, 0, a->stream>>>(g, a->rho, a->R, a->Jbx, a->Jby, a->Eb2, lam_out, a->colp);
    adj_reduce_col<<<1, RED_THREADS, 0, a->stream>>>(a->colp, g.ny, a->acc + 2);
    // Ax and Ay are adjacent: body-force sensitivities
    adj_reduce<<<1, RED_THREADS, 0, a->stream>>>(a->Ax, n, n, 2, a->acc + 6);
    ACK(cudaGetLastError(), "adjoint reverse kernels");
    return LBM_OK;
}

lbm_status ctx_status(lbm_adjoint *a, lbm_status s, const char *what)
{
    if (s != LBM_OK) {
        const char *m = a->ctx ? lbm_last_error(a->ctx) : "";
        a->err = std::string(what) + ": " + lbm_status_string(s) + (m && *m ? std::string(" (") + m + ")" : "");
    }
    return s;
}

bool same_drive(const lbm_drive &x, const lbm_drive &y)
{
    auto eq = [](double u, double v) { return u == v || (std::isnan(u) && std::isnan(v)); };
    return eq(x.dp, y.dp) && eq(x.p_ref, y.p_ref) && eq(x.gx, y.gx) && eq(x.gy, y.gy);
}

// (Re)build the FP64 forward context for a drive and the adjoint's geometry.
lbm_status adj_setup_drive(lbm_adjoint *a, const lbm_drive *drive)
{
    lbm_drive d = drive ? *drive : lbm_drive{0.0, NAN, 0.0, 0.0};
    if (a->ctx && a->have_drive && same_drive(d, a->drive)) return LBM_OK;
    if (a->ctx) { lbm_free(a->ctx); a->ctx = nullptr; }
    std::vector<double> one((size_t)a->grid.nx * a->grid.ny, 0.1);
    lbm_status s = lbm_init(&a->grid, &a->eos, a->tau, nullptr, a->wet, &d, one.data(), nullptr, 0, a->stream, &a->ctx);
    if (s != LBM_OK) { a->err = std::string("forward context: ") + lbm_status_string(s); a->ctx = nullptr; return s; }
    if ((s = lbm_set_collision(a->ctx, &a->coll)) != LBM_OK) return ctx_status(a, s, "collision");
    a->drive = d;
    a->have_drive = true;
    lbm_diag_t dg;
    s = lbm_diag(a->ctx, &dg);
    if (s != LBM_OK) return ctx_status(a, s, "forward context diag");

    AdjGeo &g = a->geo;
    g.nx = a->grid.nx; g.ny = a->grid.ny; g.walls = a->grid.walls; g.bc_x = a->grid.bc_x;
    g.fp = lbm::pitch_of(a->grid.nx);
    lbm::Thermo th{};
    double tc;
    if (lbm::thermo_of(a->eos, &th, &tc)) { a->err = "equation of state"; return LBM_ERR_PARAM; }
    g.eos_kind = th.kind; g.bpr = th.b; g.aalpha = th.aalpha;
    g.RT = a->eos.R * dg.T; g.a = a->eos.a; g.b4 = 0.25 * a->eos.b; g.k2 = a->eos.k * a->eos.k;
    g.kappa = a->eos.kappa; g.tau = a->tau; g.nu = (a->tau - 0.5) / 3.0; g.wet = a->wet;
    g.mrt = a->coll.kind == LBM_COLL_MRT;
    g.ushift = g.mrt ? 1.0 / a->coll.s_j : a->tau;
    if (g.mrt) {
        const double s_nu = a->coll.s_nu > 0 ? a->coll.s_nu : 1.0 / a->tau;
        const double r[9] = {0.0, a->coll.s_e / 36.0, a->coll.s_eps / 36.0, a->coll.s_j / 6.0, a->coll.s_q / 12.0,
                             a->coll.s_j / 6.0, a->coll.s_q / 12.0, s_nu / 4.0, s_nu / 4.0};
        for (int k = 0; k < 9; ++k) g.mrate[k] = r[k];
    }
    g.gx = d.gx; g.gy = d.gy;
    g.g_in = dg.rho_in; g.l_in = dg.rho_in_l; g.g_out = dg.rho_out; g.l_out = dg.rho_out_l;
    g.ph_g = dg.rho_g;
    g.inv_dph = dg.rho_l > dg.rho_g ? 1.0 / (dg.rho_l - dg.rho_g) : 0.0;
    // column densities are EOS roots of k^2 p0(rho) = p_ref +- dp/2, so
    // d rho / d dp = +-1 / (2 k^2 p0'(rho)); a density held at a spinodal
    // does not move with dp
    a->dgin = a->dlin = a->dgout = a->dlout = 0.0;
    if (a->grid.bc_x) {
        lbm::ChannelThermo ct;
        if (lbm::channel_thermo(a->eos, d, true, &ct)) { a->err = "column thermodynamics"; return LBM_ERR_PARAM; }
        auto rate = [&](double rho, bool sat, double sgn) {
            return sat ? 0.0 : sgn * 0.5 / (g.k2 * lbm::eos_dpressure(ct.th, rho));
        };
        a->dgin = rate(g.g_in, ct.sat[0], 1.0);
        a->dlin = rate(g.l_in, ct.sat[1], 1.0);
        a->dgout = rate(g.g_out, ct.sat[2], -1.0);
        a->dlout = rate(g.l_out, ct.sat[3], -1.0);
    }
    return LBM_OK;
}

} // namespace

extern "C" {

lbm_status lbm_adjoint_init(const lbm_grid *grid, const lbm_eos *eos, double tau, double wetting, int64_t nsteps,
                            int64_t block_steps, void *stream, lbm_adjoint **out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!grid || !eos || (grid->precision != 64 && grid->precision != 32) || nsteps < 1 || block_steps < 0)
        return LBM_ERR_ARG;
    if (grid->nx < 1 || grid->ny < 1 || 9ll * grid->nx * grid->ny >= (1ll << 31)) return LBM_ERR_ARG;
    if (!(tau > 0.5) || !std::isfinite(wetting)) return LBM_ERR_PARAM;
    lbm_adjoint *a = new (std::nothrow) lbm_adjoint();
    if (!a) return LBM_ERR_OOM;
    a->grid = *grid;
    a->eos = *eos;
    a->tau = tau;
    a->wet = wetting;
    a->nsteps = nsteps;
    a->K = block_steps > 0 ? block_steps : (int64_t)std::ceil(std::sqrt((double)nsteps));
    if (a->K > nsteps) a->K = nsteps;
    a->nblocks = (nsteps + a->K - 1) / a->K;
    a->stream = (cudaStream_t)stream;

    const size_t n = (size_t)grid->nx * grid->ny, m1 = (size_t)(grid->nx + 2) * (grid->ny + 2),
                 m2 = (size_t)(grid->nx + 4) * (grid->ny + 4), P = npop(a);
    const size_t SD = (sbytes(a) + 7) / 8;  // one stored state, in doubles
    lbm_status s = LBM_OK;
    struct { double **p; size_t count; } bufs[] = {
        {&a->ckpt, SD * a->nblocks}, {&a->blk, SD * a->K}, {&a->lam0, P}, {&a->lam1, P},
        {&a->rho, n}, {&a->jx, n}, {&a->jy, n}, {&a->Fx, n}, {&a->Fy, n}, {&a->L1, m1},
        {&a->Ax, 2 * n}, {&a->Jbx, n}, {&a->Jby, n}, {&a->R, n}, {&a->Ls, n}, {&a->Cx, n}, {&a->Cy, n},
        {&a->Lb1, m1}, {&a->Pb1, m1}, {&a->Eb2, m2}, {&a->tw, 4 * (size_t)grid->nx},
        {&a->colp, 4 * (size_t)grid->ny}, {&a->acc, 8}, {&a->rho0, n}};
    for (auto &b : bufs)
        if (s == LBM_OK) s = adj_alloc(a, b.p, b.count);
    if (s != LBM_OK) { lbm_adjoint_free(a); return s; }
    a->Ay = a->Ax + n;              // adjacent, summed in one reduction
    a->pw = a->tw + 2 * grid->nx;   // likewise
    // the forward context is built by the first forward, for its drive
    lbm::Thermo th{};
    double tc;
    if (lbm::thermo_of(*eos, &th, &tc)) { lbm_adjoint_free(a); return LBM_ERR_PARAM; }
    *out = a;
    return LBM_OK;
}

lbm_status lbm_adjoint_forward(lbm_adjoint *a, const lbm_drive *drive, const double *rho0, double *J)
{
    if (!a || !rho0 || !J) return LBM_ERR_ARG;
    a->forward_done = false;
    lbm_status s = adj_setup_drive(a, drive);
    if (s != LBM_OK) return s;
    const long long n = (long long)a->grid.nx * a->grid.ny;
    const size_t SB = sbytes(a);
    ACK(cudaMemcpyAsync(a->rho0, rho0, n * sizeof(double), cudaMemcpyDefault, a->stream), "rho0 copy");
    ACK(cudaMemsetAsync(a->ckpt, 0, SB, a->stream), "adjoint memset");  // padding columns
    if (a->grid.precision == 32)
        adj_init_f<float><<<blocks(n), TPB, 0, a->stream>>>(a->geo, a->rho0, (float *)a->ckpt);
    else
        adj_init_f<double><<<blocks(n), TPB, 0, a->stream>>>(a->geo, a->rho0, a->ckpt);
    ACK(cudaGetLastError(), "adjoint init kernel");
    ACK(cudaMemsetAsync(a->acc, 0, 8 * sizeof(double), a->stream), "adjoint memset");
    // everything below is enqueued on the context's stream: no host round trip per step
    ACK(lbm_ctx_load_state(a->ctx, a->ckpt), "load initial state");
    for (int64_t t = 0; t < a->nsteps; ++t) {
        if (t > 0 && t % a->K == 0)
            ACK(lbm_ctx_copy_state(a->ctx, state_at(a->ckpt, (size_t)(t / a->K), SB)), "checkpoint");
        // the objective reads the state in the context's own buffer
        if ((s = adj_objective(a, lbm_ctx_state(a->ctx))) != LBM_OK) return s;
        if (t + 1 < a->nsteps && (s = lbm_step(a->ctx, 1)) != LBM_OK) return ctx_status(a, s, "forward step");
    }
    double h[2];
    ACK(cudaMemcpyAsync(h, a->acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, a->stream), "objective copy");
    ACK(cudaStreamSynchronize(a->stream), "forward sync");
    J[0] = h[0];
    J[1] = h[1];
    a->forward_done = true;
    return LBM_OK;
}

lbm_status lbm_adjoint_backward(lbm_adjoint *a, double w_tau, double w_p, double *grad_rho0, double *grad_drive)
{
    if (!a || !grad_rho0 || !grad_drive) return LBM_ERR_ARG;
    if (!a->forward_done) { a->err = "backward before forward"; return LBM_ERR_STATE; }
    if (!std::isfinite(w_tau) || !std::isfinite(w_p)) return LBM_ERR_ARG;
    a->geo.w_tau = w_tau;
    a->geo.w_p = w_p;
    const long long n = (long long)a->grid.nx * a->grid.ny;
    const size_t P = npop(a), SB = sbytes(a);
    ACK(cudaMemsetAsync(a->acc, 0, 8 * sizeof(double), a->stream), "adjoint memset");
    ACK(cudaMemsetAsync(a->lam1, 0, P * sizeof(double), a->stream), "adjoint memset");
    double *lin = a->lam1, *lout = a->lam0;
    lbm_status s;
    for (int64_t b = a->nblocks - 1; b >= 0; --b) {
        const int64_t n0 = b * a->K, n1 = std::min(a->nsteps, n0 + a->K);
        const void *ck = state_at(a->ckpt, (size_t)b, SB);
        if (n1 - n0 > 1) {
            ACK(lbm_ctx_load_state(a->ctx, ck), "load checkpoint");
            for (int64_t m = 1; m < n1 - n0; ++m) {
                if ((s = lbm_step(a->ctx, 1)) != LBM_OK) return ctx_status(a, s, "recompute step");
                ACK(lbm_ctx_copy_state(a->ctx, state_at(a->blk, (size_t)m, SB)), "recompute copy");
            }
        }
        for (int64_t t = n1 - 1; t >= n0; --t) {
            const void *state = t == n0 ? ck : state_at(a->blk, (size_t)(t - n0), SB);
            if ((s = adj_reverse_step(a, state, lin, lout)) != LBM_OK) return s;
            std::swap(lin, lout);
        }
    }
    adj_grad_rho0<<<blocks(n), TPB, 0, a->stream>>>(lin, (int)n, a->rho0);
    ACK(cudaGetLastError(), "gradient kernel");
    ACK(cudaMemcpyAsync(grad_rho0, a->rho0, n * sizeof(double), cudaMemcpyDefault, a->stream), "gradient copy");
    double h[8];
    ACK(cudaMemcpyAsync(h, a->acc, 8 * sizeof(double), cudaMemcpyDeviceToHost, a->stream), "gradient copy");
    ACK(cudaStreamSynchronize(a->stream), "backward sync");
    // h[2..5]: sensitivities to the column densities (gas_in, liq_in, gas_out, liq_out)
    grad_drive[0] = h[2] * a->dgin + h[3] * a->dlin + h[4] * a->dgout + h[5] * a->dlout;
    grad_drive[1] = h[6];
    grad_drive[2] = h[7];
    return LBM_OK;
}

lbm_status lbm_adjoint_set_collision(lbm_adjoint *a, const lbm_collision *c)
{
    if (!a) return LBM_ERR_ARG;
    const lbm_collision prev = a->coll;
    a->coll = c ? *c : lbm_collision{};
    if (a->ctx) {
        lbm_status s = lbm_set_collision(a->ctx, &a->coll);
        if (s != LBM_OK) { a->coll = prev; return s; }
    } else if (a->coll.kind == LBM_COLL_MRT) {
        for (double r : {a->coll.s_e, a->coll.s_eps, a->coll.s_j, a->coll.s_q})
            if (!(r > 0.0 && r < 2.0)) { a->coll = prev; return LBM_ERR_ARG; }
    } else if (a->coll.kind != LBM_COLL_BGK) {
        a->coll = prev;
        return LBM_ERR_ARG;
    }
    a->have_drive = false;    // rebuild the geometry with the new collision
    a->forward_done = false;  // earlier checkpoints belong to the old operator
    return LBM_OK;
}

const char *lbm_adjoint_last_error(const lbm_adjoint *a) { return a ? a->err.c_str() : ""; }

void lbm_adjoint_free(lbm_adjoint *a)
{
    if (!a) return;
    if (a->ctx) lbm_free(a->ctx);
    for (void *p : a->allocs) cudaFree(p);
    delete a;
}

} // extern "C"
