// Discrete adjoint of the fused step with checkpoint-and-recompute.
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
// recomputed from a checkpoint by the forward context and kept in HBM. The
// reverse arithmetic is FP64, or FP32 on request (lbm_adjoint_set_precision);
// sums over steps are FP64 either way.
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

// T: the reverse sweep's arithmetic type (double, or float where the forward
// is FP32 and the gradient's bound is far above FP32 rounding)
template <typename T>
__device__ __forceinline__ T wq(int i) { return lbm::w_<T>(i); }

template <typename T>
struct AdjGeo {
    int nx, ny, walls, bc_x;
    int fp;                       // plane pitch of a stored state: rows of nine planes, f[(y * 9 + i) * fp + x]
    int eos_kind;                 // 0 Carnahan-Starling, 1 Peng-Robinson
    T RT, a, b4, k2, kappa, tau, inv_tau, nu, wet, gx, gy;
    T bpr, aalpha;                // PR: b and a alpha(T)
    T g_in, l_in, g_out, l_out, ph_g, inv_dph;  // inv_dph = 0: single phase, no blend
    T w_tau, w_p;
    // collision: BGK (mrt = 0) or MRT with rates over the squared row norms of
    // the moment basis (mrate[k] = s_k / |M_k|^2); the equilibrium velocity is
    // u + ushift F / rho with ushift = tau (BGK) or 1 / s_j (MRT)
    int mrt;
    T ushift, mrate[9];
};

// the FP64 parameters rounded to the reverse sweep's type
template <typename T>
AdjGeo<T> geo_as(const AdjGeo<double> &d)
{
    AdjGeo<T> g;
    g.nx = d.nx; g.ny = d.ny; g.walls = d.walls; g.bc_x = d.bc_x; g.fp = d.fp; g.eos_kind = d.eos_kind;
    g.RT = (T)d.RT; g.a = (T)d.a; g.b4 = (T)d.b4; g.k2 = (T)d.k2; g.kappa = (T)d.kappa; g.tau = (T)d.tau;
    g.inv_tau = (T)d.inv_tau; g.nu = (T)d.nu; g.wet = (T)d.wet; g.gx = (T)d.gx; g.gy = (T)d.gy;
    g.bpr = (T)d.bpr; g.aalpha = (T)d.aalpha;
    g.g_in = (T)d.g_in; g.l_in = (T)d.l_in; g.g_out = (T)d.g_out; g.l_out = (T)d.l_out;
    g.ph_g = (T)d.ph_g; g.inv_dph = (T)d.inv_dph; g.w_tau = (T)d.w_tau; g.w_p = (T)d.w_p;
    g.mrt = d.mrt; g.ushift = (T)d.ushift;
    for (int k = 0; k < 9; ++k) g.mrate[k] = (T)d.mrate[k];
    return g;
}

// Lallemand-Luo moment basis (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy)
// over the D2Q9 velocities: entry (k, i) per class of velocity (rest, axis,
// diagonal), folded at compile time inside unrolled loops.
__device__ __forceinline__ constexpr int mrow(int k, int i)
{
    return k == 0 ? 1
         : k == 1 ? (i == 0 ? -4 : (i <= 4 ? -1 : 2))
         : k == 2 ? (i == 0 ? 4 : (i <= 4 ? -2 : 1))
         : k == 3 ? ex_(i)
         : k == 4 ? ex_(i) * (i <= 4 ? -2 : 1)
         : k == 5 ? ey_(i)
         : k == 6 ? ey_(i) * (i <= 4 ? -2 : 1)
         : k == 7 ? ex_(i) * ex_(i) - ey_(i) * ey_(i)
         : ex_(i) * ey_(i);
}

// t += c v for a small integer constant c (no operation for c = 0)
template <typename T>
__device__ __forceinline__ void acc_c(T &t, int c, T v)
{
    if (c == 1) t += v;
    else if (c == -1) t -= v;
    else if (c != 0) t = fma((T)c, v, t);
}

// v -> K v with K = M^-1 S M = M^T diag(s_k / |M_k|^2) M. K is symmetric, so
// the same map transposes the MRT relaxation f* = f - K (f - f_eq).
template <typename T>
__device__ __forceinline__ void mrt_apply(const AdjGeo<T> &g, const T (&v)[9], T (&out)[9])
{
    T m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        T t = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) acc_c(t, mrow(k, i), v[i]);
        m[k] = t * g.mrate[k];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        T t = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) acc_c(t, mrow(k, i), m[k]);
        out[i] = t;
    }
}

template <typename T>
__device__ __forceinline__ bool solid_row(const AdjGeo<T> &g, int y) { return g.walls && (y == 0 || y == g.ny - 1); }
template <typename T>
__device__ __forceinline__ bool pcol(const AdjGeo<T> &g, int x) { return g.bc_x && (x == 0 || x == g.nx - 1); }
__device__ __forceinline__ int pmod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// EOS p0 and dp0/drho: Carnahan-Starling (eta = b rho / 4) or Peng-Robinson
// (x = b rho, D = 1 + 2x - x^2).
template <typename T>
__device__ __forceinline__ T cs_p0(const AdjGeo<T> &g, T r)
{
    if (g.eos_kind == 1) {
        const T x = g.bpr * r;
        return r * g.RT / (T(1) - x) - g.aalpha * r * r / (T(1) + x * (T(2) - x));
    }
    const T eta = g.b4 * r, om = T(1) - eta;
    return r * g.RT * (T(1) + eta * (T(1) + eta * (T(1) - eta))) / (om * om * om) - g.a * r * r;
}
template <typename T>
__device__ __forceinline__ T cs_dp0(const AdjGeo<T> &g, T r)
{
    if (g.eos_kind == 1) {
        const T x = g.bpr * r, om = T(1) - x, D = T(1) + x * (T(2) - x);
        return g.RT / (om * om) - T(2) * g.aalpha * r * (T(1) + x) / (D * D);
    }
    const T eta = g.b4 * r, om = T(1) - eta, om2 = om * om;
    return g.RT * (T(1) + eta * (T(4) + eta * (T(4) + eta * (T(-4) + eta)))) / (om2 * om2) - T(2) * g.a * r;
}
template <typename T>
__device__ __forceinline__ T phi_of(const AdjGeo<T> &g, T r) { return g.k2 * cs_p0(g, r) - r / T(3); }

template <typename T>
__device__ __forceinline__ int map_y(const AdjGeo<T> &g, int y)
{
    if (g.walls) return y <= 0 ? 1 - y : (y >= g.ny - 1 ? 2 * g.ny - 3 - y : y);
    return pmod(y, g.ny);
}
template <typename T>
__device__ __forceinline__ int map_x(const AdjGeo<T> &g, int x)
{
    if (g.bc_x) return x < 0 ? 0 : (x > g.nx - 1 ? g.nx - 1 : x);
    return pmod(x, g.nx);
}
// Density seen by a stencil at (x, y), up to two nodes outside the lattice:
// mirror images behind walls (plus the wetting offset), clamp beyond pressure
// columns, wrap on periodic axes.
template <typename T>
__device__ __forceinline__ T ghost_rho(const AdjGeo<T> &g, const T *rho, int x, int y)
{
    const bool beyond = g.walls && (y <= 0 || y >= g.ny - 1);
    return rho[map_y(g, y) * g.nx + map_x(g, x)] + (beyond ? g.wet : T(0));
}

// gx, gy += 3 w_i e_i v: direction i's term of the lattice gradient, zero
// components skipped (i is a constant inside unrolled loops)
template <typename T>
__device__ __forceinline__ void grad_term(T &gx, T &gy, int i, T v)
{
    if (ex_(i) != 0) gx += T(3) * wq<T>(i) * T(ex_(i)) * v;
    if (ey_(i) != 0) gy += T(3) * wq<T>(i) * T(ey_(i)) * v;
}

// Ring-1 (fluid plus one node) and ring-2 extended grids.
template <typename T>
__device__ __forceinline__ int ri1(const AdjGeo<T> &g, int x, int y) { return (y + 1) * (g.nx + 2) + (x + 1); }
template <typename T>
__device__ __forceinline__ bool in_r1(const AdjGeo<T> &g, int x, int y)
{
    return x >= -1 && x <= g.nx && y >= -1 && y <= g.ny;
}
template <typename T>
__device__ __forceinline__ bool in_lat(const AdjGeo<T> &g, int x, int y)
{
    return x >= 0 && x < g.nx && y >= 0 && y < g.ny;
}

// Phase weight of a pressure column whose neighbour has density rf, and its
// derivative (zero where clamped).
template <typename T>
__device__ __forceinline__ T col_theta(const AdjGeo<T> &g, T rf, T &dth)
{
    dth = 0;
    if (!(g.inv_dph > T(0))) return 0;
    T th = (rf - g.ph_g) * g.inv_dph;
    if (th < T(0)) return 0;
    if (th > T(1)) return 1;
    if (th > T(0) && th < T(1)) dth = g.inv_dph;
    return th;
}

// ---- forward recompute of the fields of one state ---------------------------

// S: the stored state's type (double, or float for an FP32 forward)
template <typename S, typename T>
__global__ void adj_moments(AdjGeo<T> g, const S *__restrict__ f, T *rho, T *jx, T *jy)
{
    const int n = g.nx * g.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int x = c % g.nx, y = c / g.nx;
    if (solid_row(g, y)) { rho[c] = jx[c] = jy[c] = 0; return; }
    const S *fr = f + (size_t)y * 9 * g.fp;  // row y of the state
    if (pcol(g, x)) {
        const int xf = x == 0 ? 1 : g.nx - 2;
        T rf = 0;
        for (int i = 0; i < 9; ++i) rf += (T)fr[i * g.fp + xf];
        T dth;
        const T th = col_theta(g, rf, dth);
        const T gg = x == 0 ? g.g_in : g.g_out, ll = x == 0 ? g.l_in : g.l_out;
        rho[c] = gg + th * (ll - gg);
        jx[c] = jy[c] = 0;
        return;
    }
    T r = 0, X = 0, Y = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const T fi = (T)fr[i * g.fp + x];
        r += fi;
        acc_c(X, ex_(i), fi);
        acc_c(Y, ey_(i), fi);
    }
    rho[c] = r;
    jx[c] = X;
    jy[c] = Y;
}

// lap(rho) = 6 sum_i w_i (rho(x + e_i) - rho(x)) and the EOS potential
// phi(rho) on the ring-1 grid (phi once per point: the force reads it at
// eight neighbours).
template <typename T>
__global__ void adj_lap(AdjGeo<T> g, const T *__restrict__ rho, T *L1, T *Phi1)
{
    const int w = g.nx + 2, m = w * (g.ny + 2);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int x = t % w - 1, y = t / w - 1;
    const T e0 = ghost_rho(g, rho, x, y);
    T s = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) s += T(6) * wq<T>(i) * (ghost_rho(g, rho, x + ex_(i), y + ey_(i)) - e0);
    L1[t] = s;
    Phi1[t] = phi_of(g, e0);
}

// F = -grad phi + kappa rho grad L + G at fluid nodes (grad = 3 sum_i w_i e_i).
template <typename T>
__global__ void adj_force(AdjGeo<T> g, const T *__restrict__ rho, const T *__restrict__ L1,
                          const T *__restrict__ Phi1, T *Fx, T *Fy)
{
    const int n = g.nx * g.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int x = c % g.nx, y = c / g.nx;
    if (solid_row(g, y) || pcol(g, x)) { Fx[c] = Fy[c] = 0; return; }
    T gpx = 0, gpy = 0, glx = 0, gly = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int q = ri1(g, x + ex_(i), y + ey_(i));
        grad_term(gpx, gpy, i, Phi1[q]);
        grad_term(glx, gly, i, L1[q]);
    }
    Fx[c] = -gpx + g.kappa * rho[c] * glx + g.gx;
    Fy[c] = -gpy + g.kappa * rho[c] * gly + g.gy;
}

template <typename T>
__device__ __forceinline__ void grad_rho(const AdjGeo<T> &g, const T *rho, int x, int y, T &gx, T &gy)
{
    gx = gy = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) grad_term(gx, gy, i, ghost_rho(g, rho, x + ex_(i), y + ey_(i)));
}

// Wall shear and wall pressure per (side, column), added to their FP64 sums
// over the steps: 2 nx entries each.
template <typename T>
__global__ void adj_wall_terms(AdjGeo<T> g, const T *__restrict__ rho, const T *__restrict__ jx,
                               const T *__restrict__ Fx, const T *__restrict__ L1, double *tw, double *pw)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * g.nx) return;
    const int side = t / g.nx, x = t % g.nx;
    if (!g.walls || pcol(g, x)) return;
    const int y1 = side ? g.ny - 2 : 1, y2 = side ? g.ny - 3 : 2;
    const int c1 = y1 * g.nx + x, c2 = y2 * g.nx + x;
    const T r1 = rho[c1], r2 = rho[c2];
    const T m1 = jx[c1] + T(0.5) * Fx[c1], v2 = (jx[c2] + T(0.5) * Fx[c2]) / r2;
    tw[t] += (double)(g.nu * (T(9) * m1 - r1 * v2) / T(3));
    T grx, gry;
    grad_rho(g, rho, x, y1, grx, gry);
    pw[t] += (double)(g.k2 * cs_p0(g, r1) - g.kappa * r1 * L1[ri1(g, x, y1)] -
                      T(0.5) * g.kappa * (grx * grx + gry * gry));
}

// ---- reverse step ---------------------------------------------------------

// Local part of the reverse step at every lattice node: reverse streaming,
// reverse collision, the pressure column fed by this node, and the wall
// objective terms of this node. Outputs Fbar (A), jbar, the local rho-bar (R;
// a column's own entry is written by its interior neighbour), the objective
// sources of Lbar and Ebar (Ls, Cx, Cy) and (1 - 1/tau) f*-bar into lam_out;
// Fbar is also added to its FP64 per-node sum over the steps (AS).
template <typename T>
__global__ void adj_local(AdjGeo<T> g, const T *__restrict__ lam_in, const T *__restrict__ rho,
                          const T *__restrict__ jx, const T *__restrict__ jy, const T *__restrict__ Fx,
                          const T *__restrict__ Fy, const T *__restrict__ L1, T *lam_out, T *Ax, T *Ay,
                          T *Jbx, T *Jby, T *R, T *Ls, T *Cx, T *Cy, double *AS)
{
    const int n = g.nx * g.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int x = c % g.nx, y = c / g.nx;
    Ls[c] = Cx[c] = Cy[c] = 0;
    Ax[c] = Ay[c] = Jbx[c] = Jby[c] = 0;
    if (solid_row(g, y) || pcol(g, x)) {
        if (solid_row(g, y)) R[c] = 0;
        for (int i = 0; i < 9; ++i) lam_out[i * n + c] = 0;
        return;
    }
    const T omt = T(1) - g.inv_tau;
    const T r = rho[c], jX = jx[c], jY = jy[c], FX = Fx[c], FY = Fy[c];

    // reverse streaming: f*_i(x) went to x + e_i, or back to x as opp(i)
    T gb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int tx = x + ex_(i), ty = y + ey_(i);
        if (g.walls && (ty == 0 || ty == g.ny - 1)) { gb[i] = lam_in[opp_(i) * n + c]; continue; }
        if (!g.walls) ty = pmod(ty, g.ny);
        if (!g.bc_x) tx = pmod(tx, g.nx);
        gb[i] = lam_in[i * n + ty * g.nx + tx];
    }

    // collision f* = f - K (f - f_eq(rho, u_eq)), u_eq = (j + ushift F) / rho,
    // K = I / tau (BGK) or M^-1 S M (MRT): f-bar = g - K g, f_eq-bar = K g
    const T inv_r = T(1) / r;
    T lam[9], kg[9];
    if (g.mrt) {
        mrt_apply(g, gb, kg);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) kg[i] = gb[i] * g.inv_tau;
    }
    // f_eq_i = w_i rho (1 + 3 e_i.u + 4.5 (e_i.u)^2 - 1.5 u^2) is quadratic in
    // e_i, so its reverse needs only the moments of w_i f_eq-bar_i up to
    // second order
    T M0 = 0, Mx = 0, My = 0, Mxx = 0, Myy = 0, Mxy = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        lam[i] = gb[i] - kg[i];
        const T a = wq<T>(i) * kg[i];
        M0 += a;
        acc_c(Mx, ex_(i), a);
        acc_c(My, ey_(i), a);
        acc_c(Mxx, ex_(i) * ex_(i), a);
        acc_c(Myy, ey_(i) * ey_(i), a);
        acc_c(Mxy, ex_(i) * ey_(i), a);
    }
    const T uex = (jX + g.ushift * FX) * inv_r, uey = (jY + g.ushift * FY) * inv_r;
    const T usq = uex * uex + uey * uey;
    T rb = M0 * (T(1) - T(1.5) * usq) + T(3) * (uex * Mx + uey * My) +
           T(4.5) * (uex * uex * Mxx + T(2) * uex * uey * Mxy + uey * uey * Myy);
    // u_eq-bar / rho: the rho factor of f_eq cancels the 1 / rho of u_eq
    const T ubx = T(3) * Mx + T(9) * (uex * Mxx + uey * Mxy) - T(3) * uex * M0;
    const T uby = T(3) * My + T(9) * (uex * Mxy + uey * Myy) - T(3) * uey * M0;
    T jbx = ubx, jby = uby;
    T ax = g.ushift * ubx, ay = g.ushift * uby;
    rb -= ubx * uex + uby * uey;

    // wall objective terms (interior columns; a row may serve both walls on
    // very low channels)
    if (g.walls) {
        for (int side = 0; side < 2; ++side) {
            const int y1 = side ? g.ny - 2 : 1, y2 = side ? g.ny - 3 : 2;
            if (y == y1) {
                const int c2 = y2 * g.nx + x;
                const T v2 = (jx[c2] + T(0.5) * Fx[c2]) / rho[c2];
                jbx += g.w_tau * T(3) * g.nu;
                ax += g.w_tau * T(1.5) * g.nu;
                rb += -g.w_tau * g.nu / T(3) * v2;
                rb += g.w_p * (g.k2 * cs_dp0(g, r) - g.kappa * L1[ri1(g, x, y)]);
                Ls[c] += -g.w_p * g.kappa * r;
                T grx, gry;
                grad_rho(g, rho, x, y, grx, gry);
                Cx[c] += -g.w_p * g.kappa * grx;
                Cy[c] += -g.w_p * g.kappa * gry;
            }
            if (y == y2) {
                const T r1v = rho[y1 * g.nx + x];
                const T v2 = (jX + T(0.5) * FX) * inv_r;
                jbx += -g.w_tau * g.nu / T(3) * r1v * inv_r;
                ax += -g.w_tau * g.nu / T(6) * r1v * inv_r;
                rb += g.w_tau * g.nu / T(3) * r1v * v2 * inv_r;
            }
        }
    }

    // pressure column fed by this node:
    // f*_i(x_b) = f_eq_i(rho_b, v_f) + (1 - 1/tau)(f_i(x_f) - f_eq_i(rho_f, v_f)),
    // v_f = (j_f + F_f / 2) / rho_f
    if (g.bc_x && (x == 1 || x == g.nx - 2)) {
        const int xb = x == 1 ? 0 : g.nx - 1, cb = y * g.nx + xb;
        T gc[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int tx = xb + ex_(i), ty = y + ey_(i);
            gc[i] = 0;
            if (g.walls && (ty == 0 || ty == g.ny - 1)) continue;  // into the column's own (unread) slots
            if (!g.walls) ty = pmod(ty, g.ny);
            if (tx < 0 || tx >= g.nx) continue;                      // leaves the lattice
            gc[i] = lam_in[i * n + ty * g.nx + tx];
        }
        const T rbv = rho[cb];
        const T vx = (jX + T(0.5) * FX) * inv_r, vy = (jY + T(0.5) * FY) * inv_r;
        const T vsq = vx * vx + vy * vy;
        T rbb = 0, vbx = 0, vby = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const T ev = T(ex_(i)) * vx + T(ey_(i)) * vy;
            const T q = wq<T>(i) * (T(1) + T(3) * ev + T(4.5) * ev * ev - T(1.5) * vsq);
            lam[i] += omt * gc[i];
            rbb += gc[i] * q;
            rb -= omt * gc[i] * q;
            const T s = gc[i] * (rbv - omt * r) * wq<T>(i);
            vbx += s * (T(3 * ex_(i)) + T(9) * ev * T(ex_(i)) - T(3) * vx);
            vby += s * (T(3 * ey_(i)) + T(9) * ev * T(ey_(i)) - T(3) * vy);
        }
        R[cb] = rbb;
        jbx += vbx * inv_r;
        jby += vby * inv_r;
        ax += T(0.5) * vbx * inv_r;
        ay += T(0.5) * vby * inv_r;
        rb -= (vbx * vx + vby * vy) * inv_r;
    }

    // F = ... + kappa rho grad L: the rho factor
    T glx = 0, gly = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) grad_term(glx, gly, i, L1[ri1(g, x + ex_(i), y + ey_(i))]);
    rb += g.kappa * (ax * glx + ay * gly);

#pragma unroll
    for (int i = 0; i < 9; ++i) lam_out[i * n + c] = lam[i];
    Ax[c] = ax;
    Ay[c] = ay;
    AS[c] += (double)ax;  // sums over the steps: the body-force sensitivities
    AS[n + c] += (double)ay;
    Jbx[c] = jbx;
    Jby[c] = jby;
    R[c] = rb;
}

// Lbar and phibar on the ring-1 grid: transposed gradients of the force.
template <typename T>
__global__ void adj_lbar(AdjGeo<T> g, const T *__restrict__ rho, const T *__restrict__ Ax,
                         const T *__restrict__ Ay, const T *__restrict__ Ls, T *Lb1, T *Pb1)
{
    const int w = g.nx + 2, m = w * (g.ny + 2);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int x = t % w - 1, y = t / w - 1;
    T lb = in_lat(g, x, y) ? Ls[y * g.nx + x] : T(0), pb = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int qx = x - ex_(i), qy = y - ey_(i);
        if (!in_lat(g, qx, qy)) continue;
        const int q = qy * g.nx + qx;
        T s = 0;
        if (ex_(i) != 0) s += T(ex_(i)) * Ax[q];
        if (ey_(i) != 0) s += T(ey_(i)) * Ay[q];
        s *= T(3) * wq<T>(i);
        lb += g.kappa * rho[q] * s;
        pb -= s;
    }
    Lb1[t] = lb;
    Pb1[t] = pb;
}

// Ebar (adjoint of the ghost-extended density) on the ring-2 grid.
template <typename T>
__global__ void adj_ebar(AdjGeo<T> g, const T *__restrict__ rho, const T *__restrict__ Lb1,
                         const T *__restrict__ Pb1, const T *__restrict__ Cx, const T *__restrict__ Cy, T *Eb2)
{
    const int w = g.nx + 4, m = w * (g.ny + 4);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int x = t % w - 2, y = t / w - 2;
    T eb = 0;
    if (in_r1(g, x, y)) {
        const T e = ghost_rho(g, rho, x, y);
        eb += Pb1[ri1(g, x, y)] * (g.k2 * cs_dp0(g, e) - T(1) / T(3));
        eb -= T(6) * (T(1) - wq<T>(0)) * Lb1[ri1(g, x, y)];
    }
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int qx = x - ex_(i), qy = y - ey_(i);
        if (in_lat(g, qx, qy)) {
            const int q = qy * g.nx + qx;
            T s = 0;
            if (ex_(i) != 0) s += T(ex_(i)) * Cx[q];
            if (ey_(i) != 0) s += T(ey_(i)) * Cy[q];
            eb += T(3) * wq<T>(i) * s;
        }
        if (in_r1(g, qx, qy)) eb += T(6) * wq<T>(i) * Lb1[ri1(g, qx, qy)];
    }
    Eb2[t] = eb;
}

// Sum of Ebar over the extended points whose ghost density is node (x, y).
template <typename T>
__device__ T gather_pre(const AdjGeo<T> &g, const T *Eb2, int x, int y)
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
    T s = 0;
    for (int b = 0; b < nyp; ++b)
        for (int a = 0; a < nxp; ++a) s += Eb2[(py[b] + 2) * (g.nx + 4) + (px[a] + 2)];
    return s;
}

// Final gather: lambda^n_i(x) = (1 - 1/tau) f*-bar + rhobar + jbar . e_i.
// Interior neighbours of pressure columns also take the column's rho-bar
// through the phase weight and add the column-density sensitivities to their
// FP64 sums over the steps (colp).
template <typename T>
__global__ void adj_final(AdjGeo<T> g, const T *__restrict__ rho, const T *__restrict__ R,
                          const T *__restrict__ Jbx, const T *__restrict__ Jby, const T *__restrict__ Eb2,
                          T *lam_out, double *colp)
{
    const int n = g.nx * g.ny;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int x = c % g.nx, y = c / g.nx;
    if (solid_row(g, y) || pcol(g, x)) return;  // adj_local zeroed these
    T rb = R[c] + gather_pre(g, Eb2, x, y);
    if (g.bc_x && (x == 1 || x == g.nx - 2)) {
        const int side = x == 1 ? 0 : 1, xb = side ? g.nx - 1 : 0;
        const T rbb = R[y * g.nx + xb] + gather_pre(g, Eb2, xb, y);
        T dth;
        const T th = col_theta(g, rho[c], dth);
        const T gg = side ? g.g_out : g.g_in, ll = side ? g.l_out : g.l_in;
        rb += rbb * dth * (ll - gg);
        colp[(side * g.ny + y) * 2 + 0] += (double)(rbb * (T(1) - th));
        colp[(side * g.ny + y) * 2 + 1] += (double)(rbb * th);
    }
    const T bx = Jbx[c], by = Jby[c];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        T v = rb;
        acc_c(v, ex_(i), bx);
        acc_c(v, ey_(i), by);
        lam_out[i * n + c] += v;
    }
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
__global__ void adj_init_f(AdjGeo<double> g, const double *__restrict__ rho0, S *f)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.nx * g.ny) return;
    const int x = c % g.nx, y = c / g.nx;
    for (int i = 0; i < 9; ++i) f[((size_t)y * 9 + i) * g.fp + x] = (S)(wq<double>(i) * rho0[c]);
}

template <typename T>
__global__ void adj_grad_rho0(const T *__restrict__ lam, int n, double *g)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += wq<double>(i) * (double)lam[i * n + c];
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
    AdjGeo<double> geo{};
    int rprec = 64;  // reverse sweep (and objective) arithmetic: 64 or 32
    double dgin = 0, dlin = 0, dgout = 0, dlout = 0;  // d rho_column / d dp
    // device buffers (the reverse sweep's fields and adjoint populations are
    // sized for doubles and hold floats with rprec = 32)
    double *ckpt = nullptr, *blk = nullptr, *lam0 = nullptr, *lam1 = nullptr;
    double *rho = nullptr, *jx = nullptr, *jy = nullptr, *Fx = nullptr, *Fy = nullptr, *L1 = nullptr, *Phi1 = nullptr;
    double *Ax = nullptr, *Ay = nullptr, *Jbx = nullptr, *Jby = nullptr, *R = nullptr, *Ls = nullptr;
    double *Cx = nullptr, *Cy = nullptr, *Lb1 = nullptr, *Pb1 = nullptr, *Eb2 = nullptr;
    double *tw = nullptr, *pw = nullptr, *colp = nullptr, *acc = nullptr, *rho0 = nullptr, *AS = nullptr;
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

template <typename T>
T *as(double *p) { return reinterpret_cast<T *>(p); }

template <typename T>
lbm_status adj_fields(lbm_adjoint *a, const AdjGeo<T> &g, const void *f)
{
    const long long n = (long long)g.nx * g.ny, m1 = (long long)(g.nx + 2) * (g.ny + 2);
    if (a->grid.precision == 32)
        adj_moments<float, T><<<blocks(n), TPB, 0, a->stream>>>(g, (const float *)f, as<T>(a->rho), as<T>(a->jx),
                                                                 as<T>(a->jy));
    else
        adj_moments<double, T><<<blocks(n), TPB, 0, a->stream>>>(g, (const double *)f, as<T>(a->rho),
                                                                  as<T>(a->jx), as<T>(a->jy));
    adj_lap<T><<<blocks(m1), TPB, 0, a->stream>>>(g, as<T>(a->rho), as<T>(a->L1), as<T>(a->Phi1));
    adj_force<T><<<blocks(n), TPB, 0, a->stream>>>(g, as<T>(a->rho), as<T>(a->L1), as<T>(a->Phi1), as<T>(a->Fx),
                                                   as<T>(a->Fy));
    ACK(cudaGetLastError(), "adjoint field kernels");
    return LBM_OK;
}

template <typename T>
lbm_status adj_objective_t(lbm_adjoint *a, const void *f)
{
    const AdjGeo<T> g = geo_as<T>(a->geo);
    lbm_status s = adj_fields<T>(a, g, f);
    if (s != LBM_OK) return s;
    adj_wall_terms<T><<<blocks(2LL * g.nx), TPB, 0, a->stream>>>(g, as<T>(a->rho), as<T>(a->jx), as<T>(a->Fx),
                                                                 as<T>(a->L1), a->tw, a->pw);
    ACK(cudaGetLastError(), "adjoint objective kernels");
    return LBM_OK;
}

lbm_status adj_objective(lbm_adjoint *a, const void *f)
{
    return a->rprec == 32 ? adj_objective_t<float>(a, f) : adj_objective_t<double>(a, f);
}

template <typename T>
lbm_status adj_reverse_step_t(lbm_adjoint *a, const void *f, const double *lam_in, double *lam_out)
{
    const AdjGeo<T> g = geo_as<T>(a->geo);
    lbm_status s = adj_fields<T>(a, g, f);
    if (s != LBM_OK) return s;
    const long long n = (long long)g.nx * g.ny, m1 = (long long)(g.nx + 2) * (g.ny + 2),
                    m2 = (long long)(g.nx + 4) * (g.ny + 4);
    T *lo = as<T>(lam_out);
    adj_local<T><<<blocks(n), TPB, 0, a->stream>>>(g, (const T *)lam_in, as<T>(a->rho), as<T>(a->jx), as<T>(a->jy),
                                                   as<T>(a->Fx), as<T>(a->Fy), as<T>(a->L1), lo, as<T>(a->Ax),
                                                   as<T>(a->Ay), as<T>(a->Jbx), as<T>(a->Jby), as<T>(a->R),
                                                   as<T>(a->Ls), as<T>(a->Cx), as<T>(a->Cy), a->AS);
    adj_lbar<T><<<blocks(m1), TPB, 0, a->stream>>>(g, as<T>(a->rho), as<T>(a->Ax), as<T>(a->Ay), as<T>(a->Ls),
                                                   as<T>(a->Lb1), as<T>(a->Pb1));
    adj_ebar<T><<<blocks(m2), TPB, 0, a->stream>>>(g, as<T>(a->rho), as<T>(a->Lb1), as<T>(a->Pb1), as<T>(a->Cx),
                                                   as<T>(a->Cy), as<T>(a->Eb2));
    adj_final<T><<<blocks(n), TPB, 0, a->stream>>>(g, as<T>(a->rho), as<T>(a->R), as<T>(a->Jbx), as<T>(a->Jby),
                                                   as<T>(a->Eb2), lo, a->colp);
    ACK(cudaGetLastError(), "adjoint reverse kernels");
    return LBM_OK;
}

lbm_status adj_reverse_step(lbm_adjoint *a, const void *f, const double *lam_in, double *lam_out)
{
    return a->rprec == 32 ? adj_reverse_step_t<float>(a, f, lam_in, lam_out)
                          : adj_reverse_step_t<double>(a, f, lam_in, lam_out);
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

    AdjGeo<double> &g = a->geo;
    g.nx = a->grid.nx; g.ny = a->grid.ny; g.walls = a->grid.walls; g.bc_x = a->grid.bc_x;
    g.fp = lbm::pitch_of(a->grid.nx);
    lbm::Thermo th{};
    double tc;
    if (lbm::thermo_of(a->eos, &th, &tc)) { a->err = "equation of state"; return LBM_ERR_PARAM; }
    g.eos_kind = th.kind; g.bpr = th.b; g.aalpha = th.aalpha;
    g.RT = a->eos.R * dg.T; g.a = a->eos.a; g.b4 = 0.25 * a->eos.b; g.k2 = a->eos.k * a->eos.k;
    g.kappa = a->eos.kappa; g.tau = a->tau; g.inv_tau = 1.0 / a->tau; g.nu = (a->tau - 0.5) / 3.0; g.wet = a->wet;
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
        {&a->rho, n}, {&a->jx, n}, {&a->jy, n}, {&a->Fx, n}, {&a->Fy, n}, {&a->L1, m1}, {&a->Phi1, m1},
        {&a->Ax, 2 * n}, {&a->Jbx, n}, {&a->Jby, n}, {&a->R, n}, {&a->Ls, n}, {&a->Cx, n}, {&a->Cy, n},
        {&a->Lb1, m1}, {&a->Pb1, m1}, {&a->Eb2, m2}, {&a->tw, 4 * (size_t)grid->nx},
        {&a->colp, 4 * (size_t)grid->ny}, {&a->acc, 8}, {&a->rho0, n}, {&a->AS, 2 * n}};
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
    ACK(cudaMemsetAsync(a->tw, 0, 4 * (size_t)a->grid.nx * sizeof(double), a->stream), "adjoint memset");
    // everything below is enqueued on the context's stream: no host round trip per step
    ACK(lbm_ctx_load_state(a->ctx, a->ckpt), "load initial state");
    for (int64_t t = 0; t < a->nsteps; ++t) {
        if (t > 0 && t % a->K == 0)
            ACK(lbm_ctx_copy_state(a->ctx, state_at(a->ckpt, (size_t)(t / a->K), SB)), "checkpoint");
        // the objective reads the state in the context's own buffer
        if ((s = adj_objective(a, lbm_ctx_state(a->ctx))) != LBM_OK) return s;
        if (t + 1 < a->nsteps && (s = lbm_step(a->ctx, 1)) != LBM_OK) return ctx_status(a, s, "forward step");
    }
    // tw and pw are adjacent: two series of 2 nx per-column sums over the steps
    adj_reduce<<<1, RED_THREADS, 0, a->stream>>>(a->tw, 2LL * a->grid.nx, 2LL * a->grid.nx, 2, a->acc);
    ACK(cudaGetLastError(), "adjoint objective sum");
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
    ACK(cudaMemsetAsync(a->AS, 0, 2 * (size_t)n * sizeof(double), a->stream), "adjoint memset");
    ACK(cudaMemsetAsync(a->colp, 0, 4 * (size_t)a->grid.ny * sizeof(double), a->stream), "adjoint memset");
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
    // per-node and per-row sums over the steps, reduced once
    adj_reduce_col<<<1, RED_THREADS, 0, a->stream>>>(a->colp, a->grid.ny, a->acc + 2);
    adj_reduce<<<1, RED_THREADS, 0, a->stream>>>(a->AS, n, n, 2, a->acc + 6);
    if (a->rprec == 32)
        adj_grad_rho0<float><<<blocks(n), TPB, 0, a->stream>>>((const float *)lin, (int)n, a->rho0);
    else
        adj_grad_rho0<double><<<blocks(n), TPB, 0, a->stream>>>(lin, (int)n, a->rho0);
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

lbm_status lbm_adjoint_set_precision(lbm_adjoint *a, int32_t reverse_precision)
{
    if (!a || (reverse_precision != 32 && reverse_precision != 64)) return LBM_ERR_ARG;
    a->rprec = reverse_precision;
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
