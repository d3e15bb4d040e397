// Fused D2Q9 EOS-multiphase time step for sm_103a (GB300).
//
// One launch performs, for every fluid node, the whole step of the method
// (arXiv 2103.08301, Sec. 2): moments, the nonideal force evaluated from the
// equation of state with a radius-2 density stencil (Eq. 2.17 in the mesh
// space of Eqs. 2.13-2.16), BGK collision with the velocity-shift forcing
// u_eq = u + tau F / rho (Sec. 2.1), the channel boundaries (half-way
// bounce-back walls, mirror ghost densities, pressure columns) and the
// streaming of Eq. 2.1, plus the wall diagnostics of Sec. 3.
//
// Data flow (HBM-bound: 36 B read + 36 B written per node in FP32):
//   - populations live in two structure-of-arrays buffers; a step reads
//     buffer A and pushes post-collision values into buffer B;
//   - each CTA owns a strip of up to BLOCK columns and marches along y over
//     a contiguous range of rows; one thread per column keeps the raw
//     populations of the last four rows in registers (one row prefetched);
//   - rho, phi = k^2 p0(rho) - rho/3 and lap(rho) of the rows in flight sit
//     in an 8-row shared-memory ring that covers the strip plus two halo
//     columns per side; the halo densities are summed from the neighbouring
//     strips' populations (served from L2), so no density array is stored;
//   - rows ya-2 .. yb+1 are read to collide rows ya .. yb-1; the work of a
//     launch is a balanced split of (strip, row) units over the CTAs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int RING = 8;      // shared-memory ring rows (power of two)
constexpr int MAX_CTAS = 8192;

enum { MODE_STEP = 0, MODE_FIELDS = 1 };

template <typename real>
struct KArgs {
    const real *__restrict__ fin;
    real *__restrict__ fout;
    long long plane;  // nx * ny
    int nx, ny;
    int W;            // strip width in columns (<= BLOCK)
    int nstrips;
    int yf0, nyf;     // first fluid row and number of fluid rows
    long long units;  // nstrips * nyf
    int nctas;        // logical CTAs of the schedule
    int reverse;      // launch the logical CTAs in reverse order
    real RT, a, b4, k2, kappa, tau, inv_tau, omb, gx, gy, wet, nu;
    // pressure columns: gas / liquid branch densities at the inlet and outlet
    // pressures, and the phase indicator theta = clamp((rho_f - ph_g) * inv_dph, 0, 1)
    real rho_in_g, rho_in_l, rho_out_g, rho_out_l, ph_g, inv_dph;
    double *mass_part;  // [nctas] mass of the state read (overwritten each step)
    double *J_acc;      // [nctas] accumulated wall shear
    real *ext;          // [nctas][4] running tw_min, tw_max, pw_min, pw_max
    int *err;           // nonzero once a bad density was met
    real *o_rho, *o_vx, *o_vy, *o_tw, *o_pw;  // MODE_FIELDS outputs (device)
};

// D2Q9 velocities, folded at compile time inside unrolled loops.
__device__ __forceinline__ constexpr int ex_(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ constexpr int ey_(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ constexpr int opp_(int i)
{
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 5 + 2) & 3) + 5);
}
template <typename real>
__device__ __forceinline__ constexpr real w_(int i)
{
    return i == 0 ? real(4.0 / 9.0) : (i <= 4 ? real(1.0 / 9.0) : real(1.0 / 36.0));
}

// Mesh-space EOS potential phi = k^2 p0(rho) - rho/3 (Eqs. 2.14, 2.17), CS p0.
template <typename real>
__device__ __forceinline__ real eos_phi(const KArgs<real> &A, real rho)
{
    real eta = A.b4 * rho;
    real om = real(1) - eta;
    real num = real(1) + eta * (real(1) + eta * (real(1) - eta));
    real p0 = rho * A.RT * num / (om * om * om) - A.a * rho * rho;
    return A.k2 * p0 - rho * real(1.0 / 3.0);
}

// f_eq_i(rho, u) of Eq. 2.2. The rest population is taken as rho minus the
// eight moving ones: the weights 4/9, 1/9, 1/36 all round up in FP32 (their
// float sum is 1 + 7.5e-9), which would otherwise add that fraction of the
// mass at every collision.
template <typename real>
__device__ __forceinline__ void feq9(real rho, real ux, real uy, real (&fe)[9])
{
    const real usq = real(1.5) * (ux * ux + uy * uy);
    real moving = real(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const real eu = real(ex_(i)) * ux + real(ey_(i)) * uy;
        fe[i] = rho * w_<real>(i) * (real(1) + real(3) * eu + real(4.5) * eu * eu - usq);
        moving += fe[i];
    }
    fe[0] = rho - moving;
}

// Density of a pressure column whose interior neighbour has density rho_f: the
// EOS root at the column pressure on the branch of the neighbour's phase,
// blended continuously across an interface (Sec. 2.2 pressure-driven ends).
template <typename real>
__device__ __forceinline__ real column_density(const KArgs<real> &A, bool outlet, real rho_f)
{
    real th = (rho_f - A.ph_g) * A.inv_dph;
    th = fmin(fmax(th, real(0)), real(1));
    const real g = outlet ? A.rho_out_g : A.rho_in_g;
    const real l = outlet ? A.rho_out_l : A.rho_in_l;
    return g + th * (l - g);
}

// Row of the stored lattice that a stencil row yy reads, and whether it is a
// mirrored wall ghost (Sec. 2.2 walls; periodic otherwise).
template <bool WALLS>
__device__ __forceinline__ int map_row(int yy, int ny, bool &mirror)
{
    if (WALLS) {
        if (yy <= 0) { mirror = true; return 1 - yy; }
        if (yy >= ny - 1) { mirror = true; return 2 * ny - 3 - yy; }
        mirror = false;
        return yy;
    }
    mirror = false;
    int r = yy % ny;
    return r < 0 ? r + ny : r;
}

// Boundary c of the balanced split of work units over logical CTAs. A cut
// never separates rows 1|2 or ny-3|ny-2, so each wall-shear pair of rows is
// processed by one CTA in one sweep.
template <bool WALLS, typename real>
__device__ __forceinline__ long long cut_units(const KArgs<real> &A, int c)
{
    long long u = ((long long)c * A.units) / A.nctas;
    if (WALLS && u > 0 && u < A.units) {
        int y = A.yf0 + (int)(u % A.nyf);
        if (y == 2 || y == A.ny - 2) u -= 1;
    }
    return u;
}

// Resident CTAs per SM the register allocation is held to (FP32: 4 x 128
// threads -> <= 128 registers; FP64 carries twice the state per thread).
template <typename real>
struct MinBlocks { static constexpr int value = sizeof(real) == 4 ? 4 : 2; };

template <typename real, bool WALLS, bool PRES, int MODE, int BLOCK>
__global__ void __launch_bounds__(BLOCK, MinBlocks<real>::value) step_kernel(const KArgs<real> A)
{
    constexpr int SW = BLOCK + 4;
    __shared__ real s_rho[RING][SW];
    __shared__ real s_phi[RING][SW];
    __shared__ real s_lap[RING][SW];
    __shared__ double s_red[BLOCK / 32][2];
    __shared__ real s_ext[BLOCK / 32][4];
    __shared__ int s_bad;

    const int tid = threadIdx.x;
    const int cta = A.reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    long long u = cut_units<WALLS>(A, cta);
    const long long u1 = cut_units<WALLS>(A, cta + 1);

    const real third = real(1.0 / 3.0), twelfth = real(1.0 / 12.0), sixth = real(1.0 / 6.0);
    double mass = 0.0, Jsum = 0.0;
    real tmin = real(INFINITY), tmax = real(-INFINITY), pmin = real(INFINITY), pmax = real(-INFINITY);
    bool bad = false;
    // wall-pair carries between rows (bottom: rows 1 -> 2; top: ny-3 -> ny-2)
    real b_rho1 = 0, b_v1 = 0, t_v2 = 0;

    while (u < u1) {
        const int s = (int)(u / A.nyf);
        const int ya = A.yf0 + (int)(u - (long long)s * A.nyf);
        const long long ue = min(u1, (long long)(s + 1) * A.nyf);
        const int yb = ya + (int)(ue - u);
        u = ue;

        const int x0 = s * A.W;
        const int xw = min(A.W, A.nx - x0);
        const bool active = tid < xw;
        const int x = x0 + tid;
        const bool pin = PRES && active && x == 0;
        const bool pout = PRES && active && x == A.nx - 1;
        const bool pcol = pin || pout;
        const int xc = pin ? 1 : (pout ? A.nx - 2 : x);  // column whose populations we load
        const int ccol = xc - x0 + 2;                     // its shared-memory column

        // Halo columns: threads 0,1 -> local -2,-1; threads 2,3 -> local xw, xw+1.
        // hmode 1: density of column hx; 2 / 3: inlet / outlet column density
        // derived from column hx = 1 / nx-2 (clamp beyond the pressure columns).
        int hmode = 0, hx = 0, hcol = 0;
        if (tid < 4) {
            const int hloc = (tid < 2) ? (tid - 2) : (xw + tid - 2);
            hcol = hloc + 2;
            const int gxh = x0 + hloc;
            if (PRES) {
                if (gxh <= 0) { hmode = 2; hx = 1; }
                else if (gxh >= A.nx - 1) { hmode = 3; hx = A.nx - 2; }
                else { hmode = 1; hx = gxh; }
            } else {
                hmode = 1;
                hx = ((gxh % A.nx) + A.nx) % A.nx;
            }
        }

        real p[4][9];
        real hp[9];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 9; ++i) p[j][i] = real(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) hp[i] = real(0);

        // Issue the loads of stencil row yy into dst (own column) / hp (halo).
        auto load_row = [&](int yy, real(&dst)[9]) {
            bool mir;
            const int ysrc = map_row<WALLS>(yy, A.ny, mir);
            if (active) {
                const real *src = A.fin + (long long)ysrc * A.nx + xc;
#pragma unroll
                for (int i = 0; i < 9; ++i) dst[i] = __ldg(src + (long long)i * A.plane);
            }
            if (hmode) {
                const real *src = A.fin + (long long)ysrc * A.nx + hx;
#pragma unroll
                for (int i = 0; i < 9; ++i) hp[i] = __ldg(src + (long long)i * A.plane);
            }
        };

        load_row(ya - 2, p[0]);

        for (int y0 = ya - 2; y0 < yb + 2; y0 += 4) {
#pragma unroll
            for (int J = 0; J < 4; ++J) {
                const int yy = y0 + J;
                if (yy < yb + 2) {
                    bool mir;
                    map_row<WALLS>(yy, A.ny, mir);
                    const real add = mir ? A.wet : real(0);
                    const int rs = yy & (RING - 1);

                    // densities of row yy (own column and halo) before reusing hp
                    real rho_own = real(0);
                    if (active) {
                        real sum = real(0);
#pragma unroll
                        for (int i = 0; i < 9; ++i) sum += p[J][i];
                        rho_own = (pcol ? column_density(A, pout, sum) : sum) + add;
                    }
                    real rho_h = real(0);
                    if (hmode) {
                        real sum = real(0);
#pragma unroll
                        for (int i = 0; i < 9; ++i) sum += hp[i];
                        rho_h = (hmode == 1 ? sum : column_density(A, hmode == 3, sum)) + add;
                    }

                    // prefetch row yy+1 (slot J+1 held row yy-3, already collided)
                    if (yy + 1 < yb + 2) load_row(yy + 1, p[(J + 1) & 3]);

                    if (active) {
                        s_rho[rs][tid + 2] = rho_own;
                        s_phi[rs][tid + 2] = eos_phi(A, rho_own);
                    }
                    if (hmode) {
                        s_rho[rs][hcol] = rho_h;
                        s_phi[rs][hcol] = eos_phi(A, rho_h);
                    }
                    __syncthreads();

                    // Laplacian of row yy-1 on local columns -1 .. xw
                    if (yy >= ya) {
                        const int lr = (yy - 1) & (RING - 1);
                        const int lm = (yy - 2) & (RING - 1), lp = yy & (RING - 1);
                        auto lap_at = [&](int c) {
                            real edges = s_rho[lr][c - 1] + s_rho[lr][c + 1] + s_rho[lm][c] + s_rho[lp][c];
                            real corners = s_rho[lm][c - 1] + s_rho[lm][c + 1] + s_rho[lp][c - 1] + s_rho[lp][c + 1];
                            s_lap[lr][c] = (real(4) * edges + corners - real(20) * s_rho[lr][c]) * sixth;
                        };
                        if (active) lap_at(tid + 2);
                        if (tid == 0) lap_at(1);
                        if (tid == 1) lap_at(xw + 2);
                    }
                    __syncthreads();

                    // collide and stream row r = yy - 2
                    const int r = yy - 2;
                    if (r >= ya && active) {
                        const real(&f)[9] = p[(J + 2) & 3];
                        const int q0 = r & (RING - 1), qm = (r - 1) & (RING - 1), qp = (r + 1) & (RING - 1);
                        const int c = ccol;
                        // isotropic gradients: grad psi = 3 sum_i w_i e_i psi(x + e_i)
                        auto grad = [&](real (*S)[SW], real &gx_, real &gy_) {
                            gx_ = (S[q0][c + 1] - S[q0][c - 1]) * third
                                  + (S[qp][c + 1] - S[qp][c - 1] + S[qm][c + 1] - S[qm][c - 1]) * twelfth;
                            gy_ = (S[qp][c] - S[qm][c]) * third
                                  + (S[qp][c + 1] + S[qp][c - 1] - S[qm][c + 1] - S[qm][c - 1]) * twelfth;
                        };
                        real gpx, gpy, glx, gly;
                        grad(s_phi, gpx, gpy);
                        grad(s_lap, glx, gly);
                        const real rho = s_rho[q0][c];
                        const real rho_b = s_rho[q0][tid + 2];  // pressure column's own density
                        const real Fx = -gpx + A.kappa * rho * glx + A.gx;
                        const real Fy = -gpy + A.kappa * rho * gly + A.gy;
                        const real jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
                        const real jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
                        const real irho = real(1) / rho;
                        const real ux = jx * irho, uy = jy * irho;
                        const real vx = ux + real(0.5) * Fx * irho, vy = uy + real(0.5) * Fy * irho;

                        if (MODE == MODE_STEP) {
                            real fs[9];
                            if (!pcol) {
                                real fe[9];
                                feq9<real>(rho, ux + A.tau * Fx * irho, uy + A.tau * Fy * irho, fe);
#pragma unroll
                                for (int i = 0; i < 9; ++i) fs[i] = f[i] + (fe[i] - f[i]) * A.inv_tau;
                            } else {
                                // non-equilibrium extrapolation from the interior neighbour
                                real fb[9], ff[9];
                                feq9<real>(rho_b, vx, vy, fb);
                                feq9<real>(rho, vx, vy, ff);
#pragma unroll
                                for (int i = 0; i < 9; ++i) fs[i] = fb[i] + A.omb * (f[i] - ff[i]);
                            }
                            // push with half-way bounce-back
                            real *dst = A.fout;
#pragma unroll
                            for (int i = 0; i < 9; ++i) {
                                const int ty = r + ey_(i);
                                if (WALLS && (ty == 0 || ty == A.ny - 1)) {
                                    dst[(long long)opp_(i) * A.plane + (long long)r * A.nx + x] = fs[i];
                                } else {
                                    int tx = x + ex_(i);
                                    if (PRES) {
                                        if (tx < 0 || tx >= A.nx) continue;
                                    } else {
                                        tx = tx < 0 ? tx + A.nx : (tx >= A.nx ? tx - A.nx : tx);
                                    }
                                    int tyw = ty;
                                    if (!WALLS) tyw = ty < 0 ? ty + A.ny : (ty >= A.ny ? ty - A.ny : ty);
                                    dst[(long long)i * A.plane + (long long)tyw * A.nx + tx] = fs[i];
                                }
                            }
                            mass += (double)(pcol ? rho_b : rho);
                            if (!(rho > real(0)) || !(rho < real(1e30))) bad = true;
                        } else {
                            const long long o = (long long)r * A.nx + x;
                            A.o_rho[o] = pcol ? rho_b : rho;
                            A.o_vx[o] = vx;
                            A.o_vy[o] = vy;
                        }

                        if (WALLS && !pcol) {
                            // wall shear: quadratic through v = 0 on the half-way plane
                            // and v at distances 1/2, 3/2 (reading of Fig. 3's tau_w)
                            auto pwall = [&]() {
                                real grx, gry;
                                grad(s_rho, grx, gry);
                                return s_phi[q0][c] + rho * third - A.kappa * rho * s_lap[q0][c]
                                       - real(0.5) * A.kappa * (grx * grx + gry * gry);
                            };
                            if (r == 1) {
                                b_rho1 = rho;
                                b_v1 = vx;
                                const real pw = pwall();
                                if (MODE == MODE_STEP) { pmin = fmin(pmin, pw); pmax = fmax(pmax, pw); }
                                else A.o_pw[x] = pw;
                            }
                            if (r == A.ny - 3) t_v2 = vx;
                            if (r == 2) {
                                const real tw = b_rho1 * A.nu * (real(9) * b_v1 - vx) * third;
                                if (MODE == MODE_STEP) { Jsum += (double)tw; tmin = fmin(tmin, tw); tmax = fmax(tmax, tw); }
                                else A.o_tw[x] = tw;
                            }
                            if (r == A.ny - 2) {
                                const real tw = rho * A.nu * (real(9) * vx - t_v2) * third;
                                const real pw = pwall();
                                if (MODE == MODE_STEP) {
                                    Jsum += (double)tw;
                                    tmin = fmin(tmin, tw); tmax = fmax(tmax, tw);
                                    pmin = fmin(pmin, pw); pmax = fmax(pmax, pw);
                                } else {
                                    A.o_tw[A.nx + x] = tw;
                                    A.o_pw[A.nx + x] = pw;
                                }
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();  // ring reuse by the next segment
    }

    if (MODE != MODE_STEP) return;

    // CTA reduction in a fixed order (deterministic for a fixed schedule)
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mass += __shfl_xor_sync(0xffffffffu, mass, o);
        Jsum += __shfl_xor_sync(0xffffffffu, Jsum, o);
        tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
        tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        pmin = fmin(pmin, __shfl_xor_sync(0xffffffffu, pmin, o));
        pmax = fmax(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
    }
    const bool anybad = __any_sync(0xffffffffu, bad);
    if (tid == 0) s_bad = 0;
    __syncthreads();
    if (lane == 0) {
        s_red[warp][0] = mass;
        s_red[warp][1] = Jsum;
        s_ext[warp][0] = tmin; s_ext[warp][1] = tmax;
        s_ext[warp][2] = pmin; s_ext[warp][3] = pmax;
        if (anybad) atomicOr(&s_bad, 1);
    }
    __syncthreads();
    if (tid == 0) {
        double m = 0.0, j = 0.0;
        real e0 = s_ext[0][0], e1 = s_ext[0][1], e2 = s_ext[0][2], e3 = s_ext[0][3];
        for (int w = 0; w < BLOCK / 32; ++w) {
            m += s_red[w][0];
            j += s_red[w][1];
            e0 = fmin(e0, s_ext[w][0]); e1 = fmax(e1, s_ext[w][1]);
            e2 = fmin(e2, s_ext[w][2]); e3 = fmax(e3, s_ext[w][3]);
        }
        A.mass_part[cta] = m;
        A.J_acc[cta] += j;
        real *e = A.ext + 4 * cta;
        e[0] = fmin(e[0], e0); e[1] = fmax(e[1], e1);
        e[2] = fmin(e[2], e2); e[3] = fmax(e[3], e3);
        if (s_bad) atomicOr(A.err, 1);
    }
}

// f = f_eq(rho0, 0) at every node.
template <typename real>
__global__ void init_kernel(const double *__restrict__ rho0, real *__restrict__ fa,
                            real *__restrict__ fb, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        real fe[9];
        feq9<real>((real)rho0[k], real(0), real(0), fe);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fa[i * n + k] = fe[i];
            fb[i * n + k] = fe[i];
        }
    }
}

// Fixed-order reduction of the per-CTA partials into out[0..6]:
// mass, J, tw_min, tw_max, pw_min, pw_max, err.
template <typename real>
__global__ void diag_kernel(const double *__restrict__ mass_part, const double *__restrict__ J_acc,
                            const real *__restrict__ ext, const int *__restrict__ err, int nctas,
                            double *__restrict__ out)
{
    __shared__ double sm[256], sj[256], se[4][256];
    const int t = threadIdx.x;
    double m = 0.0, j = 0.0;
    double e0 = INFINITY, e1 = -INFINITY, e2 = INFINITY, e3 = -INFINITY;
    for (int c = t; c < nctas; c += 256) {
        m += mass_part[c];
        j += J_acc[c];
        e0 = fmin(e0, (double)ext[4 * c + 0]);
        e1 = fmax(e1, (double)ext[4 * c + 1]);
        e2 = fmin(e2, (double)ext[4 * c + 2]);
        e3 = fmax(e3, (double)ext[4 * c + 3]);
    }
    sm[t] = m; sj[t] = j; se[0][t] = e0; se[1][t] = e1; se[2][t] = e2; se[3][t] = e3;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) {
            sm[t] += sm[t + s];
            sj[t] += sj[t + s];
            se[0][t] = fmin(se[0][t], se[0][t + s]);
            se[1][t] = fmax(se[1][t], se[1][t + s]);
            se[2][t] = fmin(se[2][t], se[2][t + s]);
            se[3][t] = fmax(se[3][t], se[3][t + s]);
        }
        __syncthreads();
    }
    if (t == 0) {
        out[0] = sm[0]; out[1] = sj[0];
        out[2] = se[0][0]; out[3] = se[1][0]; out[4] = se[2][0]; out[5] = se[3][0];
        out[6] = (double)(*err);
    }
}

template <typename real>
__global__ void reset_acc_kernel(double *mass_part, double *J_acc, real *ext, int *err, int n)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        mass_part[c] = 0.0;
        J_acc[c] = 0.0;
        ext[4 * c + 0] = real(INFINITY);
        ext[4 * c + 1] = real(-INFINITY);
        ext[4 * c + 2] = real(INFINITY);
        ext[4 * c + 3] = real(-INFINITY);
        if (c == 0) *err = 0;
    }
}

} // namespace lbm
