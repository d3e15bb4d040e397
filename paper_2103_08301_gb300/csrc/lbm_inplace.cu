// In-place streaming for single contexts: one population array instead of
// two (the AA pattern, Bailey, Myre, Walsh, Lilja and Wilson, ICPP 2009),
// plus a density plane.
//
// Even steps find the natural layout, F[x][i] = f_i(x): a node reads its own
// nine slots and writes its post-collision populations back reversed,
// F[x][opp(i)] = f*_i(x). Odd steps read f_i(x) from F[x - e_i][opp(i)] and
// write f*_i(x) to F[x + e_i][i], which restores the natural layout. Each slot
// is read and written by one node only, so neither step races. Half-way
// bounce-back (Sec. 2.2 walls) writes into the wall row's slot on even steps
// (F[x + e_i][i]) and into the node's own reversed slot on odd steps; the
// populations that leave through a pressure column are dropped.
//
// The force of Eq. 2.17 reads densities up to two nodes away, and in place a
// neighbour's slots may already hold its next state, so every step first
// writes the density sum of each fluid node into a plane of its own
// (aa_density_kernel) and then collides from that plane (aa_step_kernel_f2
// for FP32, two rows per thread on the paired FP32 instructions, and
// aa_step_kernel for FP64, one node per thread; a CTA takes one 32 x 8 tile at
// a time). A pressure column collides with its interior neighbour's
// populations (Sec. 2.2 pressure-driven ends); the density pass copies those
// into a side buffer, for the same reason.
//
// The node arithmetic is the one-row step kernel's helper sequence, in the
// same order and precision, so the populations match the two-array step bit
// for bit; only the summation order of the diagnostics differs.
//
// Traffic per node and step (FP32): 36 B read and 4 B written by the density
// pass, 36 B read, 36 B written and 4 B of densities read by the step, 116 B
// against the two-array step's 72 B; storage 40 B against 72 B.

#include <cuda_runtime.h>

#include <algorithm>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

constexpr int AA_TX = 32;                   // tile columns: one warp
constexpr int AA_TY = 8;                    // tile rows: one warp each
constexpr int AA_THREADS = AA_TX * AA_TY;   // one node per thread
constexpr int AA_SW = AA_TX + 4;            // ring columns x0-2 .. x0+AA_TX+1
constexpr int AA_ROWS = AA_TY + 4;          // ring rows y0-2 .. y0+AA_TY+1
// resident CTAs per SM the one-node-per-thread step is compiled for: 4 (64
// registers) measured fastest on 16384 x 2048 FP32 (0.992 ms against 1.20 ms
// at 80 registers and 3 CTAs, 1.15 ms at 5 CTAs with spills); FP32 contexts
// now step with the row-pair kernel below, FP64 ones with this kernel
#ifndef LBM_AA_MIN_BLOCKS
#define LBM_AA_MIN_BLOCKS 4
#endif

template <typename real>
struct SmemAA {
    real rho[AA_ROWS][AA_SW];
    real phi[AA_ROWS][AA_SW];
    real lap[AA_ROWS][AA_SW];
    real brho1[AA_TX], bv1[AA_TX], tv2[AA_TX];  // row 1 (rho, v) and row ny-3 (v) for the wall shear
    double red[AA_THREADS / 32][2];
    real ext[AA_THREADS / 32][4];
    int bad;
};

// x +- 1 on a periodic axis of n nodes (n >= 1)
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// offset of slot (x, y, i): rows of nine planes of pitch P
template <typename IX>
__device__ __forceinline__ IX aa_slot(int x, int y, int i, int P)
{
    return (IX)y * (IX)(9 * (IX)P) + (IX)i * P + x;
}

// Density sum of every fluid node into rho (plane pitch P), in the step
// kernels' summation order; pressure columns are skipped (their density is
// derived from the neighbour's), and the populations of columns 1 and nx-2
// go to side[2][ny][9] for the pressure columns' extrapolation.
template <typename real, bool WALLS, bool PRES, bool ODD, typename IX>
__global__ void __launch_bounds__(256) aa_density_kernel(const real *F, real *rho, real *side, int nx, int ny, int P,
                                                         int yf0, int nyf)
{
    const long long n = (long long)nx * nyf;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int yl = (int)(k / nx), x = (int)(k - (long long)yl * nx), y = yf0 + yl;
        if (PRES && (x == 0 || x == nx - 1)) continue;
        real f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (ODD) {
                // interior columns of a channel with pressure columns, and the
                // fluid rows of a walled one, have all their sources in the array
                const int sx = PRES ? x - ex_(i) : wrap1(x - ex_(i), nx);
                const int sy = WALLS ? y - ey_(i) : wrap1(y - ey_(i), ny);
                f[i] = F[aa_slot<IX>(sx, sy, opp_(i), P)];
            } else {
                f[i] = F[aa_slot<IX>(x, y, i, P)];
            }
        }
        real sum = add_(add_(add_(f[0], f[1]), add_(f[2], f[3])), add_(add_(f[4], f[5]), add_(f[6], f[7])));
        sum = add_(sum, f[8]);
        rho[(IX)y * P + x] = sum;
        if (PRES && (x == 1 || x == nx - 2)) {
            real *s = side + ((size_t)(x == 1 ? 0 : 1) * ny + y) * 9;
#pragma unroll
            for (int i = 0; i < 9; ++i) s[i] = f[i];
        }
    }
}

// Odd-parity layout <-> natural layout, in place: the slots (x, i) and
// (x - e_i, opp(i)) trade values, one thread per representative i in
// {1, 2, 5, 6}. Pairs with a slot outside the array (beyond a pressure
// column or a wall row) hold no population that is ever read and stay.
template <typename real, bool WALLS, bool PRES, typename IX>
__global__ void __launch_bounds__(256) aa_swap_kernel(real *F, int nx, int ny, int P)
{
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / nx), x = (int)(k - (long long)y * nx);
        const int rep[4] = {1, 2, 5, 6};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = rep[r];
            int sx = x - ex_(i), sy = y - ey_(i);
            if (PRES) { if (sx < 0 || sx >= nx) continue; }
            else sx = wrap1(sx, nx);
            if (WALLS) { if (sy < 0 || sy >= ny) continue; }
            else sy = wrap1(sy, ny);
            const IX a = aa_slot<IX>(x, y, i, P), b = aa_slot<IX>(sx, sy, opp_(i), P);
            const real t = F[a];
            F[a] = F[b];
            F[b] = t;
        }
    }
}

// Tile grid of the step: ntx x nty tiles of AA_TX x AA_TY nodes, the first
// starting sx columns left of column 0 and sy rows below the first fluid row.
// The shifts keep the outlet column off a tile's first lane (its stencil is
// its neighbour's, which reaches two columns back) and the wall-shear rows
// ny-3 | ny-2 in one tile (rows 1 | 2 always are).
struct AATiles {
    int ntx, nty, sx, sy;
};

// One step of the interior of every tile (the FP64 in-place step; FP32 takes
// aa_step_kernel_f2 below), CTAs striding over the tiles: (1) densities (with
// the mirror, pressure-column and periodic rules of the stencil) and the EOS
// potential on the tile plus two halo nodes, (2) the Laplacian on the tile
// plus one, (3) force, collision, boundaries and the in-place write of each
// node (one per thread), then the diagnostics.
template <typename real, bool WALLS, bool PRES, bool ODD, typename IX>
__global__ void __launch_bounds__(AA_THREADS, LBM_AA_MIN_BLOCKS)
    aa_step_kernel(const KArgs<real> A, real *F, const real *rho_in, const real *side, const AATiles T)
{
    __shared__ SmemAA<real> S;
    const int tid = threadIdx.x, lane = tid & 31, rl = tid >> 5;
    const int nx = A.nx, ny = A.ny, P = A.pitch;
    const real third = real(1.0 / 3.0);
    const Geom<real> G{nullptr, nullptr, nx, ny, A.W, P, A.rho_in_g, A.rho_in_l, A.rho_out_g, A.rho_out_l};
    const int yf0 = A.yf0, yf1 = A.yf0 + A.nyf;
    Acc<real, 1> acc;
    acc.reset();
    const long long ntiles = (long long)T.ntx * T.nty;
    constexpr int RN = (AA_ROWS * AA_SW + AA_THREADS - 1) / AA_THREADS;  // ring entries per thread
    struct TileGeom {
        int x0, y0, ylo, yhi;  // origin, and the stencil rows its fluid rows read
    };
    auto tile_geom = [&](long long t) {
        const int ty = (int)(t / T.ntx), tx = (int)(t - (long long)ty * T.ntx);
        TileGeom g;
        g.x0 = tx * AA_TX - T.sx;
        g.y0 = yf0 - T.sy + ty * AA_TY;
        g.ylo = max(g.y0, yf0) - 2;
        g.yhi = min(g.y0 + AA_TY, yf1) + 1;
        return g;
    };
    // the populations of this thread's node (x0 + lane, y0 + rl) of a tile
    auto load_f = [&](const TileGeom &g, real (&f)[9]) {
        const int x = g.x0 + lane, y = g.y0 + rl;
        if (!(x >= 0 && x < nx && y >= yf0 && y < yf1)) return;
        if (PRES && (x == 0 || x == nx - 1)) {
            const real *s = side + ((size_t)(x == 0 ? 0 : 1) * ny + y) * 9;
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = s[i];
            return;
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (ODD) {
                const int sx = PRES ? x - ex_(i) : wrap1(x - ex_(i), nx);
                const int sy = WALLS ? y - ey_(i) : wrap1(y - ey_(i), ny);
                f[i] = F[aa_slot<IX>(sx, sy, opp_(i), P)];
            } else {
                f[i] = F[aa_slot<IX>(x, y, i, P)];
            }
        }
    };
    // the stored density sums behind this thread's ring entries k = tid + q
    // AA_THREADS (ring row j = stencil row y0-2+j, column c = x0-2+c): the
    // mirrored row, the pressure column's interior neighbour, the periodic image
    auto load_ring = [&](const TileGeom &g, real (&r)[RN]) {
#pragma unroll
        for (int q = 0; q < RN; ++q) {
            const int k = tid + q * AA_THREADS;
            const int j = k / AA_SW, c = k - j * AA_SW;
            const int yy = g.y0 - 2 + j, gc = g.x0 - 2 + c;
            r[q] = real(0);
            if (k < AA_ROWS * AA_SW && yy >= g.ylo && yy <= g.yhi) {
                bool mir;
                const int row = map_row<WALLS>(yy, ny, mir);
                int col;
                if (PRES) {
                    col = gc <= 0 ? 1 : (gc >= nx - 1 ? nx - 2 : gc);
                } else {
                    col = gc % nx;
                    col = col < 0 ? col + nx : col;
                }
                r[q] = rho_in[(IX)row * P + col];
            }
        }
    };

    // CTAs stride over the tiles in row-major order, so that at any time the
    // grid works on a few rows of tiles whose halos meet in L2; software
    // pipeline: the next tile's populations and densities are loaded while
    // this tile computes
    long long t = blockIdx.x;
    TileGeom gcur{0, 0, 0, 0};
    real fcur[9], rcur[RN];
#pragma unroll
    for (int i = 0; i < 9; ++i) fcur[i] = real(0);
    if (t < ntiles) {
        gcur = tile_geom(t);
        load_f(gcur, fcur);
        load_ring(gcur, rcur);
    }
    for (; t < ntiles; t += gridDim.x) {
        TileGeom gnext = gcur;
        real fnext[9], rnext[RN];
#pragma unroll
        for (int i = 0; i < 9; ++i) fnext[i] = real(0);
        if (t + gridDim.x < ntiles) {
            gnext = tile_geom(t + gridDim.x);
            load_f(gnext, fnext);
            load_ring(gnext, rnext);
        }
        const int x0 = gcur.x0, y0 = gcur.y0;
        const int x = x0 + lane, y = y0 + rl;
        const bool active = x >= 0 && x < nx && y >= yf0 && y < yf1;
        const bool pin = PRES && x == 0, pout = PRES && x == nx - 1, anyp = pin || pout;
        const int lcol = (pin ? 1 : (pout ? nx - 2 : x)) - x0;  // a pressure column collides its neighbour
        const int ccol = lcol + 2;
        const int q0 = rl + 2, qm = q0 - 1, qp = q0 + 1;

        // (1) densities (mirror offset, pressure-column density) and phi of the ring
#pragma unroll
        for (int q = 0; q < RN; ++q) {
            const int k = tid + q * AA_THREADS;
            if (k < AA_ROWS * AA_SW) {
                const int j = k / AA_SW, c = k - j * AA_SW;
                const int yy = y0 - 2 + j, gc = x0 - 2 + c;
                real rho_c = real(0), ph = real(0);
                if (yy >= gcur.ylo && yy <= gcur.yhi) {
                    bool mir;
                    map_row<WALLS>(yy, ny, mir);
                    real v = rcur[q];
                    if (PRES) {
                        if (gc <= 0) v = column_density(A, G, false, v);
                        else if (gc >= nx - 1) v = column_density(A, G, true, v);
                    }
                    rho_c = add_(v, mir ? A.wet : real(0));
                    ph = eos_phi<real>(A, rho_c);
                }
                S.rho[j][c] = rho_c;
                S.phi[j][c] = ph;
            }
        }
        __syncthreads();

        // (2) Laplacian at ring rows 1 .. AA_ROWS-2, columns 1 .. AA_SW-2
        for (int k = tid; k < (AA_ROWS - 2) * (AA_SW - 2); k += AA_THREADS) {
            const int j = 1 + k / (AA_SW - 2), c = 1 + k % (AA_SW - 2);
            S.lap[j][c] = lap9<real>(row3<real, 1, AA_SW>(S.rho, j - 1, c), row3<real, 1, AA_SW>(S.rho, j, c),
                                     row3<real, 1, AA_SW>(S.rho, j + 1, c));
        }
        __syncthreads();

        // (3) force, collision, boundaries and the in-place write of the node
        real rho = real(0), vx = real(0);
        if (active) {
            const real (&f)[9] = fcur;
            real ngpx, ngpy, glx, gly;
            ngrad12<real>(row3<real, 1, AA_SW>(S.phi, qm, ccol), row3<real, 1, AA_SW>(S.phi, q0, ccol),
                          row3<real, 1, AA_SW>(S.phi, qp, ccol), ngpx, ngpy);
            grad12<real>(row3<real, 1, AA_SW>(S.lap, qm, ccol), row3<real, 1, AA_SW>(S.lap, q0, ccol),
                         row3<real, 1, AA_SW>(S.lap, qp, ccol), glx, gly);
            rho = S.rho[q0][ccol];
            const real kr = mul_(A.kappa, rho);
            const real Fx = add_(mulk(fma_(kr, glx, ngpx), 1.0 / 12.0), A.gx);
            const real Fy = add_(mulk(fma_(kr, gly, ngpy), 1.0 / 12.0), A.gy);
            const real jx = add_(add_(sub_(f[1], f[3]), sub_(f[5], f[6])), sub_(f[8], f[7]));
            const real jy = sub_(add_(sub_(f[2], f[4]), add_(f[5], f[6])), add_(f[7], f[8]));
            const real irho = rcp_(rho);
            const real ux = mul_(jx, irho), uy = mul_(jy, irho);
            const real hFi = mul_(irho, bc<real>(0.5));
            vx = fma_(hFi, Fx, ux);
            const real vy = fma_(hFi, Fy, uy);
            const real rho_own = anyp ? S.rho[q0][lane + 2] : rho;  // a pressure column's own is rho_b

            real fs[9];
            {
                // shifted equilibrium: momentum j + ushift F, velocity (j + ushift F) / rho
                const real mx = fma_(A.ushift, Fx, jx), my = fma_(A.ushift, Fy, jy);
                real fe[9];
                feq_pairs<real>(rho, mul_(mx, irho), mul_(my, irho), mx, my, fe);
                if (A.mrt) {
                    mrt_relax<real, real>(A, f, fe, fs);
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) fs[i] = fma_(sub_(fe[i], f[i]), A.inv_tau, f[i]);
                }
            }
            if (anyp) {
                // extrapolation from the interior neighbour, momentum of v = (j + F/2) / rho
                const real mvx = fma_(real(0.5), Fx, jx), mvy = fma_(real(0.5), Fy, jy);
                real fsc[9];
                column_extrapolate<real>(A, rho_own, rho, vx, vy, mvx, mvy, f, fsc);
#pragma unroll
                for (int i = 0; i < 9; ++i) fs[i] = fsc[i];
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int ty2 = y + ey_(i);
                const bool wall = WALLS && (ty2 == 0 || ty2 == ny - 1);
                int tx2 = x + ex_(i);
                bool inx = true;
                if (PRES) inx = tx2 >= 0 && tx2 < nx;
                else tx2 = wrap1(tx2, nx);
                const int tyw = WALLS ? ty2 : wrap1(ty2, ny);
                if (ODD) {
                    if (wall) F[aa_slot<IX>(x, y, opp_(i), P)] = fs[i];
                    else if (inx) F[aa_slot<IX>(tx2, tyw, i, P)] = fs[i];  // else it leaves through the column
                } else {
                    if (wall) {
                        if (inx) F[aa_slot<IX>(tx2, ty2, i, P)] = fs[i];
                    } else {
                        F[aa_slot<IX>(x, y, opp_(i), P)] = fs[i];
                    }
                }
            }
            acc.macc = add_(acc.macc, rho_own);
            acc.rmin = vmin_(acc.rmin, rho);
            acc.rmax = vmax_(acc.rmax, rho);
            if (WALLS && !anyp) {
                if (y == 1) { S.brho1[lane] = rho; S.bv1[lane] = vx; }
                if (y == ny - 3) S.tv2[lane] = vx;
            }
        }
        acc.flush();
        if (WALLS) {
            __syncthreads();  // rows 1 and ny-3 of the tile published
            if (active && !anyp && (y == 1 || y == 2 || y == ny - 2)) {
                // wall shear: quadratic through v = 0 on the half-way plane and
                // v at distances 1/2 and 3/2; wall pressure: Eq. 2.4 in mesh units
                if (y == 1) {
                    const real pw = wall_pressure<real, AA_SW>(A, S.rho, S.phi, S.lap[q0][ccol], qm, q0, qp, ccol, rho);
                    acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw);
                }
                if (y == 2) {
                    const real tw = mul_(mul_(S.brho1[lane], A.nu), mul_(fma_(real(9), S.bv1[lane], -vx), third));
                    acc.J += (double)tw; acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw);
                }
                if (y == ny - 2) {
                    const real tw = mul_(mul_(rho, A.nu), mul_(fma_(real(9), vx, -S.tv2[lane]), third));
                    const real pw = wall_pressure<real, AA_SW>(A, S.rho, S.phi, S.lap[q0][ccol], qm, q0, qp, ccol, rho);
                    acc.J += (double)tw;
                    acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw);
                    acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw);
                }
            }
        }
        __syncthreads();  // the ring is rewritten by the next tile
        gcur = gnext;
#pragma unroll
        for (int i = 0; i < 9; ++i) fcur[i] = fnext[i];
#pragma unroll
        for (int q = 0; q < RN; ++q) rcur[q] = rnext[q];
    }

    double m, j;
    real e[4];
    bool anybad;
    cta_reduce<real, AA_THREADS, 1>(acc, S, m, j, e, anybad);
    if (tid == 0) {
        const int cta = blockIdx.x;
        A.mass_part[cta] = m;
        A.J_acc[cta] += j;
        real *ex = A.ext + 4 * cta;
        ex[0] = fmin(ex[0], e[0]); ex[1] = fmax(ex[1], e[1]);
        ex[2] = fmin(ex[2], e[2]); ex[3] = fmax(ex[3], e[3]);
        if (anybad) atomicOr(A.err, 1);
    }
}


// The FP32 step with two rows per thread: the same phases, with the ring's
// densities, EOS potential and Laplacian and the node arithmetic on the paired
// FP32 instructions, which round each element as the scalar instruction does,
// so the populations are the scalar kernel's bit for bit. 128 threads: lane =
// column, warp = row pair of the 32 x 8 tile.
// The next tile's halo densities are loaded while the current tile computes;
// its populations too with LBM_AA2_PREFETCH_F = 1 (else each tile loads its
// own at its start). Measured per 16384 x 2048 step: populations at the tile's
// start, 5 CTAs per SM (88 registers) 0.837 ms (kept); 6 CTAs (80 registers,
// small spills) 0.932 ms; populations prefetched, 4 CTAs (118 registers)
// 0.882 ms, 5 CTAs (96 registers, spills) 1.017 ms.
constexpr int AA2_THREADS = AA_TX * AA_TY / 2;
#ifndef LBM_AA2_MIN_BLOCKS
#define LBM_AA2_MIN_BLOCKS 5
#endif
#ifndef LBM_AA2_PREFETCH_F
#define LBM_AA2_PREFETCH_F 0
#endif

// West, centre and east float2 packs (ring rows ra, rb) of ring column c.
__device__ __forceinline__ Row3<float2> aa_row3p(const float (*S)[AA_SW], int ra, int rb, int c)
{
    Row3<float2> r;
    r.w = make_float2(S[ra][c - 1], S[rb][c - 1]);
    r.c = make_float2(S[ra][c], S[rb][c]);
    r.e = make_float2(S[ra][c + 1], S[rb][c + 1]);
    return r;
}

template <bool WALLS, bool PRES, bool ODD, typename IX>
__global__ void __launch_bounds__(AA2_THREADS, LBM_AA2_MIN_BLOCKS)
    aa_step_kernel_f2(const KArgs<float> A, float *F, const float *rho_in, const float *side, const AATiles T)
{
    using V = float2;
    __shared__ SmemAA<float> S;
    const int tid = threadIdx.x, lane = tid & 31, pr = tid >> 5;
    const int nx = A.nx, ny = A.ny, P = A.pitch;
    const float third = 1.0f / 3.0f;
    const Geom<float> G{nullptr, nullptr, nx, ny, A.W, P, A.rho_in_g, A.rho_in_l, A.rho_out_g, A.rho_out_l};
    const int yf0 = A.yf0, yf1 = A.yf0 + A.nyf;
    Acc<float, 1> acc;
    acc.reset();
    const long long ntiles = (long long)T.ntx * T.nty;
    constexpr int NP = (AA_ROWS / 2) * AA_SW;                  // ring entries as row pairs
    constexpr int RN = (NP + AA2_THREADS - 1) / AA2_THREADS;   // per thread
    struct TileGeom {
        int x0, y0, ylo, yhi;  // origin, and the stencil rows its fluid rows read
    };
    auto tile_geom = [&](long long t) {
        const int ty = (int)(t / T.ntx), tx = (int)(t - (long long)ty * T.ntx);
        TileGeom g;
        g.x0 = tx * AA_TX - T.sx;
        g.y0 = yf0 - T.sy + ty * AA_TY;
        g.ylo = max(g.y0, yf0) - 2;
        g.yhi = min(g.y0 + AA_TY, yf1) + 1;
        return g;
    };
    // the populations of this thread's nodes (x0 + lane, y0 + 2 pr + e)
    auto load_f = [&](const TileGeom &g, V (&f)[9]) {
        const int x = g.x0 + lane;
        if (x < 0 || x >= nx) return;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int y = g.y0 + 2 * pr + e;
            if (y < yf0 || y >= yf1) continue;
            if (PRES && (x == 0 || x == nx - 1)) {
                const float *s = side + ((size_t)(x == 0 ? 0 : 1) * ny + y) * 9;
#pragma unroll
                for (int i = 0; i < 9; ++i) set_el(f[i], e, s[i]);
                continue;
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if (ODD) {
                    const int sx = PRES ? x - ex_(i) : wrap1(x - ex_(i), nx);
                    const int sy = WALLS ? y - ey_(i) : wrap1(y - ey_(i), ny);
                    set_el(f[i], e, F[aa_slot<IX>(sx, sy, opp_(i), P)]);
                } else {
                    set_el(f[i], e, F[aa_slot<IX>(x, y, i, P)]);
                }
            }
        }
    };
    // the stored density sums behind this thread's ring pair entries k = tid +
    // q AA2_THREADS (ring rows 2 jp, 2 jp + 1, column c)
    auto load_ring = [&](const TileGeom &g, V (&r)[RN]) {
#pragma unroll
        for (int q = 0; q < RN; ++q) {
            const int k = tid + q * AA2_THREADS;
            const int jp = k / AA_SW, c = k - jp * AA_SW;
            const int gc = g.x0 - 2 + c;
            int col;
            if (PRES) {
                col = gc <= 0 ? 1 : (gc >= nx - 1 ? nx - 2 : gc);
            } else {
                col = gc % nx;
                col = col < 0 ? col + nx : col;
            }
            r[q] = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int yy = g.y0 - 2 + 2 * jp + e;
                if (k < NP && yy >= g.ylo && yy <= g.yhi) {
                    bool mir;
                    const int row = map_row<WALLS>(yy, ny, mir);
                    set_el(r[q], e, rho_in[(IX)row * P + col]);
                }
            }
        }
    };

    long long t = blockIdx.x;
    TileGeom gcur{0, 0, 0, 0};
    V fcur[9], rcur[RN];
#pragma unroll
    for (int i = 0; i < 9; ++i) fcur[i] = make_float2(0.f, 0.f);
    constexpr bool PF = LBM_AA2_PREFETCH_F != 0;
    if (t < ntiles) {
        gcur = tile_geom(t);
        if (PF) load_f(gcur, fcur);
        load_ring(gcur, rcur);
    }
    for (; t < ntiles; t += gridDim.x) {
        if (!PF) load_f(gcur, fcur);
        TileGeom gnext = gcur;
        V fnext[9], rnext[RN];
#pragma unroll
        for (int i = 0; i < 9; ++i) fnext[i] = make_float2(0.f, 0.f);
        if (t + gridDim.x < ntiles) {
            gnext = tile_geom(t + gridDim.x);
            if (PF) load_f(gnext, fnext);
            load_ring(gnext, rnext);
        }
        const int x0 = gcur.x0, y0 = gcur.y0;

        // (1) densities (mirror offset, pressure-column density) and phi of the ring
#pragma unroll
        for (int q = 0; q < RN; ++q) {
            const int k = tid + q * AA2_THREADS;
            if (k < NP) {
                const int jp = k / AA_SW, c = k - jp * AA_SW, j = 2 * jp;
                const int gc = x0 - 2 + c;
                bool in[2], mir[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int yy = y0 - 2 + j + e;
                    in[e] = yy >= gcur.ylo && yy <= gcur.yhi;
                    map_row<WALLS>(yy, ny, mir[e]);
                }
                V v = rcur[q];
                if (PRES && (gc <= 0 || gc >= nx - 1)) {
                    v.x = column_density(A, G, gc > 0, v.x);
                    v.y = column_density(A, G, gc > 0, v.y);
                }
                const V rho_c = add_(v, make_float2(mir[0] ? A.wet : 0.f, mir[1] ? A.wet : 0.f));
                const V ph = eos_phi<V>(A, rho_c);
                S.rho[j][c] = in[0] ? rho_c.x : 0.f;
                S.rho[j + 1][c] = in[1] ? rho_c.y : 0.f;
                S.phi[j][c] = in[0] ? ph.x : 0.f;
                S.phi[j + 1][c] = in[1] ? ph.y : 0.f;
            }
        }
        __syncthreads();

        // (2) Laplacian at ring rows 1 .. AA_ROWS-2 in pairs, columns 1 .. AA_SW-2
        for (int k = tid; k < ((AA_ROWS - 2) / 2) * (AA_SW - 2); k += AA2_THREADS) {
            const int j = 1 + 2 * (k / (AA_SW - 2)), c = 1 + k % (AA_SW - 2);
            const V L = lap9<V>(aa_row3p(S.rho, j - 1, j, c), aa_row3p(S.rho, j, j + 1, c),
                                aa_row3p(S.rho, j + 1, j + 2, c));
            S.lap[j][c] = L.x;
            S.lap[j + 1][c] = L.y;
        }
        __syncthreads();

        // (3) force, collision, boundaries and the in-place write of the nodes
        //     (x, b) and (x, b + 1)
        const int x = x0 + lane, b = y0 + 2 * pr;
        const bool xin = x >= 0 && x < nx;
        const bool act0 = xin && b >= yf0 && b < yf1, act1 = xin && b + 1 >= yf0 && b + 1 < yf1;
        const bool pin = PRES && x == 0, pout = PRES && x == nx - 1, anyp = pin || pout;
        const int lcol = (pin ? 1 : (pout ? nx - 2 : x)) - x0;  // a pressure column collides its neighbour
        const int ccol = lcol + 2;
        const int q0 = 2 * pr + 2, qm = q0 - 1, q1 = q0 + 1, q2 = q0 + 2;  // ring rows of b-1 .. b+2
        V rho = make_float2(0.f, 0.f), vx = rho;
        if (act0 || act1) {
            const V (&f)[9] = fcur;
            V ngpx, ngpy, glx, gly;
            ngrad12<V>(aa_row3p(S.phi, qm, q0, ccol), aa_row3p(S.phi, q0, q1, ccol), aa_row3p(S.phi, q1, q2, ccol),
                       ngpx, ngpy);
            grad12<V>(aa_row3p(S.lap, qm, q0, ccol), aa_row3p(S.lap, q0, q1, ccol), aa_row3p(S.lap, q1, q2, ccol),
                      glx, gly);
            rho = make_float2(S.rho[q0][ccol], S.rho[q1][ccol]);
            const V kr = mul_(bcr<V>(A.kappa), rho);
            const V Fx = add_(mulk(fma_(kr, glx, ngpx), 1.0 / 12.0), bcr<V>(A.gx));
            const V Fy = add_(mulk(fma_(kr, gly, ngpy), 1.0 / 12.0), bcr<V>(A.gy));
            const V jx = add_(add_(sub_(f[1], f[3]), sub_(f[5], f[6])), sub_(f[8], f[7]));
            const V jy = sub_(add_(sub_(f[2], f[4]), add_(f[5], f[6])), add_(f[7], f[8]));
            const V irho = rcp_(rho);
            const V ux = mul_(jx, irho), uy = mul_(jy, irho);
            const V hFi = mul_(irho, bc<V>(0.5));
            vx = fma_(hFi, Fx, ux);
            const V vy = fma_(hFi, Fy, uy);
            const V rho_own = anyp ? make_float2(S.rho[q0][lane + 2], S.rho[q1][lane + 2]) : rho;

            V fs[9];
            {
                // shifted equilibrium: momentum j + ushift F, velocity (j + ushift F) / rho
                const V mx = fma_(bcr<V>(A.ushift), Fx, jx), my = fma_(bcr<V>(A.ushift), Fy, jy);
                V fe[9];
                feq_pairs<V>(rho, mul_(mx, irho), mul_(my, irho), mx, my, fe);
                if (A.mrt) {
                    mrt_relax<V, float>(A, f, fe, fs);
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) fs[i] = fma_(sub_(fe[i], f[i]), bcr<V>(A.inv_tau), f[i]);
                }
            }
            if (anyp) {
                // extrapolation from the interior neighbour, row by row
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    float ff[9], fsc[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) ff[i] = el(f[i], e);
                    const float mvx = fma_(0.5f, el(Fx, e), el(jx, e));
                    const float mvy = fma_(0.5f, el(Fy, e), el(jy, e));
                    column_extrapolate<float>(A, el(rho_own, e), el(rho, e), el(vx, e), el(vy, e), mvx, mvy, ff, fsc);
#pragma unroll
                    for (int i = 0; i < 9; ++i) set_el(fs[i], e, fsc[i]);
                }
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (!(e ? act1 : act0)) continue;
                const int y = b + e;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int ty2 = y + ey_(i);
                    const bool wall = WALLS && (ty2 == 0 || ty2 == ny - 1);
                    int tx2 = x + ex_(i);
                    bool inx = true;
                    if (PRES) inx = tx2 >= 0 && tx2 < nx;
                    else tx2 = wrap1(tx2, nx);
                    const int tyw = WALLS ? ty2 : wrap1(ty2, ny);
                    const float v = el(fs[i], e);
                    if (ODD) {
                        if (wall) F[aa_slot<IX>(x, y, opp_(i), P)] = v;
                        else if (inx) F[aa_slot<IX>(tx2, tyw, i, P)] = v;  // else it leaves through the column
                    } else {
                        if (wall) {
                            if (inx) F[aa_slot<IX>(tx2, ty2, i, P)] = v;
                        } else {
                            F[aa_slot<IX>(x, y, opp_(i), P)] = v;
                        }
                    }
                }
                acc.macc = add_(acc.macc, el(rho_own, e));
                acc.rmin = vmin_(acc.rmin, el(rho, e));
                acc.rmax = vmax_(acc.rmax, el(rho, e));
                if (WALLS && !anyp) {
                    if (y == 1) { S.brho1[lane] = el(rho, e); S.bv1[lane] = el(vx, e); }
                    if (y == ny - 3) S.tv2[lane] = el(vx, e);
                }
            }
        }
        acc.flush();
        if (WALLS) {
            __syncthreads();  // rows 1 and ny-3 of the tile published
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int y = b + e;
                if (!(e ? act1 : act0) || anyp || !(y == 1 || y == 2 || y == ny - 2)) continue;
                // wall shear: quadratic through v = 0 on the half-way plane and
                // v at distances 1/2 and 3/2; wall pressure: Eq. 2.4 in mesh units
                const float rk = el(rho, e), vk = el(vx, e);
                const int pz = q0 + e;
                if (y == 1) {
                    const float pw = wall_pressure<float, AA_SW>(A, S.rho, S.phi, S.lap[pz][ccol], pz - 1, pz, pz + 1,
                                                                 ccol, rk);
                    acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw);
                }
                if (y == 2) {
                    const float tw = mul_(mul_(S.brho1[lane], A.nu), mul_(fma_(9.0f, S.bv1[lane], -vk), third));
                    acc.J += (double)tw; acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw);
                }
                if (y == ny - 2) {
                    const float tw = mul_(mul_(rk, A.nu), mul_(fma_(9.0f, vk, -S.tv2[lane]), third));
                    const float pw = wall_pressure<float, AA_SW>(A, S.rho, S.phi, S.lap[pz][ccol], pz - 1, pz, pz + 1,
                                                                 ccol, rk);
                    acc.J += (double)tw;
                    acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw);
                    acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw);
                }
            }
        }
        __syncthreads();  // the ring is rewritten by the next tile
        gcur = gnext;
#pragma unroll
        for (int i = 0; i < 9; ++i) fcur[i] = PF ? fnext[i] : make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < RN; ++q) rcur[q] = rnext[q];
    }

    double m, j;
    float e[4];
    bool anybad;
    cta_reduce<float, AA2_THREADS, 1>(acc, S, m, j, e, anybad);
    if (tid == 0) {
        const int cta = blockIdx.x;
        A.mass_part[cta] = m;
        A.J_acc[cta] += j;
        float *ex = A.ext + 4 * cta;
        ex[0] = fmin(ex[0], e[0]); ex[1] = fmax(ex[1], e[1]);
        ex[2] = fmin(ex[2], e[2]); ex[3] = fmax(ex[3], e[3]);
        if (anybad) atomicOr(A.err, 1);
    }
}

// ---------------------------------------------------------------------------
// Host side: kernel selection, the tile plan and the launches.
// ---------------------------------------------------------------------------
namespace {

// v = 4 walls + 2 pressure columns + odd
template <typename real, typename IX>
void *aa_step_fn(int v)
{
    switch (v) {
    case 0: return (void *)aa_step_kernel<real, false, false, false, IX>;
    case 1: return (void *)aa_step_kernel<real, false, false, true, IX>;
    case 2: return (void *)aa_step_kernel<real, false, true, false, IX>;
    case 3: return (void *)aa_step_kernel<real, false, true, true, IX>;
    case 4: return (void *)aa_step_kernel<real, true, false, false, IX>;
    case 5: return (void *)aa_step_kernel<real, true, false, true, IX>;
    case 6: return (void *)aa_step_kernel<real, true, true, false, IX>;
    default: return (void *)aa_step_kernel<real, true, true, true, IX>;
    }
}

template <typename real, typename IX>
void *aa_density_fn(int v)
{
    switch (v) {
    case 0: return (void *)aa_density_kernel<real, false, false, false, IX>;
    case 1: return (void *)aa_density_kernel<real, false, false, true, IX>;
    case 2: return (void *)aa_density_kernel<real, false, true, false, IX>;
    case 3: return (void *)aa_density_kernel<real, false, true, true, IX>;
    case 4: return (void *)aa_density_kernel<real, true, false, false, IX>;
    case 5: return (void *)aa_density_kernel<real, true, false, true, IX>;
    case 6: return (void *)aa_density_kernel<real, true, true, false, IX>;
    default: return (void *)aa_density_kernel<real, true, true, true, IX>;
    }
}

// v = 2 walls + pressure columns
template <typename real, typename IX>
void *aa_swap_fn(int v)
{
    switch (v) {
    case 0: return (void *)aa_swap_kernel<real, false, false, IX>;
    case 1: return (void *)aa_swap_kernel<real, false, true, IX>;
    case 2: return (void *)aa_swap_kernel<real, true, false, IX>;
    default: return (void *)aa_swap_kernel<real, true, true, IX>;
    }
}

template <typename IX>
void *aa_step_f2_fn(int v)
{
    switch (v) {
    case 0: return (void *)aa_step_kernel_f2<false, false, false, IX>;
    case 1: return (void *)aa_step_kernel_f2<false, false, true, IX>;
    case 2: return (void *)aa_step_kernel_f2<false, true, false, IX>;
    case 3: return (void *)aa_step_kernel_f2<false, true, true, IX>;
    case 4: return (void *)aa_step_kernel_f2<true, false, false, IX>;
    case 5: return (void *)aa_step_kernel_f2<true, false, true, IX>;
    case 6: return (void *)aa_step_kernel_f2<true, true, false, IX>;
    default: return (void *)aa_step_kernel_f2<true, true, true, IX>;
    }
}

// FP32: the row-pair kernel (128 threads); FP64: one node per thread (256)
template <typename real>
void *step_fn(bool big, int v)
{
    if constexpr (sizeof(real) == 4) return big ? aa_step_f2_fn<long long>(v) : aa_step_f2_fn<int>(v);
    return big ? aa_step_fn<real, long long>(v) : aa_step_fn<real, int>(v);
}
template <typename real>
constexpr int step_threads() { return sizeof(real) == 4 ? AA2_THREADS : AA_THREADS; }

}  // namespace

cudaError_t aa_plan(int precision, bool big, bool walls, bool pres, int nx, int ny, int sms, AAPlan *p)
{
    AAPlan q{};
    const int nyf = walls ? ny - 2 : ny;
    q.sx = (pres && (nx - 1) % AA_TX == 0) ? 1 : 0;
    q.sy = (walls && (ny - 3) % AA_TY == 0) ? 1 : 0;
    q.ntx = (nx + q.sx + AA_TX - 1) / AA_TX;
    q.nty = (nyf + q.sy + AA_TY - 1) / AA_TY;
    int occ = 0;
    void *fn = precision == 64 ? step_fn<double>(big, 0) : step_fn<float>(big, 0);
    q.threads = precision == 64 ? step_threads<double>() : step_threads<float>();
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, q.threads, 0);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)q.ntx * q.nty;
    q.nctas = (int)std::max<long long>(1, std::min<long long>({tiles, (long long)sms * std::max(1, occ),
                                                               (long long)MAX_CTAS}));
    const long long nodes = (long long)nx * nyf;
    q.dens_blocks = (int)std::max<long long>(1, std::min<long long>((nodes + 255) / 256, (long long)sms * 8));
    *p = q;
    return cudaSuccess;
}

template <typename real>
cudaError_t aa_step(const KArgs<real> &A, real *F, real *rho, real *side, bool walls, bool pres, bool odd, bool big,
                    const AAPlan &p, cudaStream_t st)
{
    const int v = 4 * walls + 2 * pres + odd;
    int nx = A.nx, ny = A.ny, P = A.pitch, yf0 = A.yf0, nyf = A.nyf;
    const real *Fc = F;
    void *dargs[] = {(void *)&Fc, (void *)&rho, (void *)&side, (void *)&nx, (void *)&ny, (void *)&P, (void *)&yf0,
                     (void *)&nyf};
    void *dfn = big ? aa_density_fn<real, long long>(v) : aa_density_fn<real, int>(v);
    cudaError_t e = cudaLaunchKernel(dfn, dim3(p.dens_blocks), dim3(256), dargs, 0, st);
    if (e != cudaSuccess) return e;
    const AATiles T{p.ntx, p.nty, p.sx, p.sy};
    const real *rc = rho, *sc = side;
    void *sargs[] = {(void *)&A, (void *)&F, (void *)&rc, (void *)&sc, (void *)&T};
    return cudaLaunchKernel(step_fn<real>(big, v), dim3(p.nctas), dim3(step_threads<real>()), sargs, 0, st);
}

cudaError_t aa_swap(int precision, void *F, bool walls, bool pres, bool big, int nx, int ny, int P, int sms,
                    cudaStream_t st)
{
    const int v = 2 * walls + pres;
    void *fn = precision == 64 ? (big ? aa_swap_fn<double, long long>(v) : aa_swap_fn<double, int>(v))
                               : (big ? aa_swap_fn<float, long long>(v) : aa_swap_fn<float, int>(v));
    void *args[] = {(void *)&F, (void *)&nx, (void *)&ny, (void *)&P};
    const long long nodes = (long long)nx * ny;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((nodes + 255) / 256, (long long)sms * 8));
    return cudaLaunchKernel(fn, dim3(blocks), dim3(256), args, 0, st);
}

template cudaError_t aa_step<float>(const KArgs<float> &, float *, float *, float *, bool, bool, bool, bool,
                                    const AAPlan &, cudaStream_t);
template cudaError_t aa_step<double>(const KArgs<double> &, double *, double *, double *, bool, bool, bool, bool,
                                     const AAPlan &, cudaStream_t);

}  // namespace lbm
