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
//   - populations live in two buffers with rows of nine planes,
//     f[y][i][x] (row stride 9 nx; the C ABI exchanges f[i][y][x] and
//     converts); a step reads buffer A and pushes post-collision values into
//     buffer B; all indices are 32-bit (9 nx ny < 2^31);
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
    long long plane;  // nx * ny (nodes per lattice)
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

// Reciprocal: the FP32 path uses the hardware approximation (a few ulp), the
// FP64 path the IEEE division.
__device__ __forceinline__ float rcp_(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ double rcp_(double v) { return 1.0 / v; }

// ---------------------------------------------------------------------------
// Bulk asynchronous copies global -> shared (cp.async.bulk, completion counted
// on an mbarrier in bytes), used to stream population rows into a stage ring.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity; gives up after a bounded number
// of polls (each poll itself suspends for a hardware-defined interval) and
// returns false, so a lost transfer can never hang the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (bulk copy) writes.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Mesh-space EOS potential phi = k^2 p0(rho) - rho/3 (Eqs. 2.14, 2.17), CS p0.
template <typename real>
__device__ __forceinline__ real eos_phi(const KArgs<real> &A, real rho)
{
    const real eta = A.b4 * rho;
    const real om = real(1) - eta;
    const real num = real(1) + eta * (real(1) + eta * (real(1) - eta));
    const real p0 = rho * A.RT * num * rcp_(om * om * om) - A.a * rho * rho;
    return A.k2 * p0 - rho * real(1.0 / 3.0);
}

// Density of a pressure column whose interior neighbour has density rho_f: the
// EOS root at the column pressure on the branch of the neighbour's phase,
// blended continuously across an interface (Sec. 2.2 pressure-driven ends).
// Per-channel geometry of a segment: population buffers (read / written),
// lattice size, strip width and the pressure-column branch densities.
template <typename real>
struct Geom {
    const real *fin;
    real *fout;
    int nx, ny, W;
    real rho_in_g, rho_in_l, rho_out_g, rho_out_l;
};

template <typename real>
__device__ __forceinline__ real column_density(const KArgs<real> &A, const Geom<real> &G, bool outlet, real rho_f)
{
    real th = (rho_f - A.ph_g) * A.inv_dph;
    th = fmin(fmax(th, real(0)), real(1));
    const real g = outlet ? G.rho_out_g : G.rho_in_g;
    const real l = outlet ? G.rho_out_l : G.rho_in_l;
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

// Resident CTAs per SM the register allocation is held to: 512 FP32 threads
// per SM (<= 128 registers each); FP64 carries twice the state per thread.
#ifndef LBM_FP32_THREADS_PER_SM
#define LBM_FP32_THREADS_PER_SM 512
#endif
template <typename real, int BLOCK>
struct MinBlocks {
    static constexpr int value = (sizeof(real) == 4 ? LBM_FP32_THREADS_PER_SM : 256) / BLOCK;
};

// Stage ring of the staged kernel. At iteration j (after its barrier) the
// rows j-3 (collision) .. j (newest density row) are in use, rows j+1 ..
// j+STAGE_AHEAD are in flight, and row j+STAGE_AHEAD+1 is issued into the
// stage freed by row j-4: STAGE_AHEAD + 5 stages.
#ifndef LBM_STAGE_AHEAD
#define LBM_STAGE_AHEAD 1
#endif
constexpr int STAGE_AHEAD = LBM_STAGE_AHEAD;
constexpr int NSTAGE = 5 + STAGE_AHEAD;

// A stage holds one stencil row of the strip (local columns 0 .. BLOCK-1) for
// the nine planes. Each plane segment starts on a 128-byte line when the strip
// does, so a copy touches no more lines than it needs.
template <int BLOCK>
__host__ __device__ constexpr int stage_pitch() { return BLOCK; }

template <typename real, int BLOCK>
constexpr size_t staged_smem_bytes()
{
    return (size_t)NSTAGE * 9 * stage_pitch<BLOCK>() * sizeof(real) + NSTAGE * sizeof(uint64_t);
}

// Position in the stage ring (stage index and mbarrier phase parity).
struct RingPos {
    uint32_t s = 0, ph = 0;
    __device__ __forceinline__ void advance()
    {
        if (++s == NSTAGE) { s = 0; ph ^= 1u; }
    }
};

// f_eq of Eq. 2.2 built from the (i, opp(i)) pairs, which share their even
// part c and differ in the sign of their odd part o: f_i = c + o, f_opp = c - o.
// The rest population is rho minus the eight moving ones (= rho - 2 sum c), so
// f_eq carries exactly rho up to unbiased rounding.
template <typename real>
__device__ __forceinline__ void feq_pairs(real rho, real ux, real uy, real (&fe)[9])
{
    const real base = real(1) - real(1.5) * (ux * ux + uy * uy);
    const real r1 = rho * real(1.0 / 9.0), r2 = rho * real(1.0 / 36.0);
    const real s = ux + uy, d = uy - ux;  // e.u of directions 5 (1,1) and 6 (-1,1)
    const real c1 = r1 * (base + real(4.5) * ux * ux), o1 = real(3) * r1 * ux;
    const real c2 = r1 * (base + real(4.5) * uy * uy), o2 = real(3) * r1 * uy;
    const real c5 = r2 * (base + real(4.5) * s * s), o5 = real(3) * r2 * s;
    const real c6 = r2 * (base + real(4.5) * d * d), o6 = real(3) * r2 * d;
    fe[1] = c1 + o1; fe[3] = c1 - o1;
    fe[2] = c2 + o2; fe[4] = c2 - o2;
    fe[5] = c5 + o5; fe[7] = c5 - o5;
    fe[6] = c6 + o6; fe[8] = c6 - o6;
    fe[0] = rho - real(2) * ((c1 + c2) + (c5 + c6));
}

// Unscaled isotropic gradient: 12 * grad psi = (4(E - W) + (NE - NW) + (SE - SW),
//                                              4(N - S) + (NE - SE) + (NW - SW)).
template <typename real, int SW>
__device__ __forceinline__ void grad12(const real (*S)[SW], int qm, int q0, int qp, int c, real &gx,
                                       real &gy)
{
    const real E = S[q0][c + 1], W = S[q0][c - 1], N = S[qp][c], So = S[qm][c];
    const real NE = S[qp][c + 1], NW = S[qp][c - 1], SE = S[qm][c + 1], SWv = S[qm][c - 1];
    gx = real(4) * (E - W) + (NE - NW) + (SE - SWv);
    gy = real(4) * (N - So) + (NE - SE) + (NW - SWv);
}

// One fused time step (MODE_STEP) or the macroscopic fields (MODE_FIELDS).
//
// Per segment (strip of columns x0 .. x0+xw-1, fluid rows ya .. yb-1) the CTA
// runs iterations yy = ya-2 .. yb+2 with one barrier each:
//   (1) re-read (L1) the populations of the collision row r = yy-3;
//   (2) density and phi of stencil row yy from the populations prefetched in
//       the previous iteration, then prefetch row yy+1;
//   (3) Laplacian of row yy-2 (its density rows were completed before the
//       previous barrier);
//   --- barrier ---
//   (4) force, collision, boundaries and push-streaming of row r, whose phi
//       rows r-1..r+1 and Laplacian rows r-1..r+1 are now complete.
// The ring keeps 8 rows, so the writes of iteration yy+1 never touch the rows
// iteration yy still reads.
//
// STAGED: the strip's populations of each stencil row (9 plane segments of xw
// values) are streamed by one producer thread with bulk asynchronous copies
// into a ring of NSTAGE shared-memory stages, issued STAGE_AHEAD + 1 rows
// ahead; consumers read densities and collision populations from the stage
// (needs nx and the strip width to be multiples of 4 for 16-byte aligned
// copies). Otherwise each thread loads its column with one row of register
// prefetch and re-reads the collision row from L1. In both variants the four
// halo lanes load the two columns beyond each strip edge with one row of
// register prefetch.
// Per-thread diagnostic accumulators of the states read.
template <typename real>
struct Acc {
    double mass, J;
    real macc;
    int mcount;
    real tmin, tmax, pmin, pmax;
    bool bad;
    __device__ __forceinline__ void reset()
    {
        mass = 0.0; J = 0.0; macc = real(0); mcount = 0;
        tmin = pmin = real(INFINITY); tmax = pmax = real(-INFINITY);
        bad = false;
    }
};

// Static shared-memory working set of a CTA: the 8-row stencil ring (density,
// EOS potential, Laplacian; strip plus two halo columns per side) and the
// reduction scratch.
template <typename real, int BLOCK>
struct Smem {
    real rho[RING][BLOCK + 4];
    real phi[RING][BLOCK + 4];
    real lap[RING][BLOCK + 4];
    double red[BLOCK / 32][2];
    real ext[BLOCK / 32][4];
    int bad;
};

// One segment: strip s (columns s*W ..) of the lattice G, fluid rows ya .. yb-1.
// Every thread of the CTA calls it with the same arguments.
template <typename real, bool WALLS, bool PRES, int MODE, int BLOCK, bool STAGED>
__device__ __forceinline__ void run_segment(const KArgs<real> &A, const Geom<real> &G, int s, int ya, int yb,
                                            Smem<real, BLOCK> &S, real *stages, uint64_t *bars,
                                            RingPos &ring_next, Acc<real> &acc, bool &lost)
{
    constexpr int SW = BLOCK + 4;
    constexpr int PRODUCER = BLOCK - 1;  // no halo duty
    constexpr int SP = stage_pitch<BLOCK>();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const real third = real(1.0 / 3.0), twelfth = real(1.0 / 12.0), sixth = real(1.0 / 6.0);
    const int nx = G.nx, ny = G.ny;
    const int rstride = 9 * nx;  // row stride of the population layout f[y][i][x]
    // push targets of directions 1..8 relative to the source slot index
    const int o1 = nx + 1, o2 = rstride + 2 * nx, o3 = 3 * nx - 1, o4 = 4 * nx - rstride;
    const int o5 = rstride + 5 * nx + 1, o6 = rstride + 6 * nx - 1, o7 = 7 * nx - rstride - 1;
    const int o8 = 8 * nx - rstride + 1;
    real b_rho1 = 0, b_v1 = 0, t_v2 = 0;  // wall-pair carries (rows 1 -> 2, ny-3 -> ny-2)

    const int x0 = s * G.W;
    const int xw = min(G.W, nx - x0);
    const bool active = tid < xw;
    const int x = x0 + tid;
    const bool pin = PRES && active && x == 0;
    const bool pout = PRES && active && x == nx - 1;
    const bool pcol = pin || pout;
    const int xc = pin ? 1 : (pout ? nx - 2 : x);  // column whose populations this thread loads
    const int ccol = xc - x0 + 2;                  // its shared-memory column
    // pushes never wrap or leave the lattice in x
    const bool x_inner = !pcol && (PRES || (x >= 1 && x <= nx - 2));

    // Halo columns (lane 0 of warps 0..3): local -2, -1, xw, xw+1.
    // hmode 1: density of column hx; 2 / 3: inlet / outlet column density
    // derived from column hx = 1 / nx-2 (clamp beyond the pressure columns).
    int hmode = 0, hx = 0, hcol = 0;
    if (lane == 0 && warp < 4) {
        const int hloc = (warp < 2) ? (warp - 2) : (xw + warp - 2);
        hcol = hloc + 2;
        const int gxh = x0 + hloc;
        if (PRES) {
            if (gxh <= 0) { hmode = 2; hx = 1; }
            else if (gxh >= nx - 1) { hmode = 3; hx = nx - 2; }
            else { hmode = 1; hx = gxh; }
        } else {
            hmode = 1;
            hx = ((gxh % nx) + nx) % nx;
        }
    }
    // Laplacian of the two halo columns next to the strip (local -1, xw)
    const int lhalo = (lane == 1 && warp == 1) ? 1 : ((lane == 1 && warp == 2) ? xw + 2 : -1);

    const real *__restrict__ col_in = G.fin + xc;
    const real *__restrict__ hal_in = G.fin + hx;
    const int scol = xc - x0;            // this thread's column inside a stage
    const int nrows = yb - ya + 4;       // stencil rows ya-2 .. yb+1
    real pf[9], hf[9];
    real add_next = real(0);  // wetting offset of the next stencil row (mirrored wall ghost)
    // halo (and, without staging, own-column) loads of stencil row yy
    auto prefetch = [&](int yy) {
        bool mir;
        const int row = map_row<WALLS>(yy, ny, mir) * rstride;
        add_next = mir ? A.wet : real(0);
        if (!STAGED && active) {
#pragma unroll
            for (int i = 0; i < 9; ++i) pf[i] = __ldg(col_in + row + i * nx);
        }
        if (hmode) {
#pragma unroll
            for (int i = 0; i < 9; ++i) hf[i] = __ldg(hal_in + row + i * nx);
        }
    };
    // producer: stream stencil row j of this segment into stage position ip
    RingPos ring_issue = ring_next;
    auto issue = [&](int j) {
        if (j < nrows) {
            if (tid == PRODUCER) {
                bool mir;
                const int row = map_row<WALLS>(ya - 2 + j, ny, mir) * rstride;
                const uint32_t st = ring_issue.s;
                real *dst = stages + (size_t)st * 9 * SP;
                const real *src = G.fin + row + x0;
                const uint32_t bytes = (uint32_t)(xw * sizeof(real));
                mbar_arrive_expect_tx(&bars[st], 9 * bytes);
#pragma unroll
                for (int i = 0; i < 9; ++i) bulk_copy_g2s(dst + i * SP, src + i * nx, bytes, &bars[st]);
            }
            ring_issue.advance();
        }
    };
    // stage of the collision row (three rows behind the consumed row)
    RingPos ring_coll = ring_next;
    for (int k = 0; k < NSTAGE - 3; ++k) ring_coll.advance();
#pragma unroll
    for (int i = 0; i < 9; ++i) { pf[i] = real(0); hf[i] = real(0); }
    prefetch(ya - 2);
    if constexpr (STAGED) {
        for (int j = 0; j <= STAGE_AHEAD; ++j) issue(j);
        // one thread waits for the first row; the barrier publishes it
        if (tid == 0 && !mbar_wait_bounded(&bars[ring_next.s], ring_next.ph)) lost = true;
        __syncthreads();
    }

    for (int yy = ya - 2; yy <= yb + 2; ++yy) {
        const int r = yy - 3;
        const int j = yy - (ya - 2);
        const bool collide = r >= ya && r < yb;  // uniform over the CTA
        const uint32_t st_cons = ring_next.s, ph_cons = ring_next.ph, st_coll = ring_coll.s;

        // (1) populations of the collision row (read from HBM three iterations ago)
        real f[9];
        if (!STAGED && collide && active) {
            const real *src = col_in + r * rstride;
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = __ldg(src + i * nx);
        }

        // (2) density and EOS potential of stencil row yy (staged: its
        //     stage was completed before the previous barrier)
        if (yy <= yb + 1) {
            const real add = add_next;
            const int rs = yy & (RING - 1);
            real rho_own = real(0), rho_h = real(0);
            if constexpr (STAGED) {
                (void)ph_cons;
                const real *stg = stages + (size_t)st_cons * 9 * SP;
                if (active) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) pf[i] = stg[i * SP + scol];
                }
            }
            if (active) {
                real sum = ((pf[0] + pf[1]) + (pf[2] + pf[3])) + ((pf[4] + pf[5]) + (pf[6] + pf[7])) + pf[8];
                rho_own = (pcol ? column_density(A, G, pout, sum) : sum) + add;
            }
            if (hmode) {
                real sum = ((hf[0] + hf[1]) + (hf[2] + hf[3])) + ((hf[4] + hf[5]) + (hf[6] + hf[7])) + hf[8];
                rho_h = (hmode == 1 ? sum : column_density(A, G, hmode == 3, sum)) + add;
            }
            if (yy + 1 <= yb + 1) prefetch(yy + 1);
            if (active) {
                S.rho[rs][tid + 2] = rho_own;
                S.phi[rs][tid + 2] = eos_phi(A, rho_own);
            }
            if (hmode) {
                S.rho[rs][hcol] = rho_h;
                S.phi[rs][hcol] = eos_phi(A, rho_h);
            }
        }

        // (3) Laplacian of row yy-2 on local columns -1 .. xw
        if (yy >= ya + 1) {
            const int lr = (yy - 2) & (RING - 1), lm = (yy - 3) & (RING - 1), lp = (yy - 1) & (RING - 1);
            auto lap_at = [&](int c) {
                const real edges = (S.rho[lr][c - 1] + S.rho[lr][c + 1]) + (S.rho[lm][c] + S.rho[lp][c]);
                const real corners = (S.rho[lm][c - 1] + S.rho[lm][c + 1]) + (S.rho[lp][c - 1] + S.rho[lp][c + 1]);
                S.lap[lr][c] = (real(4) * edges + corners - real(20) * S.rho[lr][c]) * sixth;
            };
            if (active) lap_at(tid + 2);
            if (lhalo >= 0) lap_at(lhalo);
        }
        if constexpr (STAGED) {
            // one thread waits for the next stencil row's stage; the
            // barrier below publishes its contents to the whole CTA
            if (tid == 0 && yy + 1 <= yb + 1) {
                RingPos nxt = ring_next;
                nxt.advance();
                if (!mbar_wait_bounded(&bars[nxt.s], nxt.ph)) lost = true;
            }
        }
        __syncthreads();

        if constexpr (STAGED) {
            // the stage of row j-4 was last read by the collision of the
            // previous iteration, before this barrier: refill it
            if (tid == PRODUCER) fence_proxy_async_smem();
            issue(j + STAGE_AHEAD + 1);
        }
        if (yy <= yb + 1) ring_next.advance();

        // (4) collide and stream row r
        if (collide && active) {
            if constexpr (STAGED) {
                const real *sp = stages + (size_t)st_coll * 9 * SP + scol;
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = sp[i * SP];
            }
            const int q0 = r & (RING - 1), qm = (r - 1) & (RING - 1), qp = (r + 1) & (RING - 1);
            const int c = ccol;
            real gpx, gpy, glx, gly;
            grad12<real, SW>(S.phi, qm, q0, qp, c, gpx, gpy);
            grad12<real, SW>(S.lap, qm, q0, qp, c, glx, gly);
            const real rho = S.rho[q0][c];
            const real kr = A.kappa * rho;
            const real Fx = (kr * glx - gpx) * twelfth + A.gx;
            const real Fy = (kr * gly - gpy) * twelfth + A.gy;
            const real jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
            const real jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
            const real irho = rcp_(rho);
            const real ux = jx * irho, uy = jy * irho;
            const real hFi = real(0.5) * irho;
            const real vx = ux + hFi * Fx, vy = uy + hFi * Fy;

            if (MODE == MODE_STEP) {
                real fs[9];
                if (!pcol) {
                    const real tFi = A.tau * irho;
                    real fe[9];
                    feq_pairs<real>(rho, ux + tFi * Fx, uy + tFi * Fy, fe);
#pragma unroll
                    for (int i = 0; i < 9; ++i) fs[i] = f[i] + (fe[i] - f[i]) * A.inv_tau;
                } else {
                    // non-equilibrium extrapolation from the interior neighbour:
                    // f_eq(rho_b, v) = (rho_b / rho_f) f_eq(rho_f, v)
                    const real rho_b = S.rho[q0][tid + 2];
                    real ff[9];
                    feq_pairs<real>(rho, vx, vy, ff);
                    const real sc = rho_b * irho;
#pragma unroll
                    for (int i = 0; i < 9; ++i) fs[i] = sc * ff[i] + A.omb * (f[i] - ff[i]);
                }
                real *const out = G.fout;
                const int oi = r * rstride + x;  // slot of (x, r) in plane 0
                const bool y_inner = WALLS ? (r >= 2 && r <= ny - 3) : (r >= 1 && r <= ny - 2);
                if (x_inner && y_inner) {
                    out[oi] = fs[0];
                    out[oi + o1] = fs[1];
                    out[oi + o2] = fs[2];
                    out[oi + o3] = fs[3];
                    out[oi + o4] = fs[4];
                    out[oi + o5] = fs[5];
                    out[oi + o6] = fs[6];
                    out[oi + o7] = fs[7];
                    out[oi + o8] = fs[8];
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const int ty = r + ey_(i);
                        if (WALLS && (ty == 0 || ty == ny - 1)) {
                            // half-way bounce-back into the opposite slot of this node
                            out[oi + opp_(i) * nx] = fs[i];
                        } else {
                            int tx = x + ex_(i);
                            if (PRES) {
                                if (tx < 0 || tx >= nx) continue;  // leaves through the column
                            } else {
                                tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
                            }
                            int tyw = ty;
                            if (!WALLS) tyw = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
                            out[tyw * rstride + i * nx + tx] = fs[i];
                        }
                    }
                }
                const real mrho = pcol ? S.rho[q0][tid + 2] : rho;
                if (sizeof(real) == 8) acc.mass += (double)mrho;
                else {
                    acc.macc += mrho;
                    if (++acc.mcount == 16) { acc.mass += (double)acc.macc; acc.macc = real(0); acc.mcount = 0; }
                }
                if (!(rho > real(0)) || !(rho < real(1e30))) acc.bad = true;
            } else {
                const long long oi = (long long)r * nx + x;
                A.o_rho[oi] = pcol ? S.rho[q0][tid + 2] : rho;
                A.o_vx[oi] = vx;
                A.o_vy[oi] = vy;
            }

            if (WALLS && !pcol && (r <= 2 || r >= ny - 3)) {
                // wall shear: quadratic through v = 0 on the half-way plane and
                // v at distances 1/2 and 3/2; wall pressure: Eq. 2.4 in mesh units
                auto pwall = [&]() {
                    real grx, gry;
                    grad12<real, SW>(S.rho, qm, q0, qp, c, grx, gry);
                    grx *= twelfth;
                    gry *= twelfth;
                    return S.phi[q0][c] + rho * third - A.kappa * rho * S.lap[q0][c]
                           - real(0.5) * A.kappa * (grx * grx + gry * gry);
                };
                if (r == 1) {
                    b_rho1 = rho;
                    b_v1 = vx;
                    const real pw = pwall();
                    if (MODE == MODE_STEP) { acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw); }
                    else A.o_pw[x] = pw;
                }
                if (r == ny - 3) t_v2 = vx;
                if (r == 2) {
                    const real tw = b_rho1 * A.nu * (real(9) * b_v1 - vx) * third;
                    if (MODE == MODE_STEP) { acc.J += (double)tw; acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw); }
                    else A.o_tw[x] = tw;
                }
                if (r == ny - 2) {
                    const real tw = rho * A.nu * (real(9) * vx - t_v2) * third;
                    const real pw = pwall();
                    if (MODE == MODE_STEP) {
                        acc.J += (double)tw;
                        acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw);
                        acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw);
                    } else {
                        A.o_tw[nx + x] = tw;
                        A.o_pw[nx + x] = pw;
                    }
                }
            }
        }
        ring_coll.advance();
    }
    __syncthreads();  // ring and stage reuse by the next segment
}

// Fixed-order CTA reduction of the accumulators; thread 0 receives the totals.
template <typename real, int BLOCK>
__device__ __forceinline__ void cta_reduce(Acc<real> &acc, Smem<real, BLOCK> &S, double &m, double &j,
                                           real (&e)[4], bool &anybad)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    acc.mass += (double)acc.macc;
    acc.macc = real(0);
    acc.mcount = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.mass += __shfl_xor_sync(0xffffffffu, acc.mass, o);
        acc.J += __shfl_xor_sync(0xffffffffu, acc.J, o);
        acc.tmin = fmin(acc.tmin, __shfl_xor_sync(0xffffffffu, acc.tmin, o));
        acc.tmax = fmax(acc.tmax, __shfl_xor_sync(0xffffffffu, acc.tmax, o));
        acc.pmin = fmin(acc.pmin, __shfl_xor_sync(0xffffffffu, acc.pmin, o));
        acc.pmax = fmax(acc.pmax, __shfl_xor_sync(0xffffffffu, acc.pmax, o));
    }
    const bool wbad = __any_sync(0xffffffffu, acc.bad);
    if (tid == 0) S.bad = 0;
    __syncthreads();
    if (lane == 0) {
        S.red[warp][0] = acc.mass;
        S.red[warp][1] = acc.J;
        S.ext[warp][0] = acc.tmin; S.ext[warp][1] = acc.tmax;
        S.ext[warp][2] = acc.pmin; S.ext[warp][3] = acc.pmax;
        if (wbad) atomicOr(&S.bad, 1);
    }
    __syncthreads();
    if (tid == 0) {
        m = 0.0; j = 0.0;
        e[0] = S.ext[0][0]; e[1] = S.ext[0][1]; e[2] = S.ext[0][2]; e[3] = S.ext[0][3];
        for (int w = 0; w < BLOCK / 32; ++w) {
            m += S.red[w][0];
            j += S.red[w][1];
            e[0] = fmin(e[0], S.ext[w][0]); e[1] = fmax(e[1], S.ext[w][1]);
            e[2] = fmin(e[2], S.ext[w][2]); e[3] = fmax(e[3], S.ext[w][3]);
        }
        anybad = S.bad != 0;
    }
    __syncthreads();
}

template <typename real, bool WALLS, bool PRES, int MODE, int BLOCK, bool STAGED>
__global__ void __launch_bounds__(BLOCK, MinBlocks<real, BLOCK>::value) step_kernel(const KArgs<real> A)
{
    static_assert(BLOCK % 32 == 0 && BLOCK >= 128, "the four halo columns take one warp each");
    constexpr int SP = stage_pitch<BLOCK>();
    extern __shared__ __align__(128) unsigned char dsm[];
    real *const stages = reinterpret_cast<real *>(dsm);
    uint64_t *const bars = reinterpret_cast<uint64_t *>(dsm + (size_t)NSTAGE * 9 * SP * sizeof(real));
    __shared__ Smem<real, BLOCK> S;

    const int tid = threadIdx.x;
    const int cta = A.reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    long long u = cut_units<WALLS>(A, cta);
    const long long u1 = cut_units<WALLS>(A, cta + 1);
    const Geom<real> G{A.fin, A.fout, A.nx, A.ny, A.W, A.rho_in_g, A.rho_in_l, A.rho_out_g, A.rho_out_l};

    Acc<real> acc;
    acc.reset();
    RingPos ring_next;  // stage of the next stencil row to consume (uniform)
    bool lost = false;  // a bounded wait gave up

    if constexpr (STAGED) {
        if (tid == 0) {
            for (int st = 0; st < NSTAGE; ++st) mbar_init(&bars[st], 1);
            mbar_init_fence();
        }
        __syncthreads();
    }

    while (u < u1) {
        const int s = (int)(u / A.nyf);
        const int ya = A.yf0 + (int)(u - (long long)s * A.nyf);
        const long long ue = min(u1, (long long)(s + 1) * A.nyf);
        const int yb = ya + (int)(ue - u);
        u = ue;
        run_segment<real, WALLS, PRES, MODE, BLOCK, STAGED>(A, G, s, ya, yb, S, stages, bars, ring_next, acc,
                                                           lost);
    }

    if (STAGED && lost) atomicOr(A.err, 2);
    if (MODE != MODE_STEP) return;

    double m, j;
    real e[4];
    bool anybad;
    cta_reduce<real, BLOCK>(acc, S, m, j, e, anybad);
    if (tid == 0) {
        A.mass_part[cta] = m;
        A.J_acc[cta] += j;
        real *ex = A.ext + 4 * cta;
        ex[0] = fmin(ex[0], e[0]); ex[1] = fmax(ex[1], e[1]);
        ex[2] = fmin(ex[2], e[2]); ex[3] = fmax(ex[3], e[3]);
        if (anybad) atomicOr(A.err, 1);
    }
}

// ---------------------------------------------------------------------------
// Batched channels: one launch steps many independent channels of different
// sizes (a parameter sweep). The channels' populations are packed in one
// buffer; a host-built work list gives each CTA a run of segments (channel,
// strip, rows), balanced over the CTAs. Every segment runs the same code as
// the single-channel kernel, so each channel's populations evolve bit for bit
// as they would alone. Diagnostics are reduced per segment into fixed slots.
// ---------------------------------------------------------------------------
template <typename real>
struct BatchChan {
    long long off;  // element offset of the channel in the packed population buffers
    int nx, ny, W, pad;
    real rho_in_g, rho_in_l, rho_out_g, rho_out_l;
};

struct BatchSeg {
    int chan, strip, ya, yb;
};

template <typename real, bool WALLS, bool PRES, int BLOCK, bool STAGED>
__global__ void __launch_bounds__(BLOCK, MinBlocks<real, BLOCK>::value)
    batch_step_kernel(const KArgs<real> A, const BatchChan<real> *__restrict__ chans,
                      const BatchSeg *__restrict__ segs, const int *__restrict__ cta_begin,
                      double *__restrict__ seg_mass, double *__restrict__ seg_J, real *__restrict__ seg_ext)
{
    constexpr int SP = stage_pitch<BLOCK>();
    extern __shared__ __align__(128) unsigned char dsm[];
    real *const stages = reinterpret_cast<real *>(dsm);
    uint64_t *const bars = reinterpret_cast<uint64_t *>(dsm + (size_t)NSTAGE * 9 * SP * sizeof(real));
    __shared__ Smem<real, BLOCK> S;

    const int tid = threadIdx.x;
    const int cta = A.reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    RingPos ring_next;
    bool lost = false;
    if constexpr (STAGED) {
        if (tid == 0) {
            for (int st = 0; st < NSTAGE; ++st) mbar_init(&bars[st], 1);
            mbar_init_fence();
        }
        __syncthreads();
    }
    for (int k = cta_begin[cta]; k < cta_begin[cta + 1]; ++k) {
        const BatchSeg sg = segs[k];
        const BatchChan<real> ch = chans[sg.chan];
        const Geom<real> G{A.fin + ch.off, A.fout + ch.off, ch.nx, ch.ny, ch.W,
                           ch.rho_in_g, ch.rho_in_l, ch.rho_out_g, ch.rho_out_l};
        Acc<real> acc;
        acc.reset();
        run_segment<real, WALLS, PRES, MODE_STEP, BLOCK, STAGED>(A, G, sg.strip, sg.ya, sg.yb, S, stages, bars,
                                                                ring_next, acc, lost);
        double m, j;
        real e[4];
        bool anybad;
        cta_reduce<real, BLOCK>(acc, S, m, j, e, anybad);
        if (tid == 0) {
            seg_mass[k] = m;
            seg_J[k] += j;
            real *ex = seg_ext + 4 * (long long)k;
            ex[0] = fmin(ex[0], e[0]); ex[1] = fmax(ex[1], e[1]);
            ex[2] = fmin(ex[2], e[2]); ex[3] = fmax(ex[3], e[3]);
            if (anybad) atomicOr(A.err, 1);
        }
    }
    if (STAGED && lost) atomicOr(A.err, 2);
}

// Per-channel reduction of the segment slots in segment order (deterministic):
// out[c*7 + 0..6] = mass, J, tw_min, tw_max, pw_min, pw_max, err.
template <typename real>
__global__ void batch_diag_kernel(const double *__restrict__ seg_mass, const double *__restrict__ seg_J,
                                  const real *__restrict__ seg_ext, const BatchSeg *__restrict__ segs,
                                  int nseg, int nchan, const int *__restrict__ err, double *__restrict__ out)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nchan; c += gridDim.x * blockDim.x) {
        double m = 0.0, j = 0.0;
        double e0 = INFINITY, e1 = -INFINITY, e2 = INFINITY, e3 = -INFINITY;
        for (int k = 0; k < nseg; ++k) {
            if (segs[k].chan != c) continue;
            m += seg_mass[k];
            j += seg_J[k];
            e0 = fmin(e0, (double)seg_ext[4 * k + 0]);
            e1 = fmax(e1, (double)seg_ext[4 * k + 1]);
            e2 = fmin(e2, (double)seg_ext[4 * k + 2]);
            e3 = fmax(e3, (double)seg_ext[4 * k + 3]);
        }
        double *o = out + 7 * c;
        o[0] = m; o[1] = j; o[2] = e0; o[3] = e1; o[4] = e2; o[5] = e3; o[6] = (double)(*err);
    }
}

// f = f_eq(rho0, 0) at every node.
template <typename real>
__global__ void init_kernel(const double *__restrict__ rho0, real *__restrict__ fa,
                            real *__restrict__ fb, int nx, int n)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int y = k / nx, x = k - y * nx;
        real fe[9];
        feq_pairs<real>((real)rho0[k], real(0), real(0), fe);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fa[(9 * y + i) * nx + x] = fe[i];
            fb[(9 * y + i) * nx + x] = fe[i];
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
