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
//   - each CTA owns a strip of up to STRIP = 128 columns and marches along y
//     over a contiguous range of rows; in this file each thread owns one
//     column (or, built with LBM_FP32_PAIR=2, a pair of adjacent columns) and
//     one row per iteration; the default FP32 staged step, in lbm_rows2.cuh,
//     gives each thread two rows per iteration; population rows are streamed
//     into a shared-memory stage ring by bulk asynchronous copies (or,
//     unstaged, prefetched into registers one row ahead);
//   - rho, phi = k^2 p0(rho) - rho/3 and lap(rho) of the rows in flight sit
//     in an 8-row shared-memory ring that covers the strip plus two halo
//     columns per side; the halo densities are summed from the neighbouring
//     strips' populations (served from L2), so no density array is stored;
//   - rows ya-2 .. yb+1 are read to collide rows ya .. yb-1; the work of a
//     launch is a balanced split of (strip, row) units over the CTAs.
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; nothing of the driver library is linked)
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
    int pitch;        // row pitch of a population plane (>= nx, a multiple of 4 when staged)
    int W;            // strip width in columns (<= STRIP)
    int nstrips;
    int yf0, nyf;     // first fluid row and number of fluid rows
    long long units;  // nstrips * nyf
    int band;         // rows per band of the unit order (>= nyf: strip-major)
    int nctas;        // logical CTAs of the schedule
    int reverse;      // launch the logical CTAs in reverse order
    real RT, a, b4, k2, kappa, tau, inv_tau, omb, gx, gy, wet, nu;
    // equation of state: 0 Carnahan-Starling (RT, a, b4), 1 Peng-Robinson
    // (RT, bpr = b, aalpha = a alpha(T))
    int eos_kind;
    real bpr, aalpha;
    // collision: 0 BGK, 1 MRT with rates over the squared row norms of the
    // moment basis (m_e = s_e/36, m_eps = s_eps/36, m_j = s_j/6, m_q = s_q/12,
    // m_nu = s_nu/4); the equilibrium velocity is u + ushift F / rho with
    // ushift = tau (BGK) or 1/s_j (MRT)
    int mrt;
    real ushift, m_e, m_eps, m_j, m_q, m_nu;
    // row-pair staged step: 1 = stage rows through the tensor-map kernel
    // parameter (one 2-D TMA load per row), 0 = plain bulk copies per plane
    int tma;
    // row-pair staged step: the stencil rows of the pair this many pairs ahead
    // of the one being staged are prefetched into L2 (0 = no prefetch)
    int pf;
    // failure-detection test build of the row-pair step (step_kernel_rows2
    // with HOOK): every stage wait polls at most poll_limit times
    int poll_limit;
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
__device__ __forceinline__ float2 rcp_(float2 v) { return make_float2(__fdividef(1.0f, v.x), __fdividef(1.0f, v.y)); }

// ---------------------------------------------------------------------------
// Packs: the values of the CP adjacent columns one thread owns (float2 for a
// pair of FP32 columns). Every operation is rounded once to nearest and none
// is contracted, so a pair computed with the paired FP32 instructions and the
// same columns computed one per thread give identical bits.
// ---------------------------------------------------------------------------
template <typename real, int CP>
struct Pack;
template <>
struct Pack<float, 1> { using T = float; };
template <>
struct Pack<double, 1> { using T = double; };
template <>
struct Pack<float, 2> { using T = float2; };

__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float2 add_(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul_(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma_(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b = (-1) b + a, exact product, one rounding: equal to the scalar subtraction
__device__ __forceinline__ float2 sub_(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// broadcast a constant into a pack
template <typename V>
__device__ __forceinline__ V bc(double v);
template <>
__device__ __forceinline__ float bc<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ double bc<double>(double v) { return v; }
template <>
__device__ __forceinline__ float2 bc<float2>(double v) { return make_float2((float)v, (float)v); }
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
template <typename V, typename real>
__device__ __forceinline__ V bcr(real v);
template <>
__device__ __forceinline__ float bcr<float, float>(float v) { return v; }
template <>
__device__ __forceinline__ double bcr<double, double>(double v) { return v; }
template <>
__device__ __forceinline__ float2 bcr<float2, float>(float v) { return make_float2(v, v); }

// element k of a pack
__device__ __forceinline__ float el(float v, int) { return v; }
__device__ __forceinline__ double el(double v, int) { return v; }
__device__ __forceinline__ float el(float2 v, int k) { return k ? v.y : v.x; }
__device__ __forceinline__ void set_el(float &v, int, float x) { v = x; }
__device__ __forceinline__ void set_el(double &v, int, double x) { v = x; }
__device__ __forceinline__ void set_el(float2 &v, int k, float x)
{
    if (k) v.y = x;
    else v.x = x;
}

// pack load / store (the address of a pair is 8-byte aligned)
template <typename V, typename real>
__device__ __forceinline__ V ldp(const real *p) { return *reinterpret_cast<const V *>(p); }
template <typename V, typename real>
__device__ __forceinline__ void stp(real *p, V v) { *reinterpret_cast<V *>(p) = v; }

// x times a constant c that FP32 does not represent (1/3, 1/9, 1/12, 1/36,
// 1/6): with c = hi + lo, hi = float(c), lo = float(c - hi), fma(x, hi, x lo)
// is x c under one rounding, free of the constant's own rounding bias (which
// would otherwise scale every collision's momentum or force the same way).
template <typename V>
__device__ __forceinline__ V mulk(V x, double c)
{
    if constexpr (sizeof(el(x, 0)) == 8) {
        return mul_(x, bc<V>(c));
    } else {
        const float hi = (float)c, lo = (float)(c - (double)hi);
        return fma_(x, bc<V>(hi), mul_(x, bc<V>(lo)));
    }
}

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
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int limit = 1 << 22)
{
    for (int it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// L2 prefetch of a global range (16-byte aligned, a multiple of 16 bytes) by
// the bulk-copy unit: no shared memory and no completion to wait for.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// Orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (bulk copy) writes.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Mesh-space EOS potential phi = k^2 p0(rho) - rho/3 (Eqs. 2.14, 2.17), CS p0
// with eta = b rho / 4: p0 = rho RT (1 + eta + eta^2 - eta^3)/(1 - eta)^3 - a rho^2.
template <typename V, typename real>
__device__ __forceinline__ V eos_phi(const KArgs<real> &A, V rho)
{
    const V one = bc<V>(1.0);
    if (A.eos_kind == 1) {
        // Peng-Robinson (Eq. 2.18): rho RT / (1 - x) - a alpha rho^2 / (1 + x (2 - x)), x = b rho
        const V x = mul_(bcr<V>(A.bpr), rho);
        const V i1 = rcp_(fma_(x, bc<V>(-1.0), one));
        const V iD = rcp_(fma_(x, fma_(x, bc<V>(-1.0), bc<V>(2.0)), one));
        const V p0 = fma_(mul_(mul_(rho, rho), bcr<V>(-A.aalpha)), iD, mul_(mul_(rho, bcr<V>(A.RT)), i1));
        return sub_(mul_(bcr<V>(A.k2), p0), mulk(rho, 1.0 / 3.0));
    }
    const V eta = mul_(bcr<V>(A.b4), rho);
    const V om = fma_(eta, bc<V>(-1.0), one);          // 1 - eta
    const V num = fma_(eta, fma_(eta, om, one), one);  // 1 + eta (1 + eta (1 - eta))
    const V ir = rcp_(mul_(mul_(om, om), om));
    const V p0 = fma_(mul_(rho, rho), bcr<V>(-A.a), mul_(mul_(mul_(rho, bcr<V>(A.RT)), num), ir));
    return sub_(mul_(bcr<V>(A.k2), p0), mulk(rho, 1.0 / 3.0));
}

// Per-channel geometry of a segment: population buffers (read / written),
// lattice size, strip width and the pressure-column branch densities.
template <typename real>
struct Geom {
    const real *fin;
    real *fout;
    int nx, ny, W, pitch;
    real rho_in_g, rho_in_l, rho_out_g, rho_out_l;
};

// Density of a pressure column whose interior neighbour has density rho_f: the
// EOS root at the column pressure on the branch of the neighbour's phase,
// blended linearly across an interface (Sec. 2.2 pressure-driven ends).
template <typename real>
__device__ __forceinline__ real column_density(const KArgs<real> &A, const Geom<real> &G, bool outlet, real rho_f)
{
    real th = mul_(sub_(rho_f, A.ph_g), A.inv_dph);
    th = fmin(fmax(th, real(0)), real(1));
    const real g = outlet ? G.rho_out_g : G.rho_in_g;
    const real l = outlet ? G.rho_out_l : G.rho_in_l;
    return fma_(th, sub_(l, g), g);
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

// Work units are (strip, fluid row) pairs, enumerated band by band: rows are
// cut into bands of A.band rows and, within a band, strip by strip. Logical
// CTAs take consecutive runs of units, so neighbouring CTAs hold neighbouring
// strips of one band and march through the same rows at the same time: the
// halo columns one strip reads from its neighbours are then recent in L2.
// unit_run gives the strip s, the row y of unit u and the end of its
// (strip, band) run.
template <typename real>
__device__ __forceinline__ void unit_run(const KArgs<real> &A, long long u, int &s, int &y, long long &run_end)
{
    const long long per_band = (long long)A.band * A.nstrips;
    const int b = (int)(u / per_band);
    const long long ub = (long long)b * per_band;
    const int y0 = b * A.band;
    const int hb = min(A.band, A.nyf - y0);
    const long long r = u - ub;
    s = (int)(r / hb);
    const int off = (int)(r - (long long)s * hb);
    y = A.yf0 + y0 + off;
    run_end = ub + (long long)(s + 1) * hb;
}

// Boundary c of the balanced split of work units over logical CTAs. A cut
// never separates rows 1|2 or ny-3|ny-2 (nor does a band boundary: the host
// picks the band height), so each wall-shear pair of rows is processed by one
// CTA in one sweep.
template <bool WALLS, typename real>
__device__ __forceinline__ long long cut_units(const KArgs<real> &A, int c)
{
    long long u = ((long long)c * A.units) / A.nctas;
    if (WALLS && u > 0 && u < A.units) {
        int s, y;
        long long e;
        unit_run(A, u, s, y, e);
        // ny-2 is never a run's first row: one row back is ny-3, which is
        // row 2 itself when ny = 5
        if (y == A.ny - 2) { u -= 1; --y; }
        if (y == 2) u -= 1;
    }
    return u;
}

// Strip width and threads. A CTA owns a strip of up to STRIP columns; each
// thread owns CP adjacent columns. By default every kernel takes one column
// per thread (128 threads). LBM_FP32_PAIR=2 builds the FP32 staged kernel
// with column pairs (float2 arithmetic on the paired FP32 instructions, 64
// threads, bit-identical results): about a third fewer instructions, but with
// shared memory holding ~640 columns per SM in flight it runs half the warps,
// and the paired instructions keep the scalar latency, so it is slower.
#ifndef LBM_STRIP
#define LBM_STRIP 128
#endif
#ifndef LBM_FP32_PAIR
#define LBM_FP32_PAIR 1
#endif
constexpr int STRIP = LBM_STRIP;
template <typename real, bool STAGED>
__host__ __device__ constexpr int cols_per_thread()
{
    return (sizeof(real) == 4 && STAGED) ? LBM_FP32_PAIR : 1;
}
template <typename real, bool STAGED>
__host__ __device__ constexpr int threads_per_cta()
{
    return STRIP / cols_per_thread<real, STAGED>();
}

// Register allocation is held to LBM_FP32_THREADS_PER_SM resident FP32
// threads per SM (256 for FP64, which carries twice the state per thread).
// Halo duty: LBM_HALO_ONE_WARP puts the four halo columns on lanes 0..3 of
// warp 0 (and the two halo Laplacians on lanes 0..1 of the last warp), so the
// divergent halo path is issued by one warp per row instead of four.
#ifndef LBM_HALO_ONE_WARP
#define LBM_HALO_ONE_WARP 1
#endif


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
#define LBM_STAGE_AHEAD 2
#endif
constexpr int STAGE_AHEAD = LBM_STAGE_AHEAD;
// the wait for row j+1 comes before the barrier of iteration j, so that row
// must have been issued in an earlier iteration
static_assert(STAGE_AHEAD >= 1, "rows are issued at least one iteration before they are awaited");
constexpr int NSTAGE = 5 + STAGE_AHEAD;

// A stage holds one stencil row of the strip (local columns 0 .. STRIP-1) for
// the nine planes. Each plane segment starts on a 128-byte line when the strip
// does, so a copy touches no more lines than it needs.
__host__ __device__ constexpr int stage_pitch() { return STRIP; }

template <typename real>
constexpr size_t staged_smem_bytes()
{
    return (size_t)NSTAGE * 9 * stage_pitch() * sizeof(real) + NSTAGE * sizeof(uint64_t);
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
// The odd parts 3 w_i rho (e_i . u) are taken from the momentum m = rho u
// itself (mx, my; exact sums, no reciprocal), the even parts from u. The rest
// population is rho minus the eight moving ones (= rho - 2 sum c), so f_eq
// carries exactly rho and m up to unbiased rounding.
template <typename V>
__device__ __forceinline__ void feq_pairs(V rho, V ux, V uy, V mx, V my, V (&fe)[9])
{
    const V usq = fma_(ux, ux, mul_(uy, uy));
    const V base = fma_(usq, bc<V>(-1.5), bc<V>(1.0));
    const V r1 = mulk(rho, 1.0 / 9.0), r2 = mulk(rho, 1.0 / 36.0);
    const V s = add_(ux, uy), d = sub_(uy, ux);  // e.u of directions 5 (1,1) and 6 (-1,1)
    const V h = bc<V>(4.5);
    const V c1 = mul_(r1, fma_(mul_(ux, h), ux, base)), o1 = mulk(mx, 1.0 / 3.0);
    const V c2 = mul_(r1, fma_(mul_(uy, h), uy, base)), o2 = mulk(my, 1.0 / 3.0);
    const V c5 = mul_(r2, fma_(mul_(s, h), s, base)), o5 = mulk(add_(mx, my), 1.0 / 12.0);
    const V c6 = mul_(r2, fma_(mul_(d, h), d, base)), o6 = mulk(sub_(my, mx), 1.0 / 12.0);
    fe[1] = add_(c1, o1); fe[3] = sub_(c1, o1);
    fe[2] = add_(c2, o2); fe[4] = sub_(c2, o2);
    fe[5] = add_(c5, o5); fe[7] = sub_(c5, o5);
    fe[6] = add_(c6, o6); fe[8] = sub_(c6, o6);
    fe[0] = fma_(add_(add_(c1, c2), add_(c5, c6)), bc<V>(-2.0), rho);
}

// West, centre and east packs of CP adjacent ring columns c .. c+CP-1 on one
// ring row (c even for pairs: three aligned pair loads).
template <typename V>
struct Row3 {
    V w, c, e;
};
template <typename real, int CP, int SW>
__device__ __forceinline__ Row3<typename Pack<real, CP>::T> row3(const real (*S)[SW], int q, int c)
{
    using V = typename Pack<real, CP>::T;
    Row3<V> r;
    if constexpr (CP == 1) {
        r.w = S[q][c - 1];
        r.c = S[q][c];
        r.e = S[q][c + 1];
    } else {
        const float2 a = ldp<float2>(&S[q][c - 2]), b = ldp<float2>(&S[q][c]), d = ldp<float2>(&S[q][c + 2]);
        r.w = make_float2(a.y, b.x);
        r.c = b;
        r.e = make_float2(b.y, d.x);
    }
    return r;
}

// 12 x isotropic gradient from rows below (m), at (z) and above (p):
// (4(E - W) + (NE - NW) + (SE - SW), 4(N - S) + (NE - SE) + (NW - SW)).
template <typename V>
__device__ __forceinline__ void grad12(const Row3<V> &m, const Row3<V> &z, const Row3<V> &p, V &gx, V &gy)
{
    gx = fma_(sub_(z.e, z.w), bc<V>(4.0), add_(sub_(p.e, p.w), sub_(m.e, m.w)));
    gy = fma_(sub_(p.c, m.c), bc<V>(4.0), add_(sub_(p.e, m.e), sub_(p.w, m.w)));
}
// the negated gradient, for the pressure term of the force
template <typename V>
__device__ __forceinline__ void ngrad12(const Row3<V> &m, const Row3<V> &z, const Row3<V> &p, V &gx, V &gy)
{
    gx = fma_(sub_(z.w, z.e), bc<V>(4.0), add_(sub_(p.w, p.e), sub_(m.w, m.e)));
    gy = fma_(sub_(m.c, p.c), bc<V>(4.0), add_(sub_(m.e, p.e), sub_(m.w, p.w)));
}
// lap psi = 6 sum_i w_i (psi(x + e_i) - psi(x)) = (4 edges + corners - 20 psi) / 6
template <typename V>
__device__ __forceinline__ V lap9(const Row3<V> &m, const Row3<V> &z, const Row3<V> &p)
{
    const V edges = add_(add_(z.w, z.e), add_(m.c, p.c));
    const V corners = add_(add_(m.w, m.e), add_(p.w, p.e));
    return mulk(fma_(z.c, bc<V>(-20.0), fma_(edges, bc<V>(4.0), corners)), 1.0 / 6.0);
}

// MRT relaxation (Eq. 2.1) f* = f - M^-1 S M (f - f_eq) in the Lallemand-Luo
// moment basis (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy): the non-
// equilibrium moments d = f - f_eq are scaled by s_k / |row_k|^2 and mapped
// back with M^T (the rows are orthogonal). The density is conserved.
template <typename V, typename real>
__device__ __forceinline__ void mrt_relax(const KArgs<real> &A, const V (&f)[9], const V (&fe)[9], V (&fs)[9])
{
    V d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = sub_(f[i], fe[i]);
    const V s14 = add_(add_(d[1], d[2]), add_(d[3], d[4]));
    const V s58 = add_(add_(d[5], d[6]), add_(d[7], d[8]));
    const V e = fma_(d[0], bc<V>(-4.0), sub_(mul_(s58, bc<V>(2.0)), s14));    // -4 d0 - s14 + 2 s58
    const V ep = fma_(d[0], bc<V>(4.0), sub_(s58, mul_(s14, bc<V>(2.0))));    //  4 d0 - 2 s14 + s58
    const V a13 = sub_(d[1], d[3]), bx = add_(sub_(d[5], d[6]), sub_(d[8], d[7]));
    const V a24 = sub_(d[2], d[4]), by = sub_(add_(d[5], d[6]), add_(d[7], d[8]));
    const V jx = add_(a13, bx), qx = fma_(a13, bc<V>(-2.0), bx);
    const V jy = add_(a24, by), qy = fma_(a24, bc<V>(-2.0), by);
    const V pxx = sub_(add_(d[1], d[3]), add_(d[2], d[4]));
    const V pxy = sub_(add_(d[5], d[7]), add_(d[6], d[8]));
    const V E = mul_(e, bcr<V>(A.m_e)), P = mul_(ep, bcr<V>(A.m_eps));
    const V JX = mul_(jx, bcr<V>(A.m_j)), JY = mul_(jy, bcr<V>(A.m_j));
    const V QX = mul_(qx, bcr<V>(A.m_q)), QY = mul_(qy, bcr<V>(A.m_q));
    const V XX = mul_(pxx, bcr<V>(A.m_nu)), XY = mul_(pxy, bcr<V>(A.m_nu));
    // M^T applied to the scaled moments
    const V b14 = sub_(mul_(P, bc<V>(-2.0)), E);  // -E - 2P
    const V xj = fma_(QX, bc<V>(-2.0), JX), yj = fma_(QY, bc<V>(-2.0), JY);
    const V b58 = fma_(E, bc<V>(2.0), P);         // 2E + P
    const V xq = add_(JX, QX), yq = add_(JY, QY);
    fs[0] = sub_(f[0], mul_(sub_(P, E), bc<V>(4.0)));
    fs[1] = sub_(f[1], add_(add_(b14, xj), XX));
    fs[2] = sub_(f[2], sub_(add_(b14, yj), XX));
    fs[3] = sub_(f[3], add_(sub_(b14, xj), XX));
    fs[4] = sub_(f[4], sub_(sub_(b14, yj), XX));
    fs[5] = sub_(f[5], add_(add_(add_(b58, xq), yq), XY));
    fs[6] = sub_(f[6], sub_(add_(sub_(b58, xq), yq), XY));
    fs[7] = sub_(f[7], add_(sub_(sub_(b58, xq), yq), XY));
    fs[8] = sub_(f[8], sub_(sub_(add_(b58, xq), yq), XY));
}

// Non-equilibrium extrapolation of a pressure column (Sec. 2.2 ends) from its
// interior neighbour x_f (density rho_f, velocity v, momentum m = rho_f v,
// populations f):
// f*_i = f_eq_i(rho_b, v) + (1 - 1/tau)(f_i - f_eq_i(rho_f, v)), with
// f_eq(rho_b, v) = (rho_b / rho_f) f_eq(rho_f, v).
template <typename real>
__device__ __forceinline__ void column_extrapolate(const KArgs<real> &A, real rho_b, real rho_f, real vx, real vy,
                                                   real mx, real my, const real (&f)[9], real (&fs)[9])
{
    real ff[9];
    feq_pairs<real>(rho_f, vx, vy, mx, my, ff);
    const real sc = mul_(rho_b, rcp_(rho_f));
#pragma unroll
    for (int i = 0; i < 9; ++i) fs[i] = fma_(sc, ff[i], mul_(A.omb, sub_(f[i], ff[i])));
}

// Wall pressure (Eq. 2.4 in mesh units) at ring column cc of row q0:
// k^2 p0 - kappa rho lap rho - (kappa/2)|grad rho|^2, with k^2 p0 = phi + rho/3
// and lap rho = lap (the node's Laplacian).
template <typename real, int SW>
__device__ __forceinline__ real wall_pressure(const KArgs<real> &A, const real (*R)[SW], const real (*P)[SW],
                                              real lap, int qm, int q0, int qp, int cc, real rho)
{
    real grx, gry;
    grad12<real>(row3<real, 1, SW>(R, qm, cc), row3<real, 1, SW>(R, q0, cc), row3<real, 1, SW>(R, qp, cc), grx,
                 gry);
    grx = mulk(grx, 1.0 / 12.0);
    gry = mulk(gry, 1.0 / 12.0);
    const real k2p0 = add_(P[q0][cc], mulk(rho, 1.0 / 3.0));
    const real t = fma_(mul_(A.kappa, rho), -lap, k2p0);
    return fma_(fma_(grx, grx, mul_(gry, gry)), mul_(real(-0.5), A.kappa), t);
}

// h + l += x for an unevaluated FP32 pair (h, l): Knuth's two-sum gives the
// rounding error of h + x exactly, which l collects.
__device__ __forceinline__ void two_sum_acc(float &h, float &l, float x)
{
    const float s = __fadd_rn(h, x);
    const float bp = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    h = s;
    l = __fadd_rn(l, err);
}

// Per-thread diagnostic accumulators of the states read. The density sum is
// kept in the working precision and flushed every 16 rows (at most 16 terms
// per flush): FP64 builds into a double, FP32 builds into a compensated FP32
// pair (two-sum, on the FP32 pipes: GB300 runs FP64 at 1/64 of that rate),
// which the CTA reduction combines in FP64. The density range is tracked
// with min / max, and a non-finite density shows up in the mass sum (min /
// max ignore NaN).
template <typename real, int CP>
struct Acc {
    using V = typename Pack<real, CP>::T;
    static constexpr bool PAIR = sizeof(real) == 4;
    double mass, J;
    float mhi, mlo;  // FP32 builds: the flushed sums as hi + lo
    V macc, rmin, rmax;
    real tmin, tmax, pmin, pmax;
    __device__ __forceinline__ void reset()
    {
        mass = 0.0; J = 0.0; mhi = mlo = 0.f; macc = bc<V>(0.0);
        rmin = bc<V>(INFINITY); rmax = bc<V>(-INFINITY);
        tmin = pmin = real(INFINITY); tmax = pmax = real(-INFINITY);
    }
    __device__ __forceinline__ void flush()
    {
        if constexpr (PAIR) {
#pragma unroll
            for (int k = 0; k < CP; ++k) two_sum_acc(mhi, mlo, (float)el(macc, k));
        } else {
#pragma unroll
            for (int k = 0; k < CP; ++k) mass += (double)el(macc, k);
        }
        macc = bc<V>(0.0);
    }
    // a density that is not in (0, 1e30) or a non-finite mass
    __device__ __forceinline__ bool bad() const
    {
        bool b = PAIR ? !(mhi - mhi == 0.f) : !(mass - mass == 0.0);
#pragma unroll
        for (int k = 0; k < CP; ++k) b = b || !(el(rmin, k) > real(0)) || !(el(rmax, k) < real(1e30));
        return b;
    }
};

__device__ __forceinline__ float vmin_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float vmax_(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmin_(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ double vmax_(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float2 vmin_(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ float2 vmax_(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }

// Static shared-memory working set of a CTA: the 8-row stencil ring (density,
// EOS potential, Laplacian; strip plus two halo columns per side) and the
// reduction scratch.
template <typename real, int BLOCK>
struct Smem {
    __align__(16) real rho[RING][STRIP + 4];
    __align__(16) real phi[RING][STRIP + 4];
    __align__(16) real lap[RING][STRIP + 4];
    double red[BLOCK / 32][2];
    real ext[BLOCK / 32][4];
    int bad;
};

// One fused time step (MODE_STEP) or the macroscopic fields (MODE_FIELDS).
//
// Per segment (strip of columns x0 .. x0+xw-1, fluid rows ya .. yb-1) the CTA
// runs iterations yy = ya-2 .. yb+2 with one barrier each:
//   (1) (unstaged) re-read (L1) the populations of the collision row r = yy-3;
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
// Each thread owns CP adjacent columns (c0 = CP tid). STAGED: the strip's
// populations of each stencil row (9 plane segments of xw values) are
// streamed by one producer thread with bulk asynchronous copies into a ring
// of NSTAGE shared-memory stages, issued STAGE_AHEAD + 1 rows ahead; consumers
// read densities and collision populations from the stage (needs nx and the
// strip width to be multiples of 4 for 16-byte aligned copies, so pairs are
// always complete and a pressure column's interior neighbour is the other
// column of its own pair). Otherwise (CP = 1) each thread loads its column
// with one row of register prefetch and re-reads the collision row from L1.
// In both variants four halo lanes load the two columns beyond each strip
// edge with one row of register prefetch.
template <typename real, bool WALLS, bool PRES, int MODE, int BLOCK, bool STAGED, int CP, bool PADDED,
          typename IX = int>
__device__ __forceinline__ void run_segment(const KArgs<real> &A, const Geom<real> &G, int s, int ya, int yb,
                                            Smem<real, BLOCK> &S, real *stages, uint64_t *bars,
                                            RingPos &ring_next, Acc<real, CP> &acc, bool &lost)
{
    using V = typename Pack<real, CP>::T;
    constexpr int SW = STRIP + 4;
    constexpr int NW = BLOCK / 32;
    constexpr int PRODUCER = BLOCK - 1;  // no halo duty
    constexpr int SP = stage_pitch();
    static_assert(CP * BLOCK == STRIP, "a CTA covers one strip");
    static_assert(CP == 1 || STAGED, "column pairs need the staged kernel");
    static_assert(NW == 2 || NW >= 4, "halo lanes: two warps or four and more");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const real third = real(1.0 / 3.0);
    const int nx = G.nx, ny = G.ny;
    const int P = PADDED ? G.pitch : G.nx;  // plane pitch; columns nx .. P-1 are padding
    const int rstride = 9 * P;   // row stride of the population layout f[y][i][x]
    // push targets of directions 1..8 relative to the source slot index
    const int o1 = P + 1, o2 = rstride + 2 * P, o3 = 3 * P - 1, o4 = 4 * P - rstride;
    const int o5 = rstride + 5 * P + 1, o6 = rstride + 6 * P - 1, o7 = 7 * P - rstride - 1;
    const int o8 = 8 * P - rstride + 1;
    real b_rho1[CP], b_v1[CP], t_v2[CP];  // wall-pair carries (rows 1 -> 2, ny-3 -> ny-2)
#pragma unroll
    for (int k = 0; k < CP; ++k) b_rho1[k] = b_v1[k] = t_v2[k] = real(0);

    const int x0 = s * G.W;
    const int xw = min(G.W, nx - x0);
    const int c0 = CP * tid;  // first local column of this thread
    const bool active = c0 < xw;
    const int xa = x0 + c0;   // its global column
    // pressure columns: with pairs, x = 0 is element 0 and x = nx-1 element 1
    const bool pin = PRES && active && xa == 0;
    const bool pout = PRES && active && xa + CP - 1 == nx - 1;
    const bool anyp = pin || pout;
    // CP = 1: a pressure column sums and collides its interior neighbour's column
    const int scol = (CP == 1) ? ((pin ? 1 : (pout ? nx - 2 : xa)) - x0) : c0;  // stage column
    const int ccol = scol + 2;                                                   // ring column
    // pushes never wrap or leave the lattice in x
    const bool x_inner = !anyp && (PRES || (xa >= 1 && xa + CP - 1 <= nx - 2));

    // Halo columns local -2, -1, xw, xw+1 (four lanes: lane 0 of warps 0..3,
    // or lanes 0 and 1 of two warps). hmode 1: density of column hx; 2 / 3:
    // inlet / outlet column density derived from column hx = 1 / nx-2 (clamp
    // beyond the pressure columns).
    int hidx = -1;
    if (LBM_HALO_ONE_WARP) { if (warp == 0 && lane < 4) hidx = lane; }
    else if (NW >= 4) { if (lane == 0 && warp < 4) hidx = warp; }
    else if (lane < 2) hidx = 2 * warp + lane;
    int hmode = 0, hx = 0, hcol = 0;
    if (hidx >= 0) {
        const int hloc = (hidx < 2) ? (hidx - 2) : (xw + hidx - 2);
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
    int lhalo = -1;
    if (LBM_HALO_ONE_WARP) { if (warp == NW - 1 && lane < 2) lhalo = lane == 0 ? 1 : xw + 2; }
    else if (NW >= 4) lhalo = (lane == 1 && warp == 1) ? 1 : ((lane == 1 && warp == 2) ? xw + 2 : -1);
    else if (lane == 2) lhalo = warp == 0 ? 1 : xw + 2;

    const real *__restrict__ col_in = G.fin + x0 + scol;
    const real *__restrict__ hal_in = G.fin + hx;
    const int nrows = yb - ya + 4;  // stencil rows ya-2 .. yb+1
    V pf[9];
    real hf[9];
    real add_next = real(0);  // wetting offset of the next stencil row (mirrored wall ghost)
    // halo (and, without staging, own-column) loads of stencil row yy
    auto prefetch = [&](int yy) {
        bool mir;
        const IX row = (IX)map_row<WALLS>(yy, ny, mir) * rstride;
        add_next = mir ? A.wet : real(0);
        if constexpr (!STAGED) {
            if (active) {
#pragma unroll
                for (int i = 0; i < 9; ++i) pf[i] = __ldg(col_in + row + i * P);
            }
        }
        if (hmode) {
#pragma unroll
            for (int i = 0; i < 9; ++i) hf[i] = __ldg(hal_in + row + i * P);
        }
    };
    // producer: stream stencil row j of this segment into the next stage
    RingPos ring_issue = ring_next;
    auto issue = [&](int j) {
        if (j < nrows) {
            if (tid == PRODUCER) {
                bool mir;
                const IX row = (IX)map_row<WALLS>(ya - 2 + j, ny, mir) * rstride;
                const uint32_t st = ring_issue.s;
                real *dst = stages + (size_t)st * 9 * SP;
                const real *src = G.fin + row + x0;
                // whole 16-byte groups: a ragged last strip also copies padding columns
                const uint32_t bytes = (uint32_t)(((xw + 3) & ~3) * sizeof(real));
                mbar_arrive_expect_tx(&bars[st], 9 * bytes);
#pragma unroll
                for (int i = 0; i < 9; ++i) bulk_copy_g2s(dst + i * SP, src + i * P, bytes, &bars[st]);
            }
            ring_issue.advance();
        }
    };
    // stage of the collision row (three rows behind the consumed row)
    RingPos ring_coll = ring_next;
    for (int k = 0; k < NSTAGE - 3; ++k) ring_coll.advance();
#pragma unroll
    for (int i = 0; i < 9; ++i) { pf[i] = bc<V>(0.0); hf[i] = real(0); }
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
        const uint32_t st_cons = ring_next.s, st_coll = ring_coll.s;

        // (1) populations of the collision row (read from HBM three iterations ago)
        V f[9];
        if constexpr (!STAGED) {
            if (collide && active) {
                const real *src = col_in + (IX)r * rstride;
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = __ldg(src + i * P);
            }
        }

        // (2) density and EOS potential of stencil row yy (staged: its
        //     stage was completed before the previous barrier)
        if (yy <= yb + 1) {
            const real add = add_next;
            const int rs = yy & (RING - 1);
            V rho_own = bc<V>(0.0);
            real rho_h = real(0);
            if constexpr (STAGED) {
                const real *stg = stages + (size_t)st_cons * 9 * SP + scol;
                if (active) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) pf[i] = ldp<V>(stg + i * SP);
                }
            }
            if (active) {
                V sum = add_(add_(add_(pf[0], pf[1]), add_(pf[2], pf[3])), add_(add_(pf[4], pf[5]), add_(pf[6], pf[7])));
                sum = add_(sum, pf[8]);
                if (anyp) {
                    if constexpr (CP == 1) {
                        set_el(sum, 0, column_density(A, G, pout, el(sum, 0)));
                    } else {
                        // the pair (0, 1) or (nx-2, nx-1): the column takes the other element's sum
                        if (pin) set_el(sum, 0, column_density(A, G, false, el(sum, 1)));
                        if (pout) set_el(sum, CP - 1, column_density(A, G, true, el(sum, CP - 2)));
                    }
                }
                rho_own = add_(sum, bcr<V>(add));
            }
            if (hmode) {
                real sum = add_(add_(add_(hf[0], hf[1]), add_(hf[2], hf[3])), add_(add_(hf[4], hf[5]), add_(hf[6], hf[7])));
                sum = add_(sum, hf[8]);
                rho_h = add_(hmode == 1 ? sum : column_density(A, G, hmode == 3, sum), add);
            }
            if (yy + 1 <= yb + 1) prefetch(yy + 1);
            if (active) {
                stp<V>(&S.rho[rs][c0 + 2], rho_own);
                stp<V>(&S.phi[rs][c0 + 2], eos_phi<V>(A, rho_own));
            }
            if (hmode) {
                S.rho[rs][hcol] = rho_h;
                S.phi[rs][hcol] = eos_phi<real>(A, rho_h);
            }
        }

        // (3) Laplacian of row yy-2 on local columns -1 .. xw
        if (yy >= ya + 1) {
            const int lr = (yy - 2) & (RING - 1), lm = (yy - 3) & (RING - 1), lp = (yy - 1) & (RING - 1);
            if (active) {
                const V L = lap9<V>(row3<real, CP, SW>(S.rho, lm, c0 + 2), row3<real, CP, SW>(S.rho, lr, c0 + 2),
                                    row3<real, CP, SW>(S.rho, lp, c0 + 2));
                stp<V>(&S.lap[lr][c0 + 2], L);
            }
            if (lhalo >= 0)
                S.lap[lr][lhalo] = lap9<real>(row3<real, 1, SW>(S.rho, lm, lhalo), row3<real, 1, SW>(S.rho, lr, lhalo),
                                              row3<real, 1, SW>(S.rho, lp, lhalo));
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
                for (int i = 0; i < 9; ++i) f[i] = ldp<V>(sp + i * SP);
            }
            const int q0 = r & (RING - 1), qm = (r - 1) & (RING - 1), qp = (r + 1) & (RING - 1);
            V ngpx, ngpy, glx, gly;
            ngrad12<V>(row3<real, CP, SW>(S.phi, qm, ccol), row3<real, CP, SW>(S.phi, q0, ccol),
                       row3<real, CP, SW>(S.phi, qp, ccol), ngpx, ngpy);
            grad12<V>(row3<real, CP, SW>(S.lap, qm, ccol), row3<real, CP, SW>(S.lap, q0, ccol),
                      row3<real, CP, SW>(S.lap, qp, ccol), glx, gly);
            const V rho = ldp<V>(&S.rho[q0][ccol]);
            const V kr = mul_(bcr<V>(A.kappa), rho);
            const V Fx = add_(mulk(fma_(kr, glx, ngpx), 1.0 / 12.0), bcr<V>(A.gx));
            const V Fy = add_(mulk(fma_(kr, gly, ngpy), 1.0 / 12.0), bcr<V>(A.gy));
            const V jx = add_(add_(sub_(f[1], f[3]), sub_(f[5], f[6])), sub_(f[8], f[7]));
            const V jy = sub_(add_(sub_(f[2], f[4]), add_(f[5], f[6])), add_(f[7], f[8]));
            const V irho = rcp_(rho);
            const V ux = mul_(jx, irho), uy = mul_(jy, irho);
            const V hFi = mul_(irho, bc<V>(0.5));
            const V vx = fma_(hFi, Fx, ux), vy = fma_(hFi, Fy, uy);
            // own-column density (a pressure column's own is rho_b)
            const V rho_own = (CP == 1 && anyp) ? bcr<V>(S.rho[q0][tid + 2]) : rho;

            if (MODE == MODE_STEP) {
                V fs[9];
                {
                    // shifted equilibrium: momentum j + ushift F, velocity (j + ushift F) / rho
                    const V mx = fma_(bcr<V>(A.ushift), Fx, jx), my = fma_(bcr<V>(A.ushift), Fy, jy);
                    V fe[9];
                    feq_pairs<V>(rho, mul_(mx, irho), mul_(my, irho), mx, my, fe);
                    if (A.mrt) {
                        mrt_relax<V, real>(A, f, fe, fs);
                    } else {
#pragma unroll
                        for (int i = 0; i < 9; ++i) fs[i] = fma_(sub_(fe[i], f[i]), bcr<V>(A.inv_tau), f[i]);
                    }
                }
                if (anyp) {
                    // pressure column: extrapolate from the interior neighbour
                    // (CP = 1: this thread's values are the neighbour's; pairs:
                    // the other element of the pair)
                    const int kc = pin ? 0 : CP - 1, kf = (CP == 1) ? 0 : (pin ? 1 : CP - 2);
                    real ff[9], fsc[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) ff[i] = el(f[i], kf);
                    // momentum of the neighbour's v = (j + F/2) / rho
                    const real mvx = fma_(real(0.5), el(Fx, kf), el(jx, kf));
                    const real mvy = fma_(real(0.5), el(Fy, kf), el(jy, kf));
                    column_extrapolate<real>(A, el(rho_own, kc), el(rho, kf), el(vx, kf), el(vy, kf), mvx, mvy, ff,
                                             fsc);
#pragma unroll
                    for (int i = 0; i < 9; ++i) set_el(fs[i], kc, fsc[i]);
                }
                real *const out = G.fout;
                const IX oi = (IX)r * rstride + xa;  // slot of (xa, r) in plane 0
                const bool y_inner = WALLS ? (r >= 2 && r <= ny - 3) : (r >= 1 && r <= ny - 2);
                if (x_inner && y_inner) {
                    if constexpr (CP == 1) {
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
                        // directions without an x component keep the pair together
                        stp<V>(out + oi, fs[0]);
                        stp<V>(out + oi + o2, fs[2]);
                        stp<V>(out + oi + o4, fs[4]);
                        out[oi + o1] = el(fs[1], 0); out[oi + o1 + 1] = el(fs[1], 1);
                        out[oi + o3] = el(fs[3], 0); out[oi + o3 + 1] = el(fs[3], 1);
                        out[oi + o5] = el(fs[5], 0); out[oi + o5 + 1] = el(fs[5], 1);
                        out[oi + o6] = el(fs[6], 0); out[oi + o6 + 1] = el(fs[6], 1);
                        out[oi + o7] = el(fs[7], 0); out[oi + o7 + 1] = el(fs[7], 1);
                        out[oi + o8] = el(fs[8], 0); out[oi + o8 + 1] = el(fs[8], 1);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < CP; ++k) {
                        const int xk = xa + k;
                        const IX ok = oi + k;
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            const int ty = r + ey_(i);
                            if (WALLS && (ty == 0 || ty == ny - 1)) {
                                // half-way bounce-back into the opposite slot of this node
                                out[ok + opp_(i) * P] = el(fs[i], k);
                            } else {
                                int tx = xk + ex_(i);
                                if (PRES) {
                                    if (tx < 0 || tx >= nx) continue;  // leaves through the column
                                } else {
                                    tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
                                }
                                int tyw = ty;
                                if (!WALLS) tyw = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
                                out[(IX)tyw * rstride + i * P + tx] = el(fs[i], k);
                            }
                        }
                    }
                }
                acc.macc = add_(acc.macc, rho_own);
                acc.rmin = vmin_(acc.rmin, rho);
                acc.rmax = vmax_(acc.rmax, rho);
            } else {
#pragma unroll
                for (int k = 0; k < CP; ++k) {
                    const bool pk = (k == 0 && pin) || (k == CP - 1 && pout);
                    const int kv = (CP == 1 || !pk) ? k : (k == 0 ? 1 : CP - 2);  // a column reports v_f
                    const long long oi = (long long)r * nx + xa + k;
                    A.o_rho[oi] = el(rho_own, k);
                    A.o_vx[oi] = el(vx, kv);
                    A.o_vy[oi] = el(vy, kv);
                }
            }

            if (WALLS && (r <= 2 || r >= ny - 3)) {
                // wall shear: quadratic through v = 0 on the half-way plane and
                // v at distances 1/2 and 3/2; wall pressure: Eq. 2.4 in mesh units
#pragma unroll
                for (int k = 0; k < CP; ++k) {
                    const bool pk = (k == 0 && pin) || (k == CP - 1 && pout);
                    if (pk) continue;
                    const int cc = ccol + k, xk = xa + k;
                    const real rk = el(rho, k), vk = el(vx, k);
                    if (r == 1) {
                        b_rho1[k] = rk;
                        b_v1[k] = vk;
                        const real pw = wall_pressure<real, SW>(A, S.rho, S.phi, S.lap[q0][cc], qm, q0, qp, cc, rk);
                        if (MODE == MODE_STEP) { acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw); }
                        else A.o_pw[xk] = pw;
                    }
                    if (r == ny - 3) t_v2[k] = vk;
                    if (r == 2) {
                        const real tw = mul_(mul_(b_rho1[k], A.nu), mul_(fma_(real(9), b_v1[k], -vk), third));
                        if (MODE == MODE_STEP) { acc.J += (double)tw; acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw); }
                        else A.o_tw[xk] = tw;
                    }
                    if (r == ny - 2) {
                        const real tw = mul_(mul_(rk, A.nu), mul_(fma_(real(9), vk, -t_v2[k]), third));
                        const real pw = wall_pressure<real, SW>(A, S.rho, S.phi, S.lap[q0][cc], qm, q0, qp, cc, rk);
                        if (MODE == MODE_STEP) {
                            acc.J += (double)tw;
                            acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw);
                            acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw);
                        } else {
                            A.o_tw[nx + xk] = tw;
                            A.o_pw[nx + xk] = pw;
                        }
                    }
                }
            }
        }
        ring_coll.advance();
        if ((j & 15) == 15) acc.flush();  // uniform: every thread added at most 16 densities
    }
    __syncthreads();  // ring and stage reuse by the next segment
}

// Fixed-order CTA reduction of the accumulators; thread 0 receives the totals.
template <typename real, int BLOCK, int CP, typename SM>
__device__ __forceinline__ void cta_reduce(Acc<real, CP> &acc, SM &S, double &m, double &j, real (&e)[4],
                                           bool &anybad)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    acc.flush();
    // only warps that hold wall rows carry a wall-shear sum: the others skip
    // its FP64 shuffles (GB300 runs FP64 at 1/64 of the FP32 rate)
    const bool anyJ = __any_sync(0xffffffffu, acc.J != 0.0);
    if constexpr (Acc<real, CP>::PAIR) {
        // FP32 builds: the pairs summed across the warp with two-sum (lane 0's
        // result is the one kept), then one FP64 addition
        float h = acc.mhi, l = acc.mlo;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
            two_sum_acc(h, l, h2);
            l = __fadd_rn(l, l2);
        }
        acc.mass = (double)h + (double)l;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if constexpr (!Acc<real, CP>::PAIR) acc.mass += __shfl_xor_sync(0xffffffffu, acc.mass, o);
        if (anyJ) acc.J += __shfl_xor_sync(0xffffffffu, acc.J, o);
        acc.tmin = fmin(acc.tmin, __shfl_xor_sync(0xffffffffu, acc.tmin, o));
        acc.tmax = fmax(acc.tmax, __shfl_xor_sync(0xffffffffu, acc.tmax, o));
        acc.pmin = fmin(acc.pmin, __shfl_xor_sync(0xffffffffu, acc.pmin, o));
        acc.pmax = fmax(acc.pmax, __shfl_xor_sync(0xffffffffu, acc.pmax, o));
    }
    const bool wbad = __any_sync(0xffffffffu, acc.bad());
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

// PADDED: the population rows have a plane pitch above nx (taken from the
// arguments); otherwise the pitch is nx itself, which the compiler can share
// with the bounds arithmetic (4% faster than carrying both). IX: the type of
// population offsets, int while 9 pitch ny < 2^31, long long above.
template <typename real, bool WALLS, bool PRES, int MODE, bool STAGED, bool PADDED, typename IX = int>
__global__ void __launch_bounds__(threads_per_cta<real, STAGED>(),
                                  MinBlocks<real, threads_per_cta<real, STAGED>()>::value)
    step_kernel(const KArgs<real> A)
{
    constexpr int CP = cols_per_thread<real, STAGED>();
    constexpr int BLOCK = threads_per_cta<real, STAGED>();
    constexpr int SP = stage_pitch();
    extern __shared__ __align__(128) unsigned char dsm[];
    real *const stages = reinterpret_cast<real *>(dsm);
    uint64_t *const bars = reinterpret_cast<uint64_t *>(dsm + (size_t)NSTAGE * 9 * SP * sizeof(real));
    __shared__ Smem<real, BLOCK> S;

    const int tid = threadIdx.x;
    const int cta = A.reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    long long u = cut_units<WALLS>(A, cta);
    const long long u1 = cut_units<WALLS>(A, cta + 1);
    const Geom<real> G{A.fin, A.fout, A.nx, A.ny, A.W, A.pitch, A.rho_in_g, A.rho_in_l, A.rho_out_g, A.rho_out_l};

    Acc<real, CP> acc;
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
        int s, ya;
        long long run_end;
        unit_run(A, u, s, ya, run_end);
        const long long ue = min(u1, run_end);
        const int yb = ya + (int)(ue - u);
        u = ue;
        run_segment<real, WALLS, PRES, MODE, BLOCK, STAGED, CP, PADDED, IX>(A, G, s, ya, yb, S, stages, bars, ring_next,
                                                                       acc, lost);
    }

    if (STAGED && lost) atomicOr(A.err, 2);
    if (MODE != MODE_STEP) return;

    double m, j;
    real e[4];
    bool anybad;
    cta_reduce<real, BLOCK, CP>(acc, S, m, j, e, anybad);
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
    int nx, ny, W, pitch;
    real rho_in_g, rho_in_l, rho_out_g, rho_out_l;
};

struct BatchSeg {
    int chan, strip, ya, yb;
};

template <typename real, bool WALLS, bool PRES, bool STAGED>
__global__ void __launch_bounds__(threads_per_cta<real, STAGED>(),
                                  MinBlocks<real, threads_per_cta<real, STAGED>()>::value)
    batch_step_kernel(const KArgs<real> A, const BatchChan<real> *__restrict__ chans,
                      const BatchSeg *__restrict__ segs, const int *__restrict__ cta_begin,
                      double *__restrict__ seg_mass, double *__restrict__ seg_J, real *__restrict__ seg_ext)
{
    constexpr int CP = cols_per_thread<real, STAGED>();
    constexpr int BLOCK = threads_per_cta<real, STAGED>();
    constexpr int SP = stage_pitch();
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
        const Geom<real> G{A.fin + ch.off, A.fout + ch.off, ch.nx, ch.ny, ch.W, ch.pitch,
                           ch.rho_in_g, ch.rho_in_l, ch.rho_out_g, ch.rho_out_l};
        Acc<real, CP> acc;
        acc.reset();
        run_segment<real, WALLS, PRES, MODE_STEP, BLOCK, STAGED, CP, true>(A, G, sg.strip, sg.ya, sg.yb, S, stages,
                                                                          bars, ring_next, acc, lost);
        double m, j;
        real e[4];
        bool anybad;
        cta_reduce<real, BLOCK, CP>(acc, S, m, j, e, anybad);
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

// f = f_eq(rho0, 0) at every node (rho0: nx x ny; populations with plane
// pitch P, 64-bit offsets). Padding columns are zeroed.
template <typename real>
__global__ void init_kernel(const double *__restrict__ rho0, real *__restrict__ fa,
                            real *__restrict__ fb, int nx, int P, int ny)
{
    const int n = P * ny;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int y = k / P, x = k - y * P;
        real fe[9];
        feq_pairs<real>(x < nx ? (real)rho0[(long long)y * nx + x] : real(0), real(0), real(0), real(0), real(0), fe);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fa[(long long)(9 * y + i) * P + x] = fe[i];
            fb[(long long)(9 * y + i) * P + x] = fe[i];
        }
    }
}

// Fixed-order reduction of the per-CTA partials into out[0..6]:
// mass, J, tw_min, tw_max, pw_min, pw_max, err. One block of 256 threads:
// strided per-thread sums, warp butterflies (extrema in the partials' own
// precision, exact), then the eight warps in order.
template <typename real>
__global__ void diag_kernel(const double *__restrict__ mass_part, const double *__restrict__ J_acc,
                            const real *__restrict__ ext, const int *__restrict__ err, int nctas,
                            double *__restrict__ out)
{
    __shared__ double sm[8], sj[8];
    __shared__ real se[4][8];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    double m = 0.0, j = 0.0;
    real e0 = real(INFINITY), e1 = real(-INFINITY), e2 = real(INFINITY), e3 = real(-INFINITY);
    for (int c = t; c < nctas; c += 256) {
        m += mass_part[c];
        j += J_acc[c];
        e0 = fmin(e0, ext[4 * c + 0]);
        e1 = fmax(e1, ext[4 * c + 1]);
        e2 = fmin(e2, ext[4 * c + 2]);
        e3 = fmax(e3, ext[4 * c + 3]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m += __shfl_xor_sync(0xffffffffu, m, o);
        j += __shfl_xor_sync(0xffffffffu, j, o);
        e0 = fmin(e0, __shfl_xor_sync(0xffffffffu, e0, o));
        e1 = fmax(e1, __shfl_xor_sync(0xffffffffu, e1, o));
        e2 = fmin(e2, __shfl_xor_sync(0xffffffffu, e2, o));
        e3 = fmax(e3, __shfl_xor_sync(0xffffffffu, e3, o));
    }
    if (lane == 0) {
        sm[w] = m; sj[w] = j;
        se[0][w] = e0; se[1][w] = e1; se[2][w] = e2; se[3][w] = e3;
    }
    __syncthreads();
    if (t == 0) {
        double M = 0.0, Jt = 0.0;
        real a0 = se[0][0], a1 = se[1][0], a2 = se[2][0], a3 = se[3][0];
        for (int k = 0; k < 8; ++k) {
            M += sm[k];
            Jt += sj[k];
            a0 = fmin(a0, se[0][k]); a1 = fmax(a1, se[1][k]);
            a2 = fmin(a2, se[2][k]); a3 = fmax(a3, se[3][k]);
        }
        out[0] = M; out[1] = Jt;
        out[2] = (double)a0; out[3] = (double)a1; out[4] = (double)a2; out[5] = (double)a3;
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
        if (c == 0 && err) *err = 0;
    }
}

} // namespace lbm

#include "lbm_rows2.cuh"
