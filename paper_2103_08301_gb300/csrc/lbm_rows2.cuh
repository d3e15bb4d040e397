// Row-pair variant of the FP32 staged step (MODE_STEP): each thread owns one
// column and takes two consecutive rows per iteration, the pair held in a
// float2 and computed with the paired FP32 instructions (__ffma2_rn and
// friends), which round every element exactly as the scalar operations do.
// The arithmetic is the same pack code as the one-row kernel's, so the two
// kernels give identical bits; only the schedule differs:
//   - the loop bookkeeping, barriers and stage waits of an iteration are
//     shared by two nodes per thread, and the method's arithmetic issues one
//     instruction per two nodes;
//   - strips are at most R2_BLOCK - 4 columns wide and lane t holds local column
//     t - 2, so the two halo columns on each side are lanes of their own: no
//     divergent halo duty (which cost 8% as a one-warp duty); the stage holds
//     each stencil row with a four-column margin on both sides (columns
//     x0-4 .. x0+W+3), so the halo densities are summed from shared memory;
//   - one producer thread stages each stencil row with a single 2-D tensor
//     (TMA) load of 132 columns by 9 planes (cp.async.bulk.tensor through
//     the tensor-map kernel parameter); strips whose halo wraps around a
//     periodic x take nine plane copies and the wrap copies instead (plain
//     cp.async.bulk). The batch kernel can read its channels' maps from
//     device memory, but by default it takes the plane copies (faster there:
//     58.9k against 56.3k MLUPS on the 64-channel sweep). Nine copies per row in
//     place of one load cost 7% of the step;
//   - every thread waits on the stage's mbarrier itself, so a pair issued
//     half an iteration before it is read needs no publishing barrier; three
//     pair slots (six rows) suffice.
// Iteration k handles stencil rows yy0 = ya-2+2k and yy0+1:
//   (1) wait for their stage; density and phi of both rows (own and halo
//       columns) into the 8-row ring;                      --- barrier A ---
//   (2) issue the pair k+1 into the slot of pair k-2; Laplacian of rows
//       yy0-1, yy0 on local columns -1 .. xw;              --- barrier B ---
//   (3) force, collision, boundaries and push of rows yy0-2, yy0-1 (pair k-1,
//       k >= 2; the second row only if it is below yb).
// Restricted to strips and pitches that are multiples of 4 and, with periodic
// x, to nx a multiple of 4 (the wrapped halo columns are copied as one
// 16-byte group from each end of the row).
#pragma once

namespace lbm {

constexpr int R2_SLOTS = 3;            // pair slots of the stage ring
// Threads of a row-pair CTA (one column each).
#ifndef LBM_R2_BLOCK
#define LBM_R2_BLOCK 128
#endif
constexpr int R2_BLOCK = LBM_R2_BLOCK;
static_assert(R2_BLOCK % 32 == 0 && R2_BLOCK <= STRIP, "whole warps, at most STRIP lanes");
constexpr int R2_W = R2_BLOCK - 4;     // widest strip: the lanes cover it and two halo columns per side
// stage row pitch and tensor box width: columns x0-4 .. x0+R2_BLOCK-1, i.e. a
// strip of up to R2_W columns with 4 margin columns on each side (the bulk
// path's right wrap copy ends at xw + 7 <= R2_BLOCK + 3)
constexpr int R2_SP = R2_BLOCK + 4;
// one stencil row of nine planes, padded to a 128-byte multiple so that every
// row of every slot starts on a 128-byte boundary (tensor copy destinations)
constexpr int R2_ROW = (9 * R2_SP + 31) / 32 * 32;
constexpr int R2_SLOT = 2 * R2_ROW;    // one pair of rows

constexpr size_t rows2_smem_bytes()
{
    return (size_t)R2_SLOTS * R2_SLOT * sizeof(float) + R2_SLOTS * sizeof(uint64_t);
}

// 2-D tiled tensor load (TMA) of box (x, y) of the tensor map into shared
// memory, completing on the mbarrier's transaction count. The population
// maps are 2-D views of a buffer: x = column (pitch wide), y = 9 * row + plane;
// the box is R2_SP columns by 9 planes, so one load brings a stencil row.
// Columns outside the array (x < 0 or beyond the pitch) read as zero.
// Programmatic dependent launch: let the next grid in the stream be scheduled,
// and wait until the grids this one depends on have completed and their
// memory is visible (both no-ops for a grid launched without the attribute).
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
constexpr uint32_t R2_TMA_ROW_BYTES = 9u * R2_SP * sizeof(float);  // one box
// L2 prefetch of the same box (no shared memory, nothing to wait for)
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y) : "memory");
}

// Position in the pair-slot ring (slot and mbarrier phase parity).
struct RingPos2 {
    uint32_t s = 0, ph = 0;
    __device__ __forceinline__ void advance()
    {
        if (++s == R2_SLOTS) { s = 0; ph ^= 1u; }
    }
};

// West, centre and east float2 packs (rows ra, rb) of ring column c.
template <int SW>
__device__ __forceinline__ Row3<float2> row3p(const float (*S)[SW], int ra, int rb, int c)
{
    Row3<float2> r;
    r.w = make_float2(S[ra][c - 1], S[rb][c - 1]);
    r.c = make_float2(S[ra][c], S[rb][c]);
    r.e = make_float2(S[ra][c + 1], S[rb][c + 1]);
    return r;
}

// Static shared memory of a row-pair CTA: the 8-row rings of density, phi
// and Laplacian (one column per lane) and the reduction scratch.
struct SmemR2 {
    __align__(16) float rho[RING][R2_BLOCK + 4];
    __align__(16) float phi[RING][R2_BLOCK + 4];
    __align__(16) float lap[RING][R2_BLOCK + 4];
    double red[R2_BLOCK / 32][2];
    float ext[R2_BLOCK / 32][4];
    int bad;
};

// Both rows of a slot at stage column sc, plane i.
__device__ __forceinline__ float2 stage_pair(const float *slot, int i, int sc)
{
    return make_float2(slot[i * R2_SP + sc], slot[R2_ROW + i * R2_SP + sc]);
}


// One segment (strip s, fluid rows ya .. yb-1) of the row-pair step; see the
// file comment for the schedule. The ring rows of rho / phi / lap are indexed
// by y & (RING - 1) as in the one-row kernel.
// lost: a stage wait of this thread gave up (the step is then invalid and
// reported so; the loop runs on with whatever the stage holds). HOOK: the
// failure-detection test build (a separate instantiation, so the production
// kernel's code is untouched); skip_here: its hook applies to this segment:
// the copy of the final pair is never issued, so the wait for it gives up
// after KArgs::poll_limit polls; no later copy reuses that slot, so nothing is
// left in flight when the CTA exits.
// EARLY: stencil-row pairs issued together when a segment starts (1 .. the
// three slots, all free then); later pairs are issued one per iteration.
template <bool WALLS, bool PRES, bool PADDED, bool HOOK = false, typename IX = int, int EARLY = 1>
__device__ __forceinline__ void run_segment_r2(const KArgs<float> &A, const Geom<float> &G, int s, int ya, int yb,
                                               SmemR2 &S, float *stages, uint64_t *bars,
                                               RingPos2 &ring_next, const CUtensorMap *tmap, Acc<float, 1> &acc,
                                               bool &lost, bool skip_here)
{
    using V = float2;
    constexpr int SW = R2_BLOCK + 4;
    constexpr int PRODUCER = R2_BLOCK - 1;  // no halo duty
    constexpr int RM = RING - 1;
    const int tid = threadIdx.x;
    const float third = 1.0f / 3.0f;
    const int nx = G.nx, ny = G.ny;
    const int P = PADDED ? G.pitch : G.nx;  // plane pitch; columns nx .. P-1 are padding
    const int rstride = 9 * P;
    const int o1 = P + 1, o2 = rstride + 2 * P, o3 = 3 * P - 1, o4 = 4 * P - rstride;
    const int o5 = rstride + 5 * P + 1, o6 = rstride + 6 * P - 1, o7 = 7 * P - rstride - 1;
    const int o8 = 8 * P - rstride + 1;
    float b_rho1 = 0.f, b_v1 = 0.f, t_v2 = 0.f;  // wall-pair carries (rows 1 -> 2, ny-3 -> ny-2)

    const int x0 = s * G.W;
    const int xw = min(G.W, nx - x0);
    // Thread t holds local column l = t - 2: the strip (at most R2_W = R2_BLOCK - 4
    // columns) plus two halo columns on each side, so every column's density
    // is computed by its own lane and no halo duty exists.
    const int l = tid - 2;
    const int g = x0 + l;                    // global column (halo columns may lie outside 0 .. nx-1)
    const bool dens = l < xw + 2;            // density and phi of column l (l >= -2 always)
    const bool lapc = l >= -1 && l <= xw;    // Laplacian of column l
    const bool active = l >= 0 && l < xw;    // collided column
    // density source: the column itself (stage column l + 4), or at and beyond
    // the pressure columns the inlet / outlet density derived from column
    // 1 / nx-2 (dmode 2 / 3)
    int dmode = 0, dsc = l + 4;
    if (PRES) {
        if (g <= 0) { dmode = 2; dsc = 1 - x0 + 4; }
        else if (g >= nx - 1) { dmode = 3; dsc = nx - 2 - x0 + 4; }
    }
    const int xa = g;
    const bool pin = PRES && active && xa == 0;
    const bool pout = PRES && active && xa == nx - 1;
    const bool anyp = pin || pout;
    // a pressure column collides its interior neighbour's column
    const int lcol = (pin ? 1 : (pout ? nx - 2 : xa)) - x0;
    const int scol = lcol + 4;  // stage column
    const int ccol = lcol + 2;  // ring column
    const bool x_inner = !anyp && (PRES || (xa >= 1 && xa <= nx - 2));

    // stage copies: columns gx0 .. gx1-1 of each plane row, plus (periodic x)
    // the four columns wrapped around from the other end of the row
    const int gx0 = max(x0 - 4, 0);
    const int gx1 = min(x0 + xw + 4, G.pitch);
    const uint32_t mbytes = (uint32_t)((gx1 - gx0) * sizeof(float));
    const bool wrapL = !PRES && x0 == 0, wrapR = !PRES && x0 + xw == nx;
    const uint32_t row_bytes = 9u * (mbytes + (wrapL ? 16u : 0u) + (wrapR ? 16u : 0u));
    const int dcol = gx0 - x0 + 4;
    const int npairs = (yb - ya + 5) / 2;  // stencil rows ya-2 .. yb+1 in pairs
    RingPos2 ring_issue = ring_next;
    // tensor loads: the box starts 4 columns left of the strip; strips that
    // need wrapped halo columns (periodic x, first or last strip) keep the
    // bulk copies, whose wrap copies would race with a box's zero fill
    const bool use_tma = tmap != nullptr && !wrapL && !wrapR;
    // L2 prefetch (tensor-load path) of stencil-row pair q: the boxes the
    // stage loads of pair q will read
    auto prefetch = [&](int q) {
        if (q < npairs) {
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                bool mir;
                tma_prefetch_2d(tmap, x0 - 4, 9 * map_row<WALLS>(ya - 2 + 2 * q + t, ny, mir));
            }
        }
    };
    const int poll = HOOK ? A.poll_limit : (1 << 22);
    auto issue = [&](int q) {
        if (A.pf > 0 && use_tma && tid == PRODUCER) {
            // keep the pairs up to A.pf ahead of the staged one in flight to L2
            if (q == 0)
                for (int d = 1; d < A.pf; ++d) prefetch(d);
            prefetch(q + A.pf);
        }
        if (q < npairs) {
            if (HOOK && skip_here && q == npairs - 1) {
                // the test hook: the final pair's copy is never issued
            } else if (tid == PRODUCER && use_tma) {
                const uint32_t st = ring_issue.s;
                mbar_arrive_expect_tx(&bars[st], 2u * R2_TMA_ROW_BYTES);
                float *slot = stages + (size_t)st * R2_SLOT;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    bool mir;
                    const int row = map_row<WALLS>(ya - 2 + 2 * q + t, ny, mir);
                    tma_load_2d(slot + t * R2_ROW, tmap, x0 - 4, 9 * row, &bars[st]);
                }
            } else if (tid == PRODUCER) {
                const uint32_t st = ring_issue.s;
                mbar_arrive_expect_tx(&bars[st], 2u * row_bytes);
                float *slot = stages + (size_t)st * R2_SLOT;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    bool mir;
                    const float *src = G.fin + (IX)map_row<WALLS>(ya - 2 + 2 * q + t, ny, mir) * rstride;
                    float *dst = slot + t * R2_ROW;
#pragma unroll
                    for (int i = 0; i < 9; ++i) bulk_copy_g2s(dst + i * R2_SP + dcol, src + i * P + gx0, mbytes, &bars[st]);
                    if (wrapL) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) bulk_copy_g2s(dst + i * R2_SP, src + i * P + nx - 4, 16u, &bars[st]);
                    }
                    if (wrapR) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) bulk_copy_g2s(dst + i * R2_SP + xw + 4, src + i * P, 16u, &bars[st]);
                    }
                }
            }
            ring_issue.advance();
        }
    };

    // with EARLY > 1 the first pairs go out together, so only the first wait
    // of a segment sees the full latency of a stage load (short segments)
    static_assert(EARLY >= 1 && EARLY <= R2_SLOTS, "early pairs fit the free slots");
    if (tid == PRODUCER) fence_proxy_async_smem();  // slots last read by the previous segment
#pragma unroll
    for (int q = 0; q < EARLY; ++q) issue(q);
    for (int k = 0; k < npairs; ++k) {
        const int yy0 = ya - 2 + 2 * k;
        const uint32_t cur = ring_next.s;
        const uint32_t prev = cur == 0 ? R2_SLOTS - 1 : cur - 1;  // slot of pair k-1

        // (1) density and phi of stencil rows yy0, yy0+1
        if (!mbar_wait_bounded(&bars[cur], ring_next.ph, poll)) lost = true;
        {
            const float *slot = stages + (size_t)cur * R2_SLOT;
            bool m0, m1;
            map_row<WALLS>(yy0, ny, m0);
            map_row<WALLS>(yy0 + 1, ny, m1);
            const V add = make_float2(m0 ? A.wet : 0.f, m1 ? A.wet : 0.f);  // mirrored wall ghosts
            const int r0 = yy0 & RM, r1 = (yy0 + 1) & RM;
            if (dens) {
                V pf[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) pf[i] = stage_pair(slot, i, dsc);
                V sum = add_(add_(add_(pf[0], pf[1]), add_(pf[2], pf[3])), add_(add_(pf[4], pf[5]), add_(pf[6], pf[7])));
                sum = add_(sum, pf[8]);
                if (dmode) {
                    sum.x = column_density(A, G, dmode == 3, sum.x);
                    sum.y = column_density(A, G, dmode == 3, sum.y);
                }
                const V rho_c = add_(sum, add);
                const V ph = eos_phi<V>(A, rho_c);
                S.rho[r0][tid] = rho_c.x; S.rho[r1][tid] = rho_c.y;
                S.phi[r0][tid] = ph.x; S.phi[r1][tid] = ph.y;
            }
        }
        __syncthreads();  // A: density rows complete; the slot of pair k-2 is free

        // (2) refill the slot of pair k-2 with pair k+1; Laplacian of rows yy0-1, yy0
        if (k + 1 >= EARLY) {
            if (tid == PRODUCER) fence_proxy_async_smem();
            issue(k + 1);
        }
        if (k >= 1) {
            const int qm = (yy0 - 2) & RM, q0 = (yy0 - 1) & RM, q1 = yy0 & RM, q2 = (yy0 + 1) & RM;
            if (lapc) {
                const V L = lap9<V>(row3p<SW>(S.rho, qm, q0, tid), row3p<SW>(S.rho, q0, q1, tid),
                                    row3p<SW>(S.rho, q1, q2, tid));
                S.lap[q0][tid] = L.x; S.lap[q1][tid] = L.y;
            }
        }
        __syncthreads();  // B: Laplacian rows complete

        // (3) collide and stream rows b = yy0-2 and (if below yb) b+1
        if (k >= 2 && active) {
            const int b = yy0 - 2;
            const bool second = b + 1 < yb;
            const float *slot = stages + (size_t)prev * R2_SLOT;
            V f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = stage_pair(slot, i, scol);
            const int qm = (b - 1) & RM, q0 = b & RM, q1 = (b + 1) & RM, q2 = (b + 2) & RM;
            V ngpx, ngpy, glx, gly;
            ngrad12<V>(row3p<SW>(S.phi, qm, q0, ccol), row3p<SW>(S.phi, q0, q1, ccol), row3p<SW>(S.phi, q1, q2, ccol),
                       ngpx, ngpy);
            grad12<V>(row3p<SW>(S.lap, qm, q0, ccol), row3p<SW>(S.lap, q0, q1, ccol), row3p<SW>(S.lap, q1, q2, ccol),
                      glx, gly);
            const V rho = make_float2(S.rho[q0][ccol], S.rho[q1][ccol]);
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
            const V rho_own = anyp ? make_float2(S.rho[q0][tid], S.rho[q1][tid]) : rho;

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
                // pressure column: extrapolate from the interior neighbour, row by row
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
            float *const out = G.fout;
            const IX oi = (IX)b * rstride + xa;  // slot of (xa, b) in plane 0
            const bool y_inner = WALLS ? (b >= 2 && b + 1 <= ny - 3) : (b >= 1 && b + 1 <= ny - 2);
            if (x_inner && y_inner && second) {
                const IX oj = oi + rstride;
                out[oi] = fs[0].x;      out[oj] = fs[0].y;
                out[oi + o1] = fs[1].x; out[oj + o1] = fs[1].y;
                out[oi + o2] = fs[2].x; out[oj + o2] = fs[2].y;
                out[oi + o3] = fs[3].x; out[oj + o3] = fs[3].y;
                out[oi + o4] = fs[4].x; out[oj + o4] = fs[4].y;
                out[oi + o5] = fs[5].x; out[oj + o5] = fs[5].y;
                out[oi + o6] = fs[6].x; out[oj + o6] = fs[6].y;
                out[oi + o7] = fs[7].x; out[oj + o7] = fs[7].y;
                out[oi + o8] = fs[8].x; out[oj + o8] = fs[8].y;
            } else {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (e == 1 && !second) break;
                    const int r = b + e;
                    const IX ok = oi + (IX)e * rstride;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const int ty = r + ey_(i);
                        if (WALLS && (ty == 0 || ty == ny - 1)) {
                            // half-way bounce-back into the opposite slot of this node
                            out[ok + opp_(i) * P] = el(fs[i], e);
                        } else {
                            int tx = xa + ex_(i);
                            if (PRES) {
                                if (tx < 0 || tx >= nx) continue;  // leaves through the column
                            } else {
                                tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
                            }
                            int tyw = ty;
                            if (!WALLS) tyw = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
                            out[(IX)tyw * rstride + i * P + tx] = el(fs[i], e);
                        }
                    }
                }
            }
            // diagnostics of the state read, row by row in the one-row kernel's
            // order (its flush follows collided row r when (r - ya + 5) % 16 == 15)
            acc.macc = add_(acc.macc, rho_own.x);
            acc.rmin = vmin_(acc.rmin, rho.x);
            acc.rmax = vmax_(acc.rmax, rho.x);
            if (((b - ya + 5) & 15) == 15) acc.flush();
            if (second) {
                acc.macc = add_(acc.macc, rho_own.y);
                acc.rmin = vmin_(acc.rmin, rho.y);
                acc.rmax = vmax_(acc.rmax, rho.y);
                if (((b + 1 - ya + 5) & 15) == 15) acc.flush();
            }

            if (WALLS && !anyp && (b <= 2 || b + 1 >= ny - 3)) {
                // wall shear: quadratic through v = 0 on the half-way plane and
                // v at distances 1/2 and 3/2; wall pressure: Eq. 2.4 in mesh units
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (e == 1 && !second) break;
                    const int r = b + e;
                    const float rk = el(rho, e), vk = el(vx, e);
                    const int pm = (r - 1) & RM, pz = r & RM, pp = (r + 1) & RM;
                    if (r == 1) {
                        b_rho1 = rk;
                        b_v1 = vk;
                        const float pw = wall_pressure<float, SW>(A, S.rho, S.phi, S.lap[pz][ccol], pm, pz, pp, ccol, rk);
                        acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw);
                    }
                    if (r == ny - 3) t_v2 = vk;
                    if (r == 2) {
                        const float tw = mul_(mul_(b_rho1, A.nu), mul_(fma_(9.0f, b_v1, -vk), third));
                        acc.J += (double)tw; acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw);
                    }
                    if (r == ny - 2) {
                        const float tw = mul_(mul_(rk, A.nu), mul_(fma_(9.0f, vk, -t_v2), third));
                        const float pw = wall_pressure<float, SW>(A, S.rho, S.phi, S.lap[pz][ccol], pm, pz, pp, ccol, rk);
                        acc.J += (double)tw;
                        acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw);
                        acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw);
                    }
                }
            }
        }
        ring_next.advance();
    }
    __syncthreads();  // ring and stage reuse by the next segment
}

// The row-pair step kernel (FP32, staged, MODE_STEP); launched like
// step_kernel with rows2_smem_bytes() of dynamic shared memory.
#ifndef LBM_R2_MIN_BLOCKS
#define LBM_R2_MIN_BLOCKS (640 / LBM_R2_BLOCK)
#endif
// tmap: 2-D tensor map of A.fin (used when A.tma is set). HOOK: the
// failure-detection test build (see run_segment_r2). IX: the type of
// population offsets, int while 9 pitch ny < 2^31, long long above. EARLY:
// as run_segment_r2 (3 pays where CTAs hold short segments).
template <bool WALLS, bool PRES, bool PADDED, bool HOOK = false, typename IX = int, int EARLY = 1>
__global__ void __launch_bounds__(R2_BLOCK, LBM_R2_MIN_BLOCKS)
    step_kernel_rows2(const KArgs<float> A, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    float *const stages = reinterpret_cast<float *>(dsm);
    uint64_t *const bars = reinterpret_cast<uint64_t *>(dsm + (size_t)R2_SLOTS * R2_SLOT * sizeof(float));
    __shared__ SmemR2 S;

    const int tid = threadIdx.x;
    const int cta = A.reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    long long u = cut_units<WALLS>(A, cta);
    const long long u1 = cut_units<WALLS>(A, cta + 1);
    const Geom<float> G{A.fin, A.fout, A.nx, A.ny, A.W, A.pitch, A.rho_in_g, A.rho_in_l, A.rho_out_g, A.rho_out_l};

    Acc<float, 1> acc;
    acc.reset();
    RingPos2 ring_next;
    bool lost = false;  // a bounded wait gave up
    if (tid == 0) {
        for (int st = 0; st < R2_SLOTS; ++st) mbar_init(&bars[st], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // launched with programmatic serialization, the next step's CTAs may
    // start their set-up while this grid runs; every access to the state and
    // to the per-CTA slots follows the wait for the previous grid
    griddep_launch_dependents();
    griddep_wait();

    while (u < u1) {
        int s, ya;
        long long run_end;
        unit_run(A, u, s, ya, run_end);
        const long long ue = min(u1, run_end);
        const int yb = ya + (int)(ue - u);
        u = ue;
        // the test hook applies to the first CTA's last segment
        run_segment_r2<WALLS, PRES, PADDED, HOOK, IX, EARLY>(A, G, s, ya, yb, S, stages, bars, ring_next,
                                                  A.tma ? &tmap : nullptr, acc, lost, HOOK && cta == 0 && u == u1);
    }
    if (lost) atomicOr(A.err, 2);

    double m, j;
    float e[4];
    bool anybad;
    cta_reduce<float, R2_BLOCK, 1>(acc, S, m, j, e, anybad);
    if (tid == 0) {
        A.mass_part[cta] = m;
        A.J_acc[cta] += j;
        float *ex = A.ext + 4 * cta;
        ex[0] = fmin(ex[0], e[0]); ex[1] = fmax(ex[1], e[1]);
        ex[2] = fmin(ex[2], e[2]); ex[3] = fmax(ex[3], e[3]);
        if (anybad) atomicOr(A.err, 1);
    }
}

// Batched channels with the row-pair step: as batch_step_kernel, every
// segment of the work list through run_segment_r2 (padded-pitch body, since
// the channels of a batch mix pitches), one reduction slot per segment.
// tmaps: NULL (plane copies) or the tensor maps of the source buffer, one per
// channel, in device memory (written by the host before the launch).
template <bool WALLS, bool PRES>
__global__ void __launch_bounds__(R2_BLOCK, LBM_R2_MIN_BLOCKS)
    batch_step_kernel_rows2(const KArgs<float> A, const BatchChan<float> *__restrict__ chans,
                            const BatchSeg *__restrict__ segs, const int *__restrict__ cta_begin,
                            double *__restrict__ seg_mass, double *__restrict__ seg_J, float *__restrict__ seg_ext,
                            const CUtensorMap *__restrict__ tmaps)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    float *const stages = reinterpret_cast<float *>(dsm);
    uint64_t *const bars = reinterpret_cast<uint64_t *>(dsm + (size_t)R2_SLOTS * R2_SLOT * sizeof(float));
    __shared__ SmemR2 S;

    const int tid = threadIdx.x;
    const int cta = A.reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    RingPos2 ring_next;
    bool lost = false;
    if (tid == 0) {
        for (int st = 0; st < R2_SLOTS; ++st) mbar_init(&bars[st], 1);
        mbar_init_fence();
    }
    __syncthreads();
    for (int k = cta_begin[cta]; k < cta_begin[cta + 1]; ++k) {
        const BatchSeg sg = segs[k];
        const BatchChan<float> ch = chans[sg.chan];
        const Geom<float> G{A.fin + ch.off, A.fout + ch.off, ch.nx, ch.ny, ch.W, ch.pitch,
                            ch.rho_in_g, ch.rho_in_l, ch.rho_out_g, ch.rho_out_l};
        Acc<float, 1> acc;
        acc.reset();
        run_segment_r2<WALLS, PRES, true>(A, G, sg.strip, sg.ya, sg.yb, S, stages, bars, ring_next,
                                          tmaps ? tmaps + sg.chan : nullptr, acc, lost, false);
        double m, j;
        float e[4];
        bool anybad;
        cta_reduce<float, R2_BLOCK, 1>(acc, S, m, j, e, anybad);
        if (tid == 0) {
            seg_mass[k] = m;
            seg_J[k] += j;
            float *ex = seg_ext + 4 * (long long)k;
            ex[0] = fmin(ex[0], e[0]); ex[1] = fmax(ex[1], e[1]);
            ex[2] = fmin(ex[2], e[2]); ex[3] = fmax(ex[3], e[3]);
            if (anybad) atomicOr(A.err, 1);
        }
    }
    if (lost) atomicOr(A.err, 2);
}

}  // namespace lbm

namespace lbm {

// ---------------------------------------------------------------------------
// Persistent batch: one cooperative launch runs `nsteps` steps of every
// channel. Each segment (channel, strip, rows) keeps a step counter in global
// memory; before its step n a segment waits until every segment it depends on
// has completed n steps: the segments of its own and the two neighbouring
// strips of its channel whose rows meet [ya - 3, yb + 2] (the rows its stencil
// reads from the source buffer, and the rows whose earlier readers its pushes
// into the target buffer must not overtake; built on the host). The waits are
// bounded; one that gives up sets error bit 1 and a global abort flag, which
// ends every CTA's waiting, so nothing hangs. All CTAs are co-resident (a
// cooperative launch), so a CTA only ever waits for work that can run.
// Memory ordering: a segment's threads write the target buffer, the CTA
// barrier orders those writes before thread 0's release of the counter, and
// the waiter's acquire (thread 0) and CTA barrier order them before the
// producer thread's bulk copies, behind a generic-to-async proxy fence.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

constexpr int PERSIST_POLLS = 1 << 22;  // polls (each after a short sleep) before a dependency wait gives up

template <bool WALLS, bool PRES>
__global__ void __launch_bounds__(R2_BLOCK, LBM_R2_MIN_BLOCKS)
    batch_persistent_kernel_rows2(const KArgs<float> A, const BatchChan<float> *__restrict__ chans,
                                  const BatchSeg *__restrict__ segs, const int *__restrict__ cta_begin,
                                  double *__restrict__ seg_mass, double *__restrict__ seg_J,
                                  float *__restrict__ seg_ext, const CUtensorMap *__restrict__ tmaps, int nchan,
                                  const int *__restrict__ dep_beg, const int *__restrict__ dep, int *done,
                                  int *abort_flag, float *buf0, float *buf1, int cur0, int nsteps)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    float *const stages = reinterpret_cast<float *>(dsm);
    uint64_t *const bars = reinterpret_cast<uint64_t *>(dsm + (size_t)R2_SLOTS * R2_SLOT * sizeof(float));
    __shared__ SmemR2 S;
    __shared__ int s_stop;

    const int tid = threadIdx.x;
    constexpr int PRODUCER = R2_BLOCK - 1;
    const int cta = A.reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    RingPos2 ring_next;
    bool lost = false;
    if (tid == 0) {
        for (int st = 0; st < R2_SLOTS; ++st) mbar_init(&bars[st], 1);
        mbar_init_fence();
    }
    __syncthreads();
    for (int n = 0; n < nsteps; ++n) {
        const int src = (cur0 + n) & 1;
        float *const fin = src ? buf1 : buf0;
        float *const fout = src ? buf0 : buf1;
        for (int k = cta_begin[cta]; k < cta_begin[cta + 1]; ++k) {
            if (tid == 0) {
                // the counters are read in groups of up to 8 independent
                // relaxed loads (their latencies overlap), re-read until all
                // have reached n, then one acquire fence orders the step's reads
                int stop = 0;
                for (int j0 = dep_beg[k]; j0 < dep_beg[k + 1] && !stop; j0 += 8) {
                    const int m = min(8, dep_beg[k + 1] - j0);
                    for (int it = 0;; ++it) {
                        int v[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) v[q] = q < m ? ld_relaxed_gpu(done + dep[j0 + q]) : n;
                        bool ready = true;
#pragma unroll
                        for (int q = 0; q < 8; ++q) ready = ready && v[q] >= n;
                        if (ready) break;
                        if (it >= PERSIST_POLLS || ld_relaxed_gpu(abort_flag)) {
                            stop = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                fence_acq_rel_gpu();
                if (stop) {
                    atomicOr(A.err, 2);
                    atomicExch(abort_flag, 1);
                }
                s_stop = stop;
            }
            __syncthreads();
            if (s_stop) n = nsteps;  // uniform: leave both loops
            if (n == nsteps) break;
            if (tid == PRODUCER) fence_proxy_async_global();
            const BatchSeg sg = segs[k];
            const BatchChan<float> ch = chans[sg.chan];
            const Geom<float> G{fin + ch.off, fout + ch.off, ch.nx, ch.ny, ch.W, ch.pitch,
                                ch.rho_in_g, ch.rho_in_l, ch.rho_out_g, ch.rho_out_l};
            Acc<float, 1> acc;
            acc.reset();
            run_segment_r2<WALLS, PRES, true>(A, G, sg.strip, sg.ya, sg.yb, S, stages, bars, ring_next,
                                              tmaps ? tmaps + (size_t)src * nchan + sg.chan : nullptr, acc, lost,
                                              false);
            double m, j;
            float e[4];
            bool anybad;
            cta_reduce<float, R2_BLOCK, 1>(acc, S, m, j, e, anybad);  // ends with a CTA barrier
            if (tid == 0) {
                seg_mass[k] = m;
                seg_J[k] += j;
                float *ex = seg_ext + 4 * (long long)k;
                ex[0] = fmin(ex[0], e[0]); ex[1] = fmax(ex[1], e[1]);
                ex[2] = fmin(ex[2], e[2]); ex[3] = fmax(ex[3], e[3]);
                if (anybad) atomicOr(A.err, 1);
                fence_proxy_async_global();  // this CTA's bulk reads of the source are complete
                __threadfence();
                st_release_gpu(done + k, n + 1);
            }
        }
    }
    if (lost) atomicOr(A.err, 2);
}

}  // namespace lbm
