// The FP32 step for small grids: one CTA per 32 x 8 tile, no row pipeline.
//
// The row-pair kernel streams a strip's rows through a three-slot stage, so a
// CTA that holds only a few rows (a grid of a few hundred thousand nodes
// spread over 760 CTAs) spends most of its time filling that pipeline. Here a
// CTA stages all the stencil rows its tile needs at once (one 2-D tensor load
// of 40 columns by 9 planes per stencil row), then computes the tile in three
// phases separated by barriers: density and EOS potential on the tile plus
// two halo nodes, the Laplacian on the tile plus one, and the collision,
// boundaries and push of the tile's 32 x 8 nodes (each thread one column and
// one row pair, with the paired FP32 instructions). The node arithmetic is
// the row-pair kernel's own helper sequence in the same order, so the two
// kernels give identical populations (tested).
//
// An option (LBM_OPT_TILE, off by default) where the grid's plan gives CTAs
// short segments, for FP32 channels whose row-pair step stages with tensor
// loads (no wall mask, 32-bit offsets), with at most MAX_CTAS tiles, and
// (walls) no tile boundary between the wall-shear rows ny-3 | ny-2. Measured
// slower than the row-pair kernel on those grids: each CTA waits for its
// whole stage before it computes, and its fixed costs (the wait, four
// barriers, the FP64 reduction of its partials) are paid for 256 nodes.
#pragma once

namespace lbm {

constexpr int T_TX = 32;                   // tile columns: one warp
constexpr int T_TY = 8;                    // tile rows: four row pairs
constexpr int T_THREADS = T_TX * T_TY / 2;  // 128: lane = column, warp = row pair
constexpr int T_SW = T_TX + 4;             // ring columns x0-2 .. x0+T_TX+1
constexpr int T_ROWS = T_TY + 4;           // stencil rows y0-2 .. y0+T_TY+1
constexpr int T_BOX = T_TX + 8;            // staged columns x0-4 .. x0+T_TX+3 (16-byte aligned start)
constexpr int T_ROWF = (9 * T_BOX + 31) / 32 * 32;  // floats per staged stencil row (128-byte aligned rows)
constexpr uint32_t T_BOX_BYTES = 9u * T_BOX * sizeof(float);  // one tensor load

constexpr size_t tile_smem_bytes() { return (size_t)T_ROWS * T_ROWF * sizeof(float) + sizeof(uint64_t); }

struct SmemTile {
    __align__(16) float rho[T_ROWS][T_SW];
    __align__(16) float phi[T_ROWS][T_SW];
    __align__(16) float lap[T_ROWS][T_SW];
    float tv2[T_TX];  // v at row ny-3, for the top wall shear of row ny-2
    double red[T_THREADS / 32][2];
    float ext[T_THREADS / 32][4];
    int bad;
};

// tmap: 2-D tensor map of A.fin with boxes of T_BOX columns by 9 planes.
// ntx: tiles along x (the grid is ntx x nty tiles, tile index = CTA).
template <bool WALLS, bool PRES>
__global__ void __launch_bounds__(T_THREADS, 5)
    step_kernel_tile(const KArgs<float> A, const __grid_constant__ CUtensorMap tmap, int ntx)
{
    using V = float2;
    extern __shared__ __align__(128) unsigned char dsm[];
    float *const stage = reinterpret_cast<float *>(dsm);
    uint64_t *const bar = reinterpret_cast<uint64_t *>(dsm + (size_t)T_ROWS * T_ROWF * sizeof(float));
    __shared__ SmemTile S;

    const int tid = threadIdx.x, lane = tid & 31, pr = tid >> 5;
    const int cta = A.reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    const int nx = A.nx, ny = A.ny;
    const int P = A.pitch;
    const int rstride = 9 * P;
    const int o1 = P + 1, o2 = rstride + 2 * P, o3 = 3 * P - 1, o4 = 4 * P - rstride;
    const int o5 = rstride + 5 * P + 1, o6 = rstride + 6 * P - 1, o7 = 7 * P - rstride - 1;
    const int o8 = 8 * P - rstride + 1;
    const float third = 1.0f / 3.0f;
    const Geom<float> G{A.fin, A.fout, nx, ny, A.W, P, A.rho_in_g, A.rho_in_l, A.rho_out_g, A.rho_out_l};
    const int yf0 = WALLS ? 1 : 0, yf1 = WALLS ? ny - 1 : ny;  // fluid rows yf0 .. yf1-1
    const int x0 = (cta % ntx) * T_TX, y0 = yf0 + (cta / ntx) * T_TY;
    const int xw = min(T_TX, nx - x0), yh = min(T_TY, yf1 - y0);
    const int nrows = yh + 4;  // stencil rows y0-2 .. y0+yh+1

    Acc<float, 1> acc;
    acc.reset();
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    // launched with programmatic serialization, the next step's CTAs may start
    // their set-up now; every access to the state and the slots follows the wait
    griddep_launch_dependents();
    griddep_wait();

    // (1) stage every stencil row of the tile (mirrored or wrapped rows as the
    //     row-pair kernel maps them); columns outside the array read as zero
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)nrows * T_BOX_BYTES);
        for (int j = 0; j < nrows; ++j) {
            bool mir;
            const int row = map_row<WALLS>(y0 - 2 + j, ny, mir);
            tma_load_2d(stage + j * T_ROWF, &tmap, x0 - 4, 9 * row, bar);
        }
    }
    const bool lost = !mbar_wait_bounded(bar, 0);
    if (!PRES && (x0 < 4 || x0 + T_TX + 4 > nx)) {
        // periodic x: the staged columns beyond either end come from the other end
        for (int k = tid; k < nrows * 9 * T_BOX; k += T_THREADS) {
            const int c = k % T_BOX, ji = k / T_BOX, j = ji / 9, i = ji - 9 * j;
            const int gx = x0 - 4 + c;
            if ((gx >= 0 && gx < nx) || gx < -4 || gx > nx + 3) continue;
            bool mir;
            const int row = map_row<WALLS>(y0 - 2 + j, ny, mir);
            stage[j * T_ROWF + i * T_BOX + c] = G.fin[row * rstride + i * P + (gx < 0 ? gx + nx : gx - nx)];
        }
    }
    __syncthreads();

    // (2) density and phi at ring rows j (stencil row y0-2+j), columns c (x0-2+c)
    for (int k = tid; k < nrows * T_SW; k += T_THREADS) {
        const int j = k / T_SW, c = k - j * T_SW;
        const int g = x0 - 2 + c;
        bool mir;
        map_row<WALLS>(y0 - 2 + j, ny, mir);
        int dmode = 0, sc = c + 2;  // stage column of global column g
        if (PRES) {
            if (g <= 0) { dmode = 2; sc = 1 - x0 + 4; }
            else if (g >= nx - 1) { dmode = 3; sc = nx - 2 - x0 + 4; }
        }
        const float *sp = stage + j * T_ROWF + sc;
        float pf[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) pf[i] = sp[i * T_BOX];
        float sum = add_(add_(add_(pf[0], pf[1]), add_(pf[2], pf[3])), add_(add_(pf[4], pf[5]), add_(pf[6], pf[7])));
        sum = add_(sum, pf[8]);
        if (dmode) sum = column_density(A, G, dmode == 3, sum);
        const float rho_c = add_(sum, mir ? A.wet : 0.f);
        S.rho[j][c] = rho_c;
        S.phi[j][c] = eos_phi<float>(A, rho_c);
    }
    __syncthreads();

    // (3) Laplacian at ring rows 1 .. nrows-2, columns 1 .. T_SW-2
    for (int k = tid; k < (nrows - 2) * (T_SW - 2); k += T_THREADS) {
        const int j = 1 + k / (T_SW - 2), c = 1 + k % (T_SW - 2);
        S.lap[j][c] = lap9<float>(row3<float, 1, T_SW>(S.rho, j - 1, c), row3<float, 1, T_SW>(S.rho, j, c),
                                  row3<float, 1, T_SW>(S.rho, j + 1, c));
    }
    __syncthreads();

    // (4) collide and push rows b, b+1 of column x0 + lane
    const int b = y0 + 2 * pr;
    const bool active = lane < xw && 2 * pr < yh;
    const bool second = 2 * pr + 1 < yh;
    const int xa = x0 + lane;
    const bool pin = PRES && active && xa == 0;
    const bool pout = PRES && active && xa == nx - 1;
    const bool anyp = pin || pout;
    const int lcol = (pin ? 1 : (pout ? nx - 2 : xa)) - x0;  // a pressure column collides its neighbour
    const int scol = lcol + 4, ccol = lcol + 2;
    const bool x_inner = !anyp && (PRES || (xa >= 1 && xa <= nx - 2));
    const int q0 = 2 * pr + 2, qm = q0 - 1, q1 = q0 + 1, q2 = q0 + 2;  // ring rows of b-1 .. b+2
    V rho = make_float2(0.f, 0.f), vx = rho;
    if (active) {
        const float *s0 = stage + q0 * T_ROWF + scol, *s1 = stage + q1 * T_ROWF + scol;
        V f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = make_float2(s0[i * T_BOX], s1[i * T_BOX]);
        V ngpx, ngpy, glx, gly;
        ngrad12<V>(row3p<T_SW>(S.phi, qm, q0, ccol), row3p<T_SW>(S.phi, q0, q1, ccol),
                   row3p<T_SW>(S.phi, q1, q2, ccol), ngpx, ngpy);
        grad12<V>(row3p<T_SW>(S.lap, qm, q0, ccol), row3p<T_SW>(S.lap, q0, q1, ccol),
                  row3p<T_SW>(S.lap, q1, q2, ccol), glx, gly);
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
        const int oi = b * rstride + xa;
        const bool y_inner = WALLS ? (b >= 2 && b + 1 <= ny - 3) : (b >= 1 && b + 1 <= ny - 2);
        if (x_inner && y_inner && second) {
            const int oj = oi + rstride;
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
                const int r = b + e, ok = oi + e * rstride;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int ty = r + ey_(i);
                    if (WALLS && (ty == 0 || ty == ny - 1)) {
                        out[ok + opp_(i) * P] = el(fs[i], e);  // half-way bounce-back
                    } else {
                        int tx = xa + ex_(i);
                        if (PRES) {
                            if (tx < 0 || tx >= nx) continue;  // leaves through the column
                        } else {
                            tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
                        }
                        int tyw = ty;
                        if (!WALLS) tyw = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
                        out[tyw * rstride + i * P + tx] = el(fs[i], e);
                    }
                }
            }
        }
        acc.macc = add_(acc.macc, rho_own.x);
        acc.rmin = vmin_(acc.rmin, rho.x);
        acc.rmax = vmax_(acc.rmax, rho.x);
        if (second) {
            acc.macc = add_(acc.macc, rho_own.y);
            acc.rmin = vmin_(acc.rmin, rho.y);
            acc.rmax = vmax_(acc.rmax, rho.y);
        }
        if (WALLS && !anyp) {
            // v at row ny-3 for the top wall shear (possibly another warp's row ny-2)
            if (b == ny - 3) S.tv2[lane] = vx.x;
            if (second && b + 1 == ny - 3) S.tv2[lane] = vx.y;
        }
    }
    if (WALLS) __syncthreads();  // tv2 complete
    if (WALLS && active && !anyp && (b <= 2 || b + 1 >= ny - 3)) {
        // wall shear: quadratic through v = 0 on the half-way plane and v at
        // distances 1/2 and 3/2; wall pressure: Eq. 2.4 in mesh units
        float b_rho1 = 0.f, b_v1 = 0.f;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (e == 1 && !second) break;
            const int r = b + e;
            const float rk = el(rho, e), vk = el(vx, e);
            const int pm = q0 + e - 1, pz = q0 + e, pp = q0 + e + 1;
            if (r == 1) {
                b_rho1 = rk;
                b_v1 = vk;
                const float pw = wall_pressure<float, T_SW>(A, S.rho, S.phi, S.lap[pz][ccol], pm, pz, pp, ccol, rk);
                acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw);
            }
            if (r == 2) {
                const float tw = mul_(mul_(b_rho1, A.nu), mul_(fma_(9.0f, b_v1, -vk), third));
                acc.J += (double)tw; acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw);
            }
            if (r == ny - 2) {
                const float tw = mul_(mul_(rk, A.nu), mul_(fma_(9.0f, vk, -S.tv2[lane]), third));
                const float pw = wall_pressure<float, T_SW>(A, S.rho, S.phi, S.lap[pz][ccol], pm, pz, pp, ccol, rk);
                acc.J += (double)tw;
                acc.tmin = fmin(acc.tmin, tw); acc.tmax = fmax(acc.tmax, tw);
                acc.pmin = fmin(acc.pmin, pw); acc.pmax = fmax(acc.pmax, pw);
            }
        }
    }
    if (lost) atomicOr(A.err, 2);

    double m, j;
    float e[4];
    bool anybad;
    cta_reduce<float, T_THREADS, 1>(acc, S, m, j, e, anybad);
    if (tid == 0) {
        A.mass_part[cta] = m;
        A.J_acc[cta] += j;
        float *ex = A.ext + 4 * cta;
        ex[0] = fmin(ex[0], e[0]); ex[1] = fmax(ex[1], e[1]);
        ex[2] = fmin(ex[2], e[2]); ex[3] = fmax(ex[3], e[3]);
        if (anybad) atomicOr(A.err, 1);
    }
}

}  // namespace lbm
