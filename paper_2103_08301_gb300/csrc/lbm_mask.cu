// General wall geometry: the step on a lattice with a per-node solid mask.
//
// The paper's airway is a straight channel (Sec. 2.2), which the fast kernels
// (lbm_rows2.cuh, lbm_kernels.cuh) serve with walls derived from the row
// index. A mask marks any node solid; this path then does the same step of
// the method (moments, EOS potential, Laplacian, the force of Eq. 2.17,
// velocity-shift collision, pressure columns, push streaming) with
//   - half-way bounce-back on every link into a solid node (Eq. 2.1 streaming
//     with the no-slip rule of Sec. 2.2), and
//   - ghost densities for the stencils at solid points: the mirror rule of the
//     flat walls generalised. Along the four axis directions n, the depth d of
//     the first fluid point x + d n (d <= 2); the directions of least depth
//     each give the source x + (2d - 1) n (as deep in front of the wall as x
//     lies behind it), or x + d n where that is not fluid; without an axis
//     direction, the four diagonals likewise; without those, the fluid points
//     at knight offsets. Ghost = mean of the sources + the wetting offset. A
//     flat wall gives the channel rule exactly.
// The ghost sources are resolved on the host into a table of fluid (or
// pressure-column) nodes per ghost point, so one gather per point fills them.
//
// Data (device, allocated by the library): the solid mask (1 B/node), three
// ghost-extended arrays of (nx + 4)(ny + 4) values (density, phi, Laplacian),
// the ghost table, and the wall-row velocities and pressures of the
// diagnostics. Per step: density (reads 36 B/node FP32), columns, ghosts,
// phi and Laplacian, then force + collision + streaming (36 B read, 36 B
// written, plus the extended arrays through L1/L2) and the wall diagnostics:
// about 130 B/node against the channel kernels' 72. The arithmetic of each
// node is the channel kernels' own (the same device functions in the same
// order), so a channel run through this path matches them bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

namespace {

constexpr int MB = 256;  // threads per block of the mask kernels

struct MaskDev {
    int nx, ny, pitch, walls, bc_x, sx;  // sx = nx + 4: row stride of the extended arrays
    const uint8_t *solid;                 // nx * ny
    const uint16_t *links;                // nx * ny: bit i = the push along e_i bounces back; bit 15 = solid
    const int *gdst, *gbeg, *gsrc;        // ghost table (CSR)
    const uint8_t *gwet;
    int nghost;
};

__device__ __forceinline__ int ext(const MaskDev &m, int x, int y) { return (y + 2) * m.sx + (x + 2); }

// Sum of the nine populations of node (x, y) in the channel kernels' order.
template <typename real>
__device__ __forceinline__ real pop_sum(const real *f, int rs, int P)
{
    const real s = add_(add_(add_(f[rs], f[rs + P]), add_(f[rs + 2 * P], f[rs + 3 * P])),
                        add_(add_(f[rs + 4 * P], f[rs + 5 * P]), add_(f[rs + 6 * P], f[rs + 7 * P])));
    return add_(s, f[rs + 8 * P]);
}

template <typename real>
__global__ void __launch_bounds__(MB) mask_density_kernel(const KArgs<real> A, const MaskDev m, real *E)
{
    const int n = m.nx * m.ny;
    for (int k = blockIdx.x * MB + threadIdx.x; k < n; k += gridDim.x * MB) {
        const int y = k / m.nx, x = k - y * m.nx;
        if (m.solid[k]) continue;
        E[ext(m, x, y)] = pop_sum<real>(A.fin, y * 9 * m.pitch + x, m.pitch);
    }
}

// Pressure columns: the EOS root at the column pressure on the branch of the
// interior neighbour's phase (Sec. 2.2 ends, reading R6).
template <typename real>
__global__ void __launch_bounds__(MB) mask_columns_kernel(const KArgs<real> A, const MaskDev m, real *E)
{
    const Geom<real> G{A.fin, A.fout, A.nx, A.ny, A.W, A.pitch, A.rho_in_g, A.rho_in_l, A.rho_out_g, A.rho_out_l};
    for (int y = blockIdx.x * MB + threadIdx.x; y < m.ny; y += gridDim.x * MB) {
        if (m.walls && (y == 0 || y == m.ny - 1)) continue;
        E[ext(m, 0, y)] = add_(column_density(A, G, false, E[ext(m, 1, y)]), real(0));
        E[ext(m, m.nx - 1, y)] = add_(column_density(A, G, true, E[ext(m, m.nx - 2, y)]), real(0));
    }
}

template <typename real>
__global__ void __launch_bounds__(MB) mask_ghost_kernel(const KArgs<real> A, const MaskDev m, real *E)
{
    for (int k = blockIdx.x * MB + threadIdx.x; k < m.nghost; k += gridDim.x * MB) {
        const int b = m.gbeg[k], e = m.gbeg[k + 1];
        real v = real(0);
        if (e > b) {
            real s = E[m.gsrc[b]];
            for (int j = b + 1; j < e; ++j) s = add_(s, E[m.gsrc[j]]);
            if (e - b > 1) s = s / real(e - b);
            v = add_(s, m.gwet[k] ? A.wet : real(0));
        }
        E[m.gdst[k]] = v;
    }
}

template <typename real>
__global__ void __launch_bounds__(MB) mask_phi_lap_kernel(const KArgs<real> A, const MaskDev m, const real *E,
                                                          real *Pa, real *La)
{
    const int w = m.nx + 2, h = m.ny + 2;  // points -1 .. nx and -1 .. ny
    for (int k = blockIdx.x * MB + threadIdx.x; k < w * h; k += gridDim.x * MB) {
        const int y = k / w - 1, x = k % w - 1;
        const int c = ext(m, x, y);
        Pa[c] = eos_phi<real>(A, E[c]);
        const Row3<real> rm{E[c - m.sx - 1], E[c - m.sx], E[c - m.sx + 1]};
        const Row3<real> rz{E[c - 1], E[c], E[c + 1]};
        const Row3<real> rp{E[c + m.sx - 1], E[c + m.sx], E[c + m.sx + 1]};
        La[c] = lap9<real>(rm, rz, rp);
    }
}

template <typename real>
__device__ __forceinline__ Row3<real> row3e(const real *X, int c)
{
    return Row3<real>{X[c - 1], X[c], X[c + 1]};
}

// Force, collision, pressure columns and push streaming of every fluid node
// (MODE_STEP), or its density and velocity (MODE_FIELDS). Wall-row
// velocities and pressures go to wv[4][nx] (rows 1, 2, ny-3, ny-2) and
// pw[2][nx] (rows 1, ny-2) for the wall kernel.
template <typename real, int MODE>
__global__ void __launch_bounds__(MB) mask_collide_kernel(const KArgs<real> A, const MaskDev m, const real *E,
                                                          const real *Pa, const real *La, real *wv, real *pw)
{
    const int nx = m.nx, ny = m.ny, P = m.pitch, rstride = 9 * P, sx = m.sx;
    const int n = nx * ny;
    constexpr bool PAIR = sizeof(real) == 4;  // FP32: the mass as a compensated FP32 pair (FP64 is 1/64 rate)
    double mass = 0.0;
    float mhi = 0.f, mlo = 0.f;
    bool bad = false;
    for (int k = blockIdx.x * MB + threadIdx.x; k < n; k += gridDim.x * MB) {
        const unsigned lk = m.links[k];
        if (lk >> 15) continue;  // solid
        const int y = k / nx, xa = k - y * nx;
        const bool pin = m.bc_x && xa == 0, pout = m.bc_x && xa == nx - 1, anyp = pin || pout;
        const int xs = pin ? 1 : (pout ? nx - 2 : xa);  // a pressure column collides its interior neighbour
        const int c = ext(m, xs, y);
        real f[9];
        const int rs = y * rstride + xs;
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = A.fin[rs + i * P];
        real ngpx, ngpy, glx, gly;
        ngrad12<real>(row3e(Pa, c - sx), row3e(Pa, c), row3e(Pa, c + sx), ngpx, ngpy);
        grad12<real>(row3e(La, c - sx), row3e(La, c), row3e(La, c + sx), glx, gly);
        const real rho = E[c];
        const real kr = mul_(A.kappa, rho);
        const real Fx = add_(mulk(fma_(kr, glx, ngpx), 1.0 / 12.0), A.gx);
        const real Fy = add_(mulk(fma_(kr, gly, ngpy), 1.0 / 12.0), A.gy);
        const real jx = add_(add_(sub_(f[1], f[3]), sub_(f[5], f[6])), sub_(f[8], f[7]));
        const real jy = sub_(add_(sub_(f[2], f[4]), add_(f[5], f[6])), add_(f[7], f[8]));
        const real irho = rcp_(rho);
        const real ux = mul_(jx, irho), uy = mul_(jy, irho);
        const real hFi = mul_(irho, real(0.5));
        const real vx = fma_(hFi, Fx, ux), vy = fma_(hFi, Fy, uy);
        const real rho_own = anyp ? E[ext(m, xa, y)] : rho;
        if (MODE == MODE_FIELDS) {
            A.o_rho[k] = rho_own;
            A.o_vx[k] = vx;
            A.o_vy[k] = vy;
        } else {
            real fs[9];
            if (anyp) {
                const real mvx = fma_(real(0.5), Fx, jx), mvy = fma_(real(0.5), Fy, jy);
                column_extrapolate<real>(A, rho_own, rho, vx, vy, mvx, mvy, f, fs);
            } else {
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
            const int oi = y * rstride + xa;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if ((lk >> i) & 1u) {
                    A.fout[oi + opp_(i) * P] = fs[i];  // half-way bounce-back at a wall row or an obstacle
                    continue;
                }
                int tx = xa + ex_(i), ty = y + ey_(i);
                if (m.bc_x) {
                    if (tx < 0 || tx >= nx) continue;  // leaves through the column
                } else {
                    tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
                }
                if (!m.walls) ty = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
                A.fout[ty * rstride + i * P + tx] = fs[i];
            }
            if constexpr (PAIR) two_sum_acc(mhi, mlo, (float)rho_own);
            else mass += (double)rho_own;
            bad = bad || !(rho > real(0)) || !(rho < real(1e30));
        }
        if (m.walls && !anyp) {
            // rows 1, 2 (bottom wall) and ny-3, ny-2 (top wall); with ny = 4 or 5 a
            // row can serve both walls
            if (y == 1 || y == 2) wv[(y - 1) * nx + xa] = vx;
            if (y == ny - 3 || y == ny - 2) wv[(y - ny + 5) * nx + xa] = vx;
            if (y == 1 || y == ny - 2) {
                // Eq. 2.4 in mesh units: k^2 p0 - kappa rho lap rho - kappa/2 |grad rho|^2
                real grx, gry;
                grad12<real>(row3e(E, c - sx), row3e(E, c), row3e(E, c + sx), grx, gry);
                grx = mulk(grx, 1.0 / 12.0);
                gry = mulk(gry, 1.0 / 12.0);
                const real k2p0 = add_(Pa[c], mulk(rho, 1.0 / 3.0));
                const real t = fma_(mul_(A.kappa, rho), -La[c], k2p0);
                const real pwv = fma_(fma_(grx, grx, mul_(gry, gry)), mul_(real(-0.5), A.kappa), t);
                if (y == 1) pw[xa] = pwv;
                if (y == ny - 2) pw[nx + xa] = pwv;
            }
        }
    }
    if (MODE != MODE_STEP) return;
    // per-block mass and bad-density flag (fixed order: warp tree, then warps in order)
    __shared__ double red[MB / 32];
    __shared__ int anybad;
    if (threadIdx.x == 0) anybad = 0;
    if constexpr (PAIR) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, mhi, o), l2 = __shfl_xor_sync(0xffffffffu, mlo, o);
            two_sum_acc(mhi, mlo, h2);
            mlo = __fadd_rn(mlo, l2);
        }
        mass = (double)mhi + (double)mlo;
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mass += __shfl_xor_sync(0xffffffffu, mass, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mass;
    if (bad) anybad = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < MB / 32; ++w) s += red[w];
        A.mass_part[blockIdx.x] = s;
        if (anybad || !(s - s == 0.0)) atomicOr(A.err, 1);
    }
}

// Wall shear and wall pressure of the open wall columns (both rows next to the
// wall fluid): tau_w = rho_1 nu (9 v_1 - v_2) / 3, p_w from the collide kernel.
template <typename real, int MODE>
__global__ void __launch_bounds__(MB) mask_wall_kernel(const KArgs<real> A, const MaskDev m, const real *E,
                                                       const real *wv, const real *pw)
{
    const int nx = m.nx, ny = m.ny;
    const real third = real(1.0 / 3.0);
    double J = 0.0;
    real e[4] = {real(INFINITY), real(-INFINITY), real(INFINITY), real(-INFINITY)};
    for (int x = blockIdx.x * MB + threadIdx.x; x < nx; x += gridDim.x * MB) {
        if (m.bc_x && (x == 0 || x == nx - 1)) continue;
        if (!m.solid[nx + x] && !m.solid[2 * nx + x]) {
            const real tw = mul_(mul_(E[ext(m, x, 1)], A.nu), mul_(fma_(real(9), wv[x], -wv[nx + x]), third));
            if (MODE == MODE_FIELDS) {
                A.o_tw[x] = tw;
                A.o_pw[x] = pw[x];
            } else {
                J += (double)tw;
                e[0] = fmin(e[0], tw); e[1] = fmax(e[1], tw);
                e[2] = fmin(e[2], pw[x]); e[3] = fmax(e[3], pw[x]);
            }
        }
        if (!m.solid[(ny - 2) * nx + x] && !m.solid[(ny - 3) * nx + x]) {
            const real tw = mul_(mul_(E[ext(m, x, ny - 2)], A.nu),
                                 mul_(fma_(real(9), wv[3 * nx + x], -wv[2 * nx + x]), third));
            if (MODE == MODE_FIELDS) {
                A.o_tw[nx + x] = tw;
                A.o_pw[nx + x] = pw[nx + x];
            } else {
                J += (double)tw;
                e[0] = fmin(e[0], tw); e[1] = fmax(e[1], tw);
                e[2] = fmin(e[2], pw[nx + x]); e[3] = fmax(e[3], pw[nx + x]);
            }
        }
    }
    if (MODE != MODE_STEP) return;
    __shared__ double sj[MB];
    __shared__ real se[4][MB];
    sj[threadIdx.x] = J;
    for (int q = 0; q < 4; ++q) se[q][threadIdx.x] = e[q];
    __syncthreads();
    for (int s = MB / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sj[threadIdx.x] += sj[threadIdx.x + s];
            se[0][threadIdx.x] = fmin(se[0][threadIdx.x], se[0][threadIdx.x + s]);
            se[1][threadIdx.x] = fmax(se[1][threadIdx.x], se[1][threadIdx.x + s]);
            se[2][threadIdx.x] = fmin(se[2][threadIdx.x], se[2][threadIdx.x + s]);
            se[3][threadIdx.x] = fmax(se[3][threadIdx.x], se[3][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {  // one slot per block (the collide kernel's slot count bounds the grid)
        real *ex = A.ext + 4 * blockIdx.x;
        A.J_acc[blockIdx.x] += sj[0];
        ex[0] = fmin(ex[0], se[0][0]); ex[1] = fmax(ex[1], se[1][0]);
        ex[2] = fmin(ex[2], se[2][0]); ex[3] = fmax(ex[3], se[3][0]);
    }
}

// ---------------------------------------------------------------------------
// Host: the ghost table.
// ---------------------------------------------------------------------------

struct HostGeom {
    int nx, ny, walls, bc_x;
    const std::vector<uint8_t> *solid;
    // maps a point onto the lattice; false for rows outside a walled lattice
    bool map(int &x, int &y) const
    {
        if (bc_x) x = std::min(std::max(x, 0), nx - 1);
        else x = ((x % nx) + nx) % nx;
        if (walls) return y >= 0 && y < ny;
        y = ((y % ny) + ny) % ny;
        return true;
    }
    bool fluid(int x, int y) const { return map(x, y) && !(*solid)[(size_t)y * nx + x]; }
};

// Sources (lattice nodes) of the ghost density at solid point (x, y).
void ghost_sources(const HostGeom &g, int x, int y, std::vector<int> &sx, std::vector<int> &sy)
{
    static const int axis[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    static const int diag[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    static const int knight[8][2] = {{1, 2}, {2, 1}, {-1, 2}, {-2, 1}, {-1, -2}, {-2, -1}, {1, -2}, {2, -1}};
    sx.clear();
    sy.clear();
    for (int set = 0; set < 2 && sx.empty(); ++set) {
        const int (*dir)[2] = set ? diag : axis;
        for (int d = 1; d <= 2 && sx.empty(); ++d)
            for (int k = 0; k < 4; ++k) {
                const int dx = dir[k][0], dy = dir[k][1];
                if (!g.fluid(x + d * dx, y + d * dy) || (d == 2 && g.fluid(x + dx, y + dy))) continue;
                int px = x + (2 * d - 1) * dx, py = y + (2 * d - 1) * dy;
                if (!g.fluid(px, py)) { px = x + d * dx; py = y + d * dy; }
                g.map(px, py);
                sx.push_back(px);
                sy.push_back(py);
            }
    }
    if (sx.empty())
        for (int k = 0; k < 8; ++k) {
            int px = x + knight[k][0], py = y + knight[k][1];
            if (!g.fluid(px, py)) continue;
            g.map(px, py);
            sx.push_back(px);
            sy.push_back(py);
        }
}

}  // namespace

struct MaskPath {
    MaskDev d{};
    int precision = 32;
    size_t ne = 0;            // extended-array points
    unsigned char *mem = nullptr;
    void *E = nullptr, *Pa = nullptr, *La = nullptr, *wv = nullptr, *pw = nullptr;
    int blocks = 0;
};

int mask_blocks(const MaskPath *m) { return m ? m->blocks : 0; }

void mask_free(MaskPath *m)
{
    if (!m) return;
    cudaFree(m->mem);
    delete m;
}

// Validates the mask (with pressure columns, columns 0, 1, nx-2, nx-1 must be
// open outside the wall rows), builds the ghost table and uploads everything.
// *out = NULL with LBM_OK when the mask adds no solid node and !force.
lbm_status mask_setup(const uint8_t *mask, const lbm_grid &g, int pitch, int sms, bool force, cudaStream_t stream,
                      MaskPath **out, char *err, size_t errlen)
{
    *out = nullptr;
    const int nx = g.nx, ny = g.ny;
    std::vector<uint8_t> solid((size_t)nx * ny, 0);
    bool extra = false;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const bool wall = g.walls && (y == 0 || y == ny - 1);
            const bool ms = mask && mask[(size_t)y * nx + x] != 0;
            if (ms && !wall) {
                extra = true;
                if (g.bc_x && (x <= 1 || x >= nx - 2)) {
                    std::snprintf(err, errlen, "wall mask: solid node (%d, %d) on or next to a pressure column", x, y);
                    return LBM_ERR_ARG;
                }
            }
            solid[(size_t)y * nx + x] = (ms || wall) ? 1 : 0;
        }
    if (!extra && !force) return LBM_OK;

    HostGeom hg{nx, ny, g.walls, g.bc_x, &solid};
    const int sx = nx + 4;
    auto ext_idx = [&](int x, int y) { return (y + 2) * sx + (x + 2); };
    std::vector<int> gdst, gbeg{0}, gsrc;
    std::vector<uint8_t> gwet;
    std::vector<int> px, py;
    for (int y = -2; y <= ny + 1; ++y)
        for (int x = -2; x <= nx + 1; ++x) {
            int mx = x, my = y;
            const bool in = hg.map(mx, my);
            if (in && !solid[(size_t)my * nx + mx]) {
                if (mx == x && my == y) continue;  // a lattice node: written by the density / column kernels
                gdst.push_back(ext_idx(x, y));     // a wrapped or clamped copy
                gsrc.push_back(ext_idx(mx, my));
                gbeg.push_back((int)gsrc.size());
                gwet.push_back(0);
                continue;
            }
            ghost_sources(hg, x, y, px, py);
            gdst.push_back(ext_idx(x, y));
            for (size_t j = 0; j < px.size(); ++j) gsrc.push_back(ext_idx(px[j], py[j]));
            gbeg.push_back((int)gsrc.size());
            gwet.push_back(1);
        }

    // per-node link table: which pushes bounce back (a wall-row target first,
    // as the channel kernels order it; targets beyond a pressure column leave
    // and are not marked), and whether the node itself is solid
    static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    std::vector<uint16_t> links((size_t)nx * ny, 0);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (solid[(size_t)y * nx + x]) {  // never pushes; its targets may lie outside the lattice
                links[(size_t)y * nx + x] = (uint16_t)0x8000u;
                continue;
            }
            uint16_t l = 0;
            for (int i = 1; i < 9; ++i) {
                int tx = x + EX[i], ty = y + EY[i];
                if (g.walls && (ty == 0 || ty == ny - 1)) { l |= (uint16_t)(1u << i); continue; }
                if (g.bc_x) {
                    if (tx < 0 || tx >= nx) continue;
                } else {
                    tx = (tx + nx) % nx;
                }
                if (!g.walls) ty = (ty + ny) % ny;
                if (solid[(size_t)ty * nx + tx]) l |= (uint16_t)(1u << i);
            }
            links[(size_t)y * nx + x] = l;
        }

    MaskPath *m = new (std::nothrow) MaskPath();
    if (!m) return LBM_ERR_OOM;
    m->precision = g.precision;
    const size_t sz = g.precision == 64 ? 8 : 4;
    m->ne = (size_t)(nx + 4) * (ny + 4);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_solid = al(solid.size()), b_links = al(links.size() * 2), b_ext = al(m->ne * sz),
                 b_dst = al(gdst.size() * 4),
                 b_beg = al(gbeg.size() * 4), b_src = al(std::max<size_t>(1, gsrc.size()) * 4),
                 b_wet = al(gwet.size()), b_wv = al(4 * (size_t)nx * sz), b_pw = al(2 * (size_t)nx * sz);
    const size_t total = b_solid + b_links + 3 * b_ext + b_dst + b_beg + b_src + b_wet + b_wv + b_pw;
    if (cudaMalloc((void **)&m->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return LBM_ERR_OOM;
    }
    unsigned char *p = m->mem;
    uint8_t *d_solid = p; p += b_solid;
    uint16_t *d_links = (uint16_t *)p; p += b_links;
    m->E = p; p += b_ext;
    m->Pa = p; p += b_ext;
    m->La = p; p += b_ext;
    int *d_dst = (int *)p; p += b_dst;
    int *d_beg = (int *)p; p += b_beg;
    int *d_src = (int *)p; p += b_src;
    uint8_t *d_wet = p; p += b_wet;
    m->wv = p; p += b_wv;
    m->pw = p;
    cudaError_t e = cudaMemsetAsync(m->mem, 0, total, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_solid, solid.data(), solid.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_links, links.data(), links.size() * 2, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_dst, gdst.data(), gdst.size() * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_beg, gbeg.data(), gbeg.size() * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && !gsrc.empty())
        e = cudaMemcpyAsync(d_src, gsrc.data(), gsrc.size() * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_wet, gwet.data(), gwet.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // the host vectors die here
    if (e != cudaSuccess) {
        std::snprintf(err, errlen, "wall mask upload: %s", cudaGetErrorString(e));
        mask_free(m);
        return LBM_ERR_CUDA;
    }
    m->d = MaskDev{nx, ny, pitch, g.walls, g.bc_x, sx, d_solid, d_links, d_dst, d_beg, d_src, d_wet,
                   (int)gdst.size()};
    const long long nodes = (long long)nx * ny;
    m->blocks = (int)std::max<long long>(1, std::min<long long>((nodes + MB - 1) / MB, (long long)sms * 8));
    m->blocks = std::min(m->blocks, MAX_CTAS);
    *out = m;
    return LBM_OK;
}

namespace {
int grid_for(long long n, int cap) { return (int)std::max<long long>(1, std::min<long long>((n + MB - 1) / MB, cap)); }
}  // namespace

template <typename real>
cudaError_t mask_launch(const MaskPath *m, const KArgs<real> &A, int mode, cudaStream_t s)
{
    const MaskDev &d = m->d;
    real *E = (real *)m->E, *Pa = (real *)m->Pa, *La = (real *)m->La, *wv = (real *)m->wv, *pw = (real *)m->pw;
    const int cap = m->blocks;
    mask_density_kernel<real><<<grid_for((long long)d.nx * d.ny, cap), MB, 0, s>>>(A, d, E);
    if (d.bc_x) mask_columns_kernel<real><<<grid_for(d.ny, cap), MB, 0, s>>>(A, d, E);
    mask_ghost_kernel<real><<<grid_for(d.nghost, cap), MB, 0, s>>>(A, d, E);
    mask_phi_lap_kernel<real><<<grid_for((long long)(d.nx + 2) * (d.ny + 2), cap), MB, 0, s>>>(A, d, E, Pa, La);
    // the wall columns spread over as many blocks as fill them (at most the
    // collide kernel's block count, whose per-block slots the partials use)
    const int wb = (int)std::min<long long>(cap, ((long long)d.nx + MB - 1) / MB);
    if (mode == MODE_STEP) {
        mask_collide_kernel<real, MODE_STEP><<<m->blocks, MB, 0, s>>>(A, d, E, Pa, La, wv, pw);
        if (d.walls) mask_wall_kernel<real, MODE_STEP><<<wb, MB, 0, s>>>(A, d, E, wv, pw);
    } else {
        mask_collide_kernel<real, MODE_FIELDS><<<m->blocks, MB, 0, s>>>(A, d, E, Pa, La, wv, pw);
        if (d.walls) mask_wall_kernel<real, MODE_FIELDS><<<wb, MB, 0, s>>>(A, d, E, wv, pw);
    }
    return cudaGetLastError();
}

template cudaError_t mask_launch<float>(const MaskPath *, const KArgs<float> &, int, cudaStream_t);
template cudaError_t mask_launch<double>(const MaskPath *, const KArgs<double> &, int, cudaStream_t);

}  // namespace lbm
