// Declarations shared by the host translation units of the solver library.
#pragma once

#ifdef __CUDACC__
#include <cuda.h>  // CUtensorMap
#endif

#include <cstdint>

#include "lbm.h"

namespace lbm {

// Equation-of-state parameters at absolute temperature T: Carnahan-Starling
// (kind 0) or Peng-Robinson (kind 1, Eq. 2.18, with aalpha = a alpha(T)).
struct Thermo {
    double a, b, R, T;
    int kind = 0;
    double aalpha = 0.0;
};

double eos_pressure(const Thermo &t, double rho);
double eos_dpressure(const Thermo &t, double rho);
// Critical point (PR: alpha(Tc) = 1).
void eos_critical(int kind, double a, double b, double R, double *Tc, double *rhoc);
// Standard PR temperature function alpha(T) for acentric factor omega.
double pr_alpha(double omega, double T_over_Tc);
// Maxwell coexistence below Tc; returns nonzero at or above Tc.
int maxwell(const Thermo &t, double *rho_g, double *rho_l, double *p_sat);
// Density on the gas (liquid) branch whose EOS pressure is p. A pressure
// beyond the branch's end gives the spinodal density and sets *saturated.
// Nonzero if p <= 0 (gas) or if there is no liquid branch (T >= Tc).
int gas_density(const Thermo &t, double p, double *rho, bool *saturated = nullptr);
int liquid_density(const Thermo &t, double p, double *rho, bool *saturated = nullptr);
// Thermodynamic state of an lbm_eos: T, Tc and the Thermo; nonzero on bad parameters.
int thermo_of(const lbm_eos &e, Thermo *t, double *Tc);

// Thermodynamics of one channel: Maxwell coexistence (rho_g = rho_l = 0 above
// Tc: no phase blending) and, with pressure columns, the column densities on
// both branches at the mesh pressures p_ref +- dp/2 (p_ref NaN: k^2 p_sat).
// sat[0..3] flag a column density held at a spinodal (gas_in, liq_in,
// gas_out, liq_out). Returns nonzero if the parameters admit no columns.
struct ChannelThermo {
    Thermo th{};
    double T = 0, Tc = 0, rho_g = 0, rho_l = 0, p_sat = 0;
    double rho_in = 0, rho_out = 0, rho_in_l = 0, rho_out_l = 0;
    bool sat[4] = {false, false, false, false};
};
int channel_thermo(const lbm_eos &e, const lbm_drive &d, bool bc_x, ChannelThermo *out);
double node_noise(uint64_t seed, uint64_t node, double amp);

// Row pitch of a population plane: nx rounded up to 4 columns, so that every
// row segment of the bulk-copy staged kernel is 16-byte aligned.
inline int pitch_of(int nx) { return (nx + 3) & ~3; }

// Whether 32-bit population offsets address the grid: 9 pitch ny < 2^31
// (about 238 million nodes). Larger single-channel grids take the kernels
// with 64-bit offsets; the batch, the wall-mask path, the allocation-free
// entry and the adjoint keep the 32-bit bound.
inline bool idx32_ok(int nx, int ny) { return 9ll * pitch_of(nx) * ny < (1ll << 31); }

// Strip width for an nx-column channel: the widest up to w_max, except that
// the outlet column must not open a strip (its stencil reaches two columns
// back); widths that keep 16-byte alignment (multiples of 4) are preferred.
inline int strip_width(int nx, int w_max, bool bc_x)
{
    int W = w_max;
    if (!(bc_x && nx > W && nx % W == 1)) return W;
    for (int w = (W - 1) & ~3; w >= 4; w -= 4)
        if (nx % w != 1) return w;
    for (int w = W - 1; w >= 2; --w)
        if (nx % w != 1) return w;
    return W;
}

} // namespace lbm

// The current population state of a context in its own layout (rows of nine
// planes, plane pitch pitch_of(nx), 9 * pitch * ny values): an asynchronous
// device copy out of it / into both of its buffers, on the context's stream
// and without synchronising (the public lbm_populations / lbm_load_populations
// convert to the plane-major ABI layout and synchronise). lbm_api.cu.
#ifdef __CUDACC__
// 2-D tensor map of one FP32 population array (pitch wide, 9 * ny plane-rows)
// in the form the row-pair stage loads it (lbm_api.cu); false if the driver
// entry point is unavailable or the layout does not qualify.
bool lbm_encode_population_map(CUtensorMap *map, void *base, int pitch, int ny);
cudaError_t lbm_ctx_copy_state(lbm_ctx *ctx, void *dst);
const void *lbm_ctx_state(const lbm_ctx *ctx);  // the current state buffer itself (device)
cudaError_t lbm_ctx_load_state(lbm_ctx *ctx, const void *src);

namespace lbm {
template <typename real>
struct KArgs;
// The general-geometry step on a lattice with a solid mask (lbm_mask.cu).
// mask_setup validates the mask, builds the ghost table and allocates the
// path's device tables; *out stays NULL (LBM_OK) when the mask adds no solid
// node to the wall rows, unless `force`. mask_launch runs one step (mode
// MODE_STEP) or the fields (MODE_FIELDS) of A.fin on `stream`.
struct MaskPath;
lbm_status mask_setup(const uint8_t *mask, const lbm_grid &g, int pitch, int sms, bool force, cudaStream_t stream,
                      MaskPath **out, char *err, size_t errlen);
void mask_free(MaskPath *m);
int mask_blocks(const MaskPath *m);  // CTAs of the collide kernel (diagnostic slots)
template <typename real>
cudaError_t mask_launch(const MaskPath *m, const KArgs<real> &A, int mode, cudaStream_t stream);

// In-place streaming (the AA pattern) of a single context (lbm_inplace.cu):
// one population array F, a density plane rho (pitch * ny) and a side buffer
// (2 * ny * 9) for the pressure columns. aa_plan sizes the tile grid and the
// CTA counts; aa_step runs one step of F (even: natural layout in, odd-parity
// layout out; odd: the reverse); aa_swap turns an odd-parity F back into the
// natural layout in place.
struct AAPlan {
    int ntx, nty, sx, sy;  // tile grid of the step and its shifts
    int nctas;             // CTAs of the step (its diagnostic slots)
    int threads;           // threads per CTA of the step
    int dens_blocks;       // CTAs of the density pass
};
cudaError_t aa_plan(int precision, bool big, bool walls, bool pres, int nx, int ny, int sms, AAPlan *p);
template <typename real>
cudaError_t aa_step(const KArgs<real> &A, real *F, real *rho, real *side, bool walls, bool pres, bool odd, bool big,
                    const AAPlan &p, cudaStream_t st);
cudaError_t aa_swap(int precision, void *F, bool walls, bool pres, bool big, int nx, int ny, int P, int sms,
                    cudaStream_t st);
}  // namespace lbm
#endif

// Launchable step kernel (lbm_api.cu) for a precision (32/64), a mode
// (lbm::MODE_STEP or MODE_FIELDS), the boundary set, the staged variant and a
// row pitch above nx (padded).
void *lbm_step_kernel_ptr(int precision, int mode, bool walls, bool pres, bool staged, bool padded);
// The same kernels with 64-bit population offsets (lbm_big.cu), and the FP32
// row-pair step likewise, for grids whose 9 pitch ny slots reach 2^31.
void *lbm_big_step_kernel_ptr(int precision, int mode, bool walls, bool pres, bool staged, bool padded);
void *lbm_big_rows2_kernel_ptr(bool walls, bool pres, bool padded);
