/*
 * lbm.h — C ABI of the GB300 (sm_103a) EOS-based multiphase lattice Boltzmann
 * solver: the time-step hot path of He, Qin, Chen & Wen, "Numerical
 * simulation of pulmonary airway reopening by the EOS-based multiphase lattice
 * Boltzmann method" (arXiv 2103.08301).
 *
 * One time step (lbm_step) is, at every fluid node of a D2Q9 lattice:
 *   moments        rho = sum f_i, u = sum f_i e_i / rho                 (Sec. 2.1)
 *   nonideal force F = -grad(k^2 p0(rho) - rho/3) + kappa rho grad(lap rho) + G
 *                  with the EOS p0 evaluated directly                    (Eqs. 2.12-2.17)
 *   collision      BGK towards f_eq(rho, u + tau F / rho)               (Eq. 2.2, Sec. 2.1)
 *   boundaries     half-way bounce-back walls, mirror ghost density for
 *                  wetting, pressure inlet/outlet columns                (Sec. 2.2)
 *   streaming      f_i(x + e_i, t + 1) = f*_i(x, t)                     (Eq. 2.1)
 * The paper names the Peng-Robinson EOS (Eq. 2.18) and an MRT operator; this
 * ABI computes the Carnahan-Starling EOS, p0 = rho R T (1 + eta + eta^2 -
 * eta^3)/(1 - eta)^3 - a rho^2 with eta = b rho / 4, and the single-relaxation
 * (BGK) operator that the paper lists among its LBE variants (Sec. 2.1).
 *
 * Conventions
 *   - Lattice nodes are (x, y), 0 <= x < nx, 0 <= y < ny, node index y*nx + x.
 *   - Populations cross this ABI as nine planes f[i][y][x] (structure of
 *     arrays), i = 0..8 with e = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),
 *     (-1,-1),(1,-1). Inside a context the library keeps them row-interleaved,
 *     f[y][i][x], and converts on lbm_populations / lbm_load_populations.
 *   - Real-valued buffers use the context precision: float for precision 32,
 *     double for precision 64. Host inputs are always double.
 *   - All functions return an lbm_status; none aborts or traps. After
 *     LBM_ERR_NAN the context keeps running but its fields are meaningless
 *     until lbm_restore or lbm_load_populations.
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - Work is issued on the context's CUDA stream. lbm_step is asynchronous;
 *     lbm_fields, lbm_diag, lbm_populations and lbm_checkpoint synchronise
 *     that stream before returning.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,   /* NULL pointer, bad size or flag, buffer too small */
    LBM_ERR_PARAM = 2, /* tau <= 1/2; T >= Tc without explicit p_ref;
                          kappa < 0; k <= 0; unknown EOS kind */
    LBM_ERR_CUDA = 3,  /* a CUDA runtime call failed (lbm_last_error has the text) */
    LBM_ERR_OOM = 4,   /* device or host allocation failed */
    LBM_ERR_NAN = 5,   /* a step met a non-finite or non-positive density */
    LBM_ERR_STATE = 6, /* checkpoint of another geometry or precision */
    LBM_ERR_TIMEOUT = 7 /* a bounded wait for a staged population row gave up */
} lbm_status;

/* Lattice and geometry (Sec. 2.2: straight rigid channel of the airway model).
 * walls: 0 = periodic in y; 1 = rows 0 and ny-1 are solid no-slip walls (the
 *        channel walls; lbm_init's wall_mask adds solid nodes anywhere).
 * bc_x:  0 = periodic in x; 1 = column 0 is the pressure inlet and column
 *        nx-1 the pressure outlet.
 * Limits: nx, ny >= 4 (>= 1 for a periodic axis); pitch*ny < 2^31 nodes and
 * 9*ny < 2^31, with pitch = nx rounded up to a multiple of 4. A context whose
 * 9*pitch*ny population slots reach 2^31 (above ~238 million nodes) steps
 * with kernels that take 64-bit population offsets; the wall-mask path
 * (wall_mask, LBM_OPT_GENERAL), the batch, lbm_step_noalloc and the adjoint
 * keep 9*pitch*ny < 2^31 (LBM_ERR_ARG above). */
typedef struct {
    int32_t nx, ny;
    int32_t walls;
    int32_t bc_x;
    int32_t precision; /* 32 (float state) or 64 (double state) */
} lbm_grid;

/* Equation of state and the model coefficients of Eq. 2.17.
 * kind 0 (LBM_EOS_CS): Carnahan-Starling, p0 = rho R T (1 + e + e^2 - e^3)/(1 - e)^3
 *   - a rho^2 with e = b rho / 4 (the default of a zero-initialised field).
 * kind 1 (LBM_EOS_PR): Peng-Robinson (Eq. 2.18), p0 = rho R T / (1 - b rho)
 *   - a alpha rho^2 / (1 + 2 b rho - b^2 rho^2), alpha = [1 + (0.37464 +
 *   1.54226 omega - 0.26992 omega^2)(1 - sqrt(T/Tc))]^2 (the standard form of
 *   the temperature function, which the paper prints garbled).
 * T = T_over_Tc * Tc with Tc the EOS critical temperature (PR: alpha(Tc) = 1).
 * k: proportional coefficient (Eq. 2.13); the mesh-space EOS is k^2 p0 (Eq. 2.14).
 * kappa: gradient coefficient of Eq. 2.17, taken in mesh units.
 * omega: PR acentric factor (0.344 water, 0.011 methane); unused for CS. */
enum { LBM_EOS_CS = 0, LBM_EOS_PR = 1 };
typedef struct {
    double a, b, R;
    double T_over_Tc;
    double k;
    double kappa;
    int32_t kind;
    double omega;
} lbm_eos;

/* Driving. With bc_x = 1 the inlet and outlet columns carry the mesh
 * pressures k^2 p0 = p_ref + dp/2 and p_ref - dp/2 (pressure drop dp,
 * Sec. 2.2 / Sec. 3.3); p_ref = NaN selects k^2 p_sat(T). A column node's
 * density is the EOS root at its pressure on the branch of the phase at its
 * interior neighbour x_f: rho_b = rho_gas + theta (rho_liq - rho_gas),
 * theta = clamp((rho(x_f) - rho_g) / (rho_l - rho_g), 0, 1) with the Maxwell
 * densities rho_g, rho_l (theta = 0 above Tc). Its populations are rebuilt
 * each step by non-equilibrium extrapolation from x_f.
 * (gx, gy) is a uniform body-force density added to F. */
typedef struct {
    double dp;
    double p_ref;
    double gx, gy;
} lbm_drive;

/* Diagnostics (Sec. 3: wall pressure and wall shear; Fig. 3). Per-step
 * quantities refer to the state each step reads, so after n steps they cover
 * states 0..n-1. */
typedef struct {
    int64_t step;          /* steps taken since lbm_init / last restore */
    double mass;           /* sum of rho over non-solid nodes of state step-1
                              (pressure columns count rho_b); 0 before any step */
    double wall_shear_sum; /* sum over states and columns of tau_w(bottom) + tau_w(top) */
    double tau_wall_min, tau_wall_max; /* extrema of tau_w over walls and states */
    double p_wall_min, p_wall_max;     /* extrema of the wall pressure (Eq. 2.4) */
    int32_t nan_detected;  /* nonzero once any step met a bad density (a stage
                              wait that gave up shows as LBM_ERR_TIMEOUT from lbm_step) */
    int32_t pad_;
    /* thermodynamic set-up derived by lbm_init (host FP64); rho_in / rho_out
       are the gas-branch and rho_in_l / rho_out_l the liquid-branch densities
       at the inlet / outlet pressures */
    double T, Tc, rho_g, rho_l, p_sat, rho_in, rho_out, rho_in_l, rho_out_l;
} lbm_diag_t;

/* Bytes of device memory a context of this grid needs (two population
 * arrays plus diagnostics). 0 on invalid grid. */
size_t lbm_workspace_bytes(const lbm_grid *grid);

/* Create a context. (Failure-detection tests: the environment variable
 * LBM_FAULT=alloc makes lbm_init fail with LBM_ERR_OOM after its device
 * allocations, releasing them; LBM_FAULT=param makes it fail with
 * LBM_ERR_PARAM before any CUDA call.)
 *   grid, eos, drive: copied. drive may be NULL (no drive).
 *   tau:      BGK relaxation time, > 1/2.
 *   wall_mask: NULL, or a host array of nx*ny bytes (node y*nx + x), nonzero =
 *             solid node; copied. General geometry for the no-slip walls of
 *             Sec. 2.2: half-way bounce-back on every link into a solid node,
 *             and ghost densities at solid points for the stencils of Eq. 2.17:
 *             the flat-wall mirror rule generalised (along the axis directions
 *             of least depth d <= 2 to fluid, the point (2d-1) nodes out, or d
 *             nodes out if that is solid; else the diagonals likewise; else the
 *             fluid points at knight offsets; the mean of those densities plus
 *             `wetting`). Solid nodes keep their populations and report zero
 *             fields. With grid->walls = 1 rows 0 and ny-1 are solid whatever
 *             the mask says; with bc_x = 1 columns 0, 1, nx-2 and nx-1 must be
 *             fluid outside the wall rows (LBM_ERR_ARG otherwise). A mask that
 *             adds no solid node to the wall rows runs the channel kernels; any
 *             other runs the general-geometry kernels, whose device tables
 *             (about 13 bytes per node plus the ghost table) the library
 *             allocates even when `workspace` is given. Wall shear and wall
 *             pressure count the wall columns whose two rows next to the wall
 *             are fluid.
 *   wetting:  ghost-density offset added to mirrored wall densities
 *             (0 = neutral wetting, 90-degree contact angle).
 *   rho0:     host array of nx*ny doubles, the initial density; the
 *             populations start at f_eq(rho0, 0). Copied. Required.
 *   workspace, ws_bytes: device buffer of at least lbm_workspace_bytes(grid)
 *             bytes, 256-byte aligned, owned by the caller and kept alive
 *             until lbm_free; NULL lets the library allocate (cudaMalloc) and
 *             free it.
 *   stream:   cudaStream_t to issue all work on; NULL = legacy default stream.
 *   out:      receives the context; *out is NULL on failure.
 * Errors: LBM_ERR_ARG, LBM_ERR_PARAM, LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_init(const lbm_grid *grid, const lbm_eos *eos, double tau, const uint8_t *wall_mask,
                    double wetting, const lbm_drive *drive, const double *rho0, void *workspace,
                    size_t ws_bytes, void *stream, lbm_ctx **out);

/* In-place streaming (the AA pattern of Bailey et al., ICPP 2009): a context
 * that stores one population array instead of two, plus one density plane
 * (FP32: 40 bytes per node instead of 72), for grids that would not fit
 * otherwise. Even steps read each node's own slots and write its
 * post-collision populations back reversed; odd steps read from and write to
 * the neighbours' slots, restoring the natural layout. Each step runs two
 * kernels: the density of every fluid node into the plane (the stencil of
 * Eq. 2.17 reaches neighbours whose slots may already hold their next state),
 * then the collision from that plane; traffic is 116 bytes per node and step
 * (FP32) instead of 72. Populations are identical bit for bit to an lbm_init
 * context's; diagnostic sums agree to rounding (another summation order).
 * Arguments as lbm_init, without a wall mask (walls are the channel's rows 0
 * and ny-1 when grid->walls = 1); the workspace must hold
 * lbm_workspace_bytes_inplace(grid) bytes. Every other call works on the
 * context as on an lbm_init context, with these differences: the fields,
 * populations, checkpoint and lbm_step graph calls first bring an odd-parity
 * array back to the natural layout (one extra pass over it); checkpoints hold
 * the one array and restore only into in-place contexts (LBM_ERR_STATE
 * otherwise); LBM_OPT_GENERAL and LBM_OPT_FAULT_SKIP_COPY are rejected
 * (LBM_ERR_ARG), and the kernel-selection options (LBM_OPT_STAGED, ROWS2,
 * TMA, TILE, STRIP, CTAS_PER_SM, PREFETCH, PDL) affect only lbm_fields.
 * lbm_launch_info reports the step's CTAs, its threads per CTA (FP32: 128,
 * two rows each; FP64: 256), its 32 x 8 tiles as units, and no staging.
 * lbm_fields allocates its output scratch (3 nx ny values plus 4 nx) on first
 * use, as for any context. Errors: as lbm_init. */
size_t lbm_workspace_bytes_inplace(const lbm_grid *grid);
lbm_status lbm_init_inplace(const lbm_grid *grid, const lbm_eos *eos, double tau, double wetting,
                            const lbm_drive *drive, const double *rho0, void *workspace, size_t ws_bytes,
                            void *stream, lbm_ctx **out);

/* Advance n >= 0 time steps (one fused kernel launch each), asynchronously.
 * On a context created with a stream of its own, runs of LBM_OPT_GRAPH_STEPS
 * steps (default 64) starting from the first population buffer are replayed
 * from a CUDA graph captured on first use (identical results; changing an
 * option or the collision drops it). Returns LBM_ERR_NAN if a completed
 * earlier step met a bad density (checked without blocking), LBM_ERR_CUDA on
 * launch failure. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t n);

/* Macroscopic fields of the current state, computed on the GPU:
 *   rho, ux, uy: nx*ny values each (v = u + F/(2 rho), Sec. 2.1); solid
 *                nodes read 0; pressure columns read rho_b and v of their
 *                interior neighbour.
 *   tau_wall, p_wall: 2*nx values (bottom wall row then top wall row); zero
 *                for pressure columns and channels without walls.
 * Each pointer may be NULL (skipped), a device pointer or a host pointer, of
 * the context precision. Synchronises the stream. */
lbm_status lbm_fields(lbm_ctx *ctx, void *rho, void *ux, void *uy, void *tau_wall,
                      void *p_wall);

/* Reduce the diagnostics on the GPU (fixed order, deterministic) and return
 * them in *out (host). Synchronises the stream. */
lbm_status lbm_diag(lbm_ctx *ctx, lbm_diag_t *out);
/* lbm_diag without the synchronisation, for a caller that reads every step's
 * diagnostics while the next steps run: enqueues on the context's stream the
 * same reduction and an asynchronous copy of 7 doubles into dst (pinned host
 * or device memory, 8-byte aligned): mass, wall-shear sum, tau_w min/max,
 * p_w min/max (as lbm_diag; the extrema read +-inf before a wall row was
 * stepped) and the error word (bit 0 = bad density, bit 1 = a stage wait gave
 * up). dst is valid once the stream has passed this point (an event recorded
 * after the call, or a synchronisation). Errors: LBM_ERR_ARG (NULL or
 * misaligned dst), LBM_ERR_CUDA. */
lbm_status lbm_diag_async(lbm_ctx *ctx, double *dst);

/* Restart the diagnostic accumulators (wall-shear sum, wall shear and wall
 * pressure extrema) so that they cover the steps issued afterwards; the step
 * counter and the bad-density flag are kept. Asynchronous. Errors:
 * LBM_ERR_ARG, LBM_ERR_CUDA. */
lbm_status lbm_reset_diag(lbm_ctx *ctx);

/* Raw population state: 9*nx*ny values of the context precision, layout
 * f[i][y][x]. dst / src may be host or device pointers. */
lbm_status lbm_populations(lbm_ctx *ctx, void *dst);
lbm_status lbm_load_populations(lbm_ctx *ctx, const void *src);

/* Checkpoint / restore: populations, step counter and diagnostic
 * accumulators in a host buffer of lbm_checkpoint_bytes(ctx) bytes.
 * A restored run continues bit-identically. LBM_ERR_STATE if the buffer was
 * written by a context of another grid or precision. */
size_t lbm_checkpoint_bytes(const lbm_ctx *ctx);
lbm_status lbm_checkpoint(lbm_ctx *ctx, void *host_buf, size_t bytes);
lbm_status lbm_restore(lbm_ctx *ctx, const void *host_buf, size_t bytes);

/* Collision operator (Sec. 2.1). kind 0 (LBM_COLL_BGK): single relaxation
 * time tau, equilibrium velocity u + tau F / rho (the default). kind 1
 * (LBM_COLL_MRT): multiple relaxation times (Eq. 2.1) in the Lallemand-Luo
 * moment basis (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy) with
 * S = diag(0, s_e, s_eps, s_j, s_q, s_j, s_q, s_nu, s_nu); s_nu <= 0 means
 * 1/tau. The velocity-shift force enters through the equilibrium velocity
 * u + F / (s_j rho), so the relaxed momentum gains F per step; s_j = 1/tau
 * with every rate 1/tau is BGK. The paper's rates are s_e = 1.64,
 * s_eps = 1.54, s_q = 1.7, s_nu = 1/tau. NULL restores BGK. Applies to
 * steps issued afterwards. Errors: LBM_ERR_ARG (kind, or a rate outside
 * (0, 2) other than s_nu <= 0). */
enum { LBM_COLL_BGK = 0, LBM_COLL_MRT = 1 };
typedef struct {
    int32_t kind;
    double s_e, s_eps, s_j, s_q, s_nu;
} lbm_collision;
lbm_status lbm_set_collision(lbm_ctx *ctx, const lbm_collision *c);

/* Launch tuning and test hooks (set before stepping; changing the CTA count
 * resets the diagnostic accumulators):
 *   LBM_OPT_CTAS_PER_SM  resident CTAs per SM for the step grid (0 = from
 *                        the occupancy calculator)
 *   LBM_OPT_REVERSE      nonzero: launch the step's work units in reverse CTA
 *                        order (results must be bit-identical)
 *   LBM_OPT_STRIP        strip width in nodes (2..128)
 *   LBM_OPT_STAGED       nonzero (default): stream population rows through
 *                        shared memory with bulk asynchronous copies when nx
 *                        and the strip width are multiples of 4; zero: per-
 *                        thread register prefetch. Both give identical results.
 *   LBM_OPT_ROWS2        nonzero (default): the staged FP32 step gives each
 *                        thread two rows of its column per iteration (paired
 *                        FP32 instructions) where it applies (staged, and nx a
 *                        multiple of 4 unless x has pressure columns); zero:
 *                        one row per iteration. Both give identical results.
 *   LBM_OPT_TMA          nonzero (default, contexts and batches):
 *                        the row-pair kernel stages each stencil row with one
 *                        2-D tensor (TMA) load; zero: nine bulk copies per
 *                        row. Identical results.
 *   LBM_OPT_PREFETCH     0..4: the row-pair kernel, where it stages with
 *                        tensor loads, prefetches into L2 the stencil rows
 *                        this many row pairs ahead of the pair it stages into
 *                        shared memory (0 = none). Identical results.
 *   LBM_OPT_GENERAL      nonzero: run the general-geometry kernels even when
 *                        the wall mask adds no solid node (identical
 *                        populations; diagnostic sums to rounding); zero: the
 *                        channel kernels wherever the geometry allows.
 *   LBM_OPT_FAULT_SKIP_COPY  test hook of failure detection, 0 (default) =
 *                        off; for FP32 channels with walls, pressure columns
 *                        and nx a multiple of 4 (LBM_ERR_ARG otherwise), run
 *                        through a separate test build of the step kernel.
 *                        Nonzero: the FP32 row-pair step's first CTA never
 *                        issues the shared-memory copy of the final stencil-row
 *                        pair of its last segment, and every stage wait polls
 *                        at most 4096 times; the wait for that pair gives up
 *                        and a later lbm_step reports LBM_ERR_TIMEOUT (no copy
 *                        reuses that slot afterwards, so none is in flight when
 *                        the CTA exits). The state is then invalid;
 *                        lbm_restore recovers. */
typedef enum {
    LBM_OPT_CTAS_PER_SM = 1,
    LBM_OPT_REVERSE = 2,
    LBM_OPT_STRIP = 3,
    LBM_OPT_STAGED = 4,
    LBM_OPT_GRAPH_STEPS = 5, /* steps per CUDA graph replay (even, 0 = no graph; default 64); contexts
                                replay only on a stream of their own (not the legacy default stream) */
    LBM_OPT_ROWS2 = 6,
    LBM_OPT_TMA = 7,
    LBM_OPT_PREFETCH = 8,
    LBM_OPT_GENERAL = 9,
    LBM_OPT_FAULT_SKIP_COPY = 10,
    LBM_OPT_PERSISTENT = 11, /* batches only, see lbm_batch_step */
    LBM_OPT_BAND = 12,       /* batches only: the work order. -1 (default): one CTA per strip
                                column of every channel, tallest first (the hardware scheduler
                                balances them; with fewer columns than resident CTA slots each
                                column is cut into that many equal pieces); 0: the strip-by-strip order cut into equal runs,
                                one per resident CTA (used whenever LBM_OPT_PERSISTENT is set);
                                > 0: each channel cut into bands of that many rows (at least 8),
                                band by band and, within a band, strip by strip, cut likewise.
                                Identical results. */
    LBM_OPT_PDL = 13,        /* contexts: nonzero (default) launches the FP32 row-pair step with
                                programmatic stream serialization where the plan gives CTAs short
                                segments (under 128 rows each), so a step's launch and set-up
                                overlap the previous step's tail (the kernel waits for the previous
                                grid before any memory access); zero: plain launches. Identical
                                results. */
    LBM_OPT_TILE = 14        /* contexts: nonzero steps FP32 grids whose plan gives CTAs short
                                segments (under 128 rows each) with one CTA per 32 x 8 tile that
                                stages all its stencil rows at once, where the geometry allows
                                (tensor loads, at most 8192 tiles, with walls no tile boundary
                                between rows ny-3 | ny-2, with pressure columns nx % 32 != 1);
                                zero (default, faster on GB300): the row-pair kernel. Identical
                                results. */
} lbm_option;
lbm_status lbm_set_option(lbm_ctx *ctx, lbm_option opt, int64_t value);
/* Launch geometry of the step kernel: CTAs, threads per CTA, work units and
 * whether the staged variant runs. Any output may be NULL. */
lbm_status lbm_launch_info(const lbm_ctx *ctx, int64_t *ctas, int64_t *threads, int64_t *units,
                           int64_t *staged);

/* One time step from f_in to f_out without allocating any device memory.
 * No counterpart in the paper: this is a deployment form of lbm_step for
 * callers that cannot call cudaMalloc where they step: code running inside
 * another framework's memory pool (a raw allocation would bypass the pool's
 * accounting and limits), or a host that sizes every device buffer up front.
 * The collision is always BGK (the lbm_init default); MRT needs a context.
 *   grid, eos, tau, wetting, drive: as for lbm_init (drive may be NULL).
 *   f_in, f_out: distinct caller-owned device arrays of 9*nx*ny values of the
 *            grid precision in the library's row-interleaved layout f[y][i][x]
 *            (index (9*y + i)*nx + x), each aligned to its element size
 *            (LBM_ERR_ARG otherwise). Buffers that start on a 16-byte boundary
 *            (and nx a multiple of 4) take the staged kernels; others take
 *            the register-prefetch kernel, with identical results.
 *            f_out receives the next state; slots no population reaches
 *            (solid rows, the inflow slots of pressure columns) are left
 *            untouched, so initialise f_out from f_in if those must be defined.
 *   ctas:    CTAs of the step grid, 0 = as lbm_step chooses; at most 4096.
 *   diag_out: NULL or a device array of 7 doubles (8-byte aligned) receiving,
 *            for the state f_in: mass, wall-shear sum, tau_w min/max,
 *            p_w min/max, and the error word of the step (below).
 *   err_out: NULL or a device int32 receiving the error word of the step:
 *            bit 0 = a bad (non-finite or non-positive) density was met,
 *            bit 1 = a bounded wait for a staged population row gave up
 *            (f_out is then not valid). Written asynchronously on `stream`.
 *   stream:  cudaStream_t (NULL = legacy default stream); the call only
 *            enqueues work and does not synchronise.
 * Scratch: the per-CTA partials and the error word live in one static device
 * array (about 192 KB) that the library holds on every device it is used on
 * until the process exits. Every call reuses and first clears it, so calls
 * whose work overlaps on the GPU (for instance on different streams) race on
 * it; serialise them. The first call on a device resolves the array's device
 * address (cudaGetSymbolAddress) and should come before any stream capture.
 * Errors: LBM_ERR_ARG (bad grid or 9*pitch*ny >= 2^31, NULL, equal or
 * misaligned buffers, ctas outside 0..4096), LBM_ERR_PARAM, LBM_ERR_CUDA. */
lbm_status lbm_step_noalloc(const lbm_grid *grid, const lbm_eos *eos, double tau, double wetting,
                            const lbm_drive *drive, const void *f_in, void *f_out, int64_t ctas,
                            double *diag_out, int32_t *err_out, void *stream);

/* Release everything the library allocated. NULL-safe. */
void lbm_free(lbm_ctx *ctx);

const char *lbm_status_string(lbm_status s);
const char *lbm_last_error(const lbm_ctx *ctx);

/* Batched channels -----------------------------------------------------------
 * Many independent channels (the parameter sweeps of Sec. 3.3, Figs. 10-12:
 * pressure drop, plug length and film thickness varied per channel) stepped
 * together: one kernel launch per step covers every channel, the launches are
 * replayed from a CUDA graph, and the work of all channels is split evenly over
 * the CTAs. Each channel evolves bit for bit as it would in its own context.
 * All channels share the EOS, tau, wetting, precision and boundary kinds
 * (walls, bc_x); sizes, drives and initial densities differ. */
typedef struct lbm_batch lbm_batch; /* opaque, owned by the library */

/* n channels: grids[n] (same precision / walls / bc_x), drives[n] (may be
 * NULL), rho0s[n] host arrays of nx*ny doubles. stream: cudaStream_t or NULL
 * (the batch then creates its own non-blocking stream; graphs need a
 * non-default stream). The library allocates the packed population buffers.
 * Errors: LBM_ERR_ARG, LBM_ERR_PARAM, LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_batch_init(int32_t n, const lbm_grid *grids, const lbm_eos *eos, double tau, double wetting,
                          const lbm_drive *drives, const double *const *rho0s, void *stream, lbm_batch **out);
/* Advance every channel n steps (asynchronous): one launch per step,
 * replayed from CUDA graphs of LBM_OPT_GRAPH_STEPS steps (default 64). With
 * LBM_OPT_PERSISTENT = 1, row-pair (FP32, staged) batches run persistently
 * instead: one cooperative launch carries up to 4096 steps, every segment
 * (channel, strip, rows) waiting, bounded, for the step counters of the
 * segments next to it before each step; a wait that gives up reports
 * LBM_ERR_TIMEOUT. Identical results either way. */
lbm_status lbm_batch_step(lbm_batch *b, int64_t n);
/* Per-channel outputs, as lbm_fields / lbm_diag / lbm_populations. */
lbm_status lbm_batch_fields(lbm_batch *b, int32_t channel, void *rho, void *ux, void *uy, void *tau_wall,
                            void *p_wall);
lbm_status lbm_batch_diag(lbm_batch *b, int32_t channel, lbm_diag_t *out);
lbm_status lbm_batch_populations(lbm_batch *b, int32_t channel, void *dst);
/* As lbm_reset_diag, for every channel. */
lbm_status lbm_batch_reset_diag(lbm_batch *b);
/* Collision operator of every channel, as lbm_set_collision (NULL: BGK). */
lbm_status lbm_batch_set_collision(lbm_batch *b, const lbm_collision *c);
/* Options as lbm_set_option plus LBM_OPT_GRAPH_STEPS. Changing the launch
 * plan resets the diagnostic accumulators. */
lbm_status lbm_batch_set_option(lbm_batch *b, lbm_option opt, int64_t value);
lbm_status lbm_batch_launch_info(const lbm_batch *b, int64_t *ctas, int64_t *segments, int64_t *staged,
                                 int64_t *strip);
/* Autotuner: times trial_steps steps for each candidate launch plan (CTAs
 * per SM, strip width) on a saved copy of the state, keeps the fastest,
 * restores the state and returns the choice. With the whole-column work
 * order (LBM_OPT_BAND = -1, not persistent) only the strip width is tried
 * and best_ctas_per_sm returns the resident occupancy. Resets the
 * diagnostic accumulators. */
lbm_status lbm_batch_autotune(lbm_batch *b, int32_t trial_steps, int64_t *best_ctas_per_sm,
                              int64_t *best_strip, double *best_ms_per_step);
const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_free(lbm_batch *b); /* NULL-safe */

/* Host helpers (FP64, no GPU needed) ---------------------------------------*/

/* Critical point, Maxwell coexistence (equal pressure and chemical
 * potential, Sec. 2.1 "Verification") and saturation pressure at
 * T = T_over_Tc * Tc. LBM_ERR_PARAM above Tc. Any output may be NULL. */
lbm_status lbm_coexistence(const lbm_eos *eos, double *Tc, double *rho_g, double *rho_l,
                           double *p_sat);

/* The method's own coexistence (Sec. 2.1 "Verification": the densities a flat
 * interface relaxes to, which at lattice interface widths differ from
 * Maxwell's): a liquid slab between rows ny/4 and 3ny/4 of a periodic 4 x ny
 * box, started from the Maxwell densities (tanh profile, width 4), stepped
 * `steps` times on the current device with this EOS, tau and collision (NULL:
 * BGK) at `precision` (32 or 64). Returns the bulk densities (rows 0 and
 * ny/2) and their mesh pressures k^2 p0(rho), which agree once the slab has
 * settled (equal mechanical pressure across a flat interface); *p_gas is the
 * reference pressure at which a pressure column holds the method's own
 * saturated vapour. Any output may be NULL. Synchronises `stream` (NULL:
 * legacy default stream); allocates and frees a context of its own.
 * Errors: LBM_ERR_ARG (ny < 16, steps < 0, bad precision), LBM_ERR_PARAM
 * (T >= Tc or as lbm_init), LBM_ERR_NAN, LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_relaxed_coexistence(const lbm_eos *eos, double tau, const lbm_collision *coll, int32_t precision,
                                   int32_t ny, int64_t steps, void *stream, double *rho_g, double *rho_l,
                                   double *p_gas, double *p_liq);

/* Initial density of the airway channel (Sec. 2.2, Fig. 2): wall films of
 * thickness `film` measured from the half-way wall planes and a plug
 * covering x in [plug_x, plug_x + plug_len), smooth tanh profiles of width
 * `width`; plus uniform noise amp*(2u - 1), u from SplitMix64(seed ^ node).
 * out: host array of nx*ny doubles. */
lbm_status lbm_airway_rho0(int32_t nx, int32_t ny, double film, double plug_x, double plug_len,
                           double rho_l, double rho_g, double width, double noise_amp,
                           uint64_t seed, double *out);

/* Partial derivatives of the noise-free airway profile of lbm_airway_rho0
 * with respect to the film thickness and the plug length:
 * d_film = (rho_l - rho_g) dS/dfilm, d_plug = (rho_l - rho_g) dS/dplug_len,
 * with S = max(s_film, s_plug) differentiated along the larger profile (the
 * film where they tie). Outputs: host arrays of nx*ny doubles (either may be
 * NULL). Errors: LBM_ERR_ARG. */
lbm_status lbm_airway_rho0_tangent(int32_t nx, int32_t ny, double film, double plug_x, double plug_len,
                                   double rho_l, double rho_g, double width, double *d_film,
                                   double *d_plug);

/* Initial density of a liquid disk of radius r0 centred at (cx, cy). */
lbm_status lbm_disk_rho0(int32_t nx, int32_t ny, double cx, double cy, double r0, double rho_l,
                         double rho_g, double width, double noise_amp, uint64_t seed, double *out);

/* Liquid-plug analysis of a density field (Sec. 3: plug interfaces, rupture
 * and aerosol formation, Figs. 4, 7, 10-12), for a channel with walls at rows
 * 0 and ny-1. A node is liquid when rho > rho_mid (use (rho_l + rho_g)/2).
 *   x_rear, x_front: ends of the longest liquid run on the centre row
 *       ny/2, interpolated linearly to rho_mid (NaN if the row has no liquid);
 *   intact: 1 while some column is liquid on every fluid row (the plug still
 *       closes the channel), 0 after rupture;
 *   n_droplets, droplet_mass: liquid components (4-connected) that touch
 *       neither first fluid row - droplets detached from the wall films
 *       (aerosol) - and the sum of rho over them;
 *   wall_liquid_mass: sum of rho over liquid components touching a wall row.
 * rho: host array nx*ny (solid rows ignored). Errors: LBM_ERR_ARG. */
typedef struct {
    double x_rear, x_front;
    int32_t intact;
    int32_t n_droplets;
    double droplet_mass;
    double wall_liquid_mass;
} lbm_plug_state;
lbm_status lbm_plug_analysis(int32_t nx, int32_t ny, const double *rho, double rho_mid, lbm_plug_state *out);

/* ------------------------------------------------------------------------ */
/* Discrete adjoint                                                          */
/* ------------------------------------------------------------------------ */
/* Gradients of the time-integrated wall loads of Sec. 3 (Figs. 10-12),
 * summed over the states n = 0 .. nsteps-1 that nsteps steps read and over the
 * interior columns of both walls:
 *   J[0] = J_tau = sum_n sum_x tau_w,   J[1] = J_p = sum_n sum_x p_w,
 * tau_w and p_w as lbm_fields reports them (p_w: Eq. 2.4). The adjoint is the
 * exact transpose of the linearised step of lbm_step (a pressure column's
 * clamped phase weight contributes no derivative), run backwards over blocks
 * of block_steps steps recomputed from checkpoints kept in device memory
 * (one state, 9 pitch ny values of the forward precision with pitch = nx
 * rounded up to a multiple of 4, per checkpoint: ceil(nsteps/K) checkpoints
 * plus K states of one block; K = block_steps, or ceil(sqrt(nsteps)) if 0).
 *
 * lbm_adjoint_init: grid->precision is the precision of the forward steps and
 *   checkpoints, 64 or 32 (LBM_ERR_ARG otherwise); the reverse sweep is FP64
 *   unless lbm_adjoint_set_precision says otherwise, on the stored states
 *   widened to FP64, so with 32 the result is the gradient of the FP64 step
 *   along the FP32 trajectory. nsteps >= 1.
 *   Allocates on the current device; stream as in lbm_init.
 * lbm_adjoint_forward: runs nsteps steps from f0 = f_eq(rho0, 0) under
 *   `drive` (NULL: no drive), keeping checkpoints, and returns J (host,
 *   2 doubles). rho0: nx*ny doubles, host or device. Synchronises the stream.
 *   LBM_ERR_NAN if a step met a bad density; LBM_ERR_PARAM as lbm_init.
 * lbm_adjoint_backward: gradients of w_tau J_tau + w_p J_p for the last
 *   forward: grad_rho0 (nx*ny doubles, host or device) and grad_drive (host,
 *   3 doubles: d/d dp, d/d gx, d/d gy; dp enters through the pressure-column
 *   densities, which are EOS roots at p_ref +- dp/2). May be called several
 *   times after one forward. LBM_ERR_STATE before any forward.
 * The handle owns all its memory; lbm_adjoint_free is NULL-safe. */
typedef struct lbm_adjoint lbm_adjoint;
lbm_status lbm_adjoint_init(const lbm_grid *grid, const lbm_eos *eos, double tau, double wetting,
                            int64_t nsteps, int64_t block_steps, void *stream, lbm_adjoint **out);
lbm_status lbm_adjoint_forward(lbm_adjoint *adj, const lbm_drive *drive, const double *rho0, double *J);
lbm_status lbm_adjoint_backward(lbm_adjoint *adj, double w_tau, double w_p, double *grad_rho0,
                                double *grad_drive);
/* Collision operator of the differentiated step, as lbm_set_collision (NULL:
 * BGK); the MRT relaxation is symmetric, so its transpose is itself. Takes
 * effect at the next forward; a backward before that forward returns
 * LBM_ERR_STATE. Errors: LBM_ERR_ARG as lbm_set_collision. */
lbm_status lbm_adjoint_set_collision(lbm_adjoint *adj, const lbm_collision *c);
/* Arithmetic of the reverse sweep and of the objective's per-node terms:
 * 64 (the default) or 32. With 32 the fields recomputed from each stored
 * state, the adjoint populations and the per-step terms are FP32, on the FP32
 * pipes; the sums over steps and nodes (J, dJ/d dp, dJ/dG) and grad_rho0 stay
 * FP64. Meant for an FP32 forward whose gradients are wanted to a relative
 * 1e-3 or so (FP32 rounding compounds over the reverse steps). Takes effect at
 * the next forward or backward. Errors: LBM_ERR_ARG (adj NULL, or not 32/64). */
lbm_status lbm_adjoint_set_precision(lbm_adjoint *adj, int32_t reverse_precision);
const char *lbm_adjoint_last_error(const lbm_adjoint *adj);
void lbm_adjoint_free(lbm_adjoint *adj);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
