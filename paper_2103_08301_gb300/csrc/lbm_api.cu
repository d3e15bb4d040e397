// C ABI of the GB300 EOS-multiphase lattice Boltzmann solver (see include/lbm.h).
// Host orchestration only: argument checks, thermodynamic set-up in FP64,
// device workspace, kernel launches on the context stream, diagnostics and
// checkpoints. Every step of the method runs in the kernels of lbm_kernels.cuh.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled (fetched at run time; no link to the driver library)

#include <mutex>
#include <vector>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"
#include "lbm_tile.cuh"

namespace {

constexpr int STRIP = lbm::STRIP;  // widest strip (columns per CTA)
// threads per CTA of the step kernels of a precision and staging choice
inline int cta_threads(int precision, bool staged)
{
    if (precision == 64) return staged ? lbm::threads_per_cta<double, true>() : lbm::threads_per_cta<double, false>();
    return staged ? lbm::threads_per_cta<float, true>() : lbm::threads_per_cta<float, false>();
}
constexpr size_t ALIGN = 256;
constexpr uint64_t CKPT_MAGIC = 0x4C424D434B505431ull;  // "LBMCKPT1"

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

// Host-side fault injection for the failure-detection tests (read at every
// lbm_init): LBM_FAULT=alloc fails lbm_init as if its last device allocation
// had failed, after the workspace was allocated, so the error path's clean-up
// runs; LBM_FAULT=param fails it as if the thermodynamics had no solution.
// CTAs whose share of the work is under this many rows per strip take the
// row-pair kernel that issues a segment's first three stage pairs together
// (measured: 4096 x 512 +8.6%, 1024 x 128 +6%; 16384 x 2048, ~358 rows per
// CTA, 0.9% slower with it)
constexpr long long EARLY_ROWS = 128;

bool fault_is(const char *kind)
{
    const char *f = std::getenv("LBM_FAULT");
    return f && std::strcmp(f, kind) == 0;
}

struct Layout {
    size_t pops;      // one population array
    size_t f0, f1, mass, J, ext, err, dout, total;
    size_t rho, side;  // in-place contexts: density plane and pressure-column side buffer
};

// inplace: one population array (f1 = f0) plus the density plane and the side
// buffer of the in-place step
Layout layout_of(int nx, int ny, int precision, bool inplace = false)
{
    Layout L{};
    const size_t sz = precision == 64 ? 8 : 4;
    L.pops = align_up((size_t)9 * lbm::pitch_of(nx) * ny * sz);
    size_t o = 0;
    L.f0 = o; o += L.pops;
    if (inplace) {
        L.f1 = L.f0;
        L.rho = o; o += align_up((size_t)lbm::pitch_of(nx) * ny * sz);
        L.side = o; o += align_up((size_t)2 * 9 * ny * sz);
    } else {
        L.f1 = o; o += L.pops;
    }
    L.mass = o; o += align_up(lbm::MAX_CTAS * sizeof(double));
    L.J = o; o += align_up(lbm::MAX_CTAS * sizeof(double));
    L.ext = o; o += align_up((size_t)lbm::MAX_CTAS * 4 * sz);
    L.err = o; o += align_up(sizeof(int));
    L.dout = o; o += align_up(8 * sizeof(double));
    L.total = o;
    return L;
}

// big: a context may take 64-bit population offsets (node indices, and the
// 9 ny plane-rows of a tensor map, stay below 2^31); otherwise 9 pitch ny < 2^31.
bool grid_ok(const lbm_grid *g, bool big = false)
{
    if (!g) return false;
    if (g->precision != 32 && g->precision != 64) return false;
    if (g->walls != 0 && g->walls != 1) return false;
    if (g->bc_x != 0 && g->bc_x != 1) return false;
    if (g->nx < (g->bc_x ? 4 : 1) || g->ny < (g->walls ? 4 : 1)) return false;
    if (big) return (long long)lbm::pitch_of(g->nx) * g->ny < (1ll << 31) && 9ll * g->ny < (1ll << 31);
    return lbm::idx32_ok(g->nx, g->ny);
}

} // namespace

struct lbm_ctx {
    lbm_grid grid{};
    lbm_eos eos{};
    lbm_drive drive{};
    double tau = 1.0, wet = 0.0;
    double T = 0, Tc = 0, rho_g = 0, rho_l = 0, p_sat = 0, rho_in = 0, rho_out = 0;
    double rho_in_l = 0, rho_out_l = 0;
    lbm::Thermo th{};  // EOS at the working temperature
    lbm_collision coll{};  // BGK unless lbm_set_collision chose MRT
    cudaStream_t stream = nullptr;
    unsigned char *ws = nullptr;
    bool own_ws = false;
    Layout L{};
    int cur = 0;          // which population array holds the current state
    // in-place streaming (lbm_init_inplace): one population array, cur = 0;
    // aa_odd: the array holds the odd-parity layout (after an odd number of
    // in-place steps since it last held the natural one)
    bool inplace = false, aa_odd = false;
    lbm::AAPlan aa{};
    int64_t step = 0;
    int W = STRIP, nstrips = 0, yf0 = 0, nyf = 0;
    int W_opt = 0;  // LBM_OPT_STRIP (0: widest)
    int pitch = 0;  // plane pitch of the population rows (>= nx)
    bool big = false;  // 9 pitch ny >= 2^31: kernels with 64-bit population offsets
    bool early = false;  // row-pair kernel issuing a segment's first three stage pairs together
    bool pdl = true;     // LBM_OPT_PDL: row-pair steps launched with programmatic serialization
    long long units = 0;
    int band = 0;  // rows per band of the work-unit order
    int nctas = 0;
    int ctas_per_sm_opt = 0;
    int reverse = 0;
    int sms = 0;
    bool allow_staged = true;  // LBM_OPT_STAGED
    bool staged = false;       // bulk-copy staged kernel selected for this grid
    bool allow_rows2 = true;   // LBM_OPT_ROWS2
    bool rows2 = false;        // row-pair FP32 step kernel selected for this grid
    bool allow_tma = true;     // LBM_OPT_TMA
    int pf = 0;                // LBM_OPT_PREFETCH (row pairs ahead, 0 = off)
    // general wall geometry (lbm_mask.cu): set when the mask adds solid nodes
    // to the wall rows, or when LBM_OPT_GENERAL forces that path
    lbm::MaskPath *mask = nullptr;
    std::vector<uint8_t> mask_host;  // the caller's mask (empty: none)
    bool force_general = false;
    bool fault_skip = false;  // LBM_OPT_FAULT_SKIP_COPY (test hook)
    // graph replay of lbm_step: graph_steps launches captured from buffer 0
    // (contexts with a stream of their own; LBM_OPT_GRAPH_STEPS)
    int graph_steps = 64;
    cudaGraphExec_t graph = nullptr;
    bool tma_ok = false;       // tmap[] encoded (FP32, pitch a multiple of 4)
    CUtensorMap tmap[2];       // 2-D views of the two population buffers for the row-pair stage
    bool tile_maps_ok = false;  // tmap_tile[] encoded
    CUtensorMap tmap_tile[2];   // the same views with the tile kernel's boxes (T_BOX x 9)
    bool allow_tile = false;    // LBM_OPT_TILE (measured slower than the row-pair kernel)
    bool tile = false;          // the plan steps with step_kernel_tile (ntx tiles along x)
    int ntx = 0;
    // fields scratch (allocated on first host-pointer lbm_fields)
    unsigned char *fscratch = nullptr;
    // non-blocking NaN check
    int *h_err = nullptr;
    cudaEvent_t err_ev = nullptr;
    bool err_pending = false;
    char last_error[512] = {0};
};

namespace {

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *where)
{
    if (c) std::snprintf(c->last_error, sizeof c->last_error, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define CK(call, where)                                            \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);   \
    } while (0)

template <typename real>
lbm::KArgs<real> make_args(const lbm_ctx *ctx)
{
    lbm::KArgs<real> A{};
    const int src = ctx->cur, dst = 1 - ctx->cur;
    A.fin = (const real *)(ctx->ws + (src ? ctx->L.f1 : ctx->L.f0));
    A.fout = (real *)(ctx->ws + (dst ? ctx->L.f1 : ctx->L.f0));
    A.plane = (long long)ctx->grid.nx * ctx->grid.ny;
    A.nx = ctx->grid.nx;
    A.ny = ctx->grid.ny;
    A.pitch = ctx->pitch;
    A.W = ctx->W;
    A.nstrips = ctx->nstrips;
    A.yf0 = ctx->yf0;
    A.nyf = ctx->nyf;
    A.units = ctx->units;
    A.band = ctx->band;
    A.nctas = ctx->nctas;
    A.reverse = ctx->reverse;
    const double k = ctx->eos.k;
    A.RT = (real)(ctx->eos.R * ctx->T);
    A.a = (real)ctx->eos.a;
    A.b4 = (real)(0.25 * ctx->eos.b);
    A.k2 = (real)(k * k);
    A.kappa = (real)ctx->eos.kappa;
    A.tau = (real)ctx->tau;
    A.inv_tau = (real)(1.0 / ctx->tau);
    A.omb = (real)(1.0 - 1.0 / ctx->tau);
    A.gx = (real)ctx->drive.gx;
    A.gy = (real)ctx->drive.gy;
    A.wet = (real)ctx->wet;
    A.rho_in_g = (real)ctx->rho_in;
    A.rho_in_l = (real)ctx->rho_in_l;
    A.rho_out_g = (real)ctx->rho_out;
    A.rho_out_l = (real)ctx->rho_out_l;
    A.ph_g = (real)ctx->rho_g;
    A.inv_dph = ctx->rho_l > ctx->rho_g ? (real)(1.0 / (ctx->rho_l - ctx->rho_g)) : real(0);
    A.nu = (real)((ctx->tau - 0.5) / 3.0);
    A.eos_kind = ctx->th.kind;
    A.bpr = (real)ctx->th.b;
    A.aalpha = (real)ctx->th.aalpha;
    const lbm_collision &cl = ctx->coll;
    A.mrt = cl.kind == LBM_COLL_MRT;
    A.ushift = A.mrt ? (real)(1.0 / cl.s_j) : (real)ctx->tau;
    if (A.mrt) {
        const double s_nu = cl.s_nu > 0 ? cl.s_nu : 1.0 / ctx->tau;
        A.m_e = (real)(cl.s_e / 36.0); A.m_eps = (real)(cl.s_eps / 36.0);
        A.m_j = (real)(cl.s_j / 6.0); A.m_q = (real)(cl.s_q / 12.0); A.m_nu = (real)(s_nu / 4.0);
    }
    A.mass_part = (double *)(ctx->ws + ctx->L.mass);
    A.J_acc = (double *)(ctx->ws + ctx->L.J);
    A.ext = (real *)(ctx->ws + ctx->L.ext);
    A.err = (int *)(ctx->ws + ctx->L.err);
    return A;
}

template <typename real, int MODE, bool STAGED, bool PADDED>
void *kernel_ptr(bool walls, bool pres)
{
    using namespace lbm;
    if (walls && pres) return (void *)step_kernel<real, true, true, MODE, STAGED, PADDED>;
    if (walls) return (void *)step_kernel<real, true, false, MODE, STAGED, PADDED>;
    if (pres) return (void *)step_kernel<real, false, true, MODE, STAGED, PADDED>;
    return (void *)step_kernel<real, false, false, MODE, STAGED, PADDED>;
}

template <typename real, int MODE>
void *kernel_ptr(bool walls, bool pres, bool staged, bool padded)
{
    if (staged)
        return padded ? kernel_ptr<real, MODE, true, true>(walls, pres) : kernel_ptr<real, MODE, true, false>(walls, pres);
    return padded ? kernel_ptr<real, MODE, false, true>(walls, pres) : kernel_ptr<real, MODE, false, false>(walls, pres);
}

}  // namespace

namespace {
lbm_status aa_natural(lbm_ctx *ctx);
size_t state_bytes(const lbm_ctx *ctx)
{
    return (size_t)9 * ctx->pitch * ctx->grid.ny * (ctx->grid.precision == 64 ? 8 : 4);
}
}  // namespace

cudaError_t lbm_ctx_copy_state(lbm_ctx *ctx, void *dst)
{
    if (aa_natural(ctx) != LBM_OK) return cudaErrorLaunchFailure;
    return cudaMemcpyAsync(dst, ctx->ws + (ctx->cur ? ctx->L.f1 : ctx->L.f0), state_bytes(ctx),
                           cudaMemcpyDeviceToDevice, ctx->stream);
}

const void *lbm_ctx_state(const lbm_ctx *ctx)
{
    if (aa_natural(const_cast<lbm_ctx *>(ctx)) != LBM_OK) return nullptr;
    return ctx->ws + (ctx->cur ? ctx->L.f1 : ctx->L.f0);
}

cudaError_t lbm_ctx_load_state(lbm_ctx *ctx, const void *src)
{
    const size_t bytes = state_bytes(ctx);
    cudaError_t e = cudaMemcpyAsync(ctx->ws + ctx->L.f0, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && !ctx->inplace)
        e = cudaMemcpyAsync(ctx->ws + ctx->L.f1, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    ctx->aa_odd = false;
    return e;
}

void *lbm_step_kernel_ptr(int precision, int mode, bool walls, bool pres, bool staged, bool padded)
{
    if (precision == 64)
        return mode == lbm::MODE_STEP ? kernel_ptr<double, lbm::MODE_STEP>(walls, pres, staged, padded)
                                      : kernel_ptr<double, lbm::MODE_FIELDS>(walls, pres, staged, padded);
    return mode == lbm::MODE_STEP ? kernel_ptr<float, lbm::MODE_STEP>(walls, pres, staged, padded)
                                  : kernel_ptr<float, lbm::MODE_FIELDS>(walls, pres, staged, padded);
}

namespace {

template <bool PADDED, int EARLY>
void *rows2_kernel_ptr(bool walls, bool pres)
{
    using namespace lbm;
    if (walls && pres) return (void *)step_kernel_rows2<true, true, PADDED, false, int, EARLY>;
    if (walls) return (void *)step_kernel_rows2<true, false, PADDED, false, int, EARLY>;
    if (pres) return (void *)step_kernel_rows2<false, true, PADDED, false, int, EARLY>;
    return (void *)step_kernel_rows2<false, false, PADDED, false, int, EARLY>;
}


void *step_kernel_ptr(const lbm_ctx *ctx, int mode)
{
    const bool padded = ctx->pitch != ctx->grid.nx;
    if (ctx->big) {
        if (mode == lbm::MODE_STEP && ctx->rows2)
            return lbm_big_rows2_kernel_ptr(ctx->grid.walls, ctx->grid.bc_x, padded);
        return lbm_big_step_kernel_ptr(ctx->grid.precision, mode, ctx->grid.walls, ctx->grid.bc_x, ctx->staged,
                                       padded);
    }
    if (mode == lbm::MODE_STEP && ctx->rows2) {
        if (ctx->early)
            return padded ? rows2_kernel_ptr<true, 3>(ctx->grid.walls, ctx->grid.bc_x)
                          : rows2_kernel_ptr<false, 3>(ctx->grid.walls, ctx->grid.bc_x);
        return padded ? rows2_kernel_ptr<true, 1>(ctx->grid.walls, ctx->grid.bc_x)
                      : rows2_kernel_ptr<false, 1>(ctx->grid.walls, ctx->grid.bc_x);
    }
    return lbm_step_kernel_ptr(ctx->grid.precision, mode, ctx->grid.walls, ctx->grid.bc_x, ctx->staged, padded);
}

size_t dyn_smem(const lbm_ctx *ctx, int mode)
{
    if (!ctx->staged) return 0;
    if (mode == lbm::MODE_STEP && ctx->rows2) return lbm::rows2_smem_bytes();
    return ctx->grid.precision == 64 ? lbm::staged_smem_bytes<double>()
                                     : lbm::staged_smem_bytes<float>();
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    static std::mutex m;
    std::lock_guard<std::mutex> lock(m);
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// The 2-D view of one FP32 population buffer that the row-pair stage reads:
// x = column (pitch wide, stride 4 pitch bytes per y), y = 9 * row + plane;
// boxes of R2_SP columns by 9 planes (one stencil row), zero fill outside.
bool encode_population_map(CUtensorMap *map, void *base, int pitch, int ny, int box_cols = lbm::R2_SP)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || pitch % 4 != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)9 * (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, 9u};
    const cuuint32_t elem[2] = {1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int threads_of(const lbm_ctx *ctx, int mode)
{
    if (mode == lbm::MODE_STEP && ctx->rows2) return lbm::R2_BLOCK;
    return cta_threads(ctx->grid.precision, ctx->staged);
}

// Band height of the work-unit order: about one CTA's share of rows, so that
// consecutive CTAs hold neighbouring strips of one band (at least 8 rows; the
// whole column, i.e. strip-major order, when there are fewer CTAs than
// strips). With walls no band boundary may fall between fluid rows 1|2 or
// ny-3|ny-2 (fluid offsets 1 and nyf-1).
int band_rows(int nyf, int nstrips, int nctas, int walls)
{
    const long long share = ((long long)nyf * nstrips + nctas - 1) / nctas;
    int band = (int)std::min<long long>(nyf, std::max<long long>(8, share));
    if (walls)
        while (band < nyf && (nyf - 1) % band == 0) ++band;
    return std::max(1, band);
}

// Strip partition and the CTA count of the step grid.
lbm_status plan_launch(lbm_ctx *ctx)
{
    const int nx = ctx->grid.nx;
    const int wmax = std::min(ctx->W_opt > 0 ? ctx->W_opt : STRIP, STRIP);
    int W = lbm::strip_width(nx, wmax, ctx->grid.bc_x);
    // bulk-copy staging needs 16-byte aligned row segments
    ctx->staged = ctx->allow_staged && (ctx->pitch % 4 == 0) && (W % 4 == 0);
    // row pairs: FP32 staged grids with strips of at most R2_W columns (a
    // multiple of 4); with periodic x the wrapped halo columns are copied as
    // one 16-byte group, which needs nx a multiple of 4
    ctx->rows2 = ctx->allow_rows2 && ctx->staged && ctx->grid.precision == 32 &&
                 lbm::cols_per_thread<float, true>() == 1 && (ctx->grid.bc_x || nx % 4 == 0);
    if (ctx->rows2) {
        const int W2 = lbm::strip_width(nx, std::min(wmax, lbm::R2_W), ctx->grid.bc_x);
        if (W2 % 4 == 0) W = W2;
        else ctx->rows2 = false;
    }
    ctx->W = W;
    ctx->nstrips = (nx + W - 1) / W;
    ctx->yf0 = ctx->grid.walls ? 1 : 0;
    ctx->nyf = ctx->grid.walls ? ctx->grid.ny - 2 : ctx->grid.ny;
    ctx->units = (long long)ctx->nstrips * ctx->nyf;
    ctx->early = false;  // chosen once the CTA count is known

    for (int mode : {lbm::MODE_STEP, lbm::MODE_FIELDS}) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel_ptr(ctx, mode),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)dyn_smem(ctx, mode));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "smem attribute");
    }
    int per_sm = ctx->ctas_per_sm_opt;
    if (per_sm <= 0) {
        int occ = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, step_kernel_ptr(ctx, lbm::MODE_STEP), threads_of(ctx, lbm::MODE_STEP),
            dyn_smem(ctx, lbm::MODE_STEP));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy");
        per_sm = std::max(1, occ);
    }
    long long n = (long long)ctx->sms * per_sm;
    n = std::min<long long>(n, std::max<long long>(1, ctx->units / 2));
    n = std::min<long long>(n, lbm::MAX_CTAS);
    ctx->nctas = (int)std::max<long long>(1, n);
    ctx->band = band_rows(ctx->nyf, ctx->nstrips, ctx->nctas, ctx->grid.walls);
    if (ctx->rows2 && !ctx->big && ctx->units < EARLY_ROWS * ctx->nctas) {
        ctx->early = true;
        cudaError_t e = cudaFuncSetAttribute(step_kernel_ptr(ctx, lbm::MODE_STEP),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)dyn_smem(ctx, lbm::MODE_STEP));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "smem attribute");
    }
    // short segments with tensor-load staging: one CTA per 32 x 8 tile instead
    // (no tile boundary between the wall-shear rows ny-3 | ny-2, and the
    // outlet column never alone in a tile: its stencil reaches two columns back)
    ctx->tile = false;
    if (ctx->early && ctx->allow_tile && ctx->tile_maps_ok && ctx->allow_tma && !ctx->fault_skip) {
        const int nx = ctx->grid.nx;
        const long long ntx = (nx + lbm::T_TX - 1) / lbm::T_TX, nty = (ctx->nyf + lbm::T_TY - 1) / lbm::T_TY;
        bool ok = ntx * nty <= lbm::MAX_CTAS;
        if (ctx->grid.walls) ok = ok && (ctx->nyf - 1) % lbm::T_TY != 0;
        if (ctx->grid.bc_x) ok = ok && nx % lbm::T_TX != 1;
        if (ok) {
            void *fn = ctx->grid.walls ? (ctx->grid.bc_x ? (void *)lbm::step_kernel_tile<true, true>
                                                         : (void *)lbm::step_kernel_tile<true, false>)
                                       : (ctx->grid.bc_x ? (void *)lbm::step_kernel_tile<false, true>
                                                         : (void *)lbm::step_kernel_tile<false, false>);
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)lbm::tile_smem_bytes());
            if (e != cudaSuccess) return cuda_fail(ctx, e, "smem attribute");
            ctx->tile = true;
            ctx->ntx = (int)ntx;
            ctx->nctas = (int)(ntx * nty);
        }
    }
    return LBM_OK;
}

template <typename real, int MODE>
cudaError_t launch(lbm_ctx *ctx, const lbm::KArgs<real> &A)
{
    void *fn = step_kernel_ptr(ctx, MODE);
    if (MODE == lbm::MODE_STEP && ctx->tile) {
        // one CTA per 32 x 8 tile, every stencil row staged by a tensor load
        lbm::KArgs<real> B = A;
        fn = ctx->grid.walls ? (ctx->grid.bc_x ? (void *)lbm::step_kernel_tile<true, true>
                                               : (void *)lbm::step_kernel_tile<true, false>)
                             : (ctx->grid.bc_x ? (void *)lbm::step_kernel_tile<false, true>
                                               : (void *)lbm::step_kernel_tile<false, false>);
        int ntx = ctx->ntx;
        void *args[] = {(void *)&B, (void *)&ctx->tmap_tile[ctx->cur], (void *)&ntx};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(ctx->nctas);
        cfg.blockDim = dim3(lbm::T_THREADS);
        cfg.dynamicSmemBytes = lbm::tile_smem_bytes();
        cfg.stream = ctx->stream;
        cfg.attrs = at;
        cfg.numAttrs = ctx->pdl ? 1 : 0;
        return cudaLaunchKernelExC(&cfg, fn, args);
    }
    if (MODE == lbm::MODE_STEP && ctx->rows2) {
        // the row-pair kernel also takes the tensor map of its source buffer
        static const CUtensorMap unused{};
        lbm::KArgs<real> B = A;
        B.tma = ctx->tma_ok && ctx->allow_tma;
        B.pf = ctx->pf;
        if (ctx->fault_skip) {
            B.poll_limit = 4096;
            fn = (void *)lbm::step_kernel_rows2<true, true, false, true>;
        }
        const CUtensorMap *m = B.tma ? &ctx->tmap[ctx->cur] : &unused;
        void *args[] = {(void *)&B, (void *)m};
        if (ctx->pdl && ctx->early && !ctx->fault_skip) {
            // programmatic dependent launch: the kernel waits for the previous
            // grid before touching memory, so its launch and set-up overlap
            // the previous step's tail (short-segment plans: config 2 +2.9%;
            // the benchmark channel measured 0.1% slower with it)
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(ctx->nctas);
            cfg.blockDim = dim3(threads_of(ctx, MODE));
            cfg.dynamicSmemBytes = dyn_smem(ctx, MODE);
            cfg.stream = ctx->stream;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            return cudaLaunchKernelExC(&cfg, fn, args);
        }
        return cudaLaunchKernel(fn, dim3(ctx->nctas), dim3(threads_of(ctx, MODE)), args, dyn_smem(ctx, MODE),
                                ctx->stream);
    }
    void *args[] = {(void *)&A};
    return cudaLaunchKernel(fn, dim3(ctx->nctas), dim3(threads_of(ctx, MODE)), args, dyn_smem(ctx, MODE),
                            ctx->stream);
}

void drop_graph(lbm_ctx *ctx)
{
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
}

template <typename real>
lbm_status do_steps(lbm_ctx *ctx, int64_t n);

// graph_steps steps starting from buffer 0, captured once and replayed (the
// captured launches hold the kernel arguments of that moment: any change of
// plan, option or collision drops the graph)
template <typename real>
lbm_status build_graph(lbm_ctx *ctx)
{
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    const int cur0 = ctx->cur;
    const bool odd0 = ctx->aa_odd;
    const int64_t step0 = ctx->step;
    const int keep = ctx->graph_steps;
    ctx->graph_steps = 0;  // capture single launches
    lbm_status st = do_steps<real>(ctx, keep);
    ctx->graph_steps = keep;
    cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
    ctx->cur = cur0;  // capture records; nothing ran
    ctx->aa_odd = odd0;
    ctx->step = step0;
    if (st != LBM_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "graph end capture");
    cudaError_t e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { ctx->graph = nullptr; return cuda_fail(ctx, e, "graph instantiate"); }
    return LBM_OK;
}

// the phase lbm_step's graphs start from: buffer 0, or for in-place
// contexts the natural layout
int phase_of(const lbm_ctx *ctx) { return ctx->inplace ? (ctx->aa_odd ? 1 : 0) : ctx->cur; }

template <typename real>
lbm_status one_step(lbm_ctx *ctx)
{
    lbm::KArgs<real> A = make_args<real>(ctx);
    if (ctx->inplace) {
        cudaError_t e = lbm::aa_step<real>(A, (real *)(ctx->ws + ctx->L.f0), (real *)(ctx->ws + ctx->L.rho),
                                           (real *)(ctx->ws + ctx->L.side), ctx->grid.walls, ctx->grid.bc_x,
                                           ctx->aa_odd, ctx->big, ctx->aa, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "in-place step launch");
        ctx->aa_odd = !ctx->aa_odd;
        ctx->step += 1;
        return LBM_OK;
    }
    cudaError_t e = ctx->mask ? lbm::mask_launch<real>(ctx->mask, A, lbm::MODE_STEP, ctx->stream)
                              : launch<real, lbm::MODE_STEP>(ctx, A);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "step launch");
    ctx->cur = 1 - ctx->cur;
    ctx->step += 1;
    return LBM_OK;
}

template <typename real>
lbm_status do_steps(lbm_ctx *ctx, int64_t n)
{
    // the graph starts from buffer 0: a run that starts from buffer 1 takes one
    // single launch first
    if (ctx->graph_steps > 0 && ctx->stream && phase_of(ctx) == 1 && n > ctx->graph_steps) {
        lbm_status s = one_step<real>(ctx);
        if (s != LBM_OK) return s;
        --n;
    }
    while (ctx->graph_steps > 0 && ctx->stream && n >= ctx->graph_steps && phase_of(ctx) == 0) {
        if (!ctx->graph) {
            lbm_status s = build_graph<real>(ctx);
            if (s != LBM_OK) return s;
        }
        CK(cudaGraphLaunch(ctx->graph, ctx->stream), "graph launch");
        ctx->step += ctx->graph_steps;  // an even count: the state ends in buffer 0 (natural layout) again
        n -= ctx->graph_steps;
    }
    for (int64_t s = 0; s < n; ++s) {
        lbm_status st = one_step<real>(ctx);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

// In-place contexts: bring the array back to the natural layout (every
// reader and writer of the state outside the step expects it); asynchronous.
lbm_status aa_natural(lbm_ctx *ctx)
{
    if (!ctx->inplace || !ctx->aa_odd) return LBM_OK;
    CK(lbm::aa_swap(ctx->grid.precision, ctx->ws + ctx->L.f0, ctx->grid.walls, ctx->grid.bc_x, ctx->big, ctx->grid.nx,
                    ctx->grid.ny, ctx->pitch, ctx->sms, ctx->stream),
       "layout swap");
    ctx->aa_odd = false;
    return LBM_OK;
}

// CTAs whose diagnostic slots hold the step's partials
int diag_ctas(const lbm_ctx *ctx) { return ctx->inplace ? ctx->aa.nctas : ctx->nctas; }

template <typename real>
lbm_status do_fields(lbm_ctx *ctx, void *rho, void *ux, void *uy, void *tw, void *pw)
{
    if (lbm_status s0 = aa_natural(ctx)) return s0;
    const size_t N = (size_t)ctx->grid.nx * ctx->grid.ny, nx = ctx->grid.nx;
    const size_t sz = sizeof(real);
    if (!ctx->fscratch) {
        CK(cudaMalloc((void **)&ctx->fscratch, align_up(3 * N * sz) + align_up(4 * nx * sz)),
           "fields scratch");
    }
    real *d_rho = (real *)ctx->fscratch, *d_vx = d_rho + N, *d_vy = d_vx + N;
    real *d_tw = (real *)(ctx->fscratch + align_up(3 * N * sz)), *d_pw = d_tw + 2 * nx;
    CK(cudaMemsetAsync(ctx->fscratch, 0, align_up(3 * N * sz) + align_up(4 * nx * sz), ctx->stream),
       "fields memset");
    lbm::KArgs<real> A = make_args<real>(ctx);
    A.fout = nullptr;
    A.o_rho = d_rho; A.o_vx = d_vx; A.o_vy = d_vy; A.o_tw = d_tw; A.o_pw = d_pw;
    cudaError_t le = ctx->mask ? lbm::mask_launch<real>(ctx->mask, A, lbm::MODE_FIELDS, ctx->stream)
                               : launch<real, lbm::MODE_FIELDS>(ctx, A);
    if (le != cudaSuccess) return cuda_fail(ctx, le, "fields launch");
    struct { void *dst; real *src; size_t n; } outs[] = {
        {rho, d_rho, N}, {ux, d_vx, N}, {uy, d_vy, N}, {tw, d_tw, 2 * nx}, {pw, d_pw, 2 * nx}};
    for (auto &o : outs) {
        if (!o.dst) continue;
        CK(cudaMemcpyAsync(o.dst, o.src, o.n * sz, cudaMemcpyDefault, ctx->stream), "fields copy");
    }
    CK(cudaStreamSynchronize(ctx->stream), "fields sync");
    return LBM_OK;
}

template <typename real>
void reset_acc(lbm_ctx *ctx)
{
    lbm::reset_acc_kernel<real><<<(lbm::MAX_CTAS + 255) / 256, 256, 0, ctx->stream>>>(
        (double *)(ctx->ws + ctx->L.mass), (double *)(ctx->ws + ctx->L.J),
        (real *)(ctx->ws + ctx->L.ext), (int *)(ctx->ws + ctx->L.err), lbm::MAX_CTAS);
}

// The library stores populations row-interleaved, f[y][i][x] with plane
// pitch P >= nx; the ABI exchanges plane-major f[i][y][x]. One strided 2D
// copy per plane converts.
cudaError_t copy_planes(const lbm_ctx *ctx, void *dst, const void *src, bool to_abi)
{
    const size_t sz = ctx->grid.precision == 64 ? 8 : 4;
    const size_t nx = ctx->grid.nx, ny = ctx->grid.ny, row = nx * sz, prow = (size_t)ctx->pitch * sz;
    for (int i = 0; i < 9; ++i) {
        cudaError_t e;
        if (to_abi)
            e = cudaMemcpy2DAsync((char *)dst + i * nx * ny * sz, row, (const char *)src + i * prow, 9 * prow,
                                  row, ny, cudaMemcpyDefault, ctx->stream);
        else
            e = cudaMemcpy2DAsync((char *)dst + i * prow, 9 * prow, (const char *)src + i * nx * ny * sz, row,
                                  row, ny, cudaMemcpyDefault, ctx->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

struct CkptHeader {
    uint64_t magic;
    int32_t nx, ny, walls, bc_x, precision, nctas;
    int64_t step;
    int32_t cur, inplace;  // inplace: one population array (in the natural layout) follows
};

} // namespace

bool lbm_encode_population_map(CUtensorMap *map, void *base, int pitch, int ny)
{
    return encode_population_map(map, base, pitch, ny);
}

namespace {

// (Re)selects the general-geometry path: kept when the caller's mask adds
// solid nodes to the wall rows or LBM_OPT_GENERAL forces it; the diagnostic
// slots then follow its CTA count.
lbm_status plan_geometry(lbm_ctx *ctx)
{
    lbm::mask_free(ctx->mask);
    ctx->mask = nullptr;
    const uint8_t *m = ctx->mask_host.empty() ? nullptr : ctx->mask_host.data();
    if (ctx->big && (m || ctx->force_general)) {
        std::snprintf(ctx->last_error, sizeof ctx->last_error,
                      "the general-geometry kernels need 9 pitch ny < 2^31");
        return LBM_ERR_ARG;
    }
    lbm_status st = lbm::mask_setup(m, ctx->grid, ctx->pitch, ctx->sms, ctx->force_general, ctx->stream, &ctx->mask,
                                    ctx->last_error, sizeof ctx->last_error);
    if (st == LBM_OK && ctx->mask) ctx->nctas = lbm::mask_blocks(ctx->mask);
    return st;
}

}  // namespace


extern "C" {

const char *lbm_status_string(lbm_status s)
{
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_PARAM: return "invalid physical parameter";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_OOM: return "out of memory";
    case LBM_ERR_NAN: return "non-finite or non-positive density";
    case LBM_ERR_STATE: return "incompatible checkpoint";
    case LBM_ERR_TIMEOUT: return "a bounded wait for staged data gave up";
    }
    return "unknown status";
}

const char *lbm_last_error(const lbm_ctx *ctx) { return ctx ? ctx->last_error : ""; }

size_t lbm_workspace_bytes(const lbm_grid *grid)
{
    if (!grid_ok(grid, true)) return 0;
    return layout_of(grid->nx, grid->ny, grid->precision).total;
}

size_t lbm_workspace_bytes_inplace(const lbm_grid *grid)
{
    if (!grid_ok(grid, true)) return 0;
    return layout_of(grid->nx, grid->ny, grid->precision, true).total;
}

} // extern "C"

namespace {

lbm_status init_ctx(const lbm_grid *grid, const lbm_eos *eos, double tau, const uint8_t *wall_mask,
                    double wetting, const lbm_drive *drive, const double *rho0, void *workspace, size_t ws_bytes,
                    void *stream, bool inplace, lbm_ctx **out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!grid_ok(grid, true) || !eos || !rho0) return LBM_ERR_ARG;
    if (!(tau > 0.5) || !(eos->k > 0) || !(eos->kappa >= 0) || !(eos->a > 0) || !(eos->b > 0) ||
        !(eos->R > 0) || !(eos->T_over_Tc > 0) || !std::isfinite(wetting))
        return LBM_ERR_PARAM;

    lbm_ctx *ctx = new (std::nothrow) lbm_ctx();
    if (!ctx) return LBM_ERR_OOM;
    ctx->grid = *grid;
    ctx->eos = *eos;
    if (drive) ctx->drive = *drive;
    else { ctx->drive.dp = 0; ctx->drive.p_ref = NAN; ctx->drive.gx = ctx->drive.gy = 0; }
    ctx->tau = tau;
    ctx->wet = wetting;
    ctx->stream = (cudaStream_t)stream;

    // Thermodynamics (host FP64).
    lbm::ChannelThermo ct;
    if (lbm::channel_thermo(*eos, ctx->drive, grid->bc_x, &ct) || fault_is("param")) {
        lbm_free(ctx);
        return LBM_ERR_PARAM;
    }
    ctx->th = ct.th;
    ctx->T = ct.T; ctx->Tc = ct.Tc;
    ctx->rho_g = ct.rho_g; ctx->rho_l = ct.rho_l; ctx->p_sat = ct.p_sat;
    ctx->rho_in = ct.rho_in; ctx->rho_out = ct.rho_out;
    ctx->rho_in_l = ct.rho_in_l; ctx->rho_out_l = ct.rho_out_l;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        lbm_status s = cuda_fail(ctx, e, "device query");
        lbm_free(ctx);
        return s;
    }

    ctx->inplace = inplace;
    ctx->L = layout_of(grid->nx, grid->ny, grid->precision, inplace);
    ctx->pitch = lbm::pitch_of(grid->nx);
    ctx->big = !lbm::idx32_ok(grid->nx, grid->ny);
    if (workspace) {
        if (ws_bytes < ctx->L.total || ((uintptr_t)workspace % ALIGN) != 0) {
            lbm_free(ctx);
            return LBM_ERR_ARG;
        }
        ctx->ws = (unsigned char *)workspace;
    } else {
        e = cudaMalloc((void **)&ctx->ws, ctx->L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            lbm_free(ctx);
            return LBM_ERR_OOM;
        }
        ctx->own_ws = true;
    }
    e = cudaMallocHost((void **)&ctx->h_err, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->err_ev, cudaEventDisableTiming);
    if (e == cudaSuccess && fault_is("alloc")) e = cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        lbm_status s = cuda_fail(ctx, e, "host flag");
        lbm_free(ctx);
        return s;
    }
    *ctx->h_err = 0;

    // tensor maps of both buffers (the plan chooses kernels by them)
    if (grid->precision == 32)
        ctx->tma_ok = encode_population_map(&ctx->tmap[0], ctx->ws + ctx->L.f0, ctx->pitch, grid->ny) &&
                      encode_population_map(&ctx->tmap[1], ctx->ws + ctx->L.f1, ctx->pitch, grid->ny);
    if (grid->precision == 32)
        ctx->tile_maps_ok =
            encode_population_map(&ctx->tmap_tile[0], ctx->ws + ctx->L.f0, ctx->pitch, grid->ny, lbm::T_BOX) &&
            encode_population_map(&ctx->tmap_tile[1], ctx->ws + ctx->L.f1, ctx->pitch, grid->ny, lbm::T_BOX);
    lbm_status st = plan_launch(ctx);
    if (st != LBM_OK) { lbm_free(ctx); return st; }
    if (wall_mask) ctx->mask_host.assign(wall_mask, wall_mask + (size_t)grid->nx * grid->ny);
    st = plan_geometry(ctx);
    if (st != LBM_OK) { lbm_free(ctx); return st; }
    if (inplace) {
        e = lbm::aa_plan(grid->precision, ctx->big, grid->walls, grid->bc_x, grid->nx, grid->ny, ctx->sms, &ctx->aa);
        if (e != cudaSuccess) {
            lbm_status s = cuda_fail(ctx, e, "in-place plan");
            lbm_free(ctx);
            return s;
        }
    }

    // Initial state f = f_eq(rho0, 0) in both arrays (in-place contexts: the
    // one array, natural layout; the kernel then stores each value twice to
    // the same slot).
    const size_t N = (size_t)grid->nx * grid->ny;
    double *d_rho0 = nullptr;
    e = cudaMallocAsync((void **)&d_rho0, N * sizeof(double), ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_rho0, rho0, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        const int blocks = (int)std::min<size_t>((N + 255) / 256, (size_t)ctx->sms * 8);
        if (grid->precision == 64) {
            lbm::init_kernel<double><<<blocks, 256, 0, ctx->stream>>>(
                d_rho0, (double *)(ctx->ws + ctx->L.f0), (double *)(ctx->ws + ctx->L.f1), grid->nx, ctx->pitch,
                grid->ny);
            reset_acc<double>(ctx);
        } else {
            lbm::init_kernel<float><<<blocks, 256, 0, ctx->stream>>>(
                d_rho0, (float *)(ctx->ws + ctx->L.f0), (float *)(ctx->ws + ctx->L.f1), grid->nx, ctx->pitch,
                grid->ny);
            reset_acc<float>(ctx);
        }
        e = cudaGetLastError();
        cudaFreeAsync(d_rho0, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        lbm_status s = cuda_fail(ctx, e, "init");
        lbm_free(ctx);
        return s;
    }
    *out = ctx;
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_init(const lbm_grid *grid, const lbm_eos *eos, double tau, const uint8_t *wall_mask,
                    double wetting, const lbm_drive *drive, const double *rho0, void *workspace, size_t ws_bytes,
                    void *stream, lbm_ctx **out)
{
    return init_ctx(grid, eos, tau, wall_mask, wetting, drive, rho0, workspace, ws_bytes, stream, false, out);
}

lbm_status lbm_init_inplace(const lbm_grid *grid, const lbm_eos *eos, double tau, double wetting,
                            const lbm_drive *drive, const double *rho0, void *workspace, size_t ws_bytes,
                            void *stream, lbm_ctx **out)
{
    return init_ctx(grid, eos, tau, nullptr, wetting, drive, rho0, workspace, ws_bytes, stream, true, out);
}

lbm_status lbm_relaxed_coexistence(const lbm_eos *eos, double tau, const lbm_collision *coll, int32_t precision,
                                   int32_t ny, int64_t steps, void *stream, double *rho_g, double *rho_l,
                                   double *p_gas, double *p_liq)
{
    if (!eos || (precision != 32 && precision != 64) || ny < 16 || steps < 0) return LBM_ERR_ARG;
    lbm::Thermo th{};
    double Tc = 0, g = 0, l = 0, ps = 0;
    if (lbm::thermo_of(*eos, &th, &Tc) || lbm::maxwell(th, &g, &l, &ps)) return LBM_ERR_PARAM;
    // a liquid slab between rows ny/4 and 3ny/4 of a periodic 4 x ny box, tanh
    // profile of width 4 between the Maxwell densities
    const int nx = 4;
    std::vector<double> rho0((size_t)nx * ny);
    for (int y = 0; y < ny; ++y) {
        const double sl = 0.5 * (std::tanh(2.0 * (y - 0.25 * ny) / 4.0) - std::tanh(2.0 * (y - 0.75 * ny) / 4.0));
        for (int x = 0; x < nx; ++x) rho0[(size_t)y * nx + x] = g + (l - g) * sl;
    }
    const lbm_grid grid{nx, ny, 0, 0, precision};
    lbm_ctx *ctx = nullptr;
    lbm_status st = lbm_init(&grid, eos, tau, nullptr, 0.0, nullptr, rho0.data(), nullptr, 0, stream, &ctx);
    if (st != LBM_OK) return st;
    if (coll) st = lbm_set_collision(ctx, coll);
    if (st == LBM_OK) st = lbm_step(ctx, steps);
    std::vector<double> r64((size_t)nx * ny);
    std::vector<float> r32((size_t)nx * ny);
    if (st == LBM_OK)
        st = lbm_fields(ctx, precision == 64 ? (void *)r64.data() : (void *)r32.data(), nullptr, nullptr, nullptr,
                        nullptr);
    if (st == LBM_OK) st = lbm_step(ctx, 0);  // the bad-density flag of the last steps
    if (st == LBM_OK) {
        lbm_diag_t d;
        st = lbm_diag(ctx, &d);
        if (st == LBM_OK && d.nan_detected) st = LBM_ERR_NAN;
    }
    lbm_free(ctx);
    if (st != LBM_OK) return st;
    auto at = [&](int y) { return precision == 64 ? r64[(size_t)y * nx] : (double)r32[(size_t)y * nx]; };
    const double rg = at(0), rl = at(ny / 2), k2 = eos->k * eos->k;
    if (rho_g) *rho_g = rg;
    if (rho_l) *rho_l = rl;
    if (p_gas) *p_gas = k2 * lbm::eos_pressure(th, rg);
    if (p_liq) *p_liq = k2 * lbm::eos_pressure(th, rl);
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *ctx, int64_t n)
{
    if (!ctx || n < 0) return LBM_ERR_ARG;
    lbm_status flag = LBM_OK;
    if (ctx->err_pending && cudaEventQuery(ctx->err_ev) == cudaSuccess) {
        ctx->err_pending = false;
        // bit 0: bad density; bit 1: a bounded stage wait gave up
        if (*ctx->h_err & 1) flag = LBM_ERR_NAN;
        else if (*ctx->h_err) flag = LBM_ERR_TIMEOUT;
    }
    if (n == 0) return flag;
    lbm_status s = ctx->grid.precision == 64 ? do_steps<double>(ctx, n) : do_steps<float>(ctx, n);
    if (s != LBM_OK) return s;
    if (!ctx->err_pending) {
        cudaError_t e = cudaMemcpyAsync(ctx->h_err, ctx->ws + ctx->L.err, sizeof(int),
                                        cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->err_ev, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "error flag");
        ctx->err_pending = true;
    }
    return flag;
}

lbm_status lbm_fields(lbm_ctx *ctx, void *rho, void *ux, void *uy, void *tau_wall, void *p_wall)
{
    if (!ctx) return LBM_ERR_ARG;
    return ctx->grid.precision == 64 ? do_fields<double>(ctx, rho, ux, uy, tau_wall, p_wall)
                                     : do_fields<float>(ctx, rho, ux, uy, tau_wall, p_wall);
}

namespace {
void enqueue_diag(lbm_ctx *ctx, double *dout)
{
    if (ctx->grid.precision == 64)
        lbm::diag_kernel<double><<<1, 256, 0, ctx->stream>>>(
            (double *)(ctx->ws + ctx->L.mass), (double *)(ctx->ws + ctx->L.J),
            (double *)(ctx->ws + ctx->L.ext), (int *)(ctx->ws + ctx->L.err), diag_ctas(ctx), dout);
    else
        lbm::diag_kernel<float><<<1, 256, 0, ctx->stream>>>(
            (double *)(ctx->ws + ctx->L.mass), (double *)(ctx->ws + ctx->L.J),
            (float *)(ctx->ws + ctx->L.ext), (int *)(ctx->ws + ctx->L.err), diag_ctas(ctx), dout);
}
}  // namespace

lbm_status lbm_diag_async(lbm_ctx *ctx, double *dst)
{
    if (!ctx || !dst || ((uintptr_t)dst % 8) != 0) return LBM_ERR_ARG;
    double *dout = (double *)(ctx->ws + ctx->L.dout);
    enqueue_diag(ctx, dout);
    CK(cudaGetLastError(), "diag launch");
    CK(cudaMemcpyAsync(dst, dout, 7 * sizeof(double), cudaMemcpyDefault, ctx->stream), "diag copy");
    return LBM_OK;
}

lbm_status lbm_diag(lbm_ctx *ctx, lbm_diag_t *out)
{
    if (!ctx || !out) return LBM_ERR_ARG;
    double *dout = (double *)(ctx->ws + ctx->L.dout);
    enqueue_diag(ctx, dout);
    CK(cudaGetLastError(), "diag launch");
    double h[8];
    CK(cudaMemcpyAsync(h, dout, 7 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "diag copy");
    CK(cudaStreamSynchronize(ctx->stream), "diag sync");
    std::memset(out, 0, sizeof *out);
    out->step = ctx->step;
    out->mass = ctx->step > 0 ? h[0] : 0.0;
    out->wall_shear_sum = h[1];
    const bool any = ctx->step > 0 && ctx->grid.walls;
    out->tau_wall_min = any ? h[2] : 0.0;
    out->tau_wall_max = any ? h[3] : 0.0;
    out->p_wall_min = any ? h[4] : 0.0;
    out->p_wall_max = any ? h[5] : 0.0;
    out->nan_detected = ((int)h[6] & 1) != 0;  // bit 1 (a stage wait gave up) is lbm_step's LBM_ERR_TIMEOUT
    out->T = ctx->T; out->Tc = ctx->Tc;
    out->rho_g = ctx->rho_g; out->rho_l = ctx->rho_l; out->p_sat = ctx->p_sat;
    out->rho_in = ctx->rho_in; out->rho_out = ctx->rho_out;
    out->rho_in_l = ctx->rho_in_l; out->rho_out_l = ctx->rho_out_l;
    return LBM_OK;
}

lbm_status lbm_reset_diag(lbm_ctx *ctx)
{
    if (!ctx) return LBM_ERR_ARG;
    double *mass = (double *)(ctx->ws + ctx->L.mass), *J = (double *)(ctx->ws + ctx->L.J);
    if (ctx->grid.precision == 64)
        lbm::reset_acc_kernel<double><<<(lbm::MAX_CTAS + 255) / 256, 256, 0, ctx->stream>>>(
            mass, J, (double *)(ctx->ws + ctx->L.ext), nullptr, lbm::MAX_CTAS);
    else
        lbm::reset_acc_kernel<float><<<(lbm::MAX_CTAS + 255) / 256, 256, 0, ctx->stream>>>(
            mass, J, (float *)(ctx->ws + ctx->L.ext), nullptr, lbm::MAX_CTAS);
    CK(cudaGetLastError(), "reset diag");
    return LBM_OK;
}

lbm_status lbm_populations(lbm_ctx *ctx, void *dst)
{
    if (!ctx || !dst) return LBM_ERR_ARG;
    if (lbm_status s = aa_natural(ctx)) return s;
    CK(copy_planes(ctx, dst, ctx->ws + (ctx->cur ? ctx->L.f1 : ctx->L.f0), true), "populations copy");
    CK(cudaStreamSynchronize(ctx->stream), "populations sync");
    return LBM_OK;
}

lbm_status lbm_load_populations(lbm_ctx *ctx, const void *src)
{
    if (!ctx || !src) return LBM_ERR_ARG;
    // both arrays, so never-written slots (solid rows, unreached boundary
    // slots) agree with the loaded state
    CK(copy_planes(ctx, ctx->ws + ctx->L.f0, src, false), "load copy");
    if (!ctx->inplace) CK(copy_planes(ctx, ctx->ws + ctx->L.f1, src, false), "load copy");
    ctx->aa_odd = false;
    CK(cudaStreamSynchronize(ctx->stream), "load sync");
    return LBM_OK;
}

size_t lbm_checkpoint_bytes(const lbm_ctx *ctx)
{
    if (!ctx) return 0;
    const size_t sz = ctx->grid.precision == 64 ? 8 : 4;
    return sizeof(CkptHeader) + (ctx->inplace ? 1 : 2) * ctx->L.pops + (size_t)lbm::MAX_CTAS * (16 + 4 * sz) +
           sizeof(int);
}

lbm_status lbm_checkpoint(lbm_ctx *ctx, void *host_buf, size_t bytes)
{
    if (!ctx || !host_buf || bytes < lbm_checkpoint_bytes(ctx)) return LBM_ERR_ARG;
    const size_t sz = ctx->grid.precision == 64 ? 8 : 4;
    if (lbm_status s = aa_natural(ctx)) return s;
    const int narr = ctx->inplace ? 1 : 2;
    CkptHeader h{CKPT_MAGIC, ctx->grid.nx, ctx->grid.ny, ctx->grid.walls, ctx->grid.bc_x,
                 ctx->grid.precision, diag_ctas(ctx), ctx->step, ctx->cur, ctx->inplace ? 1 : 0};
    unsigned char *p = (unsigned char *)host_buf;
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    // both population arrays: slots no population reaches keep older values
    // (in-place contexts: the one array, in the natural layout)
    CK(cudaMemcpyAsync(p, ctx->ws + ctx->L.f0, narr * ctx->L.pops, cudaMemcpyDeviceToHost, ctx->stream), "ckpt");
    p += narr * ctx->L.pops;
    CK(cudaMemcpyAsync(p, ctx->ws + ctx->L.mass, lbm::MAX_CTAS * 8, cudaMemcpyDeviceToHost, ctx->stream), "ckpt");
    p += lbm::MAX_CTAS * 8;
    CK(cudaMemcpyAsync(p, ctx->ws + ctx->L.J, lbm::MAX_CTAS * 8, cudaMemcpyDeviceToHost, ctx->stream), "ckpt");
    p += lbm::MAX_CTAS * 8;
    CK(cudaMemcpyAsync(p, ctx->ws + ctx->L.ext, lbm::MAX_CTAS * 4 * sz, cudaMemcpyDeviceToHost, ctx->stream), "ckpt");
    p += lbm::MAX_CTAS * 4 * sz;
    CK(cudaMemcpyAsync(p, ctx->ws + ctx->L.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "ckpt");
    CK(cudaStreamSynchronize(ctx->stream), "ckpt sync");
    return LBM_OK;
}

lbm_status lbm_restore(lbm_ctx *ctx, const void *host_buf, size_t bytes)
{
    if (!ctx || !host_buf || bytes < lbm_checkpoint_bytes(ctx)) return LBM_ERR_ARG;
    CkptHeader h;
    std::memcpy(&h, host_buf, sizeof h);
    if (h.magic != CKPT_MAGIC || h.nx != ctx->grid.nx || h.ny != ctx->grid.ny || h.walls != ctx->grid.walls ||
        h.bc_x != ctx->grid.bc_x || h.precision != ctx->grid.precision || (h.inplace != 0) != ctx->inplace)
        return LBM_ERR_STATE;
    const size_t sz = ctx->grid.precision == 64 ? 8 : 4;
    const int narr = ctx->inplace ? 1 : 2;
    const unsigned char *p = (const unsigned char *)host_buf + sizeof h;
    CK(cudaMemcpyAsync(ctx->ws + ctx->L.f0, p, narr * ctx->L.pops, cudaMemcpyHostToDevice, ctx->stream), "restore");
    p += narr * ctx->L.pops;
    CK(cudaMemcpyAsync(ctx->ws + ctx->L.mass, p, lbm::MAX_CTAS * 8, cudaMemcpyHostToDevice, ctx->stream), "restore");
    p += lbm::MAX_CTAS * 8;
    CK(cudaMemcpyAsync(ctx->ws + ctx->L.J, p, lbm::MAX_CTAS * 8, cudaMemcpyHostToDevice, ctx->stream), "restore");
    p += lbm::MAX_CTAS * 8;
    CK(cudaMemcpyAsync(ctx->ws + ctx->L.ext, p, lbm::MAX_CTAS * 4 * sz, cudaMemcpyHostToDevice, ctx->stream), "restore");
    p += lbm::MAX_CTAS * 4 * sz;
    CK(cudaMemcpyAsync(ctx->ws + ctx->L.err, p, sizeof(int), cudaMemcpyHostToDevice, ctx->stream), "restore");
    CK(cudaStreamSynchronize(ctx->stream), "restore sync");
    ctx->step = h.step;
    ctx->cur = h.cur;
    ctx->aa_odd = false;
    ctx->err_pending = false;
    // Per-CTA accumulators only line up with the same launch geometry; with
    // another CTA count they stay valid as totals but the summation order changes.
    ctx->nctas = std::max(ctx->nctas, 1);
    return LBM_OK;
}

lbm_status lbm_set_collision(lbm_ctx *ctx, const lbm_collision *c)
{
    if (!ctx) return LBM_ERR_ARG;
    drop_graph(ctx);
    if (!c) { ctx->coll = lbm_collision{}; return LBM_OK; }
    if (c->kind == LBM_COLL_BGK) { ctx->coll = *c; return LBM_OK; }
    if (c->kind != LBM_COLL_MRT) return LBM_ERR_ARG;
    for (double r : {c->s_e, c->s_eps, c->s_j, c->s_q})
        if (!(r > 0.0 && r < 2.0)) return LBM_ERR_ARG;
    if (!(c->s_nu <= 0.0 || c->s_nu < 2.0) || std::isnan(c->s_nu)) return LBM_ERR_ARG;
    ctx->coll = *c;
    return LBM_OK;
}

lbm_status lbm_set_option(lbm_ctx *ctx, lbm_option opt, int64_t value)
{
    if (!ctx) return LBM_ERR_ARG;
    drop_graph(ctx);  // the captured launches hold the old arguments
    switch (opt) {
    case LBM_OPT_CTAS_PER_SM:
        if (value < 0 || value > 32) return LBM_ERR_ARG;
        ctx->ctas_per_sm_opt = (int)value;
        break;
    case LBM_OPT_REVERSE:
        ctx->reverse = value != 0;
        return LBM_OK;
    case LBM_OPT_STRIP:
        if (value < 2 || value > STRIP) return LBM_ERR_ARG;
        ctx->W_opt = (int)value;
        break;
    case LBM_OPT_STAGED:
        ctx->allow_staged = value != 0;
        break;
    case LBM_OPT_ROWS2:
        ctx->allow_rows2 = value != 0;
        break;
    case LBM_OPT_TMA:
        ctx->allow_tma = value != 0;
        break;  // re-plan: the tile kernel needs tensor loads
    case LBM_OPT_PREFETCH:
        if (value < 0 || value > 4) return LBM_ERR_ARG;
        ctx->pf = (int)value;
        return LBM_OK;
    case LBM_OPT_GENERAL:
        if (value != 0 && (ctx->big || ctx->inplace)) return LBM_ERR_ARG;  // 32-bit offsets, two arrays only
        ctx->force_general = value != 0;
        break;
    case LBM_OPT_PDL:
        ctx->pdl = value != 0;
        drop_graph(ctx);
        return LBM_OK;
    case LBM_OPT_GRAPH_STEPS:
        if (value < 0 || (value & 1) || value > 1 << 20) return LBM_ERR_ARG;
        ctx->graph_steps = (int)value;
        drop_graph(ctx);
        return LBM_OK;
    case LBM_OPT_FAULT_SKIP_COPY:
        // the test build exists for walls, pressure columns and unpadded rows
        if (value != 0) {
            if (!(ctx->rows2 && !ctx->inplace && !ctx->mask && !ctx->big && ctx->grid.walls && ctx->grid.bc_x &&
                  ctx->pitch == ctx->grid.nx))
                return LBM_ERR_ARG;
            cudaError_t e = cudaFuncSetAttribute((void *)lbm::step_kernel_rows2<true, true, false, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)lbm::rows2_smem_bytes());
            if (e != cudaSuccess) return cuda_fail(ctx, e, "smem attribute");
        }
        ctx->fault_skip = value != 0;
        break;  // re-plan: the test build is a row-pair kernel
    case LBM_OPT_TILE:
        ctx->allow_tile = value != 0;
        break;
    default:
        return LBM_ERR_ARG;
    }
    // Re-plan; per-CTA accumulators are folded into the new partition only
    // through their totals, so reset them to keep the reduction exact.
    int old = ctx->nctas;
    lbm_status s = plan_launch(ctx);
    if (s == LBM_OK) s = plan_geometry(ctx);
    if (s == LBM_OK && old != ctx->nctas) {
        if (ctx->grid.precision == 64) reset_acc<double>(ctx); else reset_acc<float>(ctx);
    }
    return s;
}

lbm_status lbm_launch_info(const lbm_ctx *ctx, int64_t *ctas, int64_t *threads, int64_t *units,
                           int64_t *staged)
{
    if (!ctx) return LBM_ERR_ARG;
    if (ctx->inplace) {
        // CTAs striding over the 32 x 8 tiles (FP32: two rows per thread)
        if (ctas) *ctas = ctx->aa.nctas;
        if (threads) *threads = ctx->aa.threads;
        if (units) *units = (int64_t)ctx->aa.ntx * ctx->aa.nty;
        if (staged) *staged = 0;
        return LBM_OK;
    }
    if (ctas) *ctas = ctx->nctas;
    if (threads) *threads = ctx->mask ? 256 : threads_of(ctx, lbm::MODE_STEP);
    if (units) *units = ctx->mask ? (int64_t)ctx->grid.nx * ctx->grid.ny : ctx->units;
    if (staged) *staged = (ctx->staged && !ctx->mask) ? 1 : 0;
    return LBM_OK;
}

void lbm_free(lbm_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream || ctx->ws) cudaStreamSynchronize(ctx->stream);
    if (ctx->own_ws && ctx->ws) cudaFree(ctx->ws);
    lbm::mask_free(ctx->mask);
    drop_graph(ctx);
    if (ctx->fscratch) cudaFree(ctx->fscratch);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    if (ctx->err_ev) cudaEventDestroy(ctx->err_ev);
    delete ctx;
}

} // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free single step.
//
// Some callers cannot allocate device memory at the point where they step the
// lattice: code running inside another framework's memory pool (a raw
// allocation would bypass the pool's accounting and limits), or an embedded
// host that sizes every device buffer up front. This entry point performs one
// step between two caller-owned population buffers and keeps the only scratch
// it needs - the per-CTA diagnostic partials and the error word - in a fixed
// device array that the library declares at file scope. Nothing is allocated
// per call.
// ---------------------------------------------------------------------------

namespace {

constexpr int NOALLOC_MAX_CTAS = 4096;

// Per-CTA partials of one step: mass, wall-shear sum, four extrema (stored as
// double so both precisions fit) and the bad-density flag.
struct NoallocScratch {
    double mass[NOALLOC_MAX_CTAS];
    double J[NOALLOC_MAX_CTAS];
    double ext[4 * NOALLOC_MAX_CTAS];
    int err;
};

constexpr int NOALLOC_MAX_DEVICES = 64;
NoallocScratch *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
std::mutex g_noalloc_mutex;

} // namespace

// The scratch itself. In host code this name is only a stand-in for the
// device object; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

namespace {

// Device address of the scratch on the current device, resolved on the first
// call made with that device current.
cudaError_t noalloc_scratch(NoallocScratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<NoallocScratch *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

template <typename real>
lbm_status noalloc_launch(lbm_ctx *c, NoallocScratch *sc, const void *f_in, void *f_out, double *diag_out,
                          int32_t *err_out)
{
    real *ext = reinterpret_cast<real *>(sc->ext);
    lbm::reset_acc_kernel<real><<<(c->nctas + 255) / 256, 256, 0, c->stream>>>(sc->mass, sc->J, ext, &sc->err,
                                                                                 c->nctas);
    lbm::KArgs<real> A = make_args<real>(c);
    A.fin = static_cast<const real *>(f_in);
    A.fout = static_cast<real *>(f_out);
    A.mass_part = sc->mass;
    A.J_acc = sc->J;
    A.ext = ext;
    A.err = &sc->err;
    cudaError_t e = launch<real, lbm::MODE_STEP>(c, A);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "noalloc step");
    if (diag_out)
        lbm::diag_kernel<real><<<1, 256, 0, c->stream>>>(sc->mass, sc->J, ext, &sc->err, c->nctas, diag_out);
    e = cudaGetLastError();
    if (e == cudaSuccess && err_out)
        e = cudaMemcpyAsync(err_out, &sc->err, sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(nullptr, e, "noalloc launch");
}

} // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_grid *grid, const lbm_eos *eos, double tau,
                                       double wetting, const lbm_drive *drive, const void *f_in,
                                       void *f_out, int64_t ctas, double *diag_out, int32_t *err_out,
                                       void *stream)
{
    if (!grid_ok(grid) || !eos || !f_in || !f_out || f_in == f_out) return LBM_ERR_ARG;
    if (ctas < 0 || ctas > NOALLOC_MAX_CTAS) return LBM_ERR_ARG;
    // buffers must hold whole values of the grid precision; the staged kernels
    // also need 16-byte aligned rows (checked below)
    const uintptr_t esz = grid->precision == 64 ? 8 : 4;
    if (((uintptr_t)f_in | (uintptr_t)f_out) % esz != 0) return LBM_ERR_ARG;
    if (((uintptr_t)diag_out) % 8 != 0 || ((uintptr_t)err_out) % 4 != 0) return LBM_ERR_ARG;
    if (!(tau > 0.5) || !(eos->k > 0) || !(eos->kappa >= 0) || !(eos->a > 0) || !(eos->b > 0) ||
        !(eos->R > 0) || !(eos->T_over_Tc > 0) || !std::isfinite(wetting))
        return LBM_ERR_PARAM;

    NoallocScratch *sc = nullptr;
    cudaError_t e = noalloc_scratch(&sc);
    if (e != cudaSuccess) return LBM_ERR_CUDA;

    // Launch plan and physics on the host stack only (no workspace).
    lbm_ctx c;
    c.grid = *grid;
    c.pitch = grid->nx;  // caller buffers: rows of 9 nx values
    c.eos = *eos;
    if (drive) c.drive = *drive;
    else { c.drive.dp = 0; c.drive.p_ref = NAN; c.drive.gx = c.drive.gy = 0; }
    c.tau = tau;
    c.wet = wetting;
    c.stream = static_cast<cudaStream_t>(stream);
    // The staged kernels copy population rows with bulk asynchronous copies,
    // which need 16-byte aligned addresses: a caller buffer that does not start
    // on a 16-byte boundary (a view with an element offset) takes the register-
    // prefetch kernel, which gives identical results.
    if (((uintptr_t)f_in | (uintptr_t)f_out) % 16 != 0) c.allow_staged = false;
    lbm::ChannelThermo ct;
    if (lbm::channel_thermo(*eos, c.drive, grid->bc_x, &ct)) return LBM_ERR_PARAM;
    c.th = ct.th;
    c.T = ct.T; c.Tc = ct.Tc;
    c.rho_g = ct.rho_g; c.rho_l = ct.rho_l; c.p_sat = ct.p_sat;
    c.rho_in = ct.rho_in; c.rho_out = ct.rho_out;
    c.rho_in_l = ct.rho_in_l; c.rho_out_l = ct.rho_out_l;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    if (plan_launch(&c) != LBM_OK) return LBM_ERR_CUDA;
    if (ctas > 0) c.nctas = (int)std::min<long long>(ctas, std::max<long long>(1, c.units / 2));
    c.nctas = std::min(c.nctas, NOALLOC_MAX_CTAS);
    c.band = band_rows(c.nyf, c.nstrips, c.nctas, c.grid.walls);
    return grid->precision == 64 ? noalloc_launch<double>(&c, sc, f_in, f_out, diag_out, err_out)
                                 : noalloc_launch<float>(&c, sc, f_in, f_out, diag_out, err_out);
}
