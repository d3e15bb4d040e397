// C ABI of batched channels (lbm_batch_*; see include/lbm.h): many independent
// airway channels of different sizes, pressure drops, plug lengths and film
// thicknesses stepped by one kernel launch per step, replayed from a CUDA
// graph - the parameter sweeps of the paper's Sec. 3.3 (Figs. 10-12) as one
// persistent job. Host orchestration only; the step is batch_step_kernel,
// which runs exactly the per-segment code of the single-channel kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace {

constexpr int STRIP = lbm::STRIP;  // widest strip (columns per CTA)
// threads per CTA of the step kernels of a precision and staging choice
inline int cta_threads(int precision, bool staged)
{
    if (precision == 64) return staged ? lbm::threads_per_cta<double, true>() : lbm::threads_per_cta<double, false>();
    return staged ? lbm::threads_per_cta<float, true>() : lbm::threads_per_cta<float, false>();
}
constexpr int DEFAULT_GRAPH_STEPS = 64;  // even: a replay ends on the buffer it started from

struct ChanHost {
    lbm_grid grid;
    lbm_drive drive;
    double rho_in = 0, rho_out = 0, rho_in_l = 0, rho_out_l = 0;
    long long off = 0;  // element offset in the packed buffers
    int pitch = 0;      // plane pitch of the channel's population rows
    int W = STRIP, nstrips = 0, yf0 = 0, nyf = 0;
    int band = 0, nbands = 1;  // work order: bands of `band` fluid rows, strip by strip within a band
    long long units = 0, unit_base = 0;
};

size_t align_elems(size_t n) { return (n + 63) / 64 * 64; }  // 256 B for float

} // namespace

struct lbm_batch {
    int n = 0, precision = 32, walls = 0, bc_x = 0;
    lbm_eos eos{};
    double tau = 1.0, wet = 0.0, T = 0, Tc = 0, rho_g = 0, rho_l = 0, p_sat = 0;
    lbm::Thermo th{};  // EOS at the working temperature
    lbm_collision coll{};  // BGK unless lbm_batch_set_collision chose MRT
    std::vector<ChanHost> ch;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    unsigned char *pop[2] = {nullptr, nullptr};
    size_t pop_elems = 0;
    int cur = 0;
    int64_t step = 0;
    // launch plan and device tables
    int sms = 0, nctas = 0, nseg = 0, per_sm = 0, ctas_per_sm_opt = 0, W_opt = 0, reverse = 0;
    int band_opt = -1;  // LBM_OPT_BAND: -1 whole strip columns, one CTA each (default); 0 strip-major
                        // balanced cut; > 0 bands of that many rows
    bool allow_staged = true, staged = false;
    bool allow_rows2 = true, rows2 = false;  // LBM_OPT_ROWS2: row-pair FP32 step
    // LBM_OPT_TMA (on by default: over whole strip columns tensor loads made the
    // 64-channel sweep 12% faster than plane copies; over the balanced cut's
    // short segments they were 4% slower); d_tmaps encoded
    bool allow_tma = true, tma_ok = false;
    int pf = 0;  // LBM_OPT_PREFETCH (row pairs ahead, 0 = off)
    CUtensorMap *d_tmaps = nullptr;          // [2][n]: tensor maps of each buffer's channels (FP32)
    void *d_chan = nullptr;
    lbm::BatchSeg *d_segs = nullptr;
    int *d_cta_begin = nullptr;
    double *d_seg_mass = nullptr, *d_seg_J = nullptr;
    void *d_seg_ext = nullptr;
    int *d_err = nullptr;
    double *d_diag = nullptr;
    std::vector<lbm::BatchSeg> segs;
    // graph of graph_steps steps starting from buffer 0
    int graph_steps = DEFAULT_GRAPH_STEPS;
    cudaGraphExec_t graph = nullptr;
    // persistent stepping (row-pair batches): one cooperative launch per chunk
    // of steps, segments ordered by step counters (LBM_OPT_PERSISTENT; off by
    // default: per-step graph launches over whole strip columns measured faster)
    bool allow_persist = false, persist = false;
    int *d_done = nullptr, *d_abort = nullptr, *d_dep_beg = nullptr, *d_dep = nullptr;
    // fields scratch and non-blocking NaN check
    unsigned char *fscratch = nullptr;
    size_t fscratch_bytes = 0;
    int *h_err = nullptr;
    cudaEvent_t err_ev = nullptr;
    bool err_pending = false;
    char last_error[512] = {0};
};

namespace {

lbm_status bfail(lbm_batch *b, cudaError_t e, const char *where)
{
    if (b) std::snprintf(b->last_error, sizeof b->last_error, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define BCK(call, where)                                          \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return bfail(b, e_, where);        \
    } while (0)

size_t sz_of(const lbm_batch *b) { return b->precision == 64 ? 8 : 4; }

template <typename real, bool STAGED>
void *batch_kernel_ptr(bool walls, bool pres)
{
    using namespace lbm;
    if (walls && pres) return (void *)batch_step_kernel<real, true, true, STAGED>;
    if (walls) return (void *)batch_step_kernel<real, true, false, STAGED>;
    if (pres) return (void *)batch_step_kernel<real, false, true, STAGED>;
    return (void *)batch_step_kernel<real, false, false, STAGED>;
}

void *batch_kernel(const lbm_batch *b)
{
    const bool w = b->walls, p = b->bc_x;
    if (b->rows2) {
        using namespace lbm;
        if (w && p) return (void *)batch_step_kernel_rows2<true, true>;
        if (w) return (void *)batch_step_kernel_rows2<true, false>;
        if (p) return (void *)batch_step_kernel_rows2<false, true>;
        return (void *)batch_step_kernel_rows2<false, false>;
    }
    if (b->precision == 64)
        return b->staged ? batch_kernel_ptr<double, true>(w, p) : batch_kernel_ptr<double, false>(w, p);
    return b->staged ? batch_kernel_ptr<float, true>(w, p) : batch_kernel_ptr<float, false>(w, p);
}

void *persist_kernel(const lbm_batch *b)
{
    using namespace lbm;
    const bool w = b->walls, p = b->bc_x;
    if (w && p) return (void *)batch_persistent_kernel_rows2<true, true>;
    if (w) return (void *)batch_persistent_kernel_rows2<true, false>;
    if (p) return (void *)batch_persistent_kernel_rows2<false, true>;
    return (void *)batch_persistent_kernel_rows2<false, false>;
}

// Dependencies of each segment for persistent stepping: the segments of the
// same channel in its own and the two neighbouring strips (wrapped for
// periodic x) whose fluid rows meet [ya - 3, yb + 2] (wrapped for periodic y):
// the rows its stencil reads, and the rows whose earlier readers its pushes
// into the target buffer must not overtake. CSR: beg[nseg + 1], dep[].
void build_deps(const lbm_batch *b, std::vector<int> &beg, std::vector<int> &dep)
{
    std::vector<std::vector<std::vector<int>>> by(b->n);  // [channel][strip] -> segments
    for (int c = 0; c < b->n; ++c) by[c].resize(b->ch[c].nstrips);
    for (int k = 0; k < b->nseg; ++k) by[b->segs[k].chan][b->segs[k].strip].push_back(k);
    beg.assign(1, 0);
    dep.clear();
    for (int k = 0; k < b->nseg; ++k) {
        const lbm::BatchSeg &g = b->segs[k];
        const ChanHost &c = b->ch[g.chan];
        const int ny = c.grid.ny, ns = c.nstrips;
        const int a = g.ya - 3, z = g.yb + 2;  // inclusive row range
        auto meets = [&](const lbm::BatchSeg &t) {
            for (int sh : {0, -ny, ny}) {
                if (b->walls && sh != 0) continue;
                if (t.ya + sh <= z && t.yb - 1 + sh >= a) return true;
            }
            return false;
        };
        std::vector<int> strips;
        for (int d = -1; d <= 1; ++d) {
            int t = g.strip + d;
            if (b->bc_x) { if (t < 0 || t >= ns) continue; }
            else t = ((t % ns) + ns) % ns;
            if (std::find(strips.begin(), strips.end(), t) == strips.end()) strips.push_back(t);
        }
        for (int t : strips)
            for (int j : by[g.chan][t])
                if (meets(b->segs[j])) dep.push_back(j);
        beg.push_back((int)dep.size());
    }
}

size_t staged_bytes(const lbm_batch *b, bool staged)
{
    if (!staged) return 0;
    return b->precision == 64 ? lbm::staged_smem_bytes<double>() : lbm::staged_smem_bytes<float>();
}

// dynamic shared memory and threads of the batch step kernel
size_t step_smem(const lbm_batch *b) { return b->rows2 ? lbm::rows2_smem_bytes() : staged_bytes(b, b->staged); }
int step_threads(const lbm_batch *b) { return b->rows2 ? lbm::R2_BLOCK : cta_threads(b->precision, b->staged); }

// Shared physics of every channel, in the kernel argument block.
template <typename real>
lbm::KArgs<real> physics_args(const lbm_batch *b)
{
    lbm::KArgs<real> A{};
    const double k = b->eos.k;
    A.RT = (real)(b->eos.R * b->T);
    A.a = (real)b->eos.a;
    A.b4 = (real)(0.25 * b->eos.b);
    A.k2 = (real)(k * k);
    A.kappa = (real)b->eos.kappa;
    A.tau = (real)b->tau;
    A.inv_tau = (real)(1.0 / b->tau);
    A.omb = (real)(1.0 - 1.0 / b->tau);
    A.wet = (real)b->wet;
    A.nu = (real)((b->tau - 0.5) / 3.0);
    A.eos_kind = b->th.kind;
    A.bpr = (real)b->th.b;
    A.aalpha = (real)b->th.aalpha;
    const lbm_collision &cl = b->coll;
    A.mrt = cl.kind == LBM_COLL_MRT;
    A.ushift = A.mrt ? (real)(1.0 / cl.s_j) : (real)b->tau;
    if (A.mrt) {
        const double s_nu = cl.s_nu > 0 ? cl.s_nu : 1.0 / b->tau;
        A.m_e = (real)(cl.s_e / 36.0); A.m_eps = (real)(cl.s_eps / 36.0);
        A.m_j = (real)(cl.s_j / 6.0); A.m_q = (real)(cl.s_q / 12.0); A.m_nu = (real)(s_nu / 4.0);
    }
    A.ph_g = (real)b->rho_g;
    A.inv_dph = b->rho_l > b->rho_g ? (real)(1.0 / (b->rho_l - b->rho_g)) : real(0);
    A.err = b->d_err;
    A.reverse = b->reverse;
    A.pf = b->pf;
    return A;
}

// Strip partition per channel, CTA count, and the balanced segment work list:
// the units (channel, strip, fluid row) of all channels in order are cut into
// nctas equal runs, never between rows 1|2 or ny-3|ny-2 of a channel.
lbm_status batch_plan(lbm_batch *b)
{
    // Row pairs need every channel staged with strips of at most R2_W columns
    // (multiples of 4) and, with periodic x, nx a multiple of 4; otherwise the
    // batch takes the one-row kernel with strips of up to STRIP columns.
    const int wopt = b->W_opt > 0 ? b->W_opt : STRIP;
    auto plan_strips = [&](int wmax) {
        long long U = 0;
        bool all4 = true, r2ok = true;
        for (auto &c : b->ch) {
            const int nx = c.grid.nx;
            const int W = lbm::strip_width(nx, std::min(wopt, wmax), b->bc_x);
            c.W = W;
            c.nstrips = (nx + W - 1) / W;
            c.yf0 = b->walls ? 1 : 0;
            c.nyf = b->walls ? c.grid.ny - 2 : c.grid.ny;
            c.units = (long long)c.nstrips * c.nyf;
            // bands never start at the row pair ny-3|ny-2 (rows 1|2 need band >= 2)
            c.band = b->band_opt > 0 ? std::min(c.nyf, std::max(8, b->band_opt)) : c.nyf;
            if (b->walls)
                while (c.band < c.nyf && (c.nyf - 1) % c.band == 0) ++c.band;
            c.nbands = (c.nyf + c.band - 1) / c.band;
            c.unit_base = U;
            U += c.units;
            all4 = all4 && (c.pitch % 4 == 0) && (W % 4 == 0);
            r2ok = r2ok && (b->bc_x || nx % 4 == 0);
        }
        b->staged = b->allow_staged && all4;
        return std::make_pair(U, r2ok && b->staged);
    };
    long long U = 0;
    b->rows2 = false;
    if (b->allow_rows2 && b->precision == 32 && lbm::cols_per_thread<float, true>() == 1) {
        auto r = plan_strips(lbm::R2_W);
        U = r.first;
        b->rows2 = r.second;
    }
    if (!b->rows2) U = plan_strips(STRIP).first;
    const size_t smem = step_smem(b);
    cudaError_t e = cudaFuncSetAttribute(batch_kernel(b), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return bfail(b, e, "smem attribute");
    int per_sm = b->ctas_per_sm_opt;
    if (per_sm <= 0) {
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel(b), step_threads(b), smem);
        if (e != cudaSuccess) return bfail(b, e, "occupancy");
        per_sm = std::max(1, occ);
    }
    // persistent stepping needs every CTA resident at once (cooperative launch)
    b->persist = false;
    if (b->rows2 && b->allow_persist) {
        int dev = 0, coop = 0, occ = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(persist_kernel(b), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persist_kernel(b), step_threads(b), smem);
        if (e != cudaSuccess) return bfail(b, e, "persistent kernel set-up");
        if (coop && occ > 0) {
            b->persist = true;
            per_sm = std::min(per_sm, occ);
        }
    }
    b->per_sm = per_sm;
    long long G = (long long)b->sms * per_sm;
    G = std::min<long long>(G, std::max<long long>(1, U / 2));
    G = std::min<long long>(G, lbm::MAX_CTAS);
    b->nctas = (int)std::max<long long>(1, G);

    // unit u -> (channel, strip, row) in the band-major order of each
    // channel; `piece_end`: the first unit after u's (band, strip) piece
    auto locate = [&](long long u, int &ci, int &s, int &row, long long *piece_end = nullptr) {
        ci = 0;
        while (ci + 1 < b->n && b->ch[ci + 1].unit_base <= u) ++ci;
        const ChanHost &c = b->ch[ci];
        const long long r = u - c.unit_base, full = (long long)c.nstrips * c.band;
        int j = (int)std::min<long long>(r / full, c.nbands - 1);
        const int h = j == c.nbands - 1 ? c.nyf - j * c.band : c.band;
        const long long rem = r - (long long)j * full;
        s = (int)(rem / h);
        row = c.yf0 + j * c.band + (int)(rem - (long long)s * h);
        if (piece_end) *piece_end = c.unit_base + (long long)j * full + (long long)(s + 1) * h;
    };
    auto cut = [&](long long k) {
        long long u = (k * U) / b->nctas;
        if (b->walls && u > 0 && u < U) {
            int ci, s, row;
            locate(u, ci, s, row);
            // one row back from ny-2 is ny-3, which is row 2 itself when ny = 5
            if (row == b->ch[ci].grid.ny - 2) { u -= 1; --row; }
            if (row == 2) u -= 1;
        }
        return u;
    };
    b->segs.clear();
    std::vector<int> begin(b->nctas + 1, 0);
    for (int k = 0; k < b->nctas; ++k) {
        begin[k] = (int)b->segs.size();
        long long u = cut(k), u1 = cut(k + 1);
        while (u < u1) {
            int ci, s, row;
            long long piece_end;
            locate(u, ci, s, row, &piece_end);
            const long long ue = std::min(u1, piece_end);
            b->segs.push_back(lbm::BatchSeg{ci, s, row, row + (int)(ue - u)});
            u = ue;
        }
    }
    begin[b->nctas] = (int)b->segs.size();
    if (b->band_opt < 0 && !b->persist) {
        // one CTA per strip column (no cuts), tallest first, so the hardware
        // scheduler hands the shorter columns to whichever CTA slot frees
        // (persistent stepping needs every CTA resident: the balanced cut)
        // (fewer columns than resident CTA slots: each column cut into equal
        // pieces, never between rows 1|2 or ny-3|ny-2, until the slots fill)
        long long ncol = 0;
        for (const auto &c : b->ch) ncol += c.nstrips;
        const long long slots = (long long)b->sms * per_sm;
        const int pieces = (int)std::max<long long>(1, (slots + ncol - 1) / std::max<long long>(1, ncol));
        b->segs.clear();
        for (int ci = 0; ci < b->n; ++ci) {
            const ChanHost &c = b->ch[ci];
            const int p = std::max(1, std::min(pieces, c.nyf / 8));
            for (int s2 = 0; s2 < c.nstrips; ++s2) {
                int ya = c.yf0;
                for (int k = 1; k <= p; ++k) {
                    int yb = c.yf0 + (int)((long long)k * c.nyf / p);
                    if (k < p && b->walls && yb == c.grid.ny - 2) --yb;
                    if (k < p && b->walls && yb == 2) --yb;
                    if (yb > ya) b->segs.push_back(lbm::BatchSeg{ci, s2, ya, yb});
                    ya = std::max(ya, yb);
                }
            }
        }
        std::stable_sort(b->segs.begin(), b->segs.end(), [](const lbm::BatchSeg &p, const lbm::BatchSeg &q) {
            return p.yb - p.ya > q.yb - q.ya;
        });
        b->nctas = (int)b->segs.size();
        begin.resize(b->nctas + 1);
        for (int k = 0; k <= b->nctas; ++k) begin[k] = k;
    }
    b->nseg = (int)b->segs.size();

    // device tables (re-allocated on every plan)
    cudaFree(b->d_segs);
    cudaFree(b->d_cta_begin);
    cudaFree(b->d_seg_mass);
    cudaFree(b->d_seg_J);
    cudaFree(b->d_seg_ext);
    b->d_segs = nullptr; b->d_cta_begin = nullptr; b->d_seg_mass = b->d_seg_J = nullptr; b->d_seg_ext = nullptr;
    const size_t ns = std::max(1, b->nseg);
    BCK(cudaMalloc((void **)&b->d_segs, ns * sizeof(lbm::BatchSeg)), "work list");
    BCK(cudaMalloc((void **)&b->d_cta_begin, (b->nctas + 1) * sizeof(int)), "work list");
    BCK(cudaMalloc((void **)&b->d_seg_mass, ns * sizeof(double)), "segment slots");
    BCK(cudaMalloc((void **)&b->d_seg_J, ns * sizeof(double)), "segment slots");
    BCK(cudaMalloc(&b->d_seg_ext, ns * 4 * sz_of(b)), "segment slots");
    cudaFree(b->d_done);
    cudaFree(b->d_abort);
    cudaFree(b->d_dep_beg);
    cudaFree(b->d_dep);
    b->d_done = b->d_abort = b->d_dep_beg = b->d_dep = nullptr;
    if (b->persist) {
        std::vector<int> dbeg, dep;
        build_deps(b, dbeg, dep);
        BCK(cudaMalloc((void **)&b->d_done, ns * sizeof(int)), "step counters");
        BCK(cudaMalloc((void **)&b->d_abort, sizeof(int)), "step counters");
        BCK(cudaMalloc((void **)&b->d_dep_beg, dbeg.size() * sizeof(int)), "dependencies");
        BCK(cudaMalloc((void **)&b->d_dep, std::max<size_t>(1, dep.size()) * sizeof(int)), "dependencies");
        BCK(cudaMemcpyAsync(b->d_dep_beg, dbeg.data(), dbeg.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream),
            "dependencies");
        if (!dep.empty())
            BCK(cudaMemcpyAsync(b->d_dep, dep.data(), dep.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream),
                "dependencies");
        BCK(cudaStreamSynchronize(b->stream), "dependencies");  // the host vectors die here
    }
    BCK(cudaMemcpyAsync(b->d_segs, b->segs.data(), b->nseg * sizeof(lbm::BatchSeg), cudaMemcpyHostToDevice,
                        b->stream), "work list copy");
    BCK(cudaMemcpyAsync(b->d_cta_begin, begin.data(), (b->nctas + 1) * sizeof(int), cudaMemcpyHostToDevice,
                        b->stream), "work list copy");
    if (b->precision == 64)
        lbm::reset_acc_kernel<double><<<(b->nseg + 255) / 256, 256, 0, b->stream>>>(
            b->d_seg_mass, b->d_seg_J, (double *)b->d_seg_ext, b->d_err, b->nseg);
    else
        lbm::reset_acc_kernel<float><<<(b->nseg + 255) / 256, 256, 0, b->stream>>>(
            b->d_seg_mass, b->d_seg_J, (float *)b->d_seg_ext, b->d_err, b->nseg);
    BCK(cudaGetLastError(), "reset");
    BCK(cudaStreamSynchronize(b->stream), "plan sync");
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return LBM_OK;
}

template <typename real>
cudaError_t batch_launch(lbm_batch *b)
{
    lbm::KArgs<real> A = physics_args<real>(b);
    A.fin = reinterpret_cast<const real *>(b->pop[b->cur]);
    A.fout = reinterpret_cast<real *>(b->pop[1 - b->cur]);
    const lbm::BatchChan<real> *chans = static_cast<const lbm::BatchChan<real> *>(b->d_chan);
    real *ext = static_cast<real *>(b->d_seg_ext);
    // the row-pair kernel takes one more argument: the source buffer's tensor maps
    const CUtensorMap *tm = b->tma_ok && b->allow_tma ? b->d_tmaps + (size_t)b->cur * b->n : nullptr;
    void *args[] = {(void *)&A, (void *)&chans, (void *)&b->d_segs, (void *)&b->d_cta_begin,
                    (void *)&b->d_seg_mass, (void *)&b->d_seg_J, (void *)&ext, b->rows2 ? (void *)&tm : nullptr};
    return cudaLaunchKernel(batch_kernel(b), dim3(b->nctas), dim3(step_threads(b)), args, step_smem(b), b->stream);
}

// Persistent stepping: `steps` steps of every channel in one cooperative launch.
cudaError_t persistent_steps(lbm_batch *b, int steps)
{
    lbm::KArgs<float> A = physics_args<float>(b);
    const lbm::BatchChan<float> *chans = static_cast<const lbm::BatchChan<float> *>(b->d_chan);
    float *ext = static_cast<float *>(b->d_seg_ext);
    const CUtensorMap *tm = b->tma_ok && b->allow_tma ? b->d_tmaps : nullptr;
    float *buf0 = reinterpret_cast<float *>(b->pop[0]), *buf1 = reinterpret_cast<float *>(b->pop[1]);
    int nchan = b->n, cur0 = b->cur;
    cudaError_t e = cudaMemsetAsync(b->d_done, 0, (size_t)std::max(1, b->nseg) * sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_abort, 0, sizeof(int), b->stream);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&A, (void *)&chans, (void *)&b->d_segs, (void *)&b->d_cta_begin, (void *)&b->d_seg_mass,
                    (void *)&b->d_seg_J, (void *)&ext, (void *)&tm, (void *)&nchan, (void *)&b->d_dep_beg,
                    (void *)&b->d_dep, (void *)&b->d_done, (void *)&b->d_abort, (void *)&buf0, (void *)&buf1,
                    (void *)&cur0, (void *)&steps};
    e = cudaLaunchCooperativeKernel(persist_kernel(b), dim3(b->nctas), dim3(step_threads(b)), args, step_smem(b),
                                    b->stream);
    if (e == cudaSuccess) {
        b->cur ^= steps & 1;
        b->step += steps;
    }
    return e;
}

cudaError_t one_step(lbm_batch *b)
{
    cudaError_t e = b->precision == 64 ? batch_launch<double>(b) : batch_launch<float>(b);
    if (e == cudaSuccess) {
        b->cur = 1 - b->cur;
        b->step += 1;
    }
    return e;
}

lbm_status build_graph(lbm_batch *b)
{
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    const int cur0 = b->cur;
    const int64_t step0 = b->step;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < b->graph_steps && e == cudaSuccess; ++s) e = one_step(b);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    b->cur = cur0;  // capture records; nothing ran
    b->step = step0;
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return bfail(b, e, "graph capture launch"); }
    if (e2 != cudaSuccess) return bfail(b, e2, "graph end capture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->graph = nullptr; return bfail(b, e, "graph instantiate"); }
    return LBM_OK;
}

template <typename real>
void fill_chan_table(const lbm_batch *b, std::vector<unsigned char> &buf)
{
    buf.resize(b->n * sizeof(lbm::BatchChan<real>));
    auto *t = reinterpret_cast<lbm::BatchChan<real> *>(buf.data());
    for (int i = 0; i < b->n; ++i) {
        const ChanHost &c = b->ch[i];
        t[i] = lbm::BatchChan<real>{c.off, c.grid.nx, c.grid.ny, c.W, c.pitch, (real)c.rho_in, (real)c.rho_in_l,
                                    (real)c.rho_out, (real)c.rho_out_l};
    }
}

lbm_status upload_chan_table(lbm_batch *b)
{
    std::vector<unsigned char> buf;
    if (b->precision == 64) fill_chan_table<double>(b, buf); else fill_chan_table<float>(b, buf);
    if (!b->d_chan) BCK(cudaMalloc(&b->d_chan, buf.size()), "channel table");
    BCK(cudaMemcpyAsync(b->d_chan, buf.data(), buf.size(), cudaMemcpyHostToDevice, b->stream), "channel table");
    BCK(cudaStreamSynchronize(b->stream), "channel table sync");
    return LBM_OK;
}

// Macroscopic fields of one channel with the single-channel kernel in fields mode.
template <typename real>
lbm_status chan_fields(lbm_batch *b, int ci, void *rho, void *ux, void *uy, void *tw, void *pw)
{
    const ChanHost &c = b->ch[ci];
    const size_t N = (size_t)c.grid.nx * c.grid.ny, nx = c.grid.nx, sz = sizeof(real);
    const size_t need = (3 * N + 4 * nx) * sz + 256;
    if (b->fscratch_bytes < need) {
        cudaFree(b->fscratch);
        b->fscratch = nullptr;
        BCK(cudaMalloc((void **)&b->fscratch, need), "fields scratch");
        b->fscratch_bytes = need;
    }
    real *d_rho = (real *)b->fscratch, *d_vx = d_rho + N, *d_vy = d_vx + N, *d_tw = d_vy + N, *d_pw = d_tw + 2 * nx;
    BCK(cudaMemsetAsync(b->fscratch, 0, need, b->stream), "fields memset");
    lbm::KArgs<real> A = physics_args<real>(b);
    A.fin = reinterpret_cast<const real *>(b->pop[b->cur]) + c.off;
    A.fout = nullptr;
    A.plane = (long long)N;
    A.nx = c.grid.nx;
    A.ny = c.grid.ny;
    A.pitch = c.pitch;
    A.W = c.W;
    A.nstrips = c.nstrips;
    A.yf0 = c.yf0;
    A.nyf = c.nyf;
    A.units = c.units;
    A.band = c.nyf;  // strip-major
    A.rho_in_g = (real)c.rho_in;
    A.rho_in_l = (real)c.rho_in_l;
    A.rho_out_g = (real)c.rho_out;
    A.rho_out_l = (real)c.rho_out_l;
    A.o_rho = d_rho; A.o_vx = d_vx; A.o_vy = d_vy; A.o_tw = d_tw; A.o_pw = d_pw;
    const bool st = b->allow_staged && c.pitch % 4 == 0 && c.W % 4 == 0;
    void *fn = lbm_step_kernel_ptr(b->precision, lbm::MODE_FIELDS, b->walls, b->bc_x, st, c.pitch != c.grid.nx);
    const size_t smem = staged_bytes(b, st);
    BCK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attribute");
    A.nctas = (int)std::max<long long>(1, std::min<long long>((long long)b->sms * 4, c.units / 2));
    void *args[] = {(void *)&A};
    BCK(cudaLaunchKernel(fn, dim3(A.nctas), dim3(cta_threads(b->precision, st)), args, smem, b->stream),
        "fields launch");
    struct { void *dst; real *src; size_t n; } outs[] = {
        {rho, d_rho, N}, {ux, d_vx, N}, {uy, d_vy, N}, {tw, d_tw, 2 * nx}, {pw, d_pw, 2 * nx}};
    for (auto &o : outs)
        if (o.dst) BCK(cudaMemcpyAsync(o.dst, o.src, o.n * sz, cudaMemcpyDefault, b->stream), "fields copy");
    BCK(cudaStreamSynchronize(b->stream), "fields sync");
    return LBM_OK;
}

} // namespace

extern "C" {

lbm_status lbm_batch_init(int32_t n, const lbm_grid *grids, const lbm_eos *eos, double tau, double wetting,
                          const lbm_drive *drives, const double *const *rho0s, void *stream, lbm_batch **out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (n <= 0 || !grids || !eos || !rho0s) return LBM_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const lbm_grid &g = grids[i];
        if (lbm_workspace_bytes(&g) == 0 || !lbm::idx32_ok(g.nx, g.ny) || !rho0s[i]) return LBM_ERR_ARG;
        if (g.precision != grids[0].precision || g.walls != grids[0].walls || g.bc_x != grids[0].bc_x)
            return LBM_ERR_ARG;
    }
    if (!(tau > 0.5) || !(eos->k > 0) || !(eos->kappa >= 0) || !(eos->a > 0) || !(eos->b > 0) ||
        !(eos->R > 0) || !(eos->T_over_Tc > 0) || !std::isfinite(wetting))
        return LBM_ERR_PARAM;

    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->n = n;
    b->precision = grids[0].precision;
    b->walls = grids[0].walls;
    b->bc_x = grids[0].bc_x;
    b->eos = *eos;
    b->tau = tau;
    b->wet = wetting;
    lbm::ChannelThermo ct0;
    const lbm_drive none{0.0, NAN, 0.0, 0.0};
    if (lbm::channel_thermo(*eos, none, false, &ct0)) { lbm_batch_free(b); return LBM_ERR_PARAM; }
    b->th = ct0.th;
    b->T = ct0.T; b->Tc = ct0.Tc;
    b->rho_g = ct0.rho_g; b->rho_l = ct0.rho_l; b->p_sat = ct0.p_sat;
    b->ch.resize(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        ChanHost &c = b->ch[i];
        c.grid = grids[i];
        if (drives) c.drive = drives[i];
        else c.drive = none;
        if (b->bc_x) {
            lbm::ChannelThermo ct;
            if (lbm::channel_thermo(*eos, c.drive, true, &ct)) { lbm_batch_free(b); return LBM_ERR_PARAM; }
            c.rho_in = ct.rho_in; c.rho_out = ct.rho_out;
            c.rho_in_l = ct.rho_in_l; c.rho_out_l = ct.rho_out_l;
        }
        c.pitch = lbm::pitch_of(c.grid.nx);
        c.off = (long long)off;
        off += align_elems((size_t)9 * c.pitch * c.grid.ny);
    }
    b->pop_elems = off;
    b->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!b->stream) {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t bytes = off * sz_of(b);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->pop[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->pop[1], bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_diag, (size_t)n * 7 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_err, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->err_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
    if (e != cudaSuccess) {
        lbm_status s = bfail(b, e, "allocation");
        lbm_batch_free(b);
        return s;
    }
    *b->h_err = 0;
    // initial states f = f_eq(rho0, 0), one channel at a time
    double *d_rho0 = nullptr;
    size_t max_nodes = 0;
    for (auto &c : b->ch) max_nodes = std::max(max_nodes, (size_t)c.grid.nx * c.grid.ny);
    e = cudaMalloc((void **)&d_rho0, max_nodes * sizeof(double));
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const ChanHost &c = b->ch[i];
        const int N = c.grid.nx * c.grid.ny;
        e = cudaMemcpyAsync(d_rho0, rho0s[i], (size_t)N * sizeof(double), cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) break;
        const int blocks = std::min((c.pitch * c.grid.ny + 255) / 256, b->sms * 8);
        if (b->precision == 64)
            lbm::init_kernel<double><<<blocks, 256, 0, b->stream>>>(d_rho0, (double *)b->pop[0] + c.off,
                                                                   (double *)b->pop[1] + c.off, c.grid.nx,
                                                                   c.pitch, c.grid.ny);
        else
            lbm::init_kernel<float><<<blocks, 256, 0, b->stream>>>(d_rho0, (float *)b->pop[0] + c.off,
                                                                  (float *)b->pop[1] + c.off, c.grid.nx,
                                                                  c.pitch, c.grid.ny);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // d_rho0 is reused
    }
    cudaFree(d_rho0);
    if (e != cudaSuccess) {
        lbm_status s = bfail(b, e, "init");
        lbm_batch_free(b);
        return s;
    }
    if (b->precision == 32) {
        // tensor maps of every channel in both buffers, for the row-pair stage
        std::vector<CUtensorMap> maps((size_t)2 * n);
        bool ok = true;
        for (int k = 0; k < 2 && ok; ++k)
            for (int i = 0; i < n && ok; ++i) {
                const ChanHost &c = b->ch[i];
                ok = lbm_encode_population_map(&maps[(size_t)k * n + i], (float *)b->pop[k] + c.off, c.pitch,
                                               c.grid.ny);
            }
        if (ok && cudaMalloc((void **)&b->d_tmaps, maps.size() * sizeof(CUtensorMap)) == cudaSuccess &&
            cudaMemcpy(b->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) ==
                cudaSuccess)
            b->tma_ok = true;
        else
            cudaGetLastError();  // plane copies instead
    }
    lbm_status s = batch_plan(b);
    if (s == LBM_OK) s = upload_chan_table(b);
    if (s != LBM_OK) { lbm_batch_free(b); return s; }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, int64_t n)
{
    if (!b || n < 0) return LBM_ERR_ARG;
    lbm_status flag = LBM_OK;
    if (b->err_pending && cudaEventQuery(b->err_ev) == cudaSuccess) {
        b->err_pending = false;
        // bit 0: bad density; bit 1: a bounded stage wait gave up
        if (*b->h_err & 1) flag = LBM_ERR_NAN;
        else if (*b->h_err) flag = LBM_ERR_TIMEOUT;
    }
    while (n > 0 && b->persist) {
        const int chunk = (int)std::min<int64_t>(n, 4096);
        BCK(persistent_steps(b, chunk), "persistent launch");
        n -= chunk;
    }
    while (n > 0) {
        if (b->graph_steps > 0 && n >= b->graph_steps && b->cur == 0) {
            if (!b->graph) {
                lbm_status s = build_graph(b);
                if (s != LBM_OK) return s;
            }
            BCK(cudaGraphLaunch(b->graph, b->stream), "graph launch");
            b->step += b->graph_steps;
            n -= b->graph_steps;
        } else {
            BCK(one_step(b), "step launch");
            n -= 1;
        }
    }
    if (!b->err_pending) {
        BCK(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "error flag");
        BCK(cudaEventRecord(b->err_ev, b->stream), "error flag");
        b->err_pending = true;
    }
    return flag;
}

lbm_status lbm_batch_fields(lbm_batch *b, int32_t channel, void *rho, void *ux, void *uy, void *tau_wall,
                            void *p_wall)
{
    if (!b || channel < 0 || channel >= b->n) return LBM_ERR_ARG;
    return b->precision == 64 ? chan_fields<double>(b, channel, rho, ux, uy, tau_wall, p_wall)
                              : chan_fields<float>(b, channel, rho, ux, uy, tau_wall, p_wall);
}

lbm_status lbm_batch_diag(lbm_batch *b, int32_t channel, lbm_diag_t *out)
{
    if (!b || !out || channel < 0 || channel >= b->n) return LBM_ERR_ARG;
    if (b->precision == 64)
        lbm::batch_diag_kernel<double><<<(b->n + 63) / 64, 64, 0, b->stream>>>(
            b->d_seg_mass, b->d_seg_J, (const double *)b->d_seg_ext, b->d_segs, b->nseg, b->n, b->d_err, b->d_diag);
    else
        lbm::batch_diag_kernel<float><<<(b->n + 63) / 64, 64, 0, b->stream>>>(
            b->d_seg_mass, b->d_seg_J, (const float *)b->d_seg_ext, b->d_segs, b->nseg, b->n, b->d_err, b->d_diag);
    BCK(cudaGetLastError(), "diag launch");
    double h[7];
    BCK(cudaMemcpyAsync(h, b->d_diag + 7 * channel, sizeof h, cudaMemcpyDeviceToHost, b->stream), "diag copy");
    BCK(cudaStreamSynchronize(b->stream), "diag sync");
    const ChanHost &c = b->ch[channel];
    std::memset(out, 0, sizeof *out);
    out->step = b->step;
    out->mass = b->step > 0 ? h[0] : 0.0;
    out->wall_shear_sum = h[1];
    const bool any = b->step > 0 && b->walls;
    out->tau_wall_min = any ? h[2] : 0.0;
    out->tau_wall_max = any ? h[3] : 0.0;
    out->p_wall_min = any ? h[4] : 0.0;
    out->p_wall_max = any ? h[5] : 0.0;
    out->nan_detected = ((int)h[6] & 1) != 0;
    out->T = b->T; out->Tc = b->Tc; out->rho_g = b->rho_g; out->rho_l = b->rho_l; out->p_sat = b->p_sat;
    out->rho_in = c.rho_in; out->rho_out = c.rho_out; out->rho_in_l = c.rho_in_l; out->rho_out_l = c.rho_out_l;
    return LBM_OK;
}

lbm_status lbm_batch_reset_diag(lbm_batch *b)
{
    if (!b) return LBM_ERR_ARG;
    if (b->precision == 64)
        lbm::reset_acc_kernel<double><<<(b->nseg + 255) / 256, 256, 0, b->stream>>>(
            b->d_seg_mass, b->d_seg_J, (double *)b->d_seg_ext, nullptr, b->nseg);
    else
        lbm::reset_acc_kernel<float><<<(b->nseg + 255) / 256, 256, 0, b->stream>>>(
            b->d_seg_mass, b->d_seg_J, (float *)b->d_seg_ext, nullptr, b->nseg);
    BCK(cudaGetLastError(), "reset diag");
    return LBM_OK;
}

lbm_status lbm_batch_populations(lbm_batch *b, int32_t channel, void *dst)
{
    if (!b || !dst || channel < 0 || channel >= b->n) return LBM_ERR_ARG;
    const ChanHost &c = b->ch[channel];
    const size_t sz = sz_of(b), nx = c.grid.nx, ny = c.grid.ny, row = nx * sz, prow = (size_t)c.pitch * sz;
    const char *src = (const char *)b->pop[b->cur] + c.off * sz;
    for (int i = 0; i < 9; ++i)
        BCK(cudaMemcpy2DAsync((char *)dst + i * nx * ny * sz, row, src + i * prow, 9 * prow, row, ny,
                              cudaMemcpyDefault, b->stream), "populations copy");
    BCK(cudaStreamSynchronize(b->stream), "populations sync");
    return LBM_OK;
}

lbm_status lbm_batch_set_collision(lbm_batch *b, const lbm_collision *c)
{
    if (!b) return LBM_ERR_ARG;
    const lbm_collision next = c ? *c : lbm_collision{};
    if (next.kind == LBM_COLL_MRT) {
        for (double r : {next.s_e, next.s_eps, next.s_j, next.s_q})
            if (!(r > 0.0 && r < 2.0)) return LBM_ERR_ARG;
        if (std::isnan(next.s_nu) || !(next.s_nu <= 0.0 || next.s_nu < 2.0)) return LBM_ERR_ARG;
    } else if (next.kind != LBM_COLL_BGK) {
        return LBM_ERR_ARG;
    }
    b->coll = next;
    // the captured graph holds the old kernel arguments
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    return LBM_OK;
}

lbm_status lbm_batch_set_option(lbm_batch *b, lbm_option opt, int64_t value)
{
    if (!b) return LBM_ERR_ARG;
    switch (opt) {
    case LBM_OPT_CTAS_PER_SM:
        if (value < 0 || value > 32) return LBM_ERR_ARG;
        b->ctas_per_sm_opt = (int)value;
        break;
    case LBM_OPT_REVERSE:
        b->reverse = value != 0;
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        return LBM_OK;
    case LBM_OPT_STRIP:
        if (value < 2 || value > STRIP) return LBM_ERR_ARG;
        b->W_opt = (int)value;
        break;
    case LBM_OPT_STAGED:
        b->allow_staged = value != 0;
        break;
    case LBM_OPT_ROWS2:
        b->allow_rows2 = value != 0;
        break;
    case LBM_OPT_TMA:
        b->allow_tma = value != 0;
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }  // captured arguments
        return LBM_OK;
    case LBM_OPT_PREFETCH:
        if (value < 0 || value > 4) return LBM_ERR_ARG;
        b->pf = (int)value;
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }  // captured arguments
        return LBM_OK;
    case LBM_OPT_PERSISTENT:
        b->allow_persist = value != 0;
        break;
    case LBM_OPT_BAND:
        if (value < -1 || value > (1 << 20)) return LBM_ERR_ARG;
        b->band_opt = (int)value;
        break;
    case LBM_OPT_GRAPH_STEPS:
        if (value < 0 || (value & 1)) return LBM_ERR_ARG;
        b->graph_steps = (int)value;
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        return LBM_OK;
    default:
        return LBM_ERR_ARG;
    }
    lbm_status s = batch_plan(b);
    return s == LBM_OK ? upload_chan_table(b) : s;
}

lbm_status lbm_batch_launch_info(const lbm_batch *b, int64_t *ctas, int64_t *segments, int64_t *staged,
                                 int64_t *strip)
{
    if (!b) return LBM_ERR_ARG;
    if (ctas) *ctas = b->nctas;
    if (segments) *segments = b->nseg;
    if (staged) *staged = b->staged ? 1 : 0;
    if (strip) *strip = b->W_opt > 0 ? b->W_opt : STRIP;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int32_t trial_steps, int64_t *best_ctas_per_sm,
                              int64_t *best_strip, double *best_ms_per_step)
{
    if (!b || trial_steps < 2) return LBM_ERR_ARG;
    // the trials advance the state: keep a copy and put it back afterwards
    const size_t bytes = b->pop_elems * sz_of(b);
    unsigned char *save = nullptr;
    BCK(cudaMalloc((void **)&save, 2 * bytes), "autotune copy");
    BCK(cudaMemcpyAsync(save, b->pop[0], bytes, cudaMemcpyDeviceToDevice, b->stream), "autotune copy");
    BCK(cudaMemcpyAsync(save + bytes, b->pop[1], bytes, cudaMemcpyDeviceToDevice, b->stream), "autotune copy");
    const int cur0 = b->cur;
    const int64_t step0 = b->step;
    const int keep_graph = b->graph_steps;
    b->graph_steps = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int occ_max = 1;
    bool whole = false;  // whole strip columns: CTAs per SM is the occupancy, not a choice
    {
        b->ctas_per_sm_opt = 0;
        b->W_opt = 0;
        lbm_status s = batch_plan(b);
        if (s != LBM_OK) { cudaFree(save); return s; }
        occ_max = std::max(1, (int)((b->nctas + b->sms - 1) / b->sms));
        whole = b->band_opt < 0 && !b->persist;
    }
    double best = 1e300;
    int best_c = 0, best_w = 0;
    const int strips[] = {128, 64};
    for (int w : strips) {
        if (w > STRIP) continue;
        for (int c = whole ? 0 : std::max(1, occ_max - 2); c <= (whole ? 0 : occ_max); ++c) {
            b->ctas_per_sm_opt = c;
            b->W_opt = w;
            if (batch_plan(b) != LBM_OK) continue;
            upload_chan_table(b);
            // time the plan the way lbm_batch_step will run it
            if (b->persist) persistent_steps(b, 2);  // warm-up
            else one_step(b);
            cudaEventRecord(e0, b->stream);
            if (b->persist) persistent_steps(b, trial_steps);
            else
                for (int s = 0; s < trial_steps; ++s) one_step(b);
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per = ms / trial_steps;
            if (per < best) { best = per; best_c = c; best_w = w; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->ctas_per_sm_opt = best_c;
    b->W_opt = best_w;
    b->graph_steps = keep_graph;
    lbm_status s = batch_plan(b);  // also clears the diagnostic slots
    if (s == LBM_OK) s = upload_chan_table(b);
    BCK(cudaMemcpyAsync(b->pop[0], save, bytes, cudaMemcpyDeviceToDevice, b->stream), "autotune restore");
    BCK(cudaMemcpyAsync(b->pop[1], save + bytes, bytes, cudaMemcpyDeviceToDevice, b->stream), "autotune restore");
    BCK(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream), "autotune restore");
    BCK(cudaStreamSynchronize(b->stream), "autotune sync");
    cudaFree(save);
    b->cur = cur0;
    b->step = step0;
    b->err_pending = false;
    if (best_ctas_per_sm) *best_ctas_per_sm = whole ? b->per_sm : best_c;
    if (best_strip) *best_strip = best_w;
    if (best_ms_per_step) *best_ms_per_step = best;
    return s;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->last_error : ""; }

void lbm_batch_free(lbm_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->pop[0]);
    cudaFree(b->pop[1]);
    cudaFree(b->d_tmaps);
    cudaFree(b->d_done);
    cudaFree(b->d_abort);
    cudaFree(b->d_dep_beg);
    cudaFree(b->d_dep);
    cudaFree(b->d_chan);
    cudaFree(b->d_segs);
    cudaFree(b->d_cta_begin);
    cudaFree(b->d_seg_mass);
    cudaFree(b->d_seg_J);
    cudaFree(b->d_seg_ext);
    cudaFree(b->d_err);
    cudaFree(b->d_diag);
    cudaFree(b->fscratch);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->err_ev) cudaEventDestroy(b->err_ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

} // extern "C"
