// aniso_api.cu -- host side of libaniso.so: handles, validation, the step
// schedule of Eq. op_2step, CUDA-graph capture, batches and diagnostics.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/aniso.h"
#include "aniso_internal.h"
#include "status.h"
#include "line5_types.h"

// NVTX range around a public call, for timeline tools (a no-op without one).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
};

using namespace aniso;

// ------------------------------------------------------------- errors

static thread_local std::string g_last_error;

extern "C" const char *aniso_last_error(void) { return g_last_error.c_str(); }

// Lets other translation units of the library report through aniso_last_error.
void aniso::record_error(const char *msg) { g_last_error = msg; }

// ------------------------------------------------------------- profiling

struct EventPair {
    cudaEvent_t a, b;
    int kind;
};

struct Profiler {
    std::vector<EventPair> pool;   // all pairs ever created
    std::vector<int> pending;      // indices whose timings have not been read
    size_t next = 0;               // next free pair for a direct (non-graph) launch
    double ms[3] = {0, 0, 0};
    long long count[3] = {0, 0, 0};

    int take(int kind)
    {
        if (next == pool.size()) {
            EventPair p;
            p.kind = kind;
            if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) return -1;
            pool.push_back(p);
        }
        pool[next].kind = kind;
        return (int)next++;
    }
    int drain()
    {
        for (int idx : pending) {
            float t = 0.f;
            cudaError_t e = cudaEventElapsedTime(&t, pool[idx].a, pool[idx].b);
            if (e != cudaSuccess) return fail(ANISO_ERR_CUDA, "event timing: %s", cudaGetErrorString(e));
            ms[pool[idx].kind] += t;
            count[pool[idx].kind] += 1;
        }
        pending.clear();
        return ANISO_OK;
    }
    void destroy()
    {
        for (auto &p : pool) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        pool.clear();
        pending.clear();
        next = 0;
    }
};

// ------------------------------------------------------------- handle

struct aniso_ctx {
    int nx = 0, ny = 0, bc = 0;
    double dx = 0, dy = 0, chi_par = 0, chi_perp = 0;
    int prec = PREC_FP64, field_fp16 = 0, kahan = 0, limiter = LIM_VANLEER, order = ANISO_ORDER_XY;
    int use_graph = 1, profile = 0, fast = 3, seg_chunks = 0, l4_warps = 0, scheme = 0, diag = 0;
    int tma_lines = 0;  // ANISO_OPT_TMA_LINES
    int tmem = 1;       // ANISO_OPT_TMEM
    int cluster = 2;    // ANISO_OPT_CLUSTER_LINES
    double nl_alpha = 0, nl_tref = 1;  // temperature-dependent diffusivity (aniso_set_nonlinear)
    void *t4 = nullptr;  // intermediate of the 4-step scheme
    void *q = nullptr;   // source term (aniso_set_source), handle precision
    cudaStream_t stream = 0;
    long long step_counter = 0;
    bool field_set = false;
    // device buffers
    void *cxx = nullptr, *cxy = nullptr, *cyy = nullptr, *cyx = nullptr;
    void *cyyT = nullptr, *cyxT = nullptr;  // transposed y coefficients (long columns)
    void *tstar = nullptr;                  // intermediate T* of a step
    void *tA = nullptr, *tB = nullptr;      // transposed scratch (long columns)
    // compensated (Kahan) low parts: of T, of T*, of the transposed scratch
    void *tlo = nullptr, *tstar_lo = nullptr, *tAlo = nullptr, *tBlo = nullptr;
    // compensated state on the cluster kernel: hi and lo interleaved by quads
    // of 4 cells (8 floats), the state between the steps of a call (kq, row
    // quads) and the intermediate (kqs, column quads)
    void *kq = nullptr, *kqs = nullptr;
    double *partials = nullptr, *result = nullptr;
    unsigned *err = nullptr;
    // graph cache
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_stream = nullptr;
    void *g_T = nullptr;
    double g_dt = 0;
    int g_nsteps = -1, g_parity = -1, g_order = -1, g_limiter = -1, g_profile = -1;
    std::vector<int> g_pairs;  // profiler pairs recorded by the graph
    Profiler prof;

    size_t cells() const { return (size_t)nx * ny; }
    size_t esz() const { return prec == PREC_FP64 ? 8 : 4; }
    size_t csz() const { return prec == PREC_FP64 ? 8 : (field_fp16 ? 2 : 4); }
    int coef_kind() const { return prec == PREC_FP64 ? 0 : (field_fp16 ? 2 : 1); }
    bool long_cols() const { return ny > MAX_COL; }
    // columns solved as transposed rows: long columns, and fixed-boundary grids
    // (only the general row kernel knows fixed boundary nodes)
    bool col_transpose() const { return long_cols() || bc == ANISO_BC_DIRICHLET; }
    bool dirichlet() const { return bc == ANISO_BC_DIRICHLET; }
    int vec() const { return prec == PREC_FP64 ? 2 : 4; }
    // Grid shapes the vectorised x-then-y path handles: both line lengths a
    // multiple of the 16-byte vector and short enough for transposed output.
    // 4: warp-per-line kernel (line4, option value 3); 6: line4 for the lines
    // it takes and the long-line kernel (line6, 2049-4096 cells, FP32) for
    // the others, x-then-y steps only; 7: as 6, with lines the cluster kernel
    // (line7) takes, or the compensated state on line7 in both directions;
    // 2: line2; 0: none of them.
    int long_kernel(int n) const
    {
        int a, b, c;
        size_t d;
        if (cluster == 2 && line7_config(prec, field_fp16, n, &a, &b, &d)) return 7;
        if (line6_config(prec, field_fp16, n, &a, &b, &c, &d)) return 6;
        if (cluster != 0 && line7_config(prec, field_fp16, n, &a, &b, &d)) return 7;
        return 0;
    }
    int fast_kind() const
    {
        int a, b, c;
        size_t d;
        if (kahan)
            return fast == 3 && cluster != 0 && line7_config(prec, field_fp16, nx, &a, &b, &d) &&
                           line7_config(prec, field_fp16, ny, &a, &b, &d)
                       ? 7
                       : 0;
        if (fast == 3) {
            const bool x4 = line4_config(prec, nx, true, l4_warps, seg_chunks, &a, &b, &c, &d);
            const bool y4 = line4_config(prec, ny, true, l4_warps, seg_chunks, &a, &b, &c, &d);
            if (x4 && y4) return 4;
            const int kx = x4 ? 4 : long_kernel(nx), ky = y4 ? 4 : long_kernel(ny);
            if (kx && ky) return (kx == 7 || ky == 7) ? 7 : 6;
        }
        if (line2_config(prec, nx, true, &a, &b, &c, &d, seg_chunks) &&
            line2_config(prec, ny, true, &a, &b, &c, &d, seg_chunks))
            return 2;
        return 0;
    }
    bool fast_shape() const { return fast_kind() != 0; }
    int max_line() const { return prec == PREC_FP64 ? MAX_LINE_FP64 : MAX_LINE_FP32; }
};

static void free_buffers(aniso_ctx *h)
{
    void **bufs[] = {&h->cxx, &h->cxy, &h->cyy,      &h->cyx,  &h->cyyT, &h->cyxT, &h->tstar,
                     &h->tA,  &h->tB,  &h->tlo, &h->tstar_lo, &h->tAlo, &h->tBlo, &h->t4,
                     &h->kq,  &h->kqs,
                     &h->q};
    for (void **b : bufs) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    }
    if (h->partials) cudaFree(h->partials);
    if (h->result) cudaFree(h->result);
    if (h->err) cudaFree(h->err);
    h->partials = h->result = nullptr;
    h->err = nullptr;
}

static void drop_graph(aniso_ctx *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->g_nsteps = -1;
    h->g_pairs.clear();
}

extern "C" int aniso_create(int nx, int ny, double dx, double dy, double chi_par, double chi_perp,
                            int bc, aniso_t *out)
{
    if (!out) return fail(ANISO_ERR_ARG, "aniso_create: out is NULL");
    *out = nullptr;
    if (nx < 3 || ny < 3) return fail(ANISO_ERR_ARG, "aniso_create: nx=%d ny=%d (need >= 3)", nx, ny);
    if (!(dx > 0) || !(dy > 0)) return fail(ANISO_ERR_ARG, "aniso_create: dx, dy must be > 0");
    if (!(chi_par > 0)) return fail(ANISO_ERR_ARG, "aniso_create: chi_par must be > 0");
    if (!(chi_perp >= 0) || chi_perp > chi_par)
        return fail(ANISO_ERR_ARG, "aniso_create: need 0 <= chi_perp <= chi_par");
    if (bc != ANISO_BC_ZEROFLUX && bc != ANISO_BC_PERIODIC && bc != ANISO_BC_DIRICHLET)
        return fail(ANISO_ERR_ARG, "aniso_create: unknown boundary condition %d", bc);
    aniso_ctx *h = new aniso_ctx;
    h->nx = nx;
    h->ny = ny;
    h->dx = dx;
    h->dy = dy;
    h->chi_par = chi_par;
    h->chi_perp = chi_perp;
    h->bc = bc;
    *out = h;
    return ANISO_OK;
}

extern "C" int aniso_set_option(aniso_t h, int key, long long v)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso_set_option: null handle");
    switch (key) {
    case ANISO_OPT_PRECISION:
        if (v != ANISO_PREC_FP64 && v != ANISO_PREC_FP32) return fail(ANISO_ERR_ARG, "bad precision %lld", v);
        if (h->field_set && v != h->prec) return fail(ANISO_ERR_STATE, "precision is fixed once the field is set");
        h->prec = (int)v;
        break;
    case ANISO_OPT_FIELD_FP16:
        if (h->field_set && (v != 0) != (h->field_fp16 != 0))
            return fail(ANISO_ERR_STATE, "field storage is fixed once the field is set");
        h->field_fp16 = v != 0;
        break;
    case ANISO_OPT_KAHAN:
        if (h->field_set && (v != 0) != (h->kahan != 0))
            return fail(ANISO_ERR_STATE, "compensated state is fixed once the field is set");
        if (v && h->scheme != ANISO_SCHEME_2STEP)
            return fail(ANISO_ERR_UNSUPPORTED, "the compensated state runs the 2-step scheme only");
        h->kahan = v != 0;
        break;
    case ANISO_OPT_SCHEME:
        if (v != ANISO_SCHEME_2STEP && v != ANISO_SCHEME_4STEP && v != ANISO_SCHEME_EXPLICIT)
            return fail(ANISO_ERR_ARG, "bad scheme %lld", v);
        if (v != ANISO_SCHEME_2STEP && h->kahan)
            return fail(ANISO_ERR_UNSUPPORTED, "the compensated state runs the 2-step scheme only");
        if (v == ANISO_SCHEME_4STEP && !h->t4) CU(cudaMalloc(&h->t4, h->cells() * 8));  // either precision
        h->scheme = (int)v;
        drop_graph(h);
        break;
    case ANISO_OPT_LIMITER:
        if (v < 0 || v > 3) return fail(ANISO_ERR_ARG, "bad limiter %lld", v);
        h->limiter = (int)v;
        break;
    case ANISO_OPT_ORDER:
        if (v < 0 || v > 2) return fail(ANISO_ERR_ARG, "bad order %lld", v);
        h->order = (int)v;
        break;
    case ANISO_OPT_STREAM:
        h->stream = (cudaStream_t)(intptr_t)v;
        drop_graph(h);
        break;
    case ANISO_OPT_GRAPH:
        h->use_graph = v != 0;
        break;
    case ANISO_OPT_PROFILE:
        if (v < 0 || v > (1 << 20)) return fail(ANISO_ERR_ARG, "bad profile value %lld", v);
        h->profile = (int)v;
        break;
    case ANISO_OPT_DIAGNOSTICS:
        h->diag = v != 0;
        break;
    case ANISO_OPT_TMEM:
        h->tmem = v != 0;
        break;
    case ANISO_OPT_CLUSTER_LINES:
        if (v < 0 || v > 2) return fail(ANISO_ERR_ARG, "bad cluster-lines value %lld", v);
        h->cluster = (int)v;
        drop_graph(h);
        break;
    case ANISO_OPT_TMA_LINES:
        if (v < 0 || v > 2) return fail(ANISO_ERR_ARG, "bad TMA-lines value %lld", v);
        h->tma_lines = (int)v;
        break;
    case ANISO_OPT_FAST_PATH:
        if (v < 0 || v > 3 || v == 2) return fail(ANISO_ERR_ARG, "bad fast-path value %lld", v);
        h->fast = (int)v;
        drop_graph(h);
        break;
    case ANISO_OPT_BLOCK_WARPS:
        if (v != 0 && v != 1 && v != 2 && v != 4 && v != 8)
            return fail(ANISO_ERR_ARG, "bad warps per block %lld (0, 1, 2, 4 or 8)", v);
        h->l4_warps = (int)v;
        drop_graph(h);
        break;
    case ANISO_OPT_SEGMENT:
        if (v < 0 || v > 64) return fail(ANISO_ERR_ARG, "bad segment length %lld", v);
        h->seg_chunks = (int)v;
        drop_graph(h);
        break;
    default:
        return fail(ANISO_ERR_ARG, "unknown option key %d", key);
    }
    return ANISO_OK;
}

extern "C" int aniso_set_field(aniso_t h, const void *bx, const void *by)
{
    TraceRange trace("aniso_set_field");
    if (!h) return fail(ANISO_ERR_ARG, "aniso_set_field: null handle");
    if (!bx || !by) return fail(ANISO_ERR_ARG, "aniso_set_field: null field pointer");
    if (h->field_fp16 && h->prec != PREC_FP32)
        return fail(ANISO_ERR_ARG, "aniso_set_field: FP16 field storage needs FP32 precision");
    if (h->kahan && h->prec != PREC_FP32)
        return fail(ANISO_ERR_ARG, "aniso_set_field: the compensated state needs FP32 precision");
    if (h->kahan && h->dirichlet())
        return fail(ANISO_ERR_UNSUPPORTED, "aniso_set_field: the compensated state needs a conserving boundary");
    if (h->nx > h->max_line() || (h->long_cols() && h->ny > h->max_line()))
        return fail(ANISO_ERR_UNSUPPORTED, "grid %dx%d exceeds the on-chip line limit %d", h->nx, h->ny,
                    h->max_line());
    if (!h->field_set) {
        const size_t n = h->cells();
        CU(cudaMalloc(&h->cxx, n * h->csz()));
        CU(cudaMalloc(&h->cxy, n * h->csz()));
        CU(cudaMalloc(&h->cyy, n * h->csz()));
        CU(cudaMalloc(&h->cyx, n * h->csz()));
        CU(cudaMalloc(&h->tstar, n * h->esz()));
        if (h->col_transpose() || h->fast_shape()) {
            CU(cudaMalloc(&h->cyyT, n * h->csz()));
            CU(cudaMalloc(&h->cyxT, n * h->csz()));
        }
        if (h->col_transpose()) {
            CU(cudaMalloc(&h->tA, n * h->esz()));
            CU(cudaMalloc(&h->tB, n * h->esz()));
        }
        if (h->kahan) {
            CU(cudaMalloc(&h->tlo, n * h->esz()));
            CU(cudaMalloc(&h->tstar_lo, n * h->esz()));
            CU(cudaMemsetAsync(h->tlo, 0, n * h->esz(), h->stream));
            if (h->col_transpose()) {
                CU(cudaMalloc(&h->tAlo, n * h->esz()));
                CU(cudaMalloc(&h->tBlo, n * h->esz()));
            }
        }
        CU(cudaMalloc(&h->partials, 4 * TOTALS_BLOCKS * sizeof(double)));
        CU(cudaMalloc(&h->result, 4 * sizeof(double)));
        CU(cudaMalloc(&h->err, sizeof(unsigned)));
        CU(cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->stream));
    }
    const double kappa = h->chi_perp / h->chi_par;
    CU(launch_face_coeffs(h->prec, h->coef_kind(), bx, by, h->nx, h->ny, h->bc, kappa, h->cxx, h->cxy,
                          h->cyy, h->cyx, h->cyyT, h->cyxT, h->stream));
    h->field_set = true;
    drop_graph(h);
    return ANISO_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// One vectorised line update (line2_kernel) of `nlines` lines of n cells.
static int enqueue_line2(aniso_ctx *h, const void *in, void *out, const void *g, const void *e, int n,
                         int nlines, int per_line, int per_cross, double lam, double mu, bool transposed,
                         int kind, cudaStream_t s, std::vector<int> *pairs, bool v4 = false,
                         const void *in_lo = nullptr, void *out_lo = nullptr, int ilv_in = 0, int ilv_out = 0)
{
    Line2Args a{};
    a.jobs = nullptr;
    a.njobs = 1;
    a.limiter = h->limiter;
    a.err = h->err;
    Line2Job &J = a.one;
    J.Tin = in;
    J.Tout = out;
    J.TinLo = in_lo;
    J.ToutLo = out_lo;
    J.g = g;
    J.e = e;
    J.lam = lam;
    J.mu = mu;
    J.n = n;
    J.nlines = nlines;
    J.per_line = per_line;
    J.per_cross = per_cross;
    J.transpose_out = transposed ? 1 : 0;
    J.ilv_in = ilv_in;
    J.ilv_out = ilv_out;
    if (v4 && h->nl_alpha != 0.0) {
        J.chi_alpha = h->nl_alpha;
        J.chi_itref = 1.0 / h->nl_tref;
    }
    int nthreads;
    size_t smem;
    bool ok = v4 ? line4_config(h->prec, n, transposed, h->l4_warps, h->seg_chunks, &J.team, &J.lines_per_block,
                                &nthreads, &smem)
                 : line2_config(h->prec, n, transposed, &J.team, &J.lines_per_block, &nthreads, &smem,
                                h->seg_chunks);
    if (v4 && ok) J.swz = line4_swizzle(h->prec, n, J.team);
    // lines above line4's limit: the long-line kernels (constant diffusivity
    // only); the compensated state runs on the cluster kernel alone
    if (v4 && in_lo) ok = false;
    const int lk = v4 && !ok && h->nl_alpha == 0.0 ? (in_lo ? 7 : h->long_kernel(n)) : 0;
    const bool v6 = lk == 6 && line6_config(h->prec, h->field_fp16, n, &J.team, &J.lines_per_block, &nthreads,
                                            &smem, h->l4_warps == 8 ? 2 : 4);
    int cs = 0;
    // (the plain state's tensor-memory form moves gamma out of shared memory;
    // the compensated one keeps it there, at two blocks an SM, and puts only
    // T_old in tensor memory)
    const bool v7 = lk == 7 && line7_config(h->prec, h->field_fp16, n, &cs, &nthreads, &smem,
                                            h->tmem != 0 && !in_lo);
    if (v7) {
        J.team = 64;
        J.lines_per_block = 4;
        a.tmem = h->tmem != 0 ? 1 : 0;
    }
    ok = ok || v6 || v7;
    if (!ok) return fail(ANISO_ERR_UNSUPPORTED, "vectorised line kernel cannot take n=%d", n);
    J.block0 = 0;
    J.nblocks = (nlines + J.lines_per_block - 1) / J.lines_per_block;
    int pidx = -1;
    const unsigned rec_flags = pairs ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (h->profile) {
        pidx = h->prof.take(kind);
        if (pidx < 0) return fail(ANISO_ERR_CUDA, "event creation failed");
        CU(cudaEventRecordWithFlags(h->prof.pool[pidx].a, s, rec_flags));
    }
    CU(v7   ? launch_line7(h->field_fp16, a, cs, smem, s)
       : v6 ? launch_line6(h->field_fp16, a, J.nblocks, nthreads, smem, s)
       : v4 ? launch_line4(h->prec, h->field_fp16, a, J.nblocks, nthreads, smem, s)
            : launch_line2(h->prec, h->field_fp16, a, J.nblocks, nthreads, smem, s, in_lo != nullptr));
    if (h->profile) {
        CU(cudaEventRecordWithFlags(h->prof.pool[pidx].b, s, rec_flags));
        if (pairs) pairs->push_back(pidx);
        else h->prof.pending.push_back(pidx);
    }
    return ANISO_OK;
}

// Fast path of one x-then-y step: the x-update reads T row-major and writes T*
// column-major; the y-update reads T*'s columns as contiguous lines (with the
// transposed y coefficients) and writes T back row-major.
// With the compensated state the low parts travel the same way (tlo <->
// tstar_lo), on the cluster kernel.
static bool use_fast(const aniso_ctx *h, const void *T)
{
    return h->fast && !h->dirichlet() && h->order == ANISO_ORDER_XY && h->cyyT && aligned16(T) &&
           aligned16(h->tstar) && (!h->kahan || (aligned16(h->tlo) && aligned16(h->tstar_lo))) &&
           h->fast_shape();
}

// One update of the fast path: dir 0 the x-update (T -> T*), 1 the y-update (T* -> T).
static int enqueue_fast_sweep(aniso_ctx *h, int dir, void *T, double dt, cudaStream_t s, std::vector<int> *pairs)
{
    const double mu = h->chi_par * dt / (h->dx * h->dy);
    const int per = h->bc == ANISO_BC_PERIODIC;
    const int fk = h->fast_kind();
    const bool v4 = fk == 4 || fk == 6 || fk == 7;  // line4, or a long-line kernel above its limit
    if (dir == 0)
        return enqueue_line2(h, T, h->tstar, h->cxx, h->cxy, h->nx, h->ny, per, per,
                             h->chi_par * dt / (h->dx * h->dx), mu, true, ANISO_KERNEL_XSWEEP, s, pairs, v4,
                             h->kahan ? h->tlo : nullptr, h->kahan ? h->tstar_lo : nullptr);
    return enqueue_line2(h, h->tstar, T, h->cyyT, h->cyxT, h->ny, h->nx, per, per, h->chi_par * dt / (h->dy * h->dy),
                         mu, true, ANISO_KERNEL_YSWEEP, s, pairs, v4, h->kahan ? h->tstar_lo : nullptr,
                         h->kahan ? h->tlo : nullptr);
}

// nsteps compensated steps on the cluster kernel: the first x-update reads
// (T, lo), the last y-update writes them; in between the state and the
// intermediate stay interleaved (kq, kqs), so that every transposed store
// fills whole 32-byte sectors.
static int enqueue_fast_steps_k(aniso_ctx *h, void *T, double dt, int nsteps, cudaStream_t s,
                                std::vector<int> *pairs)
{
    const double mu = h->chi_par * dt / (h->dx * h->dy);
    const double lamx = h->chi_par * dt / (h->dx * h->dx), lamy = h->chi_par * dt / (h->dy * h->dy);
    const int per = h->bc == ANISO_BC_PERIODIC;
    for (int k = 0; k < nsteps; ++k) {
        const bool first = k == 0, last = k == nsteps - 1;
        int rc = enqueue_line2(h, first ? T : h->kq, h->kqs, h->cxx, h->cxy, h->nx, h->ny, per, per, lamx, mu, true,
                               ANISO_KERNEL_XSWEEP, s, pairs, true, first ? h->tlo : h->kq, h->kqs, first ? 0 : 1,
                               1);
        if (rc) return rc;
        rc = enqueue_line2(h, h->kqs, last ? T : h->kq, h->cyyT, h->cyxT, h->ny, h->nx, per, per, lamy, mu, true,
                           ANISO_KERNEL_YSWEEP, s, pairs, true, h->kqs, last ? h->tlo : h->kq, 1, last ? 0 : 1);
        if (rc) return rc;
    }
    return ANISO_OK;
}

// The interleaved buffers of the compensated cluster path (allocated once,
// outside any capture).
static int ensure_kq(aniso_ctx *h)
{
    if (!h->kahan || h->kq || h->fast_kind() != 7) return ANISO_OK;
    CU(cudaMalloc(&h->kq, h->cells() * 2 * sizeof(float)));
    CU(cudaMalloc(&h->kqs, h->cells() * 2 * sizeof(float)));
    return ANISO_OK;
}

static int enqueue_fast_step(aniso_ctx *h, void *T, double dt, cudaStream_t s, std::vector<int> *pairs)
{
    int rc = enqueue_fast_sweep(h, 0, T, dt, s, pairs);
    if (rc) return rc;
    return enqueue_fast_sweep(h, 1, T, dt, s, pairs);
}

// One directional update from `in` to `out` (distinct buffers) on stream s.
// ls, ms scale the implicit (normal) and explicit (transverse) parts: the
// half-step updates of Eq. 4step use (1/2, 1) and (1/2, 0).
static int enqueue_sweep(aniso_ctx *h, int dir, const void *in, void *out, double dt, cudaStream_t s,
                         std::vector<int> *pairs, const void *in_lo = nullptr, void *out_lo = nullptr,
                         double ls = 1.0, double ms = 1.0)
{
    const bool kahan = in_lo != nullptr;
    const double lamx = ls * h->chi_par * dt / (h->dx * h->dx);
    const double lamy = ls * h->chi_par * dt / (h->dy * h->dy);
    const double mu = ms * h->chi_par * dt / (h->dx * h->dy);
    const int per = h->bc == ANISO_BC_PERIODIC;
    int pidx = -1;
    // inside a stream capture only an "external" record becomes an event
    // node that is recorded on every replay
    const unsigned rec_flags = pairs ? cudaEventRecordExternal : cudaEventRecordDefault;
    auto begin = [&](int kind) -> int {
        if (!h->profile) return ANISO_OK;
        pidx = h->prof.take(kind);
        if (pidx < 0) return fail(ANISO_ERR_CUDA, "event creation failed");
        CU(cudaEventRecordWithFlags(h->prof.pool[pidx].a, s, rec_flags));
        return ANISO_OK;
    };
    auto end = [&]() -> int {
        if (!h->profile) return ANISO_OK;
        CU(cudaEventRecordWithFlags(h->prof.pool[pidx].b, s, rec_flags));
        if (pairs) pairs->push_back(pidx);
        else h->prof.pending.push_back(pidx);
        return ANISO_OK;
    };
    auto line = [&](const void *tin, void *tout, const void *g, const void *e, int n, int nlines,
                    int per_line, int per_cross, double lam, int kind, const void *tin_lo,
                    void *tout_lo) -> int {
        LineArgs a{};
        a.jobs = nullptr;
        a.njobs = 1;
        a.limiter = h->limiter;
        a.err = h->err;
        LineJob &J = a.one;
        J.Tin = tin;
        J.Tout = tout;
        J.TinLo = tin_lo;
        J.ToutLo = tout_lo;
        J.g = g;
        J.e = e;
        J.lam = lam;
        J.mu = mu;
        J.n = n;
        J.nlines = nlines;
        J.per_line = per_line;
        J.per_cross = per_cross;
        J.pin_ends = J.pin_lines = h->dirichlet() ? 1 : 0;
        int nthreads;
        line_config(h->prec, n, &J.team, &J.lines_per_block, &nthreads);
        J.block0 = 0;
        J.nblocks = (nlines + J.lines_per_block - 1) / J.lines_per_block;
        const size_t smem = line_smem_bytes(h->prec, n, J.team, J.lines_per_block);
        int rc = begin(kind);
        if (rc) return rc;
        CU(launch_line(h->prec, h->field_fp16, a, J.nblocks, nthreads, smem, s, tin_lo != nullptr));
        return end();
    };
    int rc;
    if (dir == ANISO_DIR_X) {
        int t1, t2, t3;
        size_t t4;
        if (!kahan && !h->dirichlet() && h->fast == 3 && aligned16(in) && aligned16(out) &&
            line4_config(h->prec, h->nx, false, h->l4_warps, h->seg_chunks, &t1, &t2, &t3, &t4))
            return enqueue_line2(h, in, out, h->cxx, h->cxy, h->nx, h->ny, per, per, lamx, mu, false,
                                 ANISO_KERNEL_XSWEEP, s, pairs, true);
        // (the block-synchronous kernel also takes the compensated state)
        if (!h->dirichlet() && h->fast && aligned16(in) && aligned16(out) &&
            (!kahan || (aligned16(in_lo) && aligned16(out_lo))) &&
            line2_config(h->prec, h->nx, false, &t1, &t2, &t3, &t4, h->seg_chunks))
            return enqueue_line2(h, in, out, h->cxx, h->cxy, h->nx, h->ny, per, per, lamx, mu, false,
                                 ANISO_KERNEL_XSWEEP, s, pairs, false, in_lo, out_lo);
        return line(in, out, h->cxx, h->cxy, h->nx, h->ny, per, per, lamx, ANISO_KERNEL_XSWEEP, in_lo, out_lo);
    }
    if (!h->col_transpose()) {
        ColArgs a{};
        a.jobs = nullptr;
        a.njobs = 1;
        a.limiter = h->limiter;
        a.err = h->err;
        ColJob &J = a.one;
        J.Tin = in;
        J.Tout = out;
        J.TinLo = in_lo;
        J.ToutLo = out_lo;
        J.g = h->cyy;
        J.e = h->cyx;
        J.lam = lamy;
        J.mu = mu;
        J.nx = h->nx;
        J.ny = h->ny;
        J.per_x = per;
        J.per_y = per;
        int nthreads;
        col_config(h->prec, h->ny, &J.P, &J.Wb, &nthreads);
        J.block0 = 0;
        J.nblocks = (h->nx + J.Wb - 1) / J.Wb;
        const size_t smem = col_smem_bytes(h->prec, h->ny, J.P, J.Wb);
        if ((rc = begin(ANISO_KERNEL_YSWEEP))) return rc;
        CU(launch_col(h->prec, h->field_fp16, a, J.nblocks, nthreads, smem, s, kahan));
        return end();
    }
    // long columns: transpose, solve columns as contiguous lines, transpose back
    if ((rc = begin(ANISO_KERNEL_TRANSPOSE))) return rc;
    CU(launch_transpose((int)h->esz(), in, h->tA, h->ny, h->nx, s));
    if (kahan) CU(launch_transpose((int)h->esz(), in_lo, h->tAlo, h->ny, h->nx, s));
    if ((rc = end())) return rc;
    {
        // the columns are contiguous lines now: the vectorised kernels take them when they can
        int t1, t2, t3;
        size_t t4;
        if (!kahan && !h->dirichlet() && h->fast == 3 && aligned16(h->tA) && aligned16(h->tB) &&
            line4_config(h->prec, h->ny, false, h->l4_warps, h->seg_chunks, &t1, &t2, &t3, &t4))
            rc = enqueue_line2(h, h->tA, h->tB, h->cyyT, h->cyxT, h->ny, h->nx, per, per, lamy, mu, false,
                               ANISO_KERNEL_YSWEEP, s, pairs, true);
        else if (!h->dirichlet() && h->fast && aligned16(h->tA) && aligned16(h->tB) &&
                 (!kahan || (aligned16(h->tAlo) && aligned16(h->tBlo))) &&
                 line2_config(h->prec, h->ny, false, &t1, &t2, &t3, &t4, h->seg_chunks))
            rc = enqueue_line2(h, h->tA, h->tB, h->cyyT, h->cyxT, h->ny, h->nx, per, per, lamy, mu, false,
                               ANISO_KERNEL_YSWEEP, s, pairs, false, kahan ? h->tAlo : nullptr,
                               kahan ? h->tBlo : nullptr);
        else
            rc = line(h->tA, h->tB, h->cyyT, h->cyxT, h->ny, h->nx, per, per, lamy, ANISO_KERNEL_YSWEEP,
                      kahan ? h->tAlo : nullptr, kahan ? h->tBlo : nullptr);
        if (rc) return rc;
    }
    if ((rc = begin(ANISO_KERNEL_TRANSPOSE))) return rc;
    CU(launch_transpose((int)h->esz(), h->tB, out, h->nx, h->ny, s));
    if (kahan) CU(launch_transpose((int)h->esz(), h->tBlo, out_lo, h->nx, h->ny, s));
    return end();
}

static bool x_first(int order, long long counter)
{
    if (order == ANISO_ORDER_XY) return true;
    if (order == ANISO_ORDER_YX) return false;
    return (counter & 1) == 0;
}

// Any update order on the line4 path.  An x-update reads rows (a row-major
// array), a y-update columns (a column-major one); each writes its lines in
// place order or transposed, whichever layout the next update reads, and the
// last update leaves T row-major.  A call that starts with a y-update first
// transposes T once; the updates alternate between T and T*, and a final copy
// brings the state back to T when it ends in T*.
static bool fast_any_order(const aniso_ctx *h, const void *T)
{
    return h->fast && !h->kahan && !h->dirichlet() && !h->q && h->nl_alpha == 0.0 && h->cyyT && aligned16(T) &&
           aligned16(h->tstar) && h->fast_kind() == 4;
}

static int enqueue_steps_any_order(aniso_ctx *h, void *T, double dt, int nsteps, long long counter0,
                                   cudaStream_t s, std::vector<int> *pairs)
{
    const double lamx = h->chi_par * dt / (h->dx * h->dx);
    const double lamy = h->chi_par * dt / (h->dy * h->dy);
    const double mu = h->chi_par * dt / (h->dx * h->dy);
    const int per = h->bc == ANISO_BC_PERIODIC;
    std::vector<int> dirs;  // the updates of the call, in order
    for (int k = 0; k < nsteps; ++k) {
        const bool xf = x_first(h->order, counter0 + k);
        dirs.push_back(xf ? ANISO_DIR_X : ANISO_DIR_Y);
        dirs.push_back(xf ? ANISO_DIR_Y : ANISO_DIR_X);
    }
    void *cur = T;
    if (!dirs.empty() && dirs[0] == ANISO_DIR_Y) {  // columns of the row-major T, once
        CU(launch_transpose((int)h->esz(), T, h->tstar, h->ny, h->nx, s));
        cur = h->tstar;
    }
    for (size_t i = 0; i < dirs.size(); ++i) {
        const bool x = dirs[i] == ANISO_DIR_X;
        // the next update (or the caller, after the last) reads rows for x, columns for y
        const bool next_rows = i + 1 < dirs.size() ? dirs[i + 1] == ANISO_DIR_X : true;
        const bool transposed = x ? !next_rows : next_rows;
        void *out = cur == T ? h->tstar : T;
        const int rc = x ? enqueue_line2(h, cur, out, h->cxx, h->cxy, h->nx, h->ny, per, per, lamx, mu, transposed,
                                         ANISO_KERNEL_XSWEEP, s, pairs, true)
                         : enqueue_line2(h, cur, out, h->cyyT, h->cyxT, h->ny, h->nx, per, per, lamy, mu,
                                         transposed, ANISO_KERNEL_YSWEEP, s, pairs, true);
        if (rc) return rc;
        cur = out;
    }
    if (cur != T) CU(cudaMemcpyAsync(T, cur, h->cells() * h->esz(), cudaMemcpyDeviceToDevice, s));
    return ANISO_OK;
}

static int enqueue_steps(aniso_ctx *h, void *T, double dt, int nsteps, long long counter0,
                         cudaStream_t s, std::vector<int> *pairs)
{
    if (h->scheme == ANISO_SCHEME_EXPLICIT) {
        // explicit limited steps, T -> T* -> T ...; an odd count ends with a copy back
        ExpArgs a{};
        a.cxx = h->cxx;
        a.cxy = h->cxy;
        a.cyy = h->cyy;
        a.cyx = h->cyx;
        a.lamx = h->chi_par * dt / (h->dx * h->dx);
        a.lamy = h->chi_par * dt / (h->dy * h->dy);
        a.mu = h->chi_par * dt / (h->dx * h->dy);
        a.nx = h->nx;
        a.ny = h->ny;
        a.per = h->bc == ANISO_BC_PERIODIC;
        a.limiter = h->limiter;
        a.pin = h->dirichlet() ? 1 : 0;
        a.err = h->err;
        // rows per thread: enough threads to fill the GPU, longer strips on big grids
        const long long cols = ((h->nx + 31) / 32) * 32LL;
        a.rows = (int)std::max(1LL, std::min(32LL, cols * h->ny / (152LL * 2048)));
        const unsigned rec = pairs ? cudaEventRecordExternal : cudaEventRecordDefault;
        for (int k = 0; k < nsteps; ++k) {
            a.Tin = (k & 1) ? h->tstar : T;
            a.Tout = (k & 1) ? T : h->tstar;
            if (h->q) CU(launch_source(h->prec, const_cast<void *>(a.Tin), h->q, dt, h->cells(), s));
            int pidx = -1;
            if (h->profile) {
                pidx = h->prof.take(ANISO_KERNEL_XSWEEP);
                if (pidx < 0) return fail(ANISO_ERR_CUDA, "event creation failed");
                CU(cudaEventRecordWithFlags(h->prof.pool[pidx].a, s, rec));
            }
            CU(launch_explicit(h->prec, h->field_fp16, a, s));
            if (h->profile) {
                CU(cudaEventRecordWithFlags(h->prof.pool[pidx].b, s, rec));
                if (pairs) pairs->push_back(pidx);
                else h->prof.pending.push_back(pidx);
            }
        }
        if (nsteps & 1) CU(cudaMemcpyAsync(T, h->tstar, h->cells() * h->esz(), cudaMemcpyDeviceToDevice, s));
        return ANISO_OK;
    }
    if (h->scheme == ANISO_SCHEME_4STEP && h->order == ANISO_ORDER_XY && h->t4 && aligned16(h->t4) &&
        use_fast(h, T) && h->fast_kind() == 4) {
        // Eq. 4step on the line4 path: each direction's first half-update
        // writes its lines in place order (t4), the purely implicit second
        // half writes them transposed, so x: T -> t4 -> T* (column-major) and
        // y: T* -> t4 -> T (row-major), with no transpose pass
        const double lamx = h->chi_par * dt / (h->dx * h->dx);
        const double lamy = h->chi_par * dt / (h->dy * h->dy);
        const double mu = h->chi_par * dt / (h->dx * h->dy);
        const int per = h->bc == ANISO_BC_PERIODIC;
        for (int k = 0; k < nsteps; ++k) {
            int rc;
            if (h->q) CU(launch_source(h->prec, T, h->q, dt, h->cells(), s));
            if ((rc = enqueue_line2(h, T, h->t4, h->cxx, h->cxy, h->nx, h->ny, per, per, 0.5 * lamx, mu, false,
                                    ANISO_KERNEL_XSWEEP, s, pairs, true)))
                return rc;
            if ((rc = enqueue_line2(h, h->t4, h->tstar, h->cxx, h->cxy, h->nx, h->ny, per, per, 0.5 * lamx, 0.0,
                                    true, ANISO_KERNEL_XSWEEP, s, pairs, true)))
                return rc;
            if ((rc = enqueue_line2(h, h->tstar, h->t4, h->cyyT, h->cyxT, h->ny, h->nx, per, per, 0.5 * lamy, mu,
                                    false, ANISO_KERNEL_YSWEEP, s, pairs, true)))
                return rc;
            if ((rc = enqueue_line2(h, h->t4, T, h->cyyT, h->cyxT, h->ny, h->nx, per, per, 0.5 * lamy, 0.0, true,
                                    ANISO_KERNEL_YSWEEP, s, pairs, true)))
                return rc;
        }
        return ANISO_OK;
    }
    if (h->scheme == ANISO_SCHEME_4STEP) {
        // Eq. 4step: per direction, the semi-implicit update with its implicit
        // part over dt/2, then a fully implicit dt/2 update (no transverse term)
        for (int k = 0; k < nsteps; ++k) {
            const bool xf = x_first(h->order, counter0 + k);
            const int d1 = xf ? ANISO_DIR_X : ANISO_DIR_Y, d2 = xf ? ANISO_DIR_Y : ANISO_DIR_X;
            int rc;
            if (h->q) CU(launch_source(h->prec, T, h->q, dt, h->cells(), s));
            if ((rc = enqueue_sweep(h, d1, T, h->t4, dt, s, pairs, nullptr, nullptr, 0.5, 1.0))) return rc;
            if ((rc = enqueue_sweep(h, d1, h->t4, h->tstar, dt, s, pairs, nullptr, nullptr, 0.5, 0.0))) return rc;
            if ((rc = enqueue_sweep(h, d2, h->tstar, h->t4, dt, s, pairs, nullptr, nullptr, 0.5, 1.0))) return rc;
            if ((rc = enqueue_sweep(h, d2, h->t4, T, dt, s, pairs, nullptr, nullptr, 0.5, 0.0))) return rc;
        }
        return ANISO_OK;
    }
    if (use_fast(h, T) && h->kahan && h->kq && h->fast_kind() == 7)
        return enqueue_fast_steps_k(h, T, dt, nsteps, s, pairs);
    if (use_fast(h, T)) {
        for (int k = 0; k < nsteps; ++k) {
            if (h->q) CU(launch_source(h->prec, T, h->q, dt, h->cells(), s));
            int rc = enqueue_fast_step(h, T, dt, s, pairs);
            if (rc) return rc;
        }
        return ANISO_OK;
    }
    if (h->scheme == ANISO_SCHEME_2STEP && fast_any_order(h, T))
        return enqueue_steps_any_order(h, T, dt, nsteps, counter0, s, pairs);
    for (int k = 0; k < nsteps; ++k) {
        const bool xf = x_first(h->order, counter0 + k);
        if (h->q) CU(launch_source(h->prec, T, h->q, dt, h->cells(), s));
        int rc = enqueue_sweep(h, xf ? ANISO_DIR_X : ANISO_DIR_Y, T, h->tstar, dt, s, pairs, h->tlo, h->tstar_lo);
        if (rc) return rc;
        rc = enqueue_sweep(h, xf ? ANISO_DIR_Y : ANISO_DIR_X, h->tstar, T, dt, s, pairs, h->tstar_lo, h->tlo);
        if (rc) return rc;
    }
    return ANISO_OK;
}

static int check_ready(aniso_ctx *h, const char *who)
{
    if (!h) return fail(ANISO_ERR_ARG, "%s: null handle", who);
    if (!h->field_set) return fail(ANISO_ERR_STATE, "%s: aniso_set_field has not been called", who);
    return ANISO_OK;
}

extern "C" int aniso_set_source(aniso_t h, const void *Q)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso_set_source: null handle");
    if (!h->field_set) return fail(ANISO_ERR_STATE, "aniso_set_source: set the field first");
    if (!Q) {
        if (h->q) {
            CU(cudaStreamSynchronize(h->stream));
            cudaFree(h->q);
            h->q = nullptr;
        }
        drop_graph(h);
        return ANISO_OK;
    }
    if (h->kahan) return fail(ANISO_ERR_UNSUPPORTED, "aniso_set_source: not with the compensated state");
    if (!h->q) CU(cudaMalloc(&h->q, h->cells() * h->esz()));
    CU(cudaMemcpyAsync(h->q, Q, h->cells() * h->esz(), cudaMemcpyDeviceToDevice, h->stream));
    drop_graph(h);
    return ANISO_OK;
}

extern "C" int aniso_set_nonlinear(aniso_t h, double alpha, double t_ref)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso_set_nonlinear: null handle");
    if (!(alpha >= 0) || !(alpha < 1e3) || !(t_ref > 0) || !(t_ref < 1e300))
        return fail(ANISO_ERR_ARG, "aniso_set_nonlinear: need 0 <= alpha and t_ref > 0 (finite)");
    h->nl_alpha = alpha;
    h->nl_tref = t_ref;
    drop_graph(h);
    return ANISO_OK;
}

// What the temperature-dependent diffusivity runs on: the line4 fast path of
// the x-then-y 2-step scheme on the plain state.
static int check_nonlinear(aniso_ctx *h, const void *T, const char *who)
{
    if (h->nl_alpha == 0.0) return ANISO_OK;
    if (h->scheme != ANISO_SCHEME_2STEP || h->kahan || h->dirichlet() || h->q || h->field_fp16 ||
        h->order != ANISO_ORDER_XY || !use_fast(h, T) || h->fast_kind() != 4)
        return fail(ANISO_ERR_UNSUPPORTED,
                    "%s: the temperature-dependent diffusivity needs the 2-step x-then-y scheme on the "
                    "line4 fast path (both line lengths multiples of the 16-byte vector, at most 2048; "
                    "plain state, FP32 or FP64 field, no fixed boundary or source)", who);
    return ANISO_OK;
}

extern "C" int aniso_step(aniso_t h, void *T, double dt, int nsteps)
{
    TraceRange trace("aniso_step");
    int rc = check_ready(h, "aniso_step");
    if (rc) return rc;
    if (!T) return fail(ANISO_ERR_ARG, "aniso_step: T is NULL");
    if (!(dt > 0)) return fail(ANISO_ERR_ARG, "aniso_step: dt must be > 0");
    if (nsteps < 0) return fail(ANISO_ERR_ARG, "aniso_step: nsteps must be >= 0");
    if ((rc = check_nonlinear(h, T, "aniso_step"))) return rc;
    if (nsteps == 0) return ANISO_OK;
    if ((rc = ensure_kq(h))) return rc;
    const int parity = h->order == ANISO_ORDER_ALTERNATE ? (int)(h->step_counter & 1) : 0;
    if (h->use_graph && nsteps >= 2) {
        const bool hit = h->gexec && h->g_T == T && h->g_dt == dt && h->g_nsteps == nsteps &&
                         h->g_parity == parity && h->g_order == h->order && h->g_limiter == h->limiter &&
                         h->g_profile == h->profile;
        if (!hit) {
            drop_graph(h);
            if (!h->cap_stream) CU(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
            h->prof.next = h->prof.pool.size();  // graph pairs are never reused by direct launches
            CU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            std::vector<int> pairs;
            rc = enqueue_steps(h, T, dt, nsteps, h->step_counter, h->cap_stream, &pairs);
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (ce != cudaSuccess) return fail(ANISO_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&h->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return fail(ANISO_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
            h->g_T = T;
            h->g_dt = dt;
            h->g_nsteps = nsteps;
            h->g_parity = parity;
            h->g_order = h->order;
            h->g_limiter = h->limiter;
            h->g_profile = h->profile;
            h->g_pairs = pairs;
        }
        if (h->profile && !h->prof.pending.empty()) {
            // the graph re-records its events: read the previous replay first
            CU(cudaStreamSynchronize(h->stream));
            if ((rc = h->prof.drain())) return rc;
        }
        CU(cudaGraphLaunch(h->gexec, h->stream));
        if (h->profile) h->prof.pending.insert(h->prof.pending.end(), h->g_pairs.begin(), h->g_pairs.end());
    } else {
        if (h->profile && h->prof.next + 8 * (size_t)nsteps > 4096) {
            CU(cudaStreamSynchronize(h->stream));
            if ((rc = h->prof.drain())) return rc;
            h->prof.next = 0;
            drop_graph(h);
        }
        rc = enqueue_steps(h, T, dt, nsteps, h->step_counter, h->stream, nullptr);
        if (rc) return rc;
    }
    h->step_counter += nsteps;
    return ANISO_OK;
}

extern "C" int aniso_sweep(aniso_t h, int dir, const void *Tin, void *Tout, double dt)
{
    TraceRange trace("aniso_sweep");
    int rc = check_ready(h, "aniso_sweep");
    if (rc) return rc;
    if (!Tin || !Tout || Tin == Tout) return fail(ANISO_ERR_ARG, "aniso_sweep: need distinct Tin, Tout");
    if (dir != ANISO_DIR_X && dir != ANISO_DIR_Y) return fail(ANISO_ERR_ARG, "aniso_sweep: bad direction");
    if (!(dt > 0)) return fail(ANISO_ERR_ARG, "aniso_sweep: dt must be > 0");
    if (h->nl_alpha != 0.0)
        return fail(ANISO_ERR_UNSUPPORTED, "aniso_sweep: not with the temperature-dependent diffusivity");
    return enqueue_sweep(h, dir, Tin, Tout, dt, h->stream, nullptr);
}

static int check_err_flag(aniso_ctx *h)
{
    unsigned flag = 0;
    CU(cudaMemcpy(&flag, h->err, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) {
        CU(cudaMemset(h->err, 0, sizeof(unsigned)));
        if (flag & 2u) return fail(ANISO_ERR_TIMEOUT, "a kernel gave up waiting for its staged rows");
        return fail(ANISO_ERR_NONFINITE, "a step produced a non-finite temperature");
    }
    return ANISO_OK;
}

extern "C" int aniso_total(aniso_t h, const void *T, double *sum, double *tmin, double *tmax,
                           long long *nonfinite)
{
    int rc = check_ready(h, "aniso_total");
    if (rc) return rc;
    if (!T) return fail(ANISO_ERR_ARG, "aniso_total: T is NULL");
    CU(launch_totals(h->prec, T, h->cells(), h->partials, h->result, h->stream, h->kahan ? h->tlo : nullptr));
    double r[4];
    CU(cudaMemcpyAsync(r, h->result, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (sum) *sum = r[0];
    if (tmin) *tmin = r[1];
    if (tmax) *tmax = r[2];
    if (nonfinite) *nonfinite = (long long)r[3];
    return check_err_flag(h);
}

extern "C" int aniso_get_state(aniso_t h, long long *step_counter, void *lo_out)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso_get_state: null handle");
    if (step_counter) *step_counter = h->step_counter;
    if (lo_out && h->kahan && h->tlo)
        CU(cudaMemcpyAsync(lo_out, h->tlo, h->cells() * h->esz(), cudaMemcpyDeviceToDevice, h->stream));
    return ANISO_OK;
}

extern "C" int aniso_set_state(aniso_t h, long long step_counter, const void *lo_in)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso_set_state: null handle");
    if (step_counter < 0) return fail(ANISO_ERR_ARG, "aniso_set_state: negative step counter");
    h->step_counter = step_counter;
    if (h->kahan && h->tlo) {
        if (lo_in) CU(cudaMemcpyAsync(h->tlo, lo_in, h->cells() * h->esz(), cudaMemcpyDeviceToDevice, h->stream));
        else CU(cudaMemsetAsync(h->tlo, 0, h->cells() * h->esz(), h->stream));
    }
    return ANISO_OK;
}

extern "C" int aniso_sync(aniso_t h)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso_sync: null handle");
    CU(cudaStreamSynchronize(h->stream));
    if (!h->err) return ANISO_OK;
    return check_err_flag(h);
}

extern "C" void aniso_destroy(aniso_t h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    drop_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->prof.destroy();
    free_buffers(h);
    delete h;
}

// ------------------------------------------------------------- batches

struct aniso_batch {
    std::vector<aniso_ctx *> hs;
    cudaStream_t stream = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<void *> key_T;
    std::vector<double> key_dt;
    std::vector<int> key_n;
    std::vector<int> key_parity;
    int key_profile = -1;
    void *d_jobs = nullptr;  // device copies of all job lists of the plan
    size_t d_jobs_bytes = 0;
    Profiler prof;
    std::vector<int> g_pairs;
    int profile = 0;
    int use_graph = 1;
    // concurrent branches of one sweep (line4 occupancy classes)
    static constexpr int kSide = 6;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};
    long long kernels_per_call = 0;  // kernel nodes of the captured graph
    std::vector<void *> dev_T;       // device copies of T for aniso_step_batched_host
    // per-step diagnostics (ANISO_OPT_DIAGNOSTICS of the first handle)
    int key_diag = -1;
    int key_tma = -1;
    int key_tmem = -1;
    double *d_ring = nullptr;  // [grid][step][sum, min, max] of the last call
    size_t ring_count = 0;     // doubles
    int ring_steps = 0;        // steps per grid in the ring (the call's largest nsteps)
    DiagPart *d_part = nullptr;
    size_t part_count = 0;
};

extern "C" int aniso_batch_create(int n, const aniso_t *hs, aniso_batch_t *out)
{
    if (!out) return fail(ANISO_ERR_ARG, "aniso_batch_create: out is NULL");
    *out = nullptr;
    if (n < 1 || !hs) return fail(ANISO_ERR_ARG, "aniso_batch_create: need n >= 1 handles");
    for (int k = 0; k < n; ++k) {
        aniso_ctx *h = hs[k];
        if (!h) return fail(ANISO_ERR_ARG, "aniso_batch_create: handle %d is NULL", k);
        if (!h->field_set) return fail(ANISO_ERR_STATE, "aniso_batch_create: handle %d has no field", k);
        if (h->prec != hs[0]->prec || h->field_fp16 != hs[0]->field_fp16 || h->limiter != hs[0]->limiter ||
            h->kahan != hs[0]->kahan)
            return fail(ANISO_ERR_ARG, "aniso_batch_create: handle %d differs in precision/field/limiter/state", k);
        if (h->scheme != ANISO_SCHEME_2STEP)
            return fail(ANISO_ERR_UNSUPPORTED, "aniso_batch_create: handle %d runs another scheme than Eq. op_2step", k);
        if (h->dirichlet() || h->q)
            return fail(ANISO_ERR_UNSUPPORTED, "aniso_batch_create: handle %d has fixed boundaries or a source", k);
        if (h->nl_alpha != 0.0)
            return fail(ANISO_ERR_UNSUPPORTED, "aniso_batch_create: handle %d has a temperature-dependent diffusivity", k);
    }
    aniso_batch *b = new aniso_batch;
    b->hs.assign(hs, hs + n);
    b->stream = hs[0]->stream;
    b->profile = hs[0]->profile;
    b->use_graph = hs[0]->use_graph;
    *out = b;
    return ANISO_OK;
}

static void batch_drop(aniso_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->key_T.clear();
    b->g_pairs.clear();
}

// Build, capture and instantiate the whole batched call.
static int batch_build(aniso_batch *b, void *const *T, const double *dt, const int *nsteps)
{
    const int n = (int)b->hs.size();
    const int prec = b->hs[0]->prec;
    const int fp16 = b->hs[0]->field_fp16;
    const bool diag = b->hs[0]->diag != 0;
    int max_steps = 0;
    for (int k = 0; k < n; ++k) max_steps = std::max(max_steps, nsteps[k]);

    // Every (global step, phase) launch is one list of line jobs (x) and one
    // of column jobs (y).  Identical lists are shared.
    struct Launch {
        int kind;  // 0 line, 1 col, 2/3 line2 (x/y), 7/8 line4 (x/y), 9/10 line5 (x/y), 11/12 line6 (x/y),
                   // 6 / 13 one grid's general / fast update on its own
        size_t offset;
        int njobs, nblocks, nthreads;
        size_t smem;
        // consecutive launches with the same group >= 0 run concurrently
        // (one branch each) and are joined before the next launch
        int group = -1;
        // kind 6: one grid's sweep captured on its own (columns above the
        // on-chip limit go through the transpose path)
        int inst = -1, dir = 0;
        const void *in = nullptr, *in_lo = nullptr;
        void *out = nullptr, *out_lo = nullptr;
        double dt = 0;
        long long table = -1;  // line4: offset of the block -> job table, or -1
        int diag_region = -1;  // line4 y-update with diagnostics: its partials region
        int tmem = 0;          // line4: gamma in tensor memory
        int step = 0;          // the call's step the launch belongs to
    };
    std::vector<unsigned char> blob;
    std::vector<Launch> launches;  // in enqueue order
    auto add_line = [&](std::vector<LineJob> &jobs) {
        if (jobs.empty()) return;
        // large lines first: the block scheduler hands out blocks in order
        std::stable_sort(jobs.begin(), jobs.end(),
                         [](const LineJob &a, const LineJob &c) { return (long long)a.n * a.nlines > (long long)c.n * c.nlines; });
        int nthreads = 0;
        for (auto &J : jobs) nthreads = std::max(nthreads, J.team * J.lines_per_block);
        int blocks = 0;
        size_t smem = 0;
        for (auto &J : jobs) {
            J.lines_per_block = nthreads / J.team;
            J.block0 = blocks;
            J.nblocks = (J.nlines + J.lines_per_block - 1) / J.lines_per_block;
            blocks += J.nblocks;
            smem = std::max(smem, line_smem_bytes(prec, J.n, J.team, J.lines_per_block));
        }
        Launch L{0, blob.size(), (int)jobs.size(), blocks, nthreads, smem};
        const unsigned char *p = reinterpret_cast<const unsigned char *>(jobs.data());
        blob.insert(blob.end(), p, p + jobs.size() * sizeof(LineJob));
        while (blob.size() % 16) blob.push_back(0);
        launches.push_back(L);
    };
    auto add_col = [&](std::vector<ColJob> &jobs) {
        if (jobs.empty()) return;
        std::stable_sort(jobs.begin(), jobs.end(),
                         [](const ColJob &a, const ColJob &c) { return (long long)a.nx * a.ny > (long long)c.nx * c.ny; });
        const int nthreads = prec == PREC_FP64 ? 256 : 512;
        int blocks = 0;
        size_t smem = 0;
        for (auto &J : jobs) {
            // the launch-wide thread count fixes P * Wb
            int P, Wb, nt;
            col_config(prec, J.ny, &P, &Wb, &nt);
            Wb = nthreads / P;
            J.P = P;
            J.Wb = Wb;
            J.block0 = blocks;
            J.nblocks = (J.nx + Wb - 1) / Wb;
            blocks += J.nblocks;
            smem = std::max(smem, col_smem_bytes(prec, J.ny, P, Wb));
        }
        Launch L{1, blob.size(), (int)jobs.size(), blocks, nthreads, smem};
        const unsigned char *p = reinterpret_cast<const unsigned char *>(jobs.data());
        blob.insert(blob.end(), p, p + jobs.size() * sizeof(ColJob));
        while (blob.size() % 16) blob.push_back(0);
        launches.push_back(L);
    };

    auto add_line2 = [&](std::vector<Line2Job> &jobs, int kind_xy) {
        if (jobs.empty()) return;
        std::stable_sort(jobs.begin(), jobs.end(),
                         [](const Line2Job &a, const Line2Job &c) { return (long long)a.n * a.nlines > (long long)c.n * c.nlines; });
        int nthreads = 0;
        for (auto &J : jobs) nthreads = std::max(nthreads, J.team * J.lines_per_block);
        int blocks = 0;
        size_t smem = 0;
        for (auto &J : jobs) {
            J.lines_per_block = nthreads / J.team;
            J.block0 = blocks;
            J.nblocks = (J.nlines + J.lines_per_block - 1) / J.lines_per_block;
            blocks += J.nblocks;
            smem = std::max(smem, line2_smem_bytes(prec, J.n, J.team, J.lines_per_block));
        }
        Launch L{kind_xy == 0 ? 2 : 3, blob.size(), (int)jobs.size(), blocks, nthreads, smem};
        const unsigned char *p = reinterpret_cast<const unsigned char *>(jobs.data());
        blob.insert(blob.end(), p, p + jobs.size() * sizeof(Line2Job));
        while (blob.size() % 16) blob.push_back(0);
        launches.push_back(L);
    };

    // line4 jobs: NW-warp blocks, per-job team and lines per block; the block
    // shape (warps, chunks per lane) is the first grid's, for all.  A launch's
    // dynamic shared memory is that of its largest line, so short lines in the
    // same launch would be held to the long lines' occupancy.  The jobs are
    // therefore split by the resident blocks per SM their own shared memory
    // allows (CUDA's occupancy calculator), one launch per class, and the
    // classes of a sweep run concurrently (one graph branch each).
    int shape_rc = ANISO_OK;
    int next_group = 0;
    auto add_line4 = [&](std::vector<Line2Job> &jobs, int kind_xy, int group) {
        if (jobs.empty()) return;
        const int warps = b->hs[0]->l4_warps, seg = b->hs[0]->seg_chunks;
        std::stable_sort(jobs.begin(), jobs.end(),
                         [](const Line2Job &a, const Line2Job &c) { return (long long)a.n * a.nlines > (long long)c.n * c.nlines; });
        // one block size for the launch: the largest any job needs, then every
        // job's lines per block for that many warps
        int nthreads = 0;
        for (auto &J : jobs) {
            int nt;
            size_t sm;
            if (line4_config(prec, J.n, true, warps, seg, &J.team, &J.lines_per_block, &nt, &sm))
                nthreads = std::max(nthreads, nt);
        }
        // Per job: its resident blocks per SM in the shared-memory form and, when
        // the lines fit it, in the tensor-memory form (whose TMEM columns also
        // cap the blocks an SM holds); the form with more blocks wins.
        struct Cls {
            int occ;
            size_t sm;
            bool tm;
        };
        const bool tm_on = b->hs[0]->tmem != 0 && prec == PREC_FP32;
        std::vector<Cls> cls(jobs.size());
        for (size_t k = 0; k < jobs.size(); ++k) {
            Line2Job &J = jobs[k];
            int nt = 0;
            size_t sm = 0;
            if (!line4_config(prec, J.n, true, nthreads / 32, seg, &J.team, &J.lines_per_block, &nt, &sm) ||
                nt != nthreads)
                shape_rc = fail(ANISO_ERR_UNSUPPORTED, "batch: line length %d does not fit the block shape", J.n);
            J.swz = line4_swizzle(prec, J.n, J.team);
            int occ = line4_blocks_per_sm(prec, fp16, b->hs[0]->limiter, nthreads, sm, false);
            cls[k] = {occ > 0 ? occ : 0, sm, false};
            int t0, t1, t2;
            size_t smt = 0;
            if (tm_on && line4_config(prec, J.n, true, nthreads / 32, seg, &t0, &t1, &t2, &smt, true)) {
                const int occt = line4_blocks_per_sm(prec, fp16, b->hs[0]->limiter, nthreads, smt, true,
                                                     line4_tm_cols(J.n, J.team));
                if (occt > cls[k].occ) cls[k] = {occt, smt, true};
            }
        }
        // per form, classes in ascending occupancy (largest lines first); at
        // most three a form, the highest-occupancy ones merged
        int region = 0;
        for (int form = 1; form >= 0; --form) {
            std::vector<int> occs;
            for (auto &c : cls)
                if (c.tm == (form == 1)) occs.push_back(c.occ);
            std::sort(occs.begin(), occs.end());
            occs.erase(std::unique(occs.begin(), occs.end()), occs.end());
            // (merging never drops the lowest class: its range reaches up to the next kept one)
            while ((int)occs.size() > 3) occs.erase(occs.end() - (occs.size() >= 3 ? 2 : 1));
            for (size_t ci = 0; ci < occs.size(); ++ci) {
                const int lo = occs[ci], hi = ci + 1 < occs.size() ? occs[ci + 1] : 1 << 30;
                std::vector<Line2Job> part;
                size_t smem = 0;
                int blocks = 0;
                for (size_t k = 0; k < jobs.size(); ++k) {
                    if (cls[k].tm != (form == 1) || cls[k].occ < lo || cls[k].occ >= hi) continue;
                    Line2Job J = jobs[k];
                    smem = std::max(smem, cls[k].sm);
                    J.block0 = blocks;
                    J.nblocks = (J.nlines + J.lines_per_block - 1) / J.lines_per_block;
                    blocks += J.nblocks;
                    part.push_back(J);
                }
                if (part.empty()) continue;
                Launch L{kind_xy == 0 ? 7 : 8, blob.size(), (int)part.size(), blocks, nthreads, smem};
                L.group = group;
                L.tmem = form;
                if (kind_xy == 1 && diag) L.diag_region = region;
                ++region;
                const unsigned char *p = reinterpret_cast<const unsigned char *>(part.data());
                blob.insert(blob.end(), p, p + part.size() * sizeof(Line2Job));
                while (blob.size() % 16) blob.push_back(0);
                std::vector<int> table(blocks);
                for (size_t k = 0; k < part.size(); ++k)
                    for (int bk = 0; bk < part[k].nblocks; ++bk) table[part[k].block0 + bk] = (int)k;
                L.table = (long long)blob.size();
                const unsigned char *tp = reinterpret_cast<const unsigned char *>(table.data());
                blob.insert(blob.end(), tp, tp + table.size() * sizeof(int));
                while (blob.size() % 16) blob.push_back(0);
                launches.push_back(L);
            }
        }
    };

    // line5 jobs (TMA-staged, lines of 768-1024 cells): one launch per sweep,
    // a branch of the same group as the line4 classes
    const int tma_mode = b->hs[0]->tma_lines;
    auto add_line5 = [&](std::vector<Line5Job> &jobs, int kind_xy, int group) {
        if (jobs.empty()) return;
        std::stable_sort(jobs.begin(), jobs.end(),
                         [](const Line5Job &a, const Line5Job &c) { return (long long)a.n * a.nlines > (long long)c.n * c.nlines; });
        int tiles = 0, nthreads = 0;
        size_t stage = 0;
        for (auto &J : jobs) {
            J.block0 = tiles;
            J.nblocks = (J.nlines + J.lines_per_block - 1) / J.lines_per_block;
            tiles += J.nblocks;
            int tm, lp, nt;
            size_t st;
            line5_config(prec, fp16, J.n, &tm, &lp, &nt, &st);
            nthreads = std::max(nthreads, nt);
            stage = std::max(stage, st);
        }
        const int resident = line5_prepare(b->hs[0]->limiter, nthreads, stage);
        if (resident < 1) {
            shape_rc = fail(ANISO_ERR_CUDA, "batch: the TMA line kernel cannot be resident with %zu bytes", stage);
            return;
        }
        while (blob.size() % 128) blob.push_back(0);
        Launch L{kind_xy == 0 ? 9 : 10, blob.size(), (int)jobs.size(), tiles, nthreads, stage};
        L.group = group;
        L.inst = resident;  // the prefetch distance in tiles
        const unsigned char *p = reinterpret_cast<const unsigned char *>(jobs.data());
        blob.insert(blob.end(), p, p + jobs.size() * sizeof(Line5Job));
        std::vector<int> table(tiles);
        for (size_t k = 0; k < jobs.size(); ++k)
            for (int t = 0; t < jobs[k].nblocks; ++t) table[jobs[k].block0 + t] = (int)k;
        L.table = (long long)blob.size();
        const unsigned char *tp = reinterpret_cast<const unsigned char *>(table.data());
        blob.insert(blob.end(), tp, tp + table.size() * sizeof(int));
        while (blob.size() % 16) blob.push_back(0);
        launches.push_back(L);
    };

    // line6 jobs (lines above line4's limit): one launch per team size (the
    // kernel's block barriers need one block shape per launch)
    auto add_line6 = [&](std::vector<Line2Job> &jobs, int kind_xy, int group) {
        if (jobs.empty()) return;
        std::vector<int> teams;
        for (auto &J : jobs) teams.push_back(J.team);
        std::sort(teams.begin(), teams.end());
        teams.erase(std::unique(teams.begin(), teams.end()), teams.end());
        for (int P : teams) {
            std::vector<Line2Job> part;
            size_t smem = 0;
            int blocks = 0, nthreads = 0;
            for (auto &J0 : jobs) {
                if (J0.team != P) continue;
                Line2Job J = J0;
                int tm, lp, nt;
                size_t sm;
                line6_config(prec, fp16, J.n, &tm, &lp, &nt, &sm, J.lines_per_block);
                smem = std::max(smem, sm);
                nthreads = nt;
                J.block0 = blocks;
                J.nblocks = (J.nlines + J.lines_per_block - 1) / J.lines_per_block;
                blocks += J.nblocks;
                part.push_back(J);
            }
            Launch L{kind_xy == 0 ? 11 : 12, blob.size(), (int)part.size(), blocks, nthreads, smem};
            L.group = group;
            const unsigned char *p = reinterpret_cast<const unsigned char *>(part.data());
            blob.insert(blob.end(), p, p + part.size() * sizeof(Line2Job));
            while (blob.size() % 16) blob.push_back(0);
            std::vector<int> table(blocks);
            for (size_t k = 0; k < part.size(); ++k)
                for (int bk = 0; bk < part[k].nblocks; ++bk) table[part[k].block0 + bk] = (int)k;
            L.table = (long long)blob.size();
            const unsigned char *tp = reinterpret_cast<const unsigned char *>(table.data());
            blob.insert(blob.end(), tp, tp + table.size() * sizeof(int));
            while (blob.size() % 16) blob.push_back(0);
            launches.push_back(L);
        }
    };

    size_t step_begin = 0;
    for (int s = 0; s < max_steps; ++s) {
        for (int phase = 0; phase < 2; ++phase) {
            std::vector<LineJob> xl;
            std::vector<ColJob> yl;
            std::vector<Line2Job> fl, fl4;
            std::vector<Line5Job> fl5;
            std::vector<Line2Job> fl6;
            std::vector<Launch> solo;
            for (int k = 0; k < n; ++k) {
                if (s >= nsteps[k]) continue;
                aniso_ctx *h = b->hs[k];
                if (use_fast(h, T[k]) && h->fast_kind() == 7) {
                    // cluster-kernel grids (and the compensated state): the
                    // grid's fast update captured on its own
                    Launch L{13, 0, 0, 0, 0, 0};
                    L.inst = k;
                    L.dir = phase;
                    L.out = T[k];
                    L.dt = dt[k];
                    solo.push_back(L);
                    continue;
                }
                if (use_fast(h, T[k])) {
                    // x: T (rows) -> T* (column-major); y: T* (columns) -> T (rows)
                    const int per = h->bc == ANISO_BC_PERIODIC;
                    const double mu = h->chi_par * dt[k] / (h->dx * h->dy);
                    Line2Job J{};
                    int nt;
                    size_t sm;
                    if (phase == 0) {
                        J.Tin = T[k];
                        J.Tout = h->tstar;
                        J.g = h->cxx;
                        J.e = h->cxy;
                        J.lam = h->chi_par * dt[k] / (h->dx * h->dx);
                        J.n = h->nx;
                        J.nlines = h->ny;
                    } else {
                        J.Tin = h->tstar;
                        J.Tout = T[k];
                        J.g = h->cyyT;
                        J.e = h->cyxT;
                        J.lam = h->chi_par * dt[k] / (h->dy * h->dy);
                        J.n = h->ny;
                        J.nlines = h->nx;
                    }
                    J.mu = mu;
                    J.per_line = per;
                    J.per_cross = per;
                    J.transpose_out = 1;
                    J.diag_slot = (diag && phase == 1) ? k * max_steps + s : -1;
                    int t5, l5, n5;
                    size_t s5;
                    const int fk = h->fast_kind();
                    if ((fk == 4 || fk == 6) && tma_mode && !(diag && phase == 1) && line5_available() &&
                        line5_config(prec, fp16, J.n, &t5, &l5, &n5, &s5)) {
                        Line5Job J5{};
                        J5.Tout = J.Tout;
                        J5.lam = J.lam;
                        J5.mu = J.mu;
                        J5.n = J.n;
                        J5.nlines = J.nlines;
                        J5.per_line = J.per_line;
                        J5.per_cross = J.per_cross;
                        J5.team = t5;
                        J5.lines_per_block = l5;
                        if (line5_make_maps(J5, J.Tin, J.g, J.e, (size_t)J.n * J.nlines)) {
                            fl5.push_back(J5);
                            continue;
                        }
                    }
                    if (fk == 6 && !line4_config(prec, J.n, true, b->hs[0]->l4_warps, b->hs[0]->seg_chunks, &nt,
                                                 &nt, &nt, &sm)) {
                        // above line4's limit: the long-line kernel
                        line6_config(prec, fp16, J.n, &J.team, &J.lines_per_block, &nt, &sm,
                                     b->hs[0]->l4_warps == 8 ? 2 : 4);
                        J.diag_slot = -1;
                        fl6.push_back(J);
                    } else if (fk == 4 || fk == 6) {
                        fl4.push_back(J);  // team and block shape set by add_line4
                    } else {
                        line2_config(prec, J.n, true, &J.team, &J.lines_per_block, &nt, &sm, h->seg_chunks);
                        fl.push_back(J);
                    }
                    continue;
                }
                const bool xf = x_first(h->order, h->step_counter + s);
                const bool is_x = (phase == 0) == xf;
                const void *in = phase == 0 ? T[k] : h->tstar;
                void *outp = phase == 0 ? h->tstar : T[k];
                const void *in_lo = h->kahan ? (phase == 0 ? h->tlo : h->tstar_lo) : nullptr;
                void *out_lo = h->kahan ? (phase == 0 ? h->tstar_lo : h->tlo) : nullptr;
                if (!is_x && h->long_cols()) {
                    Launch L{6, 0, 0, 0, 0, 0};
                    L.inst = k;
                    L.dir = ANISO_DIR_Y;
                    L.in = in;
                    L.out = outp;
                    L.in_lo = in_lo;
                    L.out_lo = out_lo;
                    L.dt = dt[k];
                    solo.push_back(L);
                    continue;
                }
                const double lamx = h->chi_par * dt[k] / (h->dx * h->dx);
                const double lamy = h->chi_par * dt[k] / (h->dy * h->dy);
                const double mu = h->chi_par * dt[k] / (h->dx * h->dy);
                const int per = h->bc == ANISO_BC_PERIODIC;
                if (is_x) {
                    LineJob J{};
                    J.Tin = in;
                    J.Tout = outp;
                    J.TinLo = in_lo;
                    J.ToutLo = out_lo;
                    J.g = h->cxx;
                    J.e = h->cxy;
                    J.lam = lamx;
                    J.mu = mu;
                    J.n = h->nx;
                    J.nlines = h->ny;
                    J.per_line = per;
                    J.per_cross = per;
                    int nt;
                    line_config(prec, h->nx, &J.team, &J.lines_per_block, &nt);
                    xl.push_back(J);
                } else {
                    ColJob J{};
                    J.Tin = in;
                    J.Tout = outp;
                    J.TinLo = in_lo;
                    J.ToutLo = out_lo;
                    J.g = h->cyy;
                    J.e = h->cyx;
                    J.lam = lamy;
                    J.mu = mu;
                    J.nx = h->nx;
                    J.ny = h->ny;
                    J.per_x = per;
                    J.per_y = per;
                    yl.push_back(J);
                }
            }
            add_line2(fl, phase);
            {
                const int grp = next_group++;  // the sweep's line4 classes and line5 launch run concurrently
                add_line4(fl4, phase, grp);
                add_line5(fl5, phase, grp);
                add_line6(fl6, phase, grp);
            }
            add_line(xl);
            add_col(yl);
            launches.insert(launches.end(), solo.begin(), solo.end());
        }
        for (size_t i = step_begin; i < launches.size(); ++i) launches[i].step = s;
        step_begin = launches.size();
    }
    if (shape_rc) return shape_rc;
    // diagnostics buffers: the ring of the call and one partials region per
    // concurrent class launch of a y-update
    size_t part_blocks = 0;
    for (const Launch &L : launches)
        if (L.diag_region >= 0) part_blocks = std::max(part_blocks, (size_t)L.nblocks);
    if (diag) {
        const size_t ring = (size_t)n * (size_t)max_steps * 3;
        if (ring > b->ring_count) {
            if (b->d_ring) cudaFree(b->d_ring);
            b->d_ring = nullptr;
            b->ring_count = 0;
            CU(cudaMalloc(&b->d_ring, std::max<size_t>(ring, 3) * sizeof(double)));
            b->ring_count = ring;
        }
        b->ring_steps = max_steps;
        const size_t parts = part_blocks * (1 + aniso_batch::kSide);
        if (parts > b->part_count) {
            if (b->d_part) cudaFree(b->d_part);
            b->d_part = nullptr;
            b->part_count = 0;
            CU(cudaMalloc(&b->d_part, std::max<size_t>(parts, 1) * sizeof(DiagPart)));
            b->part_count = parts;
        }
    }
    // device copy of the job lists
    if (b->d_jobs && b->d_jobs_bytes < blob.size()) {
        cudaFree(b->d_jobs);
        b->d_jobs = nullptr;
    }
    if (!b->d_jobs) {
        CU(cudaMalloc(&b->d_jobs, std::max<size_t>(blob.size(), 16)));
        b->d_jobs_bytes = std::max<size_t>(blob.size(), 16);
    }
    CU(cudaMemcpy(b->d_jobs, blob.data(), blob.size(), cudaMemcpyHostToDevice));

    // capture
    if (!b->cap_stream) CU(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    b->prof.next = b->prof.pool.size();
    b->g_pairs.clear();
    if (!b->fork_ev) {  // branches of concurrent launches
        CU(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming));
        for (int k = 0; k < aniso_batch::kSide; ++k) {
            CU(cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking));
            CU(cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming));
        }
    }
    CU(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = ANISO_OK;
    unsigned *err = b->hs[0]->err;
    if (diag && launch_fill_nan(b->d_ring, (size_t)n * (size_t)max_steps * 3, b->cap_stream) != cudaSuccess)
        rc = fail(ANISO_ERR_CUDA, "diagnostics ring fill failed");
    auto launch_one = [&](const Launch &L, cudaStream_t st) -> cudaError_t {
        if (L.kind == 11 || L.kind == 12) {
            Line2Args a{};
            a.jobs = reinterpret_cast<const Line2Job *>(static_cast<unsigned char *>(b->d_jobs) + L.offset);
            a.njobs = L.njobs;
            a.limiter = b->hs[0]->limiter;
            a.err = err;
            a.block_job = reinterpret_cast<const int *>(static_cast<unsigned char *>(b->d_jobs) + L.table);
            return launch_line6(fp16, a, L.nblocks, L.nthreads, L.smem, st);
        }
        if (L.kind == 9 || L.kind == 10) {
            Line5Args a{};
            a.jobs = reinterpret_cast<const Line5Job *>(static_cast<unsigned char *>(b->d_jobs) + L.offset);
            a.njobs = L.njobs;
            a.total_tiles = L.nblocks;
            a.limiter = b->hs[0]->limiter;
            a.err = err;
            a.test_no_load = tma_mode == 2 ? 1 : 0;
            a.wait_limit = a.test_no_load ? 4096u : (1u << 20);
            a.tile_job = reinterpret_cast<const int *>(static_cast<unsigned char *>(b->d_jobs) + L.table);
            a.pf_dist = L.inst;
            return launch_line5(a, L.nthreads, L.smem, st);
        }
        if (L.kind == 7 || L.kind == 8) {
            Line2Args a{};
            a.jobs = reinterpret_cast<const Line2Job *>(static_cast<unsigned char *>(b->d_jobs) + L.offset);
            a.njobs = L.njobs;
            if (L.table >= 0)
                a.block_job = reinterpret_cast<const int *>(static_cast<unsigned char *>(b->d_jobs) + L.table);
            a.tmem = L.tmem;
            if (L.diag_region >= 0) {
                a.diag_part = b->d_part + (size_t)L.diag_region * part_blocks;
                cudaError_t e = launch_line4(prec, fp16, a, L.nblocks, L.nthreads, L.smem, st);
                if (e != cudaSuccess) return e;
                return launch_diag_finish(a.jobs, L.njobs, a.diag_part, b->d_ring, st);
            }
            a.limiter = b->hs[0]->limiter;
            a.err = err;
            return launch_line4(prec, fp16, a, L.nblocks, L.nthreads, L.smem, st);
        } else if (L.kind >= 2) {
            Line2Args a{};
            a.jobs = reinterpret_cast<const Line2Job *>(static_cast<unsigned char *>(b->d_jobs) + L.offset);
            a.njobs = L.njobs;
            a.limiter = b->hs[0]->limiter;
            a.err = err;
            return launch_line2(prec, fp16, a, L.nblocks, L.nthreads, L.smem, st);
        } else if (L.kind == 0) {
            LineArgs a{};
            a.jobs = reinterpret_cast<const LineJob *>(static_cast<unsigned char *>(b->d_jobs) + L.offset);
            a.njobs = L.njobs;
            a.limiter = b->hs[0]->limiter;
            a.err = err;
            return launch_line(prec, fp16, a, L.nblocks, L.nthreads, L.smem, st, b->hs[0]->kahan != 0);
        }
        ColArgs a{};
        a.jobs = reinterpret_cast<const ColJob *>(static_cast<unsigned char *>(b->d_jobs) + L.offset);
        a.njobs = L.njobs;
        a.limiter = b->hs[0]->limiter;
        a.err = err;
        return launch_col(prec, fp16, a, L.nblocks, L.nthreads, L.smem, st, b->hs[0]->kahan != 0);
    };
    for (size_t i = 0; i < launches.size() && rc == ANISO_OK;) {
        const Launch &L = launches[i];
        if (L.kind == 6 || L.kind == 13) {
            aniso_ctx *h = b->hs[L.inst];
            const int saved = h->profile;  // these sweeps are not profiled inside the batch
            h->profile = 0;
            rc = L.kind == 13 ? enqueue_fast_sweep(h, L.dir, L.out, L.dt, b->cap_stream, nullptr)
                              : enqueue_sweep(h, L.dir, L.in, L.out, L.dt, b->cap_stream, nullptr, L.in_lo, L.out_lo);
            h->profile = saved;
            if (rc) break;
            ++i;
            continue;
        }
        size_t j = i + 1;  // [i, j): one concurrent group
        // (at most 1 + kSide launches run side by side; more of the same group
        // form the next set of branches)
        while (L.group >= 0 && j < launches.size() && launches[j].group == L.group &&
               j - i < (size_t)(1 + aniso_batch::kSide))
            ++j;
        int pidx = -1;
        // (ANISO_OPT_PROFILE k: the sweeps of every k-th step carry events)
        const bool prof = b->profile && L.step % b->profile == 0;
        if (prof) {
            pidx = b->prof.take((L.kind == 0 || L.kind == 2 || L.kind == 7 || L.kind == 9 || L.kind == 11)
                                    ? ANISO_KERNEL_XSWEEP
                                    : ANISO_KERNEL_YSWEEP);
            if (pidx < 0 || cudaEventRecordWithFlags(b->prof.pool[pidx].a, b->cap_stream,
                                                     cudaEventRecordExternal) != cudaSuccess) {
                rc = fail(ANISO_ERR_CUDA, "profiling event failed");
                break;
            }
        }
        cudaError_t ce = cudaSuccess;
        if (j - i == 1) {
            ce = launch_one(L, b->cap_stream);
        } else {
            ce = cudaEventRecord(b->fork_ev, b->cap_stream);
            size_t forked = 0;  // side streams that joined the capture
            for (size_t k = i + 1; k < j && ce == cudaSuccess; ++k) {
                cudaStream_t st = b->side[k - i - 1];
                ce = cudaStreamWaitEvent(st, b->fork_ev, 0);
                if (ce == cudaSuccess) ++forked;
                if (ce == cudaSuccess) ce = launch_one(launches[k], st);
            }
            if (ce == cudaSuccess) ce = launch_one(L, b->cap_stream);
            // every forked branch is joined back, also after an error, so that
            // the capture can end and leave no stream in capture mode
            for (size_t k = 0; k < forked; ++k) {
                cudaError_t e2 = cudaEventRecord(b->join_ev[k], b->side[k]);
                if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(b->cap_stream, b->join_ev[k], 0);
                if (ce == cudaSuccess) ce = e2;
            }
        }
        if (ce != cudaSuccess) {
            rc = fail(ANISO_ERR_CUDA, "batched launch: %s", cudaGetErrorString(ce));
            break;
        }
        if (prof) {
            if (cudaEventRecordWithFlags(b->prof.pool[pidx].b, b->cap_stream, cudaEventRecordExternal) !=
                cudaSuccess) {
                rc = fail(ANISO_ERR_CUDA, "profiling event failed");
                break;
            }
            b->g_pairs.push_back(pidx);
        }
        i = j;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess) return fail(ANISO_ERR_CUDA, "batch capture: %s", cudaGetErrorString(ce));
    {
        size_t nn = 0;
        b->kernels_per_call = 0;
        if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
                for (size_t k = 0; k < nn; ++k) {
                    cudaGraphNodeType t;
                    if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                        ++b->kernels_per_call;
                }
        }
    }
    ce = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(ANISO_ERR_CUDA, "batch instantiate: %s", cudaGetErrorString(ce));
    return ANISO_OK;
}

extern "C" int aniso_step_batched(aniso_batch_t b, void *const *T, const double *dt, const int *nsteps)
{
    TraceRange trace("aniso_step_batched");
    if (!b) return fail(ANISO_ERR_ARG, "aniso_step_batched: null batch");
    if (!T || !dt || !nsteps) return fail(ANISO_ERR_ARG, "aniso_step_batched: null array");
    const int n = (int)b->hs.size();
    for (int k = 0; k < n; ++k) {
        if (!T[k]) return fail(ANISO_ERR_ARG, "aniso_step_batched: T[%d] is NULL", k);
        if (!(dt[k] > 0)) return fail(ANISO_ERR_ARG, "aniso_step_batched: dt[%d] must be > 0", k);
        if (nsteps[k] < 0) return fail(ANISO_ERR_ARG, "aniso_step_batched: nsteps[%d] < 0", k);
    }
    std::vector<int> parity(n);
    for (int k = 0; k < n; ++k)
        parity[k] = b->hs[k]->order == ANISO_ORDER_ALTERNATE ? (int)(b->hs[k]->step_counter & 1) : -b->hs[k]->order;
    const bool hit = b->gexec && b->key_profile == b->profile && b->key_diag == b->hs[0]->diag &&
                     b->key_tma == b->hs[0]->tma_lines && b->key_tmem == b->hs[0]->tmem &&
                     b->key_T == std::vector<void *>(T, T + n) &&
                     b->key_dt == std::vector<double>(dt, dt + n) &&
                     b->key_n == std::vector<int>(nsteps, nsteps + n) && b->key_parity == parity;
    if (!hit) {
        CU(cudaStreamSynchronize(b->stream));
        if (b->profile) {
            int rc = b->prof.drain();
            if (rc) return rc;
        }
        batch_drop(b);
        int rc = batch_build(b, T, dt, nsteps);
        if (rc) return rc;
        b->key_T.assign(T, T + n);
        b->key_dt.assign(dt, dt + n);
        b->key_n.assign(nsteps, nsteps + n);
        b->key_parity = parity;
        b->key_profile = b->profile;
        b->key_diag = b->hs[0]->diag;
        b->key_tma = b->hs[0]->tma_lines;
        b->key_tmem = b->hs[0]->tmem;
    }
    if (b->profile && !b->prof.pending.empty()) {
        CU(cudaStreamSynchronize(b->stream));
        int rc = b->prof.drain();
        if (rc) return rc;
    }
    CU(cudaGraphLaunch(b->gexec, b->stream));
    if (b->profile) b->prof.pending.insert(b->prof.pending.end(), b->g_pairs.begin(), b->g_pairs.end());
    for (int k = 0; k < n; ++k) b->hs[k]->step_counter += nsteps[k];
    return ANISO_OK;
}

// aniso_step_batched on host buffers: each grid's T is copied to a device
// buffer the batch owns, the batched call runs on the device, and the result
// is copied back; returns once the host arrays hold it.
extern "C" int aniso_step_batched_host(aniso_batch_t b, void *const *T_host, const double *dt, const int *nsteps)
{
    TraceRange trace("aniso_step_batched_host");
    if (!b) return fail(ANISO_ERR_ARG, "aniso_step_batched_host: null batch");
    if (!T_host || !dt || !nsteps) return fail(ANISO_ERR_ARG, "aniso_step_batched_host: null array");
    const int n = (int)b->hs.size();
    for (int k = 0; k < n; ++k)
        if (!T_host[k]) return fail(ANISO_ERR_ARG, "aniso_step_batched_host: T_host[%d] is NULL", k);
    if ((int)b->dev_T.size() != n) {
        for (int k = 0; k < n; ++k) {
            void *p = nullptr;
            if (cudaMalloc(&p, b->hs[k]->cells() * b->hs[k]->esz()) != cudaSuccess) {
                (void)cudaGetLastError();
                for (void *q : b->dev_T) cudaFree(q);
                b->dev_T.clear();
                return fail(ANISO_ERR_OOM, "aniso_step_batched_host: device copy of grid %d", k);
            }
            b->dev_T.push_back(p);
        }
    }
    for (int k = 0; k < n; ++k)
        CU(cudaMemcpyAsync(b->dev_T[k], T_host[k], b->hs[k]->cells() * b->hs[k]->esz(), cudaMemcpyHostToDevice,
                           b->stream));
    int rc = aniso_step_batched(b, b->dev_T.data(), dt, nsteps);
    if (rc) return rc;
    for (int k = 0; k < n; ++k)
        CU(cudaMemcpyAsync(T_host[k], b->dev_T[k], b->hs[k]->cells() * b->hs[k]->esz(), cudaMemcpyDeviceToHost,
                           b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return ANISO_OK;
}

extern "C" int aniso_batch_diagnostics(aniso_batch_t b, double *out, long long capacity, int *steps)
{
    if (!b) return fail(ANISO_ERR_ARG, "aniso_batch_diagnostics: null batch");
    if (!b->d_ring || b->key_diag != 1)
        return fail(ANISO_ERR_STATE, "aniso_batch_diagnostics: no batched call has run with ANISO_OPT_DIAGNOSTICS");
    const size_t count = b->hs.size() * (size_t)b->ring_steps * 3;
    if (steps) *steps = b->ring_steps;
    if (!out) return ANISO_OK;
    if (capacity < (long long)count)
        return fail(ANISO_ERR_ARG, "aniso_batch_diagnostics: need %zu doubles, got %lld", count, capacity);
    CU(cudaStreamSynchronize(b->stream));
    CU(cudaMemcpy(out, b->d_ring, count * sizeof(double), cudaMemcpyDeviceToHost));
    return ANISO_OK;
}

// Candidates of the block-shape autotuner: kernel option, warps per block
// (warp-autonomous kernel), 16-byte chunks per lane / segment.
struct Cand {
    int fast, warps, seg;
};
static const Cand kTuneCands[] = {{3, 4, 4}, {3, 8, 4}, {3, 4, 8}, {3, 8, 8}, {3, 4, 2}, {3, 8, 2},
                                  {1, 0, 4}, {1, 0, 8}};
static const int kTuneCount = (int)(sizeof(kTuneCands) / sizeof(kTuneCands[0]));

// Block-shape autotuner of the batched fast path: every candidate (kernel,
// warps per block, chunks per lane) runs `reps` timed graph replays of
// `nsteps` steps on device copies of the grids (after one untimed build and
// replay); the fastest is kept in every handle of the batch.  The caller's
// T, the handles' step counters and their profiling setting are unchanged.
extern "C" int aniso_batch_autotune(aniso_batch_t b, void *const *T, const double *dt, int nsteps, int reps,
                                    int *choice, double *best_ms)
{
    TraceRange trace("aniso_batch_autotune");
    if (!b) return fail(ANISO_ERR_ARG, "aniso_batch_autotune: null batch");
    if (!T || !dt) return fail(ANISO_ERR_ARG, "aniso_batch_autotune: null array");
    if (nsteps < 1 || reps < 1) return fail(ANISO_ERR_ARG, "aniso_batch_autotune: nsteps and reps must be >= 1");
    const int n = (int)b->hs.size();
    if (choice) *choice = -1;
    if (best_ms) *best_ms = 0.0;
    for (int k = 0; k < n; ++k) {
        if (!T[k]) return fail(ANISO_ERR_ARG, "aniso_batch_autotune: T[%d] is NULL", k);
        if (!(dt[k] > 0)) return fail(ANISO_ERR_ARG, "aniso_batch_autotune: dt[%d] must be > 0", k);
    }
    const Cand *cands = kTuneCands;
    const int ncand = kTuneCount;
    // nothing to tune unless some grid is on the fast path
    bool any = false;
    for (aniso_ctx *h : b->hs) any = any || (!h->kahan && h->order == ANISO_ORDER_XY && h->cyyT);
    if (!any) return ANISO_OK;

    struct Saved {
        int fast, warps, seg;
        long long counter;
    };
    std::vector<Saved> saved(n);
    for (int k = 0; k < n; ++k)
        saved[k] = {b->hs[k]->fast, b->hs[k]->l4_warps, b->hs[k]->seg_chunks, b->hs[k]->step_counter};
    const int saved_profile = b->profile;
    b->profile = 0;

    // device copies of the grids, 256-byte aligned
    std::vector<size_t> off(n);
    size_t total = 0;
    for (int k = 0; k < n; ++k) {
        off[k] = total;
        total += (b->hs[k]->cells() * b->hs[k]->esz() + 255) & ~(size_t)255;
    }
    void *scratch = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = ANISO_OK, best = -1;
    float best_t = 0.f;
    std::vector<void *> Ts(n);
    std::vector<int> ns(n, nsteps);
    auto apply = [&](int fast, int warps, int seg) {
        for (aniso_ctx *h : b->hs) {
            h->fast = fast;
            h->l4_warps = warps;
            h->seg_chunks = seg;
            drop_graph(h);
        }
        batch_drop(b);
    };
    if (cudaMalloc(&scratch, std::max<size_t>(total, 256)) != cudaSuccess) {
        rc = fail(ANISO_ERR_OOM, "aniso_batch_autotune: %zu bytes of scratch", total);
    } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = fail(ANISO_ERR_CUDA, "aniso_batch_autotune: event creation failed");
    } else {
        for (int k = 0; k < n; ++k) Ts[k] = static_cast<unsigned char *>(scratch) + off[k];
        for (int ci = 0; ci < ncand && rc == ANISO_OK; ++ci) {
            apply(cands[ci].fast, cands[ci].warps, cands[ci].seg);
            for (int k = 0; k < n && rc == ANISO_OK; ++k)
                if (cudaMemcpyAsync(Ts[k], T[k], b->hs[k]->cells() * b->hs[k]->esz(), cudaMemcpyDeviceToDevice,
                                    b->stream) != cudaSuccess)
                    rc = fail(ANISO_ERR_CUDA, "aniso_batch_autotune: copy failed");
            if (rc) break;
            const int r0 = aniso_step_batched(b, Ts.data(), dt, ns.data());  // build + warm
            if (r0 == ANISO_ERR_UNSUPPORTED) continue;                        // shape does not fit
            if (r0) {
                rc = r0;
                break;
            }
            if (cudaEventRecord(e0, b->stream) != cudaSuccess) {
                rc = fail(ANISO_ERR_CUDA, "aniso_batch_autotune: event record failed");
                break;
            }
            for (int r = 0; r < reps && rc == ANISO_OK; ++r) rc = aniso_step_batched(b, Ts.data(), dt, ns.data());
            if (rc) break;
            float ms = 0.f;
            if (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = fail(ANISO_ERR_CUDA, "aniso_batch_autotune: timing failed");
                break;
            }
            if (best < 0 || ms < best_t) {
                best = ci;
                best_t = ms;
            }
        }
    }
    cudaStreamSynchronize(b->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (scratch) cudaFree(scratch);
    for (int k = 0; k < n; ++k) b->hs[k]->step_counter = saved[k].counter;
    if (best >= 0 && rc == ANISO_OK) {
        apply(cands[best].fast, cands[best].warps, cands[best].seg);
        if (choice) *choice = best;
        if (best_ms) *best_ms = best_t / reps;
    } else {
        for (int k = 0; k < n; ++k) {
            aniso_ctx *h = b->hs[k];
            h->fast = saved[k].fast;
            h->l4_warps = saved[k].warps;
            h->seg_chunks = saved[k].seg;
            drop_graph(h);
        }
        batch_drop(b);
    }
    b->profile = saved_profile;
    return rc;
}

// The candidate table of aniso_batch_autotune (kernel option, warps per
// block, chunks per lane), for callers that report the choice.
extern "C" int aniso_autotune_candidate(int index, int *fast, int *warps, int *seg)
{
    if (index < 0 || index >= kTuneCount)
        return fail(ANISO_ERR_ARG, "aniso_autotune_candidate: index %d out of range", index);
    if (fast) *fast = kTuneCands[index].fast;
    if (warps) *warps = kTuneCands[index].warps;
    if (seg) *seg = kTuneCands[index].seg;
    return ANISO_OK;
}

extern "C" void aniso_batch_destroy(aniso_batch_t b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_drop(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int k = 0; k < aniso_batch::kSide; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->d_jobs) cudaFree(b->d_jobs);
    for (void *p : b->dev_T) cudaFree(p);
    if (b->d_ring) cudaFree(b->d_ring);
    if (b->d_part) cudaFree(b->d_part);
    b->prof.destroy();
    delete b;
}

extern "C" int aniso_batch_kernel_count(aniso_batch_t b, long long *kernels)
{
    if (!b || !kernels) return fail(ANISO_ERR_ARG, "aniso_batch_kernel_count: null argument");
    *kernels = b->gexec ? b->kernels_per_call : 0;
    return ANISO_OK;
}

extern "C" int aniso_kernel_times(aniso_t h, aniso_batch_t b, int kind, double *ms, long long *launches,
                                  int reset)
{
    if ((!h) == (!b)) return fail(ANISO_ERR_ARG, "aniso_kernel_times: pass exactly one of h, b");
    if (kind < 0 || kind > 2) return fail(ANISO_ERR_ARG, "aniso_kernel_times: bad kind %d", kind);
    Profiler &p = h ? h->prof : b->prof;
    CU(cudaStreamSynchronize(h ? h->stream : b->stream));
    int rc = p.drain();
    if (rc) return rc;
    if (ms) *ms = p.ms[kind];
    if (launches) *launches = p.count[kind];
    if (reset) {
        for (int k = 0; k < 3; ++k) {
            p.ms[k] = 0;
            p.count[k] = 0;
        }
    }
    return ANISO_OK;
}
