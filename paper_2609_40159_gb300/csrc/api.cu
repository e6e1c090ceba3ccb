// C ABI of the SpTRSV library (declared in include/sptrsv.h): handles, plans,
// level analysis, rewriting, single and batched solves, adjoints.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <climits>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "solve.cuh"

using namespace spt;

namespace {

// Named NVTX range for a profiler timeline (no cost without a tool attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};
constexpr long long kDefaultWaitNs = 10ll * 1000 * 1000 * 1000;  // 10 s
constexpr int kUpdateRounds = 32;  // fixpoint rounds of an incremental analysis before the full pass

bool debug_mode()
{
    static int on = -1;
    if (on < 0) {
        const char *v = getenv("SPTRSV_DEBUG");
        on = (v && v[0] && v[0] != '0') ? 1 : 0;
    }
    return on == 1;
}

sptrsv_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return SPTRSV_OK;
    if (debug_mode()) fprintf(stderr, "[sptrsv] CUDA error: %s\n", cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SPTRSV_ENOMEM : SPTRSV_ECUDA;
}

// With SPTRSV_DEBUG set, every asynchronous entry point synchronises so that
// a failing kernel is reported by the call that launched it.
sptrsv_status debug_sync(sptrsv_status st, cudaStream_t s, const char *what)
{
    if (st != SPTRSV_OK || !debug_mode()) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) fprintf(stderr, "[sptrsv] %s: %s\n", what, cudaGetErrorString(e));
    return from_cuda(e);
}

// Rows per warp from the mean row length; a heavy tail of long rows (more
// than 0.5 % of the rows with over 32 off-diagonals: one lane would walk
// each of them alone, on the dependency chain) takes a warp per row.
int default_rpw(int32_t n, int64_t nnz, int64_t long_rows = 0)
{
    if (n > 0 && long_rows * 200 > n) return 1;
    const double avg = n > 0 ? (double)nnz / n : 1.0;
    if (avg <= 12) return 32;
    if (avg <= 24) return 16;
    if (avg <= 48) return 8;
    if (avg <= 96) return 4;
    return 1;
}

int default_kt(int k)
{
    int kt = 1;
    while (kt < k && kt < 16) kt <<= 1;
    return kt;
}

bool valid_rpw(int r) { return r == 1 || r == 2 || r == 4 || r == 8 || r == 16 || r == 32; }
bool valid_kt(int k) { return k == 1 || k == 2 || k == 4 || k == 8 || k == 16; }
}  // namespace

struct sptrsv_handle_st {
    cudaStream_t stream = nullptr;
    DeviceInfo di;
    int *d_status = nullptr;
    PlanCtl *d_ctl = nullptr;
    long long *d_scratch = nullptr;  // validation result, max level, stats
    // test hook of the level analysis (sptrsv_debug_withhold_level)
    int32_t dbg_withhold = -1;
    long long dbg_wait_ns = 0;
};

struct PlanMat {
    // one system of a (possibly batched) plan
    sptrsv_csr L{};
    sptrsv_csr T{};
    bool hasT = false;
    int32_t nlevels = 0;
    int32_t *d_lev = nullptr, *d_perm = nullptr, *d_level_ptr = nullptr;
    std::vector<int32_t> h_level_ptr;
    int32_t *d_cp = nullptr, *d_crow = nullptr, *d_tmap = nullptr;
    void *d_cv = nullptr;  // L's values in CSC order (transpose solves)
    uint32_t *d_tmask = nullptr;
    // CSC of T (the adjoint's T^T gathers by column), its column mask
    int32_t *d_tcp = nullptr, *d_trow = nullptr, *d_ttmap = nullptr;
    uint32_t *d_tcmask = nullptr;
    // level-ordered batched schedule (built when first used): inverse of
    // d_perm, row groups of each direction
    int32_t *d_iperm = nullptr;
    LevelGroup *d_lgroups[2] = {nullptr, nullptr};
    int32_t n_lgroups[2] = {0, 0};
};

struct sptrsv_plan_st {
    sptrsv_handle h = nullptr;
    bool batched = false;
    sptrsv_dtype dtype = SPTRSV_F64;
    long long spin = kDefaultWaitNs;  // bounded-wait limit, nanoseconds
    int32_t withhold = -1;
    bool have_csc = false;
    std::vector<void *> owned;
    PlanCtl *d_ctl = nullptr;
    // single system
    PlanMat M;
    int mode = SPTRSV_MODE_SYNCFREE, rpw = 32, kt = 1;
    int32_t *d_chunk_fwd = nullptr, *d_chunk_tr = nullptr;
    int chunk_rpw = 0;
    uint32_t *d_flags = nullptr;
    // value-carrying ready flags of single-right-hand-side solves (16 bytes
    // per row: the solution bits and the epoch)
    unsigned long long *d_vflags = nullptr;
    int grid_level = 0, grid_sf = 0;
    int grid_level_max = 0;  // grid_level at the occupancy maximum
    int32_t max_width = 0;
    // hybrid schedule: thin-level threshold (0 = automatic) and, per
    // direction, the first level of the thin run holding every level
    int32_t thin_rows = 0, seg_rows = -1;
    int32_t *d_seg[2] = {nullptr, nullptr};
    // row-major copies of a column-major right-hand-side block and its
    // solution (sptrsv_solve_layout), grown on demand
    void *d_lay = nullptr;
    size_t lay_bytes = 0;
    // batched
    std::vector<PlanMat> mats;
    std::vector<int64_t> rhs_off, vals_off, row_off;
    BatchMat *d_mats = nullptr;
    std::vector<BatchMat> h_mats;
    // work items of each direction ([0] forward, [1] transpose): per system
    // rows per warp and rhs columns per work item, the items (system, rhs
    // column tile, geometry), their launch order, shared memory and grid
    struct Geom {
        std::vector<int32_t> rpw, tile, sched;
        BatchItem *d_items = nullptr;
        int32_t *d_order = nullptr;
        int32_t nitems = 0;
        size_t smem = 0;
        int grid = 0;
    } geo[2];
    int32_t max_items = 0;
    int last_dir = 0;  // direction of the last batched solve (for the trace)
    RowChunk *d_gchunks = nullptr, *d_tchunks = nullptr;  // all 32-row chunks; chunks with T rows
    int64_t n_gchunks = 0, n_tchunks = 0;
    RowChunk *d_ctiles = nullptr;   // tiles of the CSC value gather: (system, first entry)
    int64_t n_ctiles = 0;
    RowChunk *d_fchunks = nullptr;  // every 32-row chunk of the rewritten systems
    int64_t n_fchunks = 0;
    void *d_bt = nullptr;           // b + T b of the rewritten systems (packed like b)
    long long *d_trace = nullptr;  // per work item: start ns, end ns, SM of the last batch solve
    // steps from host buffers (sptrsv_batch_step_host): two device buffer
    // sets used alternately, a stream for the copies in and one for the
    // copies out (the solves run on the handle's stream)
    struct HostSet {
        void *b = nullptr, *w = nullptr, *x = nullptr, *gbp = nullptr, *gb = nullptr, *gv = nullptr;
        cudaEvent_t h2d = nullptr, comp = nullptr, d2h = nullptr;
        bool used = false;
    } hset[2];
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    int64_t nsteps = 0;

    template <class P> cudaError_t alloc(P **p, size_t bytes)
    {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
        if (e == cudaSuccess) { owned.push_back(q); *p = static_cast<P *>(q); }
        return e;
    }
};

// ------------------------------------------------------------------ handle
extern "C" sptrsv_status sptrsv_create(sptrsv_handle *handle, void *stream)
{
    if (!handle) return SPTRSV_EINVAL;
    *handle = nullptr;
    sptrsv_handle h = new (std::nothrow) sptrsv_handle_st;
    if (!h) return SPTRSV_ENOMEM;
    h->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&h->di.device);
    int sms = 0, smem = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->di.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->di.device);
    h->di.num_sms = sms;
    h->di.max_smem_optin = (size_t)smem;
    if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_ctl, sizeof(PlanCtl));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_scratch, 16 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_ctl, 0, sizeof(PlanCtl));
    if (e != cudaSuccess) {
        cudaFree(h->d_status); cudaFree(h->d_ctl); cudaFree(h->d_scratch);
        delete h;
        return from_cuda(e);
    }
    *handle = h;
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_destroy(sptrsv_handle h)
{
    if (!h) return SPTRSV_EINVAL;
    cudaStreamSynchronize(h->stream);
    cudaFree(h->d_status);
    cudaFree(h->d_ctl);
    cudaFree(h->d_scratch);
    delete h;
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_set_stream(sptrsv_handle h, void *stream)
{
    if (!h) return SPTRSV_EINVAL;
    h->stream = (cudaStream_t)stream;
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_get_status(sptrsv_handle h)
{
    if (!h) return SPTRSV_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    int st = 0;
    e = cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    if (st != 0) cudaMemset(h->d_status, 0, sizeof(int));
    return (sptrsv_status)st;
}

extern "C" const char *sptrsv_status_string(sptrsv_status s)
{
    switch (s) {
    case SPTRSV_OK: return "ok";
    case SPTRSV_EINVAL: return "invalid argument";
    case SPTRSV_ENOTLOWER: return "matrix is not lower triangular";
    case SPTRSV_EDIAG: return "diagonal missing, not last or zero";
    case SPTRSV_EUNSORTED: return "columns of a row are not strictly increasing";
    case SPTRSV_ETARGET: return "rewrite target outside [0, lev(i))";
    case SPTRSV_ENOMEM: return "out of device memory";
    case SPTRSV_ETIMEOUT: return "a bounded device wait gave up";
    case SPTRSV_ECUDA: return "CUDA error";
    case SPTRSV_ENOTSUP: return "not supported";
    case SPTRSV_ERANGE: return "index out of range (bounds-checked build)";
    }
    return "unknown status";
}

// -------------------------------------------------------------- internals
namespace {

sptrsv_status check_csr(const sptrsv_csr *L)
{
    if (!L || L->n < 0 || L->nnz < 0 || L->nnz >= INT_MAX) return SPTRSV_EINVAL;
    if (L->dtype != SPTRSV_F64 && L->dtype != SPTRSV_F32) return SPTRSV_EINVAL;
    if (L->n > 0 && (!L->row_ptr || !L->col_idx || !L->vals)) return SPTRSV_EINVAL;
    return SPTRSV_OK;
}

sptrsv_status validate_impl(sptrsv_handle h, const sptrsv_csr &L, int32_t *bad_row)
{
    if (bad_row) *bad_row = -1;
    if (L.n == 0) return SPTRSV_OK;
    cudaError_t e = launch_validate(L, h->d_scratch, h->stream);
    long long r = LLONG_MAX;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, h->d_scratch, sizeof(r), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    if (r == LLONG_MAX) return SPTRSV_OK;
    if (bad_row) *bad_row = (int32_t)(r / 16);
    return (sptrsv_status)(r % 16);
}

// Levels of L into lev (device, n) and their count.  Validates first.
// Levels of L; rows before 32 * (first_row / 32) keep the levels already in
// `lev` (incremental recompute after a rewrite that left them unchanged).
sptrsv_status levels_impl(sptrsv_handle h, const sptrsv_csr &L, int32_t *lev, int32_t *nlevels,
                          long long spin, int32_t first_row = 0)
{
    *nlevels = 0;
    sptrsv_status st = validate_impl(h, L, nullptr);
    if (st != SPTRSV_OK || L.n == 0) return st;
    cudaStream_t s = h->stream;
    cudaError_t e = cudaMemsetAsync(&h->d_ctl->abort_flag, 0, sizeof(int), s);
    Ctl ctl{h->d_status, &h->d_ctl->abort_flag, &h->d_ctl->ticket};
    if (h->dbg_withhold >= 0 && h->dbg_wait_ns > 0) spin = h->dbg_wait_ns;
    int32_t restart = 0;  // rows from here on are (re)computed by the sync-free pass
    if (first_row > 0 && e == cudaSuccess) {
        // after a change confined to rows >= first_row: fixpoint rounds from
        // the previous levels; a change that propagates through more than
        // kUpdateRounds rounds (a level collapse renumbers every later level)
        // or moves many rows at once is finished by the sync-free pass from
        // the first unsettled row
        bool converged = false;
        e = launch_levels_update(L, first_row, lev, ctl, spin, h->di, s, kUpdateRounds, h->dbg_withhold,
                                 &converged, &restart);
        int hab0 = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&hab0, &h->d_ctl->abort_flag, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return from_cuda(e);
        if (hab0) return SPTRSV_ETIMEOUT;
        if (converged) restart = L.n;
    }
    const int64_t c0 = restart / 32;
    if (e == cudaSuccess && 32 * c0 < L.n) {
        e = cudaMemsetAsync(lev + 32 * c0, 0xFF, sizeof(int32_t) * (size_t)(L.n - 32 * c0), s);
        if (e == cudaSuccess) e = launch_levels(L, lev, ctl, spin, h->di, s, c0, h->dbg_withhold);
    }
    int32_t *dmax = reinterpret_cast<int32_t *>(h->d_scratch + 1);
    if (e == cudaSuccess) e = launch_max(lev, L.n, dmax, s);
    int32_t hm = -1;
    int hab = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hab, &h->d_ctl->abort_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    if (hab) return SPTRSV_ETIMEOUT;
    *nlevels = hm + 1;
    return SPTRSV_OK;
}

sptrsv_status analyze_into(sptrsv_handle h, const sptrsv_csr &L, int32_t *lev, int32_t *perm,
                           int32_t *level_ptr, int64_t *cost, int32_t *nlevels, double *stats,
                           long long spin, int32_t first_row = 0)
{
    sptrsv_status st = levels_impl(h, L, lev, nlevels, spin, first_row);
    if (st != SPTRSV_OK) return st;
    cudaStream_t s = h->stream;
    cudaError_t e = level_partition(L, lev, *nlevels, perm, level_ptr, cost, s);
    if (e == cudaSuccess && stats) {
        double *dst = reinterpret_cast<double *>(h->d_scratch + 2);
        e = launch_level_stats(L.n, L.nnz, *nlevels, level_ptr, cost, dst, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(stats, dst, 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return from_cuda(e);
}

template <class T> Sys<T> sys_of(const PlanMat &M, int *chk)
{
    Sys<T> A;
    A.nnz = M.L.nnz;
    A.chk = chk;
    A.n = M.L.n;
    A.rp = M.L.row_ptr; A.ci = M.L.col_idx; A.v = (const T *)M.L.vals;
    A.cp = M.d_cp; A.crow = M.d_crow; A.tmap = M.d_tmap; A.cv = (const T *)M.d_cv;
    A.trp = M.hasT ? M.T.row_ptr : nullptr;
    A.tci = M.hasT ? M.T.col_idx : nullptr;
    A.tv = M.hasT ? (const T *)M.T.vals : nullptr;
    A.tmask = M.hasT ? M.d_tmask : nullptr;
    A.tcp = M.d_tcp; A.trow = M.d_trow; A.ttmap = M.d_ttmap;
    return A;
}

// Analysis + schedule data + optional CSC for one system of a plan.
sptrsv_status prepare_mat(sptrsv_plan p, PlanMat &M, const sptrsv_csr &L, const sptrsv_csr *T,
                          bool want_csc)
{
    sptrsv_handle h = p->h;
    cudaStream_t s = h->stream;
    M.L = L;
    const int32_t n = L.n;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    if (T && T->n > 0) {
        if (T->n != n || T->dtype != L.dtype || !T->row_ptr || (T->nnz > 0 && (!T->col_idx || !T->vals)))
            return SPTRSV_EINVAL;
        M.T = *T;
        M.hasT = true;
    }
    cudaError_t e = p->alloc(&M.d_lev, sizeof(int32_t) * nn);
    if (e == cudaSuccess) e = p->alloc(&M.d_perm, sizeof(int32_t) * nn);
    if (e == cudaSuccess) e = p->alloc(&M.d_level_ptr, sizeof(int32_t) * (nn + 1));
    int64_t *cost = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&cost, sizeof(int64_t) * nn);
    if (e != cudaSuccess) { cudaFree(cost); return from_cuda(e); }
    sptrsv_status st = analyze_into(h, L, M.d_lev, M.d_perm, M.d_level_ptr, cost, &M.nlevels, nullptr, p->spin);
    cudaFree(cost);
    if (st != SPTRSV_OK) return st;
    M.h_level_ptr.assign((size_t)M.nlevels + 1, 0);
    if (n > 0) {
        e = cudaMemcpy(M.h_level_ptr.data(), M.d_level_ptr, sizeof(int32_t) * (M.nlevels + 1), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (M.hasT) {
        const size_t tnz = (size_t)(M.T.nnz > 0 ? M.T.nnz : 1);
        e = p->alloc(&M.d_tmask, sizeof(uint32_t) * ((nn + 31) / 32));
        if (e == cudaSuccess) e = build_tmask(M.T.row_ptr, n, M.d_tmask, s);
        if (e == cudaSuccess) e = p->alloc(&M.d_tcp, sizeof(int32_t) * (nn + 1));
        if (e == cudaSuccess) e = p->alloc(&M.d_trow, sizeof(int32_t) * tnz);
        if (e == cudaSuccess) e = p->alloc(&M.d_ttmap, sizeof(int32_t) * tnz);
        if (e == cudaSuccess) e = p->alloc(&M.d_tcmask, sizeof(uint32_t) * ((nn + 31) / 32));
        if (e == cudaSuccess)
            e = M.T.nnz > 0 ? build_csc(M.T.row_ptr, M.T.col_idx, n, M.T.nnz, M.d_tcp, M.d_trow, M.d_ttmap, s)
                            : cudaMemsetAsync(M.d_tcp, 0, sizeof(int32_t) * (nn + 1), s);
        if (e == cudaSuccess) e = build_tmask(M.d_tcp, n, M.d_tcmask, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (want_csc) {
        e = p->alloc(&M.d_cp, sizeof(int32_t) * (nn + 1));
        if (e == cudaSuccess) e = p->alloc(&M.d_crow, sizeof(int32_t) * (size_t)(L.nnz > 0 ? L.nnz : 1));
        if (e == cudaSuccess) e = p->alloc(&M.d_tmap, sizeof(int32_t) * (size_t)(L.nnz > 0 ? L.nnz : 1));
        if (e == cudaSuccess)
            e = p->alloc(&M.d_cv, (L.dtype == SPTRSV_F64 ? 8 : 4) * (size_t)(L.nnz > 0 ? L.nnz : 1));
        if (e == cudaSuccess) e = build_csc(L.row_ptr, L.col_idx, n, L.nnz, M.d_cp, M.d_crow, M.d_tmap, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return SPTRSV_OK;
}

sptrsv_status ensure_chunks(sptrsv_plan p)
{
    if (p->chunk_rpw == p->rpw) return SPTRSV_OK;
    const int32_t n = p->M.L.n;
    const int64_t nch = ((int64_t)n + p->rpw - 1) / p->rpw;
    cudaError_t e = cudaSuccess;
    // chunk tables are owned; reallocate at the largest size ever needed
    if (!p->d_chunk_fwd) {
        const int64_t maxch = n > 0 ? n : 1;  // rpw = 1
        e = p->alloc(&p->d_chunk_fwd, sizeof(int32_t) * (size_t)maxch);
        if (e == cudaSuccess) e = p->alloc(&p->d_chunk_tr, sizeof(int32_t) * (size_t)maxch);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (nch > 0 && p->M.nlevels > 0) {
        e = build_chunk_levels(p->M.d_level_ptr, p->M.nlevels, n, p->rpw, false, p->d_chunk_fwd, p->h->stream);
        if (e == cudaSuccess)
            e = build_chunk_levels(p->M.d_level_ptr, p->M.nlevels, n, p->rpw, true, p->d_chunk_tr, p->h->stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    p->chunk_rpw = p->rpw;
    return SPTRSV_OK;
}

// Thin-run heads of the hybrid schedule, per direction (processing order:
// forward = level order, transpose = reverse level order): seg[l] = l for a
// thick level, the run's first level for a level of a run of consecutive
// thin levels.
sptrsv_status ensure_hybrid(sptrsv_plan p)
{
    const PlanMat &M = p->M;
    const int32_t L = M.nlevels;
    // automatic: every level thin (one synchronisation-free run in level
    // order); barriers before thick levels measured slower on every
    // workload tried (2D/3D Laplacians, power-law DAG, banded)
    const int32_t thr = p->thin_rows > 0 ? p->thin_rows : INT32_MAX;
    if (p->seg_rows == thr && p->d_seg[0]) return SPTRSV_OK;
    cudaError_t e = cudaSuccess;
    for (int d = 0; d < 2 && e == cudaSuccess; ++d)
        if (!p->d_seg[d]) e = p->alloc(&p->d_seg[d], sizeof(int32_t) * (size_t)std::max(L, 1));
    if (e != cudaSuccess) return from_cuda(e);
    std::vector<int32_t> seg((size_t)std::max(L, 1));
    for (int d = 0; d < 2 && e == cudaSuccess; ++d) {
        for (int32_t k = 0; k < L; ++k) {
            const int32_t l = d == 0 ? k : L - 1 - k;  // level of processing index k
            const bool thin = M.h_level_ptr[l + 1] - M.h_level_ptr[l] < thr;
            const int32_t l_prev = d == 0 ? k - 1 : L - k;
            const bool prev_thin = k > 0 && M.h_level_ptr[l_prev + 1] - M.h_level_ptr[l_prev] < thr;
            seg[k] = thin && prev_thin ? seg[k - 1] : k;
        }
        if (L > 0) e = cudaMemcpy(p->d_seg[d], seg.data(), sizeof(int32_t) * L, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return from_cuda(e);
    p->seg_rows = thr;
    return SPTRSV_OK;
}

// Mode from the mean level width: narrow (deep) systems stay on one SM,
// very wide levels go level by level (row-order sync-free solving keeps
// only the rows in flight near the wavefront and idles on wide, far-reaching
// levels: 9x slower than level order on the 3D Laplacian), the rest takes
// the hybrid schedule (synchronisation-free in level order: 3.8x faster than
// row order on the power-law DAG, 1.7x on the 2D Laplacian).
int auto_mode(const PlanMat &M)
{
    if (M.L.n == 0 || M.nlevels == 0) return SPTRSV_MODE_SYNCFREE;
    const double width = (double)M.L.n / M.nlevels;
    if (width < 48.0) return SPTRSV_MODE_BLOCK;
    if (width >= 2048.0) return SPTRSV_MODE_LEVEL_PERSISTENT;
    return SPTRSV_MODE_HYBRID;
}

template <class T>
sptrsv_status solve_impl(sptrsv_plan p, const void *b, void *x, int32_t nrhs, int64_t ld, bool trans)
{
    const PlanMat &M = p->M;
    if (M.L.n == 0) return SPTRSV_OK;
    if (!b || !x || nrhs < 1 || ld < nrhs) return SPTRSV_EINVAL;
    if (trans && !p->have_csc) return SPTRSV_ENOTSUP;
    cudaStream_t s = p->h->stream;
    Sys<T> A = sys_of<T>(M, p->h->d_status);
    Rhs<T> R{(const T *)b, (T *)x, ld, nrhs};
    if (trans) {
        cudaError_t eg = csc_values<T>(M.d_tmap, (const T *)M.L.vals, (T *)M.d_cv, M.L.nnz, s);
        if (eg != cudaSuccess) return from_cuda(eg);
    }
    SyncArgs sy{p->d_flags, p->d_ctl, p->withhold, Waiter{p->h->d_status, &p->d_ctl->abort_flag, p->spin}};
    // one right-hand side: the synchronisation-free waits read the values
    // from the flags themselves
    if (nrhs == 1) sy.vflags = p->d_vflags;
    const int kt = std::min(p->kt, default_kt(nrhs));
    cudaError_t e = cudaSuccess;
    int mode = p->mode;
    if (mode == SPTRSV_MODE_BLOCK && !block_mode_supported(nrhs, sizeof(T) == 8)) mode = SPTRSV_MODE_SYNCFREE;
    switch (mode) {
    case SPTRSV_MODE_LEVEL_LAUNCH:
        e = solve_level_launch<T>(A, M.d_perm, M.h_level_ptr, R, trans, s);
        break;
    case SPTRSV_MODE_LEVEL_PERSISTENT: {
        sptrsv_status st = ensure_chunks(p);
        if (st != SPTRSV_OK) return st;
        Sched S{M.d_perm, M.d_level_ptr, M.nlevels, trans ? p->d_chunk_tr : p->d_chunk_fwd,
                ((int64_t)M.L.n + p->rpw - 1) / p->rpw};
        const int64_t want = (2 * (int64_t)p->max_width / p->rpw + 7) / 8;  // blocks of 8 warps
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(p->grid_level, want));
        e = solve_level_persistent<T>(A, S, R, p->rpw, kt, trans, sy, grid, s);
        break;
    }
    case SPTRSV_MODE_HYBRID: {
        sptrsv_status st = ensure_chunks(p);
        if (st == SPTRSV_OK) st = ensure_hybrid(p);
        if (st != SPTRSV_OK) return st;
        Sched S{M.d_perm, M.d_level_ptr, M.nlevels, trans ? p->d_chunk_tr : p->d_chunk_fwd,
                ((int64_t)M.L.n + p->rpw - 1) / p->rpw, p->d_seg[trans ? 1 : 0], M.d_lev};
        e = solve_level_persistent<T>(A, S, R, p->rpw, kt, trans, sy, p->grid_level, s);
        break;
    }
    case SPTRSV_MODE_BLOCK: {
        const double width = M.nlevels > 0 ? (double)M.L.n / M.nlevels : 1.0;
        e = solve_block<T>(A, R, p->rpw, kt, trans, sy, block_warps_for(width, p->rpw), s);
        break;
    }
    default:
        e = solve_syncfree<T>(A, R, p->rpw, kt, trans, sy, p->grid_sf, s);
        break;
    }
    return debug_sync(from_cuda(e), s, trans ? "solve_transpose" : "solve");
}

}  // namespace

// --------------------------------------------------------------- validate
extern "C" sptrsv_status sptrsv_validate(sptrsv_handle h, const sptrsv_csr *L, int32_t *bad_row)
{
    if (!h) return SPTRSV_EINVAL;
    sptrsv_status st = check_csr(L);
    if (st != SPTRSV_OK) return st;
    return validate_impl(h, *L, bad_row);
}

// ---------------------------------------------------------------- analyze
extern "C" sptrsv_status sptrsv_analyze(sptrsv_handle h, const sptrsv_csr *L, int32_t *lev,
                                        int32_t *perm, int32_t *level_ptr, int64_t *level_cost,
                                        int32_t *nlevels, double stats[6])
{
    Range range("sptrsv_analyze");
    if (!h || !nlevels) return SPTRSV_EINVAL;
    sptrsv_status st = check_csr(L);
    if (st != SPTRSV_OK) return st;
    if (L->n > 0 && (!lev || !perm || !level_ptr || !level_cost)) return SPTRSV_EINVAL;
    if (L->n == 0) {
        *nlevels = 0;
        if (stats) for (int q = 0; q < 6; ++q) stats[q] = 0.0;
        if (level_ptr) cudaMemsetAsync(level_ptr, 0, sizeof(int32_t), h->stream);
        return from_cuda(cudaStreamSynchronize(h->stream));
    }
    double tmp[6];
    return analyze_into(h, *L, lev, perm, level_ptr, level_cost, nlevels, stats ? stats : tmp, kDefaultWaitNs);
}

extern "C" sptrsv_status sptrsv_analyze_incremental(sptrsv_handle h, const sptrsv_csr *L, int32_t first_row,
                                                    int32_t *lev, int32_t *perm, int32_t *level_ptr,
                                                    int64_t *level_cost, int32_t *nlevels, double stats[6])
{
    Range range("sptrsv_analyze_incremental");
    if (!h || !nlevels) return SPTRSV_EINVAL;
    sptrsv_status st = check_csr(L);
    if (st != SPTRSV_OK) return st;
    if (first_row < 0 || first_row > L->n) return SPTRSV_EINVAL;
    if (L->n == 0) return sptrsv_analyze(h, L, lev, perm, level_ptr, level_cost, nlevels, stats);
    if (!lev || !perm || !level_ptr || !level_cost) return SPTRSV_EINVAL;
    double tmp[6];
    return analyze_into(h, *L, lev, perm, level_ptr, level_cost, nlevels, stats ? stats : tmp, kDefaultWaitNs,
                        first_row);
}

extern "C" sptrsv_status sptrsv_level_summary(sptrsv_handle h, const sptrsv_csr *L, const int32_t *perm,
                                              const int32_t *level_ptr, const int64_t *level_cost,
                                              int32_t nlevels, double threshold, uint8_t *thin,
                                              int32_t *pick, int64_t summary[3])
{
    Range range("sptrsv_level_summary");
    if (!h || !L || !summary || nlevels < 0) return SPTRSV_EINVAL;
    if (nlevels > 0 && (!L->row_ptr || !perm || !level_ptr || !level_cost || !thin || !pick)) return SPTRSV_EINVAL;
    unsigned long long *d = reinterpret_cast<unsigned long long *>(h->d_scratch + 9);
    unsigned long long host[3] = {0, 0, 0};
    cudaError_t e = launch_level_summary(L->row_ptr, perm, level_ptr, level_cost, nlevels, threshold, thin, pick,
                                         d, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, d, sizeof(host), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    for (int q = 0; q < 3; ++q) summary[q] = (int64_t)host[q];
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_transpose(sptrsv_handle h, const sptrsv_csr *A, sptrsv_csr_out *At)
{
    Range range("sptrsv_transpose");
    if (!h || !A || !At || A->n < 0 || A->nnz < 0) return SPTRSV_EINVAL;
    if (A->dtype != SPTRSV_F64 && A->dtype != SPTRSV_F32) return SPTRSV_EINVAL;
    if (!At->row_ptr || (A->n > 0 && !A->row_ptr)) return SPTRSV_EINVAL;
    if (A->nnz > 0 && (!A->col_idx || !A->vals || !At->col_idx || !At->vals)) return SPTRSV_EINVAL;
    cudaStream_t s = h->stream;
    int32_t *tmap = nullptr;
    cudaError_t e = cudaMallocAsync(&tmap, sizeof(int32_t) * (size_t)(A->nnz > 0 ? A->nnz : 1), s);
    if (e == cudaSuccess) e = build_csc(A->row_ptr, A->col_idx, A->n, A->nnz, At->row_ptr, At->col_idx, tmap, s);
    if (e == cudaSuccess && A->nnz > 0)
        e = A->dtype == SPTRSV_F64
                ? csc_values<double>(tmap, (const double *)A->vals, (double *)At->vals, A->nnz, s)
                : csc_values<float>(tmap, (const float *)A->vals, (float *)At->vals, A->nnz, s);
    if (tmap) cudaFreeAsync(tmap, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return from_cuda(e);
}

// ---------------------------------------------------------------- rewrite
extern "C" sptrsv_status sptrsv_rewrite(sptrsv_handle h, const sptrsv_csr *L, const int32_t *lev,
                                        const int32_t *rows, const int32_t *targets, int32_t nrows,
                                        int64_t *nnz_Lp, int64_t *nnz_T, sptrsv_csr_out *Lp_out,
                                        sptrsv_csr_out *T_out)
{
    Range range("sptrsv_rewrite");
    if (!h || nrows < 0) return SPTRSV_EINVAL;
    sptrsv_status st = check_csr(L);
    if (st != SPTRSV_OK) return st;
    if (L->n > 0 && !lev) return SPTRSV_EINVAL;
    if (nrows > 0 && !rows) return SPTRSV_EINVAL;
    return (sptrsv_status)rewrite_run(*L, lev, rows, targets, nrows, nnz_Lp, nnz_T, Lp_out, T_out,
                                      h->di, h->stream);
}

// ------------------------------------------------------------------ plans
extern "C" sptrsv_status sptrsv_plan_create(sptrsv_handle h, const sptrsv_csr *L, const sptrsv_csr *T,
                                            const sptrsv_plan_opts *opts, sptrsv_plan *plan)
{
    Range range("sptrsv_plan_create");
    if (!h || !plan) return SPTRSV_EINVAL;
    *plan = nullptr;
    sptrsv_status st = check_csr(L);
    if (st != SPTRSV_OK) return st;
    sptrsv_plan p = new (std::nothrow) sptrsv_plan_st;
    if (!p) return SPTRSV_ENOMEM;
    p->h = h;
    p->dtype = L->dtype;
    sptrsv_plan_opts o{};
    if (opts) o = *opts;
    if (o.wait_limit_us > 0) p->spin = o.wait_limit_us * 1000;
    cudaError_t e = p->alloc(&p->d_ctl, sizeof(PlanCtl));
    if (e == cudaSuccess) e = cudaMemset(p->d_ctl, 0, sizeof(PlanCtl));
    if (e == cudaSuccess) e = p->alloc(&p->d_flags, sizeof(uint32_t) * (size_t)(L->n > 0 ? L->n : 1));
    if (e == cudaSuccess) e = cudaMemset(p->d_flags, 0, sizeof(uint32_t) * (size_t)(L->n > 0 ? L->n : 1));
    if (e == cudaSuccess) e = p->alloc(&p->d_vflags, 16 * (size_t)(L->n > 0 ? L->n : 1));
    if (e == cudaSuccess) e = cudaMemset(p->d_vflags, 0, 16 * (size_t)(L->n > 0 ? L->n : 1));
    if (e != cudaSuccess) { sptrsv_plan_destroy(p); return from_cuda(e); }
    st = prepare_mat(p, p->M, *L, T, o.build_transpose != 0);
    if (st != SPTRSV_OK) { sptrsv_plan_destroy(p); return st; }
    p->have_csc = o.build_transpose != 0;
    p->mode = o.mode != SPTRSV_MODE_AUTO ? o.mode : auto_mode(p->M);
    if (valid_rpw(o.rows_per_warp)) {
        p->rpw = o.rows_per_warp;
    } else {
        unsigned long long nlong = 0;
        unsigned long long *d = reinterpret_cast<unsigned long long *>(h->d_scratch + 8);
        cudaError_t e = launch_count_long(L->row_ptr, L->n, 32, d, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nlong, d, sizeof(nlong), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { sptrsv_plan_destroy(p); return from_cuda(e); }
        p->rpw = default_rpw(L->n, L->nnz, (int64_t)nlong);
    }
    // the hybrid schedule waits row by row on flags: 4 rows per warp (8
    // lanes a row; on the 2D Laplacian 3.2 ms against 4.2 ms with one row
    // per warp), one row per warp where long rows call for a whole warp
    // (heavy tail or long mean row: the row-length rule above gave 1)
    if (p->mode == SPTRSV_MODE_HYBRID && !valid_rpw(o.rows_per_warp)) p->rpw = p->rpw == 1 ? 1 : 4;
    p->kt = valid_kt(o.rhs_tile) ? o.rhs_tile : 16;
    if (p->mode < SPTRSV_MODE_LEVEL_LAUNCH || p->mode > SPTRSV_MODE_HYBRID) { sptrsv_plan_destroy(p); return SPTRSV_EINVAL; }
    p->grid_level = persistent_grid_level(1, p->dtype == SPTRSV_F64, h->di);
    p->grid_level_max = p->grid_level;
    {
        // warps beyond about twice the widest level only poll the progress
        // counter: cap the level-persistent grid accordingly
        int32_t maxw = 0;
        for (int32_t l = 0; l < p->M.nlevels; ++l)
            maxw = std::max(maxw, p->M.h_level_ptr[l + 1] - p->M.h_level_ptr[l]);
        p->max_width = maxw;
    }
    p->grid_sf = persistent_grid_syncfree(1, p->dtype == SPTRSV_F64, h->di);
    st = ensure_chunks(p);
    if (st == SPTRSV_OK) st = from_cuda(cudaStreamSynchronize(h->stream));
    if (st != SPTRSV_OK) { sptrsv_plan_destroy(p); return st; }
    *plan = p;
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_plan_destroy(sptrsv_plan p)
{
    if (!p) return SPTRSV_EINVAL;
    if (p->h) cudaStreamSynchronize(p->h->stream);
    for (auto &S : p->hset)
        for (cudaEvent_t ev : {S.h2d, S.comp, S.d2h})
            if (ev) cudaEventDestroy(ev);
    for (cudaStream_t st : {p->s_h2d, p->s_d2h})
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    if (p->d_lay) cudaFree(p->d_lay);
    for (void *q : p->owned) cudaFree(q);
    delete p;
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_plan_set_thin_rows(sptrsv_plan p, int32_t thin_rows)
{
    if (!p || p->batched || thin_rows < 0) return SPTRSV_EINVAL;
    p->thin_rows = thin_rows;
    return p->mode == SPTRSV_MODE_HYBRID ? ensure_hybrid(p) : SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_plan_set_blocks_per_sm(sptrsv_plan p, int32_t blocks_per_sm)
{
    if (!p || p->batched || blocks_per_sm < 0) return SPTRSV_EINVAL;
    const int sms = std::max(1, p->h->di.num_sms);
    const int cap = (int)std::min<int64_t>(p->grid_level_max, (int64_t)blocks_per_sm * sms);
    p->grid_level = blocks_per_sm == 0 ? p->grid_level_max : std::max(1, cap);
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_plan_info(sptrsv_plan p, int32_t *nlevels, int32_t *mode,
                                          int32_t *rows_per_warp, int32_t *rhs_tile)
{
    if (!p) return SPTRSV_EINVAL;
    if (nlevels) {
        if (p->batched) {
            int32_t mx = 0;
            for (const PlanMat &M : p->mats) mx = std::max(mx, M.nlevels);
            *nlevels = mx;
        } else {
            *nlevels = p->M.nlevels;
        }
    }
    if (mode) *mode = p->batched ? SPTRSV_MODE_BLOCK : p->mode;
    if (rows_per_warp) *rows_per_warp = p->batched ? (p->geo[0].rpw.empty() ? 32 : p->geo[0].rpw[0]) : p->rpw;
    if (rhs_tile) *rhs_tile = p->batched ? (p->geo[0].tile.empty() ? 4 : p->geo[0].tile[0]) : p->kt;
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_plan_set(sptrsv_plan p, int32_t mode, int32_t rows_per_warp, int32_t rhs_tile)
{
    if (!p || p->batched) return SPTRSV_EINVAL;
    if (mode < SPTRSV_MODE_AUTO || mode > SPTRSV_MODE_HYBRID) return SPTRSV_EINVAL;
    if (rows_per_warp != 0 && !valid_rpw(rows_per_warp)) return SPTRSV_EINVAL;
    if (rhs_tile != 0 && !valid_kt(rhs_tile)) return SPTRSV_EINVAL;
    p->mode = mode == SPTRSV_MODE_AUTO ? auto_mode(p->M) : mode;
    if (rows_per_warp) p->rpw = rows_per_warp;
    if (rhs_tile) p->kt = rhs_tile;
    sptrsv_status st = ensure_chunks(p);
    if (st != SPTRSV_OK) return st;
    return from_cuda(cudaStreamSynchronize(p->h->stream));
}

extern "C" sptrsv_status sptrsv_solve(sptrsv_plan p, const void *b, void *x, int32_t nrhs, int64_t ld)
{
    Range range("sptrsv_solve");
    if (!p || p->batched) return SPTRSV_EINVAL;
    return p->dtype == SPTRSV_F64 ? solve_impl<double>(p, b, x, nrhs, ld, false)
                                  : solve_impl<float>(p, b, x, nrhs, ld, false);
}

extern "C" sptrsv_status sptrsv_solve_transpose(sptrsv_plan p, const void *gx, void *gb, int32_t nrhs, int64_t ld)
{
    Range range("sptrsv_solve_transpose");
    if (!p || p->batched) return SPTRSV_EINVAL;
    return p->dtype == SPTRSV_F64 ? solve_impl<double>(p, gx, gb, nrhs, ld, true)
                                  : solve_impl<float>(p, gx, gb, nrhs, ld, true);
}

namespace {
template <class T>
sptrsv_status solve_colmajor(sptrsv_plan p, const void *b, void *x, int32_t nrhs, int64_t ld, bool trans)
{
    const int64_t n = p->M.L.n;
    const size_t need = 2 * sizeof(T) * (size_t)n * (size_t)nrhs;
    cudaStream_t s = p->h->stream;
    if (need > p->lay_bytes) {
        cudaError_t e = cudaStreamSynchronize(s);  // the old buffer may still be in use
        if (e == cudaSuccess && p->d_lay) e = cudaFree(p->d_lay);
        p->d_lay = nullptr;
        p->lay_bytes = 0;
        if (e == cudaSuccess) e = cudaMalloc(&p->d_lay, need);
        if (e != cudaSuccess) return from_cuda(e);
        p->lay_bytes = need;
    }
    T *rb = static_cast<T *>(p->d_lay);
    T *rx = rb + (size_t)n * nrhs;
    // column r of b (element (i, r) at r * ld + i) -> row-major [n x nrhs]
    cudaError_t e = transpose_dense<T>(static_cast<const T *>(b), ld, rb, nrhs, nrhs, n, s);
    if (e != cudaSuccess) return from_cuda(e);
    sptrsv_status st = solve_impl<T>(p, rb, rx, nrhs, nrhs, trans);
    if (st != SPTRSV_OK) return st;
    return from_cuda(transpose_dense<T>(rx, nrhs, static_cast<T *>(x), ld, n, nrhs, s));
}
}  // namespace

extern "C" sptrsv_status sptrsv_solve_layout(sptrsv_plan p, const void *b, void *x, int32_t nrhs, int64_t ld,
                                             int32_t layout, int32_t transpose)
{
    Range range("sptrsv_solve_layout");
    if (!p || p->batched || (layout != SPTRSV_ROW_MAJOR && layout != SPTRSV_COL_MAJOR)) return SPTRSV_EINVAL;
    const bool tr = transpose != 0;
    if (layout == SPTRSV_ROW_MAJOR || nrhs == 1) {
        // one column: both layouts are the same vector
        const int64_t ldr = layout == SPTRSV_ROW_MAJOR ? ld : 1;
        if (layout == SPTRSV_COL_MAJOR && ld < p->M.L.n) return SPTRSV_EINVAL;
        return p->dtype == SPTRSV_F64 ? solve_impl<double>(p, b, x, nrhs, ldr, tr)
                                      : solve_impl<float>(p, b, x, nrhs, ldr, tr);
    }
    if (p->M.L.n == 0) return SPTRSV_OK;
    if (!b || !x || nrhs < 1 || ld < p->M.L.n) return SPTRSV_EINVAL;
    if (tr && !p->have_csc) return SPTRSV_ENOTSUP;
    return p->dtype == SPTRSV_F64 ? solve_colmajor<double>(p, b, x, nrhs, ld, tr)
                                  : solve_colmajor<float>(p, b, x, nrhs, ld, tr);
}

extern "C" sptrsv_status sptrsv_grad_vals(sptrsv_plan p, const void *gb, const void *x, int32_t nrhs,
                                          int64_t ld, void *gvals)
{
    Range range("sptrsv_grad_vals");
    if (!p || p->batched) return SPTRSV_EINVAL;
    if (p->M.L.n == 0) return SPTRSV_OK;
    if (!gb || !x || !gvals || nrhs < 1 || ld < nrhs) return SPTRSV_EINVAL;
    cudaError_t e;
    if (p->dtype == SPTRSV_F64)
        e = grad_vals<double>(sys_of<double>(p->M, p->h->d_status), (const double *)gb, (const double *)x, ld, nrhs, (double *)gvals, p->h->stream);
    else
        e = grad_vals<float>(sys_of<float>(p->M, p->h->d_status), (const float *)gb, (const float *)x, ld, nrhs, (float *)gvals, p->h->stream);
    return from_cuda(e);
}

extern "C" sptrsv_status sptrsv_tt_apply(sptrsv_plan p, const void *gbp, void *gb, int32_t nrhs, int64_t ld)
{
    Range range("sptrsv_tt_apply");
    if (!p || p->batched) return SPTRSV_EINVAL;
    if (p->M.L.n == 0) return SPTRSV_OK;
    if (!gbp || !gb || nrhs < 1 || ld < nrhs) return SPTRSV_EINVAL;
    cudaError_t e;
    if (p->dtype == SPTRSV_F64)
        e = tt_apply<double>(sys_of<double>(p->M, p->h->d_status), (const double *)gbp, (double *)gb, ld, nrhs, p->h->stream);
    else
        e = tt_apply<float>(sys_of<float>(p->M, p->h->d_status), (const float *)gbp, (float *)gb, ld, nrhs, p->h->stream);
    return from_cuda(e);
}

extern "C" sptrsv_status sptrsv_debug_withhold_row(sptrsv_plan p, int32_t row)
{
    if (!p) return SPTRSV_EINVAL;
    p->withhold = row;
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_debug_withhold_level(sptrsv_handle h, int32_t row, int64_t wait_limit_us)
{
    if (!h || (row >= 0 && wait_limit_us <= 0)) return SPTRSV_EINVAL;
    h->dbg_withhold = row < 0 ? -1 : row;
    h->dbg_wait_ns = row < 0 ? 0 : wait_limit_us * 1000;
    return SPTRSV_OK;
}

// ----------------------------------------------------------------- batched
namespace {
bool valid_tile(int t) { return t == 1 || t == 2 || t == 4 || t == 8; }

int pow2_at_least(int v)
{
    int k = 1;
    while (k < v) k <<= 1;
    return k;
}

// Work items of one direction of a batch: every system is split into tiles
// of at most `tile` right-hand-side columns, each an independent in-order
// chain solved by one thread block.  Builds the items with their geometry,
// orders them longest estimated chain first (LPT), and sizes shared memory
// and the grid.
sptrsv_status rebuild_items(sptrsv_plan p, int dir)
{
    sptrsv_plan_st::Geom &G = p->geo[dir];
    const int32_t nmat = (int32_t)p->mats.size();
    const bool f64 = p->dtype == SPTRSV_F64;
    std::vector<BatchItem> items;
    std::vector<double> est;
    size_t smem = 16;
    for (int m = 0; m < nmat; ++m) {
        const PlanMat &M = p->mats[m];
        const int k = p->h_mats[m].k;
        const int tile = G.tile[m];
        for (int r0 = 0; r0 < k; r0 += tile) {
            BatchItem I{};
            I.mat = m;
            I.r0 = r0;
            I.kt = std::min(tile, k - r0);
            I.KT = pow2_at_least(I.kt);
            I.sched = G.sched[m];
            I.rpw = I.sched == kSchedLevel ? 32 : G.rpw[m];
            I.nw = I.sched == kSchedLevel
                       ? kBatchWarps
                       : std::min(kBatchWarps,
                                  block_warps_for(M.nlevels > 0 ? (double)M.L.n / M.nlevels : 1.0, I.rpw));
            block_geometry(I.rpw, I.KT, f64, I.nw, &I.kc, &I.P, kBatchSmemGrow);
            smem = std::max(smem, block_smem_bytes(I.rpw, I.KT, I.kc, f64, I.nw));
            items.push_back(I);
            // in order: a chain of n / 32 row groups whose cost grows with
            // the tile width; level-ordered: a chain of one or more groups per
            // level (each about a third of an in-order group); plus the
            // streamed matrix
            const double chain = I.sched == kSchedLevel ? 12.0 * (double)M.nlevels + 0.1 * (double)M.L.n
                                                        : (double)M.L.n;
            est.push_back(chain * (1.0 + 0.1 * I.KT) + 0.01 * (double)M.L.nnz);
        }
    }
    if (smem > kBlockSmemBudget) return SPTRSV_ENOTSUP;
    const int32_t ni = (int32_t)items.size();
    if (ni > p->max_items) return SPTRSV_EINVAL;
    std::vector<int32_t> order((size_t)ni);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return est[x] > est[y]; });
    cudaError_t e = cudaStreamSynchronize(p->h->stream);
    if (e == cudaSuccess && ni > 0)
        e = cudaMemcpy(G.d_items, items.data(), sizeof(BatchItem) * ni, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ni > 0)
        e = cudaMemcpy(G.d_order, order.data(), sizeof(int32_t) * ni, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return from_cuda(e);
    G.nitems = ni;
    G.smem = smem;
    G.grid = std::min(batch_grid(smem, p->h->di), std::max(ni, 1));
    return SPTRSV_OK;
}

// Tables of the level-ordered schedule of system m in direction dir: the
// inverse permutation (once per system) and the row groups: every level's
// positions cut into groups of at most 32, in level order (forward) or in
// reverse level order (transpose), each with the number of groups of the
// levels before it in that order.
sptrsv_status ensure_level_tables(sptrsv_plan p, int m, int dir)
{
    PlanMat &M = p->mats[m];
    const int32_t n = M.L.n;
    cudaError_t e = cudaSuccess;
    if (!M.d_iperm) {
        e = p->alloc(&M.d_iperm, sizeof(int32_t) * (size_t)std::max(n, 1));
        if (e == cudaSuccess) e = inverse_perm(M.d_perm, M.d_iperm, n, p->h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->h->stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (!M.d_lgroups[dir]) {
        std::vector<LevelGroup> g;
        const int32_t L = M.nlevels;
        const std::vector<int32_t> &lp = M.h_level_ptr;
        for (int32_t k = 0; k < L; ++k) {
            const int32_t l = dir == 0 ? k : L - 1 - k;
            // positions of level l in this direction's order
            const int32_t s = dir == 0 ? lp[l] : n - lp[l + 1];
            const int32_t t = dir == 0 ? lp[l + 1] : n - lp[l];
            const int32_t first = (int32_t)g.size();
            for (int32_t q = s; q < t; q += 32) g.push_back(LevelGroup{q, std::min(32, t - q), t, first});
        }
        e = p->alloc(&M.d_lgroups[dir], sizeof(LevelGroup) * std::max<size_t>(g.size(), 1));
        if (e == cudaSuccess && !g.empty())
            e = cudaMemcpy(M.d_lgroups[dir], g.data(), sizeof(LevelGroup) * g.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return from_cuda(e);
        M.n_lgroups[dir] = (int32_t)g.size();
    }
    BatchMat &B = p->h_mats[m];
    B.perm = M.d_perm;
    B.iperm = M.d_iperm;
    B.lgroups[dir] = M.d_lgroups[dir];
    B.nlgroups[dir] = M.n_lgroups[dir];
    e = cudaStreamSynchronize(p->h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_mats + m, &B, sizeof(BatchMat), cudaMemcpyHostToDevice);
    return from_cuda(e);
}

// New per-system schedules (SPTRSV_BATCH_INORDER / _LEVEL; 0 keeps) for the
// directions in `dirs`.
sptrsv_status set_schedule(sptrsv_plan p, int dirs, const int32_t *schedule)
{
    const int32_t nmat = (int32_t)p->h_mats.size();
    for (int m = 0; m < nmat; ++m)
        if (schedule[m] != 0 && schedule[m] != SPTRSV_BATCH_INORDER && schedule[m] != SPTRSV_BATCH_LEVEL)
            return SPTRSV_EINVAL;
    for (int d = 0; d < 2; ++d) {
        if (!((dirs >> d) & 1)) continue;
        sptrsv_plan_st::Geom &G = p->geo[d];
        const std::vector<int32_t> old = G.sched;
        for (int m = 0; m < nmat; ++m) {
            if (schedule[m] == SPTRSV_BATCH_LEVEL) {
                sptrsv_status st = ensure_level_tables(p, m, d);
                if (st != SPTRSV_OK) return st;
                G.sched[m] = kSchedLevel;
            } else if (schedule[m] == SPTRSV_BATCH_INORDER) {
                G.sched[m] = kSchedInOrder;
            }
        }
        sptrsv_status st = rebuild_items(p, d);
        if (st == SPTRSV_ENOTSUP) {
            G.sched = old;
            if (rebuild_items(p, d) != SPTRSV_OK) return SPTRSV_ECUDA;
        }
        if (st != SPTRSV_OK) return st;
    }
    return SPTRSV_OK;
}

// New per-system geometry for the directions in `dirs` (bit 0 forward, bit
// 1 transpose); values 0 keep the current one.  A geometry that does not fit
// in shared memory is refused and the previous one kept.
sptrsv_status set_geometry(sptrsv_plan p, int dirs, const int32_t *rows_per_warp, const int32_t *rhs_tile)
{
    const int32_t nmat = (int32_t)p->h_mats.size();
    for (int m = 0; m < nmat; ++m) {
        if (rows_per_warp && rows_per_warp[m] != 0 && !valid_rpw(rows_per_warp[m])) return SPTRSV_EINVAL;
        if (rhs_tile && rhs_tile[m] != 0 && !valid_tile(rhs_tile[m])) return SPTRSV_EINVAL;
    }
    for (int d = 0; d < 2; ++d) {
        if (!((dirs >> d) & 1)) continue;
        sptrsv_plan_st::Geom &G = p->geo[d];
        const std::vector<int32_t> old_rpw = G.rpw, old_tile = G.tile;
        for (int m = 0; m < nmat; ++m) {
            if (rows_per_warp && rows_per_warp[m]) G.rpw[m] = rows_per_warp[m];
            if (rhs_tile && rhs_tile[m]) G.tile[m] = rhs_tile[m];
        }
        sptrsv_status st = rebuild_items(p, d);
        if (st == SPTRSV_ENOTSUP) {
            G.rpw = old_rpw;
            G.tile = old_tile;
            if (rebuild_items(p, d) != SPTRSV_OK) return SPTRSV_ECUDA;
        }
        if (st != SPTRSV_OK) return st;
    }
    return SPTRSV_OK;
}
}  // namespace

extern "C" sptrsv_status sptrsv_batch_plan_create(sptrsv_handle h, int32_t nmat, const sptrsv_csr *Ls,
                                                  const sptrsv_csr *Ts, const int32_t *nrhs,
                                                  const sptrsv_plan_opts *opts, sptrsv_plan *plan)
{
    Range range("sptrsv_batch_plan_create");
    if (!h || !plan || nmat < 0 || (nmat > 0 && (!Ls || !nrhs))) return SPTRSV_EINVAL;
    *plan = nullptr;
    sptrsv_plan p = new (std::nothrow) sptrsv_plan_st;
    if (!p) return SPTRSV_ENOMEM;
    p->h = h;
    p->batched = true;
    p->dtype = nmat > 0 ? Ls[0].dtype : SPTRSV_F32;
    p->have_csc = false;
    bool want_csc = false;
    for (int m = 0; m < nmat && opts; ++m) want_csc = want_csc || opts[m].build_transpose;
    if (opts && opts[0].wait_limit_us > 0) p->spin = opts[0].wait_limit_us * 1000;
    cudaError_t e = p->alloc(&p->d_ctl, sizeof(PlanCtl));
    if (e == cudaSuccess) e = cudaMemset(p->d_ctl, 0, sizeof(PlanCtl));
    if (e != cudaSuccess) { sptrsv_plan_destroy(p); return from_cuda(e); }
    p->mats.resize((size_t)nmat);
    p->rhs_off.assign((size_t)nmat + 1, 0);
    p->vals_off.assign((size_t)nmat + 1, 0);
    p->row_off.assign((size_t)nmat + 1, 0);
    p->h_mats.resize((size_t)nmat);
    for (int d = 0; d < 2; ++d) {
        p->geo[d].rpw.assign((size_t)nmat, 32);
        p->geo[d].tile.assign((size_t)nmat, 4);
        p->geo[d].sched.assign((size_t)nmat, kSchedInOrder);
    }
    int64_t ktot = 0;
    for (int m = 0; m < nmat; ++m) {
        sptrsv_status st = check_csr(&Ls[m]);
        if (st == SPTRSV_OK && (Ls[m].dtype != p->dtype || nrhs[m] < 1)) st = SPTRSV_EINVAL;
        if (st == SPTRSV_OK && opts && opts[m].rows_per_warp != 0 && !valid_rpw(opts[m].rows_per_warp))
            st = SPTRSV_EINVAL;
        if (st == SPTRSV_OK && opts && opts[m].rhs_tile != 0 && !valid_tile(opts[m].rhs_tile))
            st = SPTRSV_EINVAL;
        if (st == SPTRSV_OK) st = prepare_mat(p, p->mats[m], Ls[m], Ts ? &Ts[m] : nullptr, want_csc);
        if (st != SPTRSV_OK) { sptrsv_plan_destroy(p); return st; }
        const PlanMat &M = p->mats[m];
        BatchMat &B = p->h_mats[m];
        B.n = M.L.n;
        B.k = nrhs[m];
        B.nnz = M.L.nnz;
        B.rp = M.L.row_ptr; B.ci = M.L.col_idx; B.v = M.L.vals;
        B.cp = M.d_cp; B.crow = M.d_crow; B.tmap = M.d_tmap; B.cv = M.d_cv;
        B.trp = M.hasT ? M.T.row_ptr : nullptr;
        B.tci = M.hasT ? M.T.col_idx : nullptr;
        B.tv = M.hasT ? M.T.vals : nullptr;
        B.tmask = M.hasT ? M.d_tmask : nullptr;
        B.tcp = M.d_tcp; B.trow = M.d_trow; B.ttmap = M.d_ttmap;
        B.rhs_off = p->rhs_off[m];
        B.vals_off = p->vals_off[m];
        B.row_off = p->row_off[m];
        p->rhs_off[m + 1] = p->rhs_off[m] + (int64_t)M.L.n * B.k;
        p->vals_off[m + 1] = p->vals_off[m] + M.L.nnz;
        p->row_off[m + 1] = p->row_off[m] + M.L.n;
        for (int d = 0; d < 2; ++d) {
            p->geo[d].rpw[m] = opts && opts[m].rows_per_warp ? opts[m].rows_per_warp : default_rpw(M.L.n, M.L.nnz);
            if (opts && opts[m].rhs_tile) p->geo[d].tile[m] = opts[m].rhs_tile;
        }
        ktot += B.k;
    }
    p->have_csc = want_csc;
    p->max_items = (int32_t)std::max<int64_t>(ktot, 1);  // tiles of one column at most
    e = p->alloc(&p->d_mats, sizeof(BatchMat) * (size_t)(nmat > 0 ? nmat : 1));
    for (int d = 0; d < 2; ++d) {
        if (e == cudaSuccess) e = p->alloc(&p->geo[d].d_items, sizeof(BatchItem) * (size_t)p->max_items);
        if (e == cudaSuccess) e = p->alloc(&p->geo[d].d_order, sizeof(int32_t) * (size_t)p->max_items);
    }
    if (e == cudaSuccess) e = p->alloc(&p->d_trace, sizeof(long long) * 3 * (size_t)p->max_items);
    if (e == cudaSuccess && nmat > 0)
        e = cudaMemcpy(p->d_mats, p->h_mats.data(), sizeof(BatchMat) * nmat, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { sptrsv_plan_destroy(p); return from_cuda(e); }
    {
        // chunk tables of the elementwise adjoint kernels: every 32-row chunk,
        // and the chunks whose T-column mask word is non-zero
        std::vector<RowChunk> g, t, f;
        std::vector<uint32_t> mask;
        e = cudaStreamSynchronize(p->h->stream);  // T-row masks are built on the handle's stream
        for (int m = 0; m < nmat && e == cudaSuccess; ++m) {
            const PlanMat &M = p->mats[m];
            const int32_t nw = (M.L.n + 31) / 32;
            for (int32_t c = 0; c < nw; ++c) g.push_back(RowChunk{m, 32 * c});
            if (!M.hasT || nw == 0) continue;
            for (int32_t c = 0; c < nw; ++c) f.push_back(RowChunk{m, 32 * c});
            mask.resize((size_t)nw);
            e = cudaMemcpy(mask.data(), M.d_tcmask, sizeof(uint32_t) * nw, cudaMemcpyDeviceToHost);
            for (int32_t c = 0; c < nw && e == cudaSuccess; ++c)
                if (mask[c]) t.push_back(RowChunk{m, 32 * c});
        }
        p->n_gchunks = (int64_t)g.size();
        p->n_tchunks = (int64_t)t.size();
        p->n_fchunks = (int64_t)f.size();
        if (e == cudaSuccess && want_csc) {
            std::vector<RowChunk> ct;
            for (int m = 0; m < nmat; ++m)
                for (int64_t q = 0; q < p->mats[m].L.nnz; q += kCscTile) ct.push_back(RowChunk{m, (int32_t)q});
            p->n_ctiles = (int64_t)ct.size();
            if (!ct.empty()) {
                e = p->alloc(&p->d_ctiles, sizeof(RowChunk) * ct.size());
                if (e == cudaSuccess)
                    e = cudaMemcpy(p->d_ctiles, ct.data(), sizeof(RowChunk) * ct.size(), cudaMemcpyHostToDevice);
            }
        }
        if (e == cudaSuccess && !f.empty()) {
            e = p->alloc(&p->d_fchunks, sizeof(RowChunk) * f.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(p->d_fchunks, f.data(), sizeof(RowChunk) * f.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = p->alloc(&p->d_bt, (p->dtype == SPTRSV_F64 ? 8 : 4) * (size_t)std::max<int64_t>(p->rhs_off[nmat], 1));
        }
        if (e == cudaSuccess) e = p->alloc(&p->d_gchunks, sizeof(RowChunk) * std::max<size_t>(g.size(), 1));
        if (e == cudaSuccess) e = p->alloc(&p->d_tchunks, sizeof(RowChunk) * std::max<size_t>(t.size(), 1));
        if (e == cudaSuccess && !g.empty())
            e = cudaMemcpy(p->d_gchunks, g.data(), sizeof(RowChunk) * g.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !t.empty())
            e = cudaMemcpy(p->d_tchunks, t.data(), sizeof(RowChunk) * t.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { sptrsv_plan_destroy(p); return from_cuda(e); }
    }
    sptrsv_status st = rebuild_items(p, 0);
    if (st == SPTRSV_OK) st = rebuild_items(p, 1);
    if (st != SPTRSV_OK) { sptrsv_plan_destroy(p); return st; }
    *plan = p;
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_batch_plan_set(sptrsv_plan p, const int32_t *rows_per_warp,
                                               const int32_t *rhs_tile)
{
    if (!p || !p->batched) return SPTRSV_EINVAL;
    return set_geometry(p, 3, rows_per_warp, rhs_tile);
}

extern "C" sptrsv_status sptrsv_batch_plan_set_direction(sptrsv_plan p, int32_t direction,
                                                         const int32_t *rows_per_warp, const int32_t *rhs_tile)
{
    if (!p || !p->batched || direction < 0 || direction > 2) return SPTRSV_EINVAL;
    return set_geometry(p, direction == 0 ? 3 : direction, rows_per_warp, rhs_tile);
}

extern "C" sptrsv_status sptrsv_batch_plan_set_schedule(sptrsv_plan p, int32_t direction, const int32_t *schedule)
{
    Range range("sptrsv_batch_plan_set_schedule");
    if (!p || !p->batched || !schedule || direction < 0 || direction > 2) return SPTRSV_EINVAL;
    return set_schedule(p, direction == 0 ? 3 : direction, schedule);
}

extern "C" sptrsv_status sptrsv_batch_offsets(sptrsv_plan p, int64_t *rhs_offset, int64_t *vals_offset)
{
    if (!p || !p->batched) return SPTRSV_EINVAL;
    if (rhs_offset) std::copy(p->rhs_off.begin(), p->rhs_off.end(), rhs_offset);
    if (vals_offset) std::copy(p->vals_off.begin(), p->vals_off.end(), vals_offset);
    return SPTRSV_OK;
}

namespace {
sptrsv_status batch_solve_impl(sptrsv_plan p, const void *b, void *x, bool trans)
{
    if (!p || !p->batched) return SPTRSV_EINVAL;
    const sptrsv_plan_st::Geom &G = p->geo[trans ? 1 : 0];
    if (G.nitems == 0) return SPTRSV_OK;
    if (!b || !x) return SPTRSV_EINVAL;
    if (trans && !p->have_csc) return SPTRSV_ENOTSUP;
    p->last_dir = trans ? 1 : 0;
    Waiter w{p->h->d_status, &p->d_ctl->abort_flag, p->spin};
    cudaError_t e = cudaSuccess;
    if (trans)
        e = p->dtype == SPTRSV_F64 ? batch_csc_values<double>(p->d_mats, p->d_ctiles, p->n_ctiles, p->h->stream)
                                   : batch_csc_values<float>(p->d_mats, p->d_ctiles, p->n_ctiles, p->h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    if (p->dtype == SPTRSV_F64)
        e = batch_solve<double>(p->d_mats, G.d_items, G.nitems, G.d_order, (const double *)b, (double *)x,
                                trans, p->d_ctl, w, G.grid, G.smem, p->d_trace, p->withhold,
                                p->d_fchunks, p->n_fchunks, (double *)p->d_bt, p->h->stream);
    else
        e = batch_solve<float>(p->d_mats, G.d_items, G.nitems, G.d_order, (const float *)b, (float *)x,
                               trans, p->d_ctl, w, G.grid, G.smem, p->d_trace, p->withhold,
                               p->d_fchunks, p->n_fchunks, (float *)p->d_bt, p->h->stream);
    return debug_sync(from_cuda(e), p->h->stream, "batch_solve");
}
}  // namespace

extern "C" sptrsv_status sptrsv_batch_solve(sptrsv_plan p, const void *b, void *x)
{
    Range range("sptrsv_batch_solve");
    return batch_solve_impl(p, b, x, false);
}

extern "C" sptrsv_status sptrsv_batch_solve_transpose(sptrsv_plan p, const void *gx, void *gb)
{
    Range range("sptrsv_batch_solve_transpose");
    return batch_solve_impl(p, gx, gb, true);
}

extern "C" sptrsv_status sptrsv_batch_trace(sptrsv_plan p, int64_t *trace)
{
    if (!p || !p->batched || !trace) return SPTRSV_EINVAL;
    const size_t nmat = p->mats.size();
    if (nmat == 0) return SPTRSV_OK;
    const sptrsv_plan_st::Geom &G = p->geo[p->last_dir];
    std::vector<long long> t(3 * (size_t)G.nitems);
    std::vector<BatchItem> items((size_t)G.nitems);
    cudaError_t e = cudaStreamSynchronize(p->h->stream);
    if (e == cudaSuccess && G.nitems > 0)
        e = cudaMemcpy(t.data(), p->d_trace, sizeof(long long) * t.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && G.nitems > 0)
        e = cudaMemcpy(items.data(), G.d_items, sizeof(BatchItem) * items.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    // per system: earliest start and latest end over its work items, and the
    // SM that started first
    for (size_t m = 0; m < nmat; ++m) {
        trace[3 * m] = INT64_MAX;
        trace[3 * m + 1] = 0;
        trace[3 * m + 2] = -1;
    }
    for (int32_t it = 0; it < G.nitems; ++it) {
        const int m = items[(size_t)it].mat;
        if (t[3 * (size_t)it] < trace[3 * m]) {
            trace[3 * m] = t[3 * (size_t)it];
            trace[3 * m + 2] = t[3 * (size_t)it + 2];
        }
        trace[3 * m + 1] = std::max<int64_t>(trace[3 * m + 1], t[3 * (size_t)it + 1]);
    }
    return SPTRSV_OK;
}

extern "C" sptrsv_status sptrsv_batch_grad_vals(sptrsv_plan p, const void *gb, const void *x, void *gvals)
{
    Range range("sptrsv_batch_grad_vals");
    if (!p || !p->batched) return SPTRSV_EINVAL;
    const int32_t nmat = (int32_t)p->mats.size();
    if (nmat == 0) return SPTRSV_OK;
    if (!gb || !x || !gvals) return SPTRSV_EINVAL;
    cudaError_t e;
    if (p->dtype == SPTRSV_F64)
        e = batch_grad_vals<double>(p->d_mats, p->d_gchunks, p->n_gchunks, (const double *)gb, (const double *)x,
                                    (double *)gvals, p->h->stream);
    else
        e = batch_grad_vals<float>(p->d_mats, p->d_gchunks, p->n_gchunks, (const float *)gb, (const float *)x,
                                   (float *)gvals, p->h->stream);
    return from_cuda(e);
}

extern "C" sptrsv_status sptrsv_batch_tt_apply(sptrsv_plan p, const void *gbp, void *gb)
{
    Range range("sptrsv_batch_tt_apply");
    if (!p || !p->batched) return SPTRSV_EINVAL;
    const int32_t nmat = (int32_t)p->mats.size();
    if (nmat == 0) return SPTRSV_OK;
    if (!gbp || !gb) return SPTRSV_EINVAL;
    cudaError_t e;
    if (p->dtype == SPTRSV_F64)
        e = batch_tt_apply<double>(p->d_mats, p->d_tchunks, p->n_tchunks, p->rhs_off[nmat], (const double *)gbp,
                                   (double *)gb, p->h->stream);
    else
        e = batch_tt_apply<float>(p->d_mats, p->d_tchunks, p->n_tchunks, p->rhs_off[nmat], (const float *)gbp,
                                  (float *)gb, p->h->stream);
    return from_cuda(e);
}

// ------------------------------------------------------ steps from host buffers
namespace {
sptrsv_status ensure_host_sets(sptrsv_plan p)
{
    if (p->s_h2d) return SPTRSV_OK;
    const int32_t nmat = (int32_t)p->mats.size();
    const size_t w = p->dtype == SPTRSV_F64 ? 8 : 4;
    const size_t rhs = w * (size_t)std::max<int64_t>(p->rhs_off[nmat], 1);
    const size_t nz = w * (size_t)std::max<int64_t>(p->vals_off[nmat], 1);
    cudaError_t e = cudaSuccess;
    for (auto &S : p->hset) {
        for (void **q : {&S.b, &S.w, &S.x, &S.gbp, &S.gb})
            if (e == cudaSuccess) e = p->alloc(q, rhs);
        if (e == cudaSuccess) e = p->alloc(&S.gv, nz);
        for (cudaEvent_t *ev : {&S.h2d, &S.comp, &S.d2h})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_d2h, cudaStreamNonBlocking);
    return from_cuda(e);
}
}  // namespace

extern "C" sptrsv_status sptrsv_batch_step_host(sptrsv_plan p, const void *b, const void *w, void *x, void *gb,
                                                void *gvals)
{
    Range range("sptrsv_batch_step_host");
    if (!p || !p->batched || !b || !w || !x || !gb || !gvals) return SPTRSV_EINVAL;
    if (!p->have_csc) return SPTRSV_ENOTSUP;
    const int32_t nmat = (int32_t)p->mats.size();
    if (nmat == 0 || p->rhs_off[nmat] == 0) return SPTRSV_OK;
    sptrsv_status st = ensure_host_sets(p);
    if (st != SPTRSV_OK) return st;
    const size_t wb = p->dtype == SPTRSV_F64 ? 8 : 4;
    const size_t rhs = wb * (size_t)p->rhs_off[nmat];
    const size_t nz = wb * (size_t)p->vals_off[nmat];
    sptrsv_plan_st::HostSet &S = p->hset[p->nsteps & 1];
    cudaStream_t hs = p->h->stream;
    // copies in, once the previous step on this set no longer reads b and w
    cudaError_t e = S.used ? cudaStreamWaitEvent(p->s_h2d, S.comp, 0) : cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.b, b, rhs, cudaMemcpyHostToDevice, p->s_h2d);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.w, w, rhs, cudaMemcpyHostToDevice, p->s_h2d);
    if (e == cudaSuccess) e = cudaEventRecord(S.h2d, p->s_h2d);
    // the step, once its inputs are in and the previous results of the set are out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hs, S.h2d, 0);
    if (e == cudaSuccess && S.used) e = cudaStreamWaitEvent(hs, S.d2h, 0);
    if (e != cudaSuccess) return from_cuda(e);
    st = sptrsv_batch_solve(p, S.b, S.x);
    if (st == SPTRSV_OK) st = sptrsv_batch_solve_transpose(p, S.w, S.gbp);
    if (st == SPTRSV_OK) st = sptrsv_batch_tt_apply(p, S.gbp, S.gb);
    if (st == SPTRSV_OK) st = sptrsv_batch_grad_vals(p, S.gbp, S.x, S.gv);
    if (st != SPTRSV_OK) return st;
    e = cudaEventRecord(S.comp, hs);
    // copies out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_d2h, S.comp, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, S.x, rhs, cudaMemcpyDeviceToHost, p->s_d2h);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gb, S.gb, rhs, cudaMemcpyDeviceToHost, p->s_d2h);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gvals, S.gv, nz, cudaMemcpyDeviceToHost, p->s_d2h);
    if (e == cudaSuccess) e = cudaEventRecord(S.d2h, p->s_d2h);
    S.used = true;
    ++p->nsteps;
    return from_cuda(e);
}

extern "C" sptrsv_status sptrsv_batch_step_wait(sptrsv_plan p)
{
    Range range("sptrsv_batch_step_wait");
    if (!p || !p->batched) return SPTRSV_EINVAL;
    cudaError_t e = cudaStreamSynchronize(p->h->stream);
    if (e == cudaSuccess && p->s_h2d) e = cudaStreamSynchronize(p->s_h2d);
    if (e == cudaSuccess && p->s_d2h) e = cudaStreamSynchronize(p->s_d2h);
    if (e != cudaSuccess) return from_cuda(e);
    int status = 0;
    e = cudaMemcpy(&status, p->h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    return (sptrsv_status)status;
}

// ------------------------------------------------------------ bounds checks
namespace {
__global__ void k_debug_check_index(int32_t index, int32_t n, int *status, int *out)
{
    const int v = chk_index(index, 0, n, status);
    if (v >= 0 && v < n) out[0] = v;  // the access a checked index feeds
}
}  // namespace

extern "C" int32_t sptrsv_checked_build(void)
{
#ifdef SPTRSV_CHECKED
    return 1;
#else
    return 0;
#endif
}

extern "C" sptrsv_status sptrsv_debug_check_index(sptrsv_handle h, int32_t index, int32_t n)
{
    if (!h || n < 1 || n > 32) return SPTRSV_EINVAL;
    k_debug_check_index<<<1, 1, 0, h->stream>>>(index, n, h->d_status, reinterpret_cast<int *>(h->d_scratch));
    return from_cuda(cudaGetLastError());
}
