// Batched solve: many independent lower-triangular systems of uneven size,
// each with its own number of right-hand sides, in ONE persistent launch.
// Thread blocks take work items -- one system and a tile of at most 8 of its
// right-hand-side columns -- from a ticket (longest estimated chain first)
// and run the block algorithm on them; no host work per system, so a batch
// solve is two kernel nodes in a CUDA graph.  The adjoint's elementwise
// parts (value gradient, T^T) walk plan-time tables of 32-row chunks.
#include "block.cuh"

namespace spt {

namespace {

constexpr int kBatchThreads = 32 * kBatchWarps;

template <class T>
__device__ __forceinline__ Sys<T> sys_of(const BatchMat &M)
{
    Sys<T> A;
    A.n = M.n;
    A.rp = M.rp; A.ci = M.ci; A.v = (const T *)M.v;
    A.cp = M.cp; A.crow = M.crow; A.tmap = M.tmap; A.cv = (const T *)M.cv;
    A.trp = M.trp; A.tci = M.tci; A.tv = (const T *)M.tv; A.tmask = M.tmask;
    A.tcp = M.tcp; A.trow = M.trow; A.ttmap = M.ttmap;
    A.nnz = M.nnz;
    A.chk = nullptr;
    return A;
}

template <class T, int KT, bool TR>
__device__ __forceinline__ bool run_one(const BatchMat &M, const BatchItem &I, unsigned char *raw,
                                        const T *b, const T *bt, T *x, const Waiter &w, int withhold)
{
    const int ring = I.kc * I.rpw;
    BlockSmem<T, KT> sm = carve_block_smem<T, KT>(raw, ring, I.kc, I.nw);
    reset_block_smem<T, KT>(sm, ring, I.kc);
    __syncthreads();
    Sys<T> A = sys_of<T>(M);
    A.chk = w.status;
    // a rewritten system's forward right-hand side b + T b was formed by the
    // fold launch before this one (bt); the solve itself reads no T
    const bool folded = !TR && bt != nullptr && M.tmask != nullptr;
    if (folded) A.tmask = nullptr;
    Rhs<T> R;
    R.b = (folded ? bt : b) + M.rhs_off + I.r0;
    R.x = x + M.rhs_off + I.r0;
    R.ld = M.k;
    R.k = I.kt;
    // test hook: a withheld row (counted over all systems) is never published
    const int64_t wh = (int64_t)withhold - M.row_off;
    const int local = (withhold >= 0 && wh >= 0 && wh < M.n) ? (int)wh : -1;
    const bool ok = I.sched == kSchedLevel
                        ? block_solve_levels<T, KT, TR>(A, R, M.perm, M.iperm, M.lgroups[TR ? 1 : 0],
                                                        M.nlgroups[TR ? 1 : 0], I.kc, I.nw, sm, w, local)
                        : block_solve_any<T, KT, TR, false>(A, R, I.rpw, I.kc, I.P, I.nw, sm, w, local);
    __syncthreads();
    release_block_smem<T, KT>(sm, I.kc);
    return ok;
}

__device__ __forceinline__ unsigned sm_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

template <class T, bool TR>
__global__ void __launch_bounds__(kBatchThreads, kBatchMinBlocks)
k_batch(const BatchMat *__restrict__ mats, const BatchItem *__restrict__ items, int32_t nitems,
        const int32_t *__restrict__ order, const T *b, const T *bt, T *x, PlanCtl *ctl, Waiter w,
        long long *trace, int withhold)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_next, s_stop;
    for (;;) {
        if (threadIdx.x == 0) {
            s_next = (int)atomicAdd(&ctl->ticket, 1ull);
            s_stop = ld_relaxed(w.abort_flag);
        }
        __syncthreads();
        const int t = s_next;
        const int stop = s_stop;
        __syncthreads();
        if (t >= nitems || stop) return;
        const int it = order[t];
        const BatchItem I = items[it];
        const BatchMat M = mats[I.mat];
        if (trace && threadIdx.x == 0) {
            trace[3 * it] = (long long)now_ns();
            trace[3 * it + 2] = (long long)sm_id();
        }
        switch (I.KT) {
        case 1: run_one<T, 1, TR>(M, I, smraw, b, bt, x, w, withhold); break;
        case 2: run_one<T, 2, TR>(M, I, smraw, b, bt, x, w, withhold); break;
        case 4: run_one<T, 4, TR>(M, I, smraw, b, bt, x, w, withhold); break;
        default: run_one<T, 8, TR>(M, I, smraw, b, bt, x, w, withhold); break;
        }
        __syncthreads();
        if (trace && threadIdx.x == 0) trace[3 * it + 1] = (long long)now_ns();
    }
}

// Row of nonzero p inside a 32-row chunk whose lanes hold the chunk's row
// starts (s = row_ptr[r0 + lane], lanes >= nrows unused): the last lane l <
// nrows with s_l <= p, by a five-step binary search over the lanes.
__device__ __forceinline__ int row_in_chunk(int s, int nrows, int p)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int cand = lo + step;
        const int v = __shfl_sync(SPT_FULL_MASK, s, cand & 31);
        if (cand < nrows && v <= p) lo = cand;
    }
    return lo;
}

// dL/dL_ij = -g_b[i,:] . x[j,:] on L's pattern.  One warp per 32-row chunk;
// the chunk's nonzeros are contiguous in CSR order and are taken 32 at a
// time, one per lane (coalesced column indices and gradient stores).
// (Groups of up to 8 lanes per nonzero, reading g_b[i,:] and x[j,:] in
// contiguous pieces, measured slower on the batched workload; so did groups
// of up to 32 lanes walking the chunk's rows: 8.4 ms instead of 3.0 ms for
// T^T and the gradient, the extra instructions outweighing the coalescing.)
template <class T>
__global__ void k_batch_grad(const BatchMat *__restrict__ mats, const RowChunk *__restrict__ chunks,
                             int64_t nchunks, const T *__restrict__ gb, const T *__restrict__ x,
                             T *__restrict__ gv)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = gw; c < nchunks; c += nw) {
        const RowChunk ch = chunks[c];
        const BatchMat &M = mats[ch.mat];
        const int nrows = min(32, M.n - ch.r0);
        const int k = M.k;
        const int s = ldro(M.rp + ch.r0 + min(lane, nrows));
        const int pe = __shfl_sync(SPT_FULL_MASK, s, nrows & 31);
        const int end = nrows == 32 ? ldro(M.rp + ch.r0 + 32) : pe;
        const int p0 = __shfl_sync(SPT_FULL_MASK, s, 0);
        const T *xb = x + M.rhs_off;
        const T *gbb = gb + M.rhs_off;
        T *out = gv + M.vals_off;
        for (int base = p0; base < end; base += 32) {
            const int p = base + lane;
            const int r = row_in_chunk(s, nrows, p);
            if (p < end) {
                const T *gi = gbb + (int64_t)(ch.r0 + r) * k;
                const T *xj = xb + (int64_t)ldro(M.ci + p) * k;
                T acc = T(0);
                for (int q = 0; q < k; ++q) acc += gi[q] * xj[q];
                out[p] = -acc;
            }
        }
    }
}

// g_b = g_b' + T^T g_b' on the rows of the rewritten systems that are
// columns of T: one warp per 32-row chunk holding at least one such column,
// one lane per row; each lane gathers its column of T (CSC, rows ascending)
// and writes its row of g_b once -- no atomics, so the result does not
// depend on the schedule.  The other rows of g_b are the copy of g_b'.
template <class T>
__global__ void k_batch_tt(const BatchMat *__restrict__ mats, const RowChunk *__restrict__ chunks,
                           int64_t nchunks, const T *__restrict__ gbp, T *gb)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = gw; c < nchunks; c += nw) {
        const RowChunk ch = chunks[c];
        const BatchMat &M = mats[ch.mat];
        const int j = ch.r0 + lane;
        if (j >= M.n) continue;
        const int qa = ldro(M.tcp + j), qe = ldro(M.tcp + j + 1);
        if (qa == qe) continue;
        const int k = M.k;
        const T *tv = (const T *)M.tv;
        const T *g0 = gbp + M.rhs_off;
        for (int r = 0; r < k; ++r) {
            T acc = g0[(int64_t)j * k + r];
            for (int q = qa; q < qe; ++q)
                acc += ldro(tv + ldro(M.ttmap + q)) * g0[(int64_t)ldro(M.trow + q) * k + r];
            gb[M.rhs_off + (int64_t)j * k + r] = acc;
        }
    }
}

// bt = b + T b for every row of the rewritten systems (the right-hand side
// of L' x = b + T b, Section 2.2), one warp per 32-row chunk of those
// systems.  The chunk's rows are contiguous in the packed layout, so the
// warp copies its 32 k elements in order (coalesced) and adds the T terms
// of the few rows that have a T row.  Formed once per forward batched solve
// so that the solve kernel reads one right-hand side per row.
template <class T>
__global__ void k_batch_tfold(const BatchMat *__restrict__ mats, const RowChunk *__restrict__ chunks,
                              int64_t nchunks, const T *__restrict__ b, T *__restrict__ bt)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = gw; c < nchunks; c += nw) {
        const RowChunk ch = chunks[c];
        const BatchMat &M = mats[ch.mat];
        const int k = M.k;
        const int nrows = min(32, M.n - ch.r0);
        const unsigned word = ldro(M.tmask + (ch.r0 >> 5));
        const T *bb = b + M.rhs_off;
        const T *tv = (const T *)M.tv;
        const int64_t e0 = (int64_t)ch.r0 * k;
        const int64_t e1 = e0 + (int64_t)nrows * k;
        for (int64_t t = e0 + lane; t < e1; t += 32) {
            T v = bb[t];
            const int i = (int)(t / k);
            if ((word >> (i & 31)) & 1u) {
                const int r = (int)(t - (int64_t)i * k);
                for (int p = ldro(M.trp + i); p < ldro(M.trp + i + 1); ++p)
                    v += ldro(tv + p) * bb[(int64_t)ldro(M.tci + p) * k + r];
            }
            bt[M.rhs_off + t] = v;
        }
    }
}

// cv = v[tmap] for every system, by tiles of kCscTile consecutive CSC
// entries of one system taken in order (tile t by block t, t + grid, ...):
// the blocks in flight work on a window of neighbouring tiles, whose source
// values stay in L2 while they are gathered.
template <class T>
__global__ void k_batch_csc_values(const BatchMat *__restrict__ mats, const RowChunk *__restrict__ tiles,
                                   int64_t ntiles)
{
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const RowChunk tl = tiles[t];
        const BatchMat &M = mats[tl.mat];
        const T *v = (const T *)M.v;
        T *cv = (T *)M.cv;
        const int64_t q1 = min((int64_t)tl.r0 + kCscTile, M.nnz);
        for (int64_t q = (int64_t)tl.r0 + threadIdx.x; q < q1; q += blockDim.x)
            cv[q] = ldro(v + ldro(M.tmap + q));
    }
}

int elementwise_grid(int64_t nchunks)
{
    // 8 warps per block; grid-stride over the chunks
    int64_t blocks = (nchunks + 7) / 8;
    return (int)std::min<int64_t>(std::max<int64_t>(blocks, 1), 152 * 16);
}

}  // namespace

namespace {
__global__ void k_inverse_perm(const int32_t *__restrict__ perm, int32_t *__restrict__ iperm, int32_t n)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        iperm[perm[q]] = (int32_t)q;
}
}  // namespace

cudaError_t inverse_perm(const int32_t *perm, int32_t *iperm, int32_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_inverse_perm<<<(int)std::min<int64_t>(((int64_t)n + 255) / 256, 152 * 16), 256, 0, s>>>(perm, iperm, n);
    return cudaGetLastError();
}

int batch_grid(size_t smem, const DeviceInfo &di)
{
    // raise the dynamic shared-memory limit of every variant at plan time,
    // so that a solve issues nothing but launches (capturable in a graph)
    const int lim = (int)kBlockSmemBudget;
    cudaFuncSetAttribute(k_batch<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_batch<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_batch<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_batch<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<float, false>, kBatchThreads, smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * di.num_sms;
}

template <class T>
cudaError_t batch_solve(const BatchMat *mats, const BatchItem *items, int32_t nitems,
                        const int32_t *order, const T *b, T *x, bool trans, PlanCtl *ctl,
                        const Waiter &w, int grid, size_t smem, long long *trace, int withhold,
                        const RowChunk *fchunks, int64_t nfchunks, T *bt, cudaStream_t s)
{
    cudaError_t e = launch_prologue<T>(ctl, s);
    if (e != cudaSuccess || nitems <= 0) return e;
    const bool fold = !trans && bt != nullptr && nfchunks > 0;
    if (fold) {
        k_batch_tfold<T><<<elementwise_grid(nfchunks), 256, 0, s>>>(mats, fchunks, nfchunks, b, bt);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (trans)
        k_batch<T, true><<<grid, kBatchThreads, smem, s>>>(mats, items, nitems, order, b, nullptr, x, ctl, w,
                                                            trace, withhold);
    else
        k_batch<T, false><<<grid, kBatchThreads, smem, s>>>(mats, items, nitems, order, b, fold ? bt : nullptr,
                                                             x, ctl, w, trace, withhold);
    return cudaGetLastError();
}

template <class T>
cudaError_t batch_grad_vals(const BatchMat *mats, const RowChunk *chunks, int64_t nchunks, const T *gb,
                            const T *x, T *gv, cudaStream_t s)
{
    if (nchunks <= 0) return cudaSuccess;
    k_batch_grad<T><<<elementwise_grid(nchunks), 256, 0, s>>>(mats, chunks, nchunks, gb, x, gv);
    return cudaGetLastError();
}

template <class T>
cudaError_t batch_tt_apply(const BatchMat *mats, const RowChunk *tchunks, int64_t ntchunks,
                           int64_t total_rhs, const T *gbp, T *gb, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(gb, gbp, sizeof(T) * (size_t)total_rhs, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess || ntchunks <= 0) return e;
    k_batch_tt<T><<<elementwise_grid(ntchunks), 256, 0, s>>>(mats, tchunks, ntchunks, gbp, gb);
    return cudaGetLastError();
}

template <class T>
cudaError_t batch_csc_values(const BatchMat *mats, const RowChunk *tiles, int64_t ntiles, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>(ntiles, 152 * 8);
    k_batch_csc_values<T><<<grid, 256, 0, s>>>(mats, tiles, ntiles);
    return cudaGetLastError();
}

#define SPT_INST(T)                                                                              \
    template cudaError_t batch_solve<T>(const BatchMat *, const BatchItem *, int32_t,             \
                                        const int32_t *, const T *, T *, bool, PlanCtl *,        \
                                        const Waiter &, int, size_t, long long *, int,           \
                                        const RowChunk *, int64_t, T *, cudaStream_t);           \
    template cudaError_t batch_grad_vals<T>(const BatchMat *, const RowChunk *, int64_t,         \
                                            const T *, const T *, T *, cudaStream_t);            \
    template cudaError_t batch_tt_apply<T>(const BatchMat *, const RowChunk *, int64_t, int64_t, \
                                           const T *, T *, cudaStream_t);                        \
    template cudaError_t batch_csc_values<T>(const BatchMat *, const RowChunk *, int64_t, cudaStream_t);
SPT_INST(double)
SPT_INST(float)
#undef SPT_INST

}  // namespace spt
