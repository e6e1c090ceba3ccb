// Batched solve: many independent lower-triangular systems of uneven size,
// each with its own number of right-hand sides, in ONE persistent launch.
// Thread blocks take whole systems from a ticket (largest estimated critical
// path first) and run the block algorithm on them; no host work per system,
// so a batch solve is two kernel nodes in a CUDA graph.
#include "block.cuh"

namespace spt {

namespace {

constexpr int kBatchThreads = 32 * kMaxBlockWarps;

template <class T>
__device__ __forceinline__ Sys<T> sys_of(const BatchMat &M)
{
    Sys<T> A;
    A.n = M.n;
    A.rp = M.rp; A.ci = M.ci; A.v = (const T *)M.v;
    A.cp = M.cp; A.crow = M.crow; A.tmap = M.tmap;
    A.trp = M.trp; A.tci = M.tci; A.tv = (const T *)M.tv; A.tmask = M.tmask;
    return A;
}

template <class T, int KT, bool TR>
__device__ __forceinline__ bool run_one(const BatchMat &M, const BatchItem &I, unsigned char *raw,
                                        const T *b, T *x, const Waiter &w)
{
    const int ring = I.kc * I.rpw;
    BlockSmem<T, KT> sm = carve_block_smem<T, KT>(raw, ring, I.kc, I.nw);
    reset_block_smem<T, KT>(sm, ring, I.kc);
    __syncthreads();
    Rhs<T> R;
    R.b = b + M.rhs_off + I.r0;
    R.x = x + M.rhs_off + I.r0;
    R.ld = M.k;
    R.k = I.kt;
    return block_solve_any<T, KT, TR>(sys_of<T>(M), R, I.rpw, I.kc, I.P, I.nw, sm, w, -1);
}

__device__ __forceinline__ unsigned sm_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

template <class T, bool TR>
__global__ void __launch_bounds__(kBatchThreads)
k_batch(const BatchMat *__restrict__ mats, const BatchItem *__restrict__ items, int32_t nitems,
        const int32_t *__restrict__ order, const T *b, T *x, PlanCtl *ctl, Waiter w,
        long long *trace)
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
        case 1: run_one<T, 1, TR>(M, I, smraw, b, x, w); break;
        case 2: run_one<T, 2, TR>(M, I, smraw, b, x, w); break;
        case 4: run_one<T, 4, TR>(M, I, smraw, b, x, w); break;
        default: run_one<T, 8, TR>(M, I, smraw, b, x, w); break;
        }
        __syncthreads();
        if (trace && threadIdx.x == 0) trace[3 * it + 1] = (long long)now_ns();
    }
}

// Global row r -> matrix index (row_off is the nmat+1 prefix of n).
__device__ __forceinline__ int mat_of_row(const int64_t *row_off, int nmat, int64_t r)
{
    int lo = 0, hi = nmat - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class T>
__global__ void k_batch_grad(const BatchMat *__restrict__ mats, int32_t nmat,
                             const int64_t *__restrict__ row_off, int64_t total_rows,
                             const T *__restrict__ gb, const T *__restrict__ x, T *__restrict__ gv)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 3, sl = lane & 7;  // 4 rows per warp, 8 lanes per row
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r4 = gw * 4; r4 < total_rows; r4 += nw * 4) {
        const int64_t r = r4 + g;
        if (r >= total_rows) continue;
        const int m = mat_of_row(row_off, nmat, r);
        const BatchMat &M = mats[m];
        const int i = (int)(r - row_off[m]);
        const int k = M.k;
        const int a = ldro(M.rp + i), e = ldro(M.rp + i + 1);
        const T *gi = gb + M.rhs_off + (int64_t)i * k;
        const T *xb = x + M.rhs_off;
        T *out = gv + M.vals_off;
        for (int p = a + sl; p < e; p += 8) {
            const T *xj = xb + (int64_t)ldro(M.ci + p) * k;
            T s = T(0);
            for (int q = 0; q < k; ++q) s += gi[q] * xj[q];
            out[p] = -s;
        }
    }
}

template <class T>
__global__ void k_batch_tt(const BatchMat *__restrict__ mats, int32_t nmat,
                           const int64_t *__restrict__ row_off, int64_t total_rows,
                           const T *__restrict__ gbp, T *gb)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = gw; r < total_rows; r += nw) {
        const int m = mat_of_row(row_off, nmat, r);
        const BatchMat &M = mats[m];
        if (M.tmask == nullptr) continue;
        const int i = (int)(r - row_off[m]);
        if (!((M.tmask[i >> 5] >> (i & 31)) & 1u)) continue;
        const int k = M.k;
        const T *tv = (const T *)M.tv;
        for (int p = M.trp[i] + lane; p < M.trp[i + 1]; p += 32) {
            const T c = tv[p];
            const int64_t j = M.tci[p];
            for (int q = 0; q < k; ++q)
                atomicAdd(gb + M.rhs_off + j * k + q, c * gbp[M.rhs_off + (int64_t)i * k + q]);
        }
    }
}

}  // namespace

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
                        const Waiter &w, int grid, size_t smem, long long *trace,
                        cudaStream_t s)
{
    cudaError_t e = launch_prologue<T>(ctl, s);
    if (e != cudaSuccess || nitems <= 0) return e;
    if (trans)
        k_batch<T, true><<<grid, kBatchThreads, smem, s>>>(mats, items, nitems, order, b, x, ctl, w, trace);
    else
        k_batch<T, false><<<grid, kBatchThreads, smem, s>>>(mats, items, nitems, order, b, x, ctl, w, trace);
    return cudaGetLastError();
}

template <class T>
cudaError_t batch_grad_vals(const BatchMat *mats, int32_t nmat, const int64_t *row_off,
                            int64_t total_rows, const T *gb, const T *x, T *gv, cudaStream_t s)
{
    if (total_rows <= 0) return cudaSuccess;
    int64_t blocks = (total_rows + 31) / 32;
    if (blocks > 65535 * 4) blocks = 65535 * 4;
    k_batch_grad<T><<<(int)blocks, 256, 0, s>>>(mats, nmat, row_off, total_rows, gb, x, gv);
    return cudaGetLastError();
}

template <class T>
cudaError_t batch_tt_apply(const BatchMat *mats, int32_t nmat, const int64_t *row_off,
                           int64_t total_rows, int64_t total_rhs, const T *gbp, T *gb,
                           cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(gb, gbp, sizeof(T) * (size_t)total_rhs, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess || total_rows <= 0) return e;
    int64_t blocks = (total_rows + 7) / 8;
    if (blocks > 65535 * 4) blocks = 65535 * 4;
    k_batch_tt<T><<<(int)blocks, 256, 0, s>>>(mats, nmat, row_off, total_rows, gbp, gb);
    return cudaGetLastError();
}

#define SPT_INST(T)                                                                              \
    template cudaError_t batch_solve<T>(const BatchMat *, const BatchItem *, int32_t,             \
                                        const int32_t *, const T *, T *, bool, PlanCtl *,        \
                                        const Waiter &, int, size_t, long long *, cudaStream_t); \
    template cudaError_t batch_grad_vals<T>(const BatchMat *, int32_t, const int64_t *, int64_t, \
                                            const T *, const T *, T *, cudaStream_t);            \
    template cudaError_t batch_tt_apply<T>(const BatchMat *, int32_t, const int64_t *, int64_t,  \
                                           int64_t, const T *, T *, cudaStream_t);
SPT_INST(double)
SPT_INST(float)
#undef SPT_INST

}  // namespace spt
