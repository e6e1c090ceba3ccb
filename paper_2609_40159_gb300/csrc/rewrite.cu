// Equation rewriting on the GPU (paper Section 2.2; rewriting list of
// Section 4.3).  For a listed row i with target level t, every predecessor j
// with lev(j) >= t is substituted, largest column first, by row j's own
// predecessors scaled by m = acc[j] / L_jj (original rows, original levels);
// the right-hand side picks up T[i][j] = -m.  The result is L' x = b + T b.
//
// One warp per rewritten row:
//   cone   -- the set U of every column the substitution touches, found
//             breadth-first: U starts as row i's predecessors and every
//             member with lev >= t adds its own predecessors (warp-parallel
//             inserts into an open-addressing hash set).  Members with
//             lev >= t are exactly the substituted columns (T row), the others
//             the surviving pattern of L' row i.
//   sort   -- U ascending (bitonic, warp-wide).
//   values -- accumulators for U in FP64; substituted columns are processed
//             from the largest down, each update a separate IEEE multiply and
//             subtract (__dmul_rn / __dsub_rn) and m an IEEE division, in the
//             order the textbook substitution applies them.
// The symbolic pass only counts |U| and the substituted columns, so the host
// can size L' and T; the numeric pass repeats the cone and fills them.
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace spt {

namespace {

constexpr int kRwThreads = 256;
constexpr int kNone = 0x7F7F7F7F;  // "row not listed" (memset byte 0x7F)

__global__ void k_rw_mark(const int32_t *rows, const int32_t *targets, int32_t nrows,
                          const int32_t *lev, int32_t n, int32_t *tgt, long long *bad)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nrows;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = rows[q];
        if (i < 0 || i >= n) { atomicMin(bad, q * 16 + SPTRSV_EINVAL); continue; }
        const int li = lev[i];
        const int t = targets ? targets[q] : li - 1;
        if (li == 0 || t < 0 || t >= li) { atomicMin(bad, q * 16 + SPTRSV_ETARGET); continue; }
        atomicMin(tgt + i, t);
    }
}

__global__ void k_rw_flags(const int32_t *tgt, int32_t n, int32_t *flag)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = tgt[i] != kNone ? 1 : 0;
}

__global__ void k_rw_compact(const int32_t *flag, const int32_t *pos, int32_t n, int32_t *list)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) list[pos[i]] = (int32_t)i;
}

// Per-warp workspace: hash keys (2*cap), U (cap), accumulators (cap doubles).
struct Ws {
    int *keys;
    int *U;
    double *acc;
    int cap;
};

__device__ __forceinline__ Ws warp_ws(char *base, int cap, int64_t wid)
{
    const size_t bytes = (size_t)cap * (2 * 4 + 4 + 8);
    char *p = base + bytes * wid;
    Ws w;
    w.acc = reinterpret_cast<double *>(p);
    w.keys = reinterpret_cast<int *>(p + (size_t)cap * 8);
    w.U = w.keys + 2 * cap;
    w.cap = cap;
    return w;
}

// Integer mixer for the open-addressing set: xor-shift / multiply rounds
// with the published "lowbias32" constants of C. Wellons' hash-prospector
// search (a well-mixed 32-bit bijection, so distinct keys never collide
// before the table mask).
__device__ __forceinline__ unsigned hash32(unsigned k)
{
    k ^= k >> 16;
    k *= 0x7feb352du;
    k ^= k >> 15;
    k *= 0x846ca68bu;
    k ^= k >> 16;
    return k;
}

// Inserts `key` (when want) into the warp's set; returns through *count the
// new size.  Appends new keys to U.  Sets *overflow when U would exceed cap.
__device__ __forceinline__ void warp_insert(const Ws &w, bool want, int key, int *count,
                                            bool *overflow)
{
    bool fresh = false;
    if (want) {
        const unsigned mask = 2u * w.cap - 1u;
        unsigned h = hash32((unsigned)key) & mask;
        for (int probe = 0; probe < 2 * w.cap; ++probe) {
            const int prev = atomicCAS(w.keys + h, -1, key);
            if (prev == -1) { fresh = true; break; }
            if (prev == key) break;
            h = (h + 1) & mask;
        }
    }
    const unsigned b = __ballot_sync(SPT_FULL_MASK, fresh);
    const int base = *count;
    if (fresh) {
        const int pos = base + __popc(b & lanemask_lt());
        if (pos < w.cap) w.U[pos] = key;
    }
    *count = base + __popc(b);
    if (*count > w.cap) *overflow = true;
}

// Builds U for row i with target t.  Returns |U| (or cap+1 on overflow) and
// the number of members with lev >= t in *nelim.
__device__ int build_cone(const Ws &w, const int32_t *rp, const int32_t *ci, const int32_t *lev,
                          int i, int t, int *nelim)
{
    const int lane = threadIdx.x & 31;
    for (int h = lane; h < 2 * w.cap; h += 32) w.keys[h] = -1;
    __syncwarp();
    int count = 0;
    bool overflow = false;
    const int a = rp[i], e = rp[i + 1] - 1;
    for (int p0 = a; p0 < e; p0 += 32) {
        const int p = p0 + lane;
        warp_insert(w, p < e, p < e ? ci[p] : 0, &count, &overflow);
        if (overflow) break;
    }
    __syncwarp();
    int ne = 0;
    for (int idx = 0; idx < count && !overflow; ++idx) {
        const int u = w.U[idx];
        if (lev[u] < t) continue;
        ++ne;
        const int ua = rp[u], ue = rp[u + 1] - 1;
        for (int p0 = ua; p0 < ue; p0 += 32) {
            const int p = p0 + lane;
            warp_insert(w, p < ue, p < ue ? ci[p] : 0, &count, &overflow);
            if (overflow) break;
        }
        __syncwarp();
    }
    *nelim = ne;
    return overflow ? w.cap + 1 : count;
}

// Ascending bitonic sort of U[0..cnt) in place (padding with INT_MAX up to a
// power of two; cnt <= cap, and cap is a power of two).
__device__ void warp_sort(const Ws &w, int cnt)
{
    const int lane = threadIdx.x & 31;
    int N = 1;
    while (N < cnt) N <<= 1;
    for (int t = cnt + lane; t < N; t += 32) w.U[t] = INT_MAX;
    __syncwarp();
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < N; t += 32) {
                const int partner = t ^ j;
                if (partner > t) {
                    const int x = w.U[t], y = w.U[partner];
                    const bool up = (t & k) == 0;
                    if ((x > y) == up) { w.U[t] = y; w.U[partner] = x; }
                }
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ int find_pos(const int *U, int cnt, int key)
{
    int lo = 0, hi = cnt - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (U[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kRwThreads)
k_rw_symbolic(const int32_t *rp, const int32_t *ci, const int32_t *lev, const int32_t *tgt,
              const int32_t *list, int32_t nrw, char *ws_base, int cap, int32_t *len_lp,
              int32_t *len_t, int *need)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const Ws w = warp_ws(ws_base, cap, gw);
    for (int64_t q = gw; q < nrw; q += nw) {
        const int i = list[q];
        int ne = 0;
        const int cnt = build_cone(w, rp, ci, lev, i, tgt[i], &ne);
        if (lane == 0) {
            if (cnt > cap) atomicMax(need, cnt);
            else {
                len_lp[i] = cnt - ne + 1;
                len_t[i] = ne;
            }
        }
        __syncwarp();
    }
}

__global__ void k_rw_lengths(const int32_t *rp, const int32_t *tgt, int32_t n, int32_t *len_lp,
                             int32_t *len_t)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (tgt[i] == kNone) {
            len_lp[i] = rp[i + 1] - rp[i];
            len_t[i] = 0;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(kRwThreads)
k_rw_numeric(const int32_t *rp, const int32_t *ci, const T *v, const int32_t *lev,
             const int32_t *tgt, const int32_t *list, int32_t nrw, char *ws_base, int cap,
             const int32_t *lp_rp, int32_t *lp_ci, T *lp_v, const int32_t *t_rp, int32_t *t_ci,
             T *t_v)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const Ws w = warp_ws(ws_base, cap, gw);
    for (int64_t q = gw; q < nrw; q += nw) {
        const int i = list[q];
        const int t = tgt[i];
        int ne = 0;
        const int cnt = build_cone(w, rp, ci, lev, i, t, &ne);
        __syncwarp();
        warp_sort(w, cnt);
        // accumulators: row i's own values, zero elsewhere
        for (int s = lane; s < cnt; s += 32) w.acc[s] = 0.0;
        __syncwarp();
        const int a = rp[i], e = rp[i + 1] - 1;
        for (int p = a + lane; p < e; p += 32) w.acc[find_pos(w.U, cnt, ci[p])] = (double)v[p];
        __syncwarp();
        // substitutions, largest column first
        for (int s = cnt - 1; s >= 0; --s) {
            const int u = w.U[s];
            if (lev[u] < t) continue;
            const int ua = rp[u], ue = rp[u + 1] - 1;
            const double m = __ddiv_rn(w.acc[s], (double)v[ue]);
            for (int p = ua + lane; p < ue; p += 32) {
                const int pos = find_pos(w.U, cnt, ci[p]);
                w.acc[pos] = __dsub_rn(w.acc[pos], __dmul_rn(m, (double)v[p]));
            }
            __syncwarp();
            if (lane == 0) w.acc[s] = __dsub_rn(0.0, m);  // T coefficient of column u
            __syncwarp();
        }
        // emit: survivors to L' (then the diagonal), substituted to T
        int o_l = lp_rp[i], o_t = t_rp[i];
        for (int s0 = 0; s0 < cnt; s0 += 32) {
            const int s = s0 + lane;
            const bool in = s < cnt;
            const int u = in ? w.U[s] : 0;
            const bool sub = in && lev[u] >= t;
            const unsigned bl = __ballot_sync(SPT_FULL_MASK, in && !sub);
            const unsigned bt = __ballot_sync(SPT_FULL_MASK, sub);
            if (in && !sub) {
                const int o = o_l + __popc(bl & lanemask_lt());
                lp_ci[o] = u;
                lp_v[o] = (T)w.acc[s];
            }
            if (sub) {
                const int o = o_t + __popc(bt & lanemask_lt());
                t_ci[o] = u;
                t_v[o] = (T)w.acc[s];
            }
            o_l += __popc(bl);
            o_t += __popc(bt);
        }
        if (lane == 0) {
            lp_ci[o_l] = i;
            lp_v[o_l] = v[e];
        }
        __syncwarp();
    }
}

template <class T>
__global__ void k_rw_copy(const int32_t *rp, const int32_t *ci, const T *v, const int32_t *tgt,
                          int32_t n, const int32_t *lp_rp, int32_t *lp_ci, T *lp_v)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < n; i += nw) {
        if (tgt[i] != kNone) continue;
        const int a = rp[i], e = rp[i + 1], o = lp_rp[i];
        for (int p = a + lane; p < e; p += 32) {
            lp_ci[o + p - a] = ci[p];
            lp_v[o + p - a] = v[p];
        }
    }
}

int blocks_for(int64_t work, int threads, int cap = 65535 * 4)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

// Host side of the rewrite; see sptrsv_rewrite in sptrsv.h.  Returns an sptrsv_status.
int rewrite_run(const sptrsv_csr &L, const int32_t *lev, const int32_t *rows,
                const int32_t *targets, int32_t nrows, int64_t *nnz_Lp, int64_t *nnz_T,
                sptrsv_csr_out *Lp_out, sptrsv_csr_out *T_out, const DeviceInfo &di,
                cudaStream_t s)
{
    const int32_t n = L.n;
    cudaError_t e = cudaSuccess;
    int32_t *tgt = nullptr, *flag = nullptr, *pos = nullptr, *list = nullptr;
    int32_t *len_lp = nullptr, *len_t = nullptr, *lp_rp_tmp = nullptr, *t_rp_tmp = nullptr;
    long long *bad = nullptr;
    int64_t *tot = nullptr;
    int *need = nullptr;
    char *ws = nullptr;
    int status = SPTRSV_OK;
    const size_t nn = (size_t)(n > 0 ? n : 1);
#define RW_CHECK(x)                                  \
    do {                                             \
        e = (x);                                     \
        if (e != cudaSuccess) { status = (e == cudaErrorMemoryAllocation) ? SPTRSV_ENOMEM : SPTRSV_ECUDA; goto done; } \
    } while (0)
    RW_CHECK(cudaMallocAsync(&tgt, sizeof(int32_t) * nn, s));
    RW_CHECK(cudaMallocAsync(&flag, sizeof(int32_t) * nn, s));
    RW_CHECK(cudaMallocAsync(&pos, sizeof(int32_t) * (nn + 1), s));
    RW_CHECK(cudaMallocAsync(&len_lp, sizeof(int32_t) * nn, s));
    RW_CHECK(cudaMallocAsync(&len_t, sizeof(int32_t) * nn, s));
    RW_CHECK(cudaMallocAsync(&bad, sizeof(long long) + sizeof(int64_t) * 2 + sizeof(int), s));
    tot = reinterpret_cast<int64_t *>(bad + 1);
    need = reinterpret_cast<int *>(tot + 2);
    RW_CHECK(cudaMemsetAsync(tgt, 0x7F, sizeof(int32_t) * nn, s));
    {
        long long init = LLONG_MAX;
        RW_CHECK(cudaMemcpyAsync(bad, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    }
    if (nrows > 0)
        k_rw_mark<<<blocks_for(nrows, 256), 256, 0, s>>>(rows, targets, nrows, lev, n, tgt, bad);
    RW_CHECK(cudaGetLastError());
    {
        long long hb = 0;
        RW_CHECK(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
        RW_CHECK(cudaStreamSynchronize(s));
        if (hb != LLONG_MAX) { status = (int)(hb & 15); goto done; }
    }
    int32_t nrw;
    {
        k_rw_flags<<<blocks_for(n, 256), 256, 0, s>>>(tgt, n, flag);
        RW_CHECK(exclusive_scan_i32(flag, pos, n, tot, s));
        int64_t h = 0;
        RW_CHECK(cudaMemcpyAsync(&h, tot, sizeof(h), cudaMemcpyDeviceToHost, s));
        RW_CHECK(cudaStreamSynchronize(s));
        nrw = (int32_t)h;
        RW_CHECK(cudaMallocAsync(&list, sizeof(int32_t) * (size_t)(nrw > 0 ? nrw : 1), s));
        k_rw_compact<<<blocks_for(n, 256), 256, 0, s>>>(flag, pos, n, list);
        RW_CHECK(cudaGetLastError());
    }
    {
        // cone capacity: start small, grow on overflow
        int cap = 1024;
        int warps = 0;
        for (;;) {
            const size_t per_warp = (size_t)cap * (2 * 4 + 4 + 8);
            warps = di.num_sms * (kRwThreads / 32) * 4;
            const size_t budget = (size_t)1 << 30;
            while (warps > 32 && (size_t)warps * per_warp > budget) warps >>= 1;
            const int64_t want = nrw > 0 ? nrw : 1;
            if (warps > want) warps = (int)want;
            // whole blocks of kRwThreads/32 warps, each with its own workspace
            warps = (warps + kRwThreads / 32 - 1) / (kRwThreads / 32) * (kRwThreads / 32);
            if (ws) cudaFreeAsync(ws, s);
            ws = nullptr;
            RW_CHECK(cudaMallocAsync(&ws, per_warp * (size_t)warps, s));
            RW_CHECK(cudaMemsetAsync(need, 0, sizeof(int), s));
            k_rw_lengths<<<blocks_for(n, 256), 256, 0, s>>>(L.row_ptr, tgt, n, len_lp, len_t);
            if (nrw > 0)
                k_rw_symbolic<<<warps * 32 / kRwThreads, kRwThreads, 0, s>>>(
                    L.row_ptr, L.col_idx, lev, tgt, list, nrw, ws, cap, len_lp, len_t, need);
            RW_CHECK(cudaGetLastError());
            int hneed = 0;
            RW_CHECK(cudaMemcpyAsync(&hneed, need, sizeof(int), cudaMemcpyDeviceToHost, s));
            RW_CHECK(cudaStreamSynchronize(s));
            if (hneed == 0) break;
            while (cap < hneed) cap <<= 1;
            if (cap > (1 << 24)) { status = SPTRSV_ENOMEM; goto done; }
        }
        int32_t *lp_rp = (Lp_out && Lp_out->row_ptr) ? Lp_out->row_ptr : nullptr;
        int32_t *t_rp = (T_out && T_out->row_ptr) ? T_out->row_ptr : nullptr;
        if (!lp_rp) { RW_CHECK(cudaMallocAsync(&lp_rp_tmp, sizeof(int32_t) * (nn + 1), s)); lp_rp = lp_rp_tmp; }
        if (!t_rp) { RW_CHECK(cudaMallocAsync(&t_rp_tmp, sizeof(int32_t) * (nn + 1), s)); t_rp = t_rp_tmp; }
        RW_CHECK(exclusive_scan_i32(len_lp, lp_rp, n, tot, s));
        RW_CHECK(exclusive_scan_i32(len_t, t_rp, n, tot + 1, s));
        int64_t h2[2] = {0, 0};
        RW_CHECK(cudaMemcpyAsync(h2, tot, sizeof(h2), cudaMemcpyDeviceToHost, s));
        RW_CHECK(cudaStreamSynchronize(s));
        if (h2[0] >= INT_MAX || h2[1] >= INT_MAX) { status = SPTRSV_ENOTSUP; goto done; }
        if (nnz_Lp) *nnz_Lp = h2[0];
        if (nnz_T) *nnz_T = h2[1];
        if (Lp_out == nullptr || Lp_out->col_idx == nullptr) goto done;  // sizing pass
        if (!Lp_out->vals || !T_out || !T_out->row_ptr || (h2[1] > 0 && (!T_out->col_idx || !T_out->vals))) {
            status = SPTRSV_EINVAL;
            goto done;
        }
        if (L.dtype == SPTRSV_F64) {
            if (nrw > 0)
                k_rw_numeric<double><<<warps * 32 / kRwThreads, kRwThreads, 0, s>>>(
                    L.row_ptr, L.col_idx, (const double *)L.vals, lev, tgt, list, nrw, ws, cap, lp_rp,
                    Lp_out->col_idx, (double *)Lp_out->vals, t_rp, T_out->col_idx, (double *)T_out->vals);
            k_rw_copy<double><<<blocks_for((int64_t)n * 32, 256), 256, 0, s>>>(
                L.row_ptr, L.col_idx, (const double *)L.vals, tgt, n, lp_rp, Lp_out->col_idx,
                (double *)Lp_out->vals);
        } else {
            if (nrw > 0)
                k_rw_numeric<float><<<warps * 32 / kRwThreads, kRwThreads, 0, s>>>(
                    L.row_ptr, L.col_idx, (const float *)L.vals, lev, tgt, list, nrw, ws, cap, lp_rp,
                    Lp_out->col_idx, (float *)Lp_out->vals, t_rp, T_out->col_idx, (float *)T_out->vals);
            k_rw_copy<float><<<blocks_for((int64_t)n * 32, 256), 256, 0, s>>>(
                L.row_ptr, L.col_idx, (const float *)L.vals, tgt, n, lp_rp, Lp_out->col_idx,
                (float *)Lp_out->vals);
        }
        RW_CHECK(cudaGetLastError());
        RW_CHECK(cudaStreamSynchronize(s));
    }
done:
#undef RW_CHECK
    cudaFreeAsync(tgt, s);
    cudaFreeAsync(flag, s);
    cudaFreeAsync(pos, s);
    cudaFreeAsync(len_lp, s);
    cudaFreeAsync(len_t, s);
    cudaFreeAsync(bad, s);
    if (list) cudaFreeAsync(list, s);
    if (ws) cudaFreeAsync(ws, s);
    if (lp_rp_tmp) cudaFreeAsync(lp_rp_tmp, s);
    if (t_rp_tmp) cudaFreeAsync(t_rp_tmp, s);
    cudaStreamSynchronize(s);
    return status;
}

}  // namespace spt
