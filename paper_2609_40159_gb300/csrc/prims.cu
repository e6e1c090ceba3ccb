// Building blocks used by the analysis, the rewrite and the plan set-up:
// exclusive scan, stable LSD radix sort of (key, value) pairs, row expansion.
#include "common.cuh"
#include "internal.h"

namespace spt {

// ------------------------------------------------------------------- scan
namespace {
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *total)
{
    __shared__ long long warp_sums[32];
    __shared__ long long block_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(SPT_FULL_MASK, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        long long s = lane < nw ? warp_sums[lane] : 0;
        long long si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(SPT_FULL_MASK, si, o);
            if (lane >= o) si += t;
        }
        if (lane < nw) warp_sums[lane] = si - s;
        if (lane == nw - 1) block_total = si;
    }
    __syncthreads();
    long long res = inc - v + warp_sums[warp];
    long long tot = block_total;
    __syncthreads();
    *total = tot;
    return res;
}

__global__ void k_scan_reduce(const int32_t *in, int64_t n, long long *partial)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long s = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + it;
        if (idx < n) s += in[idx];
    }
    long long tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_scan_partials(long long *partial, int nb, int64_t *total_dev)
{
    long long carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
        int b = b0 + threadIdx.x;
        long long v = b < nb ? partial[b] : 0;
        long long tot;
        long long ex = block_exclusive_scan(v, &tot);
        if (b < nb) partial[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_dev) *total_dev = carry;
}

__global__ void k_scan_apply(const int32_t *in, int32_t *out, int64_t n, const long long *partial)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int32_t v[kScanItems];
    long long s = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + it;
        v[it] = idx < n ? in[idx] : 0;
        s += v[it];
    }
    long long tot;
    long long ex = block_exclusive_scan(s, &tot) + partial[blockIdx.x];
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + it;
        if (idx < n) out[idx] = (int32_t)ex;
        ex += v[it];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = (int32_t)ex;
}
}  // namespace

cudaError_t exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int64_t *total_dev,
                               cudaStream_t s)
{
    if (n <= 0) {
        cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t), s);
        if (e == cudaSuccess && total_dev) e = cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s);
        return e;
    }
    const int nb = (int)((n + kScanTile - 1) / kScanTile);
    long long *partial = nullptr;
    cudaError_t e = cudaMallocAsync(&partial, sizeof(long long) * nb, s);
    if (e != cudaSuccess) return e;
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, n, partial);
    k_scan_partials<<<1, kScanThreads, 0, s>>>(partial, nb, total_dev);
    k_scan_apply<<<nb, kScanThreads, 0, s>>>(in, out, n, partial);
    e = cudaGetLastError();
    cudaFreeAsync(partial, s);
    return e;
}

// ------------------------------------------------------------- radix sort
namespace {
constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 8;
constexpr int kRadixTile = kRadixThreads * kRadixRounds;
constexpr int kRadixWarps = kRadixThreads / 32;

__global__ void k_radix_hist(const uint32_t *keys, int64_t n, int shift, int32_t *hist, int nb)
{
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r) {
        int64_t idx = base + r * kRadixThreads + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: the tile is consumed in rounds of 256 items in input order;
// inside a round, items are ranked by (warp, lane) with __match_any_sync.
__global__ void k_radix_scatter(const uint32_t *keys, const int32_t *vals, int64_t n, int shift,
                                const int32_t *offs, int nb, uint32_t *keys_out,
                                int32_t *vals_out)
{
    __shared__ int run[256];
    __shared__ int wcnt[kRadixWarps][256];
    const int tid = threadIdx.x, warp = tid >> 5;
    run[tid] = offs[(int64_t)tid * nb + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixRounds; ++r) {
        const int64_t idx = base + r * kRadixThreads + tid;
        const bool valid = idx < n;
        uint32_t key = valid ? keys[idx] : 0u;
        int32_t val = valid ? vals[idx] : 0;
        const unsigned d = valid ? ((key >> shift) & 255u) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(SPT_FULL_MASK, d);
        const int rank_w = __popc(peers & lanemask_lt());
        if (valid && rank_w == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pre = 0;
            for (int w = 0; w < warp; ++w) pre += wcnt[w][d];
            const int pos = run[d] + pre + rank_w;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        int add = 0;
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) {
            add += wcnt[w][tid];
            wcnt[w][tid] = 0;
        }
        run[tid] += add;
        __syncthreads();
    }
}
}  // namespace

cudaError_t radix_sort_pairs(const uint32_t *keys, const int32_t *vals, uint32_t *keys_out,
                             int32_t *vals_out, int64_t n, int key_bits, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int passes = key_bits <= 0 ? 1 : (key_bits + 7) / 8;
    const int nb = (int)((n + kRadixTile - 1) / kRadixTile);
    int32_t *hist = nullptr, *offs = nullptr;
    uint32_t *kbuf = nullptr;
    int32_t *vbuf = nullptr;
    cudaError_t e = cudaMallocAsync(&hist, sizeof(int32_t) * 256 * (size_t)nb, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&offs, sizeof(int32_t) * (256 * (size_t)nb + 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&kbuf, sizeof(uint32_t) * (size_t)n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&vbuf, sizeof(int32_t) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    // ping-pong so that the last pass writes keys_out / vals_out
    const uint32_t *ksrc = keys;
    const int32_t *vsrc = vals;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t *kdst = to_out ? keys_out : kbuf;
        int32_t *vdst = to_out ? vals_out : vbuf;
        k_radix_hist<<<nb, kRadixThreads, 0, s>>>(ksrc, n, 8 * p, hist, nb);
        e = exclusive_scan_i32(hist, offs, 256 * (int64_t)nb, nullptr, s);
        if (e != cudaSuccess) break;
        k_radix_scatter<<<nb, kRadixThreads, 0, s>>>(ksrc, vsrc, n, 8 * p, offs, nb, kdst, vdst);
        ksrc = kdst;
        vsrc = vdst;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFreeAsync(hist, s);
    cudaFreeAsync(offs, s);
    cudaFreeAsync(kbuf, s);
    cudaFreeAsync(vbuf, s);
    return e;
}

// ------------------------------------------------------------ expand rows
namespace {
__global__ void k_expand_rows(const int32_t *row_ptr, int32_t n, int32_t *entry_row)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < n; i += nw) {
        const int a = row_ptr[i], e = row_ptr[i + 1];
        for (int p = a + lane; p < e; p += 32) entry_row[p] = (int32_t)i;
    }
}
}  // namespace

cudaError_t expand_rows(const int32_t *row_ptr, int32_t n, int32_t *entry_row, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int blocks = (int)((((int64_t)n * 32) + 255) / 256);
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    k_expand_rows<<<blocks, 256, 0, s>>>(row_ptr, n, entry_row);
    return cudaGetLastError();
}

}  // namespace spt

// ------------------------------------------------------------------ CSC
namespace spt {
namespace {
__global__ void k_iota32(int32_t *v, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (int32_t)i;
}

__global__ void k_col_count(const int32_t *ci, int64_t nnz, int32_t *cnt)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + ci[p], 1);
}

__global__ void k_gather_rows(const int32_t *entry_row, const int32_t *tmap, int64_t nnz,
                              int32_t *crow)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x)
        crow[q] = entry_row[tmap[q]];
}

int grid_of(int64_t work)
{
    int64_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    if (b > 65535 * 4) b = 65535 * 4;
    return (int)b;
}
}  // namespace

// CSC of L: column pointers cp[n+1], row of every entry crow[nnz] (rows
// ascending inside a column, so the diagonal comes first) and the CSR
// position of every entry tmap[nnz] -- a stable sort of the entries by column.
cudaError_t build_csc(const int32_t *rp, const int32_t *ci, int32_t n, int64_t nnz, int32_t *cp,
                      int32_t *crow, int32_t *tmap, cudaStream_t s)
{
    if (n <= 0) return cudaMemsetAsync(cp, 0, sizeof(int32_t), s);
    int32_t *cnt = nullptr, *iota = nullptr, *erow = nullptr;
    uint32_t *kout = nullptr;
    cudaError_t e = cudaMallocAsync(&cnt, sizeof(int32_t) * (size_t)n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&iota, sizeof(int32_t) * (size_t)nnz, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&erow, sizeof(int32_t) * (size_t)nnz, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&kout, sizeof(uint32_t) * (size_t)nnz, s);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)n, s);
    k_col_count<<<grid_of(nnz), 256, 0, s>>>(ci, nnz, cnt);
    e = exclusive_scan_i32(cnt, cp, n, nullptr, s);
    if (e == cudaSuccess) {
        k_iota32<<<grid_of(nnz), 256, 0, s>>>(iota, nnz);
        int bits = 0;
        while (bits < 32 && ((uint32_t)(n - 1) >> bits) != 0) ++bits;
        e = radix_sort_pairs((const uint32_t *)ci, iota, kout, tmap, nnz, bits, s);
    }
    if (e == cudaSuccess) e = expand_rows(rp, n, erow, s);
    if (e == cudaSuccess) {
        k_gather_rows<<<grid_of(nnz), 256, 0, s>>>(erow, tmap, nnz, crow);
        e = cudaGetLastError();
    }
    cudaFreeAsync(cnt, s);
    cudaFreeAsync(iota, s);
    cudaFreeAsync(erow, s);
    cudaFreeAsync(kout, s);
    return e;
}
}  // namespace spt
