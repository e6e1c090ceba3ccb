// Level-set analysis on the GPU (paper Section 2.1; level table, level costs
// and their statistics of Section 4.1 / Tables 4-5).
//
//   validate  -- one warp per row: lower triangular, sorted, diagonal last.
//   levels    -- lev[i] = 0 without predecessors, else 1 + max lev[j]; computed
//                as a synchronisation-free max-plus "solve": warps take chunks
//                of 32 consecutive rows from a ticket counter (so every chunk
//                only waits on chunks already taken by running warps), rows
//                inside the chunk resolve through shared memory, rows of
//                earlier chunks are polled in global memory with bounded waits.
//   hist      -- rows and costs per level (2*offdiag+1 per row, int64).
//   stats     -- ALC, ARL, AIR and the coefficients of variation from exact
//                integer sums (the m*S2 - S1^2 difference in 128 bits, rounded
//                to double once), so that they are reproducible bit for bit.
//   partition -- perm = rows sorted by (level, row): stable radix sort by level.
#include <climits>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace spt {

namespace {

// ------------------------------------------------------------- validation
__global__ void k_validate(const int32_t *rp, const int32_t *ci, const void *vals, int dtype,
                           int32_t n, int64_t nnz, long long *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ii = gw; ii < n; ii += nw) {
        const int32_t i = (int32_t)ii;
        const int32_t a = rp[i], e = rp[i + 1];
        int code = 0;
        if (i == 0 && a != 0) code = SPTRSV_EINVAL;
        else if (a < 0 || e > nnz || e < a) code = SPTRSV_EINVAL;
        else if (e == a) code = SPTRSV_EDIAG;
        if (code == 0) {
            // first offending position in row order decides between
            // "outside [0, i]" and "not strictly increasing"
            int first_code = 0;
            for (int p0 = a; p0 < e; p0 += 32) {
                const int p = p0 + lane;
                int c = 0;
                if (p < e) {
                    const int32_t col = ci[p];
                    if (col < 0 || col > i) c = SPTRSV_ENOTLOWER;
                    else if (p > a && col <= ci[p - 1]) c = SPTRSV_EUNSORTED;
                }
                const unsigned bad = __ballot_sync(SPT_FULL_MASK, c != 0);
                if (bad) {
                    const int src = __ffs(bad) - 1;
                    first_code = __shfl_sync(SPT_FULL_MASK, c, src);
                    break;
                }
            }
            code = first_code;
            if (code == 0) {
                const bool zero = dtype == SPTRSV_F64 ? ((const double *)vals)[e - 1] == 0.0
                                                      : ((const float *)vals)[e - 1] == 0.0f;
                if (ci[e - 1] != i || zero) code = SPTRSV_EDIAG;
            }
        }
        if (code != 0 && lane == 0) atomicMin(out, (long long)i * 16 + code);
    }
}

// ----------------------------------------------------------------- levels
constexpr int kLevThreads = 256;
constexpr int kLevWarps = kLevThreads / 32;

constexpr int kLevLong = 32;  // rows with more off-diagonals are walked by the whole warp

// Levels by a synchronisation-free pass over chunks of 32 consecutive rows,
// taken by warps from a ticket: a chunk only waits on chunks already taken
// by running warps, so the pass needs no co-residency.  A level is its own
// ready flag (-1 until published, read with relaxed loads).  A chunk works
// in rounds: every row polls its dependencies on earlier chunks without
// blocking (a cursor stops at the first one not yet published); a row
// whose earlier-chunk dependencies are all seen and whose dependencies in
// the chunk are all published takes its level at once (the chunk's levels
// are kept in shared memory), so that rows are published as early as
// their own dependencies allow.  Once every row has seen all of its
// earlier-chunk dependencies, the rows left (chains inside the chunk) are
// resolved together by a 31-step shuffle sweep instead of one row per
// round.  The polls are bounded in time.
__global__ void __launch_bounds__(kLevThreads)
k_levels(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n, int32_t *lev,
         unsigned long long *ticket, Waiter w, int32_t withhold)
{
    __shared__ int slev[kLevWarps][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    volatile int *my = slev[wid];
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(ticket, 1ull);
        c = __shfl_sync(SPT_FULL_MASK, c, 0);
        const int64_t base = (int64_t)c * 32;
        if (base >= n) return;
        const int64_t i = base + lane;
        const bool valid = i < n;
        const int a = valid ? ldro(rp + i) : 0;
        const int pend = valid ? ldro(rp + i + 1) - 1 : 0;
        // long rows are polled by the whole warp (below)
        const bool islong = pend - a > kLevLong;
        int p = a;              // next entry of this row to look at
        int m = -1;             // deepest earlier-chunk dependency seen
        unsigned dmask = 0;     // dependencies on rows of this chunk
        bool ext = !valid || (!islong && a >= pend);  // every earlier-chunk dependency seen
        bool pub = !valid;      // level published (or withheld by the test hook)
        WaitClock clk;
        for (;;) {
            bool moved = false;
            // ---- 1. earlier-chunk dependencies, without blocking
            while (!ext && !islong && p < pend) {
                const int32_t j = ldro(ci + p);
                if (j >= base) {
                    dmask |= 1u << (j - base);
                } else {
                    const int lj = ld_relaxed(lev + j);
                    if (lj < 0) break;
                    m = m > lj ? m : lj;
                }
                ++p;
                moved = true;
            }
            if (!islong && p >= pend) ext = true;
            unsigned pending = __ballot_sync(SPT_FULL_MASK, islong && !ext);
            while (pending) {
                const int s = __ffs(pending) - 1;
                pending &= pending - 1;
                const int sa = __shfl_sync(SPT_FULL_MASK, a, s);
                const int se = __shfl_sync(SPT_FULL_MASK, pend, s);
                int ms = -1;
                unsigned dm = 0;
                bool wait = false;
                for (int q = sa + lane; q < se; q += 32) {
                    const int32_t j = ldro(ci + q);
                    if (j >= base) {
                        dm |= 1u << (j - base);
                    } else {
                        const int lj = ld_relaxed(lev + j);
                        wait |= lj < 0;
                        ms = ms > lj ? ms : lj;
                    }
                }
                ms = __reduce_max_sync(SPT_FULL_MASK, ms);
                dm = __reduce_or_sync(SPT_FULL_MASK, dm);
                if (!__any_sync(SPT_FULL_MASK, wait) && lane == s) {
                    m = ms;
                    dmask = dm;
                    ext = true;
                    moved = true;
                }
            }
            // ---- 2. rows whose dependencies in the chunk are all published
            const unsigned pubm = __ballot_sync(SPT_FULL_MASK, pub);
            if (ext && !pub && (dmask & ~pubm) == 0) {
                int lv = m + 1;
                for (unsigned bits = dmask; bits; bits &= bits - 1) {
                    const int ls = my[__ffs(bits) - 1] + 1;
                    lv = lv > ls ? lv : ls;
                }
                my[lane] = lv;
                if (i != withhold) st_relaxed(lev + i, lv);  // test hook: never published
                pub = true;
                moved = true;
            }
            __syncwarp();
            if (__all_sync(SPT_FULL_MASK, pub)) break;
            // ---- 3. every earlier-chunk dependency seen: the rows left are
            // chains inside the chunk, resolved by one max-plus sweep (step s
            // broadcasts row s's level, final as all of its dependencies are
            // earlier rows; every row depending on it takes it + 1)
            if (__all_sync(SPT_FULL_MASK, ext)) {
                int lv = pub ? my[lane] : m + 1;
#pragma unroll
                for (int s = 0; s < 31; ++s) {
                    const int ls = __shfl_sync(SPT_FULL_MASK, lv, s) + 1;
                    if ((dmask >> s) & 1u) lv = lv > ls ? lv : ls;
                }
                if (!pub && i != withhold) st_relaxed(lev + i, lv);
                break;
            }
            // one decision for the whole warp (the lanes' clocks may straddle
            // the limit)
            if (!__any_sync(SPT_FULL_MASK, moved) && __any_sync(SPT_FULL_MASK, clk.expired(w))) return;
        }
    }
}

__global__ void k_set_counter(unsigned long long *counter, unsigned long long v) { *counter = v; }

// Grid-wide barrier of a cooperative launch (every block resident): block
// leaders count arrivals; the last one resets the count and advances the
// generation (release), the others wait for the generation to move
// (acquire).  Bounded; false on timeout or abort.
__device__ bool grid_sync(unsigned *arrive, unsigned *gen, unsigned nblocks, const Waiter &w)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        const unsigned g = ld_acquire(gen);
        __threadfence();
        if (atomicAdd(arrive, 1u) == nblocks - 1) {
            *arrive = 0u;
            st_release(gen, g + 1u);
        } else {
            WaitClock clk;
            while (ld_acquire(gen) == g)
                if (clk.expired(w)) { s_ok = 0; break; }
        }
    }
    __syncthreads();
    return s_ok != 0;
}

constexpr int kUpdThreads = 256;
// rows changed in one round beyond which the rounds stop (a bulk change, e.g.
// a rewrite of many rows, propagates over many rounds of full passes)
constexpr int kUpdWideFront = 1024;
// candidate windows up to this many rows are scanned by one block (block
// barriers between rounds instead of grid-wide ones), for at most
// kUpdBlockRounds rounds
constexpr int kUpdNarrow = 8192;
constexpr int kUpdBlockRounds = 1 << 15;

// One round over the candidate rows [lo, hi) (stride over `nth` threads from
// `tid`): a row whose predecessors changed in round r - 1 or later (every row
// in round 1) is recomputed; returns this thread's count of changed rows and
// the smallest / largest of them.  In round 1 also the largest span
// i - (first column of row i), which bounds how far a change can reach.
__device__ __forceinline__ void upd_round(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int lo,
                                          int hi, int64_t tid, int64_t nth, int r, int32_t *lev, int32_t *stamp,
                                          int &cnt, int &mn, int &mx, int &span)
{
    for (int64_t ii = lo + tid; ii < hi; ii += nth) {
        const int i = (int)ii;
        const int a = ldro(rp + i), e = ldro(rp + i + 1) - 1;
        if (r == 1 && e > a) span = max(span, i - ldro(ci + a));
        bool cand = r == 1;
        for (int p = a; p < e && !cand; ++p) cand = ld_relaxed(stamp + ldro(ci + p)) >= r - 1;
        if (!cand) continue;
        int m = -1;
        for (int p = a; p < e; ++p) m = max(m, ld_relaxed(lev + ldro(ci + p)));
        if (m + 1 != ld_relaxed(lev + i)) {
            st_relaxed(lev + i, m + 1);
            st_relaxed(stamp + i, r);
            ++cnt;
            mn = min(mn, i);
            mx = max(mx, i);
        }
    }
}

// Block-wide sums / extremes of the four round values (all threads call it).
__device__ __forceinline__ void upd_block_reduce(int &cnt, int &mn, int &mx, int &span, int *sm)
{
    cnt = __reduce_add_sync(SPT_FULL_MASK, (unsigned)cnt);
    mn = __reduce_min_sync(SPT_FULL_MASK, mn);
    mx = __reduce_max_sync(SPT_FULL_MASK, mx);
    span = __reduce_max_sync(SPT_FULL_MASK, span);
    __syncthreads();
    if (threadIdx.x == 0) { sm[0] = 0; sm[1] = INT_MAX; sm[2] = -1; sm[3] = 0; }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sm, cnt);
        atomicMin(sm + 1, mn);
        atomicMax(sm + 2, mx);
        atomicMax(sm + 3, span);
    }
    __syncthreads();
    cnt = sm[0];
    mn = sm[1];
    mx = sm[2];
    span = sm[3];
}

// Levels after a change confined to rows >= first_row, as a fixpoint of
// lev[i] = 1 + max over predecessors (0 without), starting from the levels
// before the change (valid for every row < first_row).  Round 1 recomputes
// every row >= first_row from the current values; round r > 1 only the rows
// with a predecessor whose level changed in round r - 1 or later
// (stamp[j] = last round in which lev[j] changed, 0 = never), which lie in
// the window (smallest changed row, largest changed row + span]: span, the
// largest distance from a row to its first column, bounds how far a row's
// successors are.  A round that changes nothing ends the loop: then every row
// satisfies the recurrence, whose solution on a DAG is unique.  Rounds run
// over the whole grid with grid-wide barriers; once the window is narrow, one
// block continues alone with block barriers (a change that travels along a
// chain of single dependencies, e.g. the boundary of a grid, moves one row per
// round).  The rounds give up -- res = {2, smallest row changed in the last
// round}, every row below it final, the host finishes with the sync-free
// pass -- after max_rounds grid rounds, kUpdBlockRounds block rounds, on a
// round that changes more than kUpdWideFront rows, or when a block round's
// window grows wide; res = {1, n} at the fixpoint.  Cooperative launch (every
// block resident).
__global__ void __launch_bounds__(kUpdThreads)
k_levels_update(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n, int32_t first_row,
                int32_t *lev, int32_t *stamp, int32_t *cnt, int32_t *minrow, int32_t *maxrow, int32_t *span_max,
                int32_t *res, unsigned *bar, int max_rounds, Waiter w, int32_t withhold)
{
    __shared__ int sm[4];
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    int lo = first_row, hi = n;
    int r = 1;
    for (; r <= max_rounds; ++r) {
        int c = 0, mn = INT_MAX, mx = -1, span = 0;
        upd_round(rp, ci, lo, hi, tid, nth, r, lev, stamp, c, mn, mx, span);
        upd_block_reduce(c, mn, mx, span, sm);
        if (threadIdx.x == 0 && c) {
            atomicAdd(cnt + r, c);
            atomicMin(minrow + r, mn);
            atomicMax(maxrow + r, mx);
        }
        if (threadIdx.x == 0 && r == 1) atomicMax(span_max, span);
        // test hook: the first block never arrives at the first barrier
        if (withhold >= 0 && blockIdx.x == 0) return;
        if (!grid_sync(bar, bar + 1, gridDim.x, w)) return;
        // uniform from here on (values read after the barrier)
        const int changed = ld_relaxed(cnt + r);
        if (changed == 0) {
            if (tid == 0) { res[0] = 1; res[1] = n; }
            return;
        }
        if (changed > kUpdWideFront) {
            if (tid == 0) { res[0] = 2; res[1] = ld_relaxed(minrow + r); }
            return;
        }
        lo = ld_relaxed(minrow + r) + 1;
        const int64_t h = (int64_t)ld_relaxed(maxrow + r) + ld_relaxed(span_max) + 1;
        hi = (int)(h < (int64_t)n ? h : (int64_t)n);
        if (hi - lo <= kUpdNarrow) { ++r; break; }
    }
    if (r > max_rounds) {
        if (tid == 0) { res[0] = 2; res[1] = ld_relaxed(minrow + max_rounds); }
        return;
    }
    // narrow window: block 0 continues alone
    if (blockIdx.x != 0) return;
    const int span = ld_relaxed(span_max);
    int last_min = lo - 1;
    for (int rr = r; rr < r + kUpdBlockRounds; ++rr) {
        int c = 0, mn = INT_MAX, mx = -1, sp = 0;
        upd_round(rp, ci, lo, hi, threadIdx.x, blockDim.x, rr, lev, stamp, c, mn, mx, sp);
        upd_block_reduce(c, mn, mx, sp, sm);  // ends with a block barrier: this round's writes are visible
        if (c == 0) {
            if (threadIdx.x == 0) { res[0] = 1; res[1] = n; }
            return;
        }
        last_min = mn;
        lo = mn + 1;
        const int64_t h2 = (int64_t)mx + span + 1;
        hi = (int)(h2 < (int64_t)n ? h2 : (int64_t)n);
        if (c > kUpdWideFront || hi - lo > kUpdNarrow) break;
        // the block barrier orders this round's relaxed stores before the
        // next round's loads for the block's own threads (CTA scope)
        __threadfence_block();
    }
    if (threadIdx.x == 0) { res[0] = 2; res[1] = last_min; }
}

__global__ void k_count_long(const int32_t *rp, int32_t n, int32_t min_offdiag, unsigned long long *out)
{
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += (ldro(rp + i + 1) - ldro(rp + i) - 1) > min_offdiag;
    c = __reduce_add_sync(SPT_FULL_MASK, (unsigned)c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ------------------------------------------------------- level summary
// One warp per level: the row with the fewest dependencies (smallest row
// among equals) by a min over 64-bit keys (deps << 32 | row), the thin flag
// (cost < threshold, compared in double), and the thin-level count, largest
// row count and largest cost of a thin level (atomics into out[0..2]).
__global__ void k_level_summary(const int32_t *__restrict__ rp, const int32_t *__restrict__ perm,
                                const int32_t *__restrict__ level_ptr, const int64_t *__restrict__ cost,
                                int32_t nlevels, double threshold, uint8_t *thin, int32_t *pick,
                                unsigned long long *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t l = gw; l < nlevels; l += nw) {
        const int a = ldro(level_ptr + l), e = ldro(level_ptr + l + 1);
        unsigned long long key = ~0ull;
        for (int q = a + lane; q < e; q += 32) {
            const int i = ldro(perm + q);
            const unsigned long long deps = (unsigned)(ldro(rp + i + 1) - ldro(rp + i) - 1);
            const unsigned long long k = (deps << 32) | (unsigned)i;
            key = k < key ? k : key;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(SPT_FULL_MASK, key, o);
            key = other < key ? other : key;
        }
        if (lane == 0) {
            pick[l] = (int32_t)(key & 0xffffffffull);
            const int64_t c = ldro(cost + l);
            const bool t = (double)c < threshold;
            thin[l] = t ? 1 : 0;
            if (t) {
                atomicAdd(out, 1ull);
                atomicMax(out + 1, (unsigned long long)(e - a));
                atomicMax(out + 2, (unsigned long long)c);
            }
        }
    }
}

// ---------------------------------------------------------------- max/hist
__global__ void k_max(const int32_t *lev, int32_t n, int32_t *out)
{
    int m = -1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, lev[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(SPT_FULL_MASK, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_level_hist(const int32_t *rp, const int32_t *lev, int32_t n, int32_t *counts,
                             unsigned long long *cost)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = lev[i];
        atomicAdd(counts + l, 1);
        atomicAdd(cost + l, (unsigned long long)(2 * (rp[i + 1] - rp[i] - 1) + 1));
    }
}

__global__ void k_iota(int32_t *v, int32_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (int32_t)i;
}

// ------------------------------------------------------------------ stats
typedef unsigned __int128 u128;

// Correctly rounded u128 -> double: keep the top 64 bits with the discarded
// bits folded into a sticky bit, round those once, scale by a power of two.
__device__ double u128_to_double_rn(u128 v)
{
    const unsigned long long hi = (unsigned long long)(v >> 64);
    if (hi == 0) return __ull2double_rn((unsigned long long)v);
    const int bits = 128 - __clzll((long long)hi);  // > 64
    const int shift = bits - 64;
    unsigned long long top = (unsigned long long)(v >> shift);
    const u128 rest = v & ((((u128)1) << shift) - 1);
    if (rest != 0) top |= 1ull;
    const double t = __ull2double_rn(top);
    return t * __longlong_as_double((long long)(1023 + shift) << 52);
}

__device__ double cov_exact(long long m, long long S1, u128 S2)
{
    if (m <= 0 || S1 <= 0) return 0.0;
    const u128 a = (u128)(unsigned long long)m * S2;
    const u128 b = (u128)(unsigned long long)S1 * (u128)(unsigned long long)S1;
    const u128 d = a > b ? a - b : (u128)0;
    return __ddiv_rn(__dsqrt_rn(u128_to_double_rn(d)), __ll2double_rn(S1));
}

__global__ void __launch_bounds__(512)
k_level_stats(int32_t n, int64_t nnz, int32_t nlevels, const int32_t *level_ptr,
              const int64_t *cost, double *out)
{
    __shared__ long long s1[512], r1[512];
    __shared__ u128 s2[512], r2[512];
    long long a1 = 0, b1 = 0;
    u128 a2 = 0, b2 = 0;
    for (int l = threadIdx.x; l < nlevels; l += blockDim.x) {
        const unsigned long long c = (unsigned long long)cost[l];
        const unsigned long long r = (unsigned long long)(level_ptr[l + 1] - level_ptr[l]);
        a1 += (long long)c;
        a2 += (u128)c * c;
        b1 += (long long)r;
        b2 += (u128)r * r;
    }
    s1[threadIdx.x] = a1; s2[threadIdx.x] = a2;
    r1[threadIdx.x] = b1; r2[threadIdx.x] = b2;
    __syncthreads();
    if (threadIdx.x != 0) return;
    long long S1 = 0, R1 = 0;
    u128 S2 = 0, R2 = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
        S1 += s1[t]; S2 += s2[t]; R1 += r1[t]; R2 += r2[t];
    }
    for (int q = 0; q < 6; ++q) out[q] = 0.0;
    if (n <= 0 || nlevels <= 0) return;
    const double L = (double)nlevels;
    const double alc = __ddiv_rn(__ll2double_rn(S1), L);
    out[0] = alc;
    out[1] = __ddiv_rn((double)n, L);
    out[2] = __ddiv_rn(__ll2double_rn(nnz - (long long)n), (double)n);
    const double cv = cov_exact(nlevels, S1, S2);
    out[3] = cv;
    out[4] = cov_exact(nlevels, R1, R2);
    double relax = __dsub_rn(1.0, cv);
    if (relax < 0.0) relax = 0.0;
    out[5] = __dmul_rn(alc, __dadd_rn(1.0, relax));
}

int grid_for(int64_t work, int threads, int cap = 65535 * 4)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

cudaError_t launch_level_summary(const int32_t *rp, const int32_t *perm, const int32_t *level_ptr,
                                 const int64_t *cost, int32_t nlevels, double threshold, uint8_t *thin,
                                 int32_t *pick, unsigned long long *out_dev, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out_dev, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess || nlevels <= 0) return e;
    const int64_t blocks = std::min<int64_t>(((int64_t)nlevels + 7) / 8, 152 * 16);
    k_level_summary<<<(int)blocks, 256, 0, s>>>(rp, perm, level_ptr, cost, nlevels, threshold, thin, pick,
                                                out_dev);
    return cudaGetLastError();
}


cudaError_t launch_validate(const sptrsv_csr &L, long long *out_dev, cudaStream_t s)
{
    long long init = LLONG_MAX;
    cudaError_t e = cudaMemcpyAsync(out_dev, &init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if (L.n <= 0) return cudaSuccess;
    k_validate<<<grid_for((int64_t)L.n * 32, 256), 256, 0, s>>>(L.row_ptr, L.col_idx, L.vals,
                                                                (int)L.dtype, L.n, L.nnz, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_levels(const sptrsv_csr &L, int32_t *lev, const Ctl &ctl, long long limit_ns,
                          const DeviceInfo &di, cudaStream_t s, int64_t first_chunk, int32_t withhold)
{
    if (L.n <= 0) return cudaSuccess;
    // chunk tickets start at first_chunk: the rows before it keep their levels
    k_set_counter<<<1, 1, 0, s>>>(ctl.counters, (unsigned long long)first_chunk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels, kLevThreads, 0);
    if (per_sm < 1) per_sm = 1;
    const int64_t chunks = ((int64_t)L.n + 31) / 32 - first_chunk;
    if (chunks <= 0) return cudaSuccess;
    int64_t blocks = (int64_t)per_sm * di.num_sms;
    const int64_t need = (chunks + kLevWarps - 1) / kLevWarps;
    if (blocks > need) blocks = need;
    Waiter w{ctl.status, ctl.abort_flag, limit_ns};
    k_levels<<<(int)blocks, kLevThreads, 0, s>>>(L.row_ptr, L.col_idx, L.n, lev, ctl.counters, w, withhold);
    return cudaGetLastError();
}

cudaError_t launch_levels_update(const sptrsv_csr &L, int32_t first_row, int32_t *lev, const Ctl &ctl,
                                 long long limit_ns, const DeviceInfo &di, cudaStream_t s, int max_rounds,
                                 int32_t withhold, bool *converged, int32_t *restart_row)
{
    *converged = true;
    *restart_row = L.n;
    const int64_t rows = (int64_t)L.n - first_row;
    if (rows <= 0) return cudaSuccess;
    // scratch: stamp[n], cnt[R+1], minrow[R+1], maxrow[R+1], span, res[2],
    // barrier {count, generation}
    const size_t nstamp = (size_t)L.n, nr = (size_t)max_rounds + 1;
    int32_t *buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, sizeof(int32_t) * (nstamp + 3 * nr + 5), s);
    if (e != cudaSuccess) return e;
    int32_t *stamp = buf, *cnt = buf + nstamp, *minrow = cnt + nr, *maxrow = minrow + nr;
    int32_t *span = maxrow + nr, *res = span + 1;
    unsigned *bar = reinterpret_cast<unsigned *>(res + 2);
    e = cudaMemsetAsync(stamp, 0, sizeof(int32_t) * (nstamp + nr), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(minrow, 0x7f, sizeof(int32_t) * nr, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(maxrow, 0xff, sizeof(int32_t) * nr, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(span, 0, sizeof(int32_t) * 5, s);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels_update, kUpdThreads, 0);
    if (e == cudaSuccess) {
        int64_t grid = (int64_t)std::max(per_sm, 1) * di.num_sms;
        grid = std::min<int64_t>(grid, (rows + kUpdThreads - 1) / kUpdThreads);
        Waiter w{ctl.status, ctl.abort_flag, limit_ns};
        int32_t n = L.n;
        const int32_t *rp = L.row_ptr, *ci = L.col_idx;
        void *args[] = {(void *)&rp,     (void *)&ci,     (void *)&n,    (void *)&first_row, (void *)&lev,
                        (void *)&stamp,  (void *)&cnt,    (void *)&minrow, (void *)&maxrow, (void *)&span,
                        (void *)&res,    (void *)&bar,    (void *)&max_rounds, (void *)&w, (void *)&withhold};
        e = cudaLaunchCooperativeKernel((const void *)k_levels_update, dim3((unsigned)grid), dim3(kUpdThreads),
                                        args, 0, s);
    }
    int32_t hres[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return e;
    // res = {1, n}: fixpoint; {2, row}: rows below `row` are final; {0, 0}:
    // the launch gave up (bounded wait; the abort flag says so) -- start over
    *converged = hres[0] == 1;
    *restart_row = hres[0] == 2 ? hres[1] : (hres[0] == 1 ? L.n : 0);
    return cudaSuccess;
}

cudaError_t launch_count_long(const int32_t *rp, int32_t n, int32_t min_offdiag,
                              unsigned long long *out_dev, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n <= 0) return e;
    k_count_long<<<grid_for(n, 256, 1024), 256, 0, s>>>(rp, n, min_offdiag, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_max(const int32_t *lev, int32_t n, int32_t *maxlev_dev, cudaStream_t s)
{
    int init = -1;
    cudaError_t e = cudaMemcpyAsync(maxlev_dev, &init, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess || n <= 0) return e;
    k_max<<<grid_for(n, 256, 1024), 256, 0, s>>>(lev, n, maxlev_dev);
    return cudaGetLastError();
}

cudaError_t launch_level_hist(const sptrsv_csr &L, const int32_t *lev, int32_t nlevels,
                              int32_t *counts, int64_t *cost, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)nlevels, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cost, 0, sizeof(int64_t) * (size_t)nlevels, s);
    if (e != cudaSuccess || L.n <= 0) return e;
    k_level_hist<<<grid_for(L.n, 256), 256, 0, s>>>(L.row_ptr, lev, L.n, counts,
                                                    (unsigned long long *)cost);
    return cudaGetLastError();
}

cudaError_t launch_level_stats(int32_t n, int64_t nnz, int32_t nlevels, const int32_t *level_ptr,
                               const int64_t *cost, double *stats_dev, cudaStream_t s)
{
    k_level_stats<<<1, 512, 0, s>>>(n, nnz, nlevels, level_ptr, cost, stats_dev);
    return cudaGetLastError();
}

cudaError_t level_partition(const sptrsv_csr &L, const int32_t *lev, int32_t nlevels,
                            int32_t *perm, int32_t *level_ptr, int64_t *cost, cudaStream_t s)
{
    const int32_t n = L.n;
    if (n <= 0) return cudaMemsetAsync(level_ptr, 0, sizeof(int32_t), s);
    int32_t *counts = nullptr, *iota = nullptr;
    uint32_t *keys_out = nullptr;
    cudaError_t e = cudaMallocAsync(&counts, sizeof(int32_t) * (size_t)nlevels, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&iota, sizeof(int32_t) * (size_t)n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&keys_out, sizeof(uint32_t) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    e = launch_level_hist(L, lev, nlevels, counts, cost, s);
    if (e == cudaSuccess) e = exclusive_scan_i32(counts, level_ptr, nlevels, nullptr, s);
    if (e == cudaSuccess) {
        k_iota<<<grid_for(n, 256), 256, 0, s>>>(iota, n);
        int bits = 0;
        while (bits < 32 && ((uint32_t)(nlevels - 1) >> bits) != 0) ++bits;
        e = radix_sort_pairs((const uint32_t *)lev, iota, keys_out, perm, n, bits, s);
    }
    cudaFreeAsync(counts, s);
    cudaFreeAsync(iota, s);
    cudaFreeAsync(keys_out, s);
    return e;
}

}  // namespace spt
