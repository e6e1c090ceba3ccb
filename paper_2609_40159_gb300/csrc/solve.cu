// Forward and transpose sparse triangular solves on sm_103a.
//
// Kernels (paper Section 2.1 for the level-set method; the related-work
// section for synchronisation-free solves):
//   k_level_launch      plain level-set solve: one launch per level, one
//                       thread per row (the baseline).
//   k_level_persistent  one launch; warps take row groups in level order from
//                       a ticket and wait on a grid-wide progress counter
//                       (rows of all earlier levels done) instead of a launch
//                       boundary.
//   k_syncfree          one launch; row groups in row order; each row waits on
//                       its own predecessors' ready flags (ld.acquire /
//                       st.release), rows of the same group resolve through
//                       shared memory.
//   k_block             one thread block per system (one per tile of 8
//                       right-hand-side columns); recent solutions in a
//                       shared-memory ring, in-order row groups (for deep,
//                       narrow systems where the cross-SM round trip
//                       dominates).
//   k_csc_values        L's values in CSC order before a transpose solve.
// Every kernel handles both L x = b (rows in increasing order) and the
// adjoint L^T g_b = g_x (rows in decreasing order, reading L through its CSC).
// A rewritten system L' x = b + T b gathers its T row into the same sum.
#include "block.cuh"

namespace spt {

// ------------------------------------------------------------ prologue
__global__ void k_prologue(PlanCtl *ctl)
{
    ctl->ticket = 0ull;
    ctl->progress = 0ull;
    ctl->epoch = ctl->epoch + 1ull;
    ctl->abort_flag = 0;
}

template <class T>
cudaError_t launch_prologue(PlanCtl *ctl, cudaStream_t s)
{
    k_prologue<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

// ------------------------------------------------------- plain level set
template <class T, bool TR>
__global__ void k_level_launch(Sys<T> A, const int32_t *__restrict__ perm, int32_t q_lo,
                               int32_t q_hi, Rhs<T> R)
{
    const int q = q_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= q_hi) return;
    const int i = chk_row(A, perm[q]);
    const int a = RV<T, TR>::beg(A, i), e = RV<T, TR>::end(A, i);
    const T d = RV<T, TR>::diag(A, a, e);
    const bool ht = !TR && has_trow(A, i);
    for (int r = 0; r < R.k; ++r) {
        T s = R.b[(int64_t)i * R.ld + r];
        if (ht)
            for (int p = A.trp[i]; p < A.trp[i + 1]; ++p)
                s += A.tv[p] * R.b[(int64_t)tcol(A, p) * R.ld + r];
        for (int p = a; p < e; ++p)
            s -= RV<T, TR>::val(A, p) * R.x[(int64_t)RV<T, TR>::col(A, p) * R.ld + r];
        R.x[(int64_t)i * R.ld + r] = s / d;
    }
}

template <class T>
cudaError_t solve_level_launch(const Sys<T> &A, const int32_t *perm,
                               const std::vector<int32_t> &h_level_ptr, const Rhs<T> &R,
                               bool trans, cudaStream_t s)
{
    const int L = (int)h_level_ptr.size() - 1;
    for (int t = 0; t < L; ++t) {
        const int l = trans ? L - 1 - t : t;
        const int lo = h_level_ptr[l], hi = h_level_ptr[l + 1];
        const int blocks = (hi - lo + 255) / 256;
        if (trans) k_level_launch<T, true><<<blocks, 256, 0, s>>>(A, perm, lo, hi, R);
        else k_level_launch<T, false><<<blocks, 256, 0, s>>>(A, perm, lo, hi, R);
    }
    return cudaGetLastError();
}

// ------------------------------------------------ shared row computation
// acc[r] += sum over the row's entries handled by this lane of val * x[col]
// (all dependencies must already be complete).
template <class T, int KT, bool TR>
__device__ __forceinline__ void gather_row(const Sys<T> &A, const Rhs<T> &R, int i, int a, int e,
                                           int sl, int lpr, int r0, int kt, T (&acc)[KT])
{
    if (!TR && has_trow(A, i)) {
        const int tb = A.trp[i], te = A.trp[i + 1];
        for (int p = tb + sl; p < te; p += lpr) {
            const T tv = ldro(A.tv + p);
            const T *bb = R.b + (int64_t)tcol(A, p) * R.ld + r0;
#pragma unroll
            for (int r = 0; r < KT; ++r)
                if (r < kt) acc[r] -= tv * bb[r];
        }
    }
    for (int p = a + sl; p < e; p += lpr) {
        const T vv = RV<T, TR>::val(A, p);
        const T *xx = R.x + (int64_t)RV<T, TR>::col(A, p) * R.ld + r0;
#pragma unroll
        for (int r = 0; r < KT; ++r)
            if (r < kt) acc[r] += vv * xx[r];
    }
}

// The same for a row of a thin run whose earlier levels may still be in
// progress: a dependency in the run (processing level >= h) is read once
// its ready flag is set.  Returns false when a wait gave up.
template <class T, int KT, bool TR>
__device__ __forceinline__ bool gather_row_run(const Sys<T> &A, const Rhs<T> &R, const Sched &S, int h, int i,
                                               int a, int e, int sl, int lpr, int r0, int kt, T (&acc)[KT],
                                               const SyncArgs &sy, uint32_t epoch)
{
    if (!TR && has_trow(A, i)) {
        const int tb = A.trp[i], te = A.trp[i + 1];
        for (int p = tb + sl; p < te; p += lpr) {
            const T tv = ldro(A.tv + p);
            const T *bb = R.b + (int64_t)tcol(A, p) * R.ld + r0;
#pragma unroll
            for (int r = 0; r < KT; ++r)
                if (r < kt) acc[r] -= tv * bb[r];
        }
    }
    for (int p = a + sl; p < e; p += lpr) {
        const int j = RV<T, TR>::col(A, p);
        const int lj = chk_index(ldro(S.lev + j), 0, S.nlevels, A.chk);
        const T vv = RV<T, TR>::val(A, p);
        const bool in_run = (TR ? S.nlevels - 1 - lj : lj) >= h;
        if (in_run && sy.vflags) {
            // one right-hand side: the flag carries the value
            T xv;
            if (!wait_value(sy.vflags, j, epoch, sy.w, xv)) return false;
            acc[0] += vv * xv;
            continue;
        }
        if (in_run && !wait_flag(sy.flags + j, epoch, sy.w)) return false;
        const T *xx = R.x + (int64_t)j * R.ld + r0;
#pragma unroll
        for (int r = 0; r < KT; ++r)
            if (r < kt) acc[r] += vv * xx[r];
    }
    return true;
}

// ------------------------------------------------ persistent level set
// Row groups in level order (transpose: reverse level order) from a
// ticket; a group of level l waits until the grid-wide count of completed
// rows covers every earlier level.  Hybrid schedule (S.seg set): a level
// inside a run of thin levels waits only for the rows before the run, and
// its dependencies inside the run are waited for one by one through the
// rows' ready flags (the synchronisation-free protocol), so that the thin
// levels of a run overlap instead of taking one grid-wide hop each.
template <class T, int KT, bool TR>
__global__ void __launch_bounds__(256)
k_level_persistent(Sys<T> A, Sched S, Rhs<T> R, int rpw, SyncArgs sy)
{
    const int lane = threadIdx.x & 31;
    const int lpr = 32 / rpw;
    const int g = lane / lpr, sl = lane & (lpr - 1);
    const int n = A.n, L = S.nlevels;
    const uint32_t epoch = (uint32_t)sy.ctl->epoch;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(&sy.ctl->ticket, 1ull);
        c = __shfl_sync(SPT_FULL_MASK, c, 0);
        if ((int64_t)c >= S.nchunks) return;
        const int q0 = (int)c * rpw;
        const int q1 = min(q0 + rpw, n);
        int l = S.chunk_level[c];
        for (;;) {
            const int lstart = TR ? n - S.level_ptr[L - l] : S.level_ptr[l];
            const int lend = TR ? n - S.level_ptr[L - 1 - l] : S.level_ptr[l + 1];
            const int lo = max(q0, lstart), hi = min(q1, lend);
            // row metadata and the reciprocal diagonal do not depend on the
            // solution: load them before waiting for the previous levels
            const int q = q0 + g;
            const bool active = q >= lo && q < hi;
            const int i = active ? chk_row(A, TR ? S.perm[n - 1 - q] : S.perm[q]) : 0;
            const int a = active ? RV<T, TR>::beg(A, i) : 0;
            const int e = active ? RV<T, TR>::end(A, i) : 0;
            const T rinv = active ? T(1) / RV<T, TR>::diag(A, a, e) : T(0);
            // hybrid: the run's first level h, whose start is all this
            // group waits for (h == l: a thick level or a run's first level)
            const int h = S.seg ? S.seg[l] : l;
            const int wstart = h == l ? lstart : (TR ? n - S.level_ptr[L - h] : S.level_ptr[h]);
            int ok = 1;
            if (lane == 0) ok = wait_count(&sy.ctl->progress, (unsigned long long)wstart, sy.w);
            ok = __shfl_sync(SPT_FULL_MASK, ok, 0);
            if (!ok) return;
            __syncwarp();
            for (int r0 = 0; r0 < R.k; r0 += KT) {
                const int kt = min(KT, R.k - r0);
                T acc[KT];
#pragma unroll
                for (int r = 0; r < KT; ++r) acc[r] = T(0);
                bool got = true;
                if (active) {
                    if (h < l)
                        got = gather_row_run<T, KT, TR>(A, R, S, h, i, a, e, sl, lpr, r0, kt, acc, sy, epoch);
                    else
                        gather_row<T, KT, TR>(A, R, i, a, e, sl, lpr, r0, kt, acc);
                }
                if (__any_sync(SPT_FULL_MASK, !got)) return;
                group_reduce<T, KT>(acc, lpr);
                if (active && sl == 0) {
                    const T *bb = R.b + (int64_t)i * R.ld + r0;
                    T *xx = R.x + (int64_t)i * R.ld + r0;
#pragma unroll
                    for (int r = 0; r < KT; ++r)
                        if (r < kt) xx[r] = (bb[r] - acc[r]) * rinv;
                    // hybrid: the row's ready flag (after its last tile)
                    if (S.seg && r0 + KT >= R.k && i != sy.withhold) {
                        if (sy.vflags)
                            vflag_publish(sy.vflags, i, (bb[0] - acc[0]) * rinv, epoch);
                        else
                            st_release(sy.flags + i, epoch);
                    }
                }
            }
            // test hook: a withheld row is never counted, so that every
            // later level waits for it until the bounded wait gives up
            const unsigned held = __ballot_sync(SPT_FULL_MASK, active && sl == 0 && i == sy.withhold);
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                atomicAdd(&sy.ctl->progress, (unsigned long long)(hi - lo - __popc(held)));
            }
            if (hi >= q1) break;
            ++l;
        }
    }
}

// --------------------------------------------------------- sync-free
constexpr int kSfThreads = 256;
constexpr int kSfWarps = kSfThreads / 32;

template <class T, int KT, bool TR>
__global__ void __launch_bounds__(kSfThreads)
k_syncfree(Sys<T> A, Rhs<T> R, int rpw, SyncArgs sy)
{
    __shared__ T xs_all[kSfWarps][32 * KT];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    volatile T *xs = xs_all[wid];
    const int lpr = 32 / rpw;
    const int g = lane / lpr, sl = lane & (lpr - 1);
    const unsigned gm = lpr == 32 ? 0xffffffffu : ((1u << lpr) - 1u);
    const int n = A.n;
    const uint32_t epoch = (uint32_t)sy.ctl->epoch;
    const int64_t nchunks = ((int64_t)n + rpw - 1) / rpw;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(&sy.ctl->ticket, 1ull);
        c = __shfl_sync(SPT_FULL_MASK, c, 0);
        if ((int64_t)c >= nchunks) return;
        const int base = (int)c * rpw;
        const int pos = base + g;
        const bool valid = pos < n;
        const int i = valid ? (TR ? n - 1 - pos : pos) : 0;
        const int a = valid ? RV<T, TR>::beg(A, i) : 0;
        const int e = valid ? RV<T, TR>::end(A, i) : 0;
        const unsigned leaders = __ballot_sync(SPT_FULL_MASK, valid && sl == 0);
        for (int r0 = 0; r0 < R.k; r0 += KT) {
            const int kt = min(KT, R.k - r0);
            const bool last_tile = r0 + KT >= R.k;
            T acc[KT];
#pragma unroll
            for (int r = 0; r < KT; ++r) acc[r] = T(0);
            if (!TR && valid && has_trow(A, i)) {
                const int tb = A.trp[i], te = A.trp[i + 1];
                for (int p = tb + sl; p < te; p += lpr) {
                    const T tv = ldro(A.tv + p);
                    const T *bb = R.b + (int64_t)tcol(A, p) * R.ld + r0;
#pragma unroll
                    for (int r = 0; r < KT; ++r)
                        if (r < kt) acc[r] -= tv * bb[r];
                }
            }
            int p = a + sl;
            unsigned fin = 0;
            bool failed = false;
            for (;;) {
                const bool open = valid && !((fin >> (g * lpr)) & 1u);
                if (open) {
                    while (p < e) {
                        const int j = RV<T, TR>::col(A, p);
                        const int pj = order_pos<TR>(n, j);
                        const T vv = RV<T, TR>::val(A, p);
                        if (pj >= base) {
                            const int gj = pj - base;
                            if (!((fin >> (gj * lpr)) & 1u)) break;
#pragma unroll
                            for (int r = 0; r < KT; ++r)
                                if (r < kt) acc[r] += vv * xs[gj * KT + r];
                        } else if (sy.vflags) {
                            // one right-hand side: the flag carries the value
                            T xv;
                            if (!wait_value(sy.vflags, j, epoch, sy.w, xv)) { failed = true; break; }
                            acc[0] += vv * xv;
                        } else {
                            if (!wait_flag(sy.flags + j, epoch, sy.w)) { failed = true; break; }
                            const T *xx = R.x + (int64_t)j * R.ld + r0;
#pragma unroll
                            for (int r = 0; r < KT; ++r)
                                if (r < kt) acc[r] += vv * xx[r];
                        }
                        p += lpr;
                    }
                }
                const bool ready = !open || p >= e || failed;
                const unsigned bal = __ballot_sync(SPT_FULL_MASK, ready);
                if (__any_sync(SPT_FULL_MASK, failed)) return;
                const bool grp_ready = ((bal >> (g * lpr)) & gm) == gm;
                const bool newly = open && grp_ready;
                if (__any_sync(SPT_FULL_MASK, newly)) {
                    T red[KT];
#pragma unroll
                    for (int r = 0; r < KT; ++r) red[r] = acc[r];
                    group_reduce<T, KT>(red, lpr);
                    if (newly && sl == 0) {
                        const T d = RV<T, TR>::diag(A, a, e);
                        const T *bb = R.b + (int64_t)i * R.ld + r0;
                        T *xx = R.x + (int64_t)i * R.ld + r0;
#pragma unroll
                        for (int r = 0; r < KT; ++r)
                            if (r < kt) {
                                const T xv = (bb[r] - red[r]) / d;
                                xs[g * KT + r] = xv;
                                xx[r] = xv;
                            }
                        if (last_tile && i != sy.withhold) {
                            if (sy.vflags)
                                vflag_publish(sy.vflags, i, (bb[0] - red[0]) / d, epoch);
                            else
                                st_release(sy.flags + i, epoch);
                        }
                    }
                }
                fin |= __ballot_sync(SPT_FULL_MASK, newly && sl == 0);
                __syncwarp();
                if ((fin & leaders) == leaders) break;
            }
        }
    }
}

// Sync-free solve with one lane per row: dependencies on earlier groups are
// waited for through their ready flags, dependencies inside the group are
// resolved by the column sweep (lane s's solution broadcast at step s).
constexpr int kSwThreads = 128;
constexpr int kSwWarps = kSwThreads / 32;

template <class T, int KT, bool TR>
__global__ void __launch_bounds__(kSwThreads)
k_syncfree_sweep(Sys<T> A, Rhs<T> R, SyncArgs sy)
{
    __shared__ T coef_all[kSwWarps][1024];
    __shared__ T xbuf_all[kSwWarps][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *coef = coef_all[wid];
    T *xbuf = xbuf_all[wid];
    const int n = A.n;
    const uint32_t epoch = (uint32_t)sy.ctl->epoch;
    const int64_t nchunks = ((int64_t)n + 31) / 32;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(&sy.ctl->ticket, 1ull);
        c = __shfl_sync(SPT_FULL_MASK, c, 0);
        if ((int64_t)c >= nchunks) return;
        const int base = (int)c * 32;
        const int pos = base + lane;
        const bool valid = pos < n;
        const int i = valid ? (TR ? n - 1 - pos : pos) : 0;
        int a = 0, e = 0;
        T rinv = T(0);
        if (valid) {
            a = RV<T, TR>::beg(A, i);
            e = RV<T, TR>::end(A, i);
            rinv = T(1) / RV<T, TR>::diag(A, a, e);
        }
        for (int r0 = 0; r0 < R.k; r0 += KT) {
            const int ktile = min(KT, R.k - r0);
            const bool last_tile = r0 + KT >= R.k;
            T acc[KT], bv[KT];
#pragma unroll
            for (int r = 0; r < KT; ++r) {
                acc[r] = T(0);
                bv[r] = (valid && r < ktile) ? R.b[(int64_t)i * R.ld + r0 + r] : T(0);
            }
            if (!TR && valid && has_trow(A, i)) {
                for (int p = A.trp[i]; p < A.trp[i + 1]; ++p) {
                    const T tv = ldro(A.tv + p);
                    const T *bb = R.b + (int64_t)tcol(A, p) * R.ld + r0;
#pragma unroll
                    for (int r = 0; r < KT; ++r)
                        if (r < ktile) acc[r] -= tv * bb[r];
                }
            }
            // entries loaded kMaxBatch at a time; earlier groups waited for
            // through their flags and applied, this group's recorded for the
            // sweep
            bool failed = false;
            unsigned dmask = 0;
            if (valid) {
                for (int p0 = a; p0 < e && !failed; p0 += kMaxBatch) {
                    int jj[kMaxBatch];
                    T vvv[kMaxBatch];
#pragma unroll
                    for (int u = 0; u < kMaxBatch; ++u)
                        if (p0 + u < e) {
                            jj[u] = RV<T, TR>::col(A, p0 + u);
                            vvv[u] = RV<T, TR>::val(A, p0 + u);
                        }
#pragma unroll
                    for (int u = 0; u < kMaxBatch; ++u)
                        if (p0 + u < e && !failed) {
                            const int j = jj[u];
                            const int pj = order_pos<TR>(n, j);
                            if (pj >= base) {
                                dmask |= 1u << (pj - base);
                                coef[(pj - base) * 32 + lane] = vvv[u];
                                continue;
                            }
                            if (sy.vflags) {
                                // one right-hand side: the flag carries the value
                                T xv;
                                if (!wait_value(sy.vflags, j, epoch, sy.w, xv)) { failed = true; continue; }
                                acc[0] += vvv[u] * xv;
                                continue;
                            }
                            if (!wait_flag(sy.flags + j, epoch, sy.w)) { failed = true; continue; }
                            const T *xx = R.x + (int64_t)j * R.ld + r0;
#pragma unroll
                            for (int r = 0; r < KT; ++r)
                                if (r < ktile) acc[r] += vvv[u] * xx[r];
                        }
                }
            }
            if (__any_sync(SPT_FULL_MASK, failed)) return;
            group_sweep<T, KT>(dmask, coef, xbuf, acc, bv, rinv);
            if (valid) {
                T *xx = R.x + (int64_t)i * R.ld + r0;
#pragma unroll
                for (int r = 0; r < KT; ++r)
                    if (r < ktile) xx[r] = (bv[r] - acc[r]) * rinv;
                if (last_tile && i != sy.withhold) {
                    if (sy.vflags)
                        vflag_publish(sy.vflags, i, (bv[0] - acc[0]) * rinv, epoch);
                    else
                        st_release(sy.flags + i, epoch);
                }
            }
            __syncwarp();
        }
    }
}

constexpr int kBlockThreads = 512;

template <class T, int KT, bool TR>
__global__ void __launch_bounds__(kBlockThreads)
k_block(Sys<T> A, Rhs<T> R, int rpw, int kc, int P, int nwarps, SyncArgs sy)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    // one block per tile of KT right-hand-side columns: independent chains
    const int r0 = blockIdx.x * KT;
    R.b += r0;
    R.x += r0;
    R.k = min(KT, R.k - r0);
    const int ring = kc * rpw;
    BlockSmem<T, KT> sm = carve_block_smem<T, KT>(smraw, ring, kc, nwarps);
    reset_block_smem<T, KT>(sm, ring, kc);
    __syncthreads();
    block_solve_any<T, KT, TR, true>(A, R, rpw, kc, P, nwarps, sm, sy.w, sy.withhold);
}

size_t block_smem_bytes(int rpw, int kt, int kc, bool f64, int nw)
{
    const size_t ring = (size_t)kc * rpw;
    const size_t w = f64 ? 8 : 4;
    return (size_t)kc * 8 + ring * kt * w + (size_t)nw * (1024 + 32) * w + ring * 4 + (size_t)kc * 4 + 16;
}
// ------------------------------------------------------------- gradient
template <class T>
__global__ void k_grad_vals(Sys<T> A, const T *__restrict__ gb, const T *__restrict__ x,
                            int64_t ld, int32_t k, T *__restrict__ gv)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // 4 rows per warp, 8 lanes per row
    const int g = lane >> 3, sl = lane & 7;
    for (int64_t r4 = gw * 4; r4 < A.n; r4 += nw * 4) {
        const int64_t i = r4 + g;
        if (i >= A.n) continue;
        const int a = ldro(A.rp + i), e = ldro(A.rp + i + 1);
        const T *gi = gb + i * ld;
        for (int p = a + sl; p < e; p += 8) {
            const T *xj = x + (int64_t)ldro(A.ci + p) * ld;
            T s = T(0);
            for (int r = 0; r < k; ++r) s += gi[r] * xj[r];
            gv[p] = -s;
        }
    }
}

template <class T>
cudaError_t grad_vals(const Sys<T> &A, const T *gb, const T *x, int64_t ld, int32_t k, T *gv,
                      cudaStream_t s)
{
    if (A.n <= 0) return cudaSuccess;
    int64_t blocks = ((int64_t)A.n + 31) / 32;
    if (blocks > 65535 * 4) blocks = 65535 * 4;
    k_grad_vals<T><<<(int)blocks, 256, 0, s>>>(A, gb, x, ld, k, gv);
    return cudaGetLastError();
}

// -------------------------------------------------------------- T^T apply
template <class T>
__global__ void k_copy_rhs(const T *src, T *dst, int64_t n, int64_t ld, int32_t k)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * k;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k, r = t - i * k;
        dst[i * ld + r] = src[i * ld + r];
    }
}

// gb = gbp + T^T gbp, one thread per element of gb: row j gathers column j
// of T (CSC, rows ascending), so every element is written once, in a fixed
// order (no atomics: the result does not depend on the schedule).
template <class T>
__global__ void k_tt_gather(Sys<T> A, const T *__restrict__ gbp, T *__restrict__ gb, int64_t ld, int32_t k)
{
    const int64_t total = (int64_t)A.n * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / k;
        const int r = (int)(t - j * k);
        T acc = gbp[j * ld + r];
        const int qa = A.tcp[j], qe = A.tcp[j + 1];
        for (int q = qa; q < qe; ++q) acc += A.tv[A.ttmap[q]] * gbp[(int64_t)A.trow[q] * ld + r];
        gb[j * ld + r] = acc;
    }
}

template <class T>
cudaError_t tt_apply(const Sys<T> &A, const T *gbp, T *gb, int64_t ld, int32_t k, cudaStream_t s)
{
    if (A.n <= 0) return cudaSuccess;
    int64_t blocks = ((int64_t)A.n * k + 255) / 256;
    if (blocks > 65535 * 4) blocks = 65535 * 4;
    if (A.tmask && A.tcp)
        k_tt_gather<T><<<(int)blocks, 256, 0, s>>>(A, gbp, gb, ld, k);
    else
        k_copy_rhs<T><<<(int)blocks, 256, 0, s>>>(gbp, gb, A.n, ld, k);
    return cudaGetLastError();
}

// ------------------------------------------------------ plan helpers
__global__ void k_build_tmask(const int32_t *trp, int32_t n, uint32_t *tmask)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ((int64_t)n + 31) / 32 * 32;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool has = i < n && trp[i + 1] > trp[i];
        const unsigned m = __ballot_sync(SPT_FULL_MASK, has);
        if ((threadIdx.x & 31) == 0) tmask[i >> 5] = m;
    }
}

cudaError_t build_tmask(const int32_t *trp, int32_t n, uint32_t *tmask, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (((int64_t)n + 31) / 32 * 32 + 255) / 256;
    if (blocks > 65535) blocks = 65535;  // grid-stride keeps whole warps together
    k_build_tmask<<<(int)blocks, 256, 0, s>>>(trp, n, tmask);
    return cudaGetLastError();
}

__global__ void k_chunk_levels(const int32_t *level_ptr, int32_t L, int32_t n, int rpw, bool trans,
                               int32_t *chunk_level, int64_t nchunks)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int q0 = (int)(c * rpw);
        const int q = trans ? n - 1 - q0 : q0;  // original perm position
        // largest l with level_ptr[l] <= q
        int lo = 0, hi = L - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (level_ptr[mid] <= q) lo = mid; else hi = mid - 1;
        }
        chunk_level[c] = trans ? L - 1 - lo : lo;
    }
}

cudaError_t build_chunk_levels(const int32_t *level_ptr, int32_t nlevels, int32_t n, int rpw,
                               bool trans, int32_t *chunk_level, cudaStream_t s)
{
    const int64_t nchunks = ((int64_t)n + rpw - 1) / rpw;
    if (nchunks <= 0) return cudaSuccess;
    int64_t blocks = (nchunks + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_chunk_levels<<<(int)blocks, 256, 0, s>>>(level_ptr, nlevels, n, rpw, trans, chunk_level, nchunks);
    return cudaGetLastError();
}

// --------------------------------------------------------- dispatchers
template <class T, int KT>
static cudaError_t lp_launch(const Sys<T> &A, const Sched &S, const Rhs<T> &R, int rpw, bool trans,
                             const SyncArgs &sy, int grid, cudaStream_t s)
{
    if (trans) k_level_persistent<T, KT, true><<<grid, 256, 0, s>>>(A, S, R, rpw, sy);
    else k_level_persistent<T, KT, false><<<grid, 256, 0, s>>>(A, S, R, rpw, sy);
    return cudaGetLastError();
}

template <class T>
cudaError_t solve_level_persistent(const Sys<T> &A, const Sched &S, const Rhs<T> &R, int rpw,
                                   int kt, bool trans, const SyncArgs &sy, int grid, cudaStream_t s)
{
    cudaError_t e = launch_prologue<T>(sy.ctl, s);
    if (e != cudaSuccess || A.n <= 0) return e;
    switch (kt) {
    case 1: return lp_launch<T, 1>(A, S, R, rpw, trans, sy, grid, s);
    case 2: return lp_launch<T, 2>(A, S, R, rpw, trans, sy, grid, s);
    case 4: return lp_launch<T, 4>(A, S, R, rpw, trans, sy, grid, s);
    case 8: return lp_launch<T, 8>(A, S, R, rpw, trans, sy, grid, s);
    default: return lp_launch<T, 16>(A, S, R, rpw, trans, sy, grid, s);
    }
}

template <class T, int KT>
static cudaError_t sf_launch(const Sys<T> &A, const Rhs<T> &R, int rpw, bool trans,
                             const SyncArgs &sy, int grid, cudaStream_t s)
{
    if (rpw == 32) {
        // 128-thread blocks: twice as many blocks as the 256-thread grid
        if (trans) k_syncfree_sweep<T, KT, true><<<2 * grid, kSwThreads, 0, s>>>(A, R, sy);
        else k_syncfree_sweep<T, KT, false><<<2 * grid, kSwThreads, 0, s>>>(A, R, sy);
        return cudaGetLastError();
    }
    if (trans) k_syncfree<T, KT, true><<<grid, kSfThreads, 0, s>>>(A, R, rpw, sy);
    else k_syncfree<T, KT, false><<<grid, kSfThreads, 0, s>>>(A, R, rpw, sy);
    return cudaGetLastError();
}

template <class T>
cudaError_t solve_syncfree(const Sys<T> &A, const Rhs<T> &R, int rpw, int kt, bool trans,
                           const SyncArgs &sy, int grid, cudaStream_t s)
{
    cudaError_t e = launch_prologue<T>(sy.ctl, s);
    if (e != cudaSuccess || A.n <= 0) return e;
    switch (kt) {
    case 1: return sf_launch<T, 1>(A, R, rpw, trans, sy, grid, s);
    case 2: return sf_launch<T, 2>(A, R, rpw, trans, sy, grid, s);
    case 4: return sf_launch<T, 4>(A, R, rpw, trans, sy, grid, s);
    case 8: return sf_launch<T, 8>(A, R, rpw, trans, sy, grid, s);
    default: return sf_launch<T, 16>(A, R, rpw, trans, sy, grid, s);
    }
}


void block_geometry(int rpw, int kt, bool f64, int nwarps, int *kc, int *P, size_t grow_limit)
{
    // Throttle distance P (row groups a group may run ahead of the completed
    // prefix) is about the number of active warps; the ring holds kc >= 2P
    // groups, kc a power of two (slots are addressed with a mask).  When
    // that does not fit the shared-memory budget (many right-hand sides) the
    // ring shrinks; correctness only needs kc >= 2P >= 2.
    int k = 4;
    while (k < 2 * (nwarps + 2)) k <<= 1;
    while (k > 4 && block_smem_bytes(rpw, kt, k, f64, nwarps) > kBlockSmemBudget) k >>= 1;
    *P = k / 2;
    while (k < 4096 / rpw && block_smem_bytes(rpw, kt, k * 2, f64, nwarps) <= grow_limit)
        k <<= 1;  // a longer ring keeps more dependencies in shared memory
    *kc = k;
}

int block_warps_for(double rows_per_level, int rpw)
{
    // one lane per row (column sweep, groups complete in order): the extra
    // warps preload later groups, so use all of them
    if (rpw == 32) return kMaxBlockWarps;
    // enough row groups in flight to cover about two levels; at least two
    // warps so that one group's loads overlap the previous group's sweep
    int w = (int)(2.0 * rows_per_level / rpw + 0.999);
    if (w < 2) w = 2;
    if (w > kMaxBlockWarps) w = kMaxBlockWarps;
    return w;
}

// The dynamic shared-memory limit is raised once per kernel instantiation
// (outside any stream capture: plans run a first solve before capturing).
template <auto Kernel> static void raise_smem_once()
{
    static bool done = false;  // one flag per kernel instantiation
    if (!done) {
        cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlockSmemBudget);
        done = true;
    }
}

template <class T, int KT>
static cudaError_t blk_launch(const Sys<T> &A, const Rhs<T> &R, int rpw, bool trans,
                              const SyncArgs &sy, int nwarps, cudaStream_t s)
{
    int kc, P;
    block_geometry(rpw, KT, sizeof(T) == 8, nwarps, &kc, &P, kBlockSmemBudget / 2);
    const size_t smem = block_smem_bytes(rpw, KT, kc, sizeof(T) == 8, nwarps);
    if (smem > kBlockSmemBudget) return cudaErrorInvalidConfiguration;
    const int tiles = (R.k + KT - 1) / KT;
    if (trans) {
        raise_smem_once<k_block<T, KT, true>>();
        k_block<T, KT, true><<<tiles, kBlockThreads, smem, s>>>(A, R, rpw, kc, P, nwarps, sy);
    } else {
        raise_smem_once<k_block<T, KT, false>>();
        k_block<T, KT, false><<<tiles, kBlockThreads, smem, s>>>(A, R, rpw, kc, P, nwarps, sy);
    }
    return cudaGetLastError();
}

// Columns per thread block: the next power of two up to 8; wider right-hand
// sides run as several blocks of 8 columns.
int block_kt_for(int k)
{
    int kt = 1;
    while (kt < k && kt < 8) kt <<= 1;
    return kt;
}

bool block_mode_supported(int k, bool f64)
{
    if (k < 1) return false;
    const int kt = block_kt_for(k);
    int kc, P;
    block_geometry(32, kt, f64, kMaxBlockWarps, &kc, &P, kBlockSmemBudget / 2);
    return block_smem_bytes(32, kt, kc, f64, kMaxBlockWarps) <= kBlockSmemBudget;
}

template <class T>
cudaError_t solve_block(const Sys<T> &A, const Rhs<T> &R, int rpw, int kt, bool trans,
                        const SyncArgs &sy, int nwarps, cudaStream_t s)
{
    (void)kt;
    cudaError_t e = launch_prologue<T>(sy.ctl, s);
    if (e != cudaSuccess || A.n <= 0) return e;
    switch (block_kt_for(R.k)) {
    case 1: return blk_launch<T, 1>(A, R, rpw, trans, sy, nwarps, s);
    case 2: return blk_launch<T, 2>(A, R, rpw, trans, sy, nwarps, s);
    case 4: return blk_launch<T, 4>(A, R, rpw, trans, sy, nwarps, s);
    default: return blk_launch<T, 8>(A, R, rpw, trans, sy, nwarps, s);
    }
}

int persistent_grid_level(int kt, bool f64, const DeviceInfo &di)
{
    int per_sm = 0;
    if (f64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level_persistent<double, 1, false>, 256, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level_persistent<float, 1, false>, 256, 0);
    (void)kt;
    if (per_sm < 1) per_sm = 1;
    return per_sm * di.num_sms;
}

int persistent_grid_syncfree(int kt, bool f64, const DeviceInfo &di)
{
    int per_sm = 0;
    if (f64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_syncfree<double, 1, false>, kSfThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_syncfree<float, 1, false>, kSfThreads, 0);
    (void)kt;
    if (per_sm < 1) per_sm = 1;
    return per_sm * di.num_sms;
}

// ------------------------------------------------------ dense layouts
template <class T>
__global__ void __launch_bounds__(256)
k_transpose_dense(const T *__restrict__ src, int64_t lds, T *__restrict__ dst, int64_t ldd, int64_t rows,
                  int64_t cols)
{
    __shared__ T tile[32][33];
    const int64_t tr = (rows + 31) / 32, tc = (cols + 31) / 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int64_t t = blockIdx.x; t < tr * tc; t += gridDim.x) {
        const int64_t r0 = (t / tc) * 32, c0 = (t % tc) * 32;
        for (int y = ty; y < 32; y += 8) {
            const int64_t r = r0 + y, c = c0 + tx;
            if (r < rows && c < cols) tile[y][tx] = src[r * lds + c];
        }
        __syncthreads();
        for (int y = ty; y < 32; y += 8) {
            const int64_t c = c0 + y, r = r0 + tx;
            if (r < rows && c < cols) dst[c * ldd + r] = tile[tx][y];
        }
        __syncthreads();
    }
}

template <class T>
cudaError_t transpose_dense(const T *src, int64_t lds, T *dst, int64_t ldd, int64_t rows, int64_t cols,
                            cudaStream_t s)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const int64_t tiles = ((rows + 31) / 32) * ((cols + 31) / 32);
    k_transpose_dense<T><<<(int)std::min<int64_t>(tiles, 152 * 16), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
    return cudaGetLastError();
}

// ------------------------------------------------------ CSC values
template <class T>
__global__ void k_csc_values(const int32_t *__restrict__ tmap, const T *__restrict__ v, T *__restrict__ cv,
                             int64_t nnz)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x)
        cv[q] = ldro(v + ldro(tmap + q));
}

template <class T>
cudaError_t csc_values(const int32_t *tmap, const T *v, T *cv, int64_t nnz, cudaStream_t s)
{
    if (nnz <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((nnz + 255) / 256, 152 * 16);
    k_csc_values<T><<<(int)blocks, 256, 0, s>>>(tmap, v, cv, nnz);
    return cudaGetLastError();
}

// ------------------------------------------------ explicit instantiations
#define SPT_INST(T)                                                                                     \
    template cudaError_t launch_prologue<T>(PlanCtl *, cudaStream_t);                                   \
    template cudaError_t solve_level_launch<T>(const Sys<T> &, const int32_t *,                         \
                                               const std::vector<int32_t> &, const Rhs<T> &, bool,     \
                                               cudaStream_t);                                           \
    template cudaError_t solve_level_persistent<T>(const Sys<T> &, const Sched &, const Rhs<T> &, int, \
                                                   int, bool, const SyncArgs &, int, cudaStream_t);     \
    template cudaError_t solve_syncfree<T>(const Sys<T> &, const Rhs<T> &, int, int, bool,              \
                                           const SyncArgs &, int, cudaStream_t);                        \
    template cudaError_t solve_block<T>(const Sys<T> &, const Rhs<T> &, int, int, bool,                 \
                                        const SyncArgs &, int, cudaStream_t);                           \
    template cudaError_t grad_vals<T>(const Sys<T> &, const T *, const T *, int64_t, int32_t, T *,      \
                                      cudaStream_t);                                                    \
    template cudaError_t tt_apply<T>(const Sys<T> &, const T *, T *, int64_t, int32_t, cudaStream_t);   \
    template cudaError_t csc_values<T>(const int32_t *, const T *, T *, int64_t, cudaStream_t);          \
    template cudaError_t transpose_dense<T>(const T *, int64_t, T *, int64_t, int64_t, int64_t, cudaStream_t);
SPT_INST(double)
SPT_INST(float)
#undef SPT_INST

}  // namespace spt
