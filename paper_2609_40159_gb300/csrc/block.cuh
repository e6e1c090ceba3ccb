// Thread-block-local synchronisation-free solve of one system, used by the
// single-system block mode (solve.cu) and by the batched solve (batch.cu).
#pragma once

#include "rows.cuh"

namespace spt {

// Shared-memory layout (dynamic): kc phase barriers, ring of `ring` rows x
// KT solution values, per-warp coefficient tables and broadcast buffers,
// ring of row tags (position of the row held by the slot, -1 = empty), ring
// of chunk tags, counters {ticket, completed prefix}.  The one-lane-per-row
// path uses the ring, the coefficient tables, the completed-group counter
// (single-phase) or the barriers (two-phase); the other path uses the tags.
template <class T, int KT> struct BlockSmem {
    uint64_t *bar;  // kc phase barriers: group g arrives on bar[g % kc]
    volatile T *xr;
    T *coef;   // per active warp: [32][32] in-group coefficients
    T *xbuf;   // per active warp: KT broadcast values
    volatile int *tag;
    volatile int *cdone;
    int *ctr;
};

__device__ __forceinline__ void fence_cta() { asm volatile("fence.sc.cta;" ::: "memory"); }
__device__ __forceinline__ void fence_acq_rel_cta() { asm volatile("fence.acq_rel.cta;" ::: "memory"); }

__device__ __forceinline__ int ld_relaxed_cta_smem(const int *p)
{
    int v;
    asm volatile("ld.relaxed.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}

// Solve one system with the whole thread block.  Rows are handled in
// processing order by row groups of `rpw` rows taken from a shared ticket; a
// group may start only when every group at least P positions earlier is
// complete, so that (with kc >= 2P ring groups) a ring slot is never reused
// while a running group can still need it.  Dependencies from the same
// group resolve through the warp loop, those up to P groups back through the
// ring tags, older ones are read from global memory (complete by the
// throttle).  Returns false when a wait gave up.
template <class T, int KT, bool TR>
__device__ bool block_solve(const Sys<T> &A, const Rhs<T> &R, int rpw, int kc, int P,
                            const BlockSmem<T, KT> &sm, const Waiter &w, int withhold)
{
    const int lane = threadIdx.x & 31;
    const int lpr = 32 / rpw;
    const int g = lane / lpr, sl = lane & (lpr - 1);
    const unsigned gm = lpr == 32 ? 0xffffffffu : ((1u << lpr) - 1u);
    const int n = A.n;
    const int ring = kc * rpw;
    const int nchunks = (n + rpw - 1) / rpw;
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(sm.ctr, 1);
        c = __shfl_sync(SPT_FULL_MASK, c, 0);
        if (c >= nchunks) return true;
        int ok = 1;
        if (lane == 0 && c - P >= 0) {
            WaitClock clk;
            while (*(volatile int *)(sm.ctr + 1) <= c - P) {
                if (clk.expired(w)) { ok = 0; break; }
            }
        }
        ok = __shfl_sync(SPT_FULL_MASK, ok, 0);
        if (!ok) return false;
        fence_cta();
        const int base = c * rpw;
        const int pos = base + g;
        const bool valid = pos < n;
        const int i = valid ? (TR ? n - 1 - pos : pos) : 0;
        const int a = valid ? RV<T, TR>::beg(A, i) : 0;
        const int e = valid ? RV<T, TR>::end(A, i) : 0;
        const unsigned leaders = __ballot_sync(SPT_FULL_MASK, valid && sl == 0);
        const int kt = R.k;  // <= KT
        T acc[KT];
#pragma unroll
        for (int r = 0; r < KT; ++r) acc[r] = T(0);
        if (!TR && valid && has_trow(A, i)) {
            const int tb = A.trp[i], te = A.trp[i + 1];
            for (int p = tb + sl; p < te; p += lpr) {
                const T tv = ldro(A.tv + p);
                const T *bb = R.b + (int64_t)tcol(A, p) * R.ld;
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
                    const int cj = pj / rpw;
                    const T vv = RV<T, TR>::val(A, p);
                    if (cj == c) {
                        const int gj = pj - base;
                        if (!((fin >> (gj * lpr)) & 1u)) break;
                        const volatile T *xx = sm.xr + (pj % ring) * KT;
#pragma unroll
                        for (int r = 0; r < KT; ++r)
                            if (r < kt) acc[r] += vv * xx[r];
                    } else if (cj <= c - P) {
                        const T *xx = R.x + (int64_t)j * R.ld;
#pragma unroll
                        for (int r = 0; r < KT; ++r)
                            if (r < kt) acc[r] += vv * xx[r];
                    } else {
                        const int slot = pj % ring;
                        if (sm.tag[slot] != pj) {
                            WaitClock clk;
                            while (sm.tag[slot] != pj) {
                                if (clk.expired(w)) { failed = true; break; }
                            }
                            if (failed) break;
                        }
                        fence_cta();
                        const volatile T *xx = sm.xr + slot * KT;
#pragma unroll
                        for (int r = 0; r < KT; ++r)
                            if (r < kt) acc[r] += vv * xx[r];
                    }
                    p += lpr;
                }
            }
            const bool ready = !open || p >= e || failed;
            const unsigned bal = __ballot_sync(SPT_FULL_MASK, ready);
            if (__any_sync(SPT_FULL_MASK, failed)) return false;
            const bool grp_ready = ((bal >> (g * lpr)) & gm) == gm;
            const bool newly = open && grp_ready;
            if (__any_sync(SPT_FULL_MASK, newly)) {
                T red[KT];
#pragma unroll
                for (int r = 0; r < KT; ++r) red[r] = acc[r];
                group_reduce<T, KT>(red, lpr);
                if (newly && sl == 0) {
                    const T d = RV<T, TR>::diag(A, a, e);
                    const T *bb = R.b + (int64_t)i * R.ld;
                    T *xx = R.x + (int64_t)i * R.ld;
                    volatile T *xrr = sm.xr + (pos % ring) * KT;
#pragma unroll
                    for (int r = 0; r < KT; ++r)
                        if (r < kt) {
                            const T xv = (bb[r] - red[r]) / d;
                            xrr[r] = xv;
                            xx[r] = xv;
                        }
                    fence_cta();
                    if (i != withhold) sm.tag[pos % ring] = pos;
                }
            }
            fin |= __ballot_sync(SPT_FULL_MASK, newly && sl == 0);
            __syncwarp();
            if ((fin & leaders) == leaders) break;
        }
        // group complete: publish it and advance the completed prefix
        if (lane == 0) {
            fence_cta();
            sm.cdone[c % kc] = c;
            fence_cta();
            for (;;) {
                const int pf = *(volatile int *)(sm.ctr + 1);
                if (pf >= nchunks || sm.cdone[pf % kc] != pf) break;
                atomicCAS(sm.ctr + 1, pf, pf + 1);
            }
        }
    }
}

// Dependency of a row group on an EARLIER group of the same system (block
// mode), read from the shared-memory ring once its tag is set, or from
// global memory for groups too old for the ring (complete by the throttle).
constexpr int kMaxBatch = 8;
constexpr int kPreload = 16;  // entries of a row loaded before a group's turn

// acc[r] += v * src[r] for r < KT, with 16-byte loads when the layout allows
// (src is KT-aligned and KT*sizeof(T) is a multiple of 16).
template <class T, int KT>
__device__ __forceinline__ void axpy_vec(T v, const T *src, T (&acc)[KT])
{
    if constexpr (sizeof(T) * KT % 16 == 0) {
        constexpr int V = 16 / sizeof(T);
#pragma unroll
        for (int q = 0; q < KT / V; ++q) {
            const float4 f = reinterpret_cast<const float4 *>(src)[q];
            const T *t = reinterpret_cast<const T *>(&f);
#pragma unroll
            for (int u = 0; u < V; ++u) acc[q * V + u] += v * t[u];
        }
    } else {
#pragma unroll
        for (int r = 0; r < KT; ++r) acc[r] += v * src[r];
    }
}

template <class T, int KT>
__device__ __forceinline__ void store_vec(T *dst, const T (&v)[KT])
{
    if constexpr (sizeof(T) * KT % 16 == 0) {
        constexpr int V = 16 / sizeof(T);
#pragma unroll
        for (int q = 0; q < KT / V; ++q)
            reinterpret_cast<float4 *>(dst)[q] = *reinterpret_cast<const float4 *>(&v[q * V]);
    } else {
#pragma unroll
        for (int r = 0; r < KT; ++r) dst[r] = v[r];
    }
}

// In-group dependencies of a 32-row group, solved in registers.  Lane L
// holds the scaled candidates t_L = (b_L - sum over earlier groups) / L_LL,
// coef[s * 32 + L] = L_Ls / L_LL for every in-group dependency s < L (bit s
// of dmask; other entries of the table are not initialised) and the final
// x_L = t_L - sum_s coef[s * 32 + L] x_s: 31 steps; step s broadcasts x_s
// (final once every s' < s was applied) and every lane that depends on row
// s subtracts its share.
template <class T, int KT>
__device__ __forceinline__ void sweep_scalar(T (&t)[KT], unsigned dmask, const T *coef, int lane)
{
    const unsigned need = __reduce_or_sync(SPT_FULL_MASK, dmask);
#pragma unroll
    for (int s = 0; s < 31; ++s) {
        // warp-uniform skip of rows nobody depends on; only for wide tiles,
        // where the step costs more than the branch (a branch stops the
        // coefficient load from being hoisted onto the previous step)
        if (KT > 4 && !((need >> s) & 1u)) continue;
        const bool hit = (dmask >> s) & 1u;
        const T cf = coef[s * 32 + lane];
#pragma unroll
        for (int r = 0; r < KT; ++r) {
            const T xs = __shfl_sync(SPT_FULL_MASK, t[r], s);
            // a select, not a zero coefficient: an overflowed x_s must not
            // turn independent rows into NaN
            t[r] = hit ? fma(-cf, xs, t[r]) : t[r];
        }
    }
}

// Block-mode solve with one lane per row (groups of 32 rows, dealt to the
// warps round-robin).  Groups complete in order.  Group c:
//   1. before any wait: loads its rows' metadata, right-hand sides and first
//      kPreload entries, builds its in-group coefficient table and applies
//      the entries older than the shared-memory ring (global memory);
//   2. waits, then applies the dependencies held in the ring;
//   3. resolves the in-group dependencies (column sweep) and publishes: ring
//      values, completion (release), global copy.
// Single-phase (the batched solve, many blocks per SM): step 2 waits for
// every group < c on the completed-group counter, which every lane of the
// warp polls.  Two-phase (TWO, one block on an SM): step 2 waits for the
// groups <= c-2 only and applies their entries while group c-1 is still
// being solved; a second wait for group c-1 and its entries precede step 3.
// Two-phase completion goes through kc shared mbarriers of one arrival
// each: group g arrives (release) on bar[g % kc], completing that barrier's
// phase g / kc; a waiting warp is suspended by the hardware instead of
// polling.  A barrier's next completion (group g + kc) cannot come before
// the waiters of g (groups g + 1 and g + 2) are done, as kc >= 4.
// The chain from one completion to the next has no lane-divergent control
// flow (reconverging a divergent warp costs thousands of cycles on this
// path): loads use clamped, always-valid indices, stores of unused lanes go
// to a row of the coefficient table that is never read, selections are
// arithmetic.
// Ring slot safety: the slot of group cj is rewritten by group cj + kc only
// after every group < cj + kc is complete, i.e. after every reader of cj
// finished.  Global reads: the warp that solved group g stores g's global x
// (after publishing g) before it publishes its next group, g + nwarps.  A
// warp starting group c has itself completed c - nwarps, after acquiring
// the completion of every group < c - nwarps, which covers the global x of
// every group <= c - 2 nwarps - 1; entries at least kc >= 2 nwarps + 1
// groups back are therefore read from global memory before the warp waits.
template <class T, int KT, bool TR, bool TWO>
__device__ bool block_solve_sweep(const Sys<T> &A, const Rhs<T> &R, int kc, int P, int nwarps,
                                  const BlockSmem<T, KT> &sm, const Waiter &w, int withhold)
{
    (void)P;
    constexpr int NP = kPreload;
    const int lane = threadIdx.x & 31;
    const int n = A.n;
    const int ring = kc * 32;  // a power of two
    const int rmask = ring - 1;
    const int nchunks = (n + 31) / 32;
    const int kt = R.k;
    const int wid = threadIdx.x >> 5;
    T *coef = sm.coef + (size_t)wid * 1024;
    const T *ring0 = const_cast<const T *>(sm.xr);
    // row of position q in processing order (clamped into the system)
    auto row_at = [&](int q) { return q < n ? (TR ? n - 1 - q : q) : (TR ? n - 1 : 0); };
    // the row extents of a warp's next group are loaded one group ahead, so
    // that a group's entries are one dependent load away when it starts
    int a_nx = 0, e_nx = 0;
    if (wid < nchunks) {
        const int i0 = row_at(wid * 32 + lane);
        a_nx = RV<T, TR>::beg(A, i0);
        e_nx = RV<T, TR>::end(A, i0);
    }
    // groups are dealt round-robin: warp w solves w, w + nwarps, ...
    for (int c = wid; c < nchunks; c += nwarps) {
        const int base = c * 32;
        const int pos = base + lane;
        const bool valid = pos < n;
        const int i = row_at(pos);
        // ---- 1. independent of the solution
        const int a = a_nx;
        const int e = e_nx;
        if (c + nwarps < nchunks) {
            const int inx = row_at(pos + 32 * nwarps);
            a_nx = RV<T, TR>::beg(A, inx);
            e_nx = RV<T, TR>::end(A, inx);
        }
        const int safe = TR ? a - 1 : e;  // position of the diagonal entry
        const T rinv = valid ? T(1) / RV<T, TR>::diag(A, a, e) : T(0);
        T acc[KT], bv[KT];
#pragma unroll
        for (int r = 0; r < KT; ++r) {
            acc[r] = T(0);
            bv[r] = (valid && r < kt) ? R.b[(int64_t)i * R.ld + r] : T(0);
        }
        if (!TR && valid && has_trow(A, i)) {
            for (int p = A.trp[i]; p < A.trp[i + 1]; ++p) {
                const T tv = ldro(A.tv + p);
                const T *bb = R.b + (int64_t)tcol(A, p) * R.ld;
#pragma unroll
                for (int r = 0; r < KT; ++r)
                    if (r < kt) acc[r] -= tv * bb[r];
            }
        }
        int jj[NP];
        T vv[NP];
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const int q = a + u < e ? a + u : safe;
            jj[u] = order_pos<TR>(n, RV<T, TR>::col(A, q));
            vv[u] = RV<T, TR>::val(A, q);
        }
        unsigned dmask = 0;
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const bool in = valid && a + u < e && jj[u] >= base;
            coef[(in ? jj[u] - base : 31) * 32 + lane] = vv[u] * rinv;
            dmask |= in ? (1u << (jj[u] - base)) : 0u;
        }
        // entries beyond the first NP (long rows; in the transpose view,
        // columns longer than NP -- there the farthest entries): in-group
        // ones go to the table; the others are classified so that only the
        // rare ones in group c-1 are left for the group's turn
        const bool longrow = valid && e - a > NP;
        bool tail_near = false, tail_ring = false;
        for (int p0 = a + NP; longrow && p0 < e; p0 += 4) {
            // four entries per round of loads (clamped to the row's last
            // entry, which exists since p0 < e)
            int pjs[4];
            T vs[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int p = min(p0 + q, e - 1);
                pjs[q] = order_pos<TR>(n, RV<T, TR>::col(A, p));
                vs[q] = RV<T, TR>::val(A, p);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (p0 + q >= e) break;
                const int pj = pjs[q];
                if (pj >= base) {
                    dmask |= 1u << (pj - base);
                    coef[(pj - base) * 32 + lane] = vs[q] * rinv;
                } else if (c - (pj >> 5) < kc) {
                    if (pj >= base - 32) tail_near = true;
                    else tail_ring = true;
                }
            }
        }
        const bool anylong = __any_sync(SPT_FULL_MASK, longrow);
        bool ok = true;
        {
            // entries older than the ring (groups <= c - kc) are read from
            // global memory now, before the group's turn (see the visibility
            // argument above)
            bool any_old = false;
#pragma unroll
            for (int u = 0; u < NP; ++u)
                any_old |= valid && a + u < e && c - (jj[u] >> 5) >= kc;
            if (__any_sync(SPT_FULL_MASK, any_old)) {
#pragma unroll
                for (int u = 0; u < NP; ++u) {
                    if (valid && a + u < e && c - (jj[u] >> 5) >= kc) {
                        const T *xx = R.x + (int64_t)order_pos<TR>(n, jj[u]) * R.ld;
#pragma unroll
                        for (int r = 0; r < KT; ++r)
                            if (r < kt) acc[r] += vv[u] * xx[r];
                    }
                }
            }
            for (int p = a + NP; anylong && longrow && p < e; ++p) {
                const int j = RV<T, TR>::col(A, p);
                if (c - (order_pos<TR>(n, j) >> 5) >= kc) {
                    const T v = RV<T, TR>::val(A, p);
                    const T *xx = R.x + (int64_t)j * R.ld;
#pragma unroll
                    for (int r = 0; r < KT; ++r)
                        if (r < kt) acc[r] += v * xx[r];
                }
            }
        }

        if constexpr (!TWO) {
            // the ring pass after the turn is decided now: an entry in the
            // ring keeps its value and becomes its slot's offset; any other
            // entry reads slot 0 with weight 0.  Only loads and multiply-adds
            // are left on the dependent chain.
#pragma unroll
            for (int u = 0; u < NP; ++u) {
                const bool use = valid && a + u < e && jj[u] < base && c - (jj[u] >> 5) < kc;
                vv[u] = use ? vv[u] : T(0);
                jj[u] = use ? (jj[u] & rmask) * KT : 0;
            }
        }
        consume(rinv);
#pragma unroll
        for (int r = 0; r < KT; ++r) consume(bv[r]);
        // ---- 2. groups <= c-2 (group g's arrival is phase g / kc of
        // barrier g % kc); single-phase: all earlier groups (the completed-
        // group counter reaches c; every lane polls it), after the ring
        // entries of the row tails that are in groups <= c-2 (waited for
        // separately, so that their divergent loop runs while group c-1 is
        // being solved)
        if constexpr (TWO) {
            if (c >= 2) ok = mbar_wait(sm.bar + ((c - 2) & (kc - 1)), ((unsigned)(c - 2) / kc) & 1u, w);
        } else {
            if (__any_sync(SPT_FULL_MASK, tail_ring)) {
                WaitClock clk;
                while (ld_acquire_cta_smem(sm.ctr + 1) < c - 1)
                    if (clk.expired(w)) { ok = false; break; }
                if (!__all_sync(SPT_FULL_MASK, ok)) return false;
                for (int p = a + NP; tail_ring && p < e; ++p) {
                    const int pj = order_pos<TR>(n, RV<T, TR>::col(A, p));
                    if (pj < base - 32 && c - (pj >> 5) < kc)
                        axpy_vec<T, KT>(RV<T, TR>::val(A, p), ring0 + (pj & rmask) * KT, acc);
                }
            }
            // relaxed polls, one acquire fence once the count is reached
            // (PTX memory model: a relaxed read followed by fence.acq_rel is
            // an acquire pattern), so that a poll costs one shared load; a
            // warp two or more groups from its turn sleeps between polls, so
            // that waiting warps leave the issue slots to the working ones
            // (several work items share an SM)
            WaitClock clk;
            int done;
            while ((done = ld_relaxed_cta_smem(sm.ctr + 1)) < c) {
                if (c - done > 1) __nanosleep(200);
                if (clk.expired(w)) { ok = false; break; }
            }
            fence_acq_rel_cta();
        }
        if (!__all_sync(SPT_FULL_MASK, ok)) return false;
        if constexpr (TWO) {
            const int lim = base - 32;  // ring entries below lim are applied now
#pragma unroll
            for (int u = 0; u < NP; ++u) {
                const bool use = valid && a + u < e && jj[u] < lim && c - (jj[u] >> 5) < kc;
                axpy_vec<T, KT>(use ? vv[u] : T(0), ring0 + (use ? (jj[u] & rmask) * KT : 0), acc);
            }
        } else {
#pragma unroll
            for (int u = 0; u < NP; ++u) axpy_vec<T, KT>(vv[u], ring0 + jj[u], acc);
        }
        if constexpr (TWO) {
            if (__any_sync(SPT_FULL_MASK, tail_ring)) {
                for (int p = a + NP; tail_ring && p < e; ++p) {
                    const int pj = order_pos<TR>(n, RV<T, TR>::col(A, p));
                    if (pj < base - 32 && c - (pj >> 5) < kc)
                        axpy_vec<T, KT>(RV<T, TR>::val(A, p), ring0 + (pj & rmask) * KT, acc);
                }
            }
        } else if (__any_sync(SPT_FULL_MASK, tail_near)) {
            for (int p = a + NP; tail_near && p < e; ++p) {
                const int pj = order_pos<TR>(n, RV<T, TR>::col(A, p));
                if (pj < base && pj >= base - 32)
                    axpy_vec<T, KT>(RV<T, TR>::val(A, p), ring0 + (pj & rmask) * KT, acc);
            }
        }
        // ---- 3. group c-1 (two-phase), then this group
        if constexpr (TWO) {
            if (c >= 1) ok = mbar_wait(sm.bar + ((c - 1) & (kc - 1)), ((unsigned)(c - 1) / kc) & 1u, w);
            if (!__all_sync(SPT_FULL_MASK, ok)) return false;
#pragma unroll
            for (int u = 0; u < NP; ++u) {
                const bool prev = valid && a + u < e && jj[u] < base && jj[u] >= base - 32;
                axpy_vec<T, KT>(prev ? vv[u] : T(0), ring0 + (prev ? (jj[u] & rmask) * KT : 0), acc);
            }
            if (__any_sync(SPT_FULL_MASK, tail_near)) {
                for (int p = a + NP; tail_near && p < e; ++p) {
                    const int pj = order_pos<TR>(n, RV<T, TR>::col(A, p));
                    if (pj < base && pj >= base - 32)
                        axpy_vec<T, KT>(RV<T, TR>::val(A, p), ring0 + (pj & rmask) * KT, acc);
                }
            }
        }
        __syncwarp();
        T t[KT];
#pragma unroll
        for (int r = 0; r < KT; ++r) t[r] = (bv[r] - acc[r]) * rinv;
        sweep_scalar<T, KT>(t, dmask, coef, lane);
        // ---- publish: ring values, then (release) the completed-group
        // counter or, two-phase, the barrier arrival, then the global copy
        if (valid) store_vec<T, KT>(const_cast<T *>(sm.xr) + (pos & rmask) * KT, t);
        const bool hold = __any_sync(SPT_FULL_MASK, valid && i == withhold);
        __syncwarp();
        if (lane == 0 && !hold) {
            if constexpr (TWO)
                mbar_arrive(sm.bar + (c & (kc - 1)));
            else
                st_release_cta_smem(sm.ctr + 1, c + 1);
        }
        if (valid) {
            T *xx = R.x + (int64_t)i * R.ld;
#pragma unroll
            for (int r = 0; r < KT; ++r)
                if (r < kt) xx[r] = t[r];
        }
        __syncwarp();  // the coefficient table is rewritten by the next group
    }
    return true;
}

// Block-local level-scheduled solve: the rows in level order (transpose:
// its reverse), cut into groups of at most 32 rows of ONE level (`groups`,
// dealt to the warps round-robin, one lane per row).  The rows of a level
// do not depend on each other, so a group needs no in-group sweep, and the
// groups of one level run at the same time; a group waits only until every
// group of the earlier levels is complete (a shared counter of completed
// groups reaches its `wait`: before that count is reached, only groups of
// earlier levels can complete, as later ones are still waiting).  Progress:
// the smallest incomplete group waits for smaller groups only, and its
// warp has completed all of its earlier (smaller) groups.
// Dependencies live in a shared-memory ring addressed by processing
// position (slot = position mod ring).  While a group of level l runs, only
// groups of level l write the ring, at positions below the level's end
// `lend`; so every position q >= lend - ring still holds its own value, and
// entries at positions below base - win (win = ring - (lend - base)) are
// read from global memory instead.  Values, ring slots and global copies of
// a group are written before its completion is counted (release), and a
// waiter acquires the count, so both reads see complete values.
template <class T, int KT, bool TR>
__device__ bool block_solve_levels(const Sys<T> &A, const Rhs<T> &R, const int32_t *__restrict__ perm,
                                   const int32_t *__restrict__ iperm, const LevelGroup *__restrict__ groups,
                                   int ngroups, int kc, int nwarps, const BlockSmem<T, KT> &sm,
                                   const Waiter &w, int withhold)
{
    constexpr int NP = kPreload;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    if (wid >= nwarps) return true;
    const int n = A.n;
    const int ring = kc * 32;  // a power of two
    const int rmask = ring - 1;
    const int kt = R.k;
    const T *ring0 = const_cast<const T *>(sm.xr);
    // row at processing position q; processing position of row j
    auto row_at = [&](int q) { return chk_row(A, ldro(perm + (TR ? n - 1 - q : q))); };
    auto pos_of = [&](int j) {
        const int p = chk_index(ldro(iperm + j), 0, n, A.chk);
        return TR ? n - 1 - p : p;
    };
    // a warp's next group, its rows and their extents are loaded one group
    // ahead, and the group after it one more ahead, so that a group's
    // entries are one dependent load away when it starts
    LevelGroup gn{0, 0, 0, 0}, gnn{0, 0, 0, 0};
    int i_nx = 0, a_nx = 0, e_nx = 0;
    if (wid < ngroups) {
        gn = groups[wid];
        i_nx = row_at(gn.base + (lane < gn.cnt ? lane : 0));
        a_nx = RV<T, TR>::beg(A, i_nx);
        e_nx = RV<T, TR>::end(A, i_nx);
    }
    if (wid + nwarps < ngroups) gnn = groups[wid + nwarps];
    for (int g = wid; g < ngroups; g += nwarps) {
        const LevelGroup G = gn;
        const int i = i_nx, a = a_nx, e = e_nx;
        if (g + nwarps < ngroups) {
            gn = gnn;
            i_nx = row_at(gn.base + (lane < gn.cnt ? lane : 0));
            a_nx = RV<T, TR>::beg(A, i_nx);
            e_nx = RV<T, TR>::end(A, i_nx);
            if (g + 2 * nwarps < ngroups) gnn = groups[g + 2 * nwarps];
        }
        const int base = G.base;
        const bool valid = lane < G.cnt;
        const int pos = base + (valid ? lane : 0);
        // ---- 1. independent of the solution
        const int safe = TR ? a - 1 : e;  // position of the diagonal entry
        const T rinv = valid ? T(1) / RV<T, TR>::diag(A, a, e) : T(0);
        T acc[KT], bv[KT];
#pragma unroll
        for (int r = 0; r < KT; ++r) {
            acc[r] = T(0);
            bv[r] = (valid && r < kt) ? R.b[(int64_t)i * R.ld + r] : T(0);
        }
        if (!TR && valid && has_trow(A, i)) {
            for (int p = A.trp[i]; p < A.trp[i + 1]; ++p) {
                const T tv = ldro(A.tv + p);
                const T *bb = R.b + (int64_t)tcol(A, p) * R.ld;
#pragma unroll
                for (int r = 0; r < KT; ++r)
                    if (r < kt) acc[r] -= tv * bb[r];
            }
        }
        int jj[NP];
        T vv[NP];
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const int q = a + u < e ? a + u : safe;
            jj[u] = pos_of(RV<T, TR>::col(A, q));
            vv[u] = RV<T, TR>::val(A, q);
        }
        // ring window of this group (see above)
        const int win = max(0, ring - (G.lend - base));
        const int lo = base - win;
        bool any_glob = false;
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const bool in = valid && a + u < e;
            const bool use = in && jj[u] >= lo;
            any_glob |= in && !use;
            // ring pass decided now: an entry in the ring keeps its value and
            // becomes its slot's offset; any other entry reads slot 0 with
            // weight 0 (global ones are applied separately, once complete)
            vv[u] = use ? vv[u] : T(0);
            jj[u] = use ? (jj[u] & rmask) * KT : 0;
        }
        const bool longrow = valid && e - a > NP;
        consume(rinv);
#pragma unroll
        for (int r = 0; r < KT; ++r) consume(bv[r]);
        // ---- 2. wait for every group of the earlier levels
        bool ok = true;
        {
            WaitClock clk;
            int done;
            while ((done = ld_relaxed_cta_smem(sm.ctr + 1)) < G.wait) {
                if (G.wait - done > nwarps) __nanosleep(200);
                if (clk.expired(w)) { ok = false; break; }
            }
            fence_acq_rel_cta();
        }
        if (!__all_sync(SPT_FULL_MASK, ok)) return false;
        // ---- 3. dependencies: ring, then global memory, then long rows' tails
#pragma unroll
        for (int u = 0; u < NP; ++u) axpy_vec<T, KT>(vv[u], ring0 + jj[u], acc);
        if (__any_sync(SPT_FULL_MASK, any_glob)) {
            for (int p = a; any_glob && p < e && p < a + NP; ++p) {
                const int j = RV<T, TR>::col(A, p);
                if (pos_of(j) < lo) {
                    const T v = RV<T, TR>::val(A, p);
                    const T *xx = R.x + (int64_t)j * R.ld;
#pragma unroll
                    for (int r = 0; r < KT; ++r)
                        if (r < kt) acc[r] += v * xx[r];
                }
            }
        }
        if (__any_sync(SPT_FULL_MASK, longrow)) {
            for (int p = a + NP; longrow && p < e; ++p) {
                const int j = RV<T, TR>::col(A, p);
                const int pj = pos_of(j);
                const T v = RV<T, TR>::val(A, p);
                if (pj >= lo) {
                    axpy_vec<T, KT>(v, ring0 + (pj & rmask) * KT, acc);
                } else {
                    const T *xx = R.x + (int64_t)j * R.ld;
#pragma unroll
                    for (int r = 0; r < KT; ++r)
                        if (r < kt) acc[r] += v * xx[r];
                }
            }
        }
        T t[KT];
#pragma unroll
        for (int r = 0; r < KT; ++r) t[r] = (bv[r] - acc[r]) * rinv;
        // ---- 4. publish: ring slot and global copy, then (release) the count
        if (valid) {
            store_vec<T, KT>(const_cast<T *>(sm.xr) + (pos & rmask) * KT, t);
            T *xx = R.x + (int64_t)i * R.ld;
#pragma unroll
            for (int r = 0; r < KT; ++r)
                if (r < kt) xx[r] = t[r];
        }
        const bool hold = __any_sync(SPT_FULL_MASK, valid && i == withhold);
        __syncwarp();
        if (lane == 0 && !hold) {
            fence_acq_rel_cta();
            atomicAdd(sm.ctr + 1, 1);
        }
    }
    return true;
}

// Entry used by the kernels: `nwarps` warps of the block work on the system
// (the others return at once); one lane per row uses the column sweep,
// two-phase (TWO) or single-phase.
template <class T, int KT, bool TR, bool TWO>
__device__ __forceinline__ bool block_solve_any(const Sys<T> &A, const Rhs<T> &R, int rpw, int kc,
                                                int P, int nwarps, const BlockSmem<T, KT> &sm,
                                                const Waiter &w, int withhold)
{
    if (rpw == 32) {
        // the sweep's global reads need kc >= 2 nwarps + 1 (always true for
        // the plans' geometries; enforced here)
        const int nw = max(1, min(nwarps, (kc - 1) / 2));
        if ((int)(threadIdx.x >> 5) >= nw) return true;
        return block_solve_sweep<T, KT, TR, TWO>(A, R, kc, P, nw, sm, w, withhold);
    }
    if ((int)(threadIdx.x >> 5) >= nwarps) return true;
    return block_solve<T, KT, TR>(A, R, rpw, kc, P, sm, w, withhold);
}

template <class T, int KT>
__device__ __forceinline__ BlockSmem<T, KT> carve_block_smem(unsigned char *raw, int ring, int kc,
                                                           int nw)
{
    BlockSmem<T, KT> sm;
    sm.bar = reinterpret_cast<uint64_t *>(raw);  // kc * 8 bytes keep what follows 16-byte aligned
    T *xr = reinterpret_cast<T *>(raw + (size_t)kc * 8);
    sm.xr = xr;
    sm.coef = xr + (size_t)ring * KT;
    sm.xbuf = sm.coef + (size_t)nw * 1024;
    int *tag = reinterpret_cast<int *>(sm.xbuf + (size_t)nw * 32);
    sm.tag = tag;
    sm.cdone = tag + ring;
    sm.ctr = tag + ring + kc;
    return sm;
}

// Fresh state for one system (the barriers must not hold a live mbarrier:
// first use of the memory, or release_block_smem ran).
template <class T, int KT>
__device__ __forceinline__ void reset_block_smem(const BlockSmem<T, KT> &sm, int ring, int kc)
{
    for (int t = threadIdx.x; t < ring * KT; t += blockDim.x) sm.xr[t] = T(0);
    for (int t = threadIdx.x; t < ring; t += blockDim.x) sm.tag[t] = -1;
    for (int t = threadIdx.x; t < kc; t += blockDim.x) {
        sm.cdone[t] = -1;
        mbar_init(sm.bar + t, 1);
    }
    if (threadIdx.x == 0) { sm.ctr[0] = 0; sm.ctr[1] = 0; }
}

// After a __syncthreads that ends the work on one system: invalidate the
// barriers so that the memory can be re-initialised for the next one.
template <class T, int KT>
__device__ __forceinline__ void release_block_smem(const BlockSmem<T, KT> &sm, int kc)
{
    for (int t = threadIdx.x; t < kc; t += blockDim.x) mbar_inval(sm.bar + t);
}

}  // namespace spt
