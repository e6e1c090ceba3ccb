// Thread-block-local synchronisation-free solve of one system, used by the
// single-system block mode (solve.cu) and by the batched solve (batch.cu).
#pragma once

#include "rows.cuh"

namespace spt {

// Shared-memory layout (dynamic): ring of `ring` rows x KT solution values,
// ring of row tags (position of the row held by the slot, -1 = empty),
// ring of chunk tags, and counters {ticket, completed prefix}.
template <class T, int KT> struct BlockSmem {
    volatile T *xr;
    T *coef;   // per active warp: [32][32] in-group coefficients
    T *xbuf;   // per active warp: KT broadcast values
    volatile int *tag;
    volatile int *cdone;
    int *ctr;
};

__device__ __forceinline__ void fence_cta() { asm volatile("fence.sc.cta;" ::: "memory"); }

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
                const T *bb = R.b + (int64_t)ldro(A.tci + p) * R.ld;
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

// A group reading the ring slot of group cj: the slot cannot be reused
// before every group <= cj + kc - P is complete, so it is safe for
// cj >= c - kc + P (the tag then tells whether the value is there yet);
// older groups are complete and read from global memory.
template <class T, int KT>
__device__ __forceinline__ bool ring_dep(const BlockSmem<T, KT> &sm, const Rhs<T> &R, int ring,
                                         int c, int P, int kc, int pj, int j, T vv, T (&acc)[KT],
                                         const Waiter &w)
{
    const int kt = R.k;
    if ((pj >> 5) < c - kc + P) {
        const T *xx = R.x + (int64_t)j * R.ld;
#pragma unroll
        for (int r = 0; r < KT; ++r)
            if (r < kt) acc[r] += vv * xx[r];
        return true;
    }
    const int slot = pj % ring;
    int *tg = const_cast<int *>(sm.tag) + slot;
    if (ld_acquire_cta_smem(tg) != pj) {
        WaitClock clk;
        while (ld_acquire_cta_smem(tg) != pj)
            if (clk.expired(w)) return false;
    }
    const T *xx = const_cast<const T *>(sm.xr) + slot * KT;
#pragma unroll
    for (int r = 0; r < KT; ++r)
        if (r < kt) acc[r] += vv * xx[r];
    return true;
}

// Block-mode solve with one lane per row (groups of 32 rows).  Groups
// complete in order: group c waits (one CTA-scope acquire poll by lane 0)
// until the completed prefix reaches c, applies its dependencies on earlier
// groups (shared-memory ring for the last kc-1 groups, global memory before
// that), resolves the dependencies inside the group by the column sweep and
// publishes prefix = c+1 with a CTA-scope release.  The other warps of the
// block meanwhile load their next group's metadata and entries, so the
// loads overlap the chain.  Ring slot safety: a slot of group cj is
// rewritten by group cj + kc only after the prefix passed cj + kc, i.e. after
// every reader of cj (groups < cj + kc) has finished.
// Block-mode solve with one lane per row (groups of 32 rows).  Groups
// complete in order: group c waits until the completed prefix reaches c
// (every lane polls the same shared word, so the warp never diverges around
// the wait), applies its dependencies on earlier groups (shared-memory ring
// for the last kc-1 groups, global memory before that), resolves the
// dependencies inside the group by the column sweep and publishes
// prefix = c+1 with a CTA-scope release.  The other warps of the block
// meanwhile load their own next group's metadata and entries.  The chain
// from one group's release to the next group's release contains no
// lane-divergent control flow (reconverging a divergent warp costs
// thousands of cycles on this path): loads use clamped, always-valid
// indices, stores of unused lanes go to a row of the coefficient table that
// is never read, selections are arithmetic.  Ring slot safety: a slot of
// group cj is rewritten by group cj + kc only after the prefix passed
// cj + kc, i.e. after every reader of cj (groups < cj + kc) has finished.
template <class T, int KT, bool TR>
__device__ bool block_solve_sweep(const Sys<T> &A, const Rhs<T> &R, int kc, int P, int nwarps,
                                  const BlockSmem<T, KT> &sm, const Waiter &w, int withhold)
{
    (void)P;
    const int lane = threadIdx.x & 31;
    const int n = A.n;
    const int ring = kc * 32;  // a power of two
    const int rmask = ring - 1;
    const int nchunks = (n + 31) / 32;
    const int kt = R.k;
    const int wid = threadIdx.x >> 5;
    T *coef = sm.coef + (size_t)wid * 1024;
    int *prefix = sm.ctr + 1;
    const T *ring0 = const_cast<const T *>(sm.xr);
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(sm.ctr, 1);
        c = __shfl_sync(SPT_FULL_MASK, c, 0);
        if (c >= nchunks) return true;
        const int base = c * 32;
        const int pos = base + lane;
        const bool valid = pos < n;
        const int i = valid ? (TR ? n - 1 - pos : pos) : (TR ? n - 1 : 0);
        {
            // pull a later group's entries towards L2
            const int pn = min(pos + 32 * (nwarps + 1), n - 1);
            prefetch_row<T, TR>(A, TR ? n - 1 - pn : pn);
        }
        // ---- independent of the solution: metadata, right-hand side and
        // the first kPreload entries (clamped to the row's diagonal entry),
        // all complete before this group's turn
        const int a = RV<T, TR>::beg(A, i);
        const int e = RV<T, TR>::end(A, i);
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
                const T *bb = R.b + (int64_t)ldro(A.tci + p) * R.ld;
#pragma unroll
                for (int r = 0; r < KT; ++r)
                    if (r < kt) acc[r] -= tv * bb[r];
            }
        }
        int jj[kPreload];
        T vv[kPreload];
#pragma unroll
        for (int u = 0; u < kPreload; ++u) {
            const int q = a + u < e ? a + u : safe;
            jj[u] = RV<T, TR>::col(A, q);
            vv[u] = RV<T, TR>::val(A, q);
        }
        consume(rinv);
#pragma unroll
        for (int r = 0; r < KT; ++r) consume(bv[r]);
#pragma unroll
        for (int u = 0; u < kPreload; ++u) {
            consume(jj[u]);
            consume(vv[u]);
        }
        // ---- wait for every earlier group
        bool ok = true;
        {
            WaitClock clk;
            while (ld_acquire_cta_smem(prefix) < c)
                if (clk.expired(w)) { ok = false; break; }
        }
        if (!__all_sync(SPT_FULL_MASK, ok)) return false;
        // ---- earlier groups (ring) and this group (dmask + coef table;
        // unused entries write row 31, which the sweep never reads)
        // (ring loads first, then the coefficient stores, so that the loads
        // need not wait behind stores they might alias)
        unsigned dmask = 0;
        bool any_old = false;
#pragma unroll
        for (int u = 0; u < kPreload; ++u) {
            const bool has = valid && a + u < e;
            const int pj = order_pos<TR>(n, jj[u]);
            const bool far = has && pj < base;
            const bool old = far && (c - (pj >> 5) >= kc);
            any_old |= old;
            const bool use = far && !old;
            axpy_vec<T, KT>(use ? vv[u] : T(0), ring0 + (use ? (pj & rmask) * KT : 0), acc);
        }
#pragma unroll
        for (int u = 0; u < kPreload; ++u) {
            const bool has = valid && a + u < e;
            const int pj = order_pos<TR>(n, jj[u]);
            const bool in = has && pj >= base;
            coef[(in ? pj - base : 31) * 32 + lane] = vv[u];
            dmask |= in ? (1u << (pj - base)) : 0u;
        }
        if (__any_sync(SPT_FULL_MASK, any_old)) {
#pragma unroll
            for (int u = 0; u < kPreload; ++u) {
                const bool has = valid && a + u < e;
                const int pj = order_pos<TR>(n, jj[u]);
                if (has && pj < base && c - (pj >> 5) >= kc) {
                    const T *xx = R.x + (int64_t)jj[u] * R.ld;
#pragma unroll
                    for (int r = 0; r < KT; ++r)
                        if (r < kt) acc[r] += vv[u] * xx[r];
                }
            }
        }
        for (int p = a + kPreload; valid && p < e; ++p) {  // long rows
            const int j = RV<T, TR>::col(A, p);
            const T v = RV<T, TR>::val(A, p);
            const int pj = order_pos<TR>(n, j);
            if (pj >= base) {
                dmask |= 1u << (pj - base);
                coef[(pj - base) * 32 + lane] = v;
            } else if (c - (pj >> 5) < kc) {
                axpy_vec<T, KT>(v, ring0 + (pj & rmask) * KT, acc);
            } else {
                const T *xx = R.x + (int64_t)j * R.ld;
#pragma unroll
                for (int r = 0; r < KT; ++r)
                    if (r < kt) acc[r] += v * xx[r];
            }
        }
        __syncwarp();
        // ---- in-group dependencies: unrolled column sweep on the scaled
        // candidates t = (b - acc) / L_ii; a dependency on row s is one
        // t -= (coef / L_ii) * x_s after x_s's shuffle broadcast
        T t[KT];
#pragma unroll
        for (int r = 0; r < KT; ++r) t[r] = (bv[r] - acc[r]) * rinv;
        const unsigned need = __reduce_or_sync(SPT_FULL_MASK, dmask);
#pragma unroll
        for (int s2 = 0; s2 < 31; ++s2) {
            if (KT > 4 && !((need >> s2) & 1u)) continue;  // warp-uniform
            const bool hit = (dmask >> s2) & 1u;
            const T cv = coef[s2 * 32 + lane];
            const T cfr = cv * rinv;
#pragma unroll
            for (int r = 0; r < KT; ++r) {
                const T xs = __shfl_sync(SPT_FULL_MASK, t[r], s2);
                // a select, not a zero coefficient: an overflowed x_s must
                // not turn independent rows into NaN
                t[r] = hit ? t[r] - cfr * xs : t[r];
            }
        }
        // ---- publish: ring values, then the prefix (CTA-scope release),
        // then the global copy (its readers are kc >= nwarps+2 groups later
        // and synchronise through later releases)
        if (valid) store_vec<T, KT>(const_cast<T *>(sm.xr) + (pos & rmask) * KT, t);
        const bool hold = __any_sync(SPT_FULL_MASK, valid && i == withhold);
        __syncwarp();
        if (lane == 0 && !hold) st_release_cta_smem(prefix, c + 1);
        if (valid) {
            T *xx = R.x + (int64_t)i * R.ld;
#pragma unroll
            for (int r = 0; r < KT; ++r)
                if (r < kt) xx[r] = t[r];
        }
    }
}

// Entry used by the kernels: `nwarps` warps of the block work on the system
// (the others return at once); one lane per row uses the column sweep.
template <class T, int KT, bool TR>
__device__ __forceinline__ bool block_solve_any(const Sys<T> &A, const Rhs<T> &R, int rpw, int kc,
                                                int P, int nwarps, const BlockSmem<T, KT> &sm,
                                                const Waiter &w, int withhold)
{
    if ((int)(threadIdx.x >> 5) >= nwarps) return true;
    if (rpw == 32) return block_solve_sweep<T, KT, TR>(A, R, kc, P, nwarps, sm, w, withhold);
    return block_solve<T, KT, TR>(A, R, rpw, kc, P, sm, w, withhold);
}

template <class T, int KT>
__device__ __forceinline__ BlockSmem<T, KT> carve_block_smem(unsigned char *raw, int ring, int kc,
                                                           int nw)
{
    BlockSmem<T, KT> sm;
    T *xr = reinterpret_cast<T *>(raw);
    sm.xr = xr;
    sm.coef = xr + (size_t)ring * KT;
    sm.xbuf = sm.coef + (size_t)nw * 1024;
    int *tag = reinterpret_cast<int *>(sm.xbuf + (size_t)nw * 32);
    sm.tag = tag;
    sm.cdone = tag + ring;
    sm.ctr = tag + ring + kc;
    return sm;
}

template <class T, int KT>
__device__ __forceinline__ void reset_block_smem(const BlockSmem<T, KT> &sm, int ring, int kc)
{
    for (int t = threadIdx.x; t < ring * KT; t += blockDim.x) sm.xr[t] = T(0);
    for (int t = threadIdx.x; t < ring; t += blockDim.x) sm.tag[t] = -1;
    for (int t = threadIdx.x; t < kc; t += blockDim.x) sm.cdone[t] = -1;
    if (threadIdx.x == 0) { sm.ctr[0] = 0; sm.ctr[1] = 0; }
}

}  // namespace spt
