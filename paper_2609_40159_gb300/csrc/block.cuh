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

template <class T, int KT>
__device__ __forceinline__ BlockSmem<T, KT> carve_block_smem(unsigned char *raw, int ring, int kc)
{
    BlockSmem<T, KT> sm;
    T *xr = reinterpret_cast<T *>(raw);
    sm.xr = xr;
    int *tag = reinterpret_cast<int *>(xr + (size_t)ring * KT);
    sm.tag = tag;
    sm.cdone = tag + ring;
    sm.ctr = tag + ring + kc;
    return sm;
}

template <class T, int KT>
__device__ __forceinline__ void reset_block_smem(const BlockSmem<T, KT> &sm, int ring, int kc)
{
    for (int t = threadIdx.x; t < ring; t += blockDim.x) sm.tag[t] = -1;
    for (int t = threadIdx.x; t < kc; t += blockDim.x) sm.cdone[t] = -1;
    if (threadIdx.x == 0) { sm.ctr[0] = 0; sm.ctr[1] = 0; }
}

}  // namespace spt
