// Row views of a system for the solve kernels: the forward solve reads L by
// rows (CSR), the transpose solve reads L by columns (CSC, values gathered
// into CSC order before the solve).
#pragma once

#include "solve.cuh"

namespace spt {

// ------------------------------------------------------------- row views
template <class T, bool TR> struct RV;

// (chk_*: identity in the product build, bounds checks in SPTRSV_CHECKED)
template <class T> __device__ __forceinline__ int chk_row(const Sys<T> &A, int i)
{
    return chk_index(i, 0, A.n, A.chk);
}
template <class T> __device__ __forceinline__ int chk_pos(const Sys<T> &A, int p)
{
    return chk_index(p, 0, (int)A.nnz, A.chk);
}

template <class T> struct RV<T, false> {
    static __device__ __forceinline__ int beg(const Sys<T> &A, int i) { return ldro(A.rp + chk_row(A, i)); }
    static __device__ __forceinline__ int end(const Sys<T> &A, int i) { return ldro(A.rp + chk_row(A, i) + 1) - 1; }
    static __device__ __forceinline__ T diag(const Sys<T> &A, int, int e) { return ldro(A.v + chk_pos(A, e)); }
    static __device__ __forceinline__ int col(const Sys<T> &A, int p) { return chk_row(A, ldro(A.ci + chk_pos(A, p))); }
    static __device__ __forceinline__ T val(const Sys<T> &A, int p) { return ldro(A.v + chk_pos(A, p)); }
};

template <class T> struct RV<T, true> {
    static __device__ __forceinline__ int beg(const Sys<T> &A, int i) { return ldro(A.cp + chk_row(A, i)) + 1; }
    static __device__ __forceinline__ int end(const Sys<T> &A, int i) { return ldro(A.cp + chk_row(A, i) + 1); }
    static __device__ __forceinline__ T diag(const Sys<T> &A, int b, int) { return ldro(A.cv + chk_pos(A, b - 1)); }
    static __device__ __forceinline__ int col(const Sys<T> &A, int q) { return chk_row(A, ldro(A.crow + chk_pos(A, q))); }
    static __device__ __forceinline__ T val(const Sys<T> &A, int q) { return ldro(A.cv + chk_pos(A, q)); }
};

// Column of entry p of T (the rewritten right-hand side's extra terms).
template <class T> __device__ __forceinline__ int tcol(const Sys<T> &A, int p)
{
    return chk_row(A, ldro(A.tci + p));
}

template <class T>
__device__ __forceinline__ bool has_trow(const Sys<T> &A, int i)
{
    return A.tmask != nullptr && ((ldro(A.tmask + (i >> 5)) >> (i & 31)) & 1u);
}

// Position of a row in processing order (forward: i, transpose: n-1-i).
template <bool TR> __device__ __forceinline__ int order_pos(int n, int i) { return TR ? n - 1 - i : i; }

// Make a loaded value "used" here: the load must complete before this
// point, so that a warp waiting for its turn holds all of its operands
// instead of stalling on them after the turn comes.
__device__ __forceinline__ void consume(int v) { asm volatile("" ::"r"(v)); }
__device__ __forceinline__ void consume(float v) { asm volatile("" ::"f"(v)); }
__device__ __forceinline__ void consume(double v) { asm volatile("" ::"d"(v)); }

// Prefetch into L2 the first line of a row's entries (indices and values).
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <class T, bool TR>
__device__ __forceinline__ void prefetch_row(const Sys<T> &A, int i)
{
    if (!TR) {
        const int a = ldro(A.rp + i);
        prefetch_l2(A.ci + a);
        prefetch_l2(A.v + a);
    } else {
        const int a = ldro(A.cp + i);
        prefetch_l2(A.crow + a);
        prefetch_l2(A.cv + a);
    }
}

template <class T, int KT>
__device__ __forceinline__ void group_reduce(T (&acc)[KT], int lpr)
{
    for (int o = lpr >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < KT; ++r) acc[r] += shfl_xor(acc[r], o);
}

// Column sweep over the dependencies INSIDE a group of 32 rows (one row per
// lane, in processing order).  dmask: bit s is set when this lane's row
// depends on row s of the group; coef[s*32 + lane] holds that coefficient
// (per-warp table).  Steps visit only rows that some lane depends on: lane s
// forms its solution candidate (b - acc) / L_ii -- final, since all of its
// own in-group dependencies are earlier rows -- and broadcasts it (warp
// shuffles for up to 4 right-hand sides, a per-warp shared buffer for more);
// every lane that depends on row s adds coef * x_s.
template <class T, int KT>
__device__ __forceinline__ void group_sweep(unsigned dmask, const T *coef, T *xbuf, T (&acc)[KT],
                                            const T (&bv)[KT], T rinv)
{
    const int lane = threadIdx.x & 31;
    unsigned need = __reduce_or_sync(0xffffffffu, dmask);
    while (need) {
        const int s = __ffs(need) - 1;
        need &= need - 1;
        const bool hit = (dmask >> s) & 1u;
        const T c = hit ? coef[s * 32 + lane] : T(0);
        if (KT <= 4) {
#pragma unroll
            for (int r = 0; r < KT; ++r) {
                const T t = (bv[r] - acc[r]) * rinv;
                const T xs = __shfl_sync(0xffffffffu, t, s);
                if (hit) acc[r] += c * xs;
            }
        } else {
            if (lane == s) {
#pragma unroll
                for (int r = 0; r < KT; ++r) xbuf[r] = (bv[r] - acc[r]) * rinv;
            }
            __syncwarp();
            if (hit) {
#pragma unroll
                for (int r = 0; r < KT; ++r) acc[r] += c * xbuf[r];
            }
            __syncwarp();
        }
    }
}

}  // namespace spt
