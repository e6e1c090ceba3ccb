// Row views of a system for the solve kernels: the forward solve reads L by
// rows (CSR), the transpose solve reads L by columns (CSC + value map).
#pragma once

#include "solve.cuh"

namespace spt {

// ------------------------------------------------------------- row views
template <class T, bool TR> struct RV;

template <class T> struct RV<T, false> {
    static __device__ __forceinline__ int beg(const Sys<T> &A, int i) { return ldro(A.rp + i); }
    static __device__ __forceinline__ int end(const Sys<T> &A, int i) { return ldro(A.rp + i + 1) - 1; }
    static __device__ __forceinline__ T diag(const Sys<T> &A, int, int e) { return ldro(A.v + e); }
    static __device__ __forceinline__ int col(const Sys<T> &A, int p) { return ldro(A.ci + p); }
    static __device__ __forceinline__ T val(const Sys<T> &A, int p) { return ldro(A.v + p); }
};

template <class T> struct RV<T, true> {
    static __device__ __forceinline__ int beg(const Sys<T> &A, int i) { return ldro(A.cp + i) + 1; }
    static __device__ __forceinline__ int end(const Sys<T> &A, int i) { return ldro(A.cp + i + 1); }
    static __device__ __forceinline__ T diag(const Sys<T> &A, int b, int) { return ldro(A.v + ldro(A.tmap + b - 1)); }
    static __device__ __forceinline__ int col(const Sys<T> &A, int q) { return ldro(A.crow + q); }
    static __device__ __forceinline__ T val(const Sys<T> &A, int q) { return ldro(A.v + ldro(A.tmap + q)); }
};

template <class T>
__device__ __forceinline__ bool has_trow(const Sys<T> &A, int i)
{
    return A.tmask != nullptr && ((ldro(A.tmask + (i >> 5)) >> (i & 31)) & 1u);
}

// Position of a row in processing order (forward: i, transpose: n-1-i).
template <bool TR> __device__ __forceinline__ int order_pos(int n, int i) { return TR ? n - 1 - i : i; }

template <class T, int KT>
__device__ __forceinline__ void group_reduce(T (&acc)[KT], int lpr)
{
    for (int o = lpr >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < KT; ++r) acc[r] += shfl_xor(acc[r], o);
}

}  // namespace spt
