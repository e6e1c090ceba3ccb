// Device-side helpers shared by the sm_103a kernels of the SpTRSV library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sptrsv.h"

#define SPT_FULL_MASK 0xffffffffu

namespace spt {

// ---------------------------------------------------------------- status word
// The first error recorded wins; the host reads and clears it.
__device__ __forceinline__ void set_status(int *status, int code)
{
    atomicCAS(status, 0, code);
}

// ------------------------------------------------------------ bounds checks
// SPTRSV_CHECKED builds (a debug variant of the library, the stand-in for a
// memory checker): every index a solve gathers through must lie in
// [lo, hi); one outside is recorded as SPTRSV_ERANGE in the status word
// (when the kernel has one) and replaced by lo, so that the access it feeds
// stays inside its array.  The product build compiles the identity.
__device__ __forceinline__ int chk_index(int v, int lo, int hi, int *status)
{
#ifdef SPTRSV_CHECKED
    if (v < lo || v >= hi) {
        if (status) set_status(status, SPTRSV_ERANGE);
        return lo;
    }
#else
    (void)lo; (void)hi; (void)status;
#endif
    return v;
}

// -------------------------------------------------- memory-model primitives
// Ready flags are published with st.release.gpu after the solution values and
// polled with ld.acquire.gpu before the values are read (PTX memory model:
// the release/acquire pair orders the value stores before the loads).
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(int *p, int v)
{
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// CTA-scope release/acquire on shared memory (ring tags of the block mode).
__device__ __forceinline__ int ld_acquire_cta_smem(const int *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    int v;
    asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta_smem(int *p, int v)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("st.release.cta.shared.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// ------------------------------------------------------- shared mbarriers
// Phase-completion barriers in shared memory.  A waiter blocked in
// try_wait is suspended by the hardware until the phase completes (or a
// hardware time limit passes), so waiting warps do not take issue slots from
// the warps doing the work.
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Arrive with release semantics at CTA scope (orders this thread's earlier
// writes, and those ordered before it by __syncwarp, before the completion).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
// True once the phase of the given parity has completed (acquire, CTA scope).
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Read-only (for the whole kernel) matrix data: non-coherent path.
template <class T> __device__ __forceinline__ T ldro(const T *p) { return __ldg(p); }

// ------------------------------------------------------------- bounded waits
// Every wait in this library is bounded in time (%globaltimer, nanoseconds):
// after `limit_ns` it records SPTRSV_ETIMEOUT, raises the shared abort flag
// and returns false, so that all other waiters also leave instead of
// spinning on work that will never come.
struct Waiter {
    int *status;
    int *abort_flag;
    long long limit_ns;
};

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool aborted(const Waiter &w)
{
    return ld_relaxed(w.abort_flag) != 0;
}

__device__ __forceinline__ void give_up(const Waiter &w)
{
    set_status(w.status, SPTRSV_ETIMEOUT);
    st_relaxed(w.abort_flag, 1);
}

// Bounded-wait bookkeeping, cheap enough for tight shared-memory spins: the
// elapsed time comes from the SM-local clock64 (compared against the limit
// at 2.2 GHz, at or above the GB300 maximum SM clock, so the wall-time limit
// is never undercut by much), the global abort flag is read only every
// 4096 polls.
struct WaitClock {
    long long start = 0;
    unsigned polls = 0;
    __device__ __forceinline__ bool expired(const Waiter &w)
    {
        ++polls;
        if ((polls & 63u) != 0) return false;
        const long long t = clock64();
        if (start == 0) { start = t; return false; }
        if ((polls & 4095u) == 0 && aborted(w)) return true;
        if ((double)(t - start) > 2.2 * (double)w.limit_ns) { give_up(w); return true; }
        return false;
    }
};

// Bound for waits whose every poll may block in hardware (mbarrier
// try_wait): the clock is read at every poll, the abort flag every 64.
struct WaitClockEach {
    long long start = 0;
    unsigned polls = 0;
    __device__ __forceinline__ bool expired(const Waiter &w)
    {
        const long long t = clock64();
        if (start == 0) { start = t; return false; }
        if ((++polls & 63u) == 0 && aborted(w)) return true;
        if ((double)(t - start) > 2.2 * (double)w.limit_ns) { give_up(w); return true; }
        return false;
    }
};

// Wait for phase `parity` of a shared mbarrier, bounded.  Every lane of the
// warp calls it (no divergence around the wait); false on timeout / abort.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, const Waiter &w)
{
    if (mbar_try_wait(bar, parity)) return true;
    WaitClockEach clk;
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clk.expired(w)) return false;
    }
}

// Global-memory polls sleep 32 ns between attempts, so that thousands of
// waiting warps leave issue slots and L2 bandwidth to the producers.  The
// sleep is not lengthened.  Measured against a sleep doubling up to 512 ns:
// with value-carrying flags a hop is one L2 round trip, and the longer
// sleeps added their length to the hops of the hybrid solve, the automatic
// choice for such systems (lap2d 1024^2 FP64 4.24 -> 3.2 ms, power-law
// 116 -> 82 ms); the row-order synchronisation-free and level-persistent
// modes, whose waiters sit far ahead of the wavefront, lose about 20 % on
// the power-law DAG with the short sleep and gain a little on lap2d.
struct Backoff {
    __device__ __forceinline__ void pause() { __nanosleep(32); }
};

// Wait until flag == want.  Returns false on timeout / abort.
__device__ __forceinline__ bool wait_flag(const uint32_t *flag, uint32_t want, const Waiter &w)
{
    if (ld_acquire(flag) == want) return true;
    WaitClock clk;
    Backoff bo;
    for (;;) {
        if (ld_acquire(flag) == want) return true;
        if (clk.expired(w)) return false;
        bo.pause();
    }
}

// Wait until *counter >= target (64-bit monotone progress counter).
__device__ __forceinline__ bool wait_count(const unsigned long long *counter,
                                           unsigned long long target, const Waiter &w)
{
    if (ld_acquire_u64(counter) >= target) return true;
    WaitClock clk;
    Backoff bo;
    for (;;) {
        if (ld_acquire_u64(counter) >= target) return true;
        if (clk.expired(w)) return false;
        bo.pause();
    }
}

// ------------------------------------------------- value-carrying flags
// With one right-hand side a row's ready flag can carry the row's solution:
// the solve's epoch and the value's bits in one flag word, written once per
// solve.  A waiter has the value as soon as it sees the flag (one L2 round
// trip instead of two), and since nothing else is read through the flag,
// relaxed accesses suffice: the producer needs no release fence.  FP32: one
// 64-bit word {bits, epoch}.  FP64: two 64-bit halves {low bits, epoch} and
// {high bits, epoch}, each checked on its own, so that only the per-half
// single-copy atomicity of aligned 64-bit accesses is relied on.
__device__ __forceinline__ void vflag_publish(unsigned long long *f, int64_t i, float x, uint32_t epoch)
{
    const unsigned long long v = ((unsigned long long)epoch << 32) | __float_as_uint(x);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(f + i), "l"(v) : "memory");
}
__device__ __forceinline__ void vflag_publish(unsigned long long *f, int64_t i, double x, uint32_t epoch)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned long long lo = ((unsigned long long)epoch << 32) | (bits & 0xffffffffull);
    const unsigned long long hi = ((unsigned long long)epoch << 32) | (bits >> 32);
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(f + 2 * i), "l"(lo), "l"(hi) : "memory");
}
__device__ __forceinline__ bool vflag_try(const unsigned long long *f, int64_t j, uint32_t epoch, float &x)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(f + j) : "memory");
    x = __uint_as_float((uint32_t)v);
    return (uint32_t)(v >> 32) == epoch;
}
__device__ __forceinline__ bool vflag_try(const unsigned long long *f, int64_t j, uint32_t epoch, double &x)
{
    unsigned long long lo, hi;
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "l"(f + 2 * j) : "memory");
    x = __longlong_as_double((long long)((hi << 32) | (lo & 0xffffffffull)));
    return (uint32_t)(lo >> 32) == epoch && (uint32_t)(hi >> 32) == epoch;
}

// Wait until row j's value flag carries this solve's epoch; the value is
// returned in x.  Returns false on timeout / abort.
template <class T>
__device__ __forceinline__ bool wait_value(const unsigned long long *f, int64_t j, uint32_t epoch,
                                           const Waiter &w, T &x)
{
    if (vflag_try(f, j, epoch, x)) return true;
    WaitClock clk;
    Backoff bo;
    for (;;) {
        if (vflag_try(f, j, epoch, x)) return true;
        if (clk.expired(w)) return false;
        bo.pause();
    }
}

// ------------------------------------------------------------------ warp ops
template <class T> __device__ __forceinline__ T shfl_xor(T v, int m)
{
    return __shfl_xor_sync(SPT_FULL_MASK, v, m);
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace spt
