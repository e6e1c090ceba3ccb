// Allocation-free forward solve: sptrsv_solve_noalloc.
//
// Who needs it: callers that must not allocate device memory when they
// solve -- an application that hands the whole device memory budget to its
// own pool at start-up, a real-time loop where cudaMalloc's implicit
// device-wide synchronisation and unpredictable latency are not acceptable,
// or a plug-in whose host process forbids its modules to allocate.  The
// regular path needs a handle and a plan, both of which allocate (status
// word, ready flags, level schedule).  This entry point needs neither: its
// scratch -- one ready flag per row and a small control block -- lives in a
// statically allocated device array of this library.  The caller still
// passes the matrix, the right-hand sides and the output.
//
// The solve is the synchronisation-free forward substitution: warps take
// groups of 32 consecutive rows from a ticket; rows of the same group
// resolve through shared memory, earlier rows through their ready flags
// (ld.acquire / st.release), every wait bounded in time.
#include <cstddef>
#include <mutex>

#include "rows.cuh"

namespace {

using namespace spt;

struct NoallocCtl {
    unsigned long long ticket;
    unsigned long long epoch;
    int abort_flag;
    int status;
};

constexpr size_t kCtlBytes = 256;
constexpr size_t kScratchBytes = kCtlBytes + sizeof(uint32_t) * (size_t)SPTRSV_NOALLOC_MAX_ROWS;
constexpr long long kNoallocWaitNs = 10ll * 1000 * 1000 * 1000;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// The scratch of every call on this device: control block, then the flags.
// Zero at module load; flags never need clearing because each call tags them
// with a new epoch; the control block's ticket and error words are cleared
// by the first kernel of every call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__global__ void k_noalloc_begin(unsigned char *scratch)
{
    NoallocCtl *ctl = reinterpret_cast<NoallocCtl *>(scratch);
    ctl->ticket = 0ull;
    ctl->epoch = ctl->epoch + 1ull;
    ctl->abort_flag = 0;
    ctl->status = 0;
}

template <class T>
__global__ void __launch_bounds__(kThreads)
k_noalloc_syncfree(int32_t n, int64_t nnz, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                   const T *__restrict__ v, const T *b, T *x, int64_t ld, int32_t k,
                   unsigned char *scratch)
{
    __shared__ T xs_all[kThreads / 32][32];
    NoallocCtl *ctl = reinterpret_cast<NoallocCtl *>(scratch);
    uint32_t *flags = reinterpret_cast<uint32_t *>(scratch + kCtlBytes);
    const Waiter w{&ctl->status, &ctl->abort_flag, kNoallocWaitNs};
    const int lane = threadIdx.x & 31;
    volatile T *xs = xs_all[threadIdx.x >> 5];
    const uint32_t epoch = (uint32_t)ctl->epoch;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(&ctl->ticket, 1ull);
        c = __shfl_sync(SPT_FULL_MASK, c, 0);
        const int64_t base = (int64_t)c * 32;
        if (base >= n) return;
        const int i = (int)(base + lane);
        const bool valid = i < n;
        const int a = valid ? ldro(rp + i) : 0;
        const int e = valid ? ldro(rp + i + 1) - 1 : 0;
        // L is not validated here; the checks that keep every access of a
        // malformed row in bounds cost a few compares per row and one per
        // entry: row pointers outside [0, nnz] or decreasing, a row whose
        // last entry is not its diagonal (or that has none), and (below) a
        // column outside [0, i) before the diagonal, which is not lower
        // triangular and could also never complete
        int bad = 0;
        if (valid) {
            if (a < 0 || (int64_t)e >= nnz || e + 1 < a) bad = SPTRSV_EINVAL;
            else if (e < a || ldro(ci + e) != i) bad = SPTRSV_EDIAG;
        }
        if (__any_sync(SPT_FULL_MASK, bad != 0)) {
            if (bad) { set_status(&ctl->status, bad); st_relaxed(&ctl->abort_flag, 1); }
            return;
        }
        const unsigned rows = __ballot_sync(SPT_FULL_MASK, valid);
        for (int r = 0; r < k; ++r) {
            T acc = T(0);
            int p = a;
            unsigned fin = 0;
            bool failed = false;
            for (;;) {
                const bool open = valid && !((fin >> lane) & 1u);
                if (open) {
                    while (p < e) {
                        const int j = ldro(ci + p);
                        if (j < 0 || j >= i) {
                            set_status(&ctl->status, SPTRSV_ENOTLOWER);
                            st_relaxed(&ctl->abort_flag, 1);
                            failed = true;
                            break;
                        }
                        T xj;
                        if (j >= base) {
                            if (!((fin >> (j - base)) & 1u)) break;
                            xj = xs[j - base];
                        } else {
                            if (!wait_flag(flags + j, epoch, w)) { failed = true; break; }
                            xj = x[(int64_t)j * ld + r];
                        }
                        acc += ldro(v + p) * xj;
                        ++p;
                    }
                }
                if (__any_sync(SPT_FULL_MASK, failed)) return;
                const bool newly = open && p >= e;
                if (newly) {
                    const T xv = (b[(int64_t)i * ld + r] - acc) / ldro(v + e);
                    xs[lane] = xv;
                    x[(int64_t)i * ld + r] = xv;
                    if (r == k - 1) st_release(flags + i, epoch);
                }
                fin |= __ballot_sync(SPT_FULL_MASK, newly);
                __syncwarp();
                if ((fin & rows) == rows) break;
            }
        }
    }
}

// Per-device set-up: the device address of the scratch array (the host-side
// name is only a stand-in) and the persistent grid size.
struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;
    int grid = 0;
};

DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

cudaError_t setup_device(int dev, DeviceSetup **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &d = g_setup[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int sms = 0, per_sm = 0, per_sm32 = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_noalloc_syncfree<double>, kThreads, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, k_noalloc_syncfree<float>, kThreads, 0);
        if (e != cudaSuccess) return e;
        d.scratch = static_cast<unsigned char *>(ptr);
        d.grid = (per_sm < per_sm32 ? per_sm : per_sm32) * sms;
        if (d.grid < 1) d.grid = sms > 0 ? sms : 1;
        d.ready = true;
    }
    *out = &d;
    return cudaSuccess;
}

}  // namespace

extern "C" sptrsv_status sptrsv_solve_noalloc(const sptrsv_csr *L, const void *b, void *x,
                                              int32_t nrhs, int64_t ld, void *stream)
{
    if (!L || L->n < 0 || L->nnz < 0) return SPTRSV_EINVAL;
    if (L->n > SPTRSV_NOALLOC_MAX_ROWS) return SPTRSV_ENOTSUP;  // beyond the static scratch
    if (L->dtype != SPTRSV_F64 && L->dtype != SPTRSV_F32) return SPTRSV_EINVAL;
    if (L->n == 0) return SPTRSV_OK;
    if (!L->row_ptr || !L->col_idx || !L->vals || !b || !x || nrhs < 1 || ld < nrhs)
        return SPTRSV_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPTRSV_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return SPTRSV_ENOTSUP;
    DeviceSetup *d = nullptr;
    if (setup_device(dev, &d) != cudaSuccess) {
        cudaGetLastError();
        return SPTRSV_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t groups = ((int64_t)L->n + 31) / 32;
    int64_t grid = d->grid;
    const int64_t need = (groups + kThreads / 32 - 1) / (kThreads / 32);
    if (grid > need) grid = need;
    k_noalloc_begin<<<1, 1, 0, s>>>(d->scratch);
    if (L->dtype == SPTRSV_F64)
        k_noalloc_syncfree<double><<<(int)grid, kThreads, 0, s>>>(
            L->n, L->nnz, L->row_ptr, L->col_idx, (const double *)L->vals, (const double *)b, (double *)x, ld,
            nrhs, d->scratch);
    else
        k_noalloc_syncfree<float><<<(int)grid, kThreads, 0, s>>>(
            L->n, L->nnz, L->row_ptr, L->col_idx, (const float *)L->vals, (const float *)b, (float *)x, ld,
            nrhs, d->scratch);
    if (cudaGetLastError() != cudaSuccess) return SPTRSV_ECUDA;
    // wait for the solve and report a bounded wait that gave up
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, d->scratch + offsetof(NoallocCtl, status), sizeof(int),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SPTRSV_ECUDA;
    }
    return (sptrsv_status)status;
}
