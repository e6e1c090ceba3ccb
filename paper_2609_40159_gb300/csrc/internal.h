// Host-side interface between the C ABI layer (api.cu) and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "sptrsv.h"

namespace spt {

// Per-device launch facts.
struct DeviceInfo {
    int device = 0;
    int num_sms = 0;
    size_t max_smem_optin = 0;
};

// Device scratch owned by a handle: status word, abort flag, counters.
struct Ctl {
    int *status;        // first error
    int *abort_flag;    // raised by a wait that gave up
    unsigned long long *counters;  // [0] ticket, [1] progress, [2] epoch, [3] spare
};

// ------------------------------------------------------------------ prims.cu
// Exclusive scan of n int32 counts into out[0..n] (out[n] = total), int64
// accumulation; the total is also left in *total_dev (device) when non-null.
cudaError_t exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int64_t *total_dev,
                               cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs by key < 2^key_bits.
// Buffers: keys/vals in, keys_out/vals_out out; tmp arrays of the same sizes.
cudaError_t radix_sort_pairs(const uint32_t *keys, const int32_t *vals, uint32_t *keys_out,
                             int32_t *vals_out, int64_t n, int key_bits, cudaStream_t s);
// CSC of a CSR lower-triangular matrix with the CSR position of every entry.
cudaError_t build_csc(const int32_t *rp, const int32_t *ci, int32_t n, int64_t nnz, int32_t *cp,
                      int32_t *crow, int32_t *tmap, cudaStream_t s);
// Row index of every stored entry: entry_row[p] = i for row_ptr[i] <= p < row_ptr[i+1].
cudaError_t expand_rows(const int32_t *row_ptr, int32_t n, int32_t *entry_row, cudaStream_t s);

// ---------------------------------------------------------------- analyze.cu
// Validation: writes (first bad row, code) to *out_dev as row*16+code packed
// in an int64 (INT64_MAX when the matrix is valid).
cudaError_t launch_validate(const sptrsv_csr &L, long long *out_dev, cudaStream_t s);
// Levels (sync-free max-plus over the DAG).  lev must be pre-filled with -1.
// Levels of rows >= 32 * first_chunk (earlier rows must already hold theirs).
// withhold >= 0: test hook, that row's level is never published.
cudaError_t launch_levels(const sptrsv_csr &L, int32_t *lev, const Ctl &ctl,
                          long long limit_ns, const DeviceInfo &di, cudaStream_t s,
                          int64_t first_chunk = 0, int32_t withhold = -1);
// Levels after a change confined to rows >= first_row (lev: the levels before
// the change): fixpoint rounds in one cooperative launch (synchronises).
// *converged: the rounds reached the fixpoint; otherwise every row below
// *restart_row is final and the rest must be recomputed (launch_levels).
cudaError_t launch_levels_update(const sptrsv_csr &L, int32_t first_row, int32_t *lev, const Ctl &ctl,
                                 long long limit_ns, const DeviceInfo &di, cudaStream_t s, int max_rounds,
                                 int32_t withhold, bool *converged, int32_t *restart_row);
// Thin flags, fewest-dependency row per level, and (thin count, max rows in
// a thin level, max cost of a thin level) -> out_dev[0..2].
cudaError_t launch_level_summary(const int32_t *rp, const int32_t *perm, const int32_t *level_ptr,
                                 const int64_t *cost, int32_t nlevels, double threshold, uint8_t *thin,
                                 int32_t *pick, unsigned long long *out_dev, cudaStream_t s);
// Number of rows with more than min_offdiag off-diagonals -> *out_dev.
cudaError_t launch_count_long(const int32_t *rp, int32_t n, int32_t min_offdiag,
                              unsigned long long *out_dev, cudaStream_t s);
// Level of every row -> max level (nlevels-1) in *maxlev_dev.
cudaError_t launch_max(const int32_t *lev, int32_t n, int32_t *maxlev_dev, cudaStream_t s);
// Histogram of rows and costs per level; counts[nlevels], cost[nlevels].
cudaError_t launch_level_hist(const sptrsv_csr &L, const int32_t *lev, int32_t nlevels,
                              int32_t *counts, int64_t *cost, cudaStream_t s);
// Stats of the level table; writes 6 doubles to stats_dev.
cudaError_t launch_level_stats(int32_t n, int64_t nnz, int32_t nlevels, const int32_t *level_ptr,
                               const int64_t *cost, double *stats_dev, cudaStream_t s);
// Full partition (perm, level_ptr, cost) given lev and nlevels.
cudaError_t level_partition(const sptrsv_csr &L, const int32_t *lev, int32_t nlevels,
                            int32_t *perm, int32_t *level_ptr, int64_t *cost, cudaStream_t s);

// --------------------------------------------------------------- rewrite.cu
int rewrite_run(const sptrsv_csr &L, const int32_t *lev, const int32_t *rows,
                const int32_t *targets, int32_t nrows, int64_t *nnz_Lp, int64_t *nnz_T,
                sptrsv_csr_out *Lp_out, sptrsv_csr_out *T_out, const DeviceInfo &di,
                cudaStream_t s);

}  // namespace spt
