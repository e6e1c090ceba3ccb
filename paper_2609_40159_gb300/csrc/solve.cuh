// Solve-side data views and launchers (forward solve, transpose solve,
// value gradient, T application) shared by solve.cu, batch.cu and api.cu.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace spt {

// A lower-triangular system as the kernels see it.
template <class T> struct Sys {
    int32_t n;
    const int32_t *rp;    // CSR of L
    const int32_t *ci;
    const T *v;
    const int32_t *cp;    // CSC of L (transpose solve): column pointers,
    const int32_t *crow;  //   row of every CSC entry (diagonal first),
    const int32_t *tmap;  //   CSR position of every CSC entry,
    const T *cv;          //   value of every CSC entry (v[tmap[q]], gathered
                          //   before each transpose solve)
    const int32_t *trp;   // T of a rewritten system (rows with entries only)
    const int32_t *tci;
    const T *tv;
    const uint32_t *tmask;  // bit i set when row i has a T row; null = no T
    const int32_t *tcp;     // CSC of T (adjoint of b + T b): column pointers,
    const int32_t *trow;    //   row of every CSC entry (ascending),
    const int32_t *ttmap;   //   CSR position of every CSC entry
    int64_t nnz;            // entries of L (bounds of the checked build)
    int *chk;               // status word of the checked build's bounds checks
};

// Level schedule.
struct Sched {
    const int32_t *perm;
    const int32_t *level_ptr;
    int32_t nlevels;
    const int32_t *chunk_level;  // level of the first row of every row group
    int64_t nchunks;
    // hybrid schedule (null: every level waits for all earlier levels):
    // seg[l] = first level (in processing order) of the run of thin levels
    // that holds level l (l itself for a thick level); lev = row levels
    const int32_t *seg;
    const int32_t *lev;
};

template <class T> struct Rhs {
    const T *b;
    T *x;
    int64_t ld;
    int32_t k;
};

// Per-plan device control block.
struct PlanCtl {
    unsigned long long ticket;
    unsigned long long progress;
    unsigned long long epoch;
    unsigned long long spare;
    int abort_flag;
    int pad[3];
};

struct SyncArgs {
    uint32_t *flags;
    PlanCtl *ctl;
    int32_t withhold;
    Waiter w;
    // value-carrying flags (16 bytes per row), used instead of flags + x
    // when the solve has one right-hand side; nullptr otherwise
    unsigned long long *vflags = nullptr;
};

// ---------------------------------------------------------------- launchers
// All return cudaSuccess or the launch error; T = double or float.
template <class T>
cudaError_t launch_prologue(PlanCtl *ctl, cudaStream_t s);

template <class T>
cudaError_t solve_level_launch(const Sys<T> &A, const int32_t *perm,
                               const std::vector<int32_t> &h_level_ptr, const Rhs<T> &R,
                               bool trans, cudaStream_t s);

template <class T>
cudaError_t solve_level_persistent(const Sys<T> &A, const Sched &S, const Rhs<T> &R, int rpw,
                                   int kt, bool trans, const SyncArgs &sy, int grid,
                                   cudaStream_t s);

template <class T>
cudaError_t solve_syncfree(const Sys<T> &A, const Rhs<T> &R, int rpw, int kt, bool trans,
                           const SyncArgs &sy, int grid, cudaStream_t s);

template <class T>
cudaError_t solve_block(const Sys<T> &A, const Rhs<T> &R, int rpw, int kt, bool trans,
                        const SyncArgs &sy, int nwarps, cudaStream_t s);

template <class T>
cudaError_t grad_vals(const Sys<T> &A, const T *gb, const T *x, int64_t ld, int32_t k, T *gv,
                      cudaStream_t s);

template <class T>
cudaError_t tt_apply(const Sys<T> &A, const T *gbp, T *gb, int64_t ld, int32_t k,
                     cudaStream_t s);

cudaError_t build_tmask(const int32_t *trp, int32_t n, uint32_t *tmask, cudaStream_t s);
cudaError_t build_chunk_levels(const int32_t *level_ptr, int32_t nlevels, int32_t n, int rpw,
                               bool trans, int32_t *chunk_level, cudaStream_t s);

// Occupancy-derived persistent grid sizes.
int persistent_grid_level(int kt, bool f64, const DeviceInfo &di);
int persistent_grid_syncfree(int kt, bool f64, const DeviceInfo &di);
// Block mode: whether (k, dtype) fits the shared-memory ring.
bool block_mode_supported(int k, bool f64);
int block_kt_for(int k);
// Ring geometry of the block mode for `nwarps` active warps: kc row groups in
// the ring, throttle distance P.
// Ring length kc (row groups, a power of two >= 2 (nwarps + 2)) and
// throttle distance P of the block algorithm; the ring grows while the
// block's shared memory stays within grow_limit bytes.
void block_geometry(int rpw, int kt, bool f64, int nwarps, int *kc, int *P, size_t grow_limit);
// Active warps of the block mode for a system with the given level width.
int block_warps_for(double rows_per_level, int rpw);
size_t block_smem_bytes(int rpw, int kt, int kc, bool f64, int nw);
// Most warps of a block-mode thread block that work on one system.
constexpr int kMaxBlockWarps = 8;
// Batched solve: warps per thread block and the minimum number of resident
// blocks per SM the kernel is compiled for (0 = no register constraint).
constexpr int kBatchWarps = 4;
constexpr int kBatchMinBlocks = 0;
// Shared memory a batched work item may grow its ring to: several items per
// SM (each a latency-bound chain) beat longer rings.
constexpr size_t kBatchSmemGrow = 48 * 1024;
constexpr size_t kBlockSmemBudget = 200 * 1024;

// ---------------------------------------------------------------- batched
// Up to 32 rows of one level, in the processing order of one direction
// (forward: level order; transpose: its reverse).  Positions [base,
// base+cnt) of that order; the group's level ends at position lend; wait =
// number of groups of the levels before it in that order (the group may
// start once that many groups are complete).
struct LevelGroup {
    int32_t base, cnt, lend, wait;
};

// Per-matrix descriptor of a batched plan (device resident).
struct BatchMat {
    int32_t n;
    int32_t k;        // right-hand sides (leading dimension of its blocks)
    int64_t nnz;
    const int32_t *rp, *ci;
    const void *v;
    const int32_t *cp, *crow, *tmap;
    void *cv;  // CSC values, gathered before each transpose solve
    const int32_t *trp, *tci;
    const void *tv;
    const uint32_t *tmask;
    const int32_t *tcp, *trow, *ttmap;  // CSC of T
    int64_t rhs_off;   // element offset of the [n x k] block in packed buffers
    int64_t vals_off;  // element offset of the nnz values in packed gradients
    int64_t row_off;   // first global row of the matrix
    // level-ordered schedule (set once a direction of the system uses it):
    // rows in level order, the inverse permutation, and per direction the
    // row groups of that order (transpose: levels from the last to the first)
    const int32_t *perm, *iperm;
    const LevelGroup *lgroups[2];
    int32_t nlgroups[2];
};

// Schedules of a batched work item.
constexpr int32_t kSchedInOrder = 0;  // row groups in row order, completed one after another
constexpr int32_t kSchedLevel = 1;    // row groups of one level, levels one after another

// Work item of a batched solve: the columns [r0, r0+kt) of one system's
// right-hand sides (the columns are independent problems, so a system with
// many right-hand sides becomes several items solved by different blocks).
struct BatchItem {
    int32_t mat;
    int32_t r0;
    int32_t kt;       // columns of this item
    int32_t KT;       // register tile (power of two >= kt)
    int32_t rpw;      // rows per warp
    int32_t kc;       // ring row groups (block mode)
    int32_t P;        // throttle distance in row groups
    int32_t nw;       // active warps of the thread block
    int32_t sched;    // kSchedInOrder or kSchedLevel
};

// 32 consecutive rows (fewer at a system's end) of one system of a batch.
struct RowChunk {
    int32_t mat;
    int32_t r0;  // a multiple of 32
};

// One persistent launch: thread blocks take work items in `order` from the
// control block's ticket and solve each with the block algorithm; trace
// receives (start ns, end ns, SM) per item.  Forward solves of batches with
// rewritten systems first form bt = b + T b on every 32-row chunk of those
// systems (fchunks, nfchunks; bt: plan-owned, packed like b) and the solve
// reads bt for them.
template <class T>
cudaError_t batch_solve(const BatchMat *mats, const BatchItem *items, int32_t nitems,
                        const int32_t *order, const T *b, T *x, bool trans, PlanCtl *ctl,
                        const Waiter &w, int grid, size_t smem, long long *trace, int withhold,
                        const RowChunk *fchunks, int64_t nfchunks, T *bt, cudaStream_t s);
// cv[q] = v[tmap[q]]: the values of L in CSC order, so that the transpose
// solves read them without the indirection (refreshed before every
// transpose solve: the plan does not assume that L's values stay fixed).
template <class T>
cudaError_t csc_values(const int32_t *tmap, const T *v, T *cv, int64_t nnz, cudaStream_t s);
// Tiles: (system, first CSC entry) of kCscTile entries each, every system
// with a CSC, in system order.
constexpr int kCscTile = 4096;
template <class T>
cudaError_t batch_csc_values(const BatchMat *mats, const RowChunk *tiles, int64_t ntiles, cudaStream_t s);

// Value gradients of all matrices; chunks covers every row of every system
// (device table of nchunks entries).
template <class T>
cudaError_t batch_grad_vals(const BatchMat *mats, const RowChunk *chunks, int64_t nchunks, const T *gb,
                            const T *x, T *gv, cudaStream_t s);
// gb = gbp + T^T gbp for every rewritten matrix (packed buffers); tchunks
// lists the chunks that hold at least one column of T (rows of gb that
// receive a T^T term).
template <class T>
cudaError_t batch_tt_apply(const BatchMat *mats, const RowChunk *tchunks, int64_t ntchunks,
                           int64_t total_rhs, const T *gbp, T *gb, cudaStream_t s);
int batch_grid(size_t smem, const DeviceInfo &di);
// dst[c * ldd + r] = src[r * lds + c] for r < rows, c < cols (32 x 32
// tiles through shared memory: both sides read and written along rows).
template <class T>
cudaError_t transpose_dense(const T *src, int64_t lds, T *dst, int64_t ldd, int64_t rows, int64_t cols,
                            cudaStream_t s);
// iperm[perm[q]] = q for q < n.
cudaError_t inverse_perm(const int32_t *perm, int32_t *iperm, int32_t n, cudaStream_t s);

}  // namespace spt
