/*
 * sptrsv.h -- C ABI of the GB300 (sm_103a) sparse triangular solve library.
 *
 * The operations follow the paper "Reinforcement Learning-Guided Graph
 * Transformations for SpTRSV Optimization":
 *   - Section 2.1: the sparse triangular solve L x = b, where every row is a
 *     node of the dependency DAG and every off-diagonal L[i][j] an edge j -> i;
 *     the level-set method partitions the DAG into levels of independent rows.
 *   - Section 2.2: equation rewriting, a preprocessing step that replaces a
 *     row's dependencies by their predecessors so that it moves to an earlier
 *     level; the result is again a CSR lower-triangular system fed to an
 *     unchanged level-set solver.
 *   - Section 4.1 and Tables 4-5: level costs, ALC / ARL / AIR, the coefficient
 *     of variation of level costs and row counts and the thin-level threshold.
 *   - Related work (synchronisation-free solves): rows start as soon as their
 *     own predecessors are done, with lightweight flags instead of barriers.
 *
 * Conventions for every call:
 *   - A matrix is CSR with int32 row_ptr[n+1] and col_idx[nnz]; columns of a
 *     row strictly increase, all are < i except the last, which is the
 *     diagonal i; the diagonal is non-zero.  Values are FP64 or FP32.
 *   - Array arguments are DEVICE pointers owned by the caller unless stated
 *     otherwise; the library never frees them.  Host scalars/outputs are
 *     marked "(host)".
 *   - Dense right-hand sides and solutions are [n x nrhs] row-major with
 *     leading dimension ld >= nrhs (elements), in the matrix's value type.
 *   - Every call returns a status code and never throws.  Work is enqueued on
 *     the handle's stream; calls return before the GPU finishes unless they
 *     say they synchronise.  Faults found by the GPU (e.g. a bounded wait that
 *     gave up) are recorded in a device status word and returned by
 *     sptrsv_get_status().
 *   - A plan keeps pointers to the caller's matrix arrays; they must stay
 *     valid and unmodified in structure for the plan's lifetime (values may
 *     change between solves).
 */
#ifndef SPTRSV_GB300_H
#define SPTRSV_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPTRSV_OK = 0,
    SPTRSV_EINVAL = 1,     /* bad argument (null pointer, size, row index)   */
    SPTRSV_ENOTLOWER = 2,  /* a column > i, or < 0                           */
    SPTRSV_EDIAG = 3,      /* diagonal missing, not last, or zero            */
    SPTRSV_EUNSORTED = 4,  /* columns of a row not strictly increasing       */
    SPTRSV_ETARGET = 5,    /* rewrite target t < 0 or t >= lev(i), lev(i)==0 */
    SPTRSV_ENOMEM = 6,     /* device allocation failed                       */
    SPTRSV_ETIMEOUT = 7,   /* a bounded device wait gave up                  */
    SPTRSV_ECUDA = 8,      /* a CUDA runtime call failed                     */
    SPTRSV_ENOTSUP = 9,    /* option not supported for this input            */
    SPTRSV_ERANGE = 10     /* an index out of its array's range, found by the
                              bounds checks of an SPTRSV_CHECKED build       */
} sptrsv_status;

typedef enum { SPTRSV_F64 = 0, SPTRSV_F32 = 1 } sptrsv_dtype;

/* Matrix descriptor (device pointers, caller-owned). */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const void *vals;
    sptrsv_dtype dtype;
} sptrsv_csr;

/* Writable descriptor used for rewrite outputs (device pointers). */
typedef struct {
    int32_t *row_ptr;  /* n+1 */
    int32_t *col_idx;  /* nnz */
    void *vals;        /* nnz, same dtype as the input */
} sptrsv_csr_out;

typedef enum {
    SPTRSV_MODE_AUTO = 0,
    /* Plain level-set solve (Section 2.1): one kernel launch per level,
     * one thread per row.  This is the baseline the other modes must beat. */
    SPTRSV_MODE_LEVEL_LAUNCH = 1,
    /* Level-set solve in ONE persistent launch: warps take row groups in
     * level order and wait on a grid-wide progress counter for the previous
     * level instead of a launch boundary.                                    */
    SPTRSV_MODE_LEVEL_PERSISTENT = 2,
    /* Synchronisation-free solve: row groups taken in row order, each row
     * waits on its own predecessors' ready flags (acquire/release).          */
    SPTRSV_MODE_SYNCFREE = 3,
    /* Synchronisation-free solve inside one thread block: flags and recent
     * solution values live in shared memory; for deep, narrow systems where
     * the cross-SM flag round trip would dominate.                           */
    SPTRSV_MODE_BLOCK = 4,
    /* Hybrid of the level-set and synchronisation-free schedules (Section 7,
     * related work): rows in level order as in LEVEL_PERSISTENT; a thick
     * level waits for every earlier level, a maximal run of consecutive thin
     * levels (fewer rows than the plan's thin_rows) waits once for the rows
     * before the run, and inside the run each row waits only for its own
     * predecessors' ready flags.                                             */
    SPTRSV_MODE_HYBRID = 5
} sptrsv_mode;

typedef struct {
    int32_t mode;            /* sptrsv_mode; AUTO picks from the level profile */
    int32_t rows_per_warp;   /* 1,2,4,8,16,32 (lanes per row = 32/rows_per_warp); 0 = auto */
    int32_t rhs_tile;        /* right-hand sides per pass: 1,2,4,8,16; 0 = auto.
                                Block mode and batched plans: columns per
                                thread block (1,2,4,8); wider right-hand
                                sides run as independent column tiles      */
    int32_t build_transpose; /* non-zero: prepare sptrsv_solve_transpose / grad  */
    int64_t wait_limit_us;   /* longest a device wait may take before the solve
                                gives up with SPTRSV_ETIMEOUT (microseconds);
                                0 = default (10 s)                            */
} sptrsv_plan_opts;

typedef struct sptrsv_handle_st *sptrsv_handle;
typedef struct sptrsv_plan_st *sptrsv_plan;

/* ------------------------------------------------------------------ handle */
/* Creates a handle bound to the current CUDA device and to `stream` (a
 * cudaStream_t; NULL = the legacy default stream).                         */
sptrsv_status sptrsv_create(sptrsv_handle *handle, void *stream);
sptrsv_status sptrsv_destroy(sptrsv_handle handle);
sptrsv_status sptrsv_set_stream(sptrsv_handle handle, void *stream);
/* Synchronises the stream, returns the first error any kernel recorded since
 * the last call (SPTRSV_OK if none) and clears it.                          */
sptrsv_status sptrsv_get_status(sptrsv_handle handle);
const char *sptrsv_status_string(sptrsv_status status);

/* ---------------------------------------------------------------- validate */
/* Checks that L is a lower-triangular CSR with sorted columns and a non-zero
 * diagonal stored last (Section 2.1).  Synchronises.  On failure returns the
 * code of the first offending row in row order and writes that row to
 * *bad_row (host, may be NULL).                                             */
sptrsv_status sptrsv_validate(sptrsv_handle handle, const sptrsv_csr *L, int32_t *bad_row);

/* ----------------------------------------------------------------- analyze */
/* Level-set analysis of L (Section 2.1; level table and costs of Section 4.1):
 *   lev[i]        level of row i: 0 without off-diagonals, else
 *                 1 + max over predecessors (longest path from a source);
 *   perm[n]       rows sorted by (level, row);
 *   level_ptr[]   level l occupies perm[level_ptr[l] .. level_ptr[l+1]);
 *                 caller allocates n+1 entries (worst case);
 *   level_cost[]  sum over the level's rows of 2*offdiag(i)+1 (int64);
 *                 caller allocates n entries (worst case);
 *   *nlevels      (host) number of levels;
 *   stats[6]      (host) ALC, ARL, AIR, CV of level costs, CV of rows per
 *                 level (population), thin threshold ALC*(1+max(0,1-CV)).
 * Validates L first (codes as sptrsv_validate).  Synchronises.              */
sptrsv_status sptrsv_analyze(sptrsv_handle handle, const sptrsv_csr *L, int32_t *lev,
                             int32_t *perm, int32_t *level_ptr, int64_t *level_cost,
                             int32_t *nlevels, double stats[6]);

/* The same analysis after a change confined to rows >= first_row (e.g. a
 * rewrite whose rewritten rows are all >= first_row, Section 2.2: rewriting
 * row i changes row i only, so every earlier row keeps its level).  lev is
 * in/out: on entry it must hold the levels of the matrix BEFORE the change
 * (e.g. from sptrsv_analyze of that matrix); only levels that the change
 * actually moves are recomputed: rounds over the rows >= first_row, the
 * first recomputing all of them, each later one only the rows with a
 * predecessor changed in the round before, until a round changes nothing
 * (one launch, the environment step of the paper's Section 4.1: a rewrite
 * usually moves one row).  A change that propagates through more than 32
 * rounds (a level that empties renumbers every later level), or that moves
 * more than 1024 rows in one round (a bulk rewrite), is finished by the
 * full sync-free pass from its first unsettled row.  Then perm,
 * level_ptr, level_cost, *nlevels and stats as sptrsv_analyze.  first_row
 * outside [0, n] is SPTRSV_EINVAL; first_row = 0 is sptrsv_analyze.  The
 * results equal sptrsv_analyze's when the entry levels are right; wrong
 * entry levels are not detected.  Synchronises.                             */
sptrsv_status sptrsv_analyze_incremental(sptrsv_handle handle, const sptrsv_csr *L, int32_t first_row,
                                         int32_t *lev, int32_t *perm, int32_t *level_ptr,
                                         int64_t *level_cost, int32_t *nlevels, double stats[6]);

/* What the paper's environment observes after each rewrite (Section 4.1:
 * thin levels; Section 4.3: the node a move takes from a level is the one
 * with the fewest dependencies), from an analysis of L:
 *   perm, level_ptr, level_cost, nlevels  as returned by sptrsv_analyze
 *                 (device arrays);
 *   threshold     thin-level threshold (e.g. stats[5] of sptrsv_analyze);
 *   thin[l]       (device, nlevels bytes) 1 when level_cost[l] < threshold
 *                 (compared in double), else 0;
 *   pick[l]       (device, nlevels entries) the row of level l with the
 *                 fewest off-diagonals, the smallest row among equals;
 *   summary[3]    (host) number of thin levels, largest row count of a thin
 *                 level, largest cost of a thin level (0 without thin levels).
 * SPTRSV_EINVAL for missing arrays or nlevels < 0.  Synchronises.           */
sptrsv_status sptrsv_level_summary(sptrsv_handle handle, const sptrsv_csr *L, const int32_t *perm,
                                   const int32_t *level_ptr, const int64_t *level_cost, int32_t nlevels,
                                   double threshold, uint8_t *thin, int32_t *pick, int64_t summary[3]);

/* At = A^T for a square CSR matrix A (n x n): At->row_ptr (n+1),
 * At->col_idx and At->vals (nnz each, A's dtype) are caller-allocated
 * device arrays; columns come out strictly increasing inside every row.
 * The transpose of an upper-triangular matrix U whose rows store the
 * diagonal first is a lower-triangular matrix in this library's layout, so
 * U x = b is solved as the transpose solve of a plan for U^T (the paper's
 * preconditioner use needs both triangles).  Validates nothing beyond the
 * pointers (validate the result).  Synchronises.                           */
sptrsv_status sptrsv_transpose(sptrsv_handle handle, const sptrsv_csr *A, sptrsv_csr_out *At);

/* ----------------------------------------------------------------- rewrite */
/* Equation rewriting (Section 2.2) by row substitution.  rows[q] (device,
 * nrows entries) is rewritten towards target level targets[q] (device; NULL
 * means lev(i)-1): every predecessor j with lev(j) >= t is replaced, largest
 * column first, by row j's own predecessors with coefficients scaled by
 * m = acc[j] / L_jj, using the ORIGINAL rows and the ORIGINAL levels `lev`
 * (device, from sptrsv_analyze).  The result is L' (same n) and T (n rows,
 * no diagonal) with L' x = b + T b.  A row listed twice keeps its smallest
 * target.  Two-phase: with Lp_out == NULL the call only computes the sizes
 * (*nnz_Lp, *nnz_T, host); call again with buffers of those sizes.  Both
 * phases synchronise.  Errors: SPTRSV_EINVAL for a row outside [0, n),
 * SPTRSV_ETARGET for a target outside [0, lev(i)) or lev(i) == 0.           */
sptrsv_status sptrsv_rewrite(sptrsv_handle handle, const sptrsv_csr *L, const int32_t *lev,
                             const int32_t *rows, const int32_t *targets, int32_t nrows,
                             int64_t *nnz_Lp, int64_t *nnz_T,
                             sptrsv_csr_out *Lp_out, sptrsv_csr_out *T_out);

/* ------------------------------------------------------------------- solve */
/* Builds a reusable solve plan for L (and, for a rewritten system, T: the
 * solve then computes x = L^{-1} (b + T b), the T gather fused into the rows
 * that have one).  Runs the level analysis internally and synchronises.
 * opts may be NULL (defaults).                                              */
sptrsv_status sptrsv_plan_create(sptrsv_handle handle, const sptrsv_csr *L, const sptrsv_csr *T,
                                 const sptrsv_plan_opts *opts, sptrsv_plan *plan);
sptrsv_status sptrsv_plan_destroy(sptrsv_plan plan);
/* (host outputs, each may be NULL) number of levels of the plan's schedule,
 * the mode, rows per warp and rhs tile the plan uses.                       */
sptrsv_status sptrsv_plan_info(sptrsv_plan plan, int32_t *nlevels, int32_t *mode,
                               int32_t *rows_per_warp, int32_t *rhs_tile);
/* Changes the mode / rows per warp / rhs tile of an existing plan (used by
 * the autotuner); builds whatever schedule data the new mode needs.         */
sptrsv_status sptrsv_plan_set(sptrsv_plan plan, int32_t mode, int32_t rows_per_warp,
                              int32_t rhs_tile);

/* x = L^{-1} b  (or L^{-1} (b + T b)).  Asynchronous.  b and x must not
 * overlap.                                                                  */
sptrsv_status sptrsv_solve(sptrsv_plan plan, const void *b, void *x, int32_t nrhs, int64_t ld);

/* Adjoint of the solve: g_b = L^{-T} g_x, processed in reverse level /
 * reverse row order.  Requires build_transpose.  Asynchronous.  First
 * gathers L's current values into CSC order (one elementwise launch, plan-
 * owned buffer), so values may change between calls.                      */
sptrsv_status sptrsv_solve_transpose(sptrsv_plan plan, const void *gx, void *gb, int32_t nrhs,
                                     int64_t ld);

/* Multi-right-hand-side solve (SpTRSM) in either dense layout:
 *   SPTRSV_ROW_MAJOR  [n x nrhs], element (i, r) at i * ld + r, ld >= nrhs
 *                     (the layout of sptrsv_solve);
 *   SPTRSV_COL_MAJOR  every right-hand side a contiguous column: element
 *                     (i, r) at r * ld + i, ld >= n.
 * transpose = 0: x = L^{-1} b (or L^{-1} (b + T b)); 1: x = L^{-T} b as
 * sptrsv_solve_transpose (needs build_transpose).  A column-major block is
 * converted to the row-major layout the kernels gather from (each row's
 * right-hand sides contiguous) by tiled shared-memory transposes into a
 * plan-owned buffer of 2 n nrhs elements, allocated on first use and when
 * nrhs grows (so that call synchronises), and the solution is converted
 * back.  Returns SPTRSV_EINVAL for another layout or ld too small.
 * Asynchronous otherwise.                                                  */
typedef enum { SPTRSV_ROW_MAJOR = 0, SPTRSV_COL_MAJOR = 1 } sptrsv_layout;
sptrsv_status sptrsv_solve_layout(sptrsv_plan plan, const void *b, void *x, int32_t nrhs, int64_t ld,
                                  int32_t layout, int32_t transpose);

/* Value gradient on L's pattern: gvals[p] = -sum_r gb[i,r] * x[j,r] for the
 * stored entry p = (i, j), diagonal included.  Asynchronous.                */
sptrsv_status sptrsv_grad_vals(sptrsv_plan plan, const void *gb, const void *x, int32_t nrhs,
                               int64_t ld, void *gvals);

/* Adjoint of b -> b + T b for a rewritten plan: gb = gbp + T^T gbp.        */
sptrsv_status sptrsv_tt_apply(sptrsv_plan plan, const void *gbp, void *gb, int32_t nrhs,
                              int64_t ld);

/* ----------------------------------------------------------------- batched */
/* One plan over nmat independent systems (Ls, Ts, nrhs: host arrays of nmat
 * entries; Ts may be NULL or hold entries with n == 0 for "no T"; opts may
 * be NULL or an array of nmat per-matrix options).  All matrices share the
 * dtype of Ls[0].  Right-hand sides, solutions and gradients are PACKED:
 * matrix m's [n_m x nrhs_m] block (ld = nrhs_m) starts at element
 * rhs_offset[m] of one buffer, its value gradient at vals_offset[m];
 * sptrsv_batch_offsets returns both (host arrays of nmat+1 entries).        */
sptrsv_status sptrsv_batch_plan_create(sptrsv_handle handle, int32_t nmat, const sptrsv_csr *Ls,
                                       const sptrsv_csr *Ts, const int32_t *nrhs,
                                       const sptrsv_plan_opts *opts, sptrsv_plan *plan);
sptrsv_status sptrsv_batch_offsets(sptrsv_plan plan, int64_t *rhs_offset, int64_t *vals_offset);
/* Thin-level threshold of SPTRSV_MODE_HYBRID: levels with fewer rows than
 * thin_rows form the synchronisation-free runs (1 = no thin level, i.e. the
 * level-persistent schedule; 0 = automatic = every level thin, one run:
 * barriers before thick levels were slower on every workload measured).
 * Returns SPTRSV_EINVAL for a negative value or a batched plan.
 * Synchronises.                                                           */
sptrsv_status sptrsv_plan_set_thin_rows(sptrsv_plan plan, int32_t thin_rows);
/* Resident thread blocks per SM of the level-persistent and hybrid solves'
 * persistent grids (256 threads each): 0 = as many as fit (the default);
 * otherwise at most that many.  Their waiting warps poll global memory, so
 * fewer of them can be faster.  Any value is correct: a row group only
 * waits on groups taken before it.  Returns SPTRSV_EINVAL for a negative
 * value or a batched plan.                                                */
sptrsv_status sptrsv_plan_set_blocks_per_sm(sptrsv_plan plan, int32_t blocks_per_sm);

/* Re-tunes a batched plan (used by the autotuner; no analysis is repeated).
 *   rows_per_warp  host, nmat entries (1,2,4,8,16,32; 0 = keep) or NULL:
 *                  row-group width of every system;
 *   rhs_tile       host, nmat entries (1,2,4,8; 0 = keep) or NULL: columns
 *                  per work item; system m runs as ceil(nrhs_m / rhs_tile_m)
 *                  independent work items.
 * Returns SPTRSV_EINVAL for a value outside those sets, SPTRSV_ENOTSUP when
 * the geometry does not fit in shared memory (the plan keeps its previous
 * geometry).  Synchronises.                                               */
sptrsv_status sptrsv_batch_plan_set(sptrsv_plan plan, const int32_t *rows_per_warp,
                                    const int32_t *rhs_tile);
/* The same for one direction: direction 1 = forward solves only, 2 =
 * transpose solves only (0 = both, as sptrsv_batch_plan_set).  The forward
 * and transpose solves of a batch keep separate geometries, since their
 * dependency structures differ (rows of L vs columns of L); an autotuner
 * times and sets each on its own.  Synchronises.                          */
sptrsv_status sptrsv_batch_plan_set_direction(sptrsv_plan plan, int32_t direction,
                                              const int32_t *rows_per_warp, const int32_t *rhs_tile);
/* Schedule of each system's work items (Section 2.1: the level-set
 * schedule, and the synchronisation-free alternative of the related work),
 * for one direction as above (0 = both):
 *   schedule  host, nmat entries:
 *     SPTRSV_BATCH_INORDER  rows in row order, groups of 32 rows completed
 *                           one after another, dependencies inside a group
 *                           resolved in registers (the default);
 *     SPTRSV_BATCH_LEVEL    rows in level order (the plan's analysis; the
 *                           transpose solve takes the levels last to
 *                           first), groups of at most 32 rows of one
 *                           level, every group of a level at the same
 *                           time, each level after the previous one;
 *     0                     keep.
 * The first switch of a system to SPTRSV_BATCH_LEVEL builds its tables
 * (inverse permutation: 4 bytes per row; 16 bytes per group).  Returns
 * SPTRSV_EINVAL for another value, SPTRSV_ENOTSUP when the geometry does
 * not fit in shared memory (the previous schedules are kept).
 * Synchronises.                                                           */
#define SPTRSV_BATCH_INORDER 1
#define SPTRSV_BATCH_LEVEL 2
sptrsv_status sptrsv_batch_plan_set_schedule(sptrsv_plan plan, int32_t direction,
                                             const int32_t *schedule);
/* All systems in one persistent launch (plus a tiny reset launch; the
 * transpose solve also gathers the values into CSC order first): no host
 * work per matrix, so the call can be captured in a CUDA graph.            */
sptrsv_status sptrsv_batch_solve(sptrsv_plan plan, const void *b, void *x);
sptrsv_status sptrsv_batch_solve_transpose(sptrsv_plan plan, const void *gx, void *gb);
sptrsv_status sptrsv_batch_grad_vals(sptrsv_plan plan, const void *gb, const void *x,
                                     void *gvals);
sptrsv_status sptrsv_batch_tt_apply(sptrsv_plan plan, const void *gbp, void *gb);

/* One forward + adjoint step of a batch whose data live in HOST memory (the
 * call of an application that keeps its right-hand sides on the host):
 *   b      host, packed right-hand sides (rhs_offset[nmat] elements of the
 *          plan's dtype);
 *   w      host, packed dL/dx of the same layout;
 *   x      host out: x = L^{-1} b (rewritten systems: L'^{-1} (b + T b));
 *   gb     host out: dL/db = L^{-T} w (rewritten: g + T^T g, g = L'^{-T} w);
 *   gvals  host out: dL/dvals on each system's pattern (vals_offset[nmat]
 *          elements; rewritten systems: on L').
 * Enqueues the copies of b and w to the device, the four batched calls
 * above and the copies back, and returns without waiting.  Consecutive
 * steps alternate between two plan-owned device buffer sets, so that one
 * step's copies overlap the neighbouring steps' solves.  The host buffers
 * must stay valid and unchanged until sptrsv_batch_step_wait returns;
 * page-locked host memory lets the copies run asynchronously.  The first
 * call allocates the two sets (2 x (5 rhs_offset[nmat] + vals_offset[nmat])
 * elements) and two copy streams; the solves run on the handle's stream.
 * Needs a plan built with the transpose (else SPTRSV_ENOTSUP).             */
sptrsv_status sptrsv_batch_step_host(sptrsv_plan plan, const void *b, const void *w, void *x, void *gb,
                                     void *gvals);
/* Waits for every step enqueued by sptrsv_batch_step_host and returns the
 * handle's device status (SPTRSV_OK, or e.g. SPTRSV_ETIMEOUT).             */
sptrsv_status sptrsv_batch_step_wait(sptrsv_plan plan);

/* ------------------------------------------------------------ bounds checks */
/* The library also builds as a bounds-checked debug variant
 * (libsptrsv_gb300_checked.so, compiled with SPTRSV_CHECKED): every index a
 * solve gathers through -- row extents, column indices, positions of the
 * level order, levels, columns of T -- is checked against its array's
 * range; an index outside is recorded as SPTRSV_ERANGE in the handle's
 * status word and replaced by a valid one, so that the access stays inside
 * the array.  sptrsv_checked_build returns 1 in that variant, 0 in the
 * product library (where the checks compile to nothing).
 * sptrsv_debug_check_index runs one checked index through the same check
 * (index against [0, n), 1 <= n <= 32), for tests of the reporting path:
 * in the checked variant an index outside records SPTRSV_ERANGE.          */
int32_t sptrsv_checked_build(void);
sptrsv_status sptrsv_debug_check_index(sptrsv_handle handle, int32_t index, int32_t n);

/* --------------------------------------------------- allocation-free solve */
/* The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate device memory when they solve (an application whose
 * own pool owns the device memory budget, a real-time loop that cannot take
 * cudaMalloc's implicit synchronisation, a plug-in whose host forbids
 * allocation).  It needs no handle and no plan: x = L^{-1} b by the
 * synchronisation-free forward solve, with its scratch (one ready flag per
 * row plus a control block) in a static device array of this library,
 * sized for at most SPTRSV_NOALLOC_MAX_ROWS rows (4 MiB, held on every
 * device that loads the library until the process exits).
 *   L       matrix descriptor (device arrays; not fully validated here --
 *           validate it once with sptrsv_validate -- but the kernel keeps
 *           every access of a malformed row inside the arrays and reports
 *           it: row pointers outside [0, nnz] or decreasing are
 *           SPTRSV_EINVAL, a row whose last entry is not its diagonal
 *           SPTRSV_EDIAG, a column outside [0, i) SPTRSV_ENOTLOWER; the
 *           solution is then undefined);
 *   b, x    [n x nrhs] row-major with leading dimension ld (device);
 *   stream  cudaStream_t to run on (NULL = legacy default stream).
 * Returns SPTRSV_ENOTSUP when n > SPTRSV_NOALLOC_MAX_ROWS (nothing is
 * launched), SPTRSV_EINVAL for bad arguments, SPTRSV_ETIMEOUT when a bounded
 * wait gave up, SPTRSV_ECUDA for a CUDA failure.  Synchronises the stream
 * before returning.  The first call on a device looks up the device address
 * of the scratch array (and may load the library's GPU code): make it before
 * any stream capture.  All calls on a device share the one scratch array,
 * so calls that overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.  Calls no cudaMalloc / cudaFree.     */
#define SPTRSV_NOALLOC_MAX_ROWS (1 << 20)
sptrsv_status sptrsv_solve_noalloc(const sptrsv_csr *L, const void *b, void *x, int32_t nrhs,
                                   int64_t ld, void *stream);

/* ------------------------------------------------------------- diagnostics */
/* Trace of the last batched solve of `plan`: for every system m,
 * trace[3m] and trace[3m+1] are the GPU global-timer values (ns) when a
 * thread block started and finished it, trace[3m+2] the SM it ran on
 * (host array of 3*nmat entries).  Synchronises.                            */
sptrsv_status sptrsv_batch_trace(sptrsv_plan plan, int64_t *trace);

/* Test hook for the bounded waits: makes the next solves of `plan` skip
 * publishing row `row` (-1 clears it), so that any row waiting on it gives
 * up after wait_limit_us and the solve reports SPTRSV_ETIMEOUT.  For a
 * batched plan rows are counted over the systems in order (row i of system
 * m is n_0 + ... + n_{m-1} + i).  The level-persistent mode leaves the row
 * out of its progress counter instead, so every later level waits.         */
sptrsv_status sptrsv_debug_withhold_row(sptrsv_plan plan, int32_t row);

/* The same hook for the level analysis of `handle` (sptrsv_analyze, the
 * incremental analysis and plan creation): row `row`'s level is never
 * published, every wait of those calls gives up after wait_limit_us (> 0)
 * and they return SPTRSV_ETIMEOUT; row = -1 clears the hook.               */
sptrsv_status sptrsv_debug_withhold_level(sptrsv_handle handle, int32_t row, int64_t wait_limit_us);

#ifdef __cplusplus
}
#endif

#endif /* SPTRSV_GB300_H */
