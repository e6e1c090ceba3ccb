"""Seeded synthetic inputs for the SpTRSV hot path.

This module only *draws* inputs: sparse lower-triangular CSR matrices,
right-hand sides, loss weights and the list of rows handed to the rewrite
step.  It contains none of the method's arithmetic (no level analysis, no
solve, no rewrite); both the CPU oracle and the CUDA library consume what it
returns, and neither of them is imported here.

The matrices stand in for the SuiteSparse matrices of the paper's Table 2,
which are not available: banded random systems (n, nnz and level counts in
the paper's ranges), 2D/3D Laplacian lower triangles (closed-form level
structure), and a power-law DAG with skewed level costs.

Conventions (all generators):
  * CSR, int32 ``row_ptr[n+1]`` and ``col_idx[nnz]``, values float64 or
    float32; columns strictly increasing within a row, the diagonal stored
    last (the dependency DAG of the paper's Section 2.1: edge j -> i for every
    off-diagonal L[i, j]).
  * Right-hand sides are dense ``[n, k]`` row-major arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR",
    "band_random",
    "lap2d",
    "lap3d",
    "powerlaw",
    "chain",
    "diagonal",
    "rhs",
    "batch_spec",
    "batch_spec_parallel",
    "BatchItem",
    "narrowest_levels_list",
    "small_levels_list",
    "leading_block",
]


@dataclass
class CSR:
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col_idx: np.ndarray  # int32 [nnz]
    vals: np.ndarray     # float64 or float32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.n >= 0 else 0

    def astype(self, dtype) -> "CSR":
        return CSR(self.n, self.row_ptr, self.col_idx, self.vals.astype(dtype))

    def dense(self) -> np.ndarray:
        """Dense copy (small cases only)."""
        A = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        A[rows, self.col_idx] = self.vals
        return A


def _assemble(n: int, k: np.ndarray, cols_sorted: np.ndarray,
              rng: np.random.Generator) -> CSR:
    """Build a CSR from per-row off-diagonal counts ``k`` and the flattened,
    per-row ascending off-diagonal columns.  Off-diagonal values ~ U(-1, 1)
    (drawn in CSR order); diagonal = 1 + sum |off-diagonal| (stored last)."""
    k = k.astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(k + 1, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    noff = int(k.sum())
    off_vals = rng.uniform(-1.0, 1.0, size=noff)
    rows_of_off = np.repeat(np.arange(n, dtype=np.int64), k)
    # rank of each off-diagonal entry inside its row
    first_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(k, out=first_off[1:])
    rank = np.arange(noff, dtype=np.int64) - first_off[rows_of_off]
    pos = row_ptr[rows_of_off] + rank
    col_idx = np.empty(nnz, dtype=np.int32)
    vals = np.empty(nnz, dtype=np.float64)
    col_idx[pos] = cols_sorted
    vals[pos] = off_vals
    dpos = row_ptr[1:] - 1
    col_idx[dpos] = np.arange(n, dtype=np.int32)
    absum = np.bincount(rows_of_off, weights=np.abs(off_vals), minlength=n)
    vals[dpos] = 1.0 + absum
    if nnz >= 2**31:
        raise ValueError("nnz does not fit int32 row pointers")
    return CSR(n, row_ptr.astype(np.int32), col_idx, vals)


def _subset_rows_dense(rng, lo, m, k, out_cols, out_offsets):
    """Uniform k-subsets of windows [lo, lo+m) via random keys (used where the
    window is small compared with k)."""
    if len(lo) == 0:
        return
    M = int(m.max())
    keys = rng.random((len(lo), M))
    keys[np.arange(M)[None, :] >= m[:, None]] = 2.0  # never chosen
    order = np.argsort(keys, axis=1, kind="stable")
    take = np.arange(M)[None, :] < k[:, None]
    picked = np.where(take, order, np.iinfo(np.int64).max)
    picked.sort(axis=1)
    for r in range(len(lo)):
        kk = int(k[r])
        out_cols[out_offsets[r]:out_offsets[r] + kk] = lo[r] + picked[r, :kk]


def _window_subsets(rng, n, k, lo, m):
    """For every row i choose k[i] distinct columns uniformly without
    replacement from the window [lo[i], lo[i]+m[i]); return them flattened in
    row order, ascending within each row."""
    k = np.minimum(k, m).astype(np.int64)
    offs = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(k, out=offs[1:])
    cols = np.empty(int(offs[-1]), dtype=np.int64)
    dense = (2 * k > m) & (k > 0)
    sparse = (~dense) & (k > 0)
    # dense rows: random keys, grouped by window size to bound memory
    didx = np.nonzero(dense)[0]
    if len(didx):
        for lo_b, hi_b in ((0, 64), (64, 1024), (1024, 1 << 31)):
            sel = didx[(m[didx] > lo_b) & (m[didx] <= hi_b)] if lo_b else didx[m[didx] <= hi_b]
            for s in range(0, len(sel), 1 << 16):
                part = sel[s:s + (1 << 16)]
                _subset_rows_dense(rng, lo[part], m[part], k[part], cols, offs[part])
    sidx = np.nonzero(sparse)[0]
    if len(sidx):
        K = int(k[sidx].max())
        for s in range(0, len(sidx), 1 << 17):
            part = sidx[s:s + (1 << 17)]
            kp, mp, lp = k[part], m[part], lo[part]
            R = np.floor(rng.random((len(part), K)) * mp[:, None]).astype(np.int64)
            valid = np.arange(K)[None, :] < kp[:, None]
            SENT = np.iinfo(np.int64).max
            R[~valid] = SENT
            R.sort(axis=1)
            dup = np.zeros(R.shape, dtype=bool)
            dup[:, 1:] = (R[:, 1:] == R[:, :-1]) & (R[:, 1:] != SENT)
            active = np.nonzero(dup.any(axis=1))[0]
            dup = dup[active]
            while len(active):
                # redraw the duplicates of the rows that still hold some
                sub = R[active]
                rr, cc = np.nonzero(dup)
                sub[rr, cc] = np.floor(rng.random(len(rr)) * mp[active[rr]]).astype(np.int64)
                sub.sort(axis=1)
                dup = np.zeros(sub.shape, dtype=bool)
                dup[:, 1:] = (sub[:, 1:] == sub[:, :-1]) & (sub[:, 1:] != SENT)
                R[active] = sub
                keep = dup.any(axis=1)
                active, dup = active[keep], dup[keep]
            R = R + lp[:, None]
            flat = R[valid]  # row-major: the first k[r] (ascending) of each row
            within = np.arange(int(kp.sum())) - np.repeat(np.cumsum(kp) - kp, kp)
            cols[np.repeat(offs[part], kp) + within] = flat
    return k, cols


def band_random(n: int, band: int, kmin: int, kmax: int, seed=None, *,
                rng: np.random.Generator | None = None, dtype=np.float64) -> CSR:
    """Random banded lower-triangular system.

    Row i gets k_i ~ U{kmin..kmax} off-diagonals, capped at min(i, band),
    at distinct columns drawn uniformly without replacement from
    [max(0, i-band), i); off-diagonal values U(-1, 1); diagonal
    1 + sum |off-diagonal| (strict diagonal dominance).
    """
    rng = rng if rng is not None else np.random.default_rng(seed)
    i = np.arange(n, dtype=np.int64)
    k = rng.integers(kmin, kmax + 1, size=n)
    lo = np.maximum(0, i - band)
    m = i - lo
    k, cols = _window_subsets(rng, n, k, lo, m)
    return _assemble(n, k, cols, rng).astype(dtype)


def lap2d(N: int, dtype=np.float64) -> CSR:
    """Lower triangle of the 5-point Laplacian on an N x N grid, natural
    (row-major) ordering: row i = r*N + c holds -1 at i-N (r > 0), -1 at i-1
    (c > 0) and 4 on the diagonal."""
    n = N * N
    i = np.arange(n, dtype=np.int64)
    r, c = i // N, i % N
    has_s = r > 0
    has_w = c > 0
    k = has_s.astype(np.int64) + has_w.astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(k + 1, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    p = row_ptr[:-1].copy()
    col[p[has_s]] = (i - N)[has_s]
    val[p[has_s]] = -1.0
    p = p + has_s
    col[p[has_w]] = (i - 1)[has_w]
    val[p[has_w]] = -1.0
    p = p + has_w
    col[p] = i
    val[p] = 4.0
    return CSR(n, row_ptr.astype(np.int32), col, val.astype(dtype))


def lap3d(N: int, dtype=np.float64) -> CSR:
    """Lower triangle of the 7-point Laplacian on an N^3 grid, natural
    ordering i = (s*N + r)*N + c: -1 at i-N^2, i-N, i-1 where present, 6 on
    the diagonal."""
    n = N * N * N
    i = np.arange(n, dtype=np.int64)
    s, r, c = i // (N * N), (i // N) % N, i % N
    hs, hr, hc = s > 0, r > 0, c > 0
    k = hs.astype(np.int64) + hr + hc
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(k + 1, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    p = row_ptr[:-1].copy()
    for has, off in ((hs, N * N), (hr, N), (hc, 1)):
        col[p[has]] = (i - off)[has]
        val[p[has]] = -1.0
        p = p + has
    col[p] = i
    val[p] = 6.0
    return CSR(n, row_ptr.astype(np.int32), col, val.astype(dtype))


def _zipf_truncated(rng, alpha, kmax, size):
    ks = np.arange(1, kmax + 1, dtype=np.float64)
    p = ks ** (-alpha)
    cdf = np.cumsum(p / p.sum())
    cdf[-1] = 1.0
    return (np.searchsorted(cdf, rng.random(size), side="right") + 1).astype(np.int64)


def powerlaw(n: int, alpha: float = 2.1, cap: int = 512, near: int = 256,
             p_near: float = 0.7, seed=None, dtype=np.float64) -> CSR:
    """Power-law irregular DAG.

    Row i > 0 gets k_i ~ Zipf(alpha) truncated to {1..cap}, capped at i.
    Each column is, with probability p_near, uniform in the near band
    [max(0, i-near), i) and otherwise uniform in [0, i); duplicates are
    redrawn from the same mixture.  Rows whose window is too small for that
    (2*k_i > i) take a uniform k_i-subset of [0, i).  Values as in
    ``band_random``.
    """
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.int64)
    k = _zipf_truncated(rng, alpha, cap, n)
    k[0] = 0
    k = np.minimum(k, i)
    dense = (2 * k > i) & (k > 0)
    offs = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(k, out=offs[1:])
    cols = np.empty(int(offs[-1]), dtype=np.int64)
    didx = np.nonzero(dense)[0]
    for s in range(0, len(didx), 4096):
        part = didx[s:s + 4096]
        _subset_rows_dense(rng, np.zeros(len(part), np.int64), i[part], k[part], cols, offs[part])
    sidx = np.nonzero((~dense) & (k > 0))[0]
    ent_row = np.repeat(sidx, k[sidx])

    def draw(rows):
        lo_near = np.maximum(0, rows - near)
        use_near = rng.random(len(rows)) < p_near
        u = rng.random(len(rows))
        c_near = lo_near + np.floor(u * (rows - lo_near)).astype(np.int64)
        c_far = np.floor(u * rows).astype(np.int64)
        return np.where(use_near, c_near, c_far)

    c = draw(ent_row)
    while True:
        key = ent_row * n + c
        order = np.argsort(key, kind="stable")
        ent_row, c = ent_row[order], c[order]
        dup = np.zeros(len(c), dtype=bool)
        dup[1:] = (ent_row[1:] == ent_row[:-1]) & (c[1:] == c[:-1])
        if not dup.any():
            break
        c[dup] = draw(ent_row[dup])
    start = np.searchsorted(ent_row, ent_row, side="left")
    cols[offs[ent_row] + (np.arange(len(c)) - start)] = c
    return _assemble(n, k, cols, rng).astype(dtype)


def chain(n: int, dtype=np.float64, seed=None) -> CSR:
    """Bidiagonal chain: row i depends on i-1 (n levels)."""
    rng = np.random.default_rng(seed)
    k = np.minimum(np.arange(n), 1)
    cols = np.arange(n, dtype=np.int64)[k.astype(bool)] - 1
    return _assemble(n, k, cols, rng).astype(dtype)


def diagonal(n: int, dtype=np.float64, seed=None) -> CSR:
    """Diagonal-only matrix (one level)."""
    rng = np.random.default_rng(seed)
    return _assemble(n, np.zeros(n, np.int64), np.zeros(0, np.int64), rng).astype(dtype)


def rhs(n: int, k: int, seed=None, dtype=np.float64, rng=None) -> np.ndarray:
    """Dense right-hand sides, ``[n, k]`` row-major, entries U(-1, 1)."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n, k)).astype(dtype)


def leading_block(A: CSR, m: int) -> CSR:
    """Leading principal m x m block of a lower-triangular CSR (still lower
    triangular with the diagonal last in every row)."""
    rp = A.row_ptr[: m + 1].astype(np.int64)
    col = A.col_idx[: rp[-1]]
    keep = col < m  # always true for lower-triangular rows < m
    assert keep.all()
    return CSR(m, rp.astype(np.int32), col.copy(), A.vals[: rp[-1]].copy())


@dataclass
class BatchItem:
    A: CSR
    nrhs: int
    band: int
    b: np.ndarray
    rewritten: bool


def batch_spec(nmat: int = 512, seed: int = 3, n_lo: int = 1000, n_hi: int = 200_000,
               w_lo: int = 16, w_hi: int = 1024, dtype=np.float32, with_rhs: bool = True,
               k_hi: float = 32.0):
    """Batch of independent lower-triangular systems.

    Matrix m uses ``np.random.default_rng(SeedSequence(seed).spawn(nmat)[m])``:
    n ~ logU[n_lo, n_hi], band w ~ logU[w_lo, w_hi], off-diagonals per row
    ~ U{4..16} capped at min(i, w) in [i-w, i), nrhs = round(logU[1, k_hi])
    (k_hi = 32 for the benchmark's batch); odd-indexed matrices are marked
    for a pre-applied rewrite.
    """
    children = np.random.SeedSequence(seed).spawn(nmat)
    return [_batch_one((m, ss, n_lo, n_hi, w_lo, w_hi, dtype, with_rhs, k_hi))
            for m, ss in enumerate(children)]


def _batch_one(args):
    m, ss, n_lo, n_hi, w_lo, w_hi, dtype, with_rhs, k_hi = args
    rng = np.random.default_rng(ss)
    n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    w = int(round(math.exp(rng.uniform(math.log(w_lo), math.log(w_hi)))))
    k = int(round(math.exp(rng.uniform(0.0, math.log(k_hi)))))
    A = band_random(n, w, 4, 16, rng=rng, dtype=dtype)
    b = rhs(n, k, rng=rng, dtype=dtype) if with_rhs else None
    return BatchItem(A, k, w, b, rewritten=(m % 2 == 1))


def batch_spec_parallel(nmat: int = 512, seed: int = 3, workers: int | None = None, **kw):
    """``batch_spec`` computed by a pool of worker processes (spawned, so it
    is safe after CUDA has been initialised); identical output, since every
    system draws from its own child seed."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    n_lo, n_hi = kw.get("n_lo", 1000), kw.get("n_hi", 200_000)
    w_lo, w_hi = kw.get("w_lo", 16), kw.get("w_hi", 1024)
    dtype, with_rhs = kw.get("dtype", np.float32), kw.get("with_rhs", True)
    k_hi = kw.get("k_hi", 32.0)
    children = np.random.SeedSequence(seed).spawn(nmat)
    jobs = [(m, ss, n_lo, n_hi, w_lo, w_hi, dtype, with_rhs, k_hi) for m, ss in enumerate(children)]
    workers = workers or min(32, os.cpu_count() or 4)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_batch_one, jobs, chunksize=4))


# ----------------------------------------------------------------------------
# Rewrite lists.  These stand in for the rewriting list that the paper's
# policy (or its heuristic strategies) hands to the rewriting module
# (Section 4.3: triplets <node, source level, target level>).  They read the
# level partition produced by an analysis; they compute nothing of the method.
# ----------------------------------------------------------------------------

def _chunks_to_list(picked_levels, level_ptr, perm, D):
    rows, targets = [], []
    picked = sorted(set(int(l) for l in picked_levels))
    runs, cur = [], []
    for l in picked:
        if cur and l == cur[-1] + 1:
            cur.append(l)
        else:
            if cur:
                runs.append(cur)
            cur = [l]
    if cur:
        runs.append(cur)
    for run in runs:
        for s in range(0, len(run), D):
            chunk = run[s:s + D]
            t = chunk[0] - 1
            for l in chunk:
                seg = perm[level_ptr[l]:level_ptr[l + 1]]
                rows.append(np.asarray(seg, dtype=np.int32))
                targets.append(np.full(len(seg), t, dtype=np.int32))
    if not rows:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    return np.concatenate(rows), np.concatenate(targets)


def narrowest_levels_list(nlevels, level_ptr, perm, frac=0.01, D=8):
    """Narrowest-level rule: candidate levels l >= 1 sorted by (rows, l)
    ascending are taken until they hold at least ceil(frac*n) rows; picked
    levels are grouped into maximal runs of consecutive levels, each run is
    cut into chunks of at most D levels, and every row of a chunk gets the
    target (first level of the chunk) - 1."""
    level_ptr = np.asarray(level_ptr)
    n = int(level_ptr[nlevels])
    nrows = np.diff(level_ptr[: nlevels + 1])
    need = math.ceil(frac * n)
    cand = sorted(range(1, nlevels), key=lambda l: (int(nrows[l]), l))
    picked, acc = [], 0
    for l in cand:
        if acc >= need:
            break
        picked.append(l)
        acc += int(nrows[l])
    return _chunks_to_list(picked, level_ptr, np.asarray(perm), D)


def small_levels_list(nlevels, level_ptr, perm, max_rows=4, D=8):
    """Every level l >= 1 holding fewer than ``max_rows`` rows, chunked as in
    ``narrowest_levels_list``."""
    level_ptr = np.asarray(level_ptr)
    nrows = np.diff(level_ptr[: nlevels + 1])
    picked = [l for l in range(1, nlevels) if nrows[l] < max_rows]
    return _chunks_to_list(picked, level_ptr, np.asarray(perm), D)
