"""Shared helpers of the GPU parity tests (inputs from ``synthetic``,
expected values from ``oracle``)."""
import numpy as np

import synthetic as S

TOL = {np.float64: 1e-12, np.float32: 1e-5}


def relerr(x, ref):
    x = np.asarray(x, dtype=np.float64).reshape(ref.shape)
    d = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (d if d > 0 else 1.0)


def widened(A):
    """The same system with FP64 values (what the oracle solves)."""
    return S.CSR(A.n, A.row_ptr, A.col_idx, A.vals.astype(np.float64))


def wide_level(n, seed=0):
    """Row 0 plus n-1 rows that depend only on row 0: two levels, one wide."""
    rng = np.random.default_rng(seed)
    k = np.ones(n, np.int64)
    k[0] = 0
    cols = np.zeros(n - 1, np.int64)
    return S._assemble(n, k, cols, rng)


def two_wide_levels(m, seed=0):
    """m independent rows, then m rows that each depend on 3 random rows of
    the first m: two levels of m rows (wider than a shared-memory ring when
    m is large)."""
    rng = np.random.default_rng(seed)
    k = np.concatenate([np.zeros(m, np.int64), np.full(m, 3, np.int64)])
    cols = np.concatenate([np.sort(rng.choice(m, 3, replace=False)) for _ in range(m)])
    return S._assemble(2 * m, k, cols, rng)


def long_row(n=2000, width=512, seed=0):
    """Random band matrix whose last row has `width` off-diagonals."""
    A = S.band_random(n - 1, 40, 0, 6, seed=seed)
    rng = np.random.default_rng(seed + 1)
    cols = np.sort(rng.choice(n - 1, size=width, replace=False))
    offv = rng.uniform(-1, 1, width)
    rp = np.concatenate([A.row_ptr, [A.row_ptr[-1] + width + 1]]).astype(np.int32)
    ci = np.concatenate([A.col_idx, cols, [n - 1]]).astype(np.int32)
    v = np.concatenate([A.vals, offv, [1.0 + np.abs(offv).sum()]])
    return S.CSR(n, rp, ci, v)


def cases_small():
    """(name, CSR) edge cases and small workloads, several tiles + ragged tails."""
    return [
        ("n1", S.band_random(1, 4, 0, 4, seed=1)),
        ("diag", S.diagonal(1000, seed=2)),
        ("chain", S.chain(3001, seed=3)),
        ("wide_level", wide_level(40_001)),
        ("long_row", long_row()),
        ("cfg0", S.band_random(2000, 64, 0, 8, seed=0)),
        ("lap2d_97", S.lap2d(97)),
        ("lap3d_23", S.lap3d(23)),
        ("band_deep", S.band_random(30_011, 20, 4, 16, seed=5)),
        ("band_wide", S.band_random(50_003, 1024, 4, 16, seed=6)),
        ("powerlaw", S.powerlaw(60_000, alpha=2.1, seed=7)),
    ]
