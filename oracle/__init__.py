"""CPU oracle for the SpTRSV hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, sequential FP64 restatement of what the paper's method
computes (see ``sptrsv_oracle.c`` for the definitions and the sections they
come from), exposed to Python through ctypes.  Only ``tests/``, the smoke
check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may use
it; the CUDA library never imports or links it, and the two share no code.

FP32 inputs are widened to FP64 before they reach the C code, so the oracle
solves exactly the system the stored FP32 values define.

Parity status of each function (what pins it in ``tests/test_oracle.py``):
  solve, solve_transpose, grad_vals  -- dense triangular solves (numpy) on
      small systems, manufactured solutions, Higham's backward-error bound,
      central finite differences;
  levels, partition                  -- brute-force longest path on tiny DAGs,
      closed forms (2D/3D grid, chain, diagonal);
  stats                              -- the paper's printed ALC/ARL/AIR and
      threshold values (Tables 4-5), textbook population CV (numpy);
      the ddof of CV is not fixed by the paper: "parity unpinned" for the
      choice of population over sample variance;
  rewrite, solve_rewritten, tt_apply -- a worked 3x3 example, the 2D
      Laplacian closed form, solution equality, level invariants.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sptrsv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ENOTLOWER, EDIAG, EUNSORTED, ETARGET, ENOMEM = range(7)


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (gcc, -O2,
    -ffp-contract=off so that no multiply-add is fused)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        _lib = _load(_LIB)
    return _lib


def _load(path):
    """Load an oracle library image and declare its signatures (the tests
    also use this to load deliberately broken builds of the same source)."""
    lib = C.CDLL(path)
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    i32 = C.c_int32
    lib.orc_validate.argtypes = [i32, i32p, i32p, f64p, C.POINTER(C.c_int32)]
    lib.orc_validate.restype = C.c_int
    lib.orc_solve.argtypes = [i32, i32p, i32p, f64p, i32, f64p, f64p]
    lib.orc_solve_transpose.argtypes = [i32, i32p, i32p, f64p, i32, f64p, f64p]
    lib.orc_grad_vals.argtypes = [i32, i32p, i32p, i32, f64p, f64p, f64p]
    lib.orc_levels.argtypes = [i32, i32p, i32p, i32p]
    lib.orc_levels.restype = i32
    lib.orc_partition.argtypes = [i32, i32p, i32p, i32, i32p, i32p, i64p]
    lib.orc_stats.argtypes = [i32, C.c_int64, i32, i32p, i64p, f64p]
    lib.orc_thin_threshold.argtypes = [C.c_double, C.c_double, C.c_double]
    lib.orc_thin_threshold.restype = C.c_double
    lib.orc_level_summary.argtypes = [i32, i32p, i32, i32p, i32p, i64p, C.c_double, C.c_void_p, i32p, i64p]
    vp = C.c_void_p
    lib.orc_rewrite.argtypes = [i32, i32p, i32p, f64p, i32p, i32, i32p, vp,
                                i32p, vp, vp, i32p, vp, vp, C.POINTER(C.c_int32)]
    lib.orc_rewrite.restype = C.c_int
    lib.orc_solve_rewritten.argtypes = [i32, i32p, i32p, f64p, i32p, i32p, f64p, i32,
                                        f64p, f64p]
    lib.orc_tt_apply.argtypes = [i32, i32p, i32p, f64p, i32, f64p, f64p]
    return lib


def use_library(path=None):
    """Point the wrapper at another build of ``sptrsv_oracle.c`` (None = the
    default one).  Test helper for the mutation tests."""
    global _lib
    _lib = None if path is None else _load(path)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _mat(A):
    return int(A.n), _i32(A.row_ptr), _i32(A.col_idx), _f64(A.vals)


def _rhs2d(b, n):
    b = np.asarray(b)
    if b.ndim == 1:
        b = b.reshape(n, 1)
    return _f64(b), b.shape[1]


class OracleError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"oracle status {status} at {where}")
        self.status = status
        self.where = where


def validate(A):
    """Returns (status, first offending row or -1)."""
    n, rp, ci, v = _mat(A)
    bad = C.c_int32(-1)
    st = _L().orc_validate(n, rp, ci, v, C.byref(bad))
    return int(st), int(bad.value)


def solve(A, b):
    """x = L^{-1} b by forward substitution in row order (FP64)."""
    n, rp, ci, v = _mat(A)
    b2, k = _rhs2d(b, n)
    x = np.zeros((n, k), np.float64)
    _L().orc_solve(n, rp, ci, v, k, b2, x)
    return x


def solve_transpose(A, gx):
    """g_b = L^{-T} g_x by backward column sweep (FP64)."""
    n, rp, ci, v = _mat(A)
    g2, k = _rhs2d(gx, n)
    gb = np.zeros((n, k), np.float64)
    _L().orc_solve_transpose(n, rp, ci, v, k, g2, gb)
    return gb


def grad_vals(A, gb, x):
    """dLoss/dL_ij = -sum_r gb[i,r] x[j,r] on L's pattern (FP64)."""
    n, rp, ci, _ = _mat(A)
    gb2, k = _rhs2d(gb, n)
    x2, k2 = _rhs2d(x, n)
    assert k == k2
    gv = np.zeros(int(rp[-1]) if n else 0, np.float64)
    _L().orc_grad_vals(n, rp, ci, k, gb2, x2, gv)
    return gv


def levels(A):
    """Kahn-style levels; returns (lev[n] int32, nlevels)."""
    n, rp, ci, _ = _mat(A)
    lev = np.zeros(max(n, 1), np.int32)
    nl = _L().orc_levels(n, rp, ci, lev)
    return lev[:n], int(nl)


def partition(A, lev, nlevels):
    """(perm[n], level_ptr[nlevels+1], cost[nlevels] int64)."""
    n, rp, _, _ = _mat(A)
    perm = np.zeros(max(n, 1), np.int32)
    lp = np.zeros(nlevels + 1, np.int32)
    cost = np.zeros(max(nlevels, 1), np.int64)
    _L().orc_partition(n, rp, _i32(lev), nlevels, perm, lp, cost)
    return perm[:n], lp, cost[:nlevels]


def stats(n, nnz, nlevels, level_ptr, cost):
    """[ALC, ARL, AIR, CV(cost), CV(rows), thin threshold (alpha=1)]."""
    out = np.zeros(6, np.float64)
    _L().orc_stats(int(n), int(nnz), int(nlevels), _i32(level_ptr),
                   np.ascontiguousarray(cost, dtype=np.int64) if nlevels else np.zeros(1, np.int64),
                   out)
    return out


def thin_threshold(alc, cv, alpha=1.0):
    return float(_L().orc_thin_threshold(float(alc), float(cv), float(alpha)))


def level_summary(A, an, threshold=None):
    """Thin levels and the per-level row with the fewest dependencies:
    (thin[nlevels] uint8, pick[nlevels] int32, [thin count, max rows in a
    thin level, max cost of a thin level]).  threshold defaults to the
    analysis' thin-level threshold (alpha = 1)."""
    n, rp, _, _ = _mat(A)
    nl = int(an["nlevels"])
    thr = float(an["stats"][5]) if threshold is None else float(threshold)
    thin = np.zeros(max(nl, 1), np.uint8)
    pick = np.zeros(max(nl, 1), np.int32)
    out = np.zeros(3, np.int64)
    cost = np.ascontiguousarray(an["cost"], dtype=np.int64) if nl else np.zeros(1, np.int64)
    _L().orc_level_summary(n, rp, nl, _i32(an["level_ptr"]), _i32(an["perm"]) if n else np.zeros(1, np.int32),
                           cost, thr, thin.ctypes.data_as(C.c_void_p), pick, out)
    return thin[:nl], pick[:nl], out


def analyze(A):
    """Full level analysis: dict(lev, nlevels, perm, level_ptr, cost, stats)."""
    lev, nl = levels(A)
    perm, lp, cost = partition(A, lev, nl)
    st = stats(A.n, A.nnz, nl, lp, cost)
    return dict(lev=lev, nlevels=nl, perm=perm, level_ptr=lp, cost=cost, stats=st)


class _CSR:
    def __init__(self, n, row_ptr, col_idx, vals):
        self.n, self.row_ptr, self.col_idx, self.vals = n, row_ptr, col_idx, vals

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


def rewrite(A, lev, rows, targets=None):
    """Row-substitution rewrite; returns (L', T) as CSR-like objects with
    FP64 values.  Raises OracleError on an invalid row or target."""
    n, rp, ci, v = _mat(A)
    lev = _i32(lev)
    rows = _i32(rows)
    tg = None if targets is None else _i32(targets)
    lp_rp = np.zeros(n + 1, np.int32)
    t_rp = np.zeros(n + 1, np.int32)
    bad = C.c_int32(-1)
    tptr = None if tg is None else tg.ctypes.data_as(C.c_void_p)
    L = _L()
    st = L.orc_rewrite(n, rp, ci, v, lev, len(rows), rows, tptr, lp_rp, None, None,
                       t_rp, None, None, C.byref(bad))
    if st != OK:
        raise OracleError(st, int(bad.value))
    lp_ci = np.zeros(max(int(lp_rp[-1]), 1), np.int32)
    lp_v = np.zeros(max(int(lp_rp[-1]), 1), np.float64)
    t_ci = np.zeros(max(int(t_rp[-1]), 1), np.int32)
    t_v = np.zeros(max(int(t_rp[-1]), 1), np.float64)
    st = L.orc_rewrite(n, rp, ci, v, lev, len(rows), rows, tptr, lp_rp,
                       lp_ci.ctypes.data_as(C.c_void_p), lp_v.ctypes.data_as(C.c_void_p),
                       t_rp, t_ci.ctypes.data_as(C.c_void_p), t_v.ctypes.data_as(C.c_void_p),
                       C.byref(bad))
    if st != OK:
        raise OracleError(st, int(bad.value))
    Lp = _CSR(n, lp_rp, lp_ci[: lp_rp[-1]], lp_v[: lp_rp[-1]])
    T = _CSR(n, t_rp, t_ci[: t_rp[-1]], t_v[: t_rp[-1]])
    return Lp, T


def solve_rewritten(Lp, T, b):
    """x = L'^{-1} (b + T b)."""
    n, rp, ci, v = _mat(Lp)
    b2, k = _rhs2d(b, n)
    x = np.zeros((n, k), np.float64)
    _L().orc_solve_rewritten(n, rp, ci, v, _i32(T.row_ptr), _i32(T.col_idx), _f64(T.vals),
                             k, b2, x)
    return x


def tt_apply(T, gbp):
    """g_b = g_b' + T^T g_b'."""
    n = int(T.n)
    g2, k = _rhs2d(gbp, n)
    gb = np.zeros((n, k), np.float64)
    _L().orc_tt_apply(n, _i32(T.row_ptr), _i32(T.col_idx), _f64(T.vals), k, g2, gb)
    return gb
