"""Torch-facing wrappers over the C ABI: argument marshalling only.

PyTorch provides device memory and streams; every step of the solve path
runs in the library's CUDA kernels.  All calls use the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

_DTYPES = {torch.float64: L.SPTRSV_F64, torch.float32: L.SPTRSV_F32}


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


class Matrix:
    """Lower-triangular CSR matrix in device memory (int32 indices, FP64 or
    FP32 values), the diagonal stored last in every row."""

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor):
        if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32:
            raise TypeError("row_ptr and col_idx must be int32")
        if vals.dtype not in _DTYPES:
            raise TypeError("vals must be float64 or float32")
        for t in (row_ptr, col_idx, vals):
            if not t.is_cuda:
                raise ValueError("matrix arrays must live on a CUDA device")
            if not t.is_contiguous():
                raise ValueError("matrix arrays must be contiguous")
        self.row_ptr, self.col_idx, self.vals = row_ptr, col_idx, vals
        self.n = row_ptr.numel() - 1
        self.nnz = col_idx.numel()
        if vals.numel() != self.nnz:
            raise ValueError("vals and col_idx differ in length")

    @property
    def dtype(self):
        return self.vals.dtype

    @classmethod
    def from_host(cls, A, device="cuda", dtype=None):
        """From any object with n, row_ptr, col_idx, vals numpy arrays."""
        vals = torch.as_tensor(np.ascontiguousarray(A.vals))
        if dtype is not None:
            vals = vals.to(dtype)
        return cls(torch.as_tensor(np.ascontiguousarray(A.row_ptr, dtype=np.int32)).to(device),
                   torch.as_tensor(np.ascontiguousarray(A.col_idx, dtype=np.int32)).to(device),
                   vals.to(device))

    def desc(self) -> L.sptrsv_csr:
        return L.sptrsv_csr(self.n, self.nnz, _ptr(self.row_ptr), _ptr(self.col_idx),
                            _ptr(self.vals), _DTYPES[self.vals.dtype])

    def to_host(self):
        return (self.row_ptr.cpu().numpy(), self.col_idx.cpu().numpy(), self.vals.cpu().numpy())


class Handle:
    """Library handle bound to one CUDA stream."""

    def __init__(self, stream: torch.cuda.Stream | None = None):
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        h = L.sptrsv_handle()
        L.check(L.lib().sptrsv_create(C.byref(h), C.c_void_p(s.cuda_stream)), "sptrsv_create")
        self.h = h

    def status(self) -> int:
        """Synchronise and return (and clear) the device status word."""
        return int(L.lib().sptrsv_get_status(self.h))

    def withhold_level(self, row: int, wait_limit_us: int = 0):
        """Test hook of the bounded waits of the level analysis (see
        sptrsv_debug_withhold_level); row = -1 clears it."""
        L.check(L.lib().sptrsv_debug_withhold_level(self.h, int(row), int(wait_limit_us)),
                "sptrsv_debug_withhold_level")

    def __del__(self):
        try:
            if getattr(self, "h", None) and not L.exiting():
                L.lib().sptrsv_destroy(self.h)
        except Exception:
            pass


_handles: dict = {}


def handle() -> Handle:
    """Handle for the current device and stream (cached)."""
    s = torch.cuda.current_stream()
    key = (s.device.index, s.cuda_stream)
    h = _handles.get(key)
    if h is None:
        h = Handle(s)
        _handles[key] = h
    return h


def validate(A: Matrix):
    """(status, first offending row or -1); see sptrsv_validate."""
    bad = C.c_int32(-1)
    st = L.lib().sptrsv_validate(handle().h, C.byref(A.desc()), C.byref(bad))
    return int(st), int(bad.value)


@dataclass
class Analysis:
    lev: torch.Tensor        # [n] int32
    perm: torch.Tensor       # [n] int32
    level_ptr: torch.Tensor  # [nlevels+1] int32
    cost: torch.Tensor       # [nlevels] int64
    nlevels: int
    stats: np.ndarray        # ALC, ARL, AIR, CV(cost), CV(rows), thin threshold

    STAT_NAMES = ("alc", "arl", "air", "cv_cost", "cv_rows", "thin_threshold")


def analyze(A: Matrix, prev_lev: torch.Tensor | None = None, first_row: int = 0) -> Analysis:
    """Level analysis (sptrsv_analyze).  With prev_lev and first_row > 0 the
    levels of rows before first_row are taken from prev_lev and only the rest
    are recomputed (sptrsv_analyze_incremental): use it after a change that
    left those rows alone, e.g. a rewrite of rows >= first_row."""
    dev = A.row_ptr.device
    n = A.n
    lev = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    lp = torch.empty(n + 1, dtype=torch.int32, device=dev)
    cost = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    nl = C.c_int32(0)
    st = (C.c_double * 6)()
    if prev_lev is not None and first_row > 0:
        lev[:n].copy_(prev_lev[:n])
        L.check(L.lib().sptrsv_analyze_incremental(handle().h, C.byref(A.desc()), int(first_row), _ptr(lev),
                                                   _ptr(perm), _ptr(lp), _ptr(cost), C.byref(nl), st),
                "sptrsv_analyze_incremental")
    else:
        L.check(L.lib().sptrsv_analyze(handle().h, C.byref(A.desc()), _ptr(lev), _ptr(perm), _ptr(lp),
                                       _ptr(cost), C.byref(nl), st), "sptrsv_analyze")
    k = int(nl.value)
    return Analysis(lev[:n], perm[:n], lp[:k + 1], cost[:k], k, np.array(list(st)))


def level_summary(A: Matrix, an: Analysis, threshold: float | None = None):
    """Thin levels (cost below the threshold; default: the analysis' thin-
    level threshold) and the row with the fewest dependencies of every level
    (sptrsv_level_summary).  Returns (thin uint8 [nlevels], pick int32
    [nlevels], numpy [thin count, max rows in a thin level, max cost of a
    thin level])."""
    dev = A.row_ptr.device
    k = an.nlevels
    thr = float(an.stats[5]) if threshold is None else float(threshold)
    thin = torch.empty(max(k, 1), dtype=torch.uint8, device=dev)
    pick = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
    out = (C.c_int64 * 3)()
    L.check(L.lib().sptrsv_level_summary(handle().h, C.byref(A.desc()), _ptr(an.perm), _ptr(an.level_ptr),
                                         _ptr(an.cost), k, thr, _ptr(thin), _ptr(pick), out),
            "sptrsv_level_summary")
    return thin[:k], pick[:k], np.array(list(out), dtype=np.int64)


def transpose(A: Matrix) -> Matrix:
    """A^T of a square CSR matrix (sptrsv_transpose); the result's columns
    are strictly increasing inside every row."""
    dev = A.row_ptr.device
    rp = torch.empty(A.n + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)
    v = torch.empty(max(A.nnz, 1), dtype=A.dtype, device=dev)
    out = L.sptrsv_csr_out(_ptr(rp), _ptr(ci), _ptr(v))
    L.check(L.lib().sptrsv_transpose(handle().h, C.byref(A.desc()), C.byref(out)), "sptrsv_transpose")
    return Matrix(rp, ci[:A.nnz], v[:A.nnz])


class UpperPlan:
    """U x = b for an upper-triangular CSR matrix U whose rows store the
    diagonal first: a plan for the lower-triangular U^T, solved by its
    transpose solve (and U^T x = b by its forward solve).  The plan holds
    U^T built from U's values at creation; after changing U's values call
    refresh()."""

    def __init__(self, U: Matrix, mode="auto", rows_per_warp=0, rhs_tile=0):
        self.U = U
        self.Ut = transpose(U)
        self.plan = Plan(self.Ut, None, mode=mode, rows_per_warp=rows_per_warp, rhs_tile=rhs_tile,
                         transpose=True)

    def refresh(self):
        """Re-read U's values (the pattern must be unchanged)."""
        Ut = transpose(self.U)
        self.Ut.vals.copy_(Ut.vals)

    def solve(self, b, out=None):
        """x = U^{-1} b."""
        return self.plan.solve_transpose(b, out=out)

    def solve_transpose(self, b, out=None):
        """x = U^{-T} b."""
        return self.plan.solve(b, out=out)


def rewrite(A: Matrix, lev: torch.Tensor, rows, targets=None):
    """Row-substitution rewrite (see sptrsv_rewrite); returns (L', T)."""
    dev = A.row_ptr.device
    rows = torch.as_tensor(rows, dtype=torch.int32).to(dev).contiguous()
    tg = None if targets is None else torch.as_tensor(targets, dtype=torch.int32).to(dev).contiguous()
    nlp, nt = C.c_int64(0), C.c_int64(0)
    lp_rp = torch.empty(A.n + 1, dtype=torch.int32, device=dev)
    t_rp = torch.empty(A.n + 1, dtype=torch.int32, device=dev)
    h = handle().h
    desc = A.desc()
    lib = L.lib()
    L.check(lib.sptrsv_rewrite(h, C.byref(desc), _ptr(lev), _ptr(rows), _ptr(tg), int(rows.numel()),
                               C.byref(nlp), C.byref(nt), None, None), "sptrsv_rewrite (sizes)")
    lp_ci = torch.empty(max(nlp.value, 1), dtype=torch.int32, device=dev)
    lp_v = torch.empty(max(nlp.value, 1), dtype=A.dtype, device=dev)
    t_ci = torch.empty(max(nt.value, 1), dtype=torch.int32, device=dev)
    t_v = torch.empty(max(nt.value, 1), dtype=A.dtype, device=dev)
    o1 = L.sptrsv_csr_out(_ptr(lp_rp), _ptr(lp_ci), _ptr(lp_v))
    o2 = L.sptrsv_csr_out(_ptr(t_rp), _ptr(t_ci), _ptr(t_v))
    L.check(lib.sptrsv_rewrite(h, C.byref(desc), _ptr(lev), _ptr(rows), _ptr(tg), int(rows.numel()),
                               C.byref(nlp), C.byref(nt), C.byref(o1), C.byref(o2)), "sptrsv_rewrite")
    Lp = Matrix(lp_rp, lp_ci[: nlp.value], lp_v[: nlp.value])
    T = Matrix(t_rp, t_ci[: nt.value], t_v[: nt.value])
    return Lp, T


class Plan:
    """Reusable solve plan for L (and T of a rewritten system)."""

    def __init__(self, A: Matrix, T: Matrix | None = None, mode="auto", rows_per_warp=0,
                 rhs_tile=0, transpose=False, wait_limit_us=0):
        self.A, self.T = A, T
        opts = L.sptrsv_plan_opts(L.MODE_NAMES[mode] if isinstance(mode, str) else int(mode),
                                  rows_per_warp, rhs_tile, 1 if transpose else 0, wait_limit_us)
        p = L.sptrsv_plan()
        self._h = handle()
        tdesc = T.desc() if T is not None else None
        L.check(L.lib().sptrsv_plan_create(self._h.h, C.byref(A.desc()),
                                           C.byref(tdesc) if tdesc is not None else None,
                                           C.byref(opts), C.byref(p)), "sptrsv_plan_create")
        self.p = p

    def info(self):
        nl, m, r, k = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        L.check(L.lib().sptrsv_plan_info(self.p, C.byref(nl), C.byref(m), C.byref(r), C.byref(k)))
        return dict(nlevels=nl.value, mode=m.value, rows_per_warp=r.value, rhs_tile=k.value)

    def set(self, mode=0, rows_per_warp=0, rhs_tile=0):
        mode = L.MODE_NAMES[mode] if isinstance(mode, str) else int(mode)
        L.check(L.lib().sptrsv_plan_set(self.p, mode, rows_per_warp, rhs_tile), "sptrsv_plan_set")

    def solve_columns(self, B, transpose=False, out=None):
        """Multi-right-hand-side solve in the column-major layout: B is a
        [k, n] CUDA tensor whose row r is right-hand side r (rows may be
        padded: stride(0) >= n); returns X of the same layout with
        X[r] = L^{-1} B[r] (transpose: L^{-T} B[r]).  See
        sptrsv_solve_layout."""
        n = self.A.n
        if B.dim() != 2 or B.shape[1] != n or B.stride(1) != 1 or B.dtype != self.A.dtype or not B.is_cuda:
            raise ValueError("B must be a [k, n] CUDA tensor of the matrix dtype with unit stride along n")
        X = out if out is not None else torch.empty_strided(B.shape, B.stride(), dtype=B.dtype, device=B.device)
        if X.shape != B.shape or X.stride() != B.stride():
            raise ValueError("out must have B's shape and strides")
        L.check(L.lib().sptrsv_solve_layout(self.p, _ptr(B), _ptr(X), B.shape[0], B.stride(0),
                                            L.SPTRSV_COL_MAJOR, 1 if transpose else 0), "sptrsv_solve_layout")
        return X

    def set_thin_rows(self, thin_rows: int = 0):
        """Thin-level threshold of the hybrid mode (0 = automatic)."""
        L.check(L.lib().sptrsv_plan_set_thin_rows(self.p, int(thin_rows)), "sptrsv_plan_set_thin_rows")

    def set_blocks_per_sm(self, blocks: int = 0):
        """Resident blocks per SM of the level-persistent and hybrid grids
        (0 = as many as fit)."""
        L.check(L.lib().sptrsv_plan_set_blocks_per_sm(self.p, int(blocks)), "sptrsv_plan_set_blocks_per_sm")

    def withhold(self, row: int):
        L.check(L.lib().sptrsv_debug_withhold_row(self.p, row))

    @staticmethod
    def _rhs(b, n, dtype):
        if b.dim() == 1:
            b = b.view(n, 1)
        if b.dtype != dtype or not b.is_cuda or b.shape[0] != n or b.stride(1) != 1:
            raise ValueError("right-hand side must be an [n, k] CUDA tensor of the matrix dtype "
                             "with unit column stride")
        return b

    def solve(self, b: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        squeeze = b.dim() == 1
        b2 = self._rhs(b, self.A.n, self.A.dtype)
        x = out if out is not None else torch.empty(self.A.n, b2.shape[1], dtype=b2.dtype, device=b2.device)
        x2 = self._rhs(x, self.A.n, self.A.dtype)
        L.check(L.lib().sptrsv_solve(self.p, _ptr(b2), _ptr(x2), b2.shape[1], b2.stride(0)),
                "sptrsv_solve")
        return x.view(-1) if squeeze and out is None else x

    def solve_transpose(self, gx: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        squeeze = gx.dim() == 1
        g2 = self._rhs(gx, self.A.n, self.A.dtype)
        gb = out if out is not None else torch.empty(self.A.n, g2.shape[1], dtype=g2.dtype, device=g2.device)
        L.check(L.lib().sptrsv_solve_transpose(self.p, _ptr(g2), _ptr(gb), g2.shape[1], g2.stride(0)),
                "sptrsv_solve_transpose")
        return gb.view(-1) if squeeze and out is None else gb

    def grad_vals(self, gb: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None):
        gb2 = self._rhs(gb, self.A.n, self.A.dtype)
        x2 = self._rhs(x, self.A.n, self.A.dtype)
        gv = out if out is not None else torch.empty(self.A.nnz, dtype=self.A.dtype, device=gb2.device)
        L.check(L.lib().sptrsv_grad_vals(self.p, _ptr(gb2), _ptr(x2), gb2.shape[1], gb2.stride(0),
                                         _ptr(gv)), "sptrsv_grad_vals")
        return gv

    def tt_apply(self, gbp: torch.Tensor, out: torch.Tensor | None = None):
        squeeze = gbp.dim() == 1
        g2 = self._rhs(gbp, self.A.n, self.A.dtype)
        gb = out if out is not None else torch.empty_like(g2)
        L.check(L.lib().sptrsv_tt_apply(self.p, _ptr(g2), _ptr(gb), g2.shape[1], g2.stride(0)),
                "sptrsv_tt_apply")
        return gb.view(-1) if squeeze and out is None else gb

    def __del__(self):
        try:
            if getattr(self, "p", None) and not L.exiting():
                L.lib().sptrsv_plan_destroy(self.p)
        except Exception:
            pass


def _per_system(v, m):
    if v is None:
        return 0
    return int(v[m] if hasattr(v, "__len__") else v)


class BatchPlan:
    """One plan over many independent systems; right-hand sides, solutions
    and gradients are packed (see sptrsv_batch_plan_create).

    The plan copies the systems' values, at creation, into ONE packed tensor
    ``self.vals`` (system m's values are ``vals[vals_offset[m]:vals_offset[m+1]]``)
    and its matrices ``self.mats`` read from slices of it: value changes go
    through ``self.vals`` (or ``self.mats[m].vals``), and the batched autograd
    Function differentiates with respect to exactly this tensor."""

    def __init__(self, mats, Ts=None, nrhs=None, rows_per_warp=None, transpose=False, wait_limit_us=0,
                 rhs_tile=None):
        nmat = len(mats)
        mats = list(mats)
        if nmat:
            dt = mats[0].dtype
            if any(A.dtype != dt for A in mats):
                raise TypeError("all systems of a batch share one value dtype")
            self.vals = torch.cat([A.vals.detach().reshape(-1) for A in mats])
            views, a = [], 0
            for A in mats:
                views.append(Matrix(A.row_ptr, A.col_idx, self.vals[a:a + A.nnz]))
                a += A.nnz
            mats = views
        else:
            self.vals = torch.empty(0, dtype=torch.float32, device="cuda")
        self.mats, self.Ts = mats, list(Ts) if Ts is not None else [None] * nmat
        self.nrhs = [int(k) for k in (nrhs if nrhs is not None else [1] * nmat)]
        descs = (L.sptrsv_csr * max(nmat, 1))()
        tdescs = (L.sptrsv_csr * max(nmat, 1))()
        opts = (L.sptrsv_plan_opts * max(nmat, 1))()
        for m, A in enumerate(self.mats):
            descs[m] = A.desc()
            T = self.Ts[m]
            tdescs[m] = T.desc() if T is not None else L.sptrsv_csr(0, 0, None, None, None, 0)
            rpw = _per_system(rows_per_warp, m)
            tile = _per_system(rhs_tile, m)
            opts[m] = L.sptrsv_plan_opts(L.SPTRSV_MODE_BLOCK, rpw, tile, 1 if transpose else 0, wait_limit_us)
        ks = (C.c_int32 * max(nmat, 1))(*self.nrhs)
        self._h = handle()
        p = L.sptrsv_plan()
        L.check(L.lib().sptrsv_batch_plan_create(self._h.h, nmat, descs, tdescs, ks, opts, C.byref(p)),
                "sptrsv_batch_plan_create")
        self.p = p
        ro = (C.c_int64 * (nmat + 1))()
        vo = (C.c_int64 * (nmat + 1))()
        L.check(L.lib().sptrsv_batch_offsets(p, ro, vo))
        self.rhs_offset = np.array(list(ro), dtype=np.int64)
        self.vals_offset = np.array(list(vo), dtype=np.int64)
        self.dtype = mats[0].dtype if nmat else torch.float32

    def set_geometry(self, rows_per_warp=None, rhs_tile=None, direction="both"):
        """Row-group width and right-hand-side columns per work item, per
        system (list) or for all systems (int); None or 0 keeps the value.
        direction: "both", "forward" or "transpose" (the two directions keep
        separate geometries)."""
        nmat = len(self.mats)

        def arr(v):
            if v is None:
                return None
            return (C.c_int32 * max(nmat, 1))(*[_per_system(v, m) for m in range(nmat)])

        d = {"both": 0, "forward": 1, "transpose": 2}[direction]
        L.check(L.lib().sptrsv_batch_plan_set_direction(self.p, d, arr(rows_per_warp), arr(rhs_tile)),
                "sptrsv_batch_plan_set_direction")

    def set_schedule(self, schedule, direction="both"):
        """Schedule of each system's work items, per system (list) or for
        all systems: "inorder" (rows in row order, 32-row groups one after
        another), "level" (rows in level order, the groups of a level at the
        same time), or None (keep); direction as in set_geometry."""
        nmat = len(self.mats)
        code = {None: 0, "inorder": L.SPTRSV_BATCH_INORDER, "level": L.SPTRSV_BATCH_LEVEL}
        vals = schedule if isinstance(schedule, (list, tuple)) else [schedule] * nmat
        arr = (C.c_int32 * max(nmat, 1))(*[code[v] for v in vals])
        d = {"both": 0, "forward": 1, "transpose": 2}[direction]
        L.check(L.lib().sptrsv_batch_plan_set_schedule(self.p, d, arr), "sptrsv_batch_plan_set_schedule")

    def set_rows_per_warp(self, rpw):
        """Row-group width per system (list) or for all systems (int)."""
        self.set_geometry(rows_per_warp=rpw)

    @property
    def total_rhs(self):
        return int(self.rhs_offset[-1])

    @property
    def total_nnz(self):
        return int(self.vals_offset[-1])

    def _check(self, t, size):
        if t.dtype != self.dtype or not t.is_cuda or t.numel() != size or not t.is_contiguous():
            raise ValueError(f"packed buffer must be a contiguous CUDA {self.dtype} tensor of {size} elements")

    def solve(self, b, out=None):
        self._check(b, self.total_rhs)
        x = out if out is not None else torch.empty_like(b)
        L.check(L.lib().sptrsv_batch_solve(self.p, _ptr(b), _ptr(x)), "sptrsv_batch_solve")
        return x

    def solve_transpose(self, gx, out=None):
        self._check(gx, self.total_rhs)
        gb = out if out is not None else torch.empty_like(gx)
        L.check(L.lib().sptrsv_batch_solve_transpose(self.p, _ptr(gx), _ptr(gb)), "sptrsv_batch_solve_transpose")
        return gb

    def grad_vals(self, gb, x, out=None):
        self._check(gb, self.total_rhs)
        gv = out if out is not None else torch.empty(self.total_nnz, dtype=self.dtype, device=gb.device)
        L.check(L.lib().sptrsv_batch_grad_vals(self.p, _ptr(gb), _ptr(x), _ptr(gv)), "sptrsv_batch_grad_vals")
        return gv

    def tt_apply(self, gbp, out=None):
        self._check(gbp, self.total_rhs)
        gb = out if out is not None else torch.empty_like(gbp)
        L.check(L.lib().sptrsv_batch_tt_apply(self.p, _ptr(gbp), _ptr(gb)), "sptrsv_batch_tt_apply")
        return gb

    def step_host(self, b, w, x, gb, gvals):
        """One forward + adjoint step from HOST buffers (CPU tensors of the
        plan's dtype, contiguous; page-locked for overlapped copies): x =
        solve(b), gb = dL/db and gvals = dL/dvals for dL/dx = w.  Returns
        without waiting; the buffers must stay untouched until step_wait()."""
        for t, size in ((b, self.total_rhs), (w, self.total_rhs), (x, self.total_rhs), (gb, self.total_rhs),
                        (gvals, self.total_nnz)):
            if t.dtype != self.dtype or t.is_cuda or t.numel() != size or not t.is_contiguous():
                raise ValueError(f"host buffer must be a contiguous CPU {self.dtype} tensor of {size} elements")
        L.check(L.lib().sptrsv_batch_step_host(self.p, _ptr(b), _ptr(w), _ptr(x), _ptr(gb), _ptr(gvals)),
                "sptrsv_batch_step_host")

    def step_wait(self):
        """Waits for the steps enqueued by step_host; raises on a device error."""
        L.check(L.lib().sptrsv_batch_step_wait(self.p), "sptrsv_batch_step_wait")

    def withhold(self, m: int, i: int):
        """Test hook of the bounded waits: row i of system m is never
        published by the next solves (m = -1 clears it)."""
        row = -1 if m < 0 else int(sum(A.n for A in self.mats[:m])) + int(i)
        L.check(L.lib().sptrsv_debug_withhold_row(self.p, row))

    def trace(self):
        """[nmat, 3] int64: start ns, end ns, SM of every system in the last
        batched solve."""
        nmat = len(self.mats)
        buf = (C.c_int64 * (3 * max(nmat, 1)))()
        L.check(L.lib().sptrsv_batch_trace(self.p, buf), "sptrsv_batch_trace")
        return np.array(list(buf), dtype=np.int64)[: 3 * nmat].reshape(nmat, 3)

    def unpack(self, packed, m):
        a, b = int(self.rhs_offset[m]), int(self.rhs_offset[m + 1])
        return packed[a:b].view(self.mats[m].n, self.nrhs[m])

    def __del__(self):
        try:
            if getattr(self, "p", None) and not L.exiting():
                L.lib().sptrsv_plan_destroy(self.p)
        except Exception:
            pass
