"""The allocation-free entry point sptrsv_solve_noalloc.

It serves callers that cannot allocate device memory when they solve (an
application whose own pool owns the device memory, a real-time loop that
cannot take cudaMalloc's implicit synchronisation, a plug-in whose host
forbids allocation); its scratch is a static device array shared by all
calls.  Checked here through the C ABI against the regular solve entry point
(sptrsv_solve on a sync-free plan) and against the oracle, with the
tolerances of the other solve tests, on two calls in a row (the second call
finds the first call's flags and counters in the shared scratch); then the
size limit and malformed matrices, which must come back with an error status
and leave the device usable.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu


def _noalloc(A, b, x):
    from paper_2609_40159_gb300 import _lib as L
    from paper_2609_40159_gb300.api import _ptr
    stream = torch.cuda.current_stream().cuda_stream
    return L.lib().sptrsv_solve_noalloc(C.byref(A.desc()), _ptr(b), _ptr(x), b.shape[1],
                                        b.stride(0), C.c_void_p(stream))


def _relerr(x, ref):
    x = x.double().cpu().numpy() if torch.is_tensor(x) else np.asarray(x, np.float64)
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-12), (np.float32, 1e-5)], ids=["f64", "f32"])
def test_noalloc_matches_regular_solve_twice(dt, tol):
    import paper_2609_40159_gb300 as P
    A_h = S.band_random(70_003, 96, 2, 14, seed=21).astype(dt)
    A64 = S.CSR(A_h.n, A_h.row_ptr, A_h.col_idx, A_h.vals.astype(np.float64))
    A = P.Matrix.from_host(A_h)
    plan = P.Plan(A, mode="syncfree")
    for call, k in enumerate((3, 1)):
        b_h = S.rhs(A_h.n, k, seed=30 + call, dtype=dt)
        b = torch.as_tensor(b_h).cuda()
        ref = plan.solve(b)
        x = torch.full_like(b, float("nan"))
        st = _noalloc(A, b, x)
        assert st == 0, f"call {call}: status {st}"
        assert _relerr(x, ref.double().cpu().numpy()) <= tol, call
        assert _relerr(x, oracle.solve(A64, b_h)) <= tol, call
    assert P.handle().status() == 0


def test_noalloc_rejects_too_many_rows():
    from paper_2609_40159_gb300 import _lib as L
    d = L.sptrsv_csr(L.SPTRSV_NOALLOC_MAX_ROWS + 1, 0, None, None, None, L.SPTRSV_F64)
    st = L.lib().sptrsv_solve_noalloc(C.byref(d), None, None, 1, 1, None)
    assert st == L.SPTRSV_ENOTSUP


def _malformed(kind):
    """A 2,000-row system with one bad row (built on the CPU, all arrays
    in-bounds): every index the kernel can touch stays inside the arrays."""
    A = S.band_random(2000, 32, 1, 6, seed=5)
    rp, ci, v = A.row_ptr.copy(), A.col_idx.copy(), A.vals.copy()
    i = 900
    if kind == "diag_not_last":
        # a row whose last off-diagonal leaves room below the diagonal
        while ci[rp[i + 1] - 2] + 1 >= i:
            i += 1
    a, e = int(rp[i]), int(rp[i + 1])
    if kind == "upper":       # an off-diagonal column above the diagonal
        ci[a] = i + 40
    elif kind == "negative":  # a negative column
        ci[a] = -3
    elif kind == "diag_not_last":  # the last entry is not the diagonal
        ci[e - 1] = ci[e - 2] + 1
    return S.CSR(A.n, rp, ci, v)


@pytest.mark.parametrize("kind,code", [("upper", "SPTRSV_ENOTLOWER"), ("negative", "SPTRSV_ENOTLOWER"),
                                       ("diag_not_last", "SPTRSV_EDIAG")])
def test_noalloc_reports_malformed_rows(kind, code):
    import paper_2609_40159_gb300 as P
    from paper_2609_40159_gb300 import _lib as L
    bad = P.Matrix.from_host(_malformed(kind))
    b = torch.as_tensor(S.rhs(bad.n, 1, seed=3)).cuda()
    x = torch.zeros_like(b)
    assert _noalloc(bad, b, x) == getattr(L, code)
    # the device and the shared scratch are usable again at once
    good_h = S.band_random(2000, 32, 1, 6, seed=5)
    good = P.Matrix.from_host(good_h)
    assert _noalloc(good, b, x) == 0
    assert _relerr(x, oracle.solve(good_h, b.cpu().numpy())) <= 1e-12
