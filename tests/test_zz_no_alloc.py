"""The allocation-free entry point sptrsv_solve_noalloc.

It serves callers that cannot allocate device memory when they solve; its
scratch is a static device array shared by all calls.  Checked here through
the C ABI against the regular sync-free solve (sptrsv_solve on a plan) with
the tolerances of the other solve tests, on two calls in a row (the second
call finds the first call's flags and counters in the shared scratch), and
for the size limit.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _noalloc(A, b, x):
    from paper_2609_40159_gb300 import _lib as L
    from paper_2609_40159_gb300.api import _ptr
    stream = torch.cuda.current_stream().cuda_stream
    return L.lib().sptrsv_solve_noalloc(C.byref(A.desc()), _ptr(b), _ptr(x), b.shape[1],
                                        b.stride(0), C.c_void_p(stream))


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-12), (np.float32, 1e-5)], ids=["f64", "f32"])
def test_noalloc_matches_regular_solve_twice(dt, tol):
    import paper_2609_40159_gb300 as P
    A_h = S.band_random(70_003, 96, 2, 14, seed=21).astype(dt)
    A = P.Matrix.from_host(A_h)
    plan = P.Plan(A, mode="syncfree")
    for call, k in enumerate((3, 1)):
        b = torch.as_tensor(S.rhs(A_h.n, k, seed=30 + call, dtype=dt)).cuda()
        ref = plan.solve(b)
        x = torch.full_like(b, float("nan"))
        st = _noalloc(A, b, x)
        assert st == 0, f"call {call}: status {st}"
        r = ref.double().cpu().numpy()
        err = np.linalg.norm(x.double().cpu().numpy() - r) / np.linalg.norm(r)
        assert err <= tol, (call, err)


def test_noalloc_rejects_too_many_rows():
    from paper_2609_40159_gb300 import _lib as L
    d = L.sptrsv_csr(L.SPTRSV_NOALLOC_MAX_ROWS + 1, 0, None, None, None, L.SPTRSV_F64)
    st = L.lib().sptrsv_solve_noalloc(C.byref(d), None, None, 1, 1, None)
    assert st == L.SPTRSV_ENOTSUP
