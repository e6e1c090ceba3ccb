"""The bounds-checked debug variant of the library (SPTRSV_CHECKED) on the
GPU, in a child process that loads it in place of the product library:
its reporting path records SPTRSV_ERANGE for an index outside its range,
and on valid inputs every solve mode, the batched solve in both schedules,
the analysis and the rewrite find no out-of-range index and give the
oracle's results."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = '''
import numpy as np
import torch

import oracle
import synthetic as S
from paper_2609_40159_gb300 import _lib


def rel(x, r):
    return np.linalg.norm(np.asarray(x, np.float64).reshape(r.shape) - r) / np.linalg.norm(r)


def main():
    _lib._lib = _lib.load(_lib.LIB_CHECKED_PATH)
    import paper_2609_40159_gb300 as P
    assert _lib.lib().sptrsv_checked_build() == 1
    h = P.handle()
    # the reporting path: an index outside [0, n) is recorded, one inside is not
    _lib.check(_lib.lib().sptrsv_debug_check_index(h.h, 5, 8))
    assert h.status() == 0
    _lib.check(_lib.lib().sptrsv_debug_check_index(h.h, 9, 8))
    assert h.status() == _lib.SPTRSV_ERANGE
    _lib.check(_lib.lib().sptrsv_debug_check_index(h.h, -1, 8))
    assert h.status() == _lib.SPTRSV_ERANGE
    assert h.status() == 0
    cases = [S.lap2d(60), S.band_random(5000, 80, 1, 12, seed=3), S.powerlaw(20_000, seed=4)]
    for A_h in cases:
        A = P.Matrix.from_host(A_h)
        an = P.analyze(A)
        ref = oracle.analyze(A_h)
        assert np.array_equal(an.lev.cpu().numpy(), ref["lev"])
        rows, tg = S.narrowest_levels_list(ref["nlevels"], ref["level_ptr"], ref["perm"], 0.02, 8)
        Lp, T = P.rewrite(A, an.lev, rows, tg)
        b_h = S.rhs(A_h.n, 3, seed=1)
        b = torch.as_tensor(b_h).cuda()
        x_ref, g_ref = oracle.solve(A_h, b_h), oracle.solve_transpose(A_h, b_h)
        for M, TT in ((A, None), (Lp, T)):
            plan = P.Plan(M, TT, transpose=True)
            for mode in ("level_launch", "level", "syncfree", "block", "hybrid"):
                for rpw in (1, 32):
                    plan.set(mode, rpw, 4)
                    assert rel(plan.solve(b).cpu().numpy(), x_ref) <= 1e-12, (mode, rpw)
                    if TT is None:
                        assert rel(plan.solve_transpose(b).cpu().numpy(), g_ref) <= 1e-12, (mode, rpw)
                    assert h.status() == 0, (mode, rpw)
    items = S.batch_spec(nmat=12, seed=7, n_lo=300, n_hi=5000, dtype=np.float64)
    bp = P.BatchPlan([P.Matrix.from_host(it.A) for it in items], None, [it.nrhs for it in items], transpose=True)
    bb = torch.cat([torch.as_tensor(it.b).reshape(-1) for it in items]).cuda()
    for sched in ("inorder", "level"):
        bp.set_schedule(sched)
        x = bp.solve(bb)
        g = bp.solve_transpose(bb)
        assert h.status() == 0, sched
        for m, it in enumerate(items):
            assert rel(bp.unpack(x, m).cpu().numpy(), oracle.solve(it.A, it.b)) <= 1e-12, (sched, m)
            assert rel(bp.unpack(g, m).cpu().numpy(), oracle.solve_transpose(it.A, it.b)) <= 1e-12, (sched, m)
    torch.cuda.synchronize()
    del bp, plan
    P.api._handles.clear()  # the cached handle too
    print("checked-ok", flush=True)


main()  # the plans and handles die here, before the interpreter tears CUDA down
'''


def test_checked_variant_on_gpu():
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.path.join(ROOT, "tests") + os.pathsep +
               os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "checked-ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
