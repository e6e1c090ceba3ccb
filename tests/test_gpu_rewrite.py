"""Equation rewriting on the GPU vs the CPU oracle: L' and T patterns must
match bit for bit; values too (same IEEE operation order), FP32 values are
the oracle's FP64 values rounded once."""
import numpy as np
import pytest

import oracle
import synthetic as S
from helpers import relerr, widened

pytestmark = pytest.mark.gpu


def _run(A_h, rows, tg, dtype=np.float64):
    import paper_2609_40159_gb300 as P
    A = P.Matrix.from_host(A_h)
    an = P.analyze(A)
    ref_lev, _ = oracle.levels(widened(A_h))
    assert np.array_equal(an.lev.cpu().numpy(), ref_lev)
    Lp, T = P.rewrite(A, an.lev, rows, tg)
    Lr, Tr = oracle.rewrite(widened(A_h), ref_lev, rows, tg)
    assert np.array_equal(Lp.row_ptr.cpu().numpy(), Lr.row_ptr)
    assert np.array_equal(Lp.col_idx.cpu().numpy(), Lr.col_idx)
    assert np.array_equal(T.row_ptr.cpu().numpy(), Tr.row_ptr)
    assert np.array_equal(T.col_idx.cpu().numpy(), Tr.col_idx)
    assert np.array_equal(Lp.vals.cpu().numpy(), Lr.vals.astype(dtype))
    assert np.array_equal(T.vals.cpu().numpy(), Tr.vals.astype(dtype))
    return P, A, Lp, T, Lr, Tr


def test_rewrite_cfg0_small_levels():
    A_h = S.band_random(2000, 64, 0, 8, seed=0)
    an = oracle.analyze(A_h)
    rows, tg = S.small_levels_list(an["nlevels"], an["level_ptr"], an["perm"], 4, 8)
    P, A, Lp, T, Lr, Tr = _run(A_h, rows, tg)
    # the rewritten system has the original solution and fewer levels
    b = S.rhs(A_h.n, 1, seed=3)
    x = oracle.solve(A_h, b)
    assert relerr(oracle.solve_rewritten(Lr, Tr, b), x) <= 1e-12
    an2 = P.analyze(Lp)
    assert an2.nlevels < an["nlevels"]


def test_rewrite_lap2d_full_narrowest():
    A_h = S.lap2d(1024)
    an = oracle.analyze(A_h)
    rows, tg = S.narrowest_levels_list(an["nlevels"], an["level_ptr"], an["perm"], 0.01, 8)
    assert len(rows) >= 10486
    _run(A_h, rows, tg)


@pytest.mark.parametrize("seed", [0, 1])
def test_rewrite_deep_targets_and_duplicates(seed):
    A_h = S.band_random(20_000, 300, 4, 16, seed=seed)
    lev, _ = oracle.levels(A_h)
    rng = np.random.default_rng(seed)
    cand = np.nonzero(lev >= 2)[0]
    rows = rng.choice(cand, size=400, replace=False).astype(np.int32)
    tg = (lev[rows] - rng.integers(1, 4, size=400)).clip(0).astype(np.int32)
    rows = np.concatenate([rows, rows[:50]])
    tg = np.concatenate([tg, np.maximum(tg[:50] - 1, 0)]).astype(np.int32)
    _run(A_h, rows, tg)


def test_rewrite_fp32_values_rounded_once():
    A_h = S.band_random(8000, 128, 4, 16, seed=4).astype(np.float32)
    lev, nl = oracle.levels(A_h)
    perm, lp, _ = oracle.partition(A_h, lev, nl)
    rows, tg = S.narrowest_levels_list(nl, lp, perm, 0.02, 8)
    _run(A_h, rows, tg, dtype=np.float32)


def test_rewrite_powerlaw():
    A_h = S.powerlaw(200_000, alpha=2.1, seed=2)
    an = oracle.analyze(A_h)
    rows, tg = S.narrowest_levels_list(an["nlevels"], an["level_ptr"], an["perm"], 0.01, 8)
    _run(A_h, rows, tg)


def test_rewrite_errors():
    import paper_2609_40159_gb300 as P
    A_h = S.band_random(500, 10, 1, 4, seed=2)
    A = P.Matrix.from_host(A_h)
    an = P.analyze(A)
    lev = an.lev.cpu().numpy()
    z = int(np.nonzero(lev == 0)[0][0])
    i = int(np.nonzero(lev >= 2)[0][0])
    with pytest.raises(P._lib.SpTRSVError) as e:
        P.rewrite(A, an.lev, [i, z], [0, 0])
    assert e.value.status == P._lib.SPTRSV_ETARGET
    with pytest.raises(P._lib.SpTRSVError) as e:
        P.rewrite(A, an.lev, [i], [int(lev[i])])
    assert e.value.status == P._lib.SPTRSV_ETARGET
    with pytest.raises(P._lib.SpTRSVError) as e:
        P.rewrite(A, an.lev, [A_h.n + 3], [0])
    assert e.value.status == P._lib.SPTRSV_EINVAL
    Lp, T = P.rewrite(A, an.lev, [], [])
    assert np.array_equal(Lp.col_idx.cpu().numpy(), A_h.col_idx) and T.nnz == 0
