"""Level analysis and validation on the GPU vs the CPU oracle: levels, the
level partition, costs and the statistics must match bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from helpers import cases_small, widened

pytestmark = pytest.mark.gpu


def _check(A_h):
    import paper_2609_40159_gb300 as P
    A = P.Matrix.from_host(A_h)
    an = P.analyze(A)
    ref = oracle.analyze(A_h)
    assert an.nlevels == ref["nlevels"]
    assert np.array_equal(an.lev.cpu().numpy(), ref["lev"])
    assert np.array_equal(an.perm.cpu().numpy(), ref["perm"])
    assert np.array_equal(an.level_ptr.cpu().numpy(), ref["level_ptr"])
    assert np.array_equal(an.cost.cpu().numpy(), ref["cost"])
    assert np.array_equal(an.stats, ref["stats"]), (an.stats, ref["stats"])  # bit-exact
    return an


@pytest.mark.parametrize("name,A", cases_small(), ids=[c[0] for c in cases_small()])
def test_analyze_small(name, A):
    _check(A)


def test_analyze_fp32_same_as_fp64():
    _check(S.band_random(5000, 100, 4, 16, seed=9).astype(np.float32))


def test_analyze_long_rows_with_chains_in_chunk():
    """Rows longer than the cooperative threshold (up to 40 off-diagonals in a
    band of 48) that depend on rows of their own 32-row chunk as well as on
    earlier chunks, mixed with short rows: the warp-wide polls, the
    per-row early publishing and the chunk's max-plus sweep together, vs the
    oracle."""
    _check(S.band_random(20_000, 48, 20, 40, seed=13))
    _check(S.band_random(9_001, 40, 0, 39, seed=14))


def test_analysis_bounded_wait_reports_timeout():
    """A row whose level is never published (test hook): the level analysis
    gives up after the hook's wait limit with SPTRSV_ETIMEOUT (returned by
    the call and recorded in the status word), the context stays usable, and
    the next analysis equals the oracle's again."""
    import paper_2609_40159_gb300 as P
    A_h = S.band_random(20_000, 48, 1, 8, seed=12)
    A = P.Matrix.from_host(A_h)
    h = P.handle()
    assert h.status() == 0
    h.withhold_level(7000, wait_limit_us=20_000)
    try:
        with pytest.raises(P.SpTRSVError) as e:
            P.analyze(A)
        assert e.value.status == P._lib.SPTRSV_ETIMEOUT
        assert h.status() == P._lib.SPTRSV_ETIMEOUT
    finally:
        h.withhold_level(-1)
    _check(A_h)
    assert h.status() == 0


@pytest.mark.parametrize("gen", ["lap2d_1024", "lap3d_128", "powerlaw_4M"])
def test_analyze_full_size(gen):
    A = {"lap2d_1024": lambda: S.lap2d(1024), "lap3d_128": lambda: S.lap3d(128),
         "powerlaw_4M": lambda: S.powerlaw(4_000_000, alpha=2.1, seed=2)}[gen]()
    an = _check(A)
    if gen == "lap2d_1024":
        assert an.nlevels == 2047
    if gen == "lap3d_128":
        assert an.nlevels == 382


def test_analyze_deterministic():
    import paper_2609_40159_gb300 as P
    A = P.Matrix.from_host(S.powerlaw(300_000, seed=4))
    a1, a2 = P.analyze(A), P.analyze(A)
    for f in ("lev", "perm", "level_ptr", "cost"):
        assert torch.equal(getattr(a1, f), getattr(a2, f))
    assert np.array_equal(a1.stats, a2.stats)


def test_empty_matrix():
    import paper_2609_40159_gb300 as P
    A = P.Matrix(torch.zeros(1, dtype=torch.int32, device="cuda"),
                 torch.zeros(0, dtype=torch.int32, device="cuda"),
                 torch.zeros(0, dtype=torch.float64, device="cuda"))
    an = P.analyze(A)
    assert an.nlevels == 0 and np.all(an.stats == 0)


def _broken(kind):
    A = S.band_random(300, 10, 1, 4, seed=1)
    rp, ci, v = A.row_ptr.copy(), A.col_idx.copy(), A.vals.copy()
    if kind == "zero_diag":
        v[rp[41] - 1] = 0.0
    elif kind == "upper":
        ci[rp[77]] = 200
    elif kind == "unsorted":
        a = rp[150]
        ci[a], ci[a + 1] = ci[a + 1], ci[a]
    elif kind == "no_diag":
        ci[rp[201] - 1] = 199
    elif kind == "negative":
        ci[rp[90]] = -1
    elif kind == "repeated":
        ci[rp[120] + 1] = ci[rp[120]]
    elif kind == "range_before_order":  # one position both negative and decreasing
        ci[rp[130] + 1] = -5
    elif kind == "rowptr_decreasing":
        rp[61] = rp[60] - 1
    elif kind == "first_row_wins":
        ci[rp[250]] = 280
        v[rp[13] - 1] = 0.0
    elif kind == "empty_row":
        a, e = int(rp[170]), int(rp[171])
        rp[171:] -= e - a
        ci, v = np.delete(ci, np.s_[a:e]), np.delete(v, np.s_[a:e])
    return S.CSR(A.n, rp, ci, v)


@pytest.mark.parametrize("kind", ["zero_diag", "upper", "unsorted", "no_diag", "negative", "repeated",
                                  "range_before_order", "rowptr_decreasing", "first_row_wins", "empty_row"])
def test_validate_codes_match_oracle(kind):
    import paper_2609_40159_gb300 as P
    A_h = _broken(kind)
    st, row = P.validate(P.Matrix.from_host(A_h))
    assert (st, row) == oracle.validate(A_h)
    assert st != 0
    with pytest.raises(P._lib.SpTRSVError):
        P.analyze(P.Matrix.from_host(A_h))


@pytest.mark.parametrize("gen", ["band", "lap2d_256", "powerlaw"])
def test_incremental_after_rewrite(gen):
    """Rewriting changes only the listed rows, so every earlier row keeps its
    level: the incremental analysis of L' from the first rewritten row,
    seeded with L's levels, equals the full analysis of L' and the oracle
    (levels, partition, costs and statistics bit for bit)."""
    import paper_2609_40159_gb300 as P
    A_h = {"band": lambda: S.band_random(20_000, 64, 2, 10, seed=21),
           "lap2d_256": lambda: S.lap2d(256),
           "powerlaw": lambda: S.powerlaw(100_000, seed=22)}[gen]()
    A = P.Matrix.from_host(A_h)
    an = P.analyze(A)
    rows, tg = S.narrowest_levels_list(an.nlevels, an.level_ptr.cpu().numpy(), an.perm.cpu().numpy(), 0.01, 8)
    Lp, T = P.rewrite(A, an.lev, rows, tg)
    first = int(np.min(rows))
    full = P.analyze(Lp)
    inc = P.analyze(Lp, prev_lev=an.lev, first_row=first)
    for f in ("lev", "perm", "level_ptr", "cost"):
        assert torch.equal(getattr(full, f), getattr(inc, f)), f
    assert inc.nlevels == full.nlevels and np.array_equal(inc.stats, full.stats)
    ref = oracle.analyze(oracle.rewrite(A_h, an.lev.cpu().numpy(), rows, tg)[0])
    assert np.array_equal(inc.lev.cpu().numpy(), ref["lev"])
    assert np.array_equal(inc.stats, ref["stats"])
    # first row past the end: nothing recomputed beyond the last partial chunk
    same = P.analyze(Lp, prev_lev=full.lev, first_row=Lp.n)
    assert torch.equal(same.lev, full.lev)


def _check_same_analysis(inc, full, ref):
    for f in ("lev", "perm", "level_ptr", "cost"):
        assert torch.equal(getattr(full, f), getattr(inc, f)), f
    assert inc.nlevels == full.nlevels and np.array_equal(inc.stats, full.stats)
    assert np.array_equal(inc.lev.cpu().numpy(), ref["lev"])
    assert np.array_equal(inc.perm.cpu().numpy(), ref["perm"])
    assert np.array_equal(inc.stats, ref["stats"])


@pytest.mark.parametrize("gen", ["lap2d_256", "band", "powerlaw"])
def test_incremental_single_row_moves(gen):
    """The environment's step: one more row rewritten at a time (the rewrite
    list grows by one row per move; every listed row is rewritten from the
    original rows, so consecutive systems differ in that row only).  After
    every move the incremental analysis from that row, seeded with the
    previous levels, equals the full analysis and the oracle bit for bit."""
    import paper_2609_40159_gb300 as P
    A_h = {"band": lambda: S.band_random(20_000, 64, 2, 10, seed=21),
           "lap2d_256": lambda: S.lap2d(256),
           "powerlaw": lambda: S.powerlaw(100_000, seed=22)}[gen]()
    A = P.Matrix.from_host(A_h)
    an0 = P.analyze(A)
    lev0 = an0.lev.cpu().numpy()
    rng = np.random.default_rng(5)
    cand = np.flatnonzero(lev0 >= 2)
    rows, tgs = [], []
    prev = an0
    for move in range(12):
        i = int(rng.choice(cand))
        rows.append(i)
        tgs.append(int(rng.integers(max(0, lev0[i] - 6), lev0[i])))
        Lp, _ = P.rewrite(A, an0.lev, rows, tgs)
        inc = P.analyze(Lp, prev_lev=prev.lev, first_row=i)
        full = P.analyze(Lp)
        ref = oracle.analyze(oracle.rewrite(A_h, lev0, rows, tgs)[0])
        _check_same_analysis(inc, full, ref)
        prev = inc


def test_incremental_level_collapse_falls_back():
    """A move that empties a level renumbers every later level: in a chain
    (one row per level) rewriting row 1500 two levels up moves every row after
    it, a propagation longer than the fixpoint's round limit, finished by the
    full pass from the first unsettled row; still equal to the full analysis
    and the oracle."""
    import paper_2609_40159_gb300 as P
    A_h = S.chain(3000, seed=4)
    A = P.Matrix.from_host(A_h)
    an0 = P.analyze(A)
    Lp, _ = P.rewrite(A, an0.lev, [1500], [1498])
    inc = P.analyze(Lp, prev_lev=an0.lev, first_row=1500)
    full = P.analyze(Lp)
    assert full.nlevels == 2998  # row 1500 lands on level 1498; every later row moves up two levels
    _check_same_analysis(inc, full, oracle.analyze(oracle.rewrite(A_h, an0.lev.cpu().numpy(), [1500], [1498])[0]))


def test_incremental_bounded_wait_reports_timeout():
    """The grid-wide barrier of the incremental analysis is bounded too: with
    the analysis test hook one block never arrives, the others give up after
    the hook's limit, the call returns SPTRSV_ETIMEOUT and the next one is
    right."""
    import paper_2609_40159_gb300 as P
    A_h = S.band_random(300_000, 64, 2, 10, seed=23)
    A = P.Matrix.from_host(A_h)
    an0 = P.analyze(A)
    lev0 = an0.lev.cpu().numpy()
    i = int(np.flatnonzero(lev0 >= 3)[1000])
    Lp, _ = P.rewrite(A, an0.lev, [i], [int(lev0[i]) - 2])
    h = P.handle()
    h.withhold_level(0, wait_limit_us=20_000)
    try:
        with pytest.raises(P.SpTRSVError) as e:
            P.analyze(Lp, prev_lev=an0.lev, first_row=i)
        assert e.value.status == P._lib.SPTRSV_ETIMEOUT
        assert h.status() == P._lib.SPTRSV_ETIMEOUT
    finally:
        h.withhold_level(-1)
    inc = P.analyze(Lp, prev_lev=an0.lev, first_row=i)
    _check_same_analysis(inc, P.analyze(Lp), oracle.analyze(oracle.rewrite(A_h, lev0, [i], [int(lev0[i]) - 2])[0]))
    assert h.status() == 0


def test_incremental_bad_first_row():
    import ctypes as C
    import paper_2609_40159_gb300 as P
    from paper_2609_40159_gb300 import _lib as L
    A = P.Matrix.from_host(S.band_random(1000, 16, 1, 4, seed=3))
    an = P.analyze(A)
    nl = C.c_int32(0)
    st = L.lib().sptrsv_analyze_incremental(P.handle().h, C.byref(A.desc()), A.n + 1, an.lev.data_ptr(),
                                            an.perm.data_ptr(), an.level_ptr.data_ptr(), an.cost.data_ptr(),
                                            C.byref(nl), None)
    assert st == L.SPTRSV_EINVAL


@pytest.mark.parametrize("gen", ["cfg0", "lap2d_1024", "powerlaw_1M", "band_fp32"])
def test_level_summary_matches_oracle(gen):
    """Thin flags, the fewest-dependency row of every level and the thin-level
    summary (the environment's observation after a rewrite) equal the
    oracle's, at the paper's threshold and at a threshold equal to a level
    cost (strict comparison)."""
    import paper_2609_40159_gb300 as P
    A_h = {"cfg0": lambda: S.band_random(2000, 64, 0, 8, seed=0),
           "lap2d_1024": lambda: S.lap2d(1024),
           "powerlaw_1M": lambda: S.powerlaw(1_000_000, seed=5),
           "band_fp32": lambda: S.band_random(50_000, 300, 4, 16, seed=6).astype(np.float32)}[gen]()
    A = P.Matrix.from_host(A_h)
    an = P.analyze(A)
    ref = oracle.analyze(widened(A_h) if A_h.vals.dtype != np.float64 else A_h)
    for thr in (None, float(ref["cost"][len(ref["cost"]) // 2])):
        thin, pick, out = P.level_summary(A, an, thr)
        rthin, rpick, rout = oracle.level_summary(A_h, ref, thr)
        assert np.array_equal(thin.cpu().numpy(), rthin)
        assert np.array_equal(pick.cpu().numpy(), rpick)
        assert np.array_equal(out, rout)
