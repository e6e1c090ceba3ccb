"""Forward and transpose solves, value gradients and the autograd Function on
the GPU vs the CPU oracle.  x is judged by normwise relative error: 1e-12 for
FP64, 1e-5 for FP32 values with FP32 accumulation (against the FP64 solution
of the system the FP32 values define)."""
import functools

import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from helpers import TOL, cases_small, relerr, widened

pytestmark = pytest.mark.gpu

MODES = ["level_launch", "level", "syncfree", "block", "hybrid"]
RPWS = [1, 4, 32]
KS = [1, 3, 32]


@functools.lru_cache(maxsize=None)
def _case(name):
    return dict(cases_small())[name]


@functools.lru_cache(maxsize=None)
def _ref(name, k, dt):
    A_h = _case(name).astype(dt)
    b = S.rhs(A_h.n, k, seed=k, dtype=dt)
    return A_h, b, oracle.solve(widened(A_h), b), oracle.solve_transpose(widened(A_h), b)


NAMES = [c[0] for c in cases_small()]


@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("name", NAMES)
def test_solve_all_modes(name, dt):
    import paper_2609_40159_gb300 as P
    for k in KS:
        A_h, b_h, x_ref, g_ref = _ref(name, k, dt)
        A = P.Matrix.from_host(A_h)
        b = torch.as_tensor(b_h).cuda()
        plan = P.Plan(A, transpose=True)
        for mode in MODES:
            for rpw in RPWS:
                for kt in (1, 4, 16):
                    if mode == "level_launch" and (rpw, kt) != (32, 16):
                        continue
                    plan.set(mode, rpw, kt)
                    x = plan.solve(b)
                    assert P.handle().status() == 0, (mode, rpw, kt, k)
                    e = relerr(x.cpu().numpy(), x_ref)
                    assert e <= TOL[dt], (mode, rpw, kt, k, e)
                    g = plan.solve_transpose(b)
                    assert P.handle().status() == 0, ("T", mode, rpw, kt, k)
                    e = relerr(g.cpu().numpy(), g_ref)
                    assert e <= TOL[dt], ("T", mode, rpw, kt, k, e)
        assert P.handle().status() == 0


@pytest.mark.parametrize("name", ["cfg0", "lap2d_97", "powerlaw", "long_row"])
def test_grad_vals(name):
    import paper_2609_40159_gb300 as P
    A_h = _case(name)
    b_h = S.rhs(A_h.n, 4, seed=1)
    w_h = S.rhs(A_h.n, 4, seed=2)
    A = P.Matrix.from_host(A_h)
    plan = P.Plan(A, transpose=True)
    x = plan.solve(torch.as_tensor(b_h).cuda())
    gb = plan.solve_transpose(torch.as_tensor(w_h).cuda())
    gv = plan.grad_vals(gb, x).cpu().numpy()
    ref = oracle.grad_vals(A_h, oracle.solve_transpose(A_h, w_h), oracle.solve(A_h, b_h))
    assert relerr(gv, ref) <= 1e-12


def test_rewritten_solve_and_adjoint_identity():
    import paper_2609_40159_gb300 as P
    A_h = S.band_random(20_000, 200, 4, 16, seed=3)
    an = oracle.analyze(A_h)
    rows, tg = S.narrowest_levels_list(an["nlevels"], an["level_ptr"], an["perm"], 0.02, 8)
    A = P.Matrix.from_host(A_h)
    Lp, T = P.rewrite(A, P.analyze(A).lev, rows, tg)
    b_h = S.rhs(A_h.n, 3, seed=5)
    b = torch.as_tensor(b_h).cuda()
    x_ref = oracle.solve(A_h, b_h)
    plan = P.Plan(Lp, T, transpose=True)
    orig = P.Plan(A, transpose=True)
    for mode in MODES:
        plan.set(mode, 32, 4)
        assert relerr(plan.solve(b).cpu().numpy(), x_ref) <= 1e-12, mode
        gbp = plan.solve_transpose(b)
        gb = plan.tt_apply(gbp).cpu().numpy()
        assert relerr(gb, orig.solve_transpose(b).cpu().numpy()) <= 1e-12, mode
        assert relerr(gb, oracle.solve_transpose(A_h, b_h)) <= 1e-12


def test_tt_apply_is_deterministic():
    """T^T of the adjoint is a gather over T's columns (each element of g_b
    written once, in a fixed order): repeated applications, single-system
    and batched, are bit-identical, and equal the oracle's."""
    import paper_2609_40159_gb300 as P
    A_h = S.lap2d(120)
    an = oracle.analyze(A_h)
    rows, tg = S.narrowest_levels_list(an["nlevels"], an["level_ptr"], an["perm"], 0.05, 8)
    A = P.Matrix.from_host(A_h)
    Lp, T = P.rewrite(A, P.analyze(A).lev, rows, tg)
    assert T.nnz > 0
    Lp_o, T_o = oracle.rewrite(A_h, an["lev"], rows, tg)
    g_h = S.rhs(A_h.n, 5, seed=7)
    g = torch.as_tensor(g_h).cuda()
    ref = oracle.tt_apply(T_o, g_h)
    plan = P.Plan(Lp, T, transpose=True)
    first = plan.tt_apply(g)
    for _ in range(3):
        assert torch.equal(plan.tt_apply(g), first)
    assert relerr(first.cpu().numpy(), ref) <= 1e-12
    bp = P.BatchPlan([Lp, Lp], [T, T], [5, 5], transpose=True)
    gg = torch.cat([g.reshape(-1), g.reshape(-1)])
    bfirst = bp.tt_apply(gg)
    for _ in range(3):
        assert torch.equal(bp.tt_apply(gg), bfirst)
    for m in range(2):
        assert relerr(bp.unpack(bfirst, m).cpu().numpy(), ref) <= 1e-12
    assert P.handle().status() == 0


def test_autograd_finite_differences_lap3d_block():
    import paper_2609_40159_gb300 as P
    A_h = S.leading_block(S.lap3d(128), 4096)
    A = P.Matrix.from_host(A_h)
    plan = P.Plan(A, transpose=True)
    b = torch.as_tensor(S.rhs(A_h.n, 8, seed=4)).cuda().requires_grad_(True)
    w = torch.as_tensor(S.rhs(A_h.n, 8, seed=5)).cuda()
    vals = A.vals
    vals.requires_grad_(True)
    x = P.SpTRSVFunction.apply(vals, b, plan)
    (x * w).sum().backward()
    gv, gb = vals.grad.detach().clone(), b.grad.detach().clone()
    vals.requires_grad_(False)

    def loss(bb):
        with torch.no_grad():
            return float((plan.solve(bb) * w).sum())

    rng = np.random.default_rng(0)
    for p in rng.choice(A_h.nnz, size=24, replace=False):
        h = 1e-6 * max(1.0, abs(float(A.vals[p])))
        old = float(A.vals[p])
        with torch.no_grad():
            A.vals[p] = old + h
            fp = loss(b.detach())
            A.vals[p] = old - h
            fm = loss(b.detach())
            A.vals[p] = old
        fd = (fp - fm) / (2 * h)
        assert abs(fd - float(gv[p])) <= 1e-6 * max(1.0, abs(float(gv[p])))
    for (i, r) in [(0, 0), (17, 3), (1000, 7), (4095, 1), (2047, 5)]:
        bp, bm = b.detach().clone(), b.detach().clone()
        bp[i, r] += 1e-6
        bm[i, r] -= 1e-6
        fd = (loss(bp) - loss(bm)) / 2e-6
        assert abs(fd - float(gb[i, r])) <= 1e-6 * max(1.0, abs(float(gb[i, r])))
    # and against the oracle gradient
    gref = oracle.solve_transpose(A_h, w.cpu().numpy())
    assert relerr(gb.cpu().numpy(), gref) <= 1e-12
    xref = oracle.solve(A_h, b.detach().cpu().numpy())
    assert relerr(gv.cpu().numpy(), oracle.grad_vals(A_h, gref, xref)) <= 1e-12


@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
def test_full_size_lap2d(dt):
    import paper_2609_40159_gb300 as P
    A_h = S.lap2d(1024, dtype=dt)
    b_h = S.rhs(A_h.n, 1, seed=1, dtype=dt)
    x_ref = oracle.solve(widened(A_h), b_h)
    A = P.Matrix.from_host(A_h)
    b = torch.as_tensor(b_h).cuda()
    plan = P.Plan(A, transpose=True)
    for mode in MODES:
        plan.set(mode, 32, 1)
        assert relerr(plan.solve(b).cpu().numpy(), x_ref) <= TOL[dt], mode
    assert P.handle().status() == 0


def test_full_size_lap3d_fwd_bwd():
    import paper_2609_40159_gb300 as P
    A_h = S.lap3d(128)
    b_h = S.rhs(A_h.n, 8, seed=4)
    w_h = S.rhs(A_h.n, 8, seed=5)
    A = P.Matrix.from_host(A_h)
    plan = P.Plan(A, transpose=True)
    x_ref = oracle.solve(A_h, b_h)
    g_ref = oracle.solve_transpose(A_h, w_h)
    b, w = torch.as_tensor(b_h).cuda(), torch.as_tensor(w_h).cuda()
    for mode in ["level", "syncfree", "block"]:
        plan.set(mode, 32, 8)
        x = plan.solve(b)
        assert relerr(x.cpu().numpy(), x_ref) <= 1e-12, mode
        gb = plan.solve_transpose(w)
        assert relerr(gb.cpu().numpy(), g_ref) <= 1e-12, mode
    gv = plan.grad_vals(gb, x).cpu().numpy()
    rng = np.random.default_rng(1)
    rows = np.repeat(np.arange(A_h.n), np.diff(A_h.row_ptr))
    for p in rng.choice(A_h.nnz, size=2000, replace=False):
        ref = -np.dot(g_ref[rows[p]], x_ref[A_h.col_idx[p]])
        assert abs(gv[p] - ref) <= 1e-12 * max(1.0, abs(ref))


def test_full_size_powerlaw():
    import paper_2609_40159_gb300 as P
    A_h = S.powerlaw(4_000_000, alpha=2.1, seed=2)
    b_h = S.rhs(A_h.n, 1, seed=2)
    x_ref = oracle.solve(A_h, b_h)
    A = P.Matrix.from_host(A_h)
    b = torch.as_tensor(b_h).cuda()
    plan = P.Plan(A)
    for mode, rpw in [("level", 32), ("syncfree", 32), ("syncfree", 4), ("block", 32)]:
        plan.set(mode, rpw, 1)
        assert relerr(plan.solve(b).cpu().numpy(), x_ref) <= 1e-12, mode


@pytest.mark.parametrize("mode", ["level", "syncfree", "block", "hybrid"])
def test_bounded_wait_reports_timeout(mode):
    """A row that is never published (test hook; the level-persistent mode
    leaves it out of its progress counter): the solve gives up after the
    plan's wait limit with SPTRSV_ETIMEOUT, the context stays usable and the
    next solve is right."""
    import paper_2609_40159_gb300 as P
    A_h = S.chain(5000, seed=1)
    A = P.Matrix.from_host(A_h)
    b = torch.as_tensor(S.rhs(A_h.n, 1, seed=1)).cuda()
    plan = P.Plan(A, mode=mode, rows_per_warp=1, wait_limit_us=20_000)
    h = P.handle()
    assert h.status() == 0
    plan.withhold(100)      # row 100's ready flag is never released
    plan.solve(b)
    assert h.status() == P._lib.SPTRSV_ETIMEOUT
    plan.withhold(-1)
    x = plan.solve(b)
    assert h.status() == 0
    assert relerr(x.cpu().numpy(), oracle.solve(A_h, b.cpu().numpy())) <= 1e-12


@pytest.mark.parametrize("name", ["lap2d_97", "lap3d_23", "powerlaw", "wide_level", "chain", "band_wide"])
def test_hybrid_thin_thresholds(name):
    """The hybrid schedule at every extreme of its thin-level threshold --
    no thin level (the level-persistent schedule), a few rows, a level of
    the widest size, every level thin (one synchronisation-free run) -- and
    with 1, 3 and 16 right-hand sides, forward and transpose, vs the
    oracle."""
    import paper_2609_40159_gb300 as P
    A_h = _case(name)
    A = P.Matrix.from_host(A_h)
    plan = P.Plan(A, mode="hybrid", transpose=True)
    an = oracle.analyze(A_h)
    widest = int(np.diff(an["level_ptr"]).max())
    for k in (1, 3, 16):
        b_h = S.rhs(A_h.n, k, seed=k)
        b = torch.as_tensor(b_h).cuda()
        x_ref, g_ref = oracle.solve(A_h, b_h), oracle.solve_transpose(A_h, b_h)
        for thin in (1, 8, 64, widest, 2**31 - 1, 0):
            plan.set_thin_rows(thin)
            for rpw in (1, 32):
                plan.set("hybrid", rpw, 4)
                assert relerr(plan.solve(b).cpu().numpy(), x_ref) <= 1e-12, (thin, rpw, k)
                assert relerr(plan.solve_transpose(b).cpu().numpy(), g_ref) <= 1e-12, ("T", thin, rpw, k)
    assert P.handle().status() == 0


def test_persistent_grid_any_size():
    """The level-persistent and hybrid solves with their persistent grids cut
    to 1, 2 and 3 blocks per SM and back to the occupancy maximum: the same
    results as the oracle (a row group only waits on groups taken before it,
    so any grid completes)."""
    import paper_2609_40159_gb300 as P
    A_h = S.lap2d(97)
    A = P.Matrix.from_host(A_h)
    b_h = S.rhs(A_h.n, 1, seed=4)
    b = torch.as_tensor(b_h).cuda()
    x_ref = oracle.solve(A_h, b_h)
    for mode in ("level", "hybrid"):
        plan = P.Plan(A, mode=mode)
        for bps in (1, 2, 3, 0):
            plan.set_blocks_per_sm(bps)
            assert relerr(plan.solve(b).cpu().numpy(), x_ref) <= 1e-12, (mode, bps)
    with pytest.raises(P.SpTRSVError):
        plan.set_blocks_per_sm(-1)
    assert P.handle().status() == 0


@pytest.mark.parametrize("mode", ["level", "syncfree", "block", "hybrid"])
def test_column_major_multi_rhs(mode):
    """SpTRSM in the column-major layout (every right-hand side contiguous,
    padded leading dimension too): forward and transpose vs the oracle, and
    equal to the row-major solve of the same block; 1 and 13 right-hand
    sides; a wider block later regrows the plan's buffer."""
    import paper_2609_40159_gb300 as P
    A_h = S.band_random(7001, 96, 1, 12, seed=21)
    A = P.Matrix.from_host(A_h)
    plan = P.Plan(A, mode=mode, transpose=True)
    for k, pad in ((13, 0), (1, 0), (13, 77), (40, 3)):
        Bh = S.rhs(A_h.n, k, seed=k + pad)                   # [n, k]
        store = torch.zeros(k, A_h.n + pad, dtype=torch.float64, device="cuda")
        B = store[:, :A_h.n]
        B.copy_(torch.as_tensor(Bh.T))
        X = plan.solve_columns(B)
        G = plan.solve_columns(B, transpose=True)
        assert P.handle().status() == 0
        assert relerr(X.cpu().numpy().T, oracle.solve(A_h, Bh)) <= 1e-12, (k, pad)
        assert relerr(G.cpu().numpy().T, oracle.solve_transpose(A_h, Bh)) <= 1e-12, (k, pad)
        Xr = plan.solve(torch.as_tensor(Bh).cuda())
        assert relerr(X.cpu().numpy().T, Xr.cpu().numpy()) <= 1e-14, (k, pad)
    with pytest.raises(P.SpTRSVError):
        P._lib.check(P._lib.lib().sptrsv_solve_layout(plan.p, P.api._ptr(B), P.api._ptr(X), 40, 10, 1, 0))


def test_cuda_graph_replay():
    import paper_2609_40159_gb300 as P
    A_h = S.band_random(50_000, 64, 4, 16, seed=11)
    A = P.Matrix.from_host(A_h)
    b = torch.as_tensor(S.rhs(A_h.n, 2, seed=3)).cuda()
    x = torch.empty_like(b)
    for mode in ["level", "syncfree", "block", "hybrid"]:
        plan = P.Plan(A, mode=mode)
        plan.solve(b, out=x)  # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            plan_s = P.Plan(A, mode=mode)
            plan_s.solve(b, out=x)
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                plan_s.solve(b, out=x)
        for _ in range(3):
            x.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert relerr(x.cpu().numpy(), oracle.solve(A_h, b.cpu().numpy())) <= 1e-12, mode


@pytest.mark.parametrize("mode", ["auto", "level", "syncfree", "block", "hybrid"])
@pytest.mark.parametrize("k", [1, 4])
def test_upper_triangular_solve(mode, k):
    """U x = b for an upper-triangular U (rows store the diagonal first),
    through the transpose of a lower-triangular plan: against a dense
    triangular solve and against the oracle's transpose solve of U^T."""
    import scipy.linalg as sl
    import scipy.sparse as sp
    import paper_2609_40159_gb300 as P
    Lh = S.band_random(3000, 48, 1, 9, seed=31)
    Ls = sp.csr_matrix((Lh.vals, Lh.col_idx, Lh.row_ptr), shape=(Lh.n, Lh.n))
    Us = Ls.T.tocsr()
    Us.sort_indices()  # diagonal first in every row of the upper triangle
    U = P.Matrix(torch.as_tensor(Us.indptr.astype(np.int32)).cuda(), torch.as_tensor(Us.indices.astype(np.int32)).cuda(),
                 torch.as_tensor(Us.data).cuda())
    Ut = P.transpose(U)
    assert torch.equal(Ut.row_ptr.cpu(), torch.as_tensor(Lh.row_ptr))  # U^T = L exactly
    assert torch.equal(Ut.col_idx.cpu(), torch.as_tensor(Lh.col_idx))
    assert torch.equal(Ut.vals.cpu(), torch.as_tensor(Lh.vals))
    up = P.UpperPlan(U, mode=mode)
    b = S.rhs(Lh.n, k, seed=32)
    x = up.solve(torch.as_tensor(b).cuda()).cpu().numpy()
    assert P.handle().status() == 0
    assert relerr(x, sl.solve_triangular(Us.toarray(), b, lower=False)) <= TOL[np.float64]
    assert relerr(x, oracle.solve_transpose(Lh, b)) <= TOL[np.float64]
    y = up.solve_transpose(torch.as_tensor(b).cuda()).cpu().numpy()
    assert relerr(y, oracle.solve(Lh, b)) <= TOL[np.float64]


def test_transpose_twice_is_identity():
    import paper_2609_40159_gb300 as P
    A = P.Matrix.from_host(S.powerlaw(50_000, seed=33))
    B = P.transpose(P.transpose(A))
    for f in ("row_ptr", "col_idx", "vals"):
        assert torch.equal(getattr(A, f), getattr(B, f)), f
