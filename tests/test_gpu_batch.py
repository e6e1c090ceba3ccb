"""Batched solves (many systems of uneven n, nnz and right-hand sides in one
persistent launch) vs the CPU oracle, forward and adjoint, with half of the
batch rewritten."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from helpers import TOL, relerr, widened

pytestmark = pytest.mark.gpu


def _build(items, dt, transpose=True):
    """Device matrices (one packed value buffer), rewrites of the marked
    systems, packed right-hand sides."""
    import paper_2609_40159_gb300 as P
    mats, Ts, refs = [], [], []
    for it in items:
        A_h = it.A.astype(dt)
        A = P.Matrix.from_host(A_h)
        T = None
        if it.rewritten:
            an = oracle.analyze(widened(A_h))
            rows, tg = S.narrowest_levels_list(an["nlevels"], an["level_ptr"], an["perm"], 0.01, 8)
            A, T = P.rewrite(A, P.analyze(A).lev, rows, tg)
        mats.append(A)
        Ts.append(T)
        refs.append(A_h)
    plan = P.BatchPlan(mats, Ts, [it.nrhs for it in items], transpose=transpose)
    b = torch.cat([torch.as_tensor(it.b.astype(dt)).reshape(-1) for it in items]).cuda()
    return P, plan, b, refs


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_batch_small(dt):
    items = S.batch_spec(nmat=40, seed=13, n_lo=300, n_hi=20_000, w_lo=8, w_hi=1024, dtype=dt)
    P, plan, b, refs = _build(items, dt)
    x = plan.solve(b)
    w = torch.randn_like(b)
    gbp = plan.solve_transpose(w)
    gb = plan.tt_apply(gbp)
    gv = plan.grad_vals(gbp, x)
    assert P.handle().status() == 0
    for m, it in enumerate(items):
        xm = plan.unpack(x, m).cpu().numpy()
        x_ref = oracle.solve(widened(refs[m]), it.b)
        assert relerr(xm, x_ref) <= TOL[dt], m
        wm = plan.unpack(w, m).cpu().numpy()
        g_ref = oracle.solve_transpose(widened(refs[m]), wm)
        assert relerr(plan.unpack(gb, m).cpu().numpy(), g_ref) <= TOL[dt], m
        if not it.rewritten:
            a, e = int(plan.vals_offset[m]), int(plan.vals_offset[m + 1])
            gv_ref = oracle.grad_vals(widened(refs[m]), g_ref, x_ref)
            assert relerr(gv[a:e].cpu().numpy(), gv_ref) <= (1e-12 if dt == np.float64 else 1e-4), m


@pytest.mark.parametrize("tile", [1, 2, 4, 8, "mixed"])
def test_batch_rhs_tiles(tile):
    """Every column tile width, and a different width per system: systems
    split into independent work items of at most `tile` columns, ragged last
    tiles included (nrhs up to 32)."""
    items = S.batch_spec(nmat=24, seed=29, n_lo=300, n_hi=6000, dtype=np.float64)
    P, plan, b, refs = _build(items, np.float64)
    tiles = [(1, 2, 4, 8)[m % 4] for m in range(len(items))] if tile == "mixed" else tile
    rpw = [(32, 16, 8, 4, 1)[m % 5] for m in range(len(items))] if tile == "mixed" else None
    plan.set_geometry(rows_per_warp=rpw, rhs_tile=tiles)
    x = plan.solve(b)
    w = torch.randn_like(b)
    gb = plan.solve_transpose(w)
    assert P.handle().status() == 0
    for m, it in enumerate(items):
        x_ref = oracle.solve(widened(refs[m]), it.b)
        assert relerr(plan.unpack(x, m).cpu().numpy(), x_ref) <= TOL[np.float64], m
        if not it.rewritten:
            g_ref = oracle.solve_transpose(widened(refs[m]), plan.unpack(w, m).cpu().numpy())
            assert relerr(plan.unpack(gb, m).cpu().numpy(), g_ref) <= TOL[np.float64], m
    with pytest.raises(P.SpTRSVError):
        plan.set_geometry(rhs_tile=3)


def test_batch_graph_replay_and_loop_equivalence():
    import paper_2609_40159_gb300 as P
    items = S.batch_spec(nmat=24, seed=17, n_lo=500, n_hi=8000, dtype=np.float32)
    P, plan, b, refs = _build(items, np.float32, transpose=False)
    x = torch.empty_like(b)
    plan.solve(b, out=x)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan_s = P.BatchPlan(plan.mats, plan.Ts, plan.nrhs)
        plan_s.solve(b, out=x)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan_s.solve(b, out=x)
    x.zero_()
    g.replay()
    torch.cuda.synchronize()
    for m, it in enumerate(items):
        single = P.Plan(plan.mats[m], plan.Ts[m], mode="level_launch")
        xs = single.solve(torch.as_tensor(it.b).cuda())
        assert relerr(plan_s.unpack(x, m).cpu().numpy(), xs.cpu().numpy().astype(np.float64)) <= 1e-5


def test_batch_full_size_sampled():
    """The 512-system workload of the benchmark, in the launch configuration
    the benchmark times; the oracle checks a sample of systems (the deepest,
    the largest, the most right-hand sides and random ones)."""
    items = S.batch_spec(nmat=512, seed=3)
    P, plan, b, refs = _build(items, np.float32)
    x = plan.solve(b)
    w = torch.randn_like(b)
    gb = plan.tt_apply(plan.solve_transpose(w))
    assert P.handle().status() == 0
    deep = int(np.argmax([it.A.n / it.band for it in items]))
    big = int(np.argmax([it.A.nnz for it in items]))
    wide = int(np.argmax([it.nrhs * it.A.n for it in items]))
    rng = np.random.default_rng(0)
    sample = sorted({deep, big, wide, *rng.choice(512, size=5, replace=False).tolist()})
    for m in sample:
        x_ref = oracle.solve(widened(refs[m]), items[m].b)
        assert relerr(plan.unpack(x, m).cpu().numpy(), x_ref) <= 1e-5, m
        g_ref = oracle.solve_transpose(widened(refs[m]), plan.unpack(w, m).cpu().numpy())
        assert relerr(plan.unpack(gb, m).cpu().numpy(), g_ref) <= 1e-5, m


def test_batch_edge_cases():
    """Degenerate systems in one batch: n = 1, row counts at and around the
    32-row group boundary, a diagonal system (no dependencies), a chain
    (every row depends on the one before: the longest in-group chains), a
    long-row system (rows beyond the preloaded entries), 1 and 32
    right-hand sides, forward and adjoint; and an empty batch."""
    import paper_2609_40159_gb300 as P
    from helpers import long_row
    systems = [S.band_random(1, 4, 0, 4, seed=1), S.band_random(31, 8, 0, 6, seed=2),
               S.band_random(32, 8, 1, 6, seed=3), S.band_random(33, 40, 1, 20, seed=4),
               S.diagonal(100, seed=5), S.chain(1000, seed=6), long_row(),
               S.band_random(4097, 700, 10, 40, seed=7)]
    nrhs = [1, 32, 3, 32, 5, 32, 2, 9]
    rng = np.random.default_rng(8)
    mats = [P.Matrix.from_host(A) for A in systems]
    plan = P.BatchPlan(mats, None, nrhs, transpose=True)
    bs = [rng.uniform(-1, 1, (A.n, k)) for A, k in zip(systems, nrhs)]
    b = torch.cat([torch.as_tensor(v).reshape(-1) for v in bs]).cuda()
    for tile in (1, 8):
        plan.set_geometry(rhs_tile=tile)
        x = plan.solve(b)
        gb = plan.solve_transpose(b)
        assert P.handle().status() == 0
        for m, A in enumerate(systems):
            assert relerr(plan.unpack(x, m).cpu().numpy(), oracle.solve(A, bs[m])) <= TOL[np.float64], (tile, m)
            assert relerr(plan.unpack(gb, m).cpu().numpy(), oracle.solve_transpose(A, bs[m])) <= TOL[np.float64], (tile, m)
    empty = P.BatchPlan([], None, [], transpose=True)
    z = torch.empty(0, dtype=torch.float32, device="cuda")
    empty.solve(z)
    assert P.handle().status() == 0
