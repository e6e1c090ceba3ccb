"""Batched solves (many systems of uneven n, nnz and right-hand sides in one
persistent launch) vs the CPU oracle, forward and adjoint, with half of the
batch rewritten.  For a rewritten system the oracle's own rewrite of the
original (FP64-widened) system gives L' and T, and the value gradient is
compared on L''s pattern."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from helpers import TOL, relerr, widened

pytestmark = pytest.mark.gpu

GV_TOL = {np.float64: 1e-12, np.float32: 1e-4}


class Ref:
    """What the oracle says about one system of a batch."""

    def __init__(self, A_h, Lp=None, T=None):
        self.A = widened(A_h)
        self.Lp = None if Lp is None else S.CSR(Lp.n, Lp.row_ptr, Lp.col_idx, Lp.vals)
        self.T = T

    def solve(self, b):
        return oracle.solve(self.A, b)

    def grads(self, b, w):
        """(x, g_b, g_vals) of loss = <w, x>: g_vals on the pattern the
        solve reads (L', for a rewritten system), g_b through T^T."""
        if self.Lp is None:
            x = oracle.solve(self.A, b)
            gb = oracle.solve_transpose(self.A, w)
            return x, gb, oracle.grad_vals(self.A, gb, x)
        x = oracle.solve_rewritten(self.Lp, self.T, b)
        gbp = oracle.solve_transpose(self.Lp, w)
        return x, oracle.tt_apply(self.T, gbp), oracle.grad_vals(self.Lp, gbp, x)


def _build(items, dt, transpose=True, refs_for=None):
    """Device matrices, GPU rewrites of the marked systems, the batch plan,
    packed right-hand sides and the oracle's view of every system (its own
    rewrite for the rewritten ones; refs_for limits the oracle rewrites to a
    subset of systems)."""
    import paper_2609_40159_gb300 as P
    mats, Ts, refs = [], [], []
    for m, it in enumerate(items):
        A_h = it.A.astype(dt)
        A = P.Matrix.from_host(A_h)
        T = None
        ref = Ref(A_h)
        if it.rewritten:
            an = oracle.analyze(widened(A_h))
            rows, tg = S.narrowest_levels_list(an["nlevels"], an["level_ptr"], an["perm"], 0.01, 8)
            A, T = P.rewrite(A, P.analyze(A).lev, rows, tg)
            if refs_for is None or m in refs_for:
                ref = Ref(A_h, *oracle.rewrite(widened(A_h), an["lev"], rows, tg))
        mats.append(A)
        Ts.append(T)
        refs.append(ref)
    plan = P.BatchPlan(mats, Ts, [it.nrhs for it in items], transpose=transpose)
    b = torch.cat([torch.as_tensor(it.b.astype(dt)).reshape(-1) for it in items]).cuda()
    return P, plan, b, refs


def _check_system(plan, m, it, ref, x, w, gb, gv, dt):
    x_ref, gb_ref, gv_ref = ref.grads(it.b, plan.unpack(w, m).cpu().numpy())
    assert relerr(plan.unpack(x, m).cpu().numpy(), x_ref) <= TOL[dt], ("x", m)
    assert relerr(plan.unpack(gb, m).cpu().numpy(), gb_ref) <= TOL[dt], ("g_b", m)
    a, e = int(plan.vals_offset[m]), int(plan.vals_offset[m + 1])
    assert e - a == len(gv_ref), ("pattern", m)
    assert relerr(gv[a:e].cpu().numpy(), gv_ref) <= GV_TOL[dt], ("g_vals", m)


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_batch_small(dt):
    """Forward solve, transpose solve, T^T and the value gradient of every
    system, rewritten ones included (g_vals on L')."""
    items = S.batch_spec(nmat=40, seed=13, n_lo=300, n_hi=20_000, w_lo=8, w_hi=1024, dtype=dt)
    P, plan, b, refs = _build(items, dt)
    assert sum(it.rewritten for it in items) >= 10
    x = plan.solve(b)
    w = torch.randn_like(b)
    gbp = plan.solve_transpose(w)
    gb = plan.tt_apply(gbp)
    gv = plan.grad_vals(gbp, x)
    assert P.handle().status() == 0
    for m, it in enumerate(items):
        _check_system(plan, m, it, refs[m], x, w, gb, gv, dt)


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
    gbp = plan.solve_transpose(w)
    gb = plan.tt_apply(gbp)
    gv = plan.grad_vals(gbp, x)
    assert P.handle().status() == 0
    for m, it in enumerate(items):
        _check_system(plan, m, it, refs[m], x, w, gb, gv, np.float64)
    with pytest.raises(P.SpTRSVError):
        plan.set_geometry(rhs_tile=3)


def test_batch_graph_replay_vs_oracle():
    """The batched forward solve captured in a CUDA graph and replayed three
    times (the control block is reset inside the graph) equals the oracle's
    solution every time."""
    import paper_2609_40159_gb300 as P
    items = S.batch_spec(nmat=24, seed=17, n_lo=500, n_hi=8000, dtype=np.float32)
    P, plan, b, refs = _build(items, np.float32, transpose=False)
    x = torch.empty_like(b)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan_s = P.BatchPlan(plan.mats, plan.Ts, plan.nrhs)
        plan_s.solve(b, out=x)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan_s.solve(b, out=x)
    for _ in range(3):
        x.zero_()
        g.replay()
        torch.cuda.synchronize()
        for m, it in enumerate(items):
            assert relerr(plan_s.unpack(x, m).cpu().numpy(), refs[m].solve(it.b)) <= TOL[np.float32], m
    assert P.handle().status() == 0


def test_batch_full_size_sampled():
    """The 512-system workload of the benchmark, in the launch configuration
    the benchmark times (forward, transpose, T^T, value gradient); the oracle
    checks a sample of systems (the deepest, the largest, the most right-hand
    sides, rewritten and original ones at random)."""
    items = S.batch_spec(nmat=512, seed=3)
    deep = int(np.argmax([it.A.n / it.band for it in items]))
    big = int(np.argmax([it.A.nnz for it in items]))
    wide = int(np.argmax([it.nrhs * it.A.n for it in items]))
    rng = np.random.default_rng(0)
    sample = sorted({deep, big, wide, *rng.choice(512, size=6, replace=False).tolist()})
    assert any(items[m].rewritten for m in sample) and not all(items[m].rewritten for m in sample)
    P, plan, b, refs = _build(items, np.float32, refs_for=set(sample))
    x = plan.solve(b)
    w = torch.randn_like(b)
    gbp = plan.solve_transpose(w)
    gb = plan.tt_apply(gbp)
    gv = plan.grad_vals(gbp, x)
    assert P.handle().status() == 0
    for m in sample:
        _check_system(plan, m, items[m], refs[m], x, w, gb, gv, np.float32)


def test_batch_autograd_function():
    """batch_solve as a torch.autograd.Function on a mixed batch (half of it
    rewritten): gradients with respect to the packed values and right-hand
    sides against the oracle, and against central finite differences of
    loss = <w, x> at sampled coordinates (FP64, relative 1e-6)."""
    import paper_2609_40159_gb300 as P
    items = S.batch_spec(nmat=10, seed=41, n_lo=200, n_hi=3000, w_lo=8, w_hi=256, k_hi=6,
                         dtype=np.float64)
    P, plan, b0, refs = _build(items, np.float64)
    vals = plan.vals
    vals.requires_grad_(True)
    b = b0.clone().requires_grad_(True)
    w = torch.randn_like(b0)
    x = P.batch_solve(plan, b)
    (x * w).sum().backward()
    gv, gb = vals.grad.detach().clone(), b.grad.detach().clone()
    vals.requires_grad_(False)
    with pytest.raises(ValueError):
        P.batch_solve(plan, b0, vals.clone())
    xd = x.detach()
    for m, it in enumerate(items):
        _check_system(plan, m, it, refs[m], xd, w, gb, gv, np.float64)

    def loss(bb):
        with torch.no_grad():
            return float((plan.solve(bb) * w).sum())

    for p in rng_choice(plan.total_nnz, 24):
        old = float(vals[p])
        h = 1e-6 * max(1.0, abs(old))
        with torch.no_grad():
            vals[p] = old + h
            fp = loss(b0)
            vals[p] = old - h
            fm = loss(b0)
            vals[p] = old
        fd = (fp - fm) / (2 * h)
        assert abs(fd - float(gv[p])) <= 1e-6 * max(1.0, abs(float(gv[p]))), p
    for q in rng_choice(plan.total_rhs, 12):
        bp, bm = b0.clone(), b0.clone()
        bp[q] += 1e-6
        bm[q] -= 1e-6
        fd = (loss(bp) - loss(bm)) / 2e-6
        assert abs(fd - float(gb[q])) <= 1e-6 * max(1.0, abs(float(gb[q]))), q
    assert P.handle().status() == 0


def rng_choice(n, k, seed=7):
    return np.random.default_rng(seed).choice(n, size=min(k, n), replace=False).tolist()


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
        gv = plan.grad_vals(gb, x)
        assert P.handle().status() == 0
        for m, A in enumerate(systems):
            xr, gr = oracle.solve(A, bs[m]), oracle.solve_transpose(A, bs[m])
            assert relerr(plan.unpack(x, m).cpu().numpy(), xr) <= TOL[np.float64], (tile, m)
            assert relerr(plan.unpack(gb, m).cpu().numpy(), gr) <= TOL[np.float64], (tile, m)
            a, e = int(plan.vals_offset[m]), int(plan.vals_offset[m + 1])
            assert relerr(gv[a:e].cpu().numpy(), oracle.grad_vals(A, gr, xr)) <= 1e-12, (tile, m)
    empty = P.BatchPlan([], None, [], transpose=True)
    z = torch.empty(0, dtype=torch.float32, device="cuda")
    empty.solve(z)
    assert P.handle().status() == 0


@pytest.mark.parametrize("trans", [False, True], ids=["fwd", "transpose"])
def test_batch_bounded_wait_reports_timeout(trans):
    """A row of one system that is never published (test hook): the batched
    solve gives up after the plan's wait limit with SPTRSV_ETIMEOUT, leaves
    the context usable, and the next solve is right again."""
    import paper_2609_40159_gb300 as P
    systems = [S.band_random(3000, 16, 1, 6, seed=1), S.chain(4000, seed=2), S.band_random(500, 8, 1, 4, seed=3)]
    mats = [P.Matrix.from_host(A) for A in systems]
    plan = P.BatchPlan(mats, None, [1, 2, 1], transpose=True, wait_limit_us=20_000)
    rng = np.random.default_rng(3)
    bs = [rng.uniform(-1, 1, (A.n, k)) for A, k in zip(systems, [1, 2, 1])]
    b = torch.cat([torch.as_tensor(v).reshape(-1) for v in bs]).cuda()
    h = P.handle()
    assert h.status() == 0
    run = plan.solve_transpose if trans else plan.solve
    plan.withhold(1, 1500)      # row 1500 of the chain is never published
    run(b)
    assert h.status() == P._lib.SPTRSV_ETIMEOUT
    plan.withhold(-1, 0)
    x = run(b)
    assert h.status() == 0
    ref = oracle.solve_transpose if trans else oracle.solve
    for m, A in enumerate(systems):
        assert relerr(plan.unpack(x, m).cpu().numpy(), ref(A, bs[m])) <= TOL[np.float64], m

@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_batch_level_schedule(dt):
    """The level-ordered schedule (the groups of one level at the same time,
    levels one after another; transpose: levels last to first) on every
    system, then on every other system with a different tile per system:
    forward solve, transpose solve, T^T and g_vals vs the oracle, rewritten
    systems included; then back to the in-order schedule."""
    items = S.batch_spec(nmat=40, seed=13, n_lo=300, n_hi=20_000, w_lo=8, w_hi=1024, dtype=dt)
    P, plan, b, refs = _build(items, dt)
    nm = len(items)
    for sched, tiles in (("level", None),
                         (["level", "inorder"] * (nm // 2), [(1, 2, 4, 8)[m % 4] for m in range(nm)]),
                         ("inorder", 4)):
        plan.set_schedule(sched)
        if tiles is not None:
            plan.set_geometry(rhs_tile=tiles)
        x = plan.solve(b)
        w = torch.randn_like(b)
        gbp = plan.solve_transpose(w)
        gb = plan.tt_apply(gbp)
        gv = plan.grad_vals(gbp, x)
        assert P.handle().status() == 0
        for m, it in enumerate(items):
            _check_system(plan, m, it, refs[m], x, w, gb, gv, dt)
    with pytest.raises(P.SpTRSVError):
        P._lib.check(P._lib.lib().sptrsv_batch_plan_set_schedule(
            plan.p, 0, (__import__("ctypes").c_int32 * nm)(*([3] * nm))))


def test_batch_level_schedule_edge_cases():
    """Level-ordered schedule on degenerate level structures: levels wider
    than the shared-memory ring (dependencies read from global memory), one
    level of 5,000 rows, 1-row levels (a chain), n = 1, row counts around
    the 32-row group, a long row, a wide band; forward and transpose, tiles
    1 and 8, each direction scheduled on its own."""
    import paper_2609_40159_gb300 as P
    from helpers import long_row, two_wide_levels
    systems = [two_wide_levels(6000, seed=1), S.diagonal(5000, seed=2), S.chain(1000, seed=3),
               S.band_random(1, 4, 0, 4, seed=4), S.band_random(31, 8, 0, 6, seed=5),
               S.band_random(33, 40, 1, 20, seed=6), long_row(), S.band_random(4097, 700, 10, 40, seed=7),
               S.lap2d(70)]
    nrhs = [3, 1, 32, 1, 5, 32, 2, 9, 4]
    rng = np.random.default_rng(8)
    mats = [P.Matrix.from_host(A) for A in systems]
    plan = P.BatchPlan(mats, None, nrhs, transpose=True)
    bs = [rng.uniform(-1, 1, (A.n, k)) for A, k in zip(systems, nrhs)]
    b = torch.cat([torch.as_tensor(v).reshape(-1) for v in bs]).cuda()
    plan.set_schedule("level", direction="forward")
    plan.set_schedule("level", direction="transpose")
    for tile in (1, 8):
        plan.set_geometry(rhs_tile=tile)
        x = plan.solve(b)
        gb = plan.solve_transpose(b)
        assert P.handle().status() == 0
        for m, A in enumerate(systems):
            xr, gr = oracle.solve(A, bs[m]), oracle.solve_transpose(A, bs[m])
            assert relerr(plan.unpack(x, m).cpu().numpy(), xr) <= TOL[np.float64], (tile, m)
            assert relerr(plan.unpack(gb, m).cpu().numpy(), gr) <= TOL[np.float64], (tile, m)


@pytest.mark.parametrize("trans", [False, True], ids=["fwd", "transpose"])
def test_batch_level_schedule_bounded_wait(trans):
    """A withheld row under the level-ordered schedule: the groups of the
    later levels give up after the wait limit with SPTRSV_ETIMEOUT, and the
    next solve is right again."""
    import paper_2609_40159_gb300 as P
    systems = [S.lap2d(40), S.band_random(3000, 64, 1, 6, seed=2)]
    mats = [P.Matrix.from_host(A) for A in systems]
    plan = P.BatchPlan(mats, None, [1, 2], transpose=True, wait_limit_us=20_000)
    plan.set_schedule("level")
    rng = np.random.default_rng(3)
    bs = [rng.uniform(-1, 1, (A.n, k)) for A, k in zip(systems, [1, 2])]
    b = torch.cat([torch.as_tensor(v).reshape(-1) for v in bs]).cuda()
    h = P.handle()
    run = plan.solve_transpose if trans else plan.solve
    plan.withhold(1, 1500)
    run(b)
    assert h.status() == P._lib.SPTRSV_ETIMEOUT
    plan.withhold(-1, 0)
    x = run(b)
    assert h.status() == 0
    ref = oracle.solve_transpose if trans else oracle.solve
    for m, A in enumerate(systems):
        assert relerr(plan.unpack(x, m).cpu().numpy(), ref(A, bs[m])) <= TOL[np.float64], m


def test_batch_step_from_host_buffers():
    """sptrsv_batch_step_host: three steps in flight from pinned host
    buffers (different inputs, the two device buffer sets alternating), then
    one wait: x, g_b and g_vals of every step equal the oracle's, rewritten
    systems included."""
    dt = np.float32
    items = S.batch_spec(nmat=16, seed=41, n_lo=300, n_hi=8000, dtype=dt)
    P, plan, b, refs = _build(items, dt)
    n_rhs, n_nz = plan.total_rhs, plan.total_nnz
    gen = torch.Generator().manual_seed(5)
    steps = []
    for t in range(3):
        hb = torch.empty(n_rhs, dtype=torch.float32).pin_memory()
        hb.copy_(b.cpu() * (1.0 + t))
        hw = torch.empty(n_rhs, dtype=torch.float32).pin_memory()
        hw.copy_(torch.randn(n_rhs, generator=gen))
        outs = [torch.empty(n, dtype=torch.float32).pin_memory() for n in (n_rhs, n_rhs, n_nz)]
        plan.step_host(hb, hw, *outs)
        steps.append((hb, hw, outs))
    plan.step_wait()
    assert P.handle().status() == 0
    for t, (hb, hw, (hx, hgb, hgv)) in enumerate(steps):
        for m, it in enumerate(items):
            a, e = int(plan.rhs_offset[m]), int(plan.rhs_offset[m + 1])
            bm = hb[a:e].numpy().reshape(it.A.n, it.nrhs).astype(np.float64)
            wm = hw[a:e].numpy().reshape(it.A.n, it.nrhs).astype(np.float64)
            x_ref, gb_ref, gv_ref = refs[m].grads(bm, wm)
            assert relerr(hx[a:e].numpy(), x_ref) <= TOL[dt], (t, m)
            assert relerr(hgb[a:e].numpy(), gb_ref) <= TOL[dt], (t, m)
            va, ve = int(plan.vals_offset[m]), int(plan.vals_offset[m + 1])
            assert relerr(hgv[va:ve].numpy(), gv_ref) <= GV_TOL[dt], (t, m)
