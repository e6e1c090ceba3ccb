"""Host logic of the batched autotuner on CPU: a stand-in plan whose
"solve time" is a makespan model of the geometry; the tuner must reach the
model's optimum (uniform tile first, then per-class refinement) and leave
the plan on its choice."""
import numpy as np
import torch

from paper_2609_40159_gb300 import autotune


class _Mat:
    def __init__(self, n, nnz, nlevels=None):
        self.n, self.nnz = n, nnz
        self.nlevels = nlevels if nlevels is not None else n // 2


class _FakeBatch:
    def __init__(self, mats, nrhs):
        self.mats, self.nrhs = mats, nrhs
        self.rpw = [0] * len(mats)
        self.tile = [8] * len(mats)
        self.sched = ["inorder"] * len(mats)
        self.calls = 0

    def set_schedule(self, schedule, direction="both"):
        self.sched = [v if v else self.sched[m] for m, v in enumerate(schedule)]

    def set_geometry(self, rows_per_warp=None, rhs_tile=None, direction="both"):
        self.direction = direction
        if rows_per_warp is not None:
            self.rpw = [r if r else self.rpw[m] for m, r in enumerate(rows_per_warp)]
        if rhs_tile is not None:
            self.tile = [t if t else self.tile[m] for m, t in enumerate(rhs_tile)]

    def solve(self, b, out=None):
        self.calls += 1
        return out

    solve_transpose = solve

    def model_ms(self):
        # per system: chain cost grows with the tile, items = ceil(k / tile);
        # short rows prefer 32 rows per warp (0 = the default, same as 32)
        cost = []
        for m, A in enumerate(self.mats):
            t, r = self.tile[m], self.rpw[m] or 32
            if self.sched[m] == "level":   # a chain of levels instead of rows
                per_item = 12 * A.nlevels * (1 + 0.3 * t)
            else:
                per_item = A.n * (1 + 0.3 * t) * (1.0 if r == 32 else 1.5)
            items = -(-self.nrhs[m] // t)
            cost.append((per_item, items))
        longest = max(c for c, _ in cost)
        total = sum(c * i for c, i in cost) / 8.0  # 8 "slots"
        return max(longest, total)


def test_tune_batch_reaches_the_model_optimum(monkeypatch):
    rng = np.random.default_rng(0)
    mats = [_Mat(int(n), int(n) * 10) for n in rng.integers(1000, 50_000, size=24)]
    nrhs = [int(k) for k in rng.integers(1, 33, size=24)]
    fake = _FakeBatch(mats, nrhs)
    monkeypatch.setattr(autotune, "time_call", lambda fn, reps=3: (fn(), fake.model_ms())[1])
    res = autotune.tune_batch(fake, torch.zeros(4), candidates=(8, 16, 32), tiles=(2, 4, 8), reps=1)
    # the plan is left on the reported choice, and that choice is the best time
    # seen up to the tuner's 0.5 % hysteresis (it ignores smaller gains as noise)
    assert abs(fake.model_ms() - res["ms"]) < 1e-9
    assert res["ms"] <= min(e["ms"] for e in res["log"] if e["ms"] is not None) / 0.995
    # exhaustive search over uniform geometries cannot beat the tuner
    best_uniform = float("inf")
    for t in (2, 4, 8):
        for r in (8, 16, 32):
            fake.set_geometry([r] * 24, [t] * 24)
            best_uniform = min(best_uniform, fake.model_ms())
    assert res["ms"] <= best_uniform / 0.995


def test_batch_classes_bucket_row_length_and_rhs():
    fake = _FakeBatch([_Mat(100, 1000), _Mat(200, 2000), _Mat(100, 100)], [1, 1, 30])
    labels = autotune.batch_classes(fake)
    assert labels[0] == labels[1] and labels[0] != labels[2]


def test_tune_batch_direction_sets_that_direction_only(monkeypatch):
    """The transpose solve is tuned on its own timing and its geometry is set
    for the transpose direction only."""
    mats = [_Mat(1000 * (m + 1), 10_000 * (m + 1)) for m in range(6)]
    fake = _FakeBatch(mats, [1, 4, 8, 16, 2, 32])
    timed = []

    def tc(fn, reps=3):
        timed.append(fn)
        fn()
        return fake.model_ms()

    monkeypatch.setattr(autotune, "time_call", tc)
    calls = []
    fake.solve_transpose = lambda b, out=None: calls.append("T") or out
    fake.solve = lambda b, out=None: calls.append("F") or out
    res = autotune.tune_batch(fake, torch.zeros(4), reps=1, direction="transpose")
    assert res["direction"] == "transpose" and fake.direction == "transpose"
    assert calls and set(calls) == {"T"}
    import pytest
    with pytest.raises(ValueError):
        autotune.tune_batch(fake, torch.zeros(4), direction="sideways")


def test_tune_batch_picks_the_level_schedule_where_it_pays(monkeypatch):
    """Systems whose levels are wide (n / levels >> 12 in the model) are
    moved to the level-ordered schedule, the others stay in row order."""
    mats = ([_Mat(40_000, 400_000, nlevels=400) for _ in range(4)] +
            [_Mat(40_000, 400_000, nlevels=30_000) for _ in range(4)])
    fake = _FakeBatch(mats, [1] * 4 + [30] * 4)   # different classes (nrhs)
    monkeypatch.setattr(autotune, "time_call", lambda fn, reps=3: (fn(), fake.model_ms())[1])
    res = autotune.tune_batch(fake, torch.zeros(4), reps=1)
    assert fake.sched[:4] == ["level"] * 4
    assert fake.sched[4:] == ["inorder"] * 4
    assert {v["schedule"] for v in res["choice"].values()} == {"level", "inorder"}


class _FakePlan:
    """Stand-in single-system plan: the solve time of a (mode, rows per warp,
    tile) choice is read from a table; the tuner must apply the table's
    minimum."""

    def __init__(self, times):
        self.A = _Mat(10_000, 50_000, nlevels=100)
        self.A.dtype = torch.float64
        self.times = times
        self.choice = None

    def info(self):
        return {"nlevels": self.A.nlevels}

    def set(self, mode=0, rows_per_warp=0, rhs_tile=0):
        self.choice = (mode, rows_per_warp, rhs_tile)

    def solve(self, b, out=None):
        return out


def test_tune_plan_applies_the_fastest_candidate(monkeypatch):
    """tune_plan (without its cache) times every mode x rows per warp x tile
    candidate once and leaves the plan on the fastest one."""
    rng = np.random.default_rng(0)
    modes, rpws, kts = ("level", "syncfree", "block", "hybrid"), (1, 4, 32), (1, 4)
    times = {(m, r, t): float(rng.uniform(1, 10)) for m in modes for r in rpws for t in kts}
    times[("hybrid", 4, 1)] = 0.5
    plan = _FakePlan(times)
    seen = []

    def tc(fn, reps=5):
        fn()
        seen.append(plan.choice)
        return times[plan.choice]

    monkeypatch.setattr(autotune, "time_call", tc)
    res = autotune.tune_plan(plan, torch.zeros(10_000, 4, dtype=torch.float64), modes=modes, rpws=rpws,
                             kts=kts, use_cache=False, reps=1)
    assert sorted(seen) == sorted(times)
    assert plan.choice == ("hybrid", 4, 1)
    assert res["best"]["mode"] == "hybrid" and res["best"]["ms"] == 0.5 and not res["cached"]
