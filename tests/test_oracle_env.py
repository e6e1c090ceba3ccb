"""Pins of the oracle's environment step (oracle/env.py) against the paper's
Algorithm 1 (target level), Algorithm 2 (reward) and Section 4.3 (masks),
with values worked out by hand, and against invariants of the move: the
moved row ends at or above its target level, the level count never grows,
the rewritten system has the original solution."""
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import env as E


# ------------------------------------------------------------ Algorithm 1
THIN = [True, False, True, True, False, True, False]
AFF = [0.0, 0.0, 0.5, 0.2, 0.0, 0.1, 0.0]


def test_target_highest_affinity_among_nearest_thin_levels():
    # thin levels above 6, nearest first: 5, 3, 2, 0; affinities 0.1, 0.2, 0.5, 0.0
    assert E.select_target(6, THIN, AFF, window=5, max_distance=16) == 2
    # only the two nearest thin levels (5 and 3) are candidates
    assert E.select_target(6, THIN, AFF, window=2, max_distance=16) == 3
    # a tie keeps the nearer level
    aff = list(AFF)
    aff[5] = 0.2
    assert E.select_target(6, THIN, aff, window=2, max_distance=16) == 5
    # the source itself is never a candidate
    assert E.select_target(3, THIN, AFF, window=5, max_distance=16) == 2


def test_target_fallback_and_invalid_moves():
    thin = [False, False, False, True, False]
    # no thin level above a thin source: the level just above (a thick target)
    assert E.select_target(3, thin, [0.0] * 5, window=5, max_distance=16) == 2
    # no thin level above a thick source: invalid
    assert E.select_target(4, [False, False, False, False, False], [0.0] * 5, window=5, max_distance=16) == -1
    # thin level 3 is above source 4: that is the target even though the source is thick
    assert E.select_target(4, thin, [0.0] * 5, window=5, max_distance=16) == 3
    # farther than MAX_REWRITE_DISTANCE: invalid
    thin = [True] + [False] * 30
    assert E.select_target(30, thin, [0.0] * 31, window=5, max_distance=16) == -1
    assert E.select_target(16, thin, [0.0] * 31, window=5, max_distance=16) == 0


# ------------------------------------------------------------ Algorithm 2
CFG = E.Config()


def test_reward_collapse_branch():
    # L_init 100, levels 81 -> 80 (critical path reduced), CV 0.50 -> 0.40,
    # source of 1 row, distance 2, no abandonment:
    #   r_cv    = 100 * (0.5 - 0.4)                         = 9.999999999999998
    #   s       = log(1 + 1 + 1) = log 3                    = 1.0986122886681098
    #   r_cpath = 1 * (100 / 80) * (1 + 1 / s)              = 2.387799033283547
    #   r_rw    = log1p(5 - 2) / 100 = log 4 / 100          = 0.013862943611198907
    #   total   = 0.8 r_cv + 0.8 r_cpath + 0.05 r_rw        = 9.910932373807395
    total, (r_cv, r_cp, r_rw, r_ab) = E.reward(CFG, 100, 0.5, 0.4, 81, 80, 1, True, 2, 0.0)
    assert r_cv == pytest.approx(10.0, rel=1e-12)
    assert r_cp == pytest.approx(2.387799033283547, rel=1e-12)
    assert r_rw == pytest.approx(0.013862943611198907, rel=1e-12)
    assert r_ab == 0.0
    assert total == pytest.approx(9.910932373807395, rel=1e-12)


def test_reward_thin_and_thick_sources_and_cv_penalty():
    # no collapse, thin source of 5 rows: r_cpath = 1 / log 7 = 0.5138983423697507
    _, (r_cv, r_cp, _, _) = E.reward(CFG, 100, 0.5, 0.5, 80, 80, 5, True, 1, 0.0)
    assert r_cv == 0.0 and r_cp == pytest.approx(0.5138983423697507, rel=1e-12)
    # thick source: r_cpath = -(1 + log 7) = -2.9459101490553135
    _, (_, r_cp, _, _) = E.reward(CFG, 100, 0.5, 0.5, 80, 80, 5, False, 1, 0.0)
    assert r_cp == pytest.approx(-2.9459101490553135, rel=1e-12)
    # CV worse by more than epsilon: -alpha; within epsilon: 0
    _, (r_cv, _, _, _) = E.reward(CFG, 100, 0.40, 0.41, 80, 80, 5, True, 1, 0.0)
    assert r_cv == -1.0
    _, (r_cv, _, _, _) = E.reward(CFG, 100, 0.40, 0.40005, 80, 80, 5, True, 1, 0.0)
    assert r_cv == 0.0


def test_reward_distance_and_abandonment():
    # distance 9 > threshold 5: r_rw = -log1p(4) / 50 = -0.032188758248682
    total, (_, _, r_rw, r_ab) = E.reward(CFG, 50, 0.5, 0.5, 40, 40, 3, True, 9, 0.75)
    assert r_rw == pytest.approx(-0.032188758248682, rel=1e-12)
    assert r_ab == -0.75
    # total = 0.8 * (1 / log 5) + 0.05 r_rw + 0.5 * (-0.75)
    assert total == pytest.approx(0.8 / math.log(5) + 0.05 * r_rw - 0.375, rel=1e-12)
    # distance equal to the threshold: -log1p(0) = 0
    _, (_, _, r_rw, _) = E.reward(CFG, 50, 0.5, 0.5, 40, 40, 3, True, 5, 0.0)
    assert r_rw == 0.0


# ------------------------------------------------------------ Section 4.3
def test_masks():
    env = E.Env(S.lap2d(12))
    m = env.valid_actions()
    assert not m[0] and m[1:].all()
    # a source level with one row left forces its collapse
    st = env.state
    one = int(np.flatnonzero(st.rows == 1)[-1])  # the last level of the grid has one row
    env.last_source = one
    m = env.valid_actions()
    assert m.sum() == 1 and m[one]
    # after a stagnant period only the X levels of highest source affinity
    env.last_source = -1
    env.since_collapse = env.cfg.stagnation_steps
    env.src_aff[:] = 0.0
    env.src_aff[[3, 7, 9, 11, 13, 15, 17]] = [0.5, 0.9, 0.1, 0.7, 0.3, 0.2, 0.8]
    m = env.valid_actions()
    assert sorted(np.flatnonzero(m).tolist()) == [3, 7, 11, 13, 17]


# ------------------------------------------------------------ episodes
def _policy(mask, src_aff, rows):
    cands = np.flatnonzero(mask)
    return int(min(cands, key=lambda l: (-src_aff[l], rows[l], l)))


@pytest.mark.parametrize("gen", ["lap2d", "band"])
def test_episode_invariants(gen):
    A = S.lap2d(20) if gen == "lap2d" else S.band_random(600, 12, 1, 5, seed=3)
    env = E.Env(A)
    b = S.rhs(A.n, 2, seed=1)
    x_ref = oracle.solve(A, b)
    nl = env.state.nlevels
    valid = 0
    for _ in range(40):
        if env.done():
            break
        ls = _policy(env.valid_actions(), env.src_aff, env.state.rows)
        r, info = env.step(ls)
        assert math.isfinite(r)
        if not info["valid"]:
            continue
        valid += 1
        st = env.state
        assert st.nlevels <= nl
        nl = st.nlevels
        assert st.lev[info["row"]] <= info["target"]
        assert len(env.src_aff) == st.nlevels == len(env.tgt_aff)
    assert valid > 5
    Lp, T = oracle.rewrite(A, env.lev0, env.rows, env.targets)
    x = oracle.solve_rewritten(Lp, T, b)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-12
