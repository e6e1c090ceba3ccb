"""The environment step of the paper's Section 4 on the GPU kernels
(paper_2609_40159_gb300.env) against the oracle's environment (oracle/env.py):
the same scripted policy drives both; after every move the GPU state --
levels, level table, costs, statistics (bit for bit), thin set, the
fewest-dependency row of every level, the chosen target, the affinities and
the reward -- equals the oracle's.  The rewritten system at the end solves to
the original solution."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from oracle import env as OE

pytestmark = pytest.mark.gpu


def _policy(mask, src_aff, rows):
    # highest source affinity, then the level with the fewest rows, then the lowest level
    cands = np.flatnonzero(mask)
    return int(min(cands, key=lambda l: (-src_aff[l], rows[l], l)))


@pytest.mark.parametrize("gen,steps", [("lap2d_40", 80), ("band_3000", 60), ("powerlaw_20k", 40)])
def test_env_matches_oracle_every_move(gen, steps):
    import paper_2609_40159_gb300 as P
    A_h = {"lap2d_40": lambda: S.lap2d(40), "band_3000": lambda: S.band_random(3000, 24, 1, 6, seed=5),
           "powerlaw_20k": lambda: S.powerlaw(20_000, seed=6)}[gen]()
    genv = P.RewriteEnv(P.Matrix.from_host(A_h))
    oenv = OE.Env(A_h)
    assert genv.threshold == oenv.threshold and genv.L_init == oenv.L_init
    valid = collapses = 0
    for t in range(steps):
        assert genv.done() == oenv.done()
        if genv.done():
            break
        gm, om = genv.valid_actions(), oenv.valid_actions()
        assert np.array_equal(gm, om), t
        ls = _policy(gm, genv.src_aff, genv.level_rows)
        assert ls == _policy(om, oenv.src_aff, oenv.state.rows)
        gr, gi = genv.step(ls)
        orw, oi = oenv.step(ls)
        assert gi["valid"] == oi["valid"] and gi["row"] == oi["row"] and gi["target"] == oi["target"], t
        assert gr == pytest.approx(orw, rel=1e-12, abs=1e-12), t
        st = oenv.state
        assert genv.nlevels == st.nlevels, t
        assert np.array_equal(genv.an.lev.cpu().numpy(), st.lev), t
        assert np.array_equal(genv.an.perm.cpu().numpy(), st.perm), t
        assert np.array_equal(genv.level_ptr, st.level_ptr), t
        assert np.array_equal(genv.cost, st.cost), t
        assert np.array_equal(genv.stats, st.stats), t          # bit for bit
        assert np.array_equal(genv.thin, st.thin), t
        assert np.array_equal(genv.pick, st.pick), t
        assert np.array_equal(genv.src_aff, oenv.src_aff) and np.array_equal(genv.tgt_aff, oenv.tgt_aff), t
        valid += gi["valid"]
        collapses += gi["valid"] and gi["collapsed"] > 0
    assert valid >= 10
    assert P.handle().status() == 0
    # the rewritten system: L' x = b + T b has the original solution
    Lp, T = genv.result()
    b = S.rhs(A_h.n, 2, seed=9)
    plan = P.Plan(Lp, T)
    x = plan.solve(torch.as_tensor(b).cuda()).cpu().numpy()
    x_ref = oracle.solve(A_h, b)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-12
