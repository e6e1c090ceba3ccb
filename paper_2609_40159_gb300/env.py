"""The paper's graph-transformation environment on the GPU kernels.

One step of the environment of the paper's Section 4: the policy picks a
source level; the row of that level with the fewest dependencies moves to a
target level chosen by Algorithm 1; the system is rewritten (sptrsv_rewrite),
its levels are recomputed incrementally from the moved row
(sptrsv_analyze_incremental) and the environment's observation -- level
costs, rows per level, thin levels, the fewest-dependency row of every level
(sptrsv_level_summary), the coefficients of variation -- is read back; the
reward follows Algorithm 2.  Every step of the path runs in the library's
kernels; this module keeps the host-side bookkeeping (the rewriting list,
per-level affinities, completion ratios, masks), which is a few arrays of
one entry per level.

Readings of the paper (its Sections 4.1-4.4 and Algorithms 1-2 leave these
open; each unstated constant is a field of ``EnvConfig``):
  * thin threshold ALC * (1 + max(0, 1 - CV)) from the initial system, fixed
    for the episode (ALC is constant through an episode, Section 4.1);
  * levels are longest-path depths recomputed after every move, so a level
    that empties disappears and the per-level state after it moves down;
  * Algorithm 1: among the SEARCH_WINDOW nearest thin levels above the
    source, the highest target affinity (ties: the nearer); without a thin
    level, the level just above when the source is thin, else invalid;
    longer than MAX_REWRITE_DISTANCE: invalid.  An invalid move changes
    nothing and earns 0;
  * the move rewrites the row towards the target level in the current
    numbering with the library's rewrite semantics (original rows and
    levels; a row moved twice keeps the smaller target);
  * Algorithm 2 with Delta CV = previous CV - current CV, s = log(2 + size of
    the source level before the move), the abandonment penalty (1 -
    completion ratio) * log1p(steps since the level was first touched);
  * affinities decay by a factor per step, the selected levels gain a boost,
    levels that are not thin get a target affinity of at most -1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import api as _api


@dataclass
class EnvConfig:
    search_window: int = 5             # Section 4.4: "the closest five upper thin levels"
    max_rewrite_distance: int = 16     # not stated in the paper
    reward_alpha: float = 1.0          # alpha of Algorithm 2, not stated
    eps: float = 1e-4                  # epsilon of Algorithm 2, not stated
    rwdist_threshold: int = 5          # threshold of r_rwdist, not stated
    affinity_decay: float = 0.9        # not stated
    affinity_boost: float = 1.0        # not stated
    stagnation_steps: int = 20         # not stated
    stagnation_keep: int = 5           # X of Section 4.3, not stated
    thin_completion_stop: float = 0.1  # not stated
    max_steps: int = 1000
    weights: tuple = (0.80, 0.80, 0.05, 0.50)  # Algorithm 2


def target_level(source, thin, tgt_aff, window, max_distance) -> int:
    """Algorithm 1: the target level for `source` (>= 1), or -1 if the move
    is invalid."""
    near = []
    for l in range(source - 1, -1, -1):
        if len(near) == window:
            break
        if thin[l]:
            near.append(l)
    if near:
        target = near[0]
        for l in near[1:]:
            if tgt_aff[l] > tgt_aff[target]:
                target = l
    elif thin[source]:
        target = source - 1
    else:
        return -1
    return target if source - target <= max_distance else -1


def step_reward(cfg, L_init, cv_before, cv_after, levels_before, levels_after, source_rows, source_thin,
                distance, abandon_penalty):
    """Algorithm 2; returns (total, (r_cv, r_cpath, r_rwdist, r_abandon))."""
    alpha = cfg.reward_alpha
    dcv = cv_before - cv_after
    r_cv = -alpha if dcv < -cfg.eps else (L_init * dcv if dcv > cfg.eps else 0.0)
    s = math.log(1.0 + source_rows + 1.0)
    if levels_after < levels_before:
        r_cp = alpha * (L_init / levels_after) * (1.0 + 1.0 / s)
    elif source_thin:
        r_cp = alpha / s
    else:
        r_cp = -1.0 * alpha * (1.0 + s)
    thr = cfg.rwdist_threshold
    r_rw = (math.log1p(max(0, thr - distance)) if distance < thr else -math.log1p(max(0, distance - thr))) / L_init
    r_ab = -abandon_penalty
    w = cfg.weights
    return w[0] * r_cv + w[1] * r_cp + w[2] * r_rw + w[3] * r_ab, (r_cv, r_cp, r_rw, r_ab)


class RewriteEnv:
    """Environment over a lower-triangular CSR matrix on the GPU."""

    def __init__(self, A: _api.Matrix, cfg: EnvConfig | None = None):
        self.cfg = cfg or EnvConfig()
        self.A = A
        self.an0 = _api.analyze(A)
        self.threshold = float(self.an0.stats[5])
        self.L_init = self.an0.nlevels
        self.rows: list = []
        self.targets: list = []
        self.moves: list = []
        self.Lp, self.T = A, None
        self._observe(A, self.an0)
        nl = self.nlevels
        self.thin_init = max(1, int(self.thin.sum()))
        self.src_aff = np.zeros(nl)
        self.tgt_aff = np.zeros(nl)
        self.init_size = self.level_rows.astype(np.int64).copy()
        self.first_touch = np.full(nl, -1, np.int64)
        self.was_target = np.zeros(nl, bool)
        self.last_source = -1
        self.t = 0
        self.since_collapse = 0

    def _observe(self, M, an):
        thin, pick, _ = _api.level_summary(M, an, self.threshold)
        self.an = an
        self.nlevels = an.nlevels
        self.level_ptr = an.level_ptr.cpu().numpy()
        self.level_rows = np.diff(self.level_ptr)
        self.cost = an.cost.cpu().numpy()
        self.thin = thin.cpu().numpy().astype(bool)
        self.pick = pick.cpu().numpy()

    @property
    def stats(self):
        return self.an.stats

    def valid_actions(self) -> np.ndarray:
        """Mask of the source levels the policy may pick (Section 4.3)."""
        mask = np.zeros(self.nlevels, bool)
        mask[1:] = True
        if self.last_source >= 1 and self.level_rows[self.last_source] == 1:
            mask[:] = False
            mask[self.last_source] = True
            return mask
        if self.since_collapse >= self.cfg.stagnation_steps:
            order = sorted(range(1, self.nlevels), key=lambda l: (-self.src_aff[l], l))
            keep = np.zeros_like(mask)
            keep[order[: self.cfg.stagnation_keep]] = True
            return keep
        return mask

    def observation(self) -> dict:
        """Per-level and global features of Table 1 (unnormalised)."""
        comp = 1.0 - self.level_rows / (self.init_size + 1.0)
        return dict(level_cost=self.cost, level_rows=self.level_rows, source_affinity=self.src_aff,
                    target_affinity=self.tgt_aff, completion_ratio=comp, thin=self.thin,
                    cv_cost=float(self.stats[3]), cv_rows=float(self.stats[4]), levels=self.nlevels,
                    rewrite_ratio=len(self.moves) / self.A.n,
                    thin_completion=float(self.thin.sum()) / self.thin_init,
                    critical_path_ratio=self.nlevels / self.L_init,
                    thin_ratio=float(self.thin.sum()) / max(self.nlevels, 1))

    def step(self, source: int):
        """One move from `source`.  Returns (reward, info)."""
        cfg = self.cfg
        if not (1 <= source < self.nlevels) or not self.valid_actions()[source]:
            raise ValueError("source level not valid")
        self.t += 1
        row = int(self.pick[source])
        target = target_level(source, self.thin, self.tgt_aff, cfg.search_window, cfg.max_rewrite_distance)
        if target < 0:
            self.since_collapse += 1
            return 0.0, dict(valid=False, row=row, source=source, target=-1)
        cv_before, levels_before = float(self.stats[3]), self.nlevels
        src_rows, src_thin = int(self.level_rows[source]), bool(self.thin[source])
        if self.first_touch[source] < 0:
            self.first_touch[source] = self.t
            self.init_size[source] = src_rows
        self.rows.append(row)
        self.targets.append(target)
        self.moves.append((row, source, target))
        Lp, T = _api.rewrite(self.A, self.an0.lev, self.rows, self.targets)
        an = _api.analyze(Lp, prev_lev=self.an.lev, first_row=row)
        self.Lp, self.T = Lp, T
        self._observe(Lp, an)
        d = levels_before - self.nlevels
        if d > 0:
            for name in ("src_aff", "tgt_aff", "init_size", "first_touch", "was_target"):
                setattr(self, name, np.delete(getattr(self, name), np.s_[source:source + d]))
        prev, prev_gone = self.last_source, False
        if prev >= 0 and d > 0:
            if source <= prev < source + d:
                prev_gone = True
            elif prev >= source + d:
                prev -= d
        penalty = 0.0
        if prev >= 1 and prev != source and not prev_gone:
            if self.was_target[prev]:
                self.init_size[prev] = int(self.level_rows[prev])
                self.first_touch[prev] = self.t
            else:
                comp = 1.0 - self.level_rows[prev] / (self.init_size[prev] + 1.0)
                penalty = (1.0 - comp) * math.log1p(self.t - self.first_touch[prev])
                if (self.level_rows == 1).any() and self.thin[prev]:
                    penalty = 0.0
        total, parts = step_reward(cfg, self.L_init, cv_before, float(self.stats[3]), levels_before, self.nlevels,
                                   src_rows, src_thin, source - target, penalty)
        self.src_aff *= cfg.affinity_decay
        self.tgt_aff *= cfg.affinity_decay
        if d == 0:
            self.src_aff[source] += cfg.affinity_boost
        self.tgt_aff[target] += cfg.affinity_boost
        thick = ~self.thin
        self.tgt_aff[thick] = np.minimum(self.tgt_aff[thick], -1.0)
        self.was_target[target] = True
        self.last_source = -1 if d > 0 else source
        self.since_collapse = 0 if d > 0 else self.since_collapse + 1
        return total, dict(valid=True, row=row, source=source, target=target, collapsed=d, parts=parts)

    def done(self) -> bool:
        return (self.thin.sum() / self.thin_init < self.cfg.thin_completion_stop or self.t >= self.cfg.max_steps
                or not self.valid_actions().any())

    def result(self):
        """The rewritten system (L', T) of the moves so far (L' x = b + T b)."""
        return self.Lp, self.T
