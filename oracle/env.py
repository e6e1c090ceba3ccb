"""Oracle of the paper's environment step -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of the graph-transformation environment of the
paper's Section 4 on top of the CPU oracle (``oracle.rewrite``,
``oracle.analyze``, ``oracle.level_summary``), written from the paper's text:

  Section 4.1  thin levels: cost below ALC * (1 + alpha * max(0, 1 - CV)),
               with ALC and CV of the episode's initial system (they stay
               constant through an episode);
  Section 4.3  actions are source levels; level 0 is never a source; the row
               moved is the one with the fewest dependencies; two masking
               heuristics (a source level with one row left forces its
               collapse; after a stagnant period only the X source levels of
               highest affinity stay valid);
  Algorithm 1  target level: the thin level of highest target affinity among
               the SEARCH_WINDOW nearest thin levels above the source; without
               one, the nearest non-empty level above when the source is thin,
               otherwise the action is invalid; a move longer than
               MAX_REWRITE_DISTANCE is invalid;
  Algorithm 2  reward 0.80 r_cv + 0.80 r_cpath + 0.05 r_rwdist + 0.50 r_abandon;
  Section 4.2  source and target affinities (decay, boost, negative for levels
               that stop being candidates), completion ratio
               1 - size / (initial size + 1), thin-level completion ratio as
               the stopping rule.

Readings (where the paper leaves a step open) are the same ones the library's
environment takes; each is a named field of ``Config``.  Levels are always
recomputed from scratch (longest-path depths, no empty levels), so a level
that empties disappears and the per-level state of the levels after it moves
down by one index.  A move is the rewrite of the picked row towards the
target level in the current numbering, applied with the library's rewrite
semantics (original rows and original levels; a row moved twice keeps its
smaller target), after which the row sits at the target level or above it.

Nothing here is imported by the CUDA library or its Python package.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

import oracle


@dataclass
class Config:
    search_window: int = 5            # SEARCH_WINDOW (Section 4.4 names "the closest five")
    max_rewrite_distance: int = 16    # MAX_REWRITE_DISTANCE (value not stated)
    reward_alpha: float = 1.0         # alpha of Algorithm 2 (value not stated)
    eps: float = 1e-4                 # epsilon of Algorithm 2 (value not stated)
    rwdist_threshold: int = 5         # threshold of the rewriting-distance reward (not stated)
    affinity_decay: float = 0.9       # affinity decay per step (not stated)
    affinity_boost: float = 1.0       # added to the selected levels' affinities (not stated)
    stagnation_steps: int = 20        # steps without a collapse before the second mask (not stated)
    stagnation_keep: int = 5          # X of Section 4.3 (not stated)
    thin_completion_stop: float = 0.1  # episode ends below this thin-level ratio (not stated)
    max_steps: int = 1000
    weights: tuple = (0.80, 0.80, 0.05, 0.50)  # Algorithm 2


def select_target(ls, thin, tgt_aff, window, max_distance):
    """Algorithm 1 for source level ls (>= 1): returns the target level or -1.
    thin[l] and tgt_aff[l] describe the current levels."""
    cands = []
    l = ls - 1
    while l >= 0 and len(cands) < window:
        if thin[l]:
            cands.append(l)
        l -= 1
    if cands:
        best = cands[0]
        for l in cands[1:]:
            if tgt_aff[l] > tgt_aff[best]:  # strict: ties keep the nearer level
                best = l
        lt = best
    elif thin[ls]:
        lt = ls - 1          # nearest non-empty level above: a thin source may go to a thick level
    else:
        return -1            # thick source and no thin level above
    if ls - lt > max_distance:
        return -1
    return lt


def reward(cfg, L_init, cv_prev, cv_now, nlevels_prev, nlevels_now, src_size, src_thin, distance,
           abandon_penalty):
    """Algorithm 2, with Delta CV = previous CV - current CV (positive when the
    level costs became more even).  Returns (total, components)."""
    a = cfg.reward_alpha
    dcv = cv_prev - cv_now
    if dcv < -cfg.eps:
        r_cv = -a
    elif dcv > cfg.eps:
        r_cv = L_init * dcv
    else:
        r_cv = 0.0
    s = math.log(1.0 + src_size + 1.0)
    if nlevels_now < nlevels_prev:
        r_cp = a * (L_init / nlevels_now) * (1.0 + 1.0 / s)
    elif src_thin:
        r_cp = a / s
    else:
        r_cp = -1.0 * a * (1.0 + s)
    thr = cfg.rwdist_threshold
    if distance < thr:
        r_rw = math.log1p(max(0, thr - distance)) / L_init
    else:
        r_rw = -math.log1p(max(0, distance - thr)) / L_init
    r_ab = -abandon_penalty
    w = cfg.weights
    total = w[0] * r_cv + w[1] * r_cp + w[2] * r_rw + w[3] * r_ab
    return total, (r_cv, r_cp, r_rw, r_ab)


@dataclass
class State:
    lev: np.ndarray
    perm: np.ndarray
    level_ptr: np.ndarray
    cost: np.ndarray
    nlevels: int
    stats: np.ndarray
    thin: np.ndarray
    pick: np.ndarray

    @property
    def rows(self):
        return np.diff(self.level_ptr)


class Env:
    """The environment on the CPU oracle."""

    def __init__(self, A, cfg: Config | None = None):
        self.cfg = cfg or Config()
        self.A = A
        an = oracle.analyze(A)
        self.lev0 = an["lev"]
        self.threshold = float(an["stats"][5])   # from the initial ALC and CV, fixed
        self.L_init = an["nlevels"]
        self.moves = []                          # (row, source level, target level)
        self.rows, self.targets = [], []
        self.Lp = A
        self.state = self._state(A, an)
        nl = self.state.nlevels
        self.thin_init = max(1, int(self.state.thin.sum()))
        self.src_aff = np.zeros(nl)
        self.tgt_aff = np.zeros(nl)
        self.init_size = self.state.rows.astype(np.int64).copy()
        self.first_touch = np.full(nl, -1, np.int64)
        self.was_target = np.zeros(nl, bool)
        self.last_source = -1
        self.t = 0
        self.since_collapse = 0

    def _state(self, M, an):
        thin, pick, _ = oracle.level_summary(M, an, self.threshold)
        return State(an["lev"], an["perm"], an["level_ptr"], an["cost"], an["nlevels"], an["stats"],
                     thin.astype(bool), pick)

    def valid_actions(self):
        st = self.state
        mask = np.zeros(st.nlevels, bool)
        mask[1:] = True
        if self.last_source >= 1 and st.rows[self.last_source] == 1:
            only = np.zeros_like(mask)
            only[self.last_source] = True
            return only
        if self.since_collapse >= self.cfg.stagnation_steps:
            cand = [l for l in range(1, st.nlevels)]
            cand.sort(key=lambda l: (-self.src_aff[l], l))
            keep = np.zeros_like(mask)
            keep[cand[: self.cfg.stagnation_keep]] = True
            return keep
        return mask

    def _delete_levels(self, at, d):
        for name in ("src_aff", "tgt_aff", "init_size", "first_touch", "was_target"):
            arr = getattr(self, name)
            setattr(self, name, np.delete(arr, np.s_[at:at + d]))

    def step(self, ls):
        """One move from source level ls.  Returns (reward, info); an invalid
        move leaves the state as it was and earns 0."""
        cfg = self.cfg
        st = self.state
        if ls < 1 or ls >= st.nlevels or not self.valid_actions()[ls]:
            raise ValueError("source level not valid")
        self.t += 1
        n = int(st.pick[ls])
        lt = select_target(ls, st.thin, self.tgt_aff, cfg.search_window, cfg.max_rewrite_distance)
        if lt < 0:
            self.since_collapse += 1
            return 0.0, dict(valid=False, row=n, source=ls, target=-1)
        cv_prev, nl_prev = float(st.stats[3]), st.nlevels
        src_size, src_thin = int(st.rows[ls]), bool(st.thin[ls])
        if self.first_touch[ls] < 0:
            self.first_touch[ls] = self.t
            self.init_size[ls] = src_size
        self.rows.append(n)
        self.targets.append(lt)
        self.moves.append((n, ls, lt))
        Lp, _ = oracle.rewrite(self.A, self.lev0, self.rows, self.targets)
        self.Lp = Lp
        an = oracle.analyze(Lp)
        new = self._state(Lp, an)
        d = nl_prev - new.nlevels
        if d > 0:
            self._delete_levels(ls, d)
        # the previous source level, renumbered
        prev = self.last_source
        prev_collapsed = False
        if prev >= 0 and d > 0:
            if ls <= prev < ls + d:
                prev_collapsed = True
            elif prev >= ls + d:
                prev -= d
        self.state = new
        # abandonment of the previous source level (Algorithm 2, r_abandon)
        penalty = 0.0
        if prev >= 1 and prev != ls and not prev_collapsed:
            if self.was_target[prev]:
                self.init_size[prev] = int(new.rows[prev])
                self.first_touch[prev] = self.t
            else:
                comp = 1.0 - new.rows[prev] / (self.init_size[prev] + 1.0)
                penalty = (1.0 - comp) * math.log1p(self.t - self.first_touch[prev])
                if (new.rows == 1).any() and new.thin[prev]:
                    penalty = 0.0
        total, parts = reward(cfg, self.L_init, cv_prev, float(new.stats[3]), nl_prev, new.nlevels, src_size,
                              src_thin, ls - lt, penalty)
        # affinities
        self.src_aff *= cfg.affinity_decay
        self.tgt_aff *= cfg.affinity_decay
        collapsed = d > 0
        if not collapsed:
            self.src_aff[ls] += cfg.affinity_boost
        self.tgt_aff[lt] += cfg.affinity_boost
        self.tgt_aff[~new.thin] = np.minimum(self.tgt_aff[~new.thin], -1.0)
        self.was_target[lt] = True
        self.last_source = -1 if collapsed else ls
        self.since_collapse = 0 if collapsed else self.since_collapse + 1
        return total, dict(valid=True, row=n, source=ls, target=lt, collapsed=d, parts=parts)

    def done(self):
        st = self.state
        return (st.thin.sum() / self.thin_init < self.cfg.thin_completion_stop or self.t >= self.cfg.max_steps
                or not self.valid_actions().any())
