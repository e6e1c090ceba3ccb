"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is against a
library routine (dense triangular solve), a closed form, a brute-force
enumeration, the paper's printed numbers (tests/golden/paper_tables.txt) or a
hand-worked example.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr_from_dense(D):
    n = D.shape[0]
    rp, ci, v = [0], [], []
    for i in range(n):
        for j in range(i + 1):
            if D[i, j] != 0.0 or j == i:
                ci.append(j)
                v.append(D[i, j])
        rp.append(len(ci))
    return S.CSR(n, np.array(rp, np.int32), np.array(ci, np.int32), np.array(v, np.float64))


# --------------------------------------------------------------------- solve
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k", [1, 3])
def test_solve_matches_dense_triangular(seed, k):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 65))
    A = S.band_random(n, band=int(rng.integers(1, 20)), kmin=0, kmax=6, seed=seed)
    b = S.rhs(n, k, seed=seed + 7)
    x = oracle.solve(A, b)
    xr = sla.solve_triangular(A.dense(), b, lower=True)
    assert np.linalg.norm(x - xr) <= 1e-13 * max(1.0, np.linalg.norm(xr))


def test_solve_manufactured_solution():
    A = S.band_random(2000, 64, 0, 8, seed=0)
    rng = np.random.default_rng(5)
    xs = rng.uniform(-1, 1, size=(A.n, 2))
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    b = np.zeros_like(xs)
    np.add.at(b, rows, A.vals[:, None] * xs[A.col_idx])
    x = oracle.solve(A, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-12


@pytest.mark.parametrize("gen", ["lap2d", "band"])
def test_solve_backward_error_bound(gen):
    # Higham: the computed x of a triangular solve satisfies
    # (L + dL) x = b with |dL| <= n*eps/(1 - n*eps) |L| (row-wise), so the
    # normwise backward error is O(n eps); the row length bounds n here.
    A = S.lap2d(48) if gen == "lap2d" else S.band_random(3000, 200, 4, 16, seed=3)
    b = S.rhs(A.n, 1, seed=9)
    x = oracle.solve(A, b)[:, 0]
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    r = b[:, 0].copy()
    np.subtract.at(r, rows, A.vals * x[A.col_idx])
    normL = np.max(np.bincount(rows, weights=np.abs(A.vals), minlength=A.n))
    eta = np.max(np.abs(r)) / (normL * np.max(np.abs(x)) + np.max(np.abs(b)))
    maxlen = int(np.max(np.diff(A.row_ptr)))
    assert eta <= 2 * maxlen * np.finfo(float).eps


def test_solve_transpose_matches_dense():
    for seed in range(5):
        A = S.band_random(60, 12, 0, 6, seed=seed)
        g = S.rhs(60, 4, seed=seed + 1)
        gb = oracle.solve_transpose(A, g)
        ref = sla.solve_triangular(A.dense().T, g, lower=False)
        assert np.linalg.norm(gb - ref) <= 1e-13 * np.linalg.norm(ref)


def test_grad_vals_dense_closed_form():
    # loss = <w, x>, x = L^{-1} b:  dloss/dL = -(L^{-T} w) x^T restricted to
    # the pattern of L (matrix calculus closed form).
    A = S.band_random(40, 10, 1, 5, seed=11)
    b = S.rhs(40, 3, seed=1)
    w = S.rhs(40, 3, seed=2)
    x = oracle.solve(A, b)
    gb = oracle.solve_transpose(A, w)
    gv = oracle.grad_vals(A, gb, x)
    Ld = A.dense()
    G = -np.linalg.solve(Ld.T, w) @ np.linalg.solve(Ld, b).T
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    assert np.allclose(gv, G[rows, A.col_idx], rtol=1e-12, atol=1e-14)


def test_grad_central_differences():
    A = S.band_random(30, 8, 1, 5, seed=12)
    b = S.rhs(30, 2, seed=3)
    w = S.rhs(30, 2, seed=4)

    def loss(vals, bb):
        B = S.CSR(A.n, A.row_ptr, A.col_idx, vals)
        return float(np.sum(w * oracle.solve(B, bb)))

    x = oracle.solve(A, b)
    gb = oracle.solve_transpose(A, w)
    gv = oracle.grad_vals(A, gb, x)
    for p in range(0, A.nnz, 7):
        h = 1e-6 * max(1.0, abs(A.vals[p]))
        vp, vm = A.vals.copy(), A.vals.copy()
        vp[p] += h
        vm[p] -= h
        fd = (loss(vp, b) - loss(vm, b)) / (2 * h)
        assert abs(fd - gv[p]) <= 1e-6 * max(1.0, abs(gv[p]))
    for i in range(0, A.n, 5):
        h = 1e-6
        bp, bm = b.copy(), b.copy()
        bp[i, 1] += h
        bm[i, 1] -= h
        fd = (loss(A.vals, bp) - loss(A.vals, bm)) / (2 * h)
        assert abs(fd - gb[i, 1]) <= 1e-6 * max(1.0, abs(gb[i, 1]))


# -------------------------------------------------------------------- levels
def _brute_longest_path_levels(A):
    """Level of i = number of edges on the longest path ending at i, by
    enumerating every path in the DAG (tiny n only)."""
    n = A.n
    preds = [list(A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1] - 1]) for i in range(n)]
    best = [0] * n

    def walk(i, depth):
        best[i] = max(best[i], depth)
        # extend forward: successors of i
        for s in range(i + 1, n):
            if i in preds[s]:
                walk(s, depth + 1)

    for src in range(n):
        if not preds[src]:
            walk(src, 0)
    return np.array(best, np.int32)


@pytest.mark.parametrize("seed", range(25))
def test_levels_brute_force_longest_path(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 13))
    A = S.band_random(n, band=int(rng.integers(1, 13)), kmin=0, kmax=4, seed=seed)
    lev, nl = oracle.levels(A)
    ref = _brute_longest_path_levels(A)
    assert np.array_equal(lev, ref)
    assert nl == (int(ref.max()) + 1 if n else 0)


def test_levels_closed_forms():
    N = 37
    lev, nl = oracle.levels(S.lap2d(N))
    i = np.arange(N * N)
    assert np.array_equal(lev, (i // N) + (i % N)) and nl == 2 * N - 1
    M = 11
    lev, nl = oracle.levels(S.lap3d(M))
    i = np.arange(M ** 3)
    assert np.array_equal(lev, i // (M * M) + (i // M) % M + i % M) and nl == 3 * M - 2
    lev, nl = oracle.levels(S.chain(50))
    assert np.array_equal(lev, np.arange(50)) and nl == 50
    lev, nl = oracle.levels(S.diagonal(9))
    assert np.array_equal(lev, np.zeros(9)) and nl == 1
    lev, nl = oracle.levels(S.diagonal(0))
    assert nl == 0 and lev.size == 0


def test_levels_full_size_closed_form_lap2d():
    lev, nl = oracle.levels(S.lap2d(1024))
    assert nl == 2047
    i = np.arange(1024 * 1024)
    assert np.array_equal(lev, i // 1024 + i % 1024)


def test_partition_definition():
    A = S.band_random(3000, 50, 0, 8, seed=4)
    lev, nl = oracle.levels(A)
    perm, lp, cost = oracle.partition(A, lev, nl)
    order = np.lexsort((np.arange(A.n), lev))           # stable (level, row) sort
    assert np.array_equal(perm, order)
    assert np.array_equal(lp, np.concatenate([[0], np.cumsum(np.bincount(lev, minlength=nl))]))
    off = np.diff(A.row_ptr) - 1
    assert np.array_equal(cost, np.bincount(lev, weights=2 * off + 1, minlength=nl).astype(np.int64))


def test_cost_laplacian_closed_form():
    # level l of the N x N grid is the antidiagonal r + c = l; a node has a
    # west neighbour iff c > 0 and a south neighbour iff r > 0, cost per node
    # 1 + 2 * (#west + #south).
    N = 40
    A = S.lap2d(N)
    lev, nl = oracle.levels(A)
    _, _, cost = oracle.partition(A, lev, nl)
    ref = np.zeros(nl, np.int64)
    for r in range(N):
        for c in range(N):
            ref[r + c] += 1 + 2 * ((c > 0) + (r > 0))
    assert np.array_equal(cost, ref)


# --------------------------------------------------------------------- stats
def _paper_rows():
    rows = []
    with open(os.path.join(GOLDEN, "paper_tables.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows.append(dict(name=p[0], n=int(p[1]), nnz=int(p[2]), L=int(p[3]), alc=float(p[4]),
                             arl=float(p[5]), air=float(p[6]), cv=float(p[7]), thr=float(p[8])))
    return rows


def _matrix_with(n, nnz, L):
    """A lower-triangular CSR with exactly n rows, nnz stored entries and L
    levels: rows 0..L-1 form a chain, the remaining off-diagonals point into
    rows 0..L-2 so that no path gets longer."""
    k = np.zeros(n, np.int64)
    k[1:L] = 1
    extra = nnz - n - (L - 1)
    rest = n - L
    base, rem = divmod(extra, rest)
    k[L:] = base
    k[L:L + rem] += 1
    assert k.max() <= L - 1
    cols = []
    for i in range(n):
        if 1 <= i < L:
            cols.append(np.array([i - 1]))
        elif i >= L:
            cols.append(np.arange(k[i]))
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(k + 1, out=rp[1:])
    ci = np.empty(rp[-1], np.int32)
    off_pos = np.delete(np.arange(rp[-1]), rp[1:] - 1)
    ci[off_pos] = cols
    ci[rp[1:] - 1] = np.arange(n)
    v = np.ones(rp[-1])
    return S.CSR(n, rp.astype(np.int32), ci, v)


@pytest.mark.parametrize("row", _paper_rows(), ids=lambda r: r["name"])
def test_stats_reproduce_paper_tuples(row):
    A = _matrix_with(row["n"], row["nnz"], row["L"])
    res = oracle.analyze(A)
    assert res["nlevels"] == row["L"]
    alc, arl, air = res["stats"][:3]
    # ALC is printed truncated; gearbox prints 1,979 for 9,080,404/4,586 =
    # 1980.03 while its threshold 2224.62 agrees with 1980.03 (misprint).
    if row["name"] == "gearbox":
        assert abs(alc - row["alc"]) < 1.1
    else:
        assert math.floor(alc) == row["alc"]
    nd = len(str(row["arl"]).split(".")[1])
    assert round(arl, nd) == row["arl"]
    nd = len(str(row["air"]).split(".")[1])
    assert round(air, nd) == row["air"]
    # thin threshold with alpha = 1 and the printed CV (2 decimals)
    thr = oracle.thin_threshold(alc, row["cv"], 1.0)
    assert abs(thr - row["thr"]) <= 0.0051 * alc + 0.01
    implied_cv = 2.0 - row["thr"] / alc if row["cv"] < 1 else None
    if implied_cv is not None:
        assert round(implied_cv, 2) == row["cv"]
    else:  # CV > 1: the relaxation term vanishes, threshold == ALC
        assert round(thr, 2) == row["thr"]


def test_cov_population_definition_and_exactness():
    rng = np.random.default_rng(0)
    for trial in range(20):
        L = int(rng.integers(1, 300))
        scale = [1, 1000, 2 ** 40][trial % 3]
        cost = rng.integers(1, 50, size=L).astype(np.int64) * scale
        rows = rng.integers(1, 9, size=L)
        lp = np.concatenate([[0], np.cumsum(rows)]).astype(np.int32)
        st = oracle.stats(int(lp[-1]), int(lp[-1]) * 2, L, lp, cost)
        c = cost.astype(np.float64)
        assert abs(st[3] - c.std() / c.mean()) <= 1e-13 * max(1e-300, c.std() / c.mean()) + 1e-15
        r = rows.astype(np.float64)
        assert abs(st[4] - r.std() / r.mean()) <= 1e-13 * max(1e-300, r.std() / r.mean()) + 1e-15
        # exact-integer value, rounded once (Python ints are exact, float() and
        # math.sqrt are correctly rounded)
        S1, S2 = int(cost.sum()), sum(int(q) * int(q) for q in cost)
        exact = math.sqrt(float(L * S2 - S1 * S1)) / float(S1)
        assert st[3] == exact
    st = oracle.stats(2, 4, 2, np.array([0, 1, 2], np.int32), np.array([1, 3], np.int64))
    assert st[3] == 0.5 and st[4] == 0.0
    st = oracle.stats(5, 5, 5, np.arange(6, dtype=np.int32), np.full(5, 7, np.int64))
    assert st[3] == 0.0 and st[0] == 7.0 and st[5] == 14.0


# ------------------------------------------------------------------- rewrite
def test_rewrite_worked_example():
    # constructed example: L = [[2,0,0],[1,2,0],[0,1,2]], levels (0,1,2);
    # rewriting row 2 to level 1 substitutes row 1 (m = 1/2).
    A = _csr_from_dense(np.array([[2.0, 0, 0], [1, 2, 0], [0, 1, 2]]))
    lev, nl = oracle.levels(A)
    assert list(lev) == [0, 1, 2]
    Lp, T = oracle.rewrite(A, lev, [2], [1])
    assert list(Lp.row_ptr) == [0, 1, 3, 5]
    assert list(Lp.col_idx[3:5]) == [0, 2] and list(Lp.vals[3:5]) == [-0.5, 2.0]
    assert list(T.row_ptr) == [0, 0, 0, 1]
    assert list(T.col_idx) == [1] and list(T.vals) == [-0.5]
    lev2, nl2 = oracle.levels(Lp)
    assert list(lev2) == [0, 1, 1] and nl2 == 2
    b = np.array([2.0, 3.0, 4.0])
    assert np.array_equal(oracle.solve(A, b)[:, 0], [1.0, 1.0, 1.5])
    assert np.array_equal(oracle.solve_rewritten(Lp, T, b)[:, 0], [1.0, 1.0, 1.5])


def test_rewrite_lap2d_closed_form():
    # interior node (r, c) rewritten one level up: its west (i-1) and south
    # (i-N) neighbours are substituted; the new row couples to (r-2, c),
    # (r-1, c-1), (r, c-2) with -1/4, -1/2, -1/4 and T holds +1/4 at i-N, i-1.
    N = 12
    A = S.lap2d(N)
    lev, _ = oracle.levels(A)
    rows = np.array([r * N + c for r in range(2, N) for c in range(2, N)], np.int32)
    Lp, T = oracle.rewrite(A, lev, rows, lev[rows] - 1)
    for i in rows:
        a, e = Lp.row_ptr[i], Lp.row_ptr[i + 1]
        assert list(Lp.col_idx[a:e]) == [i - 2 * N, i - N - 1, i - 2, i]
        assert list(Lp.vals[a:e]) == [-0.25, -0.5, -0.25, 4.0]
        a, e = T.row_ptr[i], T.row_ptr[i + 1]
        assert list(T.col_idx[a:e]) == [i - N, i - 1] and list(T.vals[a:e]) == [0.25, 0.25]


@pytest.mark.parametrize("seed", range(4))
def test_rewrite_invariants(seed):
    A = S.band_random(2000, 64, 0, 8, seed=seed)
    an = oracle.analyze(A)
    lev = an["lev"]
    rows, tg = S.small_levels_list(an["nlevels"], an["level_ptr"], an["perm"], 4, 8)
    if seed % 2:  # also deep targets
        rng = np.random.default_rng(seed)
        cand = np.nonzero(lev >= 3)[0]
        extra = rng.choice(cand, size=40, replace=False).astype(np.int32)
        rows = np.concatenate([rows, extra])
        tg = np.concatenate([tg, (lev[extra] * rng.uniform(0, 1, 40)).astype(np.int32)])
    Lp, T = oracle.rewrite(A, lev, rows, tg)
    tmin = np.full(A.n, -1)
    for r, t in zip(rows, tg):
        tmin[r] = t if tmin[r] < 0 else min(tmin[r], t)
    # same solution
    b = S.rhs(A.n, 2, seed=seed)
    x = oracle.solve(A, b)
    xp = oracle.solve_rewritten(Lp, T, b)
    assert np.linalg.norm(xp - x) / np.linalg.norm(x) <= 1e-12
    lev2, _ = oracle.levels(Lp)
    assert np.all(lev2 <= lev)                       # no level increases
    rw = np.nonzero(tmin >= 0)[0]
    assert np.all(lev2[rw] <= tmin[rw]) and np.all(tmin[rw] < lev[rw])
    for i in rw:                                      # no column at level >= t survives
        cols = Lp.col_idx[Lp.row_ptr[i]:Lp.row_ptr[i + 1] - 1]
        assert np.all(lev[cols] < tmin[i])
    # unchanged rows are copied
    keep = np.nonzero(tmin < 0)[0][:200]
    for i in keep:
        assert np.array_equal(Lp.col_idx[Lp.row_ptr[i]:Lp.row_ptr[i + 1]],
                              A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]])
        assert T.row_ptr[i] == T.row_ptr[i + 1]


def test_rewrite_one_level_round_count():
    # with t = lev(i) - 1 exactly the columns at level lev(i)-1 that row i (or
    # a substituted row) touches are eliminated, one substitution each.
    A = S.band_random(500, 20, 1, 6, seed=21)
    lev, _ = oracle.levels(A)
    rows = np.nonzero(lev >= 1)[0][::7].astype(np.int32)
    Lp, T = oracle.rewrite(A, lev, rows)
    for i in rows:
        t = lev[i] - 1
        deps = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1] - 1]
        # levels strictly decrease along edges, so only the direct deps at
        # level t can be eliminated
        expect = sorted(d for d in deps if lev[d] >= t)
        assert list(T.col_idx[T.row_ptr[i]:T.row_ptr[i + 1]]) == expect


def test_rewrite_errors_and_duplicates():
    A = S.band_random(200, 10, 1, 4, seed=2)
    lev, _ = oracle.levels(A)
    z = int(np.nonzero(lev == 0)[0][0])
    with pytest.raises(oracle.OracleError) as e:
        oracle.rewrite(A, lev, [z], [0])
    assert e.value.status == oracle.ETARGET
    i = int(np.nonzero(lev >= 3)[0][0])
    with pytest.raises(oracle.OracleError) as e:
        oracle.rewrite(A, lev, [i], [lev[i]])
    assert e.value.status == oracle.ETARGET
    with pytest.raises(oracle.OracleError) as e:
        oracle.rewrite(A, lev, [A.n], [0])
    assert e.value.status == oracle.EINVAL
    Lp1, T1 = oracle.rewrite(A, lev, [i, i], [lev[i] - 1, 1])
    Lp2, T2 = oracle.rewrite(A, lev, [i], [1])
    assert np.array_equal(Lp1.col_idx, Lp2.col_idx) and np.array_equal(T1.vals, T2.vals)


def test_rewritten_gradient_identity():
    # x is the same function of b before and after the rewrite, so
    # T^T-applied g_b' equals the original g_b.
    A = S.band_random(1500, 40, 0, 8, seed=8)
    an = oracle.analyze(A)
    rows, tg = S.narrowest_levels_list(an["nlevels"], an["level_ptr"], an["perm"], 0.05, 8)
    Lp, T = oracle.rewrite(A, an["lev"], rows, tg)
    w = S.rhs(A.n, 3, seed=1)
    gb = oracle.solve_transpose(A, w)
    gbp = oracle.solve_transpose(S.CSR(Lp.n, Lp.row_ptr, Lp.col_idx, Lp.vals), w)
    gb2 = oracle.tt_apply(T, gbp)
    assert np.linalg.norm(gb2 - gb) / np.linalg.norm(gb) <= 1e-12


def _validate_fixture():
    """A valid 60-row system with at least two off-diagonals per row from row
    10 on (rows are hand-edited below)."""
    A = S.band_random(60, 8, 2, 4, seed=1)
    return A


def _copy(A):
    return S.CSR(A.n, A.row_ptr.copy(), A.col_idx.copy(), A.vals.copy())


def _drop_row_entries(A, i):
    """Row i without any entry (row pointers shifted)."""
    a, e = int(A.row_ptr[i]), int(A.row_ptr[i + 1])
    rp = A.row_ptr.copy()
    rp[i + 1:] -= e - a
    return S.CSR(A.n, rp, np.delete(A.col_idx, np.s_[a:e]), np.delete(A.vals, np.s_[a:e]))


def test_validate_codes():
    """Every status of the validation (Section 2.1: lower triangular, columns
    sorted, a non-zero diagonal stored last), each for one planted fault with
    the exact row, and the first-offending rules: the smallest bad row wins,
    and inside a row the first bad position decides between 'outside [0, i]'
    and 'not strictly increasing'."""
    A = _validate_fixture()
    rp = A.row_ptr
    assert oracle.validate(A) == (oracle.OK, -1)
    # zero diagonal
    B = _copy(A)
    B.vals[rp[11] - 1] = 0.0
    assert oracle.validate(B) == (oracle.EDIAG, 10)
    # a column above the diagonal at the row's first position
    B = _copy(A)
    B.col_idx[rp[20]] = 30
    assert oracle.validate(B) == (oracle.ENOTLOWER, 20)
    # a negative column
    B = _copy(A)
    B.col_idx[rp[21]] = -1
    assert oracle.validate(B) == (oracle.ENOTLOWER, 21)
    # two off-diagonals swapped
    B = _copy(A)
    B.col_idx[rp[25]], B.col_idx[rp[25] + 1] = B.col_idx[rp[25] + 1], B.col_idx[rp[25]]
    assert oracle.validate(B) == (oracle.EUNSORTED, 25)
    # a repeated column is not strictly increasing
    B = _copy(A)
    B.col_idx[rp[26] + 1] = B.col_idx[rp[26]]
    assert oracle.validate(B) == (oracle.EUNSORTED, 26)
    # the last entry is not the diagonal (sorted, lower, but != i)
    B = _copy(A)
    i = next(r for r in range(35, A.n) if B.col_idx[rp[r + 1] - 2] + 1 < r)
    B.col_idx[rp[i + 1] - 1] = B.col_idx[rp[i + 1] - 2] + 1
    assert oracle.validate(B) == (oracle.EDIAG, i)
    # an empty row has no diagonal; decreasing row pointers are invalid
    assert oracle.validate(_drop_row_entries(A, 40)) == (oracle.EDIAG, 40)
    B = _copy(A)
    B.row_ptr[45] = B.row_ptr[44] - 1           # row 44 ends before it starts
    assert oracle.validate(B) == (oracle.EINVAL, 44)
    B = _copy(A)
    B.row_ptr[0] = 1
    assert oracle.validate(B) == (oracle.EINVAL, 0)
    # first offending row in row order wins
    B = _copy(A)
    B.col_idx[rp[50]] = 55
    B.vals[rp[13] - 1] = 0.0
    assert oracle.validate(B) == (oracle.EDIAG, 12)
    # inside a row, the first bad position decides
    B = _copy(A)
    B.col_idx[rp[30]] = 40                      # position 0: above the diagonal
    B.col_idx[rp[30] + 1] = 0                   # position 1: also decreasing
    assert oracle.validate(B) == (oracle.ENOTLOWER, 30)
    B = _copy(A)
    B.col_idx[rp[33] + 1] = -1                  # position 1: negative AND decreasing: the range
    assert oracle.validate(B) == (oracle.ENOTLOWER, 33)  # check comes first
    C = _copy(A)
    C.col_idx[rp[32] + 1] = C.col_idx[rp[32]]   # position 1 repeated, position 2 above the diagonal
    C.col_idx[rp[32] + 2] = 99
    assert rp[33] - rp[32] >= 4                 # row 32 has three off-diagonals and the diagonal
    assert oracle.validate(C) == (oracle.EUNSORTED, 32)


# --------------------------------------------------- environment summary
def _lap2d_closed_form(N):
    """Level l of the N x N 5-point lower triangle (natural order): rows
    (r, c) with r + c = l; deps = [c > 0] + [r > 0]; row cost 2 deps + 1."""
    L = 2 * N - 1
    cost = np.zeros(L, np.int64)
    rows = np.zeros(L, np.int64)
    pick = np.zeros(L, np.int64)
    for l in range(L):
        cells = [(r, l - r) for r in range(N) if 0 <= l - r < N]
        rows[l] = len(cells)
        cost[l] = sum(2 * ((c > 0) + (r > 0)) + 1 for r, c in cells)
        # fewest dependencies: the origin, else a boundary cell (r = 0 has the
        # smallest index), else the interior cell with the smallest r
        pick[l] = 0 if l == 0 else (l if l < N else (l - N + 1) * N + N - 1)
    return cost, rows, pick


@pytest.mark.parametrize("N", [2, 6, 17, 40])
def test_level_summary_lap2d_closed_form(N):
    A = S.lap2d(N)
    an = oracle.analyze(A)
    cost, rows, pick = _lap2d_closed_form(N)
    alc = cost.sum() / len(cost)
    cv = cost.std() / cost.mean()  # population
    thr = alc * (1 + max(0.0, 1 - cv))
    thin, pk, out = oracle.level_summary(A, an, thr)
    assert np.array_equal(pk, pick)
    assert np.array_equal(thin.astype(bool), cost < thr)
    t = cost < thr
    assert out[0] == t.sum()
    assert out[1] == (rows[t].max() if t.any() else 0)
    assert out[2] == (cost[t].max() if t.any() else 0)


@pytest.mark.parametrize("seed", range(6))
def test_level_summary_brute_force(seed):
    """Per-level minimum of (dependencies, row) by a global sort, and the
    thin set by a direct comparison, on small random systems."""
    A = S.band_random(300, 24, 0, 6, seed=100 + seed)
    an = oracle.analyze(A)
    deps = np.diff(A.row_ptr) - 1
    lev = an["lev"]
    order = np.lexsort((np.arange(A.n), deps, lev))  # by level, then deps, then row
    first = order[np.r_[0, np.flatnonzero(np.diff(lev[order])) + 1]]
    thr = 0.9 * an["cost"].mean()
    thin, pk, out = oracle.level_summary(A, an, thr)
    assert np.array_equal(pk, first)
    assert np.array_equal(thin.astype(bool), an["cost"] < thr)
    assert out[0] == int((an["cost"] < thr).sum())


def test_level_summary_default_threshold_is_the_papers():
    A = S.lap2d(9)
    an = oracle.analyze(A)
    thin, _, _ = oracle.level_summary(A, an)
    assert np.array_equal(thin.astype(bool), an["cost"] < an["stats"][5])


def test_level_summary_threshold_is_strict():
    """A level whose cost equals the threshold is not thin (Section 4.1:
    thin means a cost smaller than the threshold)."""
    A = S.lap2d(6)
    an = oracle.analyze(A)
    cost, _, _ = _lap2d_closed_form(6)
    thr = float(cost[3])  # 5 * 3 + 1 = 16, also the cost of no other level
    thin, _, out = oracle.level_summary(A, an, thr)
    assert not thin[3] and thin[2] and out[0] == int((cost < thr).sum())
