"""Pins of the oracle's aggregation, veto, test vectors, cycle schedule and recombination (no GPU).

Each test recomputes what the paper fixes from the level's own operator and test vectors with
independent code (dense or scipy linear algebra, direct energy minimisation, hand-derived
counts), so that a plausible slip in the oracle (a flipped comparison, the wrong row for the
veto, a dropped candidate, another rounding of the fractional cycle index, a stale history in
the recombination) fails one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as sopt

import graphgen as gg
import oracle

Q = 2.5          # Eq. 4
TAU = 0.05       # Eq. 9


def rows_of(L):
    return np.repeat(np.arange(L["n"]), np.diff(L["rp"]))


def affinity_np(xu, xv):
    """Eq. 3 as the squared cosine of the two test-vector profiles."""
    return float((xu @ xv) ** 2 / ((xu @ xu) * (xv @ xv)))


def strong_np(L, u):
    """Eq. 9 from u's side, recomputed: |w_uv| >= tau max_t |w_ut|."""
    a = np.abs(L["val"][L["rp"][u]:L["rp"][u + 1]])
    return a >= TAU * a.max()


def energy_ratio(w, xnb, xs):
    """Eq. 4 by direct minimisation of the nodal energy E(y) = 1/2 sum_v w_v (y - x_v)^2 per
    test vector (numerical minimisation, no moments): max_k E(x_s) / min_y E(y)."""
    q = 0.0
    for k in range(xnb.shape[1]):
        E = lambda y: 0.5 * np.sum(w * (y - xnb[:, k]) ** 2)
        res = sopt.minimize_scalar(E, bracket=(xnb[:, k].min() - 1, xnb[:, k].max() + 1), tol=1e-14)
        relaxed = res.fun
        forced = E(xs[k])
        if relaxed <= 1e-12 * max(forced, 1e-300):
            return 1.0 if forced <= 1e-12 else math.inf
        q = max(q, forced / relaxed)
    return q


AGG_GRAPHS = [
    ("aniso 28x24", lambda: gg.grid2d(28, 24, 1.0, 1e-3)),
    ("random 500", lambda: gg.random_connected(500, 1400, seed=21)),
    ("barabasi-albert 600", lambda: gg.barabasi_albert(600, 4, seed=3)),
    ("heterogeneous 3D 7^3", lambda: gg.grid3d(7, 7, 7, "loguniform", seed=2)),
]


@pytest.mark.parametrize("name,make", AGG_GRAPHS)
def test_aggregation_choices_follow_section_2(name, make):
    """Section 2 / Eq. 4 / Eq. 9, on the first aggregation level (positive weights, so the
    nodal energy is a convex quadratic):
      - every associate's seed is a neighbour, is a seed, and its edge is strong from the
        associate's side;
      - the associate passes the energy guard q <= Q for that seed;
      - no strong neighbour that ended as a seed and passes the guard has a larger affinity
        (ties: the lower index) -- final seeds were all candidates when u was visited;
      - a seed that no earlier node joined had no admissible strong neighbour among the final
        seeds (it was undecided at its own visit and found no candidate)."""
    g = make()
    H = oracle.Hierarchy(g, coarsest_max=16)
    L = next(l for l in H.levels if l["kind"] == "agg")
    assert np.all(L["val"] < 0)                       # a Laplacian level: w_uv = -A_uv > 0
    X, seed_of, n = L["X"], L["seed_of"], L["n"]
    is_seed = seed_of == np.arange(n)
    joined_by_earlier = np.zeros(n, bool)
    for u in np.flatnonzero(~is_seed):
        if seed_of[u] > u:
            joined_by_earlier[seed_of[u]] = True
    checked = 0
    for u in range(n):
        e0, e1 = L["rp"][u], L["rp"][u + 1]
        nb = L["ci"][e0:e1]
        w = -L["val"][e0:e1]
        st = strong_np(L, u)
        # candidates among the final seeds: strong, admissible
        cand = [(affinity_np(X[u], X[v]), v) for j, v in enumerate(nb)
                if st[j] and is_seed[v] and energy_ratio(w, X[nb], X[v]) <= Q]
        if not is_seed[u]:
            s = seed_of[u]
            assert s in nb and is_seed[s], (name, u, s)
            j = int(np.flatnonzero(nb == s)[0])
            assert st[j], (name, u, s)
            assert energy_ratio(w, X[nb], X[s]) <= Q * (1 + 1e-9), (name, u, s)
            c_s = affinity_np(X[u], X[s])
            for c, v in cand:
                assert c < c_s * (1 + 1e-12) or (math.isclose(c, c_s, rel_tol=1e-12) and v >= s), (name, u, s, v)
            checked += 1
        elif not joined_by_earlier[u]:
            assert not cand, (name, u, cand)
    assert checked > n // 4


def _graph_matrix(n, edges):
    u = np.array([a for a, b in edges]); v = np.array([b for a, b in edges])
    g = gg.from_edges(n, u, v, np.ones(len(edges)))
    return g, oracle.laplacian(g)


def _entry_values(g, table, default):
    """Per stored entry (u, v) of g: table.get((u, v), default)."""
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    return np.array([table.get((int(a), int(b)), default) for a, b in zip(rows, g.ci)])


def test_aggregation_candidates_ties_and_visit_order():
    # Section 2 readings on caller data (identical test-vector profiles, so every energy ratio
    # is 1 and every strong neighbour is admissible): nodes visited in ascending order; an
    # undecided node joins the strong neighbour of largest affinity among seeds and undecided
    # nodes (never an associate); ties go to the lower index; the chosen node becomes a seed.
    #   node 0: neighbours 1, 2 tie at 0.9          -> joins 1 (lower index); 1 becomes a seed
    #   node 2: neighbour 0 is an associate (0.95)  -> joins 3 (0.5); 3 becomes a seed
    #   node 4: seed 3 and undecided 5 tie at 0.5   -> joins 3
    #   node 5: seed 1 (0.5), associate 4 (0.99)     -> joins 1
    g, A = _graph_matrix(6, [(0, 1), (0, 2), (2, 3), (3, 4), (4, 5), (1, 5)])
    aff = _entry_values(g, {(0, 1): 0.9, (0, 2): 0.9, (2, 0): 0.95, (5, 4): 0.99}, 0.5)
    seed_of, nc = oracle.aggregate(A, np.ones((6, 4)), aff, np.ones(len(aff), np.uint8))
    assert seed_of.tolist() == [1, 1, 3, 3, 3, 1] and nc == 2
    # a vetoed edge is no candidate: node 0's edge to 1 weak from 0's side -> joins 2
    strong = _entry_values(g, {(0, 1): 0}, 1).astype(np.uint8)
    seed_of, _ = oracle.aggregate(A, np.ones((6, 4)), aff, strong)
    assert seed_of[0] == 2


def test_aggregation_guard_and_singletons():
    # Eq. 4 decides admissibility: node 0 has leaves 1, 2, 3 with profiles 2, -1, -1 (weights 1).
    # Relaxed energy 1/2 (4 + 1 + 1) = 3; forced onto 1: 1/2 (0 + 9 + 9) = 9, q = 3 > 2.5
    # (inadmissible although its affinity is the largest); forced onto 2: 1/2 (9 + 0 + 0) = 4.5,
    # q = 1.5 -> node 0 joins 2. Leaves 1 and 3 then see only an associate and stay singletons.
    g, A = _graph_matrix(4, [(0, 1), (0, 2), (0, 3)])
    X = np.array([[0.0] * 4, [2.0] * 4, [-1.0] * 4, [-1.0] * 4])
    aff = _entry_values(g, {(0, 1): 0.9, (0, 2): 0.6, (0, 3): 0.5}, 0.5)
    seed_of, nc = oracle.aggregate(A, X, aff, np.ones(len(aff), np.uint8))
    assert seed_of.tolist() == [2, 1, 2, 3] and nc == 3
    # with Q = 3 the strongest-affinity leaf is admissible
    seed_of, _ = oracle.aggregate(A, X, aff, np.ones(len(aff), np.uint8), Q=3.0)
    assert seed_of[0] == 1


def test_veto_is_taken_from_the_nodes_own_row():
    # Eq. 9 with the maximum over u's own incident weights. A complete graph on 6 nodes (degree
    # 5 > d_max, and the dense-level rule off, so level 0 aggregates). Edge (0,1) has weight 0.04: weak from node 0, whose
    # strongest edge is 1, but strong from node 1, whose strongest edge is 0.5 (0.04 >= 0.025).
    # Edge (0,2) sits exactly on node 0's threshold (0.05 = 0.05 * 1): strong (the test is >=).
    n = 6
    W = np.full((n, n), 0.5)
    W[0, :] = W[:, 0] = 1.0
    W[0, 1] = W[1, 0] = 0.04
    W[0, 2] = W[2, 0] = 0.05
    W[1, 3] = W[3, 1] = 0.02          # weak from 1 (0.02 < 0.025) and from 3 (max 0.5)
    np.fill_diagonal(W, 0.0)
    iu = np.triu_indices(n, 1)
    g = gg.from_edges(n, iu[0], iu[1], W[iu])
    H = oracle.Hierarchy(g, coarsest_max=2, dense_rows=0)
    L = H.levels[0]
    assert L["kind"] == "agg"
    strong = {}
    for e, u in enumerate(rows_of(L)):
        strong[(u, int(L["ci"][e]))] = bool(L["strong"][e])
    assert strong[(0, 1)] is False and strong[(1, 0)] is True
    assert strong[(0, 2)] is True and strong[(2, 0)] is True
    assert strong[(1, 3)] is False and strong[(3, 1)] is False
    assert sum(not v for v in strong.values()) == 3
    # with the veto off every edge is a candidate
    assert oracle.Hierarchy(g, coarsest_max=2, dense_rows=0, veto=0).levels[0]["strong"].all()


@pytest.mark.parametrize("name,make", [
    ("grid with degree-600 hubs", lambda: gg.grid_with_hubs(36, 36, 4, 600, seed=2)),
    ("barabasi-albert 3000", lambda: gg.barabasi_albert(3000, 4, seed=5)),
])
def test_test_vectors_are_gauss_seidel_on_Ax_eq_0(name, make):
    # Section 2: each test vector is nu = 3 Gauss-Seidel sweeps on A x = 0 from the random start.
    # A sweep in colour order pi solves (D + L_pi) x' = -U_pi x (textbook splitting); checked on
    # levels with rows far longer than 32 entries.
    g = make()
    H = oracle.Hierarchy(g, coarsest_max=16)
    lvl = next(i for i, l in enumerate(H.levels) if l["kind"] == "agg")
    L = H.levels[lvl]
    assert np.diff(L["rp"]).max() > 64
    M = L["A"].dense()
    col = L["colour"]
    pi = np.concatenate([np.flatnonzero(col == c) for c in range(L["ncol"])])
    Pm = M[np.ix_(pi, pi)]
    low, up = np.tril(Pm), np.triu(Pm, 1)
    for k in range(4):
        x = np.array([oracle.random_start(3, lvl, u, k) for u in range(L["n"])])[pi]
        for _ in range(3):
            x = sla.solve_triangular(low, -up @ x, lower=True)
        got = L["X"][pi, k]
        assert np.max(np.abs(got - x)) <= 1e-11 * np.max(np.abs(x)), (name, k)


def test_random_start_columns_are_distinct_draws():
    # every (level, node, column) has its own counter: column k >= 4 of node u is not column
    # k - 4 of node u + 1 (a narrow column field would alias them)
    for k in range(4, 16):
        assert oracle.random_start(3, 1, 10, k) != oracle.random_start(3, 1, 11, k - 4)
    vals = {oracle.random_start(3, 0, u, k) for u in range(64) for k in range(16)}
    assert len(vals) == 64 * 16


def test_k_above_sixteen_is_rejected():
    with pytest.raises(ValueError):
        oracle.Hierarchy(gg.grid2d(20, 20), K=17)


def edge_count(L):
    """|E| of a level counted from its CSR: pairs u < v with a stored entry."""
    r = rows_of(L)
    return int(np.sum(r < L["ci"]))


@pytest.mark.parametrize("make", [lambda: gg.rgg(5000, 10, seed=1), lambda: gg.grid2d(60, 60),
                                  lambda: gg.grid3d(16, 16, 16, "loguniform", seed=1)])
def test_cycle_index_follows_eq5(make):
    # Eq. 5: elimination levels 1; an aggregation level 1.5 while |E_l| > 0.1 |E|, else
    # min(2, 0.7 / tau_l) with tau_l = |E_{l+1}| / |E_l| (clamped below at 1), from edges
    # counted here on the levels' own operators.
    H = oracle.Hierarchy(make(), coarsest_max=16)
    lv = H.levels
    E = [edge_count(L) for L in lv]
    saw_fraction = False
    for l, L in enumerate(lv):
        if L["kind"] == "elim":
            assert L["gamma"] == 1.0
        elif L["kind"] == "agg":
            if E[l] > 0.1 * E[0]:
                expect = 1.5
            else:
                expect = max(1.0, min(2.0, 0.7 / (E[l + 1] / E[l])))
                saw_fraction = saw_fraction or expect != 1.5
            assert L["gamma"] == pytest.approx(expect, rel=1e-15), (l, E[l], E[l + 1])
    assert saw_fraction


def test_fractional_cycle_index_visit_counts():
    # Reading of a fractional gamma: at the j-th visit of level l (counted from 0 within one
    # cycle), level l+1 is visited floor((j+1) gamma) - floor(j gamma) times. With the cycle
    # indices below on a hierarchy of kinds e a a a e a a c the counts, derived by hand, are:
    #   L1 (gamma 2):    j=0 -> 2                                  L2: 2 visits
    #   L2 (gamma 1.5):  j=0,1 -> 1, 2                             L3: 3 visits
    #   L3 (gamma 1.5):  j=0,1,2 -> 1, 2, 1                        L4: 4 visits, L5 (after e): 4
    #   L5 (gamma 1.7):  j=0..3 -> 1, 2, 2, 1                      L6: 6 visits
    #   L6 (gamma 1.25): j=0..5 -> 1, 1, 1, 2, 1, 1                L7: 7 visits
    g = gg.grid3d(16, 16, 16, "loguniform", seed=1)
    H = oracle.Hierarchy(g, coarsest_max=16)
    kinds = [L["kind"][0] for L in H.levels]
    assert kinds == list("eaaaeaac")
    for l, gam in [(1, 2.0), (2, 1.5), (3, 1.5), (5, 1.7), (6, 1.25)]:
        H.set_gamma(l, gam)
    H.cycle(gg.rhs(g, 2))
    assert H.visit_counts() == [1, 1, 2, 3, 4, 4, 6, 7]
    # a fresh cycle restarts the counters
    H.cycle(gg.rhs(g, 3))
    assert H.visit_counts() == [1, 1, 2, 3, 4, 4, 6, 7]


@pytest.mark.parametrize("kappa", [1, 3])
def test_recombination_is_least_squares_over_saved_iterates(kappa):
    # Section 2: after each cycle, alpha = argmin || r - A E alpha ||, E = [x_j - x] over the
    # saved iterates, x <- x + E alpha; checked with numpy's least-squares solver on every cycle.
    g = gg.grid2d(24, 20, 1.0, 1e-2)
    H = oracle.Hierarchy(g, coarsest_max=16)
    b = gg.rhs(g, 2)
    out = H.stationary(b, 1e-12, 12, kappa=kappa, record=True)
    A = oracle.laplacian(g).dense()
    bb = b - b.mean()
    saved = []
    nrec = 0
    for i in range(out["iters"]):
        pre, got = out["pre"][i], out["saved"][i]
        if saved:
            E = np.stack([s - pre for s in saved], axis=1)
            alpha, *_ = np.linalg.lstsq(A @ E, bb - A @ pre, rcond=None)
            want = pre + E @ alpha
            assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want), (i, kappa)
            nrec += 1
        else:
            assert np.array_equal(got, pre)
        saved.append(got)
        saved = saved[-kappa:]
    assert nrec >= 5
