"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks an oracle routine against something other than itself: a published value,
a closed form, a dense linear-algebra definition computed with numpy/scipy, brute force on a
tiny input, or an invariant the paper states. The oracle is then trusted as the reference
for the CUDA path.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as sopt

import graphgen as gg
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dense_L(g):
    M = np.zeros((g.n, g.n))
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    M[rows, g.ci] = -g.w
    M[np.arange(g.n), np.arange(g.n)] = -M.sum(axis=1)
    return M


# ----------------------------------------------------------------------------- random stream

def test_splitmix64_published_values():
    rows = [l.split() for l in open(os.path.join(GOLD, "splitmix64.txt")) if l.strip() and not l.startswith("#")]
    assert rows
    for seed, i, val in rows:
        assert oracle.splitmix64(int(seed), int(i)) == int(val)


def test_random_start_range_and_mapping():
    # U[-1, 1) from the top 53 bits of SplitMix64 output 1 + ((level << 44) | (u << 4) | k)
    for (lvl, u, k) in [(0, 0, 0), (3, 12345, 2), (7, 10**9, 3), (2, 777, 15)]:
        z = oracle.splitmix64(3, 1 + ((lvl << 44) | (u << 4) | k))
        expect = 2.0 * ((z >> 11) / 2.0**53) - 1.0
        v = oracle.random_start(3, lvl, u, k)
        assert v == expect and -1.0 <= v < 1.0
    vals = np.array([oracle.random_start(3, 0, u, 0) for u in range(4000)])
    assert abs(vals.mean()) < 0.05 and abs(vals.var() - 1 / 3) < 0.03


# ----------------------------------------------------------------------------- Laplacian, GS

def test_laplacian_definition():
    g = gg.random_connected(60, 90, seed=4)
    A = oracle.laplacian(g)
    D = A.dense()
    assert np.allclose(D, dense_L(g))
    assert np.abs(D @ np.ones(g.n)).max() < 1e-13          # L 1 = 0
    x = np.random.default_rng(0).standard_normal(g.n)
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    energy = 0.5 * np.sum(g.w * (x[rows] - x[g.ci]) ** 2)  # sum over edges w (x_u - x_v)^2
    assert math.isclose(x @ D @ x, energy, rel_tol=1e-12)


def test_colouring_is_greedy_and_proper():
    g = gg.random_connected(80, 200, seed=5)
    A = oracle.laplacian(g)
    col, nc = oracle.colour(A)
    for u in range(g.n):
        nb = g.ci[g.rp[u]:g.rp[u + 1]]
        assert np.all(col[nb] != col[u])
        lower = set(col[nb[nb < u]].tolist())
        c = 0
        while c in lower:
            c += 1
        assert col[u] == c
    assert nc == col.max() + 1


@pytest.mark.parametrize("order", ["forward", "reverse", "lex"])
def test_gauss_seidel_matches_matrix_splitting(order):
    # A GS sweep in row order pi solves (D + L_pi) x_new = b - U_pi x_old, where L_pi / U_pi
    # are the parts of A coupling a row to rows earlier / later in pi (textbook splitting).
    g = gg.random_connected(40, 70, seed=6)
    A = oracle.laplacian(g)
    M = A.dense()
    col, nc = oracle.colour(A)
    if order == "lex":
        pi = np.arange(g.n)
    else:
        cs = range(nc) if order == "forward" else range(nc - 1, -1, -1)
        pi = np.concatenate([np.flatnonzero(col == c) for c in cs])
    P = M[np.ix_(pi, pi)]
    rng = np.random.default_rng(1)
    x0 = rng.standard_normal(g.n); b = rng.standard_normal(g.n)
    x1 = sla.solve_triangular(np.tril(P), b[pi] - np.triu(P, 1) @ x0[pi], lower=True)
    got = oracle.gs(A, x0, b, order=order)
    assert np.allclose(got[pi], x1, rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------- affinity, guard

def test_affinity_invariants():
    rng = np.random.default_rng(2)
    for _ in range(50):
        xu, xv = rng.standard_normal(4), rng.standard_normal(4)
        c = oracle.affinity(xu, xv)
        assert 0.0 <= c <= 1.0 + 1e-15
        assert math.isclose(c, oracle.affinity(xv, xu), rel_tol=1e-14)          # symmetric
        a, b = rng.uniform(-3, 3, 2)
        assert math.isclose(c, oracle.affinity(a * xu, b * xv), rel_tol=1e-12)  # scale-free
        # squared cosine of the angle between the two profiles
        ang = math.acos(np.clip(xu @ xv / np.linalg.norm(xu) / np.linalg.norm(xv), -1, 1))
        assert math.isclose(c, math.cos(ang) ** 2, rel_tol=1e-9, abs_tol=1e-12)
    assert oracle.affinity([1, 2, 3, 4], [-2, -4, -6, -8]) == pytest.approx(1.0, abs=1e-15)
    assert oracle.affinity([1, 0, 0, 0], [0, 1, 0, 0]) == 0.0


def brute_guard(w, xnb, xs):
    """q of Eq. 4 evaluated directly: per test vector, E(y) = 1/2 sum_v w_v (y - x_v)^2,
    forced = E(x_s), relaxed = min_y E(y) found numerically."""
    q = 0.0
    for k in range(xnb.shape[1]):
        E = lambda y: 0.5 * np.sum(w * (y - xnb[:, k]) ** 2)
        res = sopt.minimize_scalar(E, bracket=(xnb[:, k].min() - 1, xnb[:, k].max() + 1), tol=1e-14)
        q = max(q, E(xs[k]) / res.fun)
    return q


def test_guard_moments_match_direct_energy():
    rng = np.random.default_rng(3)
    for deg in [2, 3, 5, 9]:
        w = rng.uniform(0.5, 1.5, deg)
        xnb = rng.standard_normal((deg, 4))
        xs = xnb[0]                     # candidate seed: the first neighbour
        s0 = w.sum(); s1 = w @ xnb; s2 = w @ xnb ** 2
        q = oracle.guard_q(s0, s1, s2, xs)
        assert q >= 1.0
        assert math.isclose(q, brute_guard(w, xnb, xs), rel_tol=1e-6)


def test_guard_single_neighbour_reading():
    # one neighbour: relaxed energy is zero; forcing onto it costs nothing (ratio 1)
    x = np.array([0.3, -0.7, 0.2, 0.9])
    assert oracle.guard_q(2.0, 2.0 * x, 2.0 * x ** 2, x) == 1.0
    assert math.isinf(oracle.guard_q(2.0, 2.0 * x, 2.0 * x ** 2, x + 0.5))


# ----------------------------------------------------------------------------- elimination

def test_elimination_is_dense_schur_complement():
    for seed in range(5):
        g = gg.random_connected(50, 30, seed=10 + seed)
        A = oracle.laplacian(g)
        inF, nf, Ac = oracle.eliminate(A, 4)
        deg = np.diff(g.rp)
        assert nf == inF.sum() > 0
        # F is independent, low degree, and maximal among the low-degree nodes
        for u in np.flatnonzero(inF):
            assert deg[u] <= 4 and not inF[g.ci[g.rp[u]:g.rp[u + 1]]].any()
        for u in np.flatnonzero(~inF & (deg <= 4)):
            assert inF[g.ci[g.rp[u]:g.rp[u + 1]]].any()
        M = A.dense(); F = np.flatnonzero(inF); Cn = np.flatnonzero(~inF)
        S = M[np.ix_(Cn, Cn)] - M[np.ix_(Cn, F)] @ np.linalg.solve(M[np.ix_(F, F)], M[np.ix_(F, Cn)])
        assert np.allclose(Ac.dense(), S, rtol=1e-13, atol=1e-13)


# ----------------------------------------------------------------------------- Galerkin, pinv

def test_galerkin_matches_dense_triple_product():
    rng = np.random.default_rng(7)
    g = gg.random_connected(70, 120, seed=8)
    A = oracle.laplacian(g)
    nc = 20
    agg = np.concatenate([np.arange(nc), rng.integers(0, nc, g.n - nc)]).astype(np.int32)
    agg2 = np.where(rng.random(g.n) < 0.4, rng.integers(0, nc, g.n), -1).astype(np.int32)
    agg2[agg2 == agg] = -1
    wt = np.where(agg2 >= 0, rng.uniform(0, 1, g.n), 1.0)
    wt[np.flatnonzero(agg2 >= 0)[:3]] = 0.0   # rows snapped to w = 0
    P = np.zeros((g.n, nc))
    P[np.arange(g.n), agg] += wt
    m = agg2 >= 0
    P[np.flatnonzero(m), agg2[m]] += 1 - wt[m]
    Ac = oracle.galerkin(A, nc, agg, agg2, wt)
    ref = P.T @ A.dense() @ P
    assert np.allclose(Ac.dense(), ref, rtol=1e-13, atol=1e-13)
    assert np.allclose(ref @ np.ones(nc), 0, atol=1e-12)


def test_pinv_matches_numpy():
    g = gg.random_connected(90, 150, seed=9)
    A = oracle.laplacian(g)
    assert np.allclose(oracle.pinv(A), np.linalg.pinv(A.dense(), rcond=1e-10, hermitian=True), rtol=1e-10, atol=1e-12)


# ----------------------------------------------------------------------------- hierarchy

GRAPHS = [
    lambda: gg.grid2d(40, 40),
    lambda: gg.grid2d(40, 40, 1.0, 1e-3),
    lambda: gg.grid3d(10, 10, 10, "loguniform", seed=1),
    lambda: gg.random_connected(1500, 3000, seed=11),
    lambda: gg.barabasi_albert(1200, 4, seed=2),
]


@pytest.mark.parametrize("make", GRAPHS)
def test_hierarchy_invariants(make):
    g = make()
    H = oracle.Hierarchy(g, coarsest_max=40)
    lv = H.levels
    assert lv[-1]["kind"] == "coarsest" and all(l["kind"] != "coarsest" for l in lv[:-1])
    for l, L in enumerate(lv):
        M = L["A"].dense() if L["n"] <= 2500 else None
        if M is not None:
            assert np.allclose(M, M.T, atol=1e-13 * np.abs(M).max())
            assert np.abs(M.sum(axis=1)).max() <= 1e-12 * np.abs(M).max()
            assert np.linalg.eigvalsh(M).min() > -1e-10 * np.abs(M).max()
        if L["kind"] == "agg":
            wt, agg2 = L["wt"], L["agg2"]
            assert np.all((wt >= 0) & (wt <= 1))
            assert np.all(wt[agg2 < 0] == 1.0)
            # colour classes are independent
            rows = np.repeat(np.arange(L["n"]), np.diff(L["rp"]))
            assert np.all(L["colour"][rows] != L["colour"][L["ci"]])
            assert np.all((L["aff"] >= 0) & (L["aff"] <= 1 + 1e-15))
            # next level is P^T A P (dense check)
            if M is not None:
                P = np.zeros((L["n"], L["nc"]))
                P[np.arange(L["n"]), L["agg"]] += wt
                m = agg2 >= 0
                P[np.flatnonzero(m), agg2[m]] += 1 - wt[m]
                assert np.allclose(P.sum(axis=1), 1.0)               # P 1 = 1
                nxt = lv[l + 1]["A"].dense()
                assert np.allclose(nxt, P.T @ M @ P, rtol=1e-12, atol=1e-12 * np.abs(M).max())
        if L["kind"] == "coarsest":
            assert np.allclose(L["pinv"], np.linalg.pinv(L["A"].dense(), rcond=1e-10, hermitian=True), atol=1e-9 * np.abs(L["pinv"]).max())


def test_caliber2_weight_is_least_squares():
    # Eq. 13 against a least-squares fit of x_u - x_b on x_a - x_b over the test vectors
    g = gg.grid2d(48, 48, 1.0, 1e-3)
    H = oracle.Hierarchy(g, coarsest_max=40)
    L = next(l for l in H.levels if l["kind"] == "agg")
    X, seed_of = L["X"], L["seed_of"]
    up = np.flatnonzero((L["agg2"] >= 0) & (L["wt"] > 0.01) & (L["wt"] < 0.99))
    assert len(up) > 50
    seeds_of_agg = {}
    for u in range(L["n"]):
        seeds_of_agg[L["agg"][u]] = seed_of[u]
    for u in up[:200]:
        xa = X[seeds_of_agg[L["agg"][u]]]; xb = X[seeds_of_agg[L["agg2"][u]]]
        w, *_ = np.linalg.lstsq((xa - xb)[:, None], X[u] - xb, rcond=None)
        assert math.isclose(L["wt"][u], w[0], rel_tol=1e-9, abs_tol=1e-12)


def test_caliber2_gate_is_self_targeting():
    # Section 3.2: ~0% of nodes upgrade on an isotropic grid, nearly every locally 1-D
    # (anisotropic) non-seed node upgrades.
    iso = oracle.Hierarchy(gg.grid2d(64, 64), coarsest_max=40)
    an = oracle.Hierarchy(gg.grid2d(64, 64, 1.0, 1e-3), coarsest_max=40)
    Li = next(l for l in iso.levels if l["kind"] == "agg")
    La = next(l for l in an.levels if l["kind"] == "agg")
    assert Li["n_caliber2"] / Li["n"] < 0.03
    assoc = np.sum(La["seed_of"] != np.arange(La["n"]))
    assert La["n_caliber2"] / assoc > 0.9


def test_veto_is_inert_on_uniform_weights():
    g = gg.grid2d(32, 32)
    H = oracle.Hierarchy(g, coarsest_max=40)
    for L in H.levels:
        if L["kind"] == "agg" and L is H.levels[1]:
            assert L["strong"].all()


# ----------------------------------------------------------------------------- solves

def test_solution_matches_dense_pseudoinverse():
    for seed in range(50):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(5, 200))
        g = gg.random_connected(n, int(rng.integers(0, 3 * n)), seed=100 + seed)
        b = gg.rhs(g, seed=seed)
        H = oracle.Hierarchy(g, coarsest_max=8)
        out = H.fcg(b, tol=1e-14, maxit=300)
        ref = np.linalg.pinv(dense_L(g), rcond=1e-10, hermitian=True) @ (b - b.mean())
        assert np.linalg.norm(out["x"] - ref) <= 1e-10 * np.linalg.norm(ref), (seed, out["iters"])


def test_path_graph_closed_form_one_cycle():
    # Path 0-1-...-(n-1) with weights w_i on edge (i, i+1): the flux through edge i is
    # f_i = sum_{j<=i} b_j and phi_{i+1} - phi_i = -f_i / w_i; then remove the mean.
    n = 700
    rng = np.random.default_rng(4)
    w = rng.uniform(0.5, 1.5, n - 1)
    g = gg.path(n, w)
    b = rng.standard_normal(n); b -= b.mean()
    f = np.cumsum(b)[:-1]
    phi = np.concatenate([[0.0], np.cumsum(-f / w)])
    phi -= phi.mean()
    H = oracle.Hierarchy(g, coarsest_max=4)
    assert all(l["kind"] != "agg" for l in H.levels)       # a path is eliminated completely
    z = H.cycle(b)
    assert np.linalg.norm(z - phi) <= 1e-11 * np.linalg.norm(phi)


def test_cycle_graph_closed_form():
    # Cycle graph: edge fluxes f_i = f_0 + sum_{1<=j<=i} b_j (edge i joins i and i+1 mod n),
    # potential drops f_i / w_i must sum to zero around the loop, which fixes f_0.
    n = 500
    rng = np.random.default_rng(5)
    w = rng.uniform(0.5, 1.5, n)
    g = gg.cycle(n, w)
    b = rng.standard_normal(n); b -= b.mean()
    c = np.concatenate([[0.0], np.cumsum(b[1:])])
    f0 = -np.sum(c / w) / np.sum(1.0 / w)
    f = f0 + c
    phi = np.concatenate([[0.0], np.cumsum(-f[:-1] / w[:-1])])
    phi -= phi.mean()
    H = oracle.Hierarchy(g, coarsest_max=4)
    out = H.fcg(b, tol=1e-13, maxit=50)
    assert out["iters"] <= 2
    assert np.linalg.norm(out["x"] - phi) <= 1e-10 * np.linalg.norm(phi)


def test_star_graph_leaves_eliminated():
    g = gg.star(300, np.random.default_rng(6).uniform(0.5, 1.5, 299))
    H = oracle.Hierarchy(g, coarsest_max=1)
    L0 = H.levels[0]
    assert L0["kind"] == "elim" and H.levels[1]["n"] == 1
    b = gg.rhs(g, 3)
    out = H.fcg(b, tol=1e-13, maxit=5)
    assert out["iters"] == 1
    ref = np.linalg.pinv(dense_L(g), rcond=1e-10, hermitian=True) @ b
    assert np.linalg.norm(out["x"] - ref) <= 1e-12 * np.linalg.norm(ref)


def test_dense_level_becomes_the_coarsest():
    # a level with at most dense_rows nodes and >= n^2/8 off-diagonal entries is solved
    # directly: a dense random graph (density ~0.3) stops at level 0 and one preconditioned
    # step is the exact pseudo-inverse solution; with the rule off it is coarsened further
    rng = np.random.default_rng(11)
    n = 400
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < 0.3
    g = gg.largest_cc(gg.from_edges(n, iu[0][keep], iu[1][keep], rng.uniform(0.5, 1.5, keep.sum())))
    assert 2 * g.m >= g.n * g.n / 8
    H = oracle.Hierarchy(g, coarsest_max=16)
    assert H.nlevels == 1 and H.levels[0]["kind"] == "coarsest"
    b = gg.rhs(g, 4)
    out = H.fcg(b, tol=1e-13, maxit=5)
    ref = np.linalg.pinv(dense_L(g), rcond=1e-10, hermitian=True) @ b
    assert out["iters"] == 1
    assert np.linalg.norm(out["x"] - ref) <= 1e-11 * np.linalg.norm(ref)
    off = oracle.Hierarchy(g, coarsest_max=16, dense_rows=0)
    assert off.nlevels > 1
    # a size bound below n switches the rule off for this level
    assert oracle.Hierarchy(g, coarsest_max=16, dense_rows=g.n - 1).nlevels > 1


def _laplacian_matrix(g):
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    return oracle.Matrix(g.rp, g.ci, -g.w, np.bincount(rows, weights=g.w, minlength=g.n))


@pytest.mark.parametrize("m", [1, 2, 3, 5])
def test_chebyshev_smoother_is_the_chebyshev_error_polynomial(m):
    # one application maps the error e = x* - x to C_m((theta I - D^-1 A)/delta) e / C_m(sigma),
    # C_m the Chebyshev polynomial of the first kind, on [lambda/30, lambda]: evaluated here
    # densely from that definition, with a signed coarse-like operator (a positive entry)
    rng = np.random.default_rng(m)
    g = gg.random_connected(40, 60, seed=m)
    A = _laplacian_matrix(g)
    val = A.val.copy()
    val[0] = abs(val[0]) * 0.3                      # one positive off-diagonal (signed coarse weights)
    j = np.where((np.repeat(np.arange(g.n), np.diff(g.rp)) == g.ci[0]) & (g.ci == 0))[0][0]
    val[j] = val[0]                                 # keep it symmetric
    A = oracle.Matrix(A.rp, A.ci, val, A.diag)
    M = A.dense()
    xs = rng.standard_normal(g.n)
    b = M @ xs
    x0 = rng.standard_normal(g.n)
    x1, lam = oracle.cheb_apply(A, x0, b, m)
    D = np.diag(M)
    assert lam == pytest.approx(max(1 + np.abs(M[i] - np.diag(D)[i]).sum() / D[i] for i in range(g.n)), rel=1e-15)
    hi, lo = lam, lam / 30
    th, de = (hi + lo) / 2, (hi - lo) / 2
    Y = (th * np.eye(g.n) - M / D[:, None]) / de
    C0, C1 = np.eye(g.n), Y
    c0, c1 = 1.0, th / de
    for _ in range(m - 1):
        C0, C1 = C1, 2 * Y @ C1 - C0
        c0, c1 = c1, 2 * (th / de) * c1 - c0
    e1 = (C1 / c1) @ (xs - x0)
    assert np.linalg.norm((xs - x1) - e1) <= 1e-11 * np.linalg.norm(xs - x0)


def test_chebyshev_bound_is_two_on_a_laplacian_and_the_solver_still_solves():
    g = gg.grid2d(24, 20, 1.0, 0.05)
    _, lam = oracle.cheb_apply(_laplacian_matrix(g), np.zeros(g.n), np.zeros(g.n), 2)
    assert lam == pytest.approx(2.0, abs=1e-14)
    # every aggregation level smoothed by the polynomial (colour threshold 1)
    H = oracle.Hierarchy(g, coarsest_max=16, cheb_colours=1)
    assert all(L["cheb"] for L in H.levels if L["kind"] == "agg")
    b = gg.rhs(g, 3)
    out = H.fcg(b, tol=1e-10, maxit=100)
    ref = np.linalg.pinv(dense_L(g), rcond=1e-10, hermitian=True) @ (b - b.mean())
    assert np.linalg.norm(out["x"] - ref) <= 1e-8 * np.linalg.norm(ref)
    # and the default keeps Gauss-Seidel on levels with few colours
    assert not any(L["cheb"] for L in oracle.Hierarchy(g, coarsest_max=16).levels)


@pytest.mark.parametrize("gamma", [1.0, 2.0])
def test_symmetric_cycle_is_symmetric(gamma):
    # With nu_pre = nu_post, forward pre- and reverse post-smoothing, P^T restriction and exact
    # coarsest/elimination solves, the cycle M is a symmetric operator: <M u, v> = <u, M v>.
    g = gg.grid2d(30, 30, 1.0, 0.1)
    H = oracle.Hierarchy(g, coarsest_max=20, nu_pre=1, nu_post=1, gamma_fixed=gamma)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(g.n); v = rng.standard_normal(g.n)
    u -= u.mean(); v -= v.mean()
    a, b = H.cycle(u) @ v, u @ H.cycle(v)
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))


def test_refinements_improve_anisotropic_convergence():
    # Section 3: the veto and caliber-2 turn the anisotropic-grid stall into fast convergence.
    g = gg.grid2d(128, 128, 1.0, 1e-4)
    b = gg.rhs(g, 2)
    both = oracle.Hierarchy(g, coarsest_max=64).stationary(b, 1e-8, 60, kappa=4)
    none = oracle.Hierarchy(g, coarsest_max=64, veto=0, caliber2=0).stationary(b, 1e-8, 60, kappa=4)
    assert oracle.acf(both["hist"]) < 0.5 * oracle.acf(none["hist"])
    assert both["iters"] < none["iters"]


def test_fcg_converges_on_workload_shapes():
    for g in [gg.grid2d(64, 64), gg.grid2d(96, 96, 1.0, 1e-3), gg.grid3d(16, 16, 16, "loguniform", seed=1)]:
        b = gg.rhs(g, 2)
        out = oracle.Hierarchy(g, coarsest_max=64).fcg(b, 1e-8, 60)
        assert out["hist"][-1] <= 1e-8 and out["iters"] <= 30, (g.name, out["iters"])
        r = gg.laplacian_apply(g, out["x"]) - (b - b.mean())
        assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(b - b.mean())


def test_coarsest_size_rule():
    # default coarsest size: floor(sqrt(1.5 nnz(L))) within [1024, 4096], nnz(L) = n + 2m; on a
    # 420^2 anisotropic grid that is 1149, so its 1094-node level is the coarsest, where a fixed
    # 1024 coarsens once more; an explicit coarsest_max still decides
    g = gg.grid2d(420, 420, 1.0, 1e-3)
    nnz_l = g.n + int(g.rp[-1])
    cmax = min(4096, max(1024, math.floor(math.sqrt(1.5 * nnz_l))))
    assert cmax == 1149
    H = oracle.Hierarchy(g)
    sizes = [L["n"] for L in H.levels]
    assert H.levels[-1]["kind"] == "coarsest"
    assert 1024 < sizes[-1] <= cmax and sizes[-2] > cmax
    H2 = oracle.Hierarchy(g, coarsest_max=1024)
    sizes2 = [L["n"] for L in H2.levels]
    assert sizes2[-1] <= 1024 and len(sizes2) > len(sizes)
    assert sizes2[:len(sizes) - 1] == sizes[:-1]
