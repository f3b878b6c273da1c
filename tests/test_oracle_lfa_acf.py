"""Closed-form and printed-behaviour pins of the oracle (no GPU).

1. The two-grid local Fourier analysis of Appendix A.1 (oracle/lfa.py): its trace formula
   against the explicitly assembled 2 x 2 symbol, against the explicit dense two-grid operator
   on a periodic grid, the closed forms of the energy fractions, the caliber-1 ceiling, and the
   printed suprema (caliber-1 about 0.48, caliber-2 0.08 / 0.09 / 0.09).
2. Convergence factors the paper prints for its anisotropic grids (Table 2, Table 10, Section 3
   and the grid128 row of the ACF table, Table 3), compared in bands of +-35% (random test vectors, and
   readings where the paper is silent). Cases whose band the oracle misses are marked xfail
   with the reading responsible; strict, so that a change that brings one into its band shows.
3. The measured two-level factors of Section 3.2 (exact coarse solve, per aggregation level)
   and the self-targeting of the caliber-2 gate (Table 2).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import graphgen as gg
import oracle
from oracle import lfa


def band(paper, value, rel=0.35):
    return paper * (1 - rel) <= value <= paper * (1 + rel)


# ----------------------------------------------------------------------------- LFA

def test_lfa_trace_formula_equals_the_two_by_two_symbol():
    # Eq. (rhotrace) against the spectral radius of Eq. (tgsymbol) assembled explicitly
    rng = np.random.default_rng(0)
    for _ in range(200):
        tx = rng.uniform(-np.pi / 2, np.pi / 2)
        ty = rng.uniform(-np.pi, np.pi)
        eps = 10 ** rng.uniform(-4, 0)
        for cal in (1, 2):
            a = float(lfa.rho_trace(tx, ty, eps, cal))
            b = lfa.rho_matrix(tx, ty, eps, cal)
            assert abs(a - b) <= 1e-12 + 1e-10 * b, (tx, ty, eps, cal)


def _periodic_laplacian(N, eps):
    n = N * N
    M = np.zeros((n, n))
    for y in range(N):
        for x in range(N):
            u = x + N * y
            for dx, dy, w in ((1, 0, 1.0), (-1, 0, 1.0), (0, 1, eps), (0, -1, eps)):
                v = (x + dx) % N + N * ((y + dy) % N)
                M[u, v] -= w
                M[u, u] += w
    return M


def _periodic_two_grid(N, eps, caliber, nu=3):
    """Spectral radius (on mean-zero vectors) of the dense two-grid operator
    S^nu (I - P (P^T L P)^+ P^T L) on the periodic N x N grid, 2:1 coarsening in x: caliber-1
    P = pairs {2i, 2i+1} piecewise constant, caliber-2 P = linear interpolation between the
    even points; S = I - M^{-1} L with M the Gauss-Seidel part (diagonal, west and south
    neighbours), circulant on the periodic grid."""
    n, nc = N * N, (N // 2) * N
    L = _periodic_laplacian(N, eps)
    P = np.zeros((n, nc))
    M = np.zeros((n, n))
    for y in range(N):
        for x in range(N):
            u, i = x + N * y, x // 2
            if caliber == 1 or x % 2 == 0:
                P[u, i + (N // 2) * y] = 1.0
            else:
                P[u, i + (N // 2) * y] = 0.5
                P[u, (i + 1) % (N // 2) + (N // 2) * y] = 0.5
            M[u, u] = 2 + 2 * eps
            M[u, (x - 1) % N + N * y] -= 1.0
            M[u, x + N * ((y - 1) % N)] -= eps
    S = np.eye(n) - np.linalg.solve(M, L)
    T = np.linalg.matrix_power(S, nu) @ (np.eye(n) - P @ np.linalg.pinv(P.T @ L @ P) @ P.T @ L)
    Q = np.eye(n) - 1.0 / n
    return float(np.max(np.abs(np.linalg.eigvals(Q @ T @ Q))))


@pytest.mark.parametrize("eps", [1e-1, 1e-2])
@pytest.mark.parametrize("caliber", [1, 2])
def test_lfa_matches_the_explicit_periodic_two_grid_operator(eps, caliber):
    # The symbols (Eq. Lsymbol, the Gauss-Seidel symbol, Eq. Psymbols) describe the operator
    # exactly on the periodic grid's own frequencies theta = 2 pi (k, l) / N.
    N = 16
    best = 0.0
    for k in range(-N // 4 + 1, N // 4 + 1):
        for l in range(-N // 2 + 1, N // 2 + 1):
            if (k, l) != (0, 0):
                best = max(best, float(lfa.rho_trace(2 * np.pi * k / N, 2 * np.pi * l / N, eps, caliber)))
    assert abs(_periodic_two_grid(N, eps, caliber) - best) <= 2e-3 * best


def test_lfa_energy_fractions_closed_forms():
    # Eq. (betas): eps -> 0 gives beta_c1 = 1/2 for every theta_x and beta_c2 = c = cos^2(theta_x/2)
    for tx in (1e-3, 0.3, 0.9, 1.4):
        assert lfa.beta(tx, 0.8, 1e-15, 1) == pytest.approx(0.5, abs=1e-9)
        assert lfa.beta(tx, 0.8, 1e-15, 2) == pytest.approx(np.cos(tx / 2) ** 2, abs=1e-9)


def test_lfa_caliber1_ceiling():
    # Eq. (c1ceiling): on modes smooth in x, S(theta) -> 1 and beta_c1 = 1/2. The paper takes the
    # x-harmonic as fully smoothed (S(theta*) -> 0, rho -> 1/2); exactly, at theta* = (pi, .) with
    # eps -> 0 the Gauss-Seidel symbol is 1 - 4/3 = -1/3, so rho -> (1 + (-1/3)^3) / 2 = 13/27,
    # the 0.48 the paper prints. Caliber-2 (beta -> 1) leaves only the smoothed harmonic.
    for ty in (0.5, 1.5, 3.0):
        assert complex(lfa.s_symbol(np.pi, ty, 1e-14)) == pytest.approx(-1 / 3, abs=1e-9)
        assert float(lfa.rho_trace(1e-6, ty, 1e-24, 1)) == pytest.approx(13 / 27, abs=1e-5)
        assert float(lfa.rho_trace(1e-6, ty, 1e-24, 2)) == pytest.approx(1 / 27, abs=1e-5)
    assert 0.5 - 13 / 27 < 0.02


def test_lfa_printed_suprema():
    # Appendix A.1 and Table 10: sup rho_c1 about 0.48 (the 1/2 ceiling), sup rho_c2 0.08 / 0.09 /
    # 0.09 at eps = 1e-1 / 1e-2 / 1e-4
    for eps in (1e-1, 1e-2, 1e-4):
        assert 0.47 <= lfa.sup_rho(eps, 1) <= 0.50
    for eps, paper in ((1e-1, 0.08), (1e-2, 0.09), (1e-4, 0.09)):
        v = lfa.sup_rho(eps, 2)
        assert 0.07 <= v <= 0.10 and abs(v - paper) <= 0.01, (eps, v)


# ----------------------------------------------------------------------------- printed ACFs

def stationary_acf(g, kappa, **opts):
    """Median ACF of the stationary solver over five test-vector seeds (the factor depends on
    the random sample, Section 3.1)."""
    b = gg.rhs(g, 2)
    acfs = [oracle.acf(oracle.Hierarchy(g, coarsest_max=16, seed=s, **opts).stationary(b, 1e-8, 300, kappa=kappa)["hist"])
            for s in range(3, 8)]
    return float(np.median(acfs))


READING_ML = ("the oracle's cycle is the gamma-cycle of Eq. 5 with per-cycle visit counts "
              "floor((j+1) gamma) - floor(j gamma) and recombination on the finest level only; the "
              "paper's near-textbook factors on isotropic and mildly anisotropic grids need cycle "
              "details it does not state (measured: 0.39-0.52 here, against the MATLAB LAMG "
              "reference's 0.21 on grid128)")


@pytest.mark.parametrize("eps,paper", [(1.0, 0.74), (1e-1, 0.76), (1e-2, 0.77), (1e-4, 0.77)])
def test_flat_vcycle_caliber1_factor(eps, paper):
    # Table 10, caliber-1 "V-cycle": gamma = 1, (1,2) sweeps, no recombination, no caliber-2
    v = stationary_acf(gg.grid2d(64, 64, 1.0, eps), 0, caliber2=0, gamma_fixed=1.0)
    assert band(paper, v), v


@pytest.mark.parametrize("eps,paper", [
    pytest.param(1.0, 0.010, marks=pytest.mark.xfail(strict=True, reason=READING_ML)),
    pytest.param(1e-1, 0.274, marks=pytest.mark.xfail(strict=True, reason=READING_ML)),
    (1e-2, 0.335),
    (1e-4, 0.391),
])
def test_multilevel_caliber1_factor(eps, paper):
    # Table 10, caliber-1 "ML": gamma of Eq. 5 and recombination
    v = stationary_acf(gg.grid2d(64, 64, 1.0, eps), 4, caliber2=0)
    assert band(paper, v), v


@pytest.mark.parametrize("eps,paper", [
    pytest.param(1.0, 0.008, marks=pytest.mark.xfail(strict=True, reason=READING_ML)),
    pytest.param(1e-1, 0.007, marks=pytest.mark.xfail(strict=True, reason=READING_ML)),
    pytest.param(1e-2, 0.051, marks=pytest.mark.xfail(strict=True, reason=READING_ML)),
    pytest.param(1e-4, 0.100, marks=pytest.mark.xfail(
        strict=False, reason="at the band's upper edge: the median of the five seeds is 0.134-0.135 "
                             "(single seeds 0.126-0.144) against the printed 0.100")),
])
def test_multilevel_caliber2_factor(eps, paper):
    # Table 10, caliber-2 "ML": the full LAMG+ solver
    v = stationary_acf(gg.grid2d(64, 64, 1.0, eps), 4)
    assert band(paper, v), v


@pytest.mark.xfail(strict=True, reason=READING_ML)
def test_grid128_factor():
    # ACF table, grid128: 0.022 in 5 cycles
    assert band(0.022, stationary_acf(gg.grid2d(128, 128), 4))


@pytest.mark.parametrize("N,paper", [
    (256, 0.16),
    pytest.param(384, 0.11, marks=pytest.mark.xfail(strict=True, reason=READING_ML + "; 0.20 measured")),
])
def test_large_anisotropic_grid_with_both_refinements(N, paper):
    # Table 2 (and Section 3.1): eps = 1e-4, veto and caliber-2 on
    v = stationary_acf(gg.grid2d(N, N, 1.0, 1e-4), 4)
    assert band(paper, v), v


@pytest.mark.xfail(strict=True, reason=READING_ML + "; 17 and 18 cycles measured")
@pytest.mark.parametrize("make,paper_cycles", [(lambda: gg.grid2d(256, 256), 5),
                                               (lambda: gg.grid3d(40, 40, 40, "unit"), 9)])
def test_isotropic_grid_cycle_counts(make, paper_cycles):
    # Table 8, uniform 2D grid of 65,536 nodes (5 cycles) and 3D grid of 64,000 nodes (9 cycles)
    g = make()
    out = oracle.Hierarchy(g).stationary(gg.rhs(g, 2), 1e-8, 300, kappa=4)
    assert band(paper_cycles, out["iters"]), out["iters"]


def test_refinements_turn_the_caliber1_rate_into_the_caliber2_rate():
    # Table 2: on the 256^2, eps = 1e-4 grid caliber-1 converges much more slowly than the
    # default (0.56 against 0.16 printed)
    g = gg.grid2d(256, 256, 1.0, 1e-4)
    c1 = stationary_acf(g, 4, caliber2=0)
    c2 = stationary_acf(g, 4)
    assert band(0.56, c1) and c2 < 0.4 * c1, (c1, c2)


# ----------------------------------------------------------------------------- two-level factors

def _level_csr(L):
    n = L["n"]
    rows = np.repeat(np.arange(n), np.diff(L["rp"]))
    return sp.csr_matrix((np.concatenate([L["val"], L["diag"]]),
                          (np.concatenate([rows, np.arange(n)]), np.concatenate([L["ci"], np.arange(n)]))),
                         shape=(n, n))


def two_level_factor(L, its=40):
    """Asymptotic energy-norm factor of one aggregation level with an exact coarse solve
    (sparse LU of P^T A P with one coarse node grounded, then the mean-zero projection) and the
    paper's lexicographic Gauss-Seidel, one sweep before and two after: power iteration on the
    error propagation from a seeded random start."""
    A = _level_csr(L)
    n, nc = L["n"], L["nc"]
    P = sp.csr_matrix((L["wt"], (np.arange(n), L["agg"])), shape=(n, nc))
    m = L["agg2"] >= 0
    P = P + sp.csr_matrix((1 - L["wt"][m], (np.flatnonzero(m), L["agg2"][m])), shape=(n, nc))
    Ac = (P.T @ A @ P).tocsc()
    lu = spla.splu(Ac[1:, 1:].tocsc())
    Am = oracle.Matrix(L["rp"], L["ci"], L["val"], L["diag"])
    e = np.random.default_rng(0).standard_normal(n)
    e -= e.mean()
    z = np.zeros(n)
    rates = []
    for _ in range(its):
        e /= np.sqrt(e @ (A @ e))
        e = oracle.gs(Am, e, z, "lex", 1)
        rc = P.T @ (-(A @ e))
        ec = np.zeros(nc)
        ec[1:] = lu.solve(rc[1:])
        e = oracle.gs(Am, e + P @ ec, z, "lex", 2)
        e -= e.mean()
        rates.append(np.sqrt(e @ (A @ e)))
    return float(np.exp(np.mean(np.log(rates[-10:]))))


def test_two_level_factors_per_aggregation_level():
    # Section 3.2: on the 256^2, eps = 1e-4 grid the two-level factor with an exact coarse solve is
    # 0.46 with caliber-1 (veto on) and 0.28 with caliber-2, "at every aggregation level"
    g = gg.grid2d(256, 256, 1.0, 1e-4)
    for cal, paper in ((0, 0.46), (1, 0.28)):
        H = oracle.Hierarchy(g, caliber2=cal, coarsest_max=300)
        aggs = [L for L in H.levels if L["kind"] == "agg"][:3]
        for L in aggs:
            v = two_level_factor(L)
            assert band(paper, v), (cal, L["n"], v)


# ----------------------------------------------------------------------------- caliber-2 gate

@pytest.mark.parametrize("make,paper", [
    (lambda: gg.aniso_patch(256, 64, 1e-4), 0.06),
    (lambda: gg.aniso_patch(512, 64, 1e-4), 0.015),
    (lambda: gg.grid2d(256, 256, 1.0, 1e-4), 0.99),
])
def test_caliber2_gate_fraction(make, paper):
    # Table 2: share of locally one-dimensional nodes that take caliber-2, measured here over the
    # nodes that can take it (the non-seed nodes of the first aggregation level)
    H = oracle.Hierarchy(make(), coarsest_max=300)
    L = next(l for l in H.levels if l["kind"] == "agg")
    assoc = int(np.sum(L["seed_of"] != np.arange(L["n"])))
    v = L["n_caliber2"] / assoc
    assert band(paper, v), v


def test_caliber2_gate_is_inert_on_an_isotropic_grid():
    H = oracle.Hierarchy(gg.grid2d(256, 256), coarsest_max=300)
    L = next(l for l in H.levels if l["kind"] == "agg")
    assert L["n_caliber2"] / np.sum(L["seed_of"] != np.arange(L["n"])) < 0.01
