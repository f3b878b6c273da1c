"""The two large configurations at full size, and a per-cycle parity check on a cut of the 3D
family (needs a B300).

- 192^3 7-point grid with i.i.d. log-uniform weights in [1e-3, 1e3] (7,077,888 nodes,
  49,324,032 nonzeros of L), 16 mean-zero Gaussian right-hand sides, FP32 cycle and FP64 cycle
  inside FP64 CG;
- Chung-Lu graph of 4,000,000 nodes (exponent 2.1, mean degree 16, largest component), 32
  right-hand sides, FP64 cycle and FP32 cycle.

Every column must reach ||b - L phi|| / ||b|| <= 1e-8 by the recursive residual and 2e-8 by the
true residual recomputed here from the graph (Eq. 1), and sampled columns must agree with the
same right-hand side solved alone (1e-6: two solves that each stop at 1e-8, in another
summation order; 1e-10 for the FP64 columns, whose iterations coincide).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_2606_24791_b300 as lamg

pytestmark = pytest.mark.gpu


def true_relres(g, X, B):
    R = gg.laplacian_apply(g, X) - (B - B.mean(axis=0, keepdims=True))
    return np.linalg.norm(R, axis=0) / np.linalg.norm(B - B.mean(axis=0, keepdims=True), axis=0)


def rel(a, b):
    d = np.asarray(a) - np.asarray(b)
    return max(np.linalg.norm(d) / np.linalg.norm(b), np.abs(d).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def grid192():
    g = gg.config_graph("grid3d192_hetero")
    return g, gg.rhs(g, seed=2, k=16)


@pytest.fixture(scope="module")
def chunglu4m():
    g = gg.config_graph("chunglu4m")
    return g, gg.rhs(g, seed=2, k=32)


@pytest.mark.parametrize("precision", [lamg.FP32, lamg.FP64])
def test_grid192_16_rhs(grid192, precision):
    g, B = grid192
    assert g.n == 192 ** 3 and g.nnz_L == 49_324_032
    P = lamg.setup(g, precision=precision)
    X, sts = P.solve_batch(B, 1e-8, 200)
    assert all(s["relres"] <= 1e-8 and s["relres_true"] <= 2e-8 for s in sts)
    assert true_relres(g, X, B).max() <= 2e-8
    for j in (0, 9):
        x1, st1 = P.solve(B[:, j], 1e-8, 200)
        assert rel(X[:, j], x1) <= (1e-10 if precision == lamg.FP64 else 1e-6), j
        if precision == lamg.FP64:
            assert st1["iters"] == sts[j]["iters"]
    P.close()


@pytest.mark.parametrize("precision", [lamg.FP64, lamg.FP32])
def test_chunglu4m_32_rhs(chunglu4m, precision):
    g, B = chunglu4m
    assert g.n > 3_800_000
    P = lamg.setup(g, precision=precision)
    assert any(L["kind"] == "agg" and L["ncol"] > 32 for L in P.info)   # Chebyshev levels
    X, sts = P.solve_batch(B, 1e-8, 200)
    assert all(s["relres"] <= 1e-8 and s["relres_true"] <= 2e-8 for s in sts)
    assert true_relres(g, X, B).max() <= 2e-8
    for j in (0, 31):
        x1, st1 = P.solve(B[:, j], 1e-8, 200)
        assert rel(X[:, j], x1) <= (1e-10 if precision == lamg.FP64 else 1e-6), j
    P.close()


def test_cycle_parity_on_a_48_cube_of_the_3d_family():
    # the oracle's hierarchy of a 48^3 grid of the same family (i.i.d. log-uniform weights),
    # imported: every cycle and every CG iterate within 1e-10 of the oracle's
    g = gg.grid3d(48, 48, 48, "loguniform", seed=1)
    H = oracle.Hierarchy(g)
    levels = []
    for L in H.levels:
        d = dict(kind=L["kind"], n=L["n"], rp=L["rp"], ci=L["ci"], val=L["val"], diag=L["diag"],
                 gamma=L["gamma"], nc=L["nc"])
        if L["kind"] == "agg":
            d.update(colour=L["colour"], agg=L["agg"], agg2=L["agg2"], wt=L["wt"])
        if L["kind"] == "elim":
            d.update(cidx=L["cidx"])
        levels.append(d)
    P = lamg.import_levels(levels)
    rng = np.random.default_rng(3)
    for _ in range(2):
        r = rng.standard_normal(g.n)
        r -= r.mean()
        assert rel(P.cycle(r), H.cycle(r)) <= 1e-10
    b = gg.rhs(g, 2)
    ref = H.fcg(b, tol=1e-300, maxit=5, record=True)
    for k in range(1, ref["iters"] + 1):
        x, _ = P.solve(b, tol=1e-300, maxit=k, allow_unconverged=True)
        assert rel(x, ref["iterates"][k - 1]) <= 1e-10, k
    P.close()
