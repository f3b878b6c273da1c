"""Chebyshev smoothing on levels with many colours, GPU against the oracle (B300).

The smoothing polynomial is the same arithmetic on both sides up to summation order and the
reciprocal diagonal, so the FP64 bars are those of Gauss-Seidel levels: cycle and FCG iterates
within 1e-10 of the oracle on its own hierarchy, solutions to 1e-9 with equal iteration counts.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_2606_24791_b300 as lamg
from test_gpu_parity import oracle_levels

pytestmark = pytest.mark.gpu


def rel(a, b):
    """max(norm ratio, largest element difference / largest element): bounds the whole vector
    and every entry."""
    a, b = np.asarray(a), np.asarray(b)
    d = a - b
    return max(np.linalg.norm(d) / max(np.linalg.norm(b), 1e-300),
               np.abs(d).max(initial=0.0) / max(np.abs(b).max(initial=0.0), 1e-300))


CASES = {
    # every aggregation level smoothed by the polynomial (colour threshold 1)
    "grid_all": (lambda: gg.grid2d(40, 36, 1.0, 0.1), dict(coarsest_max=16, cheb_colours=1)),
    "hubs_all": (lambda: gg.grid_with_hubs(40, 40, 4, 500, seed=3), dict(coarsest_max=16, cheb_colours=1)),
    # the default threshold: only the coarse power-law level with 43 colours
    "chunglu5000": (lambda: gg.chung_lu(5000, 2.1, 16, seed=1), dict(coarsest_max=24)),
}


def check_cheb_buffers(ops):
    # a smoothing phase alternates the iterate between x (0) and the second buffer t (1): every
    # step reads where the iterate is, the copy t -> x runs only when the iterate is in t, and
    # every other step of the level finds the iterate in x
    where = {}
    for kind, lv, colour in ops:
        if kind == "cheb_first":
            where[lv] = colour
        elif kind == "cheb":
            src = 1 if colour >= 256 else 0
            assert where.get(lv, 0) == src, (kind, lv, colour)
            where[lv] = 1 - src
        elif kind == "cheb_copy":
            assert where.get(lv) == 1, (kind, lv)
            where[lv] = 0
        elif kind in ("resid", "restrict", "prolong"):
            assert where.get(lv, 0) == 0, (kind, lv)
    assert all(v == 0 for v in where.values()), where


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("degree", [1, 2, 3])
def test_cheb_cycle_and_iterates_match_oracle(name, degree):
    make, opts = CASES[name]
    g = make()
    o = dict(opts, cheb_degree=degree)
    H = oracle.Hierarchy(g, **o)
    assert any(L["cheb"] for L in H.levels)
    P = lamg.import_levels(oracle_levels(H), cheb_colours=o.get("cheb_colours", 32), cheb_degree=degree)
    ops = P.op_list()
    kinds = {k for k, _, _ in ops}
    assert "cheb" in kinds and not ("cheb_copy" in kinds and degree % 2 == 0)
    check_cheb_buffers(ops)
    rng = np.random.default_rng(4)
    r = rng.standard_normal(g.n)
    r -= r.mean()
    assert rel(P.cycle(r), H.cycle(r)) <= 1e-10, name
    b = gg.rhs(g, 2)
    ref = H.fcg(b, tol=1e-300, maxit=4, record=True)
    for k in range(1, ref["iters"] + 1):
        x, _ = P.solve(b, tol=1e-300, maxit=k, allow_unconverged=True)
        assert rel(x, ref["iterates"][k - 1]) <= 1e-10, (name, k)
    P.close()


def test_cheb_setup_matches_oracle_and_solves():
    g = gg.chung_lu(20000, 2.1, 16, seed=1)
    b = gg.rhs(g, 2)
    H = oracle.Hierarchy(g)
    P = lamg.setup(g, tv_order=lamg.TV_STORED)   # the oracle's hierarchy
    assert [i["n"] for i in P.info] == [L["n"] for L in H.levels]
    assert sum(L["cheb"] for L in H.levels) >= 1
    x, st = P.solve(b, 1e-8, 200)
    ref = H.fcg(b, 1e-8, 200)
    assert st["iters"] == ref["iters"] and st["relres_true"] <= 2e-8
    assert rel(x, ref["x"]) <= 1e-9
    # multi-RHS columns equal single solves; the FP32 cycle reaches the tolerance
    B = gg.rhs(g, seed=5, k=3)
    X, sts = P.solve_batch(B, 1e-8, 200)
    for j in range(3):
        xj, stj = P.solve(B[:, j], 1e-8, 200)
        assert sts[j]["iters"] == stj["iters"] and rel(X[:, j], xj) <= 1e-10
    P32 = lamg.setup(g, precision=lamg.FP32)
    x32, st32 = P32.solve(b, 1e-8, 200)
    assert st32["relres_true"] <= 2e-8
    assert np.linalg.norm(x32 - ref["x"]) <= 1e-5 * np.linalg.norm(ref["x"])   # solution accuracy, FP32 cycle
    P.close()
    P32.close()


def test_cheb_rejects_bad_degree():
    g = gg.grid2d(16, 16)
    with pytest.raises(lamg.LamgError):
        lamg.setup(g, cheb_degree=9)
    with pytest.raises(lamg.LamgError):
        lamg.setup(g, cheb_degree=0)


def test_cheb_step_timer_reports_one_launch_and_its_work():
    # lamg_time_kernel_batch's one-step unit on a Chebyshev level: one bk_cheb launch, a
    # multiply-add per stored entry and column plus six flops per row and column
    g = gg.chung_lu(20000, 2.1, 16, seed=1)
    P = lamg.setup(g)
    lv = [l for l, L in enumerate(P.info) if L["kind"] == "agg" and L["ncol"] > 32]
    assert lv
    B = gg.rhs(g, seed=3, k=4)
    P.solve_batch(B, 1e-8, 200)
    L = P.info[lv[0]]
    r = P.time_kernel_batch("cheb_step", lv[0], 4, reps=2)
    assert r["launches"] == 1 and r["ms"] > 0
    assert r["flops"] == pytest.approx(4 * (2 * L["nnz"] + 6 * L["n"]))
    with pytest.raises(Exception):
        P.time_kernel_batch("cheb_step", 0, 4, reps=1)   # level 0 is not a Chebyshev level
    P.close()
