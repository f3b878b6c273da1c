"""Many small systems in one launch (lamg_solve_many) against the oracle and single solves (B300).

Each system runs the same cycle steps as the per-step kernels (same kernel forms, same summation
order per row); only the CG reductions are summed in another order (cluster-scope instead of
grid-wide), so each result must match the oracle to the same bars as a single solve (iterates
1e-10, solutions 1e-9 with equal iteration counts) and a single lamg_solve of the same system to
1e-11 (rounding of the reductions, amplified over the iterations).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_2606_24791_b300 as lamg

pytestmark = pytest.mark.gpu


def rel(a, b):
    """max(norm ratio, largest element difference / largest element): bounds the whole vector
    and every entry."""
    a, b = np.asarray(a), np.asarray(b)
    d = a - b
    return max(np.linalg.norm(d) / max(np.linalg.norm(b), 1e-300),
               np.abs(d).max(initial=0.0) / max(np.abs(b).max(initial=0.0), 1e-300))


def small_graphs():
    return [gg.grid2d(64, 64), gg.grid2d(48, 40, 1.0, 1e-3), gg.grid3d(12, 11, 10, "loguniform", seed=2),
            gg.rgg(3000, 10, seed=4), gg.random_connected(2500, 3000, seed=5), gg.grid2d(37, 23, 1.0, 0.3),
            gg.path(500, np.random.default_rng(1).uniform(0.5, 1.5, 499)), gg.grid2d(20, 20)]


def test_many_systems_match_oracle_and_single_solves():
    gs = small_graphs()
    bs = [gg.rhs(g, seed=30 + i) for i, g in enumerate(gs)]
    hs = [lamg.setup(g, tv_order=lamg.TV_STORED) for g in gs]   # the oracle's hierarchies
    xs, sts = lamg.solve_many(hs, bs, tol=1e-8, maxit=200, hist=True)
    for g, b, h, x, st in zip(gs, bs, hs, xs, sts):
        assert st["launches"] == 1 and st["relres_true"] <= 2e-8, (g.name, st)
        ref = oracle.Hierarchy(g).fcg(b, tol=1e-8, maxit=200)
        assert st["iters"] == ref["iters"], g.name
        assert rel(x, ref["x"]) <= 1e-9, g.name
        big = ref["hist"] > 1e-11
        assert np.allclose(st["hist"][big], ref["hist"][big], rtol=1e-8), g.name
        x1, st1 = h.solve(b, 1e-8, 200)
        assert st1["iters"] == st["iters"] and rel(x, x1) <= 1e-11, g.name
    for h in hs:
        h.close()


@pytest.mark.parametrize("make,cm", [(lambda: gg.grid2d(40, 40, 1.0, 1e-3), 16),
                                     (lambda: gg.grid3d(10, 10, 10, "loguniform", seed=1), 16),
                                     (lambda: gg.barabasi_albert(1500, 4, seed=3), 16)])
def test_many_iterates_on_the_oracle_hierarchy(make, cm):
    # the oracle's own hierarchy, two copies with different right-hand sides in one launch:
    # every CG iterate within 1e-10 of the oracle's
    g = make()
    H = oracle.Hierarchy(g, coarsest_max=cm)
    from test_gpu_parity import oracle_levels
    P1 = lamg.import_levels(oracle_levels(H))
    P2 = lamg.import_levels(oracle_levels(H))
    b1, b2 = gg.rhs(g, 2), gg.rhs(g, 9)
    r1 = H.fcg(b1, tol=1e-300, maxit=5, record=True)
    r2 = H.fcg(b2, tol=1e-300, maxit=5, record=True)
    for k in range(1, 6):
        (x1, x2), _ = lamg.solve_many([P1, P2], [b1, b2], tol=1e-300, maxit=k, allow_unconverged=True)
        assert rel(x1, r1["iterates"][k - 1]) <= 1e-10, k
        assert rel(x2, r2["iterates"][k - 1]) <= 1e-10, k
    P1.close()
    P2.close()


def test_systems_the_cluster_kernel_cannot_take_are_solved_too():
    # a hub graph (rows longer than 256 entries) and an FP32-cycle hierarchy take the
    # per-step path inside the same call
    g_hub = gg.grid_with_hubs(40, 40, 4, 500, seed=1)
    g_a, g_b = gg.grid2d(50, 50), gg.grid2d(30, 30, 1.0, 0.01)
    hs = [lamg.setup(g_a), lamg.setup(g_hub), lamg.setup(g_b, precision=lamg.FP32)]
    bs = [gg.rhs(g, 3) for g in (g_a, g_hub, g_b)]
    xs, sts = lamg.solve_many(hs, bs, tol=1e-8, maxit=200)
    assert sts[0]["launches"] == 1 and sts[1]["launches"] > 1
    for g, b, x, st in zip((g_a, g_hub, g_b), bs, xs, sts):
        assert st["relres_true"] <= 2e-8
        r = gg.laplacian_apply(g, x) - (b - b.mean())
        assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(b - b.mean())
    for h in hs:
        h.close()


def test_many_equal_systems_give_equal_bits():
    g = gg.grid2d(32, 32, 1.0, 0.1)
    b = gg.rhs(g, 5)
    hs = [lamg.setup(g) for _ in range(12)]
    xs, sts = lamg.solve_many(hs, [b] * 12, tol=1e-10, maxit=200)
    for x in xs[1:]:
        assert np.array_equal(x, xs[0])
    for h in hs:
        h.close()


def test_device_pointers():
    import ctypes as C
    import torch
    gs = [gg.grid2d(30, 30), gg.grid2d(25, 35)]
    hs = [lamg.setup(g) for g in gs]
    bs = [gg.rhs(g, 7) for g in gs]
    xh, _ = lamg.solve_many(hs, bs, 1e-8, 100)
    bt = [torch.from_numpy(b).cuda() for b in bs]
    xt = [torch.zeros_like(b) for b in bt]
    so = lamg.SolveOpts(1e-8, 100, lamg.DEVICE_PTRS, None)
    st = (lamg.Stats * 2)()
    rc = lamg.lib().lamg_solve_many(2, (C.c_void_p * 2)(*[h._h for h in hs]),
                                    (C.c_void_p * 2)(*[b.data_ptr() for b in bt]),
                                    (C.c_void_p * 2)(*[x.data_ptr() for x in xt]), C.byref(so), st)
    torch.cuda.synchronize()
    assert rc == 0
    for a, x in zip(xh, xt):
        assert np.array_equal(a, x.cpu().numpy())
    for h in hs:
        h.close()
