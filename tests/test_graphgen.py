"""The seeded generators return valid symmetric graphs of the requested shapes."""
import numpy as np
import pytest

import graphgen as gg


def check(g):
    assert g.rp[0] == 0 and g.rp[-1] == len(g.ci) == len(g.w)
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    assert np.all(rows != g.ci)
    assert np.all(g.w > 0)
    for u in range(min(g.n, 500)):
        seg = g.ci[g.rp[u]:g.rp[u + 1]]
        assert np.all(np.diff(seg) > 0)
    A = {(int(a), int(b)): float(c) for a, b, c in zip(rows, g.ci, g.w)}
    for (a, b), c in list(A.items())[:5000]:
        assert A[(b, a)] == c


@pytest.mark.parametrize("make,n,m", [
    (lambda: gg.grid2d(64, 64), 4096, 8064),
    (lambda: gg.grid2d(32, 16, 1.0, 1e-3), 512, 31 * 16 + 32 * 15),
    (lambda: gg.grid3d(6, 5, 4, "loguniform"), 120, 5 * 5 * 4 + 6 * 4 * 4 + 6 * 5 * 3),
    (lambda: gg.path(10), 10, 9),
    (lambda: gg.cycle(10), 10, 10),
    (lambda: gg.star(10), 10, 9),
])
def test_shapes(make, n, m):
    g = make()
    check(g)
    assert g.n == n and g.m == m and g.nnz_L == n + 2 * m


def test_random_families_are_connected():
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg
    for g in [gg.chung_lu(3000, 2.1, 16, seed=1), gg.rgg(2000, 10, seed=1), gg.barabasi_albert(1500, 4, seed=1),
              gg.random_connected(300, 100, seed=2), gg.grid_with_hubs(20, 20, 3, 150, seed=1)]:
        check(g)
        A = sp.csr_matrix((g.w, g.ci, g.rp), shape=(g.n, g.n))
        assert csg.connected_components(A, directed=False)[0] == 1


def test_aniso_weights_and_rhs():
    g = gg.grid2d(16, 16, 1.0, 1e-3)
    assert set(np.unique(g.w)) == {1e-3, 1.0}
    b = gg.rhs(g, 2)
    assert abs(b.sum()) < 1e-12 and np.linalg.norm(b) > 0
    B = gg.rhs(g, 2, k=3)
    assert B.shape == (256, 3) and np.allclose(B.sum(axis=0), 0, atol=1e-12)
    assert np.array_equal(gg.rhs(g, 2), gg.rhs(g, 2))


def test_grid_with_hubs_degrees():
    g = gg.grid_with_hubs(30, 30, 4, 200, seed=3)
    check(g)
    deg = np.diff(g.rp)
    # each hub: its 200 grid neighbours plus the neighbouring hubs in the chain
    assert list(deg[900:]) == [201, 202, 202, 201]
    assert deg[:900].max() <= 4 + 4   # grid degree plus at most a few hub links per node
