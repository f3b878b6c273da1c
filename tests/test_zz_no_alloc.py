"""The allocation-free test-vector entry point against the allocating one and the oracle.

lamg_testvectors_noalloc serves callers that cannot allocate device memory themselves (code
running inside another framework's memory pool, plugins limited to the buffers they are given,
programs that must not allocate after start-up): it takes device inputs and output and keeps its
scratch in a fixed device array.

Collected last on purpose: it shares a device-side scratch array that persists between calls,
so it runs after every other test and also on its own in a fresh process. Tolerance: the
test-vector tests' own bar, bit-exact against lamg_testvectors in the same summation order and
against the oracle in stored order; within rounding against the oracle in the strided order on
rows of more than 32 entries.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_2606_24791_b300 as lamg

pytestmark = pytest.mark.gpu


def _device_inputs(A, col):
    import torch
    dev = torch.device("cuda", 0)
    t = dict(rp=torch.from_numpy(A.rp.astype(np.int64)).to(dev),
             ci=torch.from_numpy(A.ci.astype(np.int32)).to(dev),
             val=torch.from_numpy(A.val).to(dev),
             diag=torch.from_numpy(A.diag).to(dev),
             colour=torch.from_numpy(col.astype(np.int32)).to(dev))
    return t


def _noalloc(t, n, ncol, level, seed, K, nu, order):
    import torch
    X = torch.full((n, K), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lamg.testvectors_noalloc(n, t["rp"].data_ptr(), t["ci"].data_ptr(), t["val"].data_ptr(),
                             t["diag"].data_ptr(), t["colour"].data_ptr(), ncol, level, seed, K, nu,
                             X.data_ptr(), stream, order=order)
    torch.cuda.synchronize()
    return X.cpu().numpy()


GRAPHS = [
    ("aniso grid 96x80", lambda: gg.grid2d(96, 80, 1.0, 1e-3), 1),
    ("random 3000", lambda: gg.random_connected(3000, 9000, seed=5), 4),
    # rows of several hundred entries: one warp per row in the strided order
    ("grid with degree-600 hubs", lambda: gg.grid_with_hubs(48, 48, 6, 600, seed=2), 2),
    ("barabasi-albert 20000", lambda: gg.barabasi_albert(20000, 4, seed=1), 0),
]


@pytest.mark.parametrize("name,make,level", GRAPHS)
@pytest.mark.parametrize("order", [lamg.TV_STRIDED, lamg.TV_STORED])
def test_noalloc_testvectors_equal_allocating_entry_point_and_oracle(name, make, level, order):
    g = make()
    A = oracle.laplacian(g)
    col, ncol = oracle.colour(A)
    K, nu, seed = 4, 3, 3
    ref = lamg.testvectors(A.rp, A.ci, A.val, A.diag, col, level, seed, K, nu, order=order)
    orc = oracle.testvectors(A, level, seed, K, nu)
    long_rows = np.diff(A.rp).max() > 32
    t = _device_inputs(A, col)
    for _ in range(2):                       # two calls in a row share the scratch array
        got = _noalloc(t, g.n, ncol, level, seed, K, nu, order)
        assert np.array_equal(got, ref), name
        if order == lamg.TV_STORED or not long_rows:
            assert np.array_equal(got, orc), name
        else:
            assert np.abs(got - orc).max() <= 1e-12 * np.abs(orc).max(), name


def test_noalloc_rows_with_colours_out_of_range_keep_their_start():
    # documented contract: a row whose colour is outside [0, ncol) is never relaxed
    g = gg.grid2d(40, 30, 1.0, 0.1)
    A = oracle.laplacian(g)
    col, ncol = oracle.colour(A)
    bad = np.array([5, 77, 401])
    col = col.copy()
    col[bad] = ncol + 3
    got = _noalloc(_device_inputs(A, col), g.n, ncol, 1, 3, 4, 3, lamg.TV_STRIDED)
    for u in bad:
        assert np.array_equal(got[u], [oracle.random_start(3, 1, int(u), k) for k in range(4)])
    assert np.isfinite(got).all()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    with pytest.raises(lamg.LamgError) as e:
        lamg.testvectors_noalloc((1 << 21) + 1, 1, 1, 1, 1, 1, 4, 0, 3, 4, 3, 1)
    assert e.value.code == 1
    with pytest.raises(lamg.LamgError):
        lamg.testvectors_noalloc(100, 1, 1, 1, 1, 1, 1025, 0, 3, 4, 3, 1)
    with pytest.raises(lamg.LamgError):
        lamg.testvectors_noalloc(100, 1, 1, 1, 1, 1, 4, 0, 3, 17, 3, 1)      # K > 16
    with pytest.raises(lamg.LamgError):
        lamg.testvectors_noalloc(100, 1, 1, 1, 1, 1, 4, 0, 3, 4, 3, 1, order=2)
