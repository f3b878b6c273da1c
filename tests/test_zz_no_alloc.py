"""The allocation-free test-vector entry point (for callers that cannot allocate device memory,
e.g. code running inside another framework's memory pool) against the allocating one.

Collected last on purpose: it shares a device-side scratch array that persists between calls,
so it runs after every other test and also on its own in a fresh process.
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


@pytest.mark.parametrize("make,level", [
    (lambda: gg.grid2d(96, 80, 1.0, 1e-3), 1),
    (lambda: gg.random_connected(3000, 9000, seed=5), 4),
])
def test_noalloc_testvectors_equal_allocating_entry_point(make, level):
    import torch
    g = make()
    A = oracle.laplacian(g)
    col, ncol = oracle.colour(A)
    K, nu, seed = 4, 3, 3
    ref = lamg.testvectors(A.rp, A.ci, A.val, A.diag, col, level, seed, K, nu)
    t = _device_inputs(A, col)
    X = torch.full((g.n, K), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                       # two calls in a row share the scratch array
        X.fill_(float("nan"))
        lamg.testvectors_noalloc(g.n, t["rp"].data_ptr(), t["ci"].data_ptr(), t["val"].data_ptr(),
                                 t["diag"].data_ptr(), t["colour"].data_ptr(), ncol, level, seed, K, nu,
                                 X.data_ptr(), stream)
        torch.cuda.synchronize()
        got = X.cpu().numpy()
        # the tolerance of the other test-vector tests: bit-exact
        assert np.array_equal(got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    with pytest.raises(lamg.LamgError) as e:
        lamg.testvectors_noalloc((1 << 21) + 1, 1, 1, 1, 1, 1, 4, 0, 3, 4, 3, 1)
    assert e.value.code == 1
    with pytest.raises(lamg.LamgError):
        lamg.testvectors_noalloc(100, 1, 1, 1, 1, 1, 1025, 0, 3, 4, 3, 1)
