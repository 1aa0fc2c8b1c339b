"""GPU contribution-grid construction against the plain recursive oracle:
identical leaves (keys and levels bit for bit) and leaf means."""
import numpy as np
import pytest

import oracle
import synth
from oracle import amr_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_09882_gb300 as rt
    return rt


def _morton_order(a, L):
    """[z][y][x](...) -> Morton order at level L (the generator's encoder)."""
    n = 1 << L
    g = np.arange(n, dtype=np.uint64)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    idx = synth.interleave(x.ravel(), y.ravel(), z.ravel())
    out = np.empty((n ** 3,) + a.shape[3:], dtype=a.dtype)
    out[idx.astype(np.int64)] = a.reshape((n ** 3,) + a.shape[3:])
    return out


@pytest.mark.parametrize("L,sigma,thr,var,maxl,dtype", [
    (4, 1.0, 1.0, 0.01, 4, np.float64), (5, 2.0, 1.0, 0.01, 5, np.float32),
    (5, 1.0, 0.5, 0.3, 3, np.float32), (6, 1.5, 2.0, 0.2, 6, np.float64)])
def test_build_matches_oracle(rt, L, sigma, thr, var, maxl, dtype):
    import torch
    rng = np.random.default_rng(L * 7 + int(10 * sigma))
    n = synth.grf_lognormal(1 << L, sigma, rng).astype(dtype)
    vals = np.stack([n, (0.4 * n).astype(dtype)], axis=-1)
    k0, l0, m0 = amr_build.build(n, vals, thr, var, maxl)
    nm = torch.from_numpy(_morton_order(n, L)).cuda()
    vm = torch.from_numpy(_morton_order(vals, L)).cuda()
    keys, lev, means = rt.build_amr(nm, vm, thr, var, maxl)
    np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64), k0)
    np.testing.assert_array_equal(lev.cpu().numpy(), l0)
    rtol = 1e-12 if dtype == np.float64 else 2e-7
    np.testing.assert_allclose(means.cpu().numpy(), m0, rtol=rtol)
    # the result is a valid octree the tracer accepts
    tree = rt.Octree(keys, lev)
    assert tree.n_leaves == len(k0)
    tree.close()


def test_build_single_dense_cell(rt):
    import torch
    L = 5
    n = np.ones((1 << L,) * 3)
    n[3, 17, 30] = 50.0
    keys, lev, _ = rt.build_amr(torch.from_numpy(_morton_order(n, L)).cuda(), None, 1.0, 0.01, L)
    assert keys.numel() == 7 * L + 1
