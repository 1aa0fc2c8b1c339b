"""Non-finite or negative densities: the device check records RT_ERR_NONFINITE
with the leaf's index as the fault position (rt_trace_columns, the chunked
trace, the epilogue), the host-buffer call returns the code, and zero
densities are valid."""
import numpy as np
import pytest

from tinytrees import random_octree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_09882_gb300 as rt
    return rt


def _dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -0.5])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_bad_density_sets_nonfinite(rt, bad, dt):
    rng = np.random.default_rng(1700)
    keys, lev, _ = random_octree(rng, 1, 4, 0.4)
    S = 3
    dens = rng.uniform(0.0, 2.0, size=(keys.shape[0], S)).astype(dt)
    dens[5] = 0.0  # zeros are fine
    leaf = keys.shape[0] - 2
    dens[leaf, 2] = bad
    src = _dev(rng.random((40, 3)))
    tree = rt.Octree(_dev(keys), _dev(lev))
    mode = "fp64" if dt == np.float64 else "f32k"
    rt.trace_columns(tree, src, 1, _dev(dens), mode)
    st = tree.stats()
    assert st["status"] == 7 and st["fault_ray"] == leaf, st
    tree.reset_stats()
    rt.trace_columns_chunked(tree, src, 1, _dev(dens), 3, mode)
    st = tree.stats()
    assert st["status"] == 7 and st["fault_ray"] == leaf, st
    tree.reset_stats()
    rt.trace_epilogue(tree, src, 1, _dev(dens), "av_eff", [1.0, 1.0, 1.0], 0.5, mode=mode)
    assert tree.stats()["status"] == 7
    dens[leaf, 2] = 0.0
    tree.reset_stats()
    rt.trace_columns(tree, src, 1, _dev(dens), mode)
    assert tree.stats()["status"] == 0
    tree.close()


def test_host_call_returns_nonfinite(rt):
    import torch
    rng = np.random.default_rng(1701)
    keys, lev, _ = random_octree(rng, 1, 4, 0.4)
    dens = rng.uniform(0.1, 2.0, size=(keys.shape[0], 4)).astype(np.float32)
    dens[3, 1] = np.nan
    with pytest.raises(rt.RTError) as e:
        rt.trace_columns_host(torch.from_numpy(keys.view(np.int64)), torch.from_numpy(lev),
                              torch.from_numpy(rng.random((64, 3))), 1, torch.from_numpy(dens), "f32k")
    assert e.value.code == 7
