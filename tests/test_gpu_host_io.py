"""The host-buffer forward call (rt_trace_columns_host): columns and statistics
equal to the device-buffer call on the same inputs, for pageable and
page-locked host tensors, chunk sizes that leave a ragged last chunk, a
single chunk, no sources, and a faulting source; and within the parity bar of
the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from tinytrees import random_octree

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-5, 1e-30


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_09882_gb300 as rt
    return rt


def _case(seed=11, n_src=1000):
    rng = np.random.default_rng(seed)
    keys, lev, _ = random_octree(rng, 2, 6, 0.3)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 4)).astype(np.float32)
    src = rng.random((n_src, 3))
    return keys, lev, dens, src


def _device_columns(rt, keys, lev, dens, src, nside, mode):
    import torch
    tree = rt.Octree(torch.from_numpy(keys.view(np.int64)).cuda(), torch.from_numpy(lev).cuda())
    tree.reset_stats()
    cols = rt.trace_columns(tree, torch.from_numpy(src).cuda(), nside, torch.from_numpy(dens).cuda(), mode)
    out = cols.cpu().numpy()
    st = tree.stats()
    tree.close()
    return out, st


@pytest.mark.parametrize("mode", ["f32k", "fp64"])
@pytest.mark.parametrize("chunk,pinned", [(96, False), (96, True), (0, True), (4096, False)])
def test_host_call_equals_device_call(rt, mode, chunk, pinned):
    import torch
    keys, lev, dens, src = _case()
    want, st_dev = _device_columns(rt, keys, lev, dens, src, 2, mode)
    args = [torch.from_numpy(a) for a in (keys.view(np.int64), lev, src, dens)]
    if pinned:
        args = [a.pin_memory() for a in args]
    k, l, s, d = args
    got, st = rt.trace_columns_host(k, l, s, 2, d, mode, chunk=chunk)
    np.testing.assert_array_equal(got.numpy(), want)
    assert st["status"] == 0 and st["rays"] == st_dev["rays"] == 1000 * 48
    assert st["segments"] == st_dev["segments"]


def test_host_call_against_oracle(rt):
    import torch
    keys, lev, dens, src = _case(12, 333)
    want, _, _ = oracle.trace(keys, lev, dens.astype(np.float64), src, oracle.healpix(1))
    got, st = rt.trace_columns_host(torch.from_numpy(keys.view(np.int64)), torch.from_numpy(lev),
                                    torch.from_numpy(src), 1, torch.from_numpy(dens), "f32k", chunk=64)
    d = np.abs(got.numpy().astype(np.float64) - want)
    assert (d <= RTOL * np.abs(want) + ATOL).all()


def test_host_call_uniform_grid_with_extent_none(rt):
    import torch
    cloud = synth.uniform_cloud(4, 1.5, 21, fracs=synth.SPECIES_FRACTIONS, dtype=np.float32)
    src = synth.leaf_centres(cloud)
    want, _ = _device_columns(rt, cloud.keys, cloud.levels, cloud.dens, src, 1, "f32k")
    got, st = rt.trace_columns_host(torch.from_numpy(cloud.keys.view(np.int64)), torch.from_numpy(cloud.levels),
                                    torch.from_numpy(src), 1, torch.from_numpy(cloud.dens), "f32k", chunk=512)
    np.testing.assert_array_equal(got.numpy(), want)


def test_host_call_no_sources(rt):
    import torch
    keys, lev, dens, _ = _case()
    got, st = rt.trace_columns_host(torch.from_numpy(keys.view(np.int64)), torch.from_numpy(lev),
                                    torch.zeros((0, 3), dtype=torch.float64), 1, torch.from_numpy(dens))
    assert got.shape == (0, 12, 4) and st["rays"] == 0 and st["status"] == 0


def test_host_call_reports_a_faulting_source(rt):
    import torch
    keys, lev, dens, src = _case(13, 100)
    src[37] = (0.5, 1.5, 0.5)  # outside the unit box
    with pytest.raises(rt.RTError) as e:
        rt.trace_columns_host(torch.from_numpy(keys.view(np.int64)), torch.from_numpy(lev),
                              torch.from_numpy(src), 1, torch.from_numpy(dens), chunk=32)
    assert e.value.code == 5  # RT_ERR_SOURCE_OUTSIDE


def test_host_call_rejects_a_malformed_octree(rt):
    import torch
    keys, lev, dens, src = _case(14, 64)
    keys, lev = keys.copy(), lev.copy()
    keys[[3, 4]] = keys[[4, 3]]  # not ascending (each key keeps its level)
    lev[[3, 4]] = lev[[4, 3]]
    with pytest.raises(rt.RTError) as e:
        rt.trace_columns_host(torch.from_numpy(keys.view(np.int64)), torch.from_numpy(lev),
                              torch.from_numpy(src), 1, torch.from_numpy(dens))
    assert e.value.code == 2  # RT_ERR_UNSORTED


def test_host_call_workspace_grows_and_releases(rt):
    import torch
    small = _case(15, 64)
    big = _case(16, 2000)
    for keys, lev, dens, src in (small, big, small):
        want, _ = _device_columns(rt, keys, lev, dens, src, 1, "f32k")
        got, _ = rt.trace_columns_host(torch.from_numpy(keys.view(np.int64)), torch.from_numpy(lev),
                                       torch.from_numpy(src), 1, torch.from_numpy(dens), "f32k", chunk=256)
        np.testing.assert_array_equal(got.numpy(), want)
    rt.trace_columns_host_release()
    keys, lev, dens, src = small
    got, _ = rt.trace_columns_host(torch.from_numpy(keys.view(np.int64)), torch.from_numpy(lev),
                                   torch.from_numpy(src), 1, torch.from_numpy(dens), "f32k")
    rt.trace_columns_host_release()


@pytest.mark.parametrize("mode", ["f32k", "fp64"])
def test_host_call_extent_and_fp64_densities(rt, mode):
    import torch
    rng = np.random.default_rng(17)
    keys, lev, ext = random_octree(rng, 3, 6, 0.3, extent_cells=5)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 2))  # float64 densities
    e = np.asarray(ext, dtype=np.float64) / float(1 << 21)
    src = rng.random((500, 3)) * e
    tree = rt.Octree(torch.from_numpy(keys.view(np.int64)).cuda(), torch.from_numpy(lev).cuda(), extent=ext)
    want = rt.trace_columns(tree, torch.from_numpy(src).cuda(), 2, torch.from_numpy(dens).cuda(), mode).cpu().numpy()
    tree.close()
    got, st = rt.trace_columns_host(torch.from_numpy(keys.view(np.int64)), torch.from_numpy(lev),
                                    torch.from_numpy(src), 2, torch.from_numpy(dens), mode, extent=ext, chunk=128)
    np.testing.assert_array_equal(got.numpy(), want)
    ref, _, _ = oracle.trace(keys, lev, dens, src, oracle.healpix(2), extent=ext)
    if mode == "fp64":
        np.testing.assert_array_equal(got.numpy(), ref)
    else:
        d = np.abs(got.numpy().astype(np.float64) - ref)
        assert (d <= RTOL * np.abs(ref) + ATOL).all()
