"""Recorded paths: columns replayed from the record equal the walk's bit for
bit (same arithmetic, same order) in both modes, the adjoint from the record
equals the recomputing adjoint, and the record holds every segment."""
import numpy as np
import pytest

import oracle
import synth
from tinytrees import leaf_boxes, random_octree

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


def _cases():
    rng = np.random.default_rng(600)
    keys, lev, _ = random_octree(rng, 1, 6, 0.4)
    lo, hi = leaf_boxes(keys, lev)
    src = np.concatenate([rng.random((150, 3)), 0.5 * (lo + hi)[::3], lo[::11]])
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 3)).astype(np.float32)
    yield "amr", keys, lev, None, src, dens, 2
    c = synth.uniform_cloud(4, 2.0, 9, fracs=synth.SPECIES_FRACTIONS, dtype=np.float32)
    yield "uniform", c.keys, c.levels, None, synth.leaf_centres(c), c.dens, 1


@pytest.mark.parametrize("mode", ["f32k", "fp64"])
def test_replayed_columns_equal_walk(rt, mode):
    for name, keys, lev, ext, src, dens, nside in _cases():
        tree = rt.Octree(_dev(keys), _dev(lev), extent=ext)
        s, d = _dev(src), _dev(dens)
        walk = rt.trace_columns(tree, s, nside, d, mode).cpu().numpy()
        nseg, _ = rt.trace_paths(tree, s, nside, mode)
        p = rt.Paths(tree, s, nside, mode)
        info = p.info()
        assert info["segments"] == int(nseg.sum()) and info["rays"] == src.shape[0] * 12 * nside ** 2
        rep = p.columns(d).cpu().numpy()
        np.testing.assert_array_equal(rep, walk, err_msg=name)
        # twice in a row, and against the oracle
        np.testing.assert_array_equal(p.columns(d).cpu().numpy(), walk)
        want, _, _ = oracle.trace(keys, lev, dens.astype(np.float64), src, oracle.healpix(nside), extent=ext)
        assert np.all(np.abs(rep - want) <= 1e-5 * np.abs(want) + 1e-30)
        p.close()
        tree.close()


@pytest.mark.parametrize("mode", ["f32k", "fp64"])
def test_replayed_adjoint_equals_recomputed(rt, mode):
    import torch
    for name, keys, lev, ext, src, dens, nside in _cases():
        tree = rt.Octree(_dev(keys), _dev(lev), extent=ext)
        s = _dev(src)
        nd = 12 * nside ** 2
        g = torch.from_numpy(np.random.default_rng(1).standard_normal((src.shape[0], nd, 3))).cuda()
        a1 = rt.trace_columns_adjoint(tree, s, nside, g, mode, path_policy=1).cpu().numpy()
        a2 = rt.trace_columns_adjoint(tree, s, nside, g, mode, path_policy=2).cpu().numpy()
        p = rt.Paths(tree, s, nside, mode)
        a3 = p.adjoint(g).cpu().numpy()
        scale = np.abs(a1).max()
        np.testing.assert_allclose(a2, a1, rtol=1e-12, atol=1e-13 * scale, err_msg=name)
        np.testing.assert_allclose(a3, a1, rtol=1e-12, atol=1e-13 * scale, err_msg=name)
        p.close()
        tree.close()
