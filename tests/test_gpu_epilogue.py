"""Fused per-source epilogues (A_V,eff, escape probability, attenuation)
against the oracle's definitions evaluated on the oracle's FP64 columns."""
import numpy as np
import pytest

import oracle
import synth
from oracle import epilogue as ep
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


@pytest.mark.parametrize("mode,rtol", [("fp64", 1e-12), ("f32k", 2e-5)])
def test_epilogues_match_oracle(rt, mode, rtol):
    rng = np.random.default_rng(777)
    keys, lev, _ = random_octree(rng, 1, 6, 0.4)
    S = 3
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], S))
    lo, hi = leaf_boxes(keys, lev)
    src = np.concatenate([rng.random((200, 3)), 0.5 * (lo + hi)[::4]])
    w = [1.0, 2.0, 0.5]
    for nside in (1, 2):
        cols, _, _ = oracle.trace(keys, lev, dens, src, oracle.healpix(nside))
        tree = rt.Octree(_dev(keys), _dev(lev))
        s, d = _dev(src), _dev(dens)
        a = 0.8
        got = rt.trace_epilogue(tree, s, nside, d, "av_eff", w, a, gamma=3.02, mode=mode).cpu().numpy()
        np.testing.assert_allclose(got, ep.av_eff(cols, w, a, 3.02), rtol=rtol)
        coef = rng.uniform(0.0, 3.0, size=src.shape[0])
        coef[:5] = 0.0  # tau = 0: every term is 1
        got = rt.trace_epilogue(tree, s, nside, d, "beta", w, 0.0, coef=_dev(coef), mode=mode).cpu().numpy()
        np.testing.assert_allclose(got, ep.beta(cols, w, coef), rtol=rtol)
        assert np.all(got[:5] == 1.0)
        got = rt.trace_epilogue(tree, s, nside, d, "attenuation", w, a, mode=mode).cpu().numpy()
        np.testing.assert_allclose(got, ep.attenuation(cols, w, a), rtol=10 * rtol)
        assert tree.stats()["status"] == 0
        tree.close()


def test_av_eff_uniform_cloud_centres(rt):
    """The uniform-grid walk with the epilogue: all leaf centres of a 16^3 cloud."""
    c = synth.uniform_cloud(4, 2.0, 9, fracs=synth.SPECIES_FRACTIONS, dtype=np.float32)
    src = synth.leaf_centres(c)
    cols, _, _ = oracle.trace(c.keys, c.levels, c.dens.astype(np.float64), src, oracle.healpix(1))
    tree = rt.Octree(_dev(c.keys), _dev(c.levels))
    w = [1.0, 2.0, 0.0, 0.0]
    got = rt.trace_epilogue(tree, _dev(src), 1, _dev(c.dens), "av_eff", w, 0.3, mode="f32k").cpu().numpy()
    np.testing.assert_allclose(got, ep.av_eff(cols, w, 0.3), rtol=2e-5)
    tree.close()
