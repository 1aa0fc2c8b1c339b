"""Fused per-source epilogues (A_V,eff, escape probability, attenuation)
against the oracle's definitions evaluated on the oracle's FP64 columns.

Bars, from the columns' bar eps (FP64: the columns are bitwise the oracle's,
so only the exponential and logarithm round, 1e-12; F32-Kahan: eps = 1e-5
relative per column, and the combined column N = sum_k w_k I_k with w >= 0
keeps it):
- A_V,eff = -(1/gamma) ln((1/N_r) sum_q exp(-gamma a N_q)): its change is
  a sum_q p_q dN_q with p_q the normalized weights exp(-gamma a N_q), and
  a sum_q p_q N_q <= A_V,eff (the log-mean-exp is at least the p-weighted
  mean), so the relative error is at most eps;
- beta: each term f(tau) = (1 - e^-tau) / tau has |tau f'(tau) / f(tau)| <= 1,
  so each term and their mean are within eps;
- attenuation exp(-a N): relative error a N eps = tau eps."""
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


@pytest.mark.parametrize("mode,rtol", [("fp64", 1e-12), ("f32k", 1e-5)])
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
        want = ep.attenuation(cols, w, a)
        tau = a * np.tensordot(cols, np.asarray(w), axes=([2], [0]))
        assert np.all(np.abs(got - want) <= want * (tau + 1.0) * rtol)
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
    np.testing.assert_allclose(got, ep.av_eff(cols, w, 0.3), rtol=1e-5)
    tree.close()
