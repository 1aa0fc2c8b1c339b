"""The leaf-gather adjoint: on a full cube of equal-level leaves with source s
in leaf s, all sources at one offset inside their leaf, every ray of a
direction takes the same steps and segment lengths, and each leaf's gradient
is summed by one thread without atomics.

Checked against the oracle's FP64 gradient with the bound any summation order
obeys: |got - ref| <= rtol * (A^T |g|), the oracle's adjoint of |g| (the sum of
the magnitudes of the terms), rtol 1e-12 in FP64 and 1e-5 in F32-Kahan (FP32
products with Kahan compensation).  Also: bitwise equal gradients on repeated
calls, the scatter (path_policy 1) within the same bound, the forward's
segment count, and the fall-back to the scatter when the sources do not have
the gather's layout."""
import numpy as np
import pytest

import oracle
import synth
from tinytrees import uniform_octree

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


def _centres(keys, lev):
    return synth.leaf_centres(synth.Cloud(keys, lev, np.zeros((keys.shape[0], 1)), (1 << 21,) * 3))


def _bound_check(got, ref, mag, rtol):
    d = np.abs(got - ref)
    lim = rtol * np.abs(mag) + 1e-300
    assert np.all(d <= lim), float((d / np.maximum(mag, 1e-300)).max())


def _run(rt, tree, src, nside, g, mode, policy=0):
    tree.reset_stats()
    gd = rt.trace_columns_adjoint(tree, src, nside, g, mode, path_policy=policy)
    st = tree.stats()
    assert st["status"] == 0, st
    return gd.cpu().numpy(), st


@pytest.mark.parametrize("level,S,nside", [(3, 1, 1), (4, 4, 1), (3, 2, 2), (4, 8, 1), (2, 4, 4), (5, 4, 1), (6, 1, 1)])
def test_gather_matches_oracle(rt, level, S, nside):
    rng = np.random.default_rng(900 + 10 * level + S)
    keys, lev = uniform_octree(level)
    src_h = _centres(keys, lev)
    dirs = oracle.healpix(nside)
    g = rng.standard_normal((src_h.shape[0], dirs.shape[0], S))
    tree = rt.Octree(_dev(keys), _dev(lev))
    src = _dev(src_h)
    ref = oracle.adjoint(keys, lev, S, src_h, dirs, g)
    mag = oracle.adjoint(keys, lev, S, src_h, dirs, np.abs(g))
    gd, st = _run(rt, tree, src, nside, _dev(g), "fp64")
    assert st["gathered"] == 1
    _bound_check(gd, ref, mag, 1e-12)
    again, _ = _run(rt, tree, src, nside, _dev(g), "fp64")
    assert np.array_equal(gd.view(np.uint64), again.view(np.uint64))
    det, st_det = _run(rt, tree, src, nside, _dev(g), "fp64", policy=3)  # deterministic: the gather
    assert st_det["gathered"] == 1 and np.array_equal(gd.view(np.uint64), det.view(np.uint64))
    sc, st_sc = _run(rt, tree, src, nside, _dev(g), "fp64", policy=1)
    assert st_sc["gathered"] == 0 and st_sc["segments"] == st["segments"] and st_sc["rays"] == st["rays"]
    _bound_check(gd, sc, mag, 2e-12)
    # F32-Kahan: FP32 gradient of the columns, FP32 segment lengths
    g32 = g.astype(np.float32)
    refk = oracle.adjoint(keys, lev, S, src_h, dirs, g32.astype(np.float64))
    magk = oracle.adjoint(keys, lev, S, src_h, dirs, np.abs(g32.astype(np.float64)))
    gk, stk = _run(rt, tree, src, nside, _dev(g32), "f32k")
    assert stk["gathered"] == 1 and stk["segments"] == st["segments"]
    _bound_check(gk, refk, magk, 1e-5)
    gk2, _ = _run(rt, tree, src, nside, _dev(g32), "f32k")
    assert np.array_equal(gk.view(np.uint64), gk2.view(np.uint64))
    # the forward walk counts the same segments
    tree.reset_stats()
    rt.trace_columns(tree, src, nside, _dev(np.ones((keys.shape[0], 1), dtype=np.float32)), "f32k")
    assert tree.stats()["segments"] == st["segments"]
    tree.close()


@pytest.mark.parametrize("fine", [0, 1])
def test_gather_common_offset_not_centre(rt, fine):
    """Every source at the same off-centre offset in its leaf, on the depth-21
    lattice (fine 0) or between its points (fine 1, a non-zero sub-lattice
    fraction); the offsets are dyadic, so every sum is exact: the gather still
    applies."""
    rng = np.random.default_rng(951 + fine)
    keys, lev = uniform_octree(4)
    h = 2.0 ** -4
    off = np.array([7 / 32, -11 / 32, 3 / 64]) * h + fine * np.array([3, 5, -7]) * 2.0 ** -40
    src_h = _centres(keys, lev) + off
    dirs = oracle.healpix(2)
    g = rng.random((src_h.shape[0], dirs.shape[0], 1))
    tree = rt.Octree(_dev(keys), _dev(lev))
    ref = oracle.adjoint(keys, lev, 1, src_h, dirs, g)
    for mode, rtol in (("fp64", 1e-12), ("f32k", 1e-5)):
        gin = g if mode == "fp64" else g.astype(np.float32)
        gd, st = _run(rt, tree, _dev(src_h), 2, _dev(gin), mode)
        assert st["gathered"] == 1
        want = ref if mode == "fp64" else oracle.adjoint(keys, lev, 1, src_h, dirs, gin.astype(np.float64))
        _bound_check(gd, want, want, rtol)  # g >= 0: the bound is relative
    tree.close()


@pytest.mark.parametrize("how", ["one_moved", "permuted", "fewer"])
def test_gather_falls_back_to_scatter(rt, how):
    rng = np.random.default_rng(960)
    keys, lev = uniform_octree(3)
    src_h = _centres(keys, lev)
    if how == "one_moved":
        src_h[37, 1] += 0.1 * 2.0 ** -3
    elif how == "permuted":
        src_h = src_h[rng.permutation(src_h.shape[0])]
    else:
        src_h = src_h[:-1]
    dirs = oracle.healpix(1)
    g = rng.standard_normal((src_h.shape[0], 12, 2))
    tree = rt.Octree(_dev(keys), _dev(lev))
    ref = oracle.adjoint(keys, lev, 2, src_h, dirs, g)
    mag = oracle.adjoint(keys, lev, 2, src_h, dirs, np.abs(g))
    gd, st = _run(rt, tree, _dev(src_h), 1, _dev(g), "fp64")
    assert st["gathered"] == 0
    _bound_check(gd, ref, mag, 1e-12)
    # deterministic: the ordered sum over a record, the same bits twice
    d1, _ = _run(rt, tree, _dev(src_h), 1, _dev(g), "fp64", policy=3)
    d2, _ = _run(rt, tree, _dev(src_h), 1, _dev(g), "fp64", policy=3)
    _bound_check(d1, ref, mag, 1e-12)
    assert np.array_equal(d1.view(np.uint64), d2.view(np.uint64))
    tree.close()


def test_gather_accumulates_into_grad(rt):
    """grad_dens is accumulated into, as for the scatter (each direction's sum
    is added in turn, so the result equals base + once up to rounding)."""
    import torch
    rng = np.random.default_rng(970)
    keys, lev = uniform_octree(3)
    src = _dev(_centres(keys, lev))
    g = _dev(rng.random((keys.shape[0], 12, 1)))
    tree = rt.Octree(_dev(keys), _dev(lev))
    once = rt.trace_columns_adjoint(tree, src, 1, g, "fp64")
    base = torch.from_numpy(rng.random((keys.shape[0], 1))).cuda()
    acc = rt.trace_columns_adjoint(tree, src, 1, g, "fp64", grad_dens=base.clone())
    torch.testing.assert_close(acc, base + once, rtol=1e-14, atol=0)
    tree.close()


@pytest.mark.parametrize("level", [0, 1])
def test_gather_smallest_cubes(rt, level):
    """A single leaf (level 0) and a 2^3 cube: the shortest tables, a row of
    one or two leaves in a 32-lane warp."""
    rng = np.random.default_rng(980 + level)
    keys, lev = uniform_octree(level)
    src_h = _centres(keys, lev)
    dirs = oracle.healpix(2)
    g = rng.random((src_h.shape[0], dirs.shape[0], 2))
    tree = rt.Octree(_dev(keys), _dev(lev))
    ref = oracle.adjoint(keys, lev, 2, src_h, dirs, g)
    gd, st = _run(rt, tree, _dev(src_h), 2, _dev(g), "fp64")
    assert st["gathered"] == 1
    _bound_check(gd, ref, ref, 1e-12)
    gk, st = _run(rt, tree, _dev(src_h), 2, _dev(g.astype(np.float32)), "f32k")
    refk = oracle.adjoint(keys, lev, 2, src_h, dirs, g.astype(np.float32).astype(np.float64))
    _bound_check(gk, refk, refk, 1e-5)
    tree.close()
