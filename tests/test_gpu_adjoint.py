"""GPU adjoint: against the oracle's FP64 gradient, the dot-product identity
<g, A n> = <A^T g, n>, central finite differences of an attenuation loss, and
the torch.autograd.Function wrapper.

Bars against the oracle, per leaf j, with mag = A^T |g| (the oracle's adjoint
of |g|, the sum of the magnitudes of the terms of grad_j):
- FP64: |got - ref| <= 1e-12 mag (the products are rounded once and any
  summation order of n terms is within (n - 1) 2^-53 mag);
- F32-Kahan: |got - ref| <= 1e-5 mag + 1e-11 max|g|.  Each segment length is
  the FP32 rounding of a double-float time difference: relative error 2^-24
  plus an absolute error below 2^-40 box lengths, which matters only for the
  near-tie slivers a ray cuts through a cell corner; the first term bounds the
  relative part (a few 2^-24 with the FP32 product and the compensated sum),
  the second the slivers, a few dozen per leaf at most.
A leaf entered through a sliver whose exit time rounds one ulp below the
previous exit gets a segment of about -1e-17 on both sides (the definition's
clamp of the non-stepped axes into the current leaf), so mag is taken as |mag|."""
import numpy as np
import pytest

import oracle
import synth
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


# mag may be a few 1e-17 below zero at a leaf the walk enters through a
# one-ulp sliver of negative length (see the readings of the definition), hence |mag|.
def _check_fp64(got, ref, mag):
    d = np.abs(got - ref)
    mag = np.abs(mag)
    assert np.all(d <= 1e-12 * mag + 1e-30), float((d / np.maximum(mag, 1e-300)).max())


def _check_f32k(got, ref, mag, g):
    d = np.abs(got - ref)
    mag = np.abs(mag)
    assert np.all(d <= 1e-5 * mag + 1e-11 * np.abs(g).max()), float((d / np.maximum(mag, 1e-300)).max())


@pytest.mark.parametrize("seed", range(4))
def test_adjoint_matches_oracle(rt, seed):
    rng = np.random.default_rng(300 + seed)
    keys, lev, _ = random_octree(rng, 1, 6, 0.4)
    S = 1 + seed % 3
    src = np.concatenate([rng.random((150, 3)), synth.leaf_centres(
        synth.Cloud(keys, lev, np.zeros((keys.shape[0], 1)), (1 << 21,) * 3))[:50]])
    nside = 1 + (seed % 2)
    dirs = oracle.healpix(nside)
    g = rng.standard_normal((src.shape[0], dirs.shape[0], S))
    ref = oracle.adjoint(keys, lev, S, src, dirs, g)
    mag = oracle.adjoint(keys, lev, S, src, dirs, np.abs(g))
    tree = rt.Octree(_dev(keys), _dev(lev))
    gd = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g), "fp64").cpu().numpy()
    _check_fp64(gd, ref, mag)
    g32 = g.astype(np.float32).astype(np.float64)
    gk = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g.astype(np.float32)), "f32k").cpu().numpy()
    refk = oracle.adjoint(keys, lev, S, src, dirs, g32)
    _check_f32k(gk, refk, oracle.adjoint(keys, lev, S, src, dirs, np.abs(g32)), g32)
    assert tree.stats()["status"] == 0
    tree.close()


@pytest.mark.parametrize("S", [1, 4])
def test_uniform_grid_adjoint_matches_oracle(rt, S):
    """The uniform-grid walks (the 512^3 bench's adjoint path): leaf centres,
    which take the x/y-locked and zero-fraction forms, and off-lattice
    sources, Nside 1 and 2."""
    from tinytrees import uniform_octree
    rng = np.random.default_rng(400 + S)
    keys, lev = uniform_octree(4)
    cloud = synth.Cloud(keys, lev, np.zeros((keys.shape[0], 1)), (1 << 21,) * 3)
    src = np.concatenate([synth.leaf_centres(cloud)[::7], rng.random((100, 3))])
    tree = rt.Octree(_dev(keys), _dev(lev))
    for nside in (1, 2):
        dirs = oracle.healpix(nside)
        g = rng.standard_normal((src.shape[0], dirs.shape[0], S))
        ref = oracle.adjoint(keys, lev, S, src, dirs, g)
        mag = oracle.adjoint(keys, lev, S, src, dirs, np.abs(g))
        gd = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g), "fp64").cpu().numpy()
        _check_fp64(gd, ref, mag)
        g32 = g.astype(np.float32)
        gk = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g32), "f32k").cpu().numpy()
        g64 = g32.astype(np.float64)
        refk = oracle.adjoint(keys, lev, S, src, dirs, g64)
        _check_f32k(gk, refk, oracle.adjoint(keys, lev, S, src, dirs, np.abs(g64)), g64)
    assert tree.stats()["status"] == 0
    tree.close()


@pytest.mark.parametrize("policy", [0, 2, 3])
def test_c4_adjoint_matches_oracle(rt, policy):
    """The differentiable workload itself (64^3 base refined once above p85,
    537,398 leaves, one species, Nside 2) on 3000 random leaf-centre sources,
    the same on both sides, with gradients of both signs; recomputed paths
    (policy 0, the scatter on a general octree), a recorded path (policy 2)
    and the deterministic form (policy 3: an ordered sum over a record, the
    same bits on a second call)."""
    cloud, src_all, nside = synth.workload_amr64_grad()
    rng = np.random.default_rng(44)
    src = src_all[np.sort(rng.choice(src_all.shape[0], size=3000, replace=False))]
    dirs = oracle.healpix(nside)
    g = rng.standard_normal((src.shape[0], dirs.shape[0], 1))
    tree = rt.Octree(_dev(cloud.keys), _dev(cloud.levels))
    ref = oracle.adjoint(cloud.keys, cloud.levels, 1, src, dirs, g)
    mag = oracle.adjoint(cloud.keys, cloud.levels, 1, src, dirs, np.abs(g))
    gd = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g), "fp64", path_policy=policy).cpu().numpy()
    _check_fp64(gd, ref, mag)
    g32 = g.astype(np.float32).astype(np.float64)
    refk = oracle.adjoint(cloud.keys, cloud.levels, 1, src, dirs, g32)
    magk = oracle.adjoint(cloud.keys, cloud.levels, 1, src, dirs, np.abs(g32))
    gk = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g.astype(np.float32)), "f32k",
                                  path_policy=policy).cpu().numpy()
    _check_f32k(gk, refk, magk, g32)
    if policy == 3:
        again = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g.astype(np.float32)), "f32k",
                                         path_policy=3).cpu().numpy()
        assert np.array_equal(gk.view(np.uint64), again.view(np.uint64))
        gd2 = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g), "fp64", path_policy=3).cpu().numpy()
        assert np.array_equal(gd.view(np.uint64), gd2.view(np.uint64))
    touched = mag[:, 0] > 0
    rel = np.abs(gk - refk)[touched, 0] / mag[touched, 0]
    print("policy", policy, "leaves touched", int(touched.sum()), "f32k max rel (of mag)", float(rel.max()))
    assert tree.stats()["status"] == 0
    tree.close()


def test_dot_product_identity(rt):
    import torch
    rng = np.random.default_rng(11)
    cloud, src, nside = synth.workload_amr64_grad()
    sel = rng.choice(src.shape[0], size=4000, replace=False)
    s = _dev(src[sel])
    tree = rt.Octree(_dev(cloud.keys), _dev(cloud.levels))
    n = torch.from_numpy(rng.random((cloud.n_leaves, 1))).cuda()
    g = torch.from_numpy(rng.standard_normal((4000, 48, 1))).cuda()
    cols = rt.trace_columns(tree, s, nside, n, "fp64")
    grad = rt.trace_columns_adjoint(tree, s, nside, g, "fp64")
    lhs = float((g * cols).sum())
    rhs = float((grad * n).sum())
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    tree.close()


def _loss_parts(cols, alpha, w):
    import torch
    av = cols[..., 0] * (alpha / 1.6e21)
    return w * torch.exp(-2.5 * av)


def test_finite_differences_attenuation_loss(rt):
    """64^3 base refined once above p85, one species, all leaf centres, Nside 2.
    A_V = alpha N / 1.6e21 with alpha giving mean A_V = 5; loss =
    sum w exp(-2.5 A_V), w ~ U[0, 1].  dLoss/dn from the adjoint (F32-Kahan
    walk) against central differences (step 1e-4 n_j, FP64 forward) on 200
    random leaves: relative error <= 1e-4."""
    import torch
    cloud, src, nside = synth.workload_amr64_grad()
    rng = np.random.default_rng(4)
    tree = rt.Octree(_dev(cloud.keys), _dev(cloud.levels))
    s = _dev(src)
    n = torch.from_numpy(cloud.dens.astype(np.float64)).cuda()
    cols = rt.trace_columns(tree, s, nside, n, "fp64")
    alpha = 5.0 * 1.6e21 / float(cols.mean())
    w = torch.from_numpy(rng.random((src.shape[0], 48))).cuda()
    # gradient of the loss w.r.t. the columns, then the adjoint trace
    av = cols[..., 0] * (alpha / 1.6e21)
    gcol = (w * (-2.5 * alpha / 1.6e21) * torch.exp(-2.5 * av))[..., None]
    grad = rt.trace_columns_adjoint(tree, s, nside, gcol, "f32k")[:, 0].cpu().numpy()
    leaves = rng.choice(cloud.n_leaves, size=200, replace=False)
    out_p = torch.empty_like(cols)
    out_m = torch.empty_like(cols)
    rel = []
    for j in leaves:
        nj = float(n[j, 0])
        h = 1e-4 * nj
        n[j, 0] = nj + h
        rt.trace_columns(tree, s, nside, n, "fp64", out=out_p)
        n[j, 0] = nj - h
        rt.trace_columns(tree, s, nside, n, "fp64", out=out_m)
        n[j, 0] = nj
        dl = float((_loss_parts(out_p, alpha, w) - _loss_parts(out_m, alpha, w)).sum())
        fd = dl / (2 * h)
        rel.append(abs(grad[j] - fd) / max(abs(fd), 1e-300))
    rel = np.array(rel)
    assert tree.stats()["status"] == 0
    assert rel.max() <= 1e-4, (rel.max(), np.median(rel))
    tree.close()


def test_autograd_function(rt):
    import torch
    rng = np.random.default_rng(21)
    keys, lev, _ = random_octree(rng, 1, 5, 0.4)
    tree = rt.Octree(_dev(keys), _dev(lev))
    src = _dev(rng.random((64, 3)))
    dens = torch.from_numpy(rng.random((keys.shape[0], 2))).float().cuda().requires_grad_(True)
    cols = rt.Columns.apply(dens, tree, src, 2, "f32k")
    w = torch.from_numpy(rng.random(cols.shape)).float().cuda()
    (w * cols).sum().backward()
    # the same step from a path record: the same columns and gradient
    paths = rt.Paths(tree, src, 2, "f32k")
    dens2 = dens.detach().clone().requires_grad_(True)
    cols2 = rt.Columns.apply(dens2, tree, src, 2, "f32k", paths)
    assert torch.equal(cols2, cols)
    (w * cols2).sum().backward()
    torch.testing.assert_close(dens2.grad, dens.grad, rtol=1e-6, atol=0)
    paths.close()
    g = oracle.adjoint(keys, lev, 2, rng.random((0, 3)), oracle.healpix(2), np.zeros((0, 48, 2)))
    ref = oracle.adjoint(keys, lev, 2, src.cpu().numpy(), oracle.healpix(2),
                         w.cpu().numpy().astype(np.float64))
    assert g.shape == ref.shape
    # w >= 0, so A^T |w| = ref: the F32-Kahan bar is relative (the float32 cast
    # of the gradient adds 2^-24)
    _check_f32k(dens.grad.cpu().numpy().astype(np.float64), ref, ref, w.cpu().numpy())
    tree.close()
