"""GPU adjoint: against the oracle's FP64 gradient, the dot-product identity
<g, A n> = <A^T g, n>, central finite differences of an attenuation loss, and
the torch.autograd.Function wrapper."""
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
    tree = rt.Octree(_dev(keys), _dev(lev))
    gd = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g), "fp64").cpu().numpy()
    scale = np.abs(ref).max()
    np.testing.assert_allclose(gd, ref, rtol=1e-12, atol=1e-13 * scale)
    gk = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g.astype(np.float32)), "f32k").cpu().numpy()
    refk = oracle.adjoint(keys, lev, S, src, dirs, g.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(gk, refk, rtol=2e-6, atol=1e-6 * scale)
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
        scale = np.abs(ref).max()
        gd = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g), "fp64").cpu().numpy()
        np.testing.assert_allclose(gd, ref, rtol=1e-12, atol=1e-13 * scale)
        g32 = g.astype(np.float32)
        gk = rt.trace_columns_adjoint(tree, _dev(src), nside, _dev(g32), "f32k").cpu().numpy()
        refk = oracle.adjoint(keys, lev, S, src, dirs, g32.astype(np.float64))
        np.testing.assert_allclose(gk, refk, rtol=2e-6, atol=1e-6 * scale)
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
    g = oracle.adjoint(keys, lev, 2, rng.random((0, 3)), oracle.healpix(2), np.zeros((0, 48, 2)))
    ref = oracle.adjoint(keys, lev, 2, src.cpu().numpy(), oracle.healpix(2),
                         w.cpu().numpy().astype(np.float64))
    assert g.shape == ref.shape
    np.testing.assert_allclose(dens.grad.cpu().numpy(), ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())
    tree.close()
