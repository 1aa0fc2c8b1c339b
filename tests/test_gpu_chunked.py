"""Chunked contribution grid (Alg. 1): the leaves split into Morton-range
chunks traced one at a time, densities streamed from host memory (or read in
place), every ray's walk carried from chunk to chunk.

Bars: columns bit for bit those of rt_trace_columns in both modes (the same
walk, the same order of additions), path fingerprints equal to rt_trace_paths',
the oracle's columns on sampled sources (F32-Kahan 1e-5 relative, FP64
bitwise); a source outside the cloud (mask 0) gets zero columns."""
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


def _same(a, b):
    import torch
    return bool(torch.equal(a.view(torch.int64) if a.dtype == torch.float64 else a.view(torch.int32),
                            b.view(torch.int64) if b.dtype == torch.float64 else b.view(torch.int32)))


@pytest.mark.parametrize("seed,n_chunks", [(0, 1), (1, 3), (2, 7), (3, -1)])
def test_chunked_small_trees(rt, seed, n_chunks):
    """Random octrees (one in a box that is not a power of two), sources on and
    off the leaf lattice, Nside 1 and 2; n_chunks -1 makes every leaf its own
    chunk."""
    import torch
    rng = np.random.default_rng(1200 + seed)
    ext = None
    if seed == 2:
        keys, lev, ext = random_octree(rng, 3, 6, 0.3, extent_cells=5)
    else:
        keys, lev, _ = random_octree(rng, 1, 5, 0.4)
    box = 1.0 if ext is None else ext[0] * 2.0 ** -21
    lo, hi = leaf_boxes(keys, lev)
    src = np.concatenate([rng.random((150, 3)) * box, 0.5 * (lo + hi)[::3]])
    S = 1 + seed % 4
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], S))
    tree = rt.Octree(_dev(keys), _dev(lev), extent=ext)
    nc = keys.shape[0] if n_chunks < 0 else n_chunks
    for nside in (1, 2):
        dirs = oracle.healpix(nside)
        want, h_or, n_or = oracle.trace(keys, lev, dens, src, dirs, extent=ext)
        for mode, dt in (("fp64", np.float64), ("f32k", np.float32)):
            d_host = torch.from_numpy(dens.astype(dt)).pin_memory()
            ref = rt.trace_columns(tree, _dev(src), nside, d_host.cuda(), mode)
            got, nseg, hsh = rt.trace_columns_chunked(tree, _dev(src), nside, d_host, nc, mode, paths=True)
            assert _same(got, ref), (mode, nside)
            np.testing.assert_array_equal(nseg.cpu().numpy().astype(np.uint64), n_or)
            np.testing.assert_array_equal(hsh.cpu().numpy().view(np.uint64), h_or)
            g = got.double().cpu().numpy()
            if mode == "fp64":
                np.testing.assert_array_equal(g, want)
            else:
                assert np.all(np.abs(g - want) <= 1e-5 * np.abs(want) + 1e-30)
            assert tree.stats()["status"] == 0
    tree.close()


def test_chunked_source_mask(rt):
    import torch
    rng = np.random.default_rng(1300)
    keys, lev, _ = random_octree(rng, 2, 5, 0.3)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 2)).astype(np.float32)
    lo, hi = leaf_boxes(keys, lev)
    src = 0.5 * (lo + hi)
    # "inside the cloud": the density of the source's own leaf (its first
    # species) at or above the median
    inside = dens[:, 0] >= np.median(dens[:, 0])
    tree = rt.Octree(_dev(keys), _dev(lev))
    got, nseg, _ = rt.trace_columns_chunked(tree, _dev(src), 2, _dev(dens), 4, "f32k",
                                            mask=torch.from_numpy(inside).cuda(), paths=True)
    g = got.double().cpu().numpy()
    assert np.all(g[~inside] == 0.0) and np.all(nseg.cpu().numpy()[~inside] == 0)
    want, _, _ = oracle.trace(keys, lev, dens.astype(np.float64), src[inside], oracle.healpix(2))
    assert np.all(np.abs(g[inside] - want) <= 1e-5 * np.abs(want) + 1e-30)
    st = tree.stats()
    assert st["status"] == 0 and st["rays"] == int(inside.sum()) * 48
    tree.close()


@pytest.mark.parametrize("n_chunks", [2, 8])
def test_chunked_amr128(rt, n_chunks):
    """The 128^3-base AMR workload (4.7M leaves, 1M mass-weighted sources, Nside
    2, 4 FP32 species) split into 2 and 8 chunks, densities streamed from
    page-locked host memory: bitwise equal to the unchunked trace in both
    modes, paths equal, 200 sources against the oracle."""
    import torch
    from synth import torchgen
    keys, lev, dens, ntot, ext = torchgen.amr_cloud(128, 2, 90.0, 1.5, 2, device="cuda")
    src = torchgen.mass_weighted_sources(keys, lev, ntot, 1_000_000, 102)
    tree = rt.Octree(keys, lev, extent=ext)
    d_host = dens.cpu().pin_memory()
    rng = np.random.default_rng(1400 + n_chunks)
    idx = np.sort(rng.choice(src.shape[0], size=200, replace=False))
    want, h_or, n_or = oracle.trace(keys.cpu().numpy().view(np.uint64), lev.cpu().numpy(),
                                    dens.cpu().numpy().astype(np.float64), src[torch.from_numpy(idx).cuda()].cpu().numpy(),
                                    oracle.healpix(2), extent=ext)
    sel = torch.from_numpy(idx).cuda()
    for mode in ("f32k", "fp64"):
        ref = rt.trace_columns(tree, src, 2, dens, mode)
        nref, href = rt.trace_paths(tree, src, 2, mode)
        tree.reset_stats()
        got, nseg, hsh = rt.trace_columns_chunked(tree, src, 2, d_host, n_chunks, mode, paths=True)
        st = tree.stats()
        assert st["status"] == 0 and st["segments"] == int(nref.sum(dtype=torch.int64))
        assert _same(got, ref), mode
        assert torch.equal(nseg, nref) and torch.equal(hsh, href)
        g = got[sel].double().cpu().numpy()
        if mode == "fp64":
            np.testing.assert_array_equal(g, want)
        else:
            assert np.all(np.abs(g - want) <= 1e-5 * np.abs(want) + 1e-30)
        del ref, got, nseg, hsh, nref, href
    tree.close()


def test_chunked_empty_and_all_masked(rt):
    import torch
    rng = np.random.default_rng(1310)
    keys, lev, _ = random_octree(rng, 1, 4, 0.4)
    dens = _dev(rng.uniform(0.1, 2.0, size=(keys.shape[0], 4)).astype(np.float32))
    tree = rt.Octree(_dev(keys), _dev(lev))
    none = rt.trace_columns_chunked(tree, _dev(np.zeros((0, 3))), 1, dens, 3, "f32k")
    assert none.shape == (0, 12, 4)
    src = _dev(rng.random((50, 3)))
    got, nseg, hsh = rt.trace_columns_chunked(tree, src, 1, dens, 3, "f32k",
                                              mask=torch.zeros(50, dtype=torch.uint8, device="cuda"), paths=True)
    assert torch.count_nonzero(got) == 0 and torch.count_nonzero(nseg) == 0 and torch.count_nonzero(hsh) == 0
    with pytest.raises(rt.RTError):
        rt.trace_columns_chunked(tree, src, 1, dens, keys.shape[0] + 1, "f32k")  # more chunks than leaves
    tree.close()
