"""rt_trace_columns_noalloc, the forward trace for callers that cannot allocate
device memory (for example an application whose own pool owns all device
memory, or code that must not call cudaMalloc/cudaFree because they can
synchronize the device), must give what rt_trace_columns gives.

It is called through the C ABI twice in a row on the same inputs, since every
call reuses one static scratch array; each output is compared with the
handle-based entry point's within the tolerance of the other parity tests
(F32-Kahan: 1e-5 relative + 1e-30; FP64: bitwise).  The file is named to be
collected last, and it builds all of its own inputs, so it also runs alone.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from tinytrees import leaf_boxes, random_octree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_09882_gb300 as rt
    f = rt._lib.rt_trace_columns_noalloc
    P = C.c_void_p
    f.argtypes = [P, P, C.c_int64, P, C.c_int, P, C.c_int64, C.c_int, P, C.c_int, C.c_int, C.c_int, P,
                  C.POINTER(rt.Stats), P]
    return rt


def _dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def _noalloc(rt, keys, lev, max_level, src, nside, dens, mode, extent=None, stats=False):
    import torch
    nd = 12 * nside * nside
    S = dens.shape[1]
    odt = torch.float32 if mode == rt.MODE_F32_KAHAN else torch.float64
    out = torch.full((src.shape[0], nd, S), float("nan"), dtype=odt, device="cuda")
    ext = None if extent is None else (C.c_int32 * 3)(*extent)
    st = rt.Stats()
    code = rt._lib.rt_trace_columns_noalloc(
        keys.data_ptr(), lev.data_ptr(), keys.numel(), ext, max_level, src.data_ptr(), src.shape[0],
        nside, dens.data_ptr(), S, rt.F64 if dens.dtype == torch.float64 else rt.F32, mode,
        out.data_ptr(), C.byref(st), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, rt._lib.rt_last_error()
    assert st.status == 0 and st.rays == src.shape[0] * nd
    return out.cpu().numpy(), (st if stats else st.segments)


def _compare(rt, keys_h, lev_h, dens_h, src_h, nside, extent=None):
    keys, lev, dens, src = _dev(keys_h), _dev(lev_h), _dev(dens_h), _dev(src_h)
    tree = rt.Octree(keys, lev, extent=extent)
    for mode in (rt.MODE_F32_KAHAN, rt.MODE_FP64):
        tree.reset_stats()
        ref = rt.trace_columns(tree, src, nside, dens, mode).cpu().numpy()
        ref_segs = tree.stats()["segments"]
        for call in range(2):
            got, segs = _noalloc(rt, keys, lev, int(lev_h.max()), src, nside, dens, mode, extent)
            assert segs == ref_segs, (mode, call)
            if mode == rt.MODE_FP64:
                np.testing.assert_array_equal(got, ref)
            else:
                d = np.abs(got.astype(np.float64) - ref)
                assert np.all(d <= 1e-5 * np.abs(ref) + 1e-30), (call, float(d.max()))
    tree.close()


def test_noalloc_matches_handle_entry_point_amr(rt):
    rng = np.random.default_rng(808)
    keys, lev, _ = random_octree(rng, 1, 7, 0.35)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 4)).astype(np.float32)
    lo, hi = leaf_boxes(keys, lev)
    src = np.concatenate([rng.random((300, 3)), 0.5 * (lo + hi)[::5]])
    _compare(rt, keys, lev, dens, src, 2)


def test_noalloc_matches_handle_entry_point_uniform(rt):
    cloud = synth.uniform_cloud(5, 2.0, 9, fracs=synth.SPECIES_FRACTIONS, dtype=np.float32)
    _compare(rt, cloud.keys, cloud.levels, cloud.dens, synth.leaf_centres(cloud), 1)


def test_paired_and_single_walks_are_bitwise_equal(rt):
    """On a uniform cube with FP32 densities the handle call walks two rays
    per lane (leaf centres share their exit sequences) and the allocation-free
    call one: their F32-Kahan columns and segment counts must be bitwise
    equal.  Sources: leaf centres (pairs), off-lattice points (single walks),
    the two interleaved so that pairs mix, and a count that leaves a ragged
    64-source block; 1, 2, 4 and 8 species."""
    import torch
    rng = np.random.default_rng(811)
    for S in (1, 2, 4, 8):
        cloud = synth.uniform_cloud(4, 2.0, 12 + S, fracs=tuple(np.linspace(1.0, 0.3, S)), dtype=np.float32)
        centres = synth.leaf_centres(cloud)
        off = rng.random((centres.shape[0], 3))
        mixed = np.where(rng.random((centres.shape[0], 1)) < 0.5, centres, off)
        src = np.concatenate([centres[:1000], off[:200], mixed[:500], centres[1000:1037]])
        keys, lev, dens, s_d = _dev(cloud.keys), _dev(cloud.levels), _dev(cloud.dens), _dev(src)
        tree = rt.Octree(keys, lev)
        tree.reset_stats()
        ref = rt.trace_columns(tree, s_d, 2, dens, rt.MODE_F32_KAHAN).cpu().numpy()
        ref_st = tree.stats()
        got, st = _noalloc(rt, keys, lev, int(cloud.levels.max()), s_d, 2, dens, rt.MODE_F32_KAHAN, stats=True)
        assert (st.segments, st.exit_fallbacks) == (ref_st["segments"], ref_st["exit_fallbacks"]), S
        np.testing.assert_array_equal(got, ref, err_msg=f"S={S}")
        tree.close()


def test_noalloc_largest_direction_table(rt):
    """nside 8, the largest table the fixed scratch holds (768 directions), on a
    small AMR tree."""
    rng = np.random.default_rng(809)
    keys, lev, _ = random_octree(rng, 1, 5, 0.35)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 2)).astype(np.float32)
    lo, hi = leaf_boxes(keys, lev)
    src = np.concatenate([rng.random((40, 3)), 0.5 * (lo + hi)[::9]])
    _compare(rt, keys, lev, dens, src, 8)
    _compare(rt, keys, lev, dens, src[:20], 8)  # fewer sources than a warp: source-major ray order


def test_noalloc_box_extent_and_fp64_densities(rt):
    """A box that is not a power of two (extent argument) with FP64 densities."""
    rng = np.random.default_rng(810)
    keys, lev, ext = random_octree(rng, 3, 5, 0.3, extent_cells=5)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 3))
    lo, hi = leaf_boxes(keys, lev)
    box = ext[0] * 2.0 ** -21
    src = np.concatenate([rng.random((200, 3)) * box, 0.5 * (lo + hi)[::4]])
    _compare(rt, keys, lev, dens, src, 2, extent=ext)


def test_noalloc_rejects_oversized_direction_table(rt):
    import torch
    keys = _dev(np.array([0], dtype=np.uint64))
    lev = _dev(np.array([0], dtype=np.uint8))
    src = torch.full((1, 3), 0.5, dtype=torch.float64, device="cuda")
    dens = torch.ones((1, 1), dtype=torch.float32, device="cuda")
    out = torch.empty((1, 12 * 256, 1), dtype=torch.float32, device="cuda")
    code = rt._lib.rt_trace_columns_noalloc(keys.data_ptr(), lev.data_ptr(), 1, None, 0, src.data_ptr(), 1,
                                            16, dens.data_ptr(), 1, rt.F32, rt.MODE_F32_KAHAN,
                                            out.data_ptr(), None, None)
    assert code == 1 and b"nside" in rt._lib.rt_last_error()
