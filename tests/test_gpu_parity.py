"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.

Bars (from the method's targets): visited-leaf sequences bit-exact (segment
count and 64-bit path hash per ray) in both modes; FP64-mode columns bitwise
equal to the oracle's; F32-Kahan columns within |d| <= 1e-5 |ref| + 1e-30.
"""
import numpy as np
import pytest

import oracle
import synth
from tinytrees import leaf_boxes, random_octree, uniform_octree

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-5, 1e-30


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


def _col_err(got, want):
    d = np.abs(got.astype(np.float64) - want)
    ok = d <= RTOL * np.abs(want) + ATOL
    rel = d / np.maximum(np.abs(want), 1e-300)
    return ok, rel


def _check_case(rt, keys, lev, dens, src, nside, extent=None, modes=("f32k", "fp64"),
                force_table=False, label=""):
    dirs = oracle.healpix(nside)
    want, h_or, n_or = oracle.trace(keys, lev, np.asarray(dens, dtype=np.float64), src, dirs, extent=extent)
    tree = rt.Octree(_dev(keys), _dev(lev), extent=extent)
    if force_table:
        tree.set_lookup(False)
    s_d = _dev(src)
    d_d = _dev(dens)
    for mode in modes:
        tree.reset_stats()
        cols = rt.trace_columns(tree, s_d, nside, d_d, mode).cpu().numpy()
        nseg, hsh = rt.trace_paths(tree, s_d, nside, mode)
        st = tree.stats()
        assert st["status"] == 0, (label, mode, st)
        np.testing.assert_array_equal(nseg.cpu().numpy().astype(np.uint64), n_or, err_msg=f"{label} {mode} nseg")
        np.testing.assert_array_equal(hsh.cpu().numpy().view(np.uint64), h_or, err_msg=f"{label} {mode} hash")
        if mode == "fp64":
            np.testing.assert_array_equal(cols, want, err_msg=f"{label} fp64 columns")
        else:
            ok, rel = _col_err(cols, want)
            assert ok.all(), (label, float(rel.max()))
        assert st["segments"] == 2 * int(n_or.sum()), (label, mode, st)  # columns + paths calls
    tree.close()
    return want


# ----------------------------------------------------------------- uniform

@pytest.mark.parametrize("force_table", [False, True])
def test_uniform32_all_centres(rt, force_table):
    """32^3 uniform grid, one FP64 species, every leaf centre, Nside 1."""
    cloud, src, nside = synth.workload_uniform32()
    _check_case(rt, cloud.keys, cloud.levels, cloud.dens, src, nside, force_table=force_table,
                label="uniform32")


def test_uniform_multi_species_f32(rt):
    cloud = synth.uniform_cloud(4, 2.0, 9, fracs=synth.SPECIES_FRACTIONS, dtype=np.float32)
    src = synth.leaf_centres(cloud)
    for nside in (1, 2, 4):
        _check_case(rt, cloud.keys, cloud.levels, cloud.dens, src, nside, label=f"uni16 nside{nside}")


# ------------------------------------------------------------ random trees

def _structured_sources(rng, keys, lev, n_random=64):
    lo, hi = leaf_boxes(keys, lev)
    pick = rng.choice(keys.shape[0], size=min(16, keys.shape[0]), replace=False)
    mid = 0.5 * (lo[pick] + hi[pick])
    pts = [rng.random((n_random, 3)), mid, lo[pick],
           np.column_stack([lo[pick, 0], mid[:, 1], lo[pick, 2]]),
           np.column_stack([mid[:, 0], lo[pick, 1], mid[:, 2]])]
    return np.concatenate(pts)


@pytest.mark.parametrize("seed", range(8))
def test_random_octrees_structured_sources(rt, seed):
    """Random AMR trees with sources at centres, corners, edges and faces
    (exact and near ties), Nside 1, 2 and 4, S = 3."""
    rng = np.random.default_rng(1000 + seed)
    keys, lev, _ = random_octree(rng, 1, 5, 0.45)
    dens = rng.uniform(0.01, 100.0, size=(keys.shape[0], 3)).astype(np.float32)
    src = _structured_sources(rng, keys, lev)
    for nside in (1, 2, 4):
        _check_case(rt, keys, lev, dens, src, nside, label=f"rand{seed} nside{nside}")


@pytest.mark.parametrize("seed", range(3))
def test_non_power_of_two_extent(rt, seed):
    rng = np.random.default_rng(2000 + seed)
    keys, lev, ext = random_octree(rng, 3, 6, 0.3, extent_cells=5 + seed)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 2)).astype(np.float32)
    lo, hi = leaf_boxes(keys, lev)
    src = np.concatenate([0.5 * (lo + hi), lo[::7]])
    _check_case(rt, keys, lev, dens, src, 2, extent=ext, label=f"ext{seed}")


def test_deep_levels_and_species_counts(rt):
    """Leaves down to level 12 and S from 1 to 8 (vector and scalar loads)."""
    rng = np.random.default_rng(77)
    keys, lev, _ = random_octree(rng, 2, 12, 0.12)
    src = _structured_sources(rng, keys, lev, n_random=32)
    for S in (1, 2, 4, 5, 8):
        dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], S)).astype(np.float32)
        _check_case(rt, keys, lev, dens, src, 1, label=f"deep S{S}")


def test_fp64_densities_in_f32k_mode(rt):
    rng = np.random.default_rng(78)
    keys, lev, _ = random_octree(rng, 1, 6, 0.4)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 2))
    src = rng.random((200, 3))
    _check_case(rt, keys, lev, dens, src, 2, label="f64dens")


# ------------------------------------------------------------ AMR workload

def test_amr128_sampled_sources(rt):
    """128^3 base, two refinement levels above p90 (about 4.7M leaves), 4 FP32
    species, mass-weighted sources (a sample of 20000), Nside 2."""
    cloud, src, nside = synth.workload_amr128(n_src=20000)
    want = _check_case(rt, cloud.keys, cloud.levels, cloud.dens, src, nside, modes=("f32k",),
                       label="amr128")
    assert cloud.n_leaves > 4_000_000
    assert np.all(want >= 0)


# ------------------------------------------------------------------ faults

def test_source_outside_sets_status_and_zeros(rt):
    import torch
    keys, lev = uniform_octree(3)
    tree = rt.Octree(_dev(keys), _dev(lev))
    dens = torch.ones((keys.shape[0], 1), dtype=torch.float32, device="cuda")
    src = torch.tensor([[0.5, 0.5, 0.5], [1.0, 0.5, 0.5], [0.2, float("nan"), 0.1],
                        [0.3, 0.3, -5e-324], [float("inf"), 0.1, 0.1], [0.1, -float("inf"), 0.1],
                        [0.1, 0.1, float(np.nextafter(1.0, 2.0))], [-1e-300, 0.5, 0.5]],
                       dtype=torch.float64, device="cuda")
    for mode in ("f32k", "fp64"):
        tree.reset_stats()
        cols = rt.trace_columns(tree, src, 1, dens, mode).cpu().numpy()
        st = tree.stats()
        assert st["status"] == 5 and st["fault_ray"] >= 12
        assert np.all(cols[1:] == 0) and np.all(cols[0] > 0)
    tree.close()


def test_step_cap_stops_rays_with_status(rt):
    import torch
    keys, lev = uniform_octree(4)
    tree = rt.Octree(_dev(keys), _dev(lev))
    tree.set_step_cap(3)
    dens = torch.ones((keys.shape[0], 1), dtype=torch.float32, device="cuda")
    src = _dev(np.array([[0.03, 0.03, 0.03]]))
    rt.trace_columns(tree, src, 1, dens, "f32k")
    assert tree.stats()["status"] == 6
    tree.set_step_cap(0)
    tree.reset_stats()
    rt.trace_columns(tree, src, 1, dens, "f32k")
    assert tree.stats()["status"] == 0
    tree.close()


def test_step_cap_on_paired_rays(rt):
    """The step cap on the two-rays-per-lane walk: leaf centres of a uniform
    cube (paired), in a full and a ragged 64-source block, with a cap shorter
    than some rays, so that one ray of a pair stops while the other goes on.
    A ray within the cap keeps its columns bit for bit, a longer one stops at
    the cap with zero columns and the step-limit status, and the segment count
    is the sum of min(path length, cap)."""
    keys, lev = uniform_octree(4)
    rng = np.random.default_rng(77)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 4)).astype(np.float32)
    src = synth.leaf_centres(synth.Cloud(keys, lev, np.zeros((keys.shape[0], 1)), (1 << 21,) * 3))[:100]
    _, _, n_or = oracle.trace(keys, lev, dens.astype(np.float64), src, oracle.healpix(1))
    cap = 6
    short = n_or <= cap
    assert short.any() and (~short).any()
    tree = rt.Octree(_dev(keys), _dev(lev))
    d_d, s_d = _dev(dens), _dev(src)
    full = rt.trace_columns(tree, s_d, 1, d_d, "f32k").cpu().numpy()
    tree.set_step_cap(cap)
    tree.reset_stats()
    capped = rt.trace_columns(tree, s_d, 1, d_d, "f32k").cpu().numpy()
    st = tree.stats()
    assert st["status"] == 6, st
    assert st["segments"] == int(np.minimum(n_or, cap).sum()), st
    np.testing.assert_array_equal(capped[short], full[short])
    assert np.all(capped[~short] == 0)
    tree.close()


def test_invalid_octrees_match_oracle_codes(rt):
    rng = np.random.default_rng(3)
    keys, lev, _ = random_octree(rng, 1, 4, 0.4)
    cases = []
    k = keys.copy(); k[[3, 4]] = k[[4, 3]]; cases.append((k, lev, None))
    i = int(np.nonzero(lev < 21)[0][0])
    k = keys.copy(); k[i] += np.uint64(1); cases.append((k, lev, None))
    l2 = lev.copy(); l2[5] = 22; cases.append((keys, l2, None))
    cases.append((np.delete(keys, 7), np.delete(lev, 7), None))
    j = int(np.nonzero(lev == lev.max())[0][0])
    l3 = lev.copy(); l3[j] = lev[j] - 1; cases.append((keys, l3, None))
    cases.append((keys, lev, (1 << 20, 1 << 21, 1 << 21)))
    k = keys.copy(); k[[3, 4]] = k[[4, 3]]; k[i] += np.uint64(1); cases.append((k, lev, None))
    for kk, ll, ext in cases:
        code = oracle.validate(kk, ll, ext)
        assert code != 0
        with pytest.raises(rt.RTError) as e:
            rt.Octree(_dev(kk), _dev(ll), extent=ext)
        assert e.value.code == code


def test_bad_arguments_are_rejected(rt):
    import torch
    keys, lev = uniform_octree(2)
    tree = rt.Octree(_dev(keys), _dev(lev))
    dens = torch.ones((keys.shape[0], 9), dtype=torch.float32, device="cuda")
    src = _dev(np.array([[0.5, 0.5, 0.5]]))
    with pytest.raises(rt.RTError):
        rt.trace_columns(tree, src, 1, dens, "f32k")          # S = 9 > 8
    with pytest.raises(rt.RTError):
        rt.trace_columns(tree, src, 3, dens[:, :1], "f32k")   # nside 3
    out = rt.trace_columns(tree, src[:0], 1, dens[:, :1], "f32k")
    assert out.shape == (0, 12, 1)
    tree.close()


def test_few_sources_many_directions(rt):
    """Angular-convergence shape: a handful of sources at high Nside (the
    source-major ray order, a warp walks 32 directions of one source)."""
    rng = np.random.default_rng(91)
    keys, lev, _ = random_octree(rng, 2, 7, 0.3)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 1))
    src = np.array([[0.5, 0.5, 0.5], [0.3125, 0.7, 0.41], [0.1, 0.9, 0.5]])
    for nside in (8, 16):
        _check_case(rt, keys, lev, dens, src, nside, label=f"few nside{nside}")
    cloud = synth.uniform_cloud(5, 1.0, 4, fracs=(1.0,), dtype=np.float64)
    _check_case(rt, cloud.keys, cloud.levels, cloud.dens, np.array([[0.515625, 0.515625, 0.515625]]), 16,
                label="uniform centre nside16")


def test_extreme_source_coordinates(rt):
    """Source coordinates at the ends of what [0, 1) holds, combined per axis:
    -0.0, the smallest subnormal and the smallest normal double, values below
    and at the 2^-53 lattice spacing, the largest doubles below 0.5 and below
    1, and points 1 to 255 lattice steps below a depth-21 cell face (where the
    32-bit fraction's FP32 rounding goes up to 2^32).  Uniform grid (grid
    walks) and a random octree (tree walks), Nside 2, both modes."""
    face = 6 * 2.0 ** -21
    vals = np.array([-0.0, 0.0, 5e-324, 2.2250738585072014e-308, 2.0 ** -60, 2.0 ** -53, 3 * 2.0 ** -54,
                     np.nextafter(0.5, 0.0), 0.5, np.nextafter(1.0, 0.0), 0.25 + 2.0 ** -53,
                     face - 2.0 ** -53, face - 127 * 2.0 ** -53, face - 128 * 2.0 ** -53,
                     face - 129 * 2.0 ** -53, face - 255 * 2.0 ** -53, 0.75 - 2.0 ** -40])
    rng = np.random.default_rng(4242)
    src = np.concatenate([vals[rng.integers(0, len(vals), size=(240, 3))], np.repeat(vals[:, None], 3, axis=1)])
    assert np.signbit(src).any()  # -0.0 survives the construction
    keys, lev = uniform_octree(4)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 2)).astype(np.float32)
    _check_case(rt, keys, lev, dens, src, 2, label="uniform16 extreme sources")
    keys, lev, _ = random_octree(rng, 1, 6, 0.35)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 2)).astype(np.float32)
    _check_case(rt, keys, lev, dens, src, 2, label="octree extreme sources")


@pytest.mark.parametrize("seed", range(2))
def test_uniform_grid_off_lattice_sources(rt, seed):
    """The uniform-grid walks with sources off the cell lattice (non-zero
    fractions), on cell corners and faces, and on x = y diagonals (equal x/y
    distances: the FP64 lock-step without zero fractions), Nside 1, 2 and 4,
    both modes."""
    rng = np.random.default_rng(3000 + seed)
    keys, lev = uniform_octree(4)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 2)).astype(np.float32)
    lo, hi = leaf_boxes(keys, lev)
    pick = rng.choice(keys.shape[0], size=16, replace=False)
    a, b = rng.random(24), rng.random(24)
    pts = [rng.random((64, 3)),                                   # off the lattice
           0.5 * (lo[pick] + hi[pick]),                           # cell centres
           lo[pick],                                              # cell corners
           np.column_stack([lo[pick, 0], rng.random(16), rng.random(16)]),   # on an x face
           np.column_stack([a, a, b]),                            # x = y, off the lattice
           np.column_stack([1.0 - a, a, b])]                      # mirrored diagonal
    src = np.concatenate(pts)
    for nside in (1, 2, 4):
        _check_case(rt, keys, lev, dens, src, nside, label=f"uniform16 off-lattice {seed} nside{nside}")
