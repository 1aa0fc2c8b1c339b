"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each expected value is a hand
derivation (golden HEALPix table, Morton bit positions), a closed form (axis-ray
prefix sums, constant-density chord = domain exit distance), an invariant
(refinement invariance, linearity, mirror symmetry, adjoint = transpose), or a
brute force that does not walk (per-leaf slab chords, point sampling).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tinytrees import (domain_exit, random_octree, sampled_lengths, slab_chords, snap,
                       uniform_octree)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Morton

def test_morton_bit_positions_by_hand():
    # x bit b -> key bit 3b, y -> 3b+1, z -> 3b+2 (Sec. 2.2.1 Morton codes)
    enc = lambda x, y, z: int(oracle.morton_encode([[x, y, z]])[0])
    assert enc(1, 0, 0) == 1
    assert enc(0, 1, 0) == 2
    assert enc(0, 0, 1) == 4
    assert enc(2, 0, 0) == 8
    assert enc(3, 0, 0) == 9
    assert enc(0, 0, 1 << 20) == 1 << 62
    assert enc(5, 6, 7) == 0b111_110_101  # b0: z1 y0 x1, b1: z1 y1 x0, b2: z1 y1 x1
    assert enc((1 << 21) - 1, (1 << 21) - 1, (1 << 21) - 1) == (1 << 63) - 1


def test_morton_z_order_2cube():
    # level-1 cells sorted by key visit x fastest, then y, then z
    cells = [(x, y, z) for z in (0, 1) for y in (0, 1) for x in (0, 1)]
    keys = oracle.morton_encode([[x << 20, y << 20, z << 20] for x, y, z in cells])
    assert list(np.argsort(keys)) == list(range(8))
    assert all(int(k) == i << 60 for i, k in enumerate(keys))


def test_morton_round_trip_brute_force():
    g = np.arange(64, dtype=np.uint32)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    keys = oracle.morton_encode(xyz)
    assert len(np.unique(keys)) == xyz.shape[0]
    assert np.array_equal(oracle.morton_decode(keys), xyz)
    # 64^3 cells of a 6-bit lattice fill keys 0 .. 2^18 - 1 exactly
    assert keys.max() == (1 << 18) - 1
    rng = np.random.default_rng(11)
    r = rng.integers(0, 1 << 21, size=(20000, 3)).astype(np.uint32)
    assert np.array_equal(oracle.morton_decode(oracle.morton_encode(r)), r)
    # and the input generator's independent encoder agrees
    k2 = synth.interleave(r[:, 0].astype(np.uint64), r[:, 1].astype(np.uint64), r[:, 2].astype(np.uint64))
    assert np.array_equal(k2, oracle.morton_encode(r))


# ----------------------------------------------------------------- HEALPix

def _golden_healpix1():
    rows = []
    for line in open(os.path.join(GOLDEN, "healpix_nside1.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        vals = []
        for tok in line.split():
            sign = -1.0 if tok.startswith("-") else 1.0
            tok = tok.lstrip("-")
            if tok.startswith("sqrt("):
                a, b = tok[5:].split(")/")
                vals.append(sign * math.sqrt(int(a)) / int(b))
            else:
                vals.append(sign * float(Fraction(tok)))
        rows.append(vals)
    return np.array(rows)


def test_healpix_nside1_closed_form():
    got = oracle.healpix(1)
    want = _golden_healpix1()
    assert got.shape == (12, 3)
    np.testing.assert_allclose(got, want, rtol=0, atol=4e-16)
    # the axis rays are exact and |m_x| == |m_y| bitwise on the diagonal rings
    assert np.array_equal(got[4:8], want[4:8])
    assert np.all(np.abs(got[[0, 1, 2, 3, 8, 9, 10, 11], 0]) == np.abs(got[[0, 1, 2, 3, 8, 9, 10, 11], 1]))


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16])
def test_healpix_invariants(nside):
    d = oracle.healpix(nside)
    N = nside
    assert d.shape == (12 * N * N, 3)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=0, atol=4 * 2.2e-16)
    np.testing.assert_allclose(d.sum(axis=0), 0.0, atol=1e-13)
    # ring structure: ring i holds 4i pixels in the caps, 4N in the belt; ring z
    # values follow z = 1 - i^2/(3N^2) and z = 4/3 - 2i/(3N)
    p = 0
    for i in range(1, 4 * N):
        ii = min(i, 4 * N - i)
        cnt = 4 * ii if ii < N else 4 * N
        z = d[p:p + cnt, 2]
        if i < N:
            zt = 1 - i * i / (3 * N * N)
        elif i > 3 * N:
            zt = -(1 - ii * ii / (3 * N * N))
        else:
            zt = 4 / 3 - 2 * i / (3 * N)
        np.testing.assert_allclose(z, zt, atol=2e-16)
        phi = np.mod(np.arctan2(d[p:p + cnt, 1], d[p:p + cnt, 0]), 2 * np.pi)
        phi[np.isclose(phi, 2 * np.pi)] = 0.0
        assert np.all(np.diff(phi) > 0), "azimuth ascends within a ring"
        # equal spacing 2 pi / cnt
        np.testing.assert_allclose(np.diff(phi), 2 * np.pi / cnt, atol=1e-12)
        p += cnt
    assert p == 12 * N * N
    # north/south mirror symmetry holds bitwise
    np.testing.assert_array_equal(d[::-1][:, 2], -d[:, 2])


def test_healpix_rejects_bad_nside():
    with pytest.raises(oracle.OracleError):
        oracle.healpix(0)


# -------------------------------------------------------------- validation

def test_validate_faults():
    rng = np.random.default_rng(3)
    keys, lev, _ = random_octree(rng, 1, 4, 0.4)
    assert oracle.validate(keys, lev) == oracle.OK
    k = keys.copy(); k[[3, 4]] = k[[4, 3]]
    assert oracle.validate(k, lev) == oracle.ERR_UNSORTED
    i = int(np.nonzero(lev < 21)[0][0])
    k = keys.copy(); k[i] += np.uint64(1)
    assert oracle.validate(k, lev) == oracle.ERR_MISALIGNED
    l2 = lev.copy(); l2[5] = 22
    assert oracle.validate(keys, l2) == oracle.ERR_ARG
    # drop a leaf -> gap
    assert oracle.validate(np.delete(keys, 7), np.delete(lev, 7)) == oracle.ERR_OVERLAP_OR_GAP
    # coarsen a deep leaf whose siblings follow -> overlap
    j = int(np.nonzero(lev == lev.max())[0][0])
    l3 = lev.copy(); l3[j] = lev[j] - 1
    assert oracle.validate(keys, l3) in (oracle.ERR_OVERLAP_OR_GAP, oracle.ERR_MISALIGNED)
    # tree larger than the domain box
    assert oracle.validate(keys, lev, extent=(1 << 20, 1 << 21, 1 << 21)) == oracle.ERR_OVERLAP_OR_GAP
    # precedence: misaligned beats unsorted
    k = keys.copy(); k[[3, 4]] = k[[4, 3]]; k[i] += np.uint64(1)
    assert oracle.validate(k, lev) == oracle.ERR_MISALIGNED


def test_validate_non_power_of_two_extent():
    rng = np.random.default_rng(5)
    keys, lev, ext = random_octree(rng, 2, 4, 0.3, extent_cells=3)
    assert oracle.validate(keys, lev, extent=ext) == oracle.OK
    assert oracle.validate(keys, lev) == oracle.ERR_OVERLAP_OR_GAP


# ------------------------------------------------------------ closed forms

def test_axis_rays_prefix_sum_closed_form():
    """Uniform grid, ray along +-x / +-y from each centre:
    C_{+x}(i) = h (n_i / 2 + sum_{i' > i} n_i')."""
    L = 3
    N = 1 << L
    keys, lev = uniform_octree(L)
    rng = np.random.default_rng(7)
    dens = rng.uniform(0.1, 10.0, size=(keys.shape[0], 1))
    c = synth.deinterleave(keys) >> np.uint64(synth.D - L)
    grid = np.zeros((N, N, N))
    grid[c[:, 2], c[:, 1], c[:, 0]] = dens[:, 0]
    src = (c.astype(np.float64) + 0.5) / N
    dirs = oracle.healpix(1)[4:8]  # +x, +y, -x, -y
    cols, _, nseg = oracle.trace(keys, lev, dens, src, dirs)
    h = 1.0 / N
    ix, iy, iz = c[:, 0].astype(int), c[:, 1].astype(int), c[:, 2].astype(int)
    tail_x = np.cumsum(grid[:, :, ::-1], axis=2)[:, :, ::-1] - grid  # sum_{i'>i}
    head_x = np.cumsum(grid, axis=2) - grid                          # sum_{i'<i}
    tail_y = np.cumsum(grid[:, ::-1, :], axis=1)[:, ::-1, :] - grid
    head_y = np.cumsum(grid, axis=1) - grid
    want = np.stack([
        h * (0.5 * grid[iz, iy, ix] + tail_x[iz, iy, ix]),
        h * (0.5 * grid[iz, iy, ix] + tail_y[iz, iy, ix]),
        h * (0.5 * grid[iz, iy, ix] + head_x[iz, iy, ix]),
        h * (0.5 * grid[iz, iy, ix] + head_y[iz, iy, ix]),
    ], axis=1)
    np.testing.assert_allclose(cols[:, :, 0], want, rtol=1e-14)
    np.testing.assert_array_equal(nseg[:, 0], N - ix)
    np.testing.assert_array_equal(nseg[:, 2], ix + 1)


def test_constant_density_is_exit_distance():
    """n = 1 everywhere: every column equals the ray's length inside the box."""
    rng = np.random.default_rng(8)
    keys, lev, _ = random_octree(rng, 1, 5, 0.3)
    dens = np.ones((keys.shape[0], 1))
    src = rng.random((300, 3))
    dirs = oracle.healpix(2)
    cols, _, _ = oracle.trace(keys, lev, dens, src, dirs)
    Qs = snap(src)
    want = np.array([[domain_exit(Q, m) for m in dirs] for Q in Qs])
    np.testing.assert_allclose(cols[:, :, 0], want, rtol=1e-14)
    # and two values by hand: from the centre, pixel 0 (sqrt(10)/6, sqrt(10)/6, 2/3)
    # leaves through z = 1 at t = 0.5 / (2/3) = 0.75; pixel 4 (+x) at t = 0.5
    c, _, _ = oracle.trace(keys, lev, dens, [[0.5, 0.5, 0.5]], oracle.healpix(1))
    assert abs(c[0, 0, 0] - 0.75) < 1e-15
    assert abs(c[0, 4, 0] - 0.5) < 1e-15


def test_constant_density_non_power_of_two_extent():
    rng = np.random.default_rng(9)
    keys, lev, ext = random_octree(rng, 2, 4, 0.3, extent_cells=3)
    dens = np.ones((keys.shape[0], 1))
    src = rng.random((100, 3)) * 0.75
    dirs = oracle.healpix(1)
    cols, _, _ = oracle.trace(keys, lev, dens, src, dirs, extent=ext)
    want = np.array([[domain_exit(Q, m, ext) for m in dirs] for Q in snap(src)])
    np.testing.assert_allclose(cols[:, :, 0], want, rtol=1e-14)


# ------------------------------------------------------------- brute force

def _structured_sources(rng, keys, lev, n_random=20):
    """Random points, leaf centres, face and corner points (exact ties)."""
    from tinytrees import leaf_boxes
    lo, hi = leaf_boxes(keys, lev)
    pick = rng.choice(keys.shape[0], size=min(8, keys.shape[0]), replace=False)
    pts = [rng.random((n_random, 3)), 0.5 * (lo[pick] + hi[pick]), lo[pick],
           np.column_stack([lo[pick, 0], 0.5 * (lo[pick, 1] + hi[pick, 1]), lo[pick, 2]])]
    return np.concatenate(pts)


@pytest.mark.parametrize("seed", range(6))
def test_walk_equals_per_leaf_slab_chords(seed):
    """The walked (leaf, ds) sequence equals the set of leaves with a positive
    slab chord ordered by entry t, and each ds equals that chord."""
    rng = np.random.default_rng(100 + seed)
    keys, lev, _ = random_octree(rng, 1, 4, 0.4)
    dirs = oracle.healpix(2)
    for Q in _structured_sources(rng, keys, lev):
        Qs = snap(Q)
        for m in dirs[rng.choice(48, size=12, replace=False)]:
            leaf, ds = oracle.trace_path(keys, lev, Q, m)
            ell, tin = slab_chords(keys, lev, Qs, m)
            T = domain_exit(Qs, m)
            tol = 1e-13 * max(T, 1e-300)
            keep = ds > tol
            walked = leaf[keep]
            bf = np.nonzero(ell > tol)[0]
            bf = bf[np.argsort(tin[bf], kind="stable")]
            assert list(walked) == list(bf), (Q, m)
            np.testing.assert_allclose(ds[keep], ell[walked], rtol=0, atol=1e-14)
            # segment lengths add up to the length inside the box
            assert abs(ds.sum() - T) <= 1e-14 * max(T, 1.0)
            # no leaf is visited twice
            assert len(np.unique(leaf)) == len(leaf)


@pytest.mark.parametrize("seed", range(3))
def test_walk_lengths_match_point_sampling(seed):
    """Independent of slabs and Morton codes: midpoint sampling with a box
    containment test gives each leaf's length within two sample spacings."""
    rng = np.random.default_rng(200 + seed)
    keys, lev, _ = random_octree(rng, 1, 4, 0.4)
    for _ in range(10):
        Q = snap(rng.random(3))
        m = oracle.healpix(2)[rng.integers(48)]
        leaf, ds = oracle.trace_path(keys, lev, Q, m)
        est, dt = sampled_lengths(keys, lev, Q, m, n_samples=20000)
        got = np.zeros(keys.shape[0])
        np.add.at(got, leaf, ds)
        np.testing.assert_allclose(got, est, rtol=0, atol=2.01 * dt)


# ---------------------------------------------------------------- invariants

def test_refinement_invariance():
    """Splitting leaves into 8 equal-density children changes the paths but not
    the columns."""
    rng = np.random.default_rng(12)
    keys, lev = uniform_octree(3)
    dens = rng.uniform(0.5, 2.0, size=(keys.shape[0], 2))
    split = rng.random(keys.shape[0]) < 0.3
    k2, l2, d2 = [keys[~split]], [lev[~split]], [dens[~split]]
    lo = synth.deinterleave(keys[split])
    half = np.uint64(1) << (np.uint64(synth.D) - lev[split].astype(np.uint64) - np.uint64(1))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                c = lo + np.stack([half * np.uint64(dx), half * np.uint64(dy), half * np.uint64(dz)], 1)
                k2.append(synth.interleave(c[:, 0], c[:, 1], c[:, 2]))
                l2.append(lev[split] + 1)
                d2.append(dens[split])
    k2, l2, d2 = np.concatenate(k2), np.concatenate(l2), np.concatenate(d2)
    o = np.argsort(k2)
    k2, l2, d2 = k2[o], l2[o], d2[o]
    assert oracle.validate(k2, l2) == oracle.OK
    src = rng.random((200, 3))
    dirs = oracle.healpix(2)
    c1, _, n1 = oracle.trace(keys, lev, dens, src, dirs)
    c2, _, n2 = oracle.trace(k2, l2, d2, src, dirs)
    np.testing.assert_allclose(c2, c1, rtol=1e-13)
    assert (n2 >= n1).all() and (n2 > n1).any()


def test_linearity():
    rng = np.random.default_rng(13)
    keys, lev, _ = random_octree(rng, 1, 4, 0.4)
    n1 = rng.random((keys.shape[0], 1))
    n2 = rng.random((keys.shape[0], 1))
    src = rng.random((100, 3))
    dirs = oracle.healpix(2)
    a, b = 2.5, 0.75  # densities stay >= 0
    c12, _, _ = oracle.trace(keys, lev, a * n1 + b * n2, src, dirs)
    c1, _, _ = oracle.trace(keys, lev, n1, src, dirs)
    c2, _, _ = oracle.trace(keys, lev, n2, src, dirs)
    np.testing.assert_allclose(c12, a * c1 + b * c2, rtol=1e-12, atol=1e-14)
    # species are independent: stacking two species gives both columns
    c3, _, _ = oracle.trace(keys, lev, np.concatenate([n1, n2], 1), src, dirs)
    np.testing.assert_array_equal(c3[:, :, 0], c1[:, :, 0])
    np.testing.assert_array_equal(c3[:, :, 1], c2[:, :, 0])


def test_mirror_symmetry():
    """A field symmetric under x -> 1 - x gives equal columns for mirrored
    sources along mirrored directions."""
    L = 3
    N = 1 << L
    keys, lev = uniform_octree(L)
    c = (synth.deinterleave(keys) >> np.uint64(synth.D - L)).astype(int)
    rng = np.random.default_rng(14)
    half = rng.uniform(0.5, 3.0, size=(N, N, N))
    grid = half + half[:, :, ::-1]
    dens = grid[c[:, 2], c[:, 1], c[:, 0]][:, None]
    src = (c + 0.5) / N
    mirr = src.copy(); mirr[:, 0] = 1.0 - mirr[:, 0]
    dirs = oracle.healpix(2)
    mdirs = dirs.copy(); mdirs[:, 0] = -mdirs[:, 0]
    c1, _, _ = oracle.trace(keys, lev, dens, src, dirs)
    c2, _, _ = oracle.trace(keys, lev, dens, mirr, mdirs)
    np.testing.assert_allclose(c1, c2, rtol=1e-13)


# ------------------------------------------------------------------ adjoint

def test_adjoint_is_transpose_of_forward():
    """<g, A n> = <A^T g, n> and the explicit Jacobian from per-leaf chords."""
    rng = np.random.default_rng(15)
    keys, lev, _ = random_octree(rng, 1, 4, 0.4)
    S = 2
    src = rng.random((40, 3))
    dirs = oracle.healpix(1)
    n = rng.random((keys.shape[0], S))
    g = rng.standard_normal((40, 12, S))
    cols, _, _ = oracle.trace(keys, lev, n, src, dirs)
    grad = oracle.adjoint(keys, lev, S, src, dirs, g)
    lhs = float((g * cols).sum())
    rhs = float((grad * n).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    A = np.array([slab_chords(keys, lev, snap(Q), m)[0] for Q in src for m in dirs])  # [rays][leaves]
    np.testing.assert_allclose(A @ n, cols.reshape(-1, S), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(A.T @ g.reshape(-1, S), grad, rtol=1e-11, atol=1e-13)


def test_source_outside_is_an_error():
    keys, lev = uniform_octree(2)
    dens = np.ones((keys.shape[0], 1))
    for bad in ([1.0, 0.5, 0.5], [-1e-9, 0.5, 0.5], [np.nan, 0.5, 0.5]):
        with pytest.raises(oracle.OracleError) as e:
            oracle.trace(keys, lev, dens, [bad], oracle.healpix(1))
        assert e.value.code == oracle.ERR_SOURCE_OUTSIDE


def test_corner_crossing_worked_example():
    """Hand-worked ray with exact edge crossings: 4^3 uniform grid, source at
    the centre of cell (0,0,0), direction (sqrt(10)/6, sqrt(10)/6, 2/3)
    (HEALPix Nside 1 pixel 0).  x and y faces are met together at
    t = (k/4 - 1/8) / a (a = sqrt(10)/6) and must be stepped in one step;
    z faces at t = 1.5 (k/4 - 1/8); the ray leaves through z = 1 at 1.3125.
    Cells: (0,0,0) (0,0,1) (1,1,1) (1,1,2) (2,2,2) (2,2,3) (3,3,3), whose
    Morton indices are 0 4 7 35 56 60 63."""
    keys, lev = uniform_octree(2)
    a = math.sqrt(10) / 6
    m = oracle.healpix(1)[0]
    leaf, ds = oracle.trace_path(keys, lev, [0.125, 0.125, 0.125], m)
    assert list(leaf) == [0, 4, 7, 35, 56, 60, 63]
    ev = [0.0, 0.1875, 0.125 / a, 0.5625, 0.375 / a, 0.9375, 0.625 / a, 1.3125]
    np.testing.assert_allclose(ds, np.diff(ev), rtol=0, atol=1e-15)


# ------------------------------------------------ translation invariance

def _leaf_xyz(keys, lev, idx):
    sh = (21 - lev[idx].astype(np.int64)).astype(np.uint64)
    return (synth.deinterleave(keys[idx]) >> sh[:, None]).astype(np.int64)


@pytest.mark.parametrize("nside", [1, 2])
def test_uniform_grid_walk_is_translation_invariant(nside):
    """On a uniform grid every face-minus-source distance of a leaf-centre
    source is (k + 1/2) h, the same list for every source, so every exit time
    and every tie is the same: the steps (leaf offsets) and the segment
    lengths of two sources agree bit for bit until the nearer one leaves the
    box.  Offsets along each axis never reverse."""
    keys, lev = uniform_octree(3)
    src = synth.leaf_centres(synth.Cloud(keys, lev, np.zeros((keys.shape[0], 1)), (1 << 21,) * 3))
    rng = np.random.default_rng(31)
    for m in oracle.healpix(nside):
        pairs = rng.choice(keys.shape[0], size=(6, 2), replace=False)
        for a, b in pairs:
            la, da = oracle.trace_path(keys, lev, src[a], m)
            lb, db = oracle.trace_path(keys, lev, src[b], m)
            n = min(la.shape[0], lb.shape[0])
            oa = _leaf_xyz(keys, lev, la[:n]) - _leaf_xyz(keys, lev, la[:1])
            ob = _leaf_xyz(keys, lev, lb[:n]) - _leaf_xyz(keys, lev, lb[:1])
            assert np.array_equal(oa, ob)
            assert np.array_equal(da[:n].view(np.uint64), db[:n].view(np.uint64))
            steps = np.diff(oa, axis=0)
            assert np.all((steps * np.sign(m)[None, :]) >= 0) and np.all(np.abs(steps) <= 1)


def test_uniform_grid_adjoint_as_leaf_gather():
    """The transpose on a uniform grid with one leaf-centre source per leaf,
    written as a gather over the path of the corner source of each direction:
    grad[j] = sum_q sum_i [j - o_qi in the box] g[j - o_qi, q] ds_qi, equals the
    oracle's scatter adjoint."""
    level = 3
    keys, lev = uniform_octree(level)
    n = keys.shape[0]
    src = synth.leaf_centres(synth.Cloud(keys, lev, np.zeros((n, 1)), (1 << 21,) * 3))
    dirs = oracle.healpix(1)
    rng = np.random.default_rng(32)
    g = rng.random((n, 12, 1))
    ref = oracle.adjoint(keys, lev, 1, src, dirs, g)
    xyz = _leaf_xyz(keys, lev, np.arange(n))
    index = {tuple(v): i for i, v in enumerate(xyz)}
    N = 1 << level
    got = np.zeros(n)
    for q, m in enumerate(dirs):
        corner = np.where(m < 0, N - 1, 0)
        c = index[tuple(corner)]
        path, ds = oracle.trace_path(keys, lev, src[c], m)
        off = _leaf_xyz(keys, lev, path) - xyz[c]
        for j in range(n):
            s = xyz[j][None, :] - off
            ok = np.all((s >= 0) & (s < N), axis=1)
            for si, d in zip(s[ok], ds[ok]):
                got[j] += g[index[tuple(si)], q, 0] * d
    np.testing.assert_allclose(got, ref[:, 0], rtol=1e-13, atol=0)


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -1.0])
def test_nonfinite_or_negative_density_is_an_error(bad):
    """Densities are number densities: a ray that crosses a leaf whose density
    is NaN, infinite or negative has no column, and the trace reports the
    non-finite status (the code the library's density check records); a ray
    that does not cross it is unaffected."""
    keys, lev = uniform_octree(2)
    dens = np.ones((keys.shape[0], 2))
    dens[17, 1] = bad
    centre = synth.leaf_centres(synth.Cloud(keys, lev, np.zeros((keys.shape[0], 1)), (1 << 21,) * 3))
    with pytest.raises(oracle.OracleError) as e:  # a source inside the bad leaf crosses it first
        oracle.trace(keys, lev, dens, centre[17:18], oracle.healpix(1))
    assert e.value.code == oracle.ERR_NONFINITE
    # +x axis ray from the leaf at the -x face two rows away never enters leaf 17
    far = np.array([[0.125, 0.875, 0.875]])
    hit = oracle.trace_path(keys, lev, far[0], [1.0, 0.0, 0.0])[0]
    assert 17 not in hit
    cols, _, _ = oracle.trace(keys, lev, dens, far, np.array([[1.0, 0.0, 0.0]]))
    assert np.all(np.isfinite(cols))
    dens[17, 1] = 0.0  # zero is a valid density
    oracle.trace(keys, lev, dens, centre[17:18], oracle.healpix(1))
