"""Pins of the oracle's contribution-grid construction (recursive refinement
with the n_max >= n_PDR and 1 % variation criterion)."""
import numpy as np
import pytest

import oracle
from oracle import amr_build


def test_uniform_field_is_one_root_leaf():
    keys, lev, vals = amr_build.build(np.full((8, 8, 8), 3.0), None, 1.0, 0.01, 3)
    assert list(keys) == [0] and list(lev) == [0] and vals[0, 0] == 3.0


def test_field_below_threshold_is_not_refined():
    rng = np.random.default_rng(1)
    n = rng.uniform(0.1, 0.9, size=(8, 8, 8))
    keys, lev, _ = amr_build.build(n, None, 1.0, 0.01, 3)
    assert len(keys) == 1


def test_single_dense_cell_refines_one_path():
    # one dense cell in a constant background: at every level exactly one cell
    # (the one holding the dense cell) splits, leaving 7 leaves per level and
    # 8 at the finest: 7 L + 1 leaves
    L = 4
    n = np.ones((1 << L,) * 3)
    n[5, 9, 2] = 100.0
    keys, lev, vals = amr_build.build(n, None, 1.0, 0.01, L)
    assert len(keys) == 7 * L + 1
    assert np.bincount(lev, minlength=L + 1).tolist() == [0] + [7] * (L - 1) + [8]
    # the dense cell is a finest leaf of value 100; mass is conserved
    assert np.any((lev == L) & (vals[:, 0] == 100.0))
    vol = np.ldexp(1.0, 3 * (L - lev.astype(int)))
    assert abs((vals[:, 0] * vol).sum() - n.sum()) <= 1e-12 * n.sum()
    assert oracle.validate(keys, lev) == oracle.OK


def test_variation_threshold_boundary():
    n = np.ones((2, 2, 2))
    n[0, 0, 0] = 1.0 / 0.99  # a variation near 1 %; the threshold is set to it exactly
    mx, mn = n.max(), n.min()
    keys, lev, _ = amr_build.build(n, None, 1.0, (mx - mn) / mx, 1)
    assert len(keys) == 8                # equal to the threshold: split
    keys, lev, _ = amr_build.build(n, None, 1.0, np.nextafter((mx - mn) / mx, 1.0), 1)
    assert len(keys) == 1                # just above it: kept


@pytest.mark.parametrize("seed", range(3))
def test_random_fields_satisfy_the_criterion(seed):
    rng = np.random.default_rng(seed)
    L = 4
    n = np.exp(rng.normal(0.0, 1.0, size=(1 << L,) * 3))
    vals = np.stack([n, 2 * n], axis=-1)
    for max_level in (2, 4):
        keys, lev, means = amr_build.build(n, vals, 1.0, 0.3, max_level)
        assert oracle.validate(keys, lev) == oracle.OK
        assert lev.max() <= max_level
        xyz = oracle.morton_decode(keys)
        for j in range(len(keys)):
            l = int(lev[j])
            h = 1 << (L - l)
            c = xyz[j] >> np.uint32(21 - L)
            blk = n[c[2]:c[2] + h, c[1]:c[1] + h, c[0]:c[0] + h]
            mx, mn = blk.max(), blk.min()
            refine = mx >= 1.0 and (mx - mn) / mx >= 0.3
            assert (not refine) or l == max_level
            np.testing.assert_allclose(means[j], [blk.mean(), 2 * blk.mean()], rtol=1e-12)
            if l > 0:  # the parent met the criterion
                hp = 2 * h
                p = (c >> np.uint32(L - l + 1)) << np.uint32(L - l + 1)
                pb = n[p[2]:p[2] + hp, p[1]:p[1] + hp, p[0]:p[0] + hp]
                assert pb.max() >= 1.0 and (pb.max() - pb.min()) / pb.max() >= 0.3
