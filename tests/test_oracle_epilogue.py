"""Pins of the oracle's per-source epilogues (A_V,eff, beta, attenuation)."""
import math

import numpy as np

import oracle
from oracle import epilogue as ep
from tinytrees import uniform_octree


def test_av_eff_equal_columns_is_the_column():
    # every direction sees the same N: A_V,eff = a N exactly
    cols = np.full((3, 12, 2), 0.0)
    cols[..., 0] = [[1.0], [2.5], [0.0]]
    got = ep.av_eff(cols, [1.0, 0.0], a=2.0)
    np.testing.assert_allclose(got, [2.0, 5.0, 0.0], rtol=1e-14, atol=1e-15)


def test_av_eff_two_directions_by_hand():
    cols = np.array([[[1.0], [3.0]]])
    g, a = 3.02, 0.5
    want = -math.log(0.5 * (math.exp(-g * a * 1.0) + math.exp(-g * a * 3.0))) / g
    np.testing.assert_allclose(ep.av_eff(cols, [1.0], a=a, gamma=g), [want], rtol=1e-15)
    # shielding is dominated by the least shielded direction: below the mean column
    assert want < a * 2.0


def test_beta_limits_and_constant_tau():
    cols = np.zeros((2, 12, 1))
    cols[1] = 0.7
    b = ep.beta(cols, [1.0], coef=[5.0, 2.0])
    assert b[0] == 1.0                                   # tau = 0 in every direction
    np.testing.assert_allclose(b[1], (1 - math.exp(-1.4)) / 1.4, rtol=1e-15)
    tiny = ep.beta(np.full((1, 4, 1), 1e-12), [1.0], coef=[1.0])
    np.testing.assert_allclose(tiny, [1.0 - 0.5e-12], rtol=1e-15)


def test_attenuation_and_species_weights():
    cols = np.array([[[1.0, 2.0], [0.0, 0.5]]])
    np.testing.assert_allclose(ep.attenuation(cols, [1.0, 2.0], a=0.1),
                               [[math.exp(-0.5), math.exp(-0.1)]], rtol=1e-15)


def test_av_eff_from_the_centre_of_a_constant_cloud():
    # n = 1 in the unit box: from the centre the Nside-1 columns are 0.75 along
    # the 8 diagonal-ring rays and 0.5 along the 4 axis rays
    keys, lev = uniform_octree(2)
    cols, _, _ = oracle.trace(keys, lev, np.ones((keys.shape[0], 1)), [[0.5, 0.5, 0.5]], oracle.healpix(1))
    g, a = 3.02, 1.0
    want = -math.log((8 * math.exp(-g * 0.75) + 4 * math.exp(-g * 0.5)) / 12) / g
    np.testing.assert_allclose(ep.av_eff(cols, [1.0], a=a, gamma=g), [want], rtol=1e-14)
