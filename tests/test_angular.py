"""Pins of the sky-map pixel lookup (HEALPix RING ang2pix) that the angular-
convergence measurement uses to average Nside-64 columns over each coarser
pixel: every pixel centre lies in its own pixel, each coarse pixel holds
exactly (64/N)^2 Nside-64 pixel centres (the hierarchical equal-area
subdivision), and any direction's coarse pixel is the coarse pixel of its
finer pixel's centre (the fine pixel lies inside one coarse pixel)."""
import numpy as np
import pytest

import bench
import oracle


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 64])
def test_pixel_centres_lie_in_their_own_pixel(nside):
    pix = bench.ang2pix_ring(nside, oracle.healpix(nside))
    np.testing.assert_array_equal(pix, np.arange(12 * nside * nside))


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 32])
def test_fine_centres_split_evenly_over_coarse_pixels(nside):
    counts = np.bincount(bench.ang2pix_ring(nside, oracle.healpix(64)), minlength=12 * nside * nside)
    assert counts.min() == counts.max() == (64 // nside) ** 2


@pytest.mark.parametrize("nside", [1, 2, 4, 8])
def test_random_directions_nest(nside):
    rng = np.random.default_rng(nside)
    v = rng.standard_normal((100_000, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    fine = bench.ang2pix_ring(2 * nside, v)
    centres = oracle.healpix(2 * nside)
    np.testing.assert_array_equal(bench.ang2pix_ring(nside, v), bench.ang2pix_ring(nside, centres[fine]))
