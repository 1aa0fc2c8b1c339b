"""Test-side helpers: tiny random linear octrees and brute-force references.

The brute-force references do not walk: `slab_chords` intersects the ray with
every leaf's box independently (the slab method of Sec. 2.2.2 applied to each
leaf, with divisions instead of a per-ray reciprocal), and `sampled_lengths`
estimates the length inside each leaf by point sampling with a containment
test, using neither slabs nor Morton codes.
"""
from __future__ import annotations

import numpy as np

import synth

D = synth.D


def random_octree(rng, root_level=1, max_level=4, p_split=0.35, extent_cells=None):
    """Leaves of a random octree: cells of the root level (optionally only the
    first extent_cells per axis) split recursively with probability p_split."""
    n0 = 1 << root_level
    e = extent_cells if extent_cells is not None else n0
    todo = [(root_level, x, y, z) for z in range(e) for y in range(e) for x in range(e)]
    leaves = []
    while todo:
        lev, x, y, z = todo.pop()
        if lev < max_level and rng.random() < p_split:
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        todo.append((lev + 1, 2 * x + dx, 2 * y + dy, 2 * z + dz))
        else:
            leaves.append((lev, x, y, z))
    lev = np.array([l[0] for l in leaves], dtype=np.uint8)
    xyz = np.array([l[1:] for l in leaves], dtype=np.uint64)
    sh = (np.uint64(D) - lev.astype(np.uint64))
    keys = synth.interleave(xyz[:, 0] << sh, xyz[:, 1] << sh, xyz[:, 2] << sh)
    order = np.argsort(keys)
    ext = None
    if extent_cells is not None:
        ext = (extent_cells << (D - root_level),) * 3
    return keys[order], lev[order], ext


def uniform_octree(level):
    n = 1 << level
    g = np.arange(n, dtype=np.uint64) << np.uint64(D - level)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    keys = synth.interleave(x.ravel(), y.ravel(), z.ravel())
    order = np.argsort(keys)
    return keys[order], np.full(n ** 3, level, dtype=np.uint8)


def leaf_boxes(keys, levels):
    lo = synth.deinterleave(keys).astype(np.float64) * 2.0 ** -D
    size = np.ldexp(1.0, -levels.astype(np.int64))
    return lo, lo + size[:, None]


def snap(src):
    """Sources as the tracer sees them: truncated to the 2^-53 lattice."""
    return np.floor(np.asarray(src, dtype=np.float64) * 2.0 ** 53) * 2.0 ** -53


def domain_exit(Q, m, extent=None):
    ext = np.array(extent if extent is not None else (1 << D,) * 3, dtype=np.float64) * 2.0 ** -D
    T = np.inf
    for b in range(3):
        if m[b] > 0:
            T = min(T, (ext[b] - Q[b]) / m[b])
        elif m[b] < 0:
            T = min(T, (0.0 - Q[b]) / m[b])
    return T


def slab_chords(keys, levels, Q, m, extent=None):
    """(chord length, entry t) of the ray Q + t m, t in [0, T], for every leaf."""
    lo, hi = leaf_boxes(keys, levels)
    n = keys.shape[0]
    tnear = np.full(n, -np.inf)
    tfar = np.full(n, np.inf)
    for b in range(3):
        if m[b] != 0.0:
            t1 = (lo[:, b] - Q[b]) / m[b]
            t2 = (hi[:, b] - Q[b]) / m[b]
            tnear = np.maximum(tnear, np.minimum(t1, t2))
            tfar = np.minimum(tfar, np.maximum(t1, t2))
        else:
            inside = (lo[:, b] <= Q[b]) & (Q[b] < hi[:, b])
            tnear = np.where(inside, tnear, np.inf)
    T = domain_exit(Q, m, extent)
    a = np.maximum(tnear, 0.0)
    ell = np.minimum(tfar, T) - a
    return np.maximum(ell, 0.0), a


def sampled_lengths(keys, levels, Q, m, n_samples=20000, extent=None):
    """Length of the ray inside each leaf estimated by midpoint sampling."""
    lo, hi = leaf_boxes(keys, levels)
    T = domain_exit(Q, m, extent)
    dt = T / n_samples
    t = (np.arange(n_samples) + 0.5) * dt
    P = Q[None, :] + t[:, None] * m[None, :]
    out = np.zeros(keys.shape[0])
    for i0 in range(0, n_samples, 2000):
        p = P[i0:i0 + 2000]
        inside = np.all((p[:, None, :] >= lo[None]) & (p[:, None, :] < hi[None]), axis=2)
        out += inside.sum(axis=0) * dt
    return out, dt
