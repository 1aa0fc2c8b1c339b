"""Plain construction of the AMR contribution grid from a uniform source grid.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/).

The paper builds the contribution grid by recursive refinement (Sec. 2.2.1):
a cell that needs refinement is split into eight children until the maximum
depth (or the minimum cell size) is reached, and the terminal cells are the
leaves.  The criterion of the 3D-PDR coupling (Sec. 2.4): a cell is split only
if its maximum hydrogen density n_max >= n_PDR and its relative variation
(n_max - n_min) / n_max >= 1 %.  This module applies that recursion top-down
from the root over an N^3 source grid (N = 2^L), with the decision taken in
FP64 as `n_max >= n_pdr and (n_max - n_min) / n_max >= rel_var`.  A leaf's
value is the mean of the source cells it covers (a reading: the paper does not
say how a leaf's value is formed).

Pinned by tests/test_oracle_amr_build.py.
"""
from __future__ import annotations

import numpy as np

from . import morton_encode

D = 21


def build(n_ref, vals, n_pdr: float, rel_var: float, max_level: int):
    """n_ref: [N][N][N] ([z][y][x]) refinement density; vals: [N][N][N][S] or
    None (then vals = n_ref).  Returns keys (uint64, sorted), levels (uint8)
    and leaf means (float64 [n][S])."""
    n_ref = np.asarray(n_ref)
    N = n_ref.shape[0]
    L = N.bit_length() - 1
    assert N == 1 << L and n_ref.shape == (N, N, N)
    if vals is None:
        vals = n_ref[..., None]
    vals = np.asarray(vals, dtype=np.float64)
    max_level = min(max_level, L)
    leaves = []
    stack = [(0, 0, 0, 0)]
    while stack:
        l, x, y, z = stack.pop()
        h = 1 << (L - l)
        block = n_ref[z * h:(z + 1) * h, y * h:(y + 1) * h, x * h:(x + 1) * h]
        mx, mn = float(block.max()), float(block.min())
        split = l < max_level and mx >= n_pdr and (mx - mn) / mx >= rel_var if mx != 0.0 else False
        if split:
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        stack.append((l + 1, 2 * x + dx, 2 * y + dy, 2 * z + dz))
        else:
            mean = vals[z * h:(z + 1) * h, y * h:(y + 1) * h, x * h:(x + 1) * h].reshape(-1, vals.shape[-1]).mean(axis=0)
            leaves.append((l, x, y, z, mean))
    lev = np.array([v[0] for v in leaves], dtype=np.uint8)
    xyz = np.array([[v[1], v[2], v[3]] for v in leaves], dtype=np.uint64)
    shift = (np.uint64(D) - lev.astype(np.uint64))
    keys = morton_encode(np.stack([xyz[:, 0] << shift, xyz[:, 1] << shift, xyz[:, 2] << shift], axis=1))
    means = np.array([v[4] for v in leaves], dtype=np.float64)
    order = np.argsort(keys)
    return keys[order], lev[order], means[order]
