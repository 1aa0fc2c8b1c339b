"""Seeded synthetic inputs for the column-density tracer.

This module builds the inputs only: lognormal turbulent density fields, the
leaf-only linear octree that stores them (sorted Morton keys, levels,
per-leaf species densities) and the source points rays start from.  It holds
none of the tracing arithmetic (no ray setup, slab exits, path lengths or
column sums); both the CPU oracle and the CUDA path consume what it returns.

Conventions (shared input format, Sec. 2.2.1 of the paper: the linear octree
stores leaves as compact arrays of Morton code, refinement level and value):

* the domain is the unit cube [0, 1)^3; integer positions live on the depth-21
  lattice (2^21 cells per axis);
* a leaf at level l with integer corner (ix, iy, iz) (in level-l cells) has the
  key interleave(ix << (21 - l), iy << (21 - l), iz << (21 - l)) with x in bit
  3b, y in bit 3b + 1 and z in bit 3b + 2; keys are sorted ascending;
* densities are stored [n_leaves][S] (species fastest);
* sources are float64 [n_src][3] positions on the 2^-53 lattice.

Field recipe (stand-in for the paper's SILCC-Zoom cloud, Sec. 4): a Gaussian
random field with power spectrum P(k) ~ k^-4 on integer wavenumbers, shifted to
mean 0 and scaled to standard deviation sigma, exponentiated (n = exp(g)).  AMR
clouds define the field on their finest grid and give each leaf the mean of the
finest cells it covers; at every level the leaves above the pct-th percentile of
that level's leaf densities are split into 8 children.
"""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass, field

import numpy as np

D = 21  # anchor depth of the Morton lattice

# Species fractions for multi-species clouds (H, H2, CO, C); each leaf draws an
# independent +-20% uniform perturbation per species.
SPECIES_FRACTIONS = (1.0, 0.4, 1.0e-4, 2.0e-4)


def _rfftn(a):
    try:
        import scipy.fft as sf
        return sf.rfftn(a, workers=os.cpu_count())
    except Exception:  # pragma: no cover - numpy fallback when scipy is absent
        return np.fft.rfftn(a)


def _irfftn(a, shape):
    try:
        import scipy.fft as sf
        return sf.irfftn(a, s=shape, workers=os.cpu_count())
    except Exception:  # pragma: no cover
        return np.fft.irfftn(a, s=shape)


def spread_bits(v):
    """Insert two zero bits between the low 21 bits of each element (uint64)."""
    v = np.asarray(v, dtype=np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def interleave(x, y, z):
    """Morton key of depth-21 integer coordinates (x in bit 3b)."""
    return spread_bits(x) | (spread_bits(y) << np.uint64(1)) | (spread_bits(z) << np.uint64(2))


def grf_lognormal(n: int, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """n = exp(g) on an n^3 grid, indexed [z][y][x]; g has P(k) ~ k^-4."""
    w = rng.standard_normal((n, n, n))
    wk = _rfftn(w)
    del w
    kz = (np.fft.fftfreq(n) * n).astype(np.float64)
    kx = (np.fft.rfftfreq(n) * n).astype(np.float64)
    k2 = kz[:, None, None] ** 2 + kz[None, :, None] ** 2 + kx[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    wk /= k2  # amplitude ~ k^-2, power ~ k^-4
    wk[0, 0, 0] = 0.0
    del k2
    g = _irfftn(wk, (n, n, n))
    del wk
    g -= g.mean()
    g *= sigma / g.std()
    np.exp(g, out=g)
    return g


@dataclass
class Cloud:
    """A leaf-only linear octree with per-leaf species densities."""
    keys: np.ndarray            # uint64 [n]
    levels: np.ndarray          # uint8 [n]
    dens: np.ndarray            # float32/float64 [n][S]
    extent: tuple               # domain size in depth-21 cells per axis
    n_total: np.ndarray | None = None  # float64 [n], the underlying total density
    meta: dict = field(default_factory=dict)

    @property
    def n_leaves(self) -> int:
        return int(self.keys.shape[0])

    @property
    def n_species(self) -> int:
        return int(self.dens.shape[1])


def _species(n_total: np.ndarray, fracs, rng, dtype, noise=0.2) -> np.ndarray:
    S = len(fracs)
    out = np.empty((n_total.shape[0], S), dtype=np.float64)
    for k, f in enumerate(fracs):
        if noise:
            u = rng.uniform(-1.0, 1.0, size=n_total.shape[0])
            out[:, k] = f * n_total * (1.0 + noise * u)
        else:
            out[:, k] = f * n_total
    return out.astype(dtype)


def uniform_cloud(level: int, sigma: float, seed: int, fracs=(1.0,), dtype=np.float64,
                  noise=0.2) -> Cloud:
    """2^level cubed uniform leaves (a single-level linear octree)."""
    n = 1 << level
    rng = np.random.Generator(np.random.PCG64(seed))
    field_ = grf_lognormal(n, sigma, rng)
    shift = np.uint64(D - level)
    ax = np.arange(n, dtype=np.uint64) << shift
    mi = (spread_bits(ax)[None, None, :]
          | (spread_bits(ax)[None, :, None] << np.uint64(1))
          | (spread_bits(ax)[:, None, None] << np.uint64(2)))  # [z][y][x]
    order = (mi >> np.uint64(3 * (D - level))).ravel()
    del mi
    n_sorted = np.empty(n ** 3, dtype=np.float64)
    n_sorted[order] = field_.ravel()
    del field_, order
    keys = np.arange(n ** 3, dtype=np.uint64) << np.uint64(3 * (D - level))
    levels = np.full(n ** 3, level, dtype=np.uint8)
    dens = _species(n_sorted, fracs, rng, dtype, noise=noise if len(fracs) > 1 else 0.0)
    return Cloud(keys, levels, dens, (1 << D,) * 3, n_sorted,
                 dict(kind="uniform", level=level, sigma=sigma, seed=seed))


def _block_mean(a: np.ndarray, f: int) -> np.ndarray:
    if f == 1:
        return a
    n = a.shape[0] // f
    return a.reshape(n, f, n, f, n, f).mean(axis=(1, 3, 5))


def amr_cloud(base_cells: int, n_refine: int, pct: float, sigma: float, seed: int,
              fracs=(1.0,), dtype=np.float32, max_field: int = 512, noise=0.2) -> Cloud:
    """AMR cloud: base_cells^3 base leaves refined n_refine times above the
    pct-th percentile of each level's leaf densities.

    A base size that is not a power of two sits in a 2^ceil(log2) root with a
    domain extent of base_cells root cells per axis.  The field lives on the
    finest grid, capped at max_field cells per axis; leaves finer than the field
    take the density of their ancestor at field resolution.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    root = int(np.ceil(np.log2(base_cells)))
    fine = base_cells << n_refine
    r_field = n_refine
    while (base_cells << r_field) > max_field:
        r_field -= 1
    field_n = base_cells << r_field
    field_ = grf_lognormal(field_n, sigma, rng)

    key_list, lev_list, n_list = [], [], []
    # existing cells at the current level: integer coords (level units)
    iz, iy, ix = np.meshgrid(np.arange(base_cells), np.arange(base_cells),
                             np.arange(base_cells), indexing="ij")
    cur = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.int64)
    del ix, iy, iz
    for r in range(n_refine + 1):
        level = root + r
        if r <= r_field:
            means = _block_mean(field_, 1 << (r_field - r))  # [z][y][x] at level
            d = means[cur[:, 2], cur[:, 1], cur[:, 0]]
        else:
            # below the field resolution: inherit the ancestor's value
            up = cur >> (r - r_field)
            d = field_[up[:, 2], up[:, 1], up[:, 0]]
        if r < n_refine:
            thr = np.percentile(d, pct)
            split = d > thr
        else:
            split = np.zeros(d.shape[0], dtype=bool)
        leaf = ~split
        lc = cur[leaf].astype(np.uint64) << np.uint64(D - level)
        key_list.append(interleave(lc[:, 0], lc[:, 1], lc[:, 2]))
        lev_list.append(np.full(lc.shape[0], level, dtype=np.uint8))
        n_list.append(d[leaf])
        if r < n_refine:
            par = cur[split] * 2
            kids = [par + np.array([dx, dy, dz]) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
            cur = np.concatenate(kids, axis=0)
    del field_
    keys = np.concatenate(key_list)
    levels = np.concatenate(lev_list)
    n_total = np.concatenate(n_list).astype(np.float64)
    order = np.argsort(keys, kind="stable")
    keys, levels, n_total = keys[order], levels[order], n_total[order]
    dens = _species(n_total, fracs, rng, dtype, noise=noise if len(fracs) > 1 else 0.0)
    ext = base_cells << (D - root)
    return Cloud(keys, levels, dens, (ext, ext, ext), n_total,
                 dict(kind="amr", base_cells=base_cells, n_refine=n_refine, pct=pct,
                      sigma=sigma, seed=seed, root_level=root, finest=fine,
                      field_cells=field_n))


def deinterleave(keys):
    """Integer depth-21 corner of each key (inverse of interleave)."""
    def compact(v):
        v = v & np.uint64(0x1249249249249249)
        v = (v | (v >> np.uint64(2))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v >> np.uint64(4))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v >> np.uint64(8))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v >> np.uint64(16))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v >> np.uint64(32))) & np.uint64(0x1FFFFF)
        return v
    k = np.asarray(keys, dtype=np.uint64)
    return np.stack([compact(k), compact(k >> np.uint64(1)), compact(k >> np.uint64(2))], axis=1)


def leaf_centres(cloud: Cloud, idx=None) -> np.ndarray:
    """Centre of every leaf (or of leaves idx), float64 [n][3]; exact."""
    keys = cloud.keys if idx is None else cloud.keys[idx]
    lev = cloud.levels if idx is None else cloud.levels[idx]
    lo = deinterleave(keys).astype(np.float64)
    half = np.ldexp(1.0, (D - 1 - lev.astype(np.int64)))  # half the leaf size in depth-21 cells
    return (lo + half[:, None]) * 2.0 ** -D


def mass_weighted_sources(cloud: Cloud, n_src: int, seed: int) -> np.ndarray:
    """n_src points: leaf drawn with probability ~ n * V, position uniform in the
    half-open leaf on the 2^-53 lattice; sorted by leaf (Morton) order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    vol = np.ldexp(1.0, 3 * (D - cloud.levels.astype(np.int64)))
    w = cloud.n_total * vol
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    j = np.searchsorted(cdf, rng.random(n_src), side="right")
    j = np.minimum(j, cloud.n_leaves - 1)
    j.sort(kind="stable")
    lo = deinterleave(cloud.keys[j]).astype(np.uint64)
    size = np.uint64(1) << (np.uint64(D) - cloud.levels[j].astype(np.uint64))
    span = (size << np.uint64(32)).astype(np.uint64)
    off = np.stack([rng.integers(0, span.astype(np.int64)) for _ in range(3)], axis=1).astype(np.uint64)
    q = (lo << np.uint64(32)) + off
    return q.astype(np.float64) * 2.0 ** -53


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8)).hexdigest()


def manifest(cloud: Cloud, src: np.ndarray) -> dict:
    m = dict(cloud.meta)
    m.update(n_leaves=cloud.n_leaves, n_species=cloud.n_species, n_src=int(src.shape[0]),
             extent=list(cloud.extent),
             sha256=dict(keys=sha256(cloud.keys), levels=sha256(cloud.levels),
                         dens=sha256(cloud.dens), src=sha256(src)))
    return m


# --------------------------------------------------------------------------
# Named workloads (the paper's shapes, Sec. 3-4: 512^3 cloud, HEALPix l = 0, 1)

def workload_uniform32(seed=1):
    """32^3 uniform leaves, one FP64 species n = exp(g), sigma 1; all leaf centres; Nside 1."""
    c = uniform_cloud(5, 1.0, seed, fracs=(1.0,), dtype=np.float64)
    return c, leaf_centres(c), 1


def workload_amr128(seed=2, n_src=1_000_000):
    """128^3 base, sigma 1.5, finest 512^3, 2 levels above p90, 4 FP32 species,
    mass-weighted sources, Nside 2."""
    c = amr_cloud(128, 2, 90.0, 1.5, seed, fracs=SPECIES_FRACTIONS, dtype=np.float32)
    return c, mass_weighted_sources(c, n_src, seed + 100), 2


def workload_amr64_grad(seed=4):
    """64^3 base refined once above p85, one species, leaf-centre sources, Nside 2."""
    c = amr_cloud(64, 1, 85.0, 1.5, seed, fracs=(1.0,), dtype=np.float32)
    return c, leaf_centres(c), 2


def workload_uniform512(seed=5, level=9):
    """512^3 uniform leaves, sigma 2, 4 FP32 species, all leaf centres, Nside 1."""
    c = uniform_cloud(level, 2.0, seed, fracs=SPECIES_FRACTIONS, dtype=np.float32)
    return c, None, 1  # sources: leaf centres, generated on demand (3.2 GB at 512^3)


def batched_clouds(seed=3, n_clouds=64, base_choices=(16, 24, 32, 48, 64, 96),
                   max_refine=3, max_field=192):
    """Many independent clouds of uneven size and depth: base size and refinement
    depth drawn per cloud, 2 FP32 species, leaf-centre sources, Nside 1 or 2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_clouds):
        b = int(rng.choice(base_choices))
        r = int(rng.integers(0, max_refine + 1))
        nside = int(rng.choice((1, 2)))
        c = amr_cloud(b, r, 80.0, 1.5, 3000 + i, fracs=SPECIES_FRACTIONS[:2], dtype=np.float32,
                      max_field=max_field)
        out.append((c, leaf_centres(c), nside))
    return out


def cache_dir() -> str:
    d = os.environ.get("RT_SYNTH_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "rt_synth"))
    os.makedirs(d, exist_ok=True)
    return d


def cached_uniform512(seed=5, level=9) -> Cloud:
    """workload_uniform512's cloud, cached on disk as .npy files."""
    d = os.path.join(cache_dir(), f"uniform_l{level}_s{seed}")
    names = ("keys", "levels", "dens")
    if all(os.path.exists(os.path.join(d, n + ".npy")) for n in names):
        arrs = [np.load(os.path.join(d, n + ".npy"), mmap_mode=None) for n in names]
        return Cloud(arrs[0], arrs[1], arrs[2], (1 << D,) * 3, None,
                     dict(kind="uniform", level=level, sigma=2.0, seed=seed))
    c, _, _ = workload_uniform512(seed, level)
    os.makedirs(d, exist_ok=True)
    for n in names:
        tmp = os.path.join(d, n + ".tmp.npy")
        np.save(tmp, getattr(c, n))
        os.replace(tmp, os.path.join(d, n + ".npy"))
    return c
