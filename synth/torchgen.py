"""Device-side generator for large uniform clouds (same recipe as synth's
numpy path, drawn with torch's seeded generator so that a 512^3 cloud takes
seconds on a GPU instead of minutes on the host).  Inputs only: no tracing
arithmetic lives here.  The draws differ from the numpy path's (different
random streams); each workload is defined by whichever generator produced it,
and the oracle checks whatever arrays the CUDA path was given.
"""
from __future__ import annotations

import torch

D = 21
SPECIES_FRACTIONS = (1.0, 0.4, 1.0e-4, 2.0e-4)


def _spread(v: torch.Tensor) -> torch.Tensor:
    v = v & 0x1FFFFF
    v = (v | (v << 32)) & 0x1F00000000FFFF
    v = (v | (v << 16)) & 0x1F0000FF0000FF
    v = (v | (v << 8)) & 0x100F00F00F00F00F
    v = (v | (v << 4)) & 0x10C30C30C30C30C3
    v = (v | (v << 2)) & 0x1249249249249249
    return v


def _compact(v: torch.Tensor) -> torch.Tensor:
    v = v & 0x1249249249249249
    v = (v | (v >> 2)) & 0x10C30C30C30C30C3
    v = (v | (v >> 4)) & 0x100F00F00F00F00F
    v = (v | (v >> 8)) & 0x1F0000FF0000FF
    v = (v | (v >> 16)) & 0x1F00000000FFFF
    v = (v | (v >> 32)) & 0x1FFFFF
    return v


def grf_lognormal(n: int, sigma: float, gen: torch.Generator, device) -> torch.Tensor:
    """exp(g) on an n^3 grid [z][y][x] (float64); g has P(k) ~ k^-4."""
    w = torch.randn((n, n, n), generator=gen, device=device, dtype=torch.float64)
    wk = torch.fft.rfftn(w)
    del w
    k = torch.fft.fftfreq(n, device=device, dtype=torch.float64) * n
    kx = torch.fft.rfftfreq(n, device=device, dtype=torch.float64) * n
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + kx[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    wk /= k2
    wk[0, 0, 0] = 0
    del k2
    g = torch.fft.irfftn(wk, s=(n, n, n))
    del wk
    g -= g.mean()
    g *= sigma / g.std()
    return g.exp_()


def uniform_cloud(level: int, sigma: float, seed: int, fracs=SPECIES_FRACTIONS,
                  dtype=torch.float32, device="cuda", noise=0.2):
    """2^level cubed uniform leaves in Morton order: keys (int64), levels
    (uint8), dens [n][S] and the total density (float64), all on `device`."""
    n = 1 << level
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    field = grf_lognormal(n, sigma, gen, device)
    ax = torch.arange(n, device=device, dtype=torch.int64) << (D - level)
    sx = _spread(ax)
    mi = (sx[None, None, :] | (sx[None, :, None] << 1) | (sx[:, None, None] << 2)) >> (3 * (D - level))
    n_tot = torch.empty(n ** 3, device=device, dtype=torch.float64)
    n_tot[mi.reshape(-1)] = field.reshape(-1)
    del field, mi
    keys = torch.arange(n ** 3, device=device, dtype=torch.int64) << (3 * (D - level))
    levels = torch.full((n ** 3,), level, device=device, dtype=torch.uint8)
    S = len(fracs)
    dens = torch.empty((n ** 3, S), device=device, dtype=dtype)
    for k, f in enumerate(fracs):
        if noise and S > 1:
            u = torch.rand(n ** 3, generator=gen, device=device, dtype=torch.float64) * 2.0 - 1.0
            dens[:, k] = (f * n_tot * (1.0 + noise * u)).to(dtype)
            del u
        else:
            dens[:, k] = (f * n_tot).to(dtype)
    return keys, levels, dens, n_tot


def uniform_centres(level: int, idx: torch.Tensor) -> torch.Tensor:
    """Centres (float64 [m][3]) of the uniform-grid leaves with Morton indices idx."""
    key = idx.to(torch.int64) << (3 * (D - level))
    c = torch.stack([_compact(key), _compact(key >> 1), _compact(key >> 2)], dim=1).to(torch.float64)
    half = float(1 << (D - level - 1))
    return (c + half) * 2.0 ** -D


def amr_cloud(base_cells: int, n_refine: int, pct: float, sigma: float, seed: int,
              fracs=SPECIES_FRACTIONS, dtype=torch.float32, device="cuda", max_field: int = 512,
              noise=0.2):
    """AMR cloud with synth.amr_cloud's recipe, built on `device`: base_cells^3
    base leaves (a 2^ceil(log2) root with a box extent when base_cells is not a
    power of two), the field on the finest grid (capped at max_field cells per
    axis), at every level the leaves above the pct-th percentile of that
    level's leaf densities split into 8.  Returns keys (int64, sorted), levels
    (uint8), dens [n][S], the total density (float64) and the extent."""
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    root = (base_cells - 1).bit_length()
    r_field = n_refine
    while (base_cells << r_field) > max_field:
        r_field -= 1
    field_n = base_cells << r_field
    field = grf_lognormal(field_n, sigma, gen, device)
    g = torch.arange(base_cells, device=device, dtype=torch.int64)
    cur = torch.stack(torch.meshgrid(g, g, g, indexing="ij")[::-1], dim=-1).reshape(-1, 3)  # x, y, z
    keys_l, lev_l, n_l = [], [], []
    for r in range(n_refine + 1):
        level = root + r
        if r <= r_field:
            f = 1 << (r_field - r)
            means = field if f == 1 else torch.nn.functional.avg_pool3d(field[None, None], f)[0, 0]
            d = means[cur[:, 2], cur[:, 1], cur[:, 0]]
        else:
            up = cur >> (r - r_field)
            d = field[up[:, 2], up[:, 1], up[:, 0]]
        if r < n_refine:
            srt = torch.sort(d).values
            # numpy's linear-interpolated percentile
            pos = pct / 100.0 * (d.numel() - 1)
            lo = int(pos)
            thr = srt[lo] + (srt[min(lo + 1, d.numel() - 1)] - srt[lo]) * (pos - lo)
            split = d > thr
            del srt
        else:
            split = torch.zeros_like(d, dtype=torch.bool)
        leaf = ~split
        lc = cur[leaf] << (D - level)
        keys_l.append(_spread(lc[:, 0]) | (_spread(lc[:, 1]) << 1) | (_spread(lc[:, 2]) << 2))
        lev_l.append(torch.full((lc.shape[0],), level, device=device, dtype=torch.uint8))
        n_l.append(d[leaf])
        if r < n_refine:
            par = cur[split] * 2
            off = torch.tensor([[dx, dy, dz] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)],
                               device=device, dtype=torch.int64)
            cur = (par[None, :, :] + off[:, None, :]).reshape(-1, 3)
    del field
    keys = torch.cat(keys_l)
    levels = torch.cat(lev_l)
    n_tot = torch.cat(n_l).to(torch.float64)
    keys, order = torch.sort(keys)
    levels, n_tot = levels[order], n_tot[order]
    S = len(fracs)
    dens = torch.empty((keys.numel(), S), device=device, dtype=dtype)
    for kk, f in enumerate(fracs):
        if noise and S > 1:
            u = torch.rand(keys.numel(), generator=gen, device=device, dtype=torch.float64) * 2.0 - 1.0
            dens[:, kk] = (f * n_tot * (1.0 + noise * u)).to(dtype)
        else:
            dens[:, kk] = (f * n_tot).to(dtype)
    ext = base_cells << (D - root)
    return keys, levels, dens, n_tot, (ext, ext, ext)


def leaf_centres(keys: torch.Tensor, levels: torch.Tensor) -> torch.Tensor:
    c = torch.stack([_compact(keys), _compact(keys >> 1), _compact(keys >> 2)], dim=1).to(torch.float64)
    half = torch.ldexp(torch.ones_like(levels, dtype=torch.float64), (D - 1 - levels.to(torch.int64)))
    return (c + half[:, None]) * 2.0 ** -D


def mass_weighted_sources(keys, levels, n_tot, n_src: int, seed: int):
    """Sources drawn with probability ~ n V, uniform inside the half-open leaf on
    the 2^-53 lattice, sorted by leaf (Morton) order."""
    gen = torch.Generator(device=keys.device)
    gen.manual_seed(seed)
    vol = torch.ldexp(torch.ones_like(n_tot), 3 * (D - levels.to(torch.int64)))
    j = torch.multinomial((n_tot * vol).to(torch.float64), n_src, replacement=True, generator=gen)
    j = torch.sort(j).values
    lo = torch.stack([_compact(keys[j]), _compact(keys[j] >> 1), _compact(keys[j] >> 2)], dim=1)
    span = (1 << (D - levels[j].to(torch.int64))) << 32
    u = torch.rand((n_src, 3), generator=gen, device=keys.device, dtype=torch.float64)
    off = torch.minimum((u * span[:, None].to(torch.float64)).to(torch.int64), span[:, None] - 1)
    q = (lo << 32) + off
    return q.to(torch.float64) * 2.0 ** -53


def batched_clouds(device="cuda", seed=3, n_clouds=64, base_choices=(16, 24, 32, 48, 64, 96),
                   max_refine=3, max_field=192):
    """The 64-cloud batch: per cloud a base size from base_choices (a
    non-power-of-two base is a box extent inside a power-of-two root), 0 to
    max_refine levels above the 80th percentile, sigma 1.5, 2 FP32 species
    (H, H2), leaf-centre sources and HEALPix Nside 1 or 2, all drawn from one
    seeded stream.  Returns [(keys, levels, dens, extent, src, nside)]."""
    import numpy as np
    g = np.random.default_rng(seed)
    out = []
    for i in range(n_clouds):
        b = int(g.choice(base_choices))
        r = int(g.integers(0, max_refine + 1))
        nside = int(g.choice((1, 2)))
        k, l, d, _, ext = amr_cloud(b, r, 80.0, 1.5, 3000 + i, fracs=(1.0, 0.4), device=device,
                                    max_field=max_field)
        out.append((k, l, d, ext, leaf_centres(k, l), nside))
    return out
