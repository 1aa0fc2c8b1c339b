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
