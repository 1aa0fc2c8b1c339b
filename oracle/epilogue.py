"""Plain FP64 definitions of the per-source quantities built from the columns
(the paper's 3D-PDR coupling, Sec. 2.4, and its accuracy test, Sec. 3).

TEST INFRASTRUCTURE ONLY (like the rest of oracle/).  Every function takes the
oracle's FP64 columns I[p, q, k] ([n_src][n_dirs][S]) and a species weight
vector w ([S]) and forms the combined column N[p, q] = sum_k w_k I[p, q, k]
(a linear combination of species columns, as in the optical depth's
[n_j g_i / g_j - n_i] integrand of the discretised tau equation).

Pinned by tests/test_oracle_epilogue.py (equal columns in every direction,
the tau -> 0 limit, two-direction values worked by hand).
"""
from __future__ import annotations

import numpy as np


def combined(cols, w):
    """N[p, q] = sum_k w_k I[p, q, k]."""
    cols = np.asarray(cols, dtype=np.float64)
    return cols @ np.asarray(w, dtype=np.float64)


def av_eff(cols, w, a, gamma=3.02):
    """Effective visual extinction per source (Sec. 3, A_V,eff equation):
    -(1/gamma) ln( (1/N_rays) sum_q exp(-gamma a N[p, q]) ), with a the
    extinction per unit column (A_V0 times the box length in the column's
    length unit)."""
    N = combined(cols, w)
    return -np.log(np.mean(np.exp(-gamma * a * N), axis=1)) / gamma


def beta(cols, w, coef):
    """Escape probability per source (Sec. 2.4, discretised beta equation):
    (1/N_rays) sum_q (1 - exp(-tau_q)) / tau_q with tau_q = coef[p] N[p, q]
    (coef folds A_ij c^3 / (8 pi nu^3) / Delta u(p) and the box length);
    the q-term is 1 at tau = 0."""
    N = combined(cols, w)
    tau = np.asarray(coef, dtype=np.float64).reshape(-1, 1) * N
    with np.errstate(invalid="ignore", divide="ignore"):
        term = np.where(tau == 0.0, 1.0, -np.expm1(-tau) / tau)
    return np.mean(term, axis=1)


def attenuation(cols, w, a):
    """Attenuation factor per ray, I / I_0 = exp(-tau) with tau = a N[p, q]
    (Sec. 2.4: I = I_0 exp(-tau))."""
    return np.exp(-a * combined(cols, w))
