"""Classical one-dimensional Prony method (linear prediction + polynomial roots).

TEST INFRASTRUCTURE: an independent brute-force solver used to pin the oracle's
matrix-pencil path for d = 1, where the problem of Eq. (1) reduces to the
textbook case.  It uses no SVD and no eigendecomposition of the S_l.

For z_j = exp(-2 pi i t_j) the Prony polynomial p(z) = prod_j (z - z_j) =
sum_s p_s z^s (p_m = 1) annihilates the samples: sum_s p_s f(k+s) = 0 for every
k, because each term c_j z_j^k p(z_j) vanishes.  The coefficients p_0..p_{m-1}
solve this (overdetermined) linear system over all available windows; the nodes
are the roots of p; the coefficients c solve the Vandermonde system
f(k) = sum_j c_j z_j^k built from the powers of the roots.
"""
from __future__ import annotations

import numpy as np


def classical_prony_1d(samples: np.ndarray, n: int, m: int):
    """samples: f(k) for k = -n .. n+1 (length 2n+2).  Returns (t (m,1) sorted, c)."""
    k = np.arange(-n, n + 2)
    L = len(samples) - m
    H = np.array([[samples[a + s] for s in range(m)] for a in range(L)])
    rhs = -np.array([samples[a + m] for a in range(L)])
    p, *_ = np.linalg.lstsq(H, rhs, rcond=None)
    coeffs = np.concatenate([[1.0 + 0j], p[::-1]])         # highest degree first
    z = np.roots(coeffs)
    t = np.mod(-np.angle(z) / (2 * np.pi), 1.0)
    Vdm = np.power.outer(z, k.astype(np.float64)).T           # (K, m): z_j^k
    c, *_ = np.linalg.lstsq(Vdm, samples, rcond=None)
    order = np.argsort(t)
    return t[order][:, None], c[order]
