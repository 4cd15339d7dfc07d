"""Seeded synthetic inputs for the multivariate Prony problem (arXiv 2012.11430).

This module is shared by the tests, the benchmark and the CPU oracle's callers.
It draws the unknowns of the signal model -- nodes t_j in [0,1)^d and
coefficients c_j -- and synthesises the samples f(k) of the exponential sum
(Section 1, Eq. 1) on the sample grid {-n..n+1}^d, optionally with noise.
It holds none of the steps of Prony's method itself (no Toeplitz matrices, no
SVD, no eigenproblem, no least squares).

Grid layout (used everywhere in this project): a complex128 array of shape
(2n+2,)*d, axis l holds coordinate x_l = -n .. n+1, so point x sits at index
x + n; flattened row-major (last coordinate fastest) the linear index is
sum_l (x_l + n) * (2n+2)**(d-1-l).

Workload recipes (seeds are numpy PCG64, seed = 2012114300 + config number):
  C1  d=2, n=15, m=5,  noise-free                      (plain, small)
  C2  d=2, n=63, m=20, additive complex Gaussian, SNR 40 dB   (plain, large)
  C3  d=3, n=19, m=40, SNR 50 dB                       (precision study)
  C4  4096 problems, d=2, n~U{7..31}, m~U{2..min(12, floor(n/2)^2)}, SNR 30 dB
  C5  d=2, n=63, m=20, SNR 20 dB                       (refinement)
Nodes: uniform on [0,1)^d with wrap-around infinity-norm separation >= 2/n
(rejection sampling); coefficients c = r e^{i phi}, r~U[0.5,1.5], phi~U[0,2pi).
The paper's own efficiency workload (Section 5) is `paper_efficiency_problem`.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2012114300


@dataclasses.dataclass
class Problem:
    """One synthetic Prony instance: truth (t, c) and its sample grid."""
    name: str
    d: int
    n: int
    m: int
    t: np.ndarray          # (m, d) float64, truth nodes in [0,1)^d
    c: np.ndarray          # (m,) complex128, truth coefficients
    grid: np.ndarray       # (2n+2,)*d complex128 samples on {-n..n+1}^d
    clean: np.ndarray      # same, without noise
    snr_db: float | None = None
    rel_eps: float | None = None

    @property
    def N(self) -> int:
        return (self.n + 1) ** self.d


def torus_dist(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Componentwise wrap-around distance |((a-b+1/2) mod 1) - 1/2|."""
    return np.abs(np.mod(a - b + 0.5, 1.0) - 0.5)


def draw_nodes(rng: np.random.Generator, m: int, d: int, sep: float,
               restarts: int = 200, tries_per_node: int = 2000) -> np.ndarray:
    """m nodes on [0,1)^d, pairwise torus inf-distance >= sep.

    Sequential rejection sampling (uniform nodes); a set that gets stuck is redrawn.  When
    that keeps failing (dense packings), a jittered grid is used: g = floor(1/sep) cells per
    axis, m distinct cells drawn at random, one node per cell at the cell centre plus a
    uniform jitter of half-width (1/g - sep)/2, which keeps neighbours >= sep apart.
    A separation no packing of m nodes can reach is lowered to 1/ceil(m^(1/d))."""
    g_need = math.ceil(m ** (1.0 / d) - 1e-12)
    sep = min(sep, 1.0 / g_need)
    g = max(1, int(math.floor(1.0 / sep + 1e-12)))
    if g ** d >= m and (g ** d) < 3 * m:
        restarts = min(restarts, 3)           # dense packing: go to the jittered grid quickly
    for _ in range(restarts):
        out = np.empty((m, d))
        k = 0
        draws = 0
        while k < m and draws < tries_per_node * m:
            cand = rng.random((64, d))          # candidates tried in order, first valid one kept
            draws += 64
            if k:
                ok = np.min(np.max(torus_dist(out[None, :k, :], cand[:, None, :]), axis=2), axis=1) >= sep
                idx = np.flatnonzero(ok)
                if idx.size == 0:
                    continue
                cand = cand[idx]
            out[k] = cand[0]
            k += 1
        if k == m:
            return out
    if g ** d < m:
        raise RuntimeError(f"cannot place {m} nodes at separation {sep} in d={d}")
    cells = rng.choice(g ** d, size=m, replace=False)
    half = max(0.0, (1.0 / g - sep) / 2.0)
    out = np.empty((m, d))
    for j, cidx in enumerate(cells):
        rem = int(cidx)
        for l in range(d - 1, -1, -1):
            out[j, l] = ((rem % g) + 0.5) / g + rng.uniform(-half, half)
            rem //= g
    return np.mod(out, 1.0)


def draw_coeffs(rng: np.random.Generator, m: int) -> np.ndarray:
    r = rng.uniform(0.5, 1.5, m)
    phi = rng.uniform(0.0, 2.0 * math.pi, m)
    return r * np.exp(1j * phi)


def grid_axis(n: int) -> np.ndarray:
    """Coordinates -n .. n+1 of one grid axis."""
    return np.arange(-n, n + 2)


def synthesize(t: np.ndarray, c: np.ndarray, n: int) -> np.ndarray:
    """Noise-free samples of the signal model on the grid {-n..n+1}^d.

    Separable evaluation: exp(-2 pi i <t_j, x>) = prod_l exp(-2 pi i t_j(l) x_l),
    each factor with its phase reduced mod 1 in float64 first.
    """
    m, d = t.shape
    x = grid_axis(n).astype(np.float64)
    facs = [np.exp(-2j * np.pi * np.mod(np.outer(t[:, l], x), 1.0)) for l in range(d)]
    letters = "abcdefgh"[:d]
    spec = "j," + ",".join("j" + a for a in letters) + "->" + letters
    return np.einsum(spec, c, *facs, optimize=True)


def add_snr_noise(rng: np.random.Generator, clean: np.ndarray, snr_db: float) -> np.ndarray:
    """Additive circular complex Gaussian noise at the given SNR (dB) over the grid."""
    sig2 = np.sum(np.abs(clean) ** 2) / clean.size / (10.0 ** (snr_db / 10.0))
    s = math.sqrt(sig2 / 2.0)
    return clean + s * (rng.standard_normal(clean.shape) + 1j * rng.standard_normal(clean.shape))


def add_relative_noise(rng: np.random.Generator, clean: np.ndarray, eps: float) -> np.ndarray:
    """The paper's noise model f(k)(1+delta_k), |delta_k| <= eps (Section 4, Section 5):
    delta_k = eps * u_k with u_k uniform in the complex unit disk."""
    rad = np.sqrt(rng.random(clean.shape))
    ang = rng.uniform(0.0, 2.0 * math.pi, clean.shape)
    return clean * (1.0 + eps * rad * np.exp(1j * ang))


def make_problem(name: str, d: int, n: int, m: int, seed: int, snr_db: float | None = None,
                 rel_eps: float | None = None, sep: float | None = None) -> Problem:
    rng = np.random.Generator(np.random.PCG64(seed))
    t = draw_nodes(rng, m, d, 2.0 / n if sep is None else sep)
    c = draw_coeffs(rng, m)
    clean = synthesize(t, c, n)
    grid = clean
    if snr_db is not None:
        grid = add_snr_noise(rng, clean, snr_db)
    elif rel_eps is not None:
        grid = add_relative_noise(rng, clean, rel_eps)
    return Problem(name, d, n, m, t, c, grid, clean, snr_db, rel_eps)


def paper_efficiency_problem(d: int, m: int, n: int = 20, rel_eps: float | None = None,
                             seed: int = SEED_BASE + 9) -> Problem:
    """Section 5 workload: t_j(i) = ((i-1)m + j-1) 10^{-ceil(log10(dm))}, c_j = j + i j."""
    scale = 10.0 ** (-math.ceil(math.log10(d * m)))
    t = np.array([[((i * m) + j) * scale for i in range(d)] for j in range(m)], dtype=np.float64)
    c = np.array([(j + 1) + 1j * (j + 1) for j in range(m)])
    clean = synthesize(t, c, n)
    grid = clean
    if rel_eps:
        grid = add_relative_noise(np.random.Generator(np.random.PCG64(seed)), clean, rel_eps)
    return Problem(f"paper-d{d}-m{m}", d, n, m, t, c, grid, clean, None, rel_eps)


CONFIGS = {
    "C1": dict(d=2, n=15, m=5, snr_db=None),
    "C2": dict(d=2, n=63, m=20, snr_db=40.0),
    "C3": dict(d=3, n=19, m=40, snr_db=50.0),
    "C5": dict(d=2, n=63, m=20, snr_db=20.0),
}


def config_problem(name: str, seed_offset: int = 0) -> Problem:
    """One instance of C1, C2, C3 or C5 (seed_offset draws further instances)."""
    cfg = CONFIGS[name]
    seed = SEED_BASE + int(name[1:]) + 1000 * seed_offset
    return make_problem(name, cfg["d"], cfg["n"], cfg["m"], seed, snr_db=cfg["snr_db"])


def batch_problems(count: int = 4096, seed_offset: int = 0, n_lo: int = 7, n_hi: int = 31,
                   snr_db: float | None = 30.0, d: int = 2) -> list[Problem]:
    """C4: independent d=2 problems of uneven n and m.

    m ~ U{2..min(12, floor(n/2)^d)} keeps the separation 2/n feasible."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4 + 1000 * seed_offset))
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        m_hi = min(12, (n // 2) ** d)
        m = int(rng.integers(2, m_hi + 1))
        t = draw_nodes(rng, m, d, 2.0 / n)
        c = draw_coeffs(rng, m)
        clean = synthesize(t, c, n)
        grid = add_snr_noise(rng, clean, snr_db) if snr_db is not None else clean
        out.append(Problem(f"C4[{i}]", d, n, m, t, c, grid, clean, snr_db, None))
    return out


def match_to_truth(t_est: np.ndarray, c_est: np.ndarray, t_true: np.ndarray, c_true: np.ndarray):
    """Match estimated nodes to the truth (Hungarian assignment on torus distance).

    Returns (max componentwise torus error, relative 2-norm error of c)."""
    from scipy.optimize import linear_sum_assignment
    cost = np.max(torus_dist(t_est[:, None, :], t_true[None, :, :]), axis=2)
    r, col = linear_sum_assignment(cost)
    t_err = float(np.max(cost[r, col])) if len(r) else 0.0
    c_err = float(np.linalg.norm(c_est[r] - c_true[col]) / np.linalg.norm(c_true))
    return t_err, c_err
