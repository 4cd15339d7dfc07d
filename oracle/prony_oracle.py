"""Plain FP64 CPU oracle of the multivariate matrix-pencil Prony method.

TEST INFRASTRUCTURE ONLY: the product path never imports this module.  Only
tests/, the smoke check in __graft_entry__ and the benchmark's CPU-baseline
leg may call it.  It shares no code with the CUDA library.

Reference: N. Bosner, "Parallel Prony's method with multivariate matrix pencil
approach and its numerical aspect", arXiv 2012.11430.  Everything here is the
plain definition written out with explicit matrices and LAPACK:
  * Section 1: T = [f(k-h)], T_l = [f(k-h+e_l)] over I_n = {0..n}^d,
    reduced SVD T = U Sigma V^* (Eq. T_svd), S_l = U^* T_l V Sigma^{-1}
    (Eq. generateSl), joint diagonalisation through C_mu = sum_l mu_l S_l,
    z_j(l) = (W^{-1} S_l W)_jj (Eq. diagonalizeSl), t from the principal
    logarithm, c from argmin ||A^T c - f||_2 (Eq. ls_probl); Algorithm 1.
  * Section 2.2: the block power method for the SVD with rank determination
    by column-pivoted QR (Algorithm 3).
  * Section 2.1: Lanczos bidiagonalisation (Algorithm 2), full
    reorthogonalisation.
Readings of passages that are garbled or silent are listed beside the code
that takes them.

Conventions shared with the library boundary (not code):
  grid  complex128, shape (2n+2,)*d, coordinate x_l at index x_l + n;
  I_n   row-major, last coordinate fastest;
  t     (m, d) in [0,1)^d; results sorted lexicographically by t.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import philox

EPS64 = np.finfo(np.float64).eps


# --------------------------------------------------------------------------
# Section 1: index set, exponential sum, matrices
# --------------------------------------------------------------------------

def index_set(n: int, d: int) -> np.ndarray:
    """I_n = {0..n}^d with a fixed (row-major, last coordinate fastest) ordering.  (N, d) int."""
    axes = np.meshgrid(*([np.arange(n + 1)] * d), indexing="ij")
    return np.stack(axes, axis=-1).reshape(-1, d)


def box_set(lengths, d: int) -> np.ndarray:
    """Row-major enumeration of {0..L_0-1} x ... x {0..L_{d-1}-1}."""
    axes = np.meshgrid(*[np.arange(L) for L in lengths], indexing="ij")
    return np.stack(axes, axis=-1).reshape(-1, d)


def expsum(t: np.ndarray, c: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Eq. (1): f(k) = sum_j c_j exp(-2 pi i <t_j, k>) for integer points k (K, d).

    The phase <t_j, k> is reduced mod 1 in float64 before the exponential."""
    phase = np.mod(k.astype(np.float64) @ t.T, 1.0)          # (K, m)
    return np.exp(-2j * np.pi * phase) @ c


def sample(grid: np.ndarray, n: int, x: np.ndarray) -> np.ndarray:
    """Look up f(x) for integer points x (..., d) in {-n..n+1}^d."""
    d = x.shape[-1]
    if np.any(x < -n) or np.any(x > n + 1):
        raise IndexError("sample point outside {-n..n+1}^d")
    return grid[tuple(x[..., l] + n for l in range(d))]


def build_T(grid: np.ndarray, n: int, d: int) -> np.ndarray:
    """T = [f(k - h)]_{k,h in I_n}, N x N (Section 1)."""
    K = index_set(n, d)
    return sample(grid, n, K[:, None, :] - K[None, :, :])


def build_Tl(grid: np.ndarray, n: int, d: int, l: int) -> np.ndarray:
    """T_l = [f(k - h + e_l)]_{k,h in I_n}, l = 0..d-1 (Section 1)."""
    K = index_set(n, d)
    e = np.zeros(d, dtype=np.int64)
    e[l] = 1
    return sample(grid, n, K[:, None, :] - K[None, :, :] + e)


def data_vector(grid: np.ndarray, n: int, d: int) -> np.ndarray:
    """f = [f(k)]_{k in I_n} (Eq. ls_probl)."""
    return sample(grid, n, index_set(n, d))


def vandermonde(t: np.ndarray, n: int) -> np.ndarray:
    """A = [z_j^k]_{j, k in I_n} in C^{m x N}, z_j^k = exp(-2 pi i <t_j, k>) (Section 1)."""
    K = index_set(n, t.shape[1])
    return np.exp(-2j * np.pi * np.mod(t @ K.T.astype(np.float64), 1.0))


def T_frobenius_closed_form(grid: np.ndarray, n: int, d: int) -> float:
    """||T||_F: each difference x = k-h in {-n..n}^d occurs prod_l (n+1-|x_l|) times in T."""
    x = box_set([2 * n + 1] * d, d) - n
    w = np.prod(n + 1 - np.abs(x), axis=1).astype(np.float64)
    return float(np.sqrt(np.sum(w * np.abs(sample(grid, n, x)) ** 2)))


# --------------------------------------------------------------------------
# Reduced SVD: full LAPACK SVD (zgesvd, Section 5) and numerical rank
# --------------------------------------------------------------------------

def full_svd(T: np.ndarray):
    """All singular triplets of T by LAPACK gesvd, the paper's reference SVD (Section 5)."""
    U, s, Vh = sla.svd(T, full_matrices=False, lapack_driver="gesvd")
    return U, s, Vh.conj().T


def numerical_rank(s: np.ndarray, tol: float) -> int:
    """Smallest i with sigma_{i+1} < tol * sigma_1 (Section 5: tol = N eps_M noise-free,
    the noise level otherwise); returns the count of singular values kept."""
    if s.size == 0 or s[0] == 0.0:
        return 0
    small = np.nonzero(s < tol * s[0])[0]
    return int(small[0]) if small.size else int(s.size)


def canonicalize(U: np.ndarray, V: np.ndarray):
    """Fix the phase freedom of singular pairs (reading: u_i, v_i -> e^{-i theta} u_i, e^{-i theta} v_i
    with theta = arg of the largest-modulus entry of v_i, lowest index on ties).
    u_i sigma_i v_i^* is unchanged; S_l becomes D^* S_l D."""
    idx = np.argmax(np.abs(V), axis=0)
    ph = V[idx, np.arange(V.shape[1])]
    ph = ph / np.abs(ph)
    return U * ph.conj()[None, :], V * ph.conj()[None, :], ph


# --------------------------------------------------------------------------
# Algorithm 3: block power method for the SVD with rank determination
# --------------------------------------------------------------------------

def pivoted_qr_rank(Rv: np.ndarray, tol: float) -> int:
    """Rank from R of a column-pivoted QR: r = i-1 for the first (1-based) i with
    ||R(i:r0, i:r0)||_F <= tol ||R||_F (Section 2.2)."""
    r0 = Rv.shape[1]
    total = np.linalg.norm(Rv)
    if total == 0.0:
        return 0
    for i in range(r0):
        if np.linalg.norm(Rv[i:, i:]) <= tol * total:
            return i
    return r0


def block_power_svd(A: np.ndarray, r0: int, U0: np.ndarray, V0: np.ndarray, tol_power: float,
                    tol_rank: float, max_iter: int = 50, fixed_rank: int | None = None):
    """Algorithm 3 with explicit A (FP64, LAPACK QR).

    Readings: the Q_k^* of the column-pivoted step is the first r_k rows of R_V P^T over all
    columns (the printed square block does not match the width of U_k); later iterations use
    plain QR; `fixed_rank` replaces the detected rank by the given m (the rank is still
    detected and returned); iterations are capped at max_iter.
    Returns (U, sigma, V, detected_rank, iterations, ||R_k||_F / ||A||_F)."""
    normA = np.linalg.norm(A)
    V = V0
    U = U0
    Q = U.conj().T @ (A @ V)
    R = A @ V - U @ Q
    k = 0
    detected = None
    while np.linalg.norm(R) > tol_power * normA and k < max_iter:
        k += 1
        Ubar = A @ V
        U, _ = np.linalg.qr(Ubar)
        Vbar = A.conj().T @ U
        if k == 1:
            Vq, Rv, piv = sla.qr(Vbar, mode="economic", pivoting=True)
            detected = pivoted_qr_rank(Rv, tol_rank)
            rk = detected if fixed_rank is None else fixed_rank
            rk = max(1, min(rk, Rv.shape[1]))
            P = np.eye(Vbar.shape[1])[:, piv]
            V = Vq[:, :rk]
            Q = (Rv @ P.T)[:rk, :].conj().T
        else:
            V, Rv = np.linalg.qr(Vbar)
            Q = Rv.conj().T
        R = A @ V - U @ Q
    Uq, s, Vqh = np.linalg.svd(Q, full_matrices=False)
    r = Q.shape[1]
    return (U @ Uq[:, :r], s[:r], V @ Vqh.conj().T[:, :r], detected, k,
            float(np.linalg.norm(R) / normA) if normA else 0.0)


# --------------------------------------------------------------------------
# Algorithm 2: Lanczos bidiagonalisation with full reorthogonalisation
# --------------------------------------------------------------------------

def lanczos_bidiag(A: np.ndarray, p1: np.ndarray, tol: float, max_steps: int | None = None):
    """Algorithm 2 with full reorthogonalisation (Section 2.1): stops when alpha_i or beta_i
    falls below tol.  Returns (r, U_r, V, B) with A V_r ~ U_r B_r."""
    mrows, ncols = A.shape
    max_steps = max_steps or min(mrows, ncols)
    beta = np.linalg.norm(p1)
    v = p1 / beta
    Us, Vs, alphas, betas = [], [v], [], [beta]
    u_prev = np.zeros(mrows, dtype=A.dtype)
    for i in range(max_steps):
        r = A @ Vs[-1] - betas[-1] * u_prev if i else A @ Vs[-1]
        for u in Us:                                    # full reorthogonalisation
            r = r - u * (u.conj() @ r)
        alpha = np.linalg.norm(r)
        if alpha <= tol:
            break
        u_prev = r / alpha
        Us.append(u_prev)
        alphas.append(alpha)
        p = A.conj().T @ u_prev - alpha * Vs[-1]
        for vv in Vs:
            p = p - vv * (vv.conj() @ p)
        beta = np.linalg.norm(p)
        betas.append(beta)
        if beta <= tol:
            break
        Vs.append(p / beta)
    r = len(alphas)
    B = np.zeros((r, r + 1))
    for i in range(r):
        B[i, i] = alphas[i]
        if i + 1 < len(betas):
            B[i, i + 1] = betas[i + 1]
    return r, np.array(Us).T, np.array(Vs).T, B


# --------------------------------------------------------------------------
# Algorithm 1 steps after the SVD
# --------------------------------------------------------------------------

def build_S(Tls, U: np.ndarray, s: np.ndarray, V: np.ndarray):
    """S_l = U^* T_l V Sigma^{-1} (Eq. generateSl)."""
    return [U.conj().T @ Tl @ V / s[None, :] for Tl in Tls]


def joint_diagonalize(S, mu: np.ndarray):
    """W diagonalising C_mu = sum_l mu_l S_l (LAPACK geev); z_j(l) = (W^{-1} S_l W)_jj
    (Eq. diagonalizeSl, Eq. tildezj).  Returns (W, z) with z of shape (m, d)."""
    C = sum(mu[l] * S[l] for l in range(len(S)))
    _, W = sla.eig(C)
    z = np.stack([np.diag(np.linalg.solve(W, Sl @ W)) for Sl in S], axis=1)
    return W, z


def t_from_z(z: np.ndarray) -> np.ndarray:
    """t_j(l) from the principal value of log z_j(l).  Reading: z = exp(-2 pi i t) gives
    t = -arg(z) / (2 pi) mod 1 (the printed arctan form loses the quadrant and its sign);
    a value that rounds to 1.0 wraps to 0."""
    t = np.mod(-np.angle(z) / (2.0 * np.pi), 1.0)
    t[t >= 1.0] = 0.0
    return t


def solve_c(t: np.ndarray, f: np.ndarray, n: int) -> np.ndarray:
    """argmin_c ||A^T c - f||_2 (Eq. ls_probl) with A built from t, by LAPACK least squares."""
    c, *_ = np.linalg.lstsq(vandermonde(t, n).T, f, rcond=None)
    return c


def vandermonde_z(z: np.ndarray, n: int) -> np.ndarray:
    """A with columns built from the raw eigenvalues z_j(l) instead of exp(-2 pi i t_j(l)):
    A[j, k] = prod_l z_j(l)^{k_l}, k in I_n (powers by repeated multiplication, no logarithm)."""
    m, d = z.shape
    K = index_set(n, d)
    A = np.ones((m, len(K)), dtype=np.complex128)
    for l in range(d):
        powers = np.ones((m, n + 1), dtype=np.complex128)
        for x in range(1, n + 1):
            powers[:, x] = powers[:, x - 1] * z[:, l]
        A *= powers[:, K[:, l]]
    return A


def solve_c_z(z: np.ndarray, f: np.ndarray, n: int) -> np.ndarray:
    """argmin_c ||A^T c - f||_2 with A from the raw z_j (Section 4 reading: the perturbation
    analysis builds A from the computed z~, not from unit-modulus exp(-2 pi i t~))."""
    c, *_ = np.linalg.lstsq(vandermonde_z(z, n).T, f, rcond=None)
    return c


def ls_residual(t, c, f, n) -> float:
    """||A^T c - f||_2 / ||f||_2 (Section 5: operational accuracy estimate)."""
    nf = np.linalg.norm(f)
    return float(np.linalg.norm(vandermonde(t, n).T @ c - f) / nf) if nf else 0.0


def sort_by_t(t: np.ndarray, c: np.ndarray):
    order = np.lexsort(t.T[::-1])
    return t[order], c[order]


def power_start_blocks(seed: int, N: int, r0: int):
    """Orthonormal U_0, V_0 (Algorithm 3 input) from the Philox complex normals, by QR."""
    U0, _ = np.linalg.qr(philox.complex_normal_block(seed, philox.STREAM_U0, N, r0))
    V0, _ = np.linalg.qr(philox.complex_normal_block(seed, philox.STREAM_V0, N, r0))
    return U0, V0


def prony(grid: np.ndarray, d: int, n: int, m: int, *, svd: str = "full", seed: int = 1,
          oversample_p: int | None = None, tol_rank: float | None = None,
          tol_power: float | None = None, max_iter: int = 50, detect_rank: bool = False,
          return_internals: bool = False, vandermonde_from: str = "t"):
    """Algorithm 1 (multivariate matrix-pencil Prony), FP64, explicit matrices.

    svd = "full": LAPACK gesvd of T, keep the leading m (Section 5 reference variant);
    svd = "power": Algorithm 3 with r0 = m + p (p = m by default: starting width 2m, Section 5).
    Rank: reported with the paper's criterion (tol_rank default N eps_M); with detect_rank the
    detected rank replaces m.  vandermonde_from = "t" builds A of the least-squares problem from
    t (unit modulus, Eq. ls_probl); "z" from the raw eigenvalues z~ (Section 4 reading).  Output
    sorted lexicographically by t."""
    if grid.shape != (2 * n + 2,) * d:
        raise ValueError("grid must have shape (2n+2,)*d")
    N = (n + 1) ** d
    tol_rank = N * EPS64 if tol_rank is None else tol_rank
    T = build_T(grid, n, d)
    f = data_vector(grid, n, d)
    info = {}
    if svd == "full":
        Uf, sf, Vf = full_svd(T)
        info["rank"] = numerical_rank(sf, tol_rank)
        info["sigma_all"] = sf
        r = info["rank"] if detect_rank else m
        U, s, V = Uf[:, :r], sf[:r], Vf[:, :r]
    elif svd == "power":
        p = m if oversample_p is None else oversample_p
        r0 = min(m + p, N)
        U0, V0 = power_start_blocks(seed, N, r0)
        tp = 8 * EPS64 if tol_power is None else tol_power
        U, s, V, det, iters, res = block_power_svd(T, r0, U0, V0, tp, tol_rank, max_iter,
                                                   fixed_rank=None if detect_rank else m)
        info.update(rank=det, power_iters=iters, power_resid=res)
    else:
        raise ValueError(svd)
    U, V, _ = canonicalize(U, V)
    S = build_S([build_Tl(grid, n, d, l) for l in range(d)], U, s, V)
    mu = philox.draw_mu(seed, d)
    W, z = joint_diagonalize(S, mu)
    t = t_from_z(z)
    if vandermonde_from == "z":
        c = solve_c_z(z, f, n)
        nf = np.linalg.norm(f)
        info["ls_resid"] = float(np.linalg.norm(vandermonde_z(z, n).T @ c - f) / nf) if nf else 0.0
    else:
        c = solve_c(t, f, n)
        info["ls_resid"] = ls_residual(t, c, f, n)
    t, c = sort_by_t(t, c)
    if return_internals:
        info.update(U=U, s=s, V=V, S=S, W=W, z=z, mu=mu, T=T, f=f)
    return t, c, info


def prony_S(grid, d, n, m, svd="full", seed=1, **kw):
    """The S_l of Algorithm 1 (phase-canonical basis) and the m leading singular values."""
    N = (n + 1) ** d
    T = build_T(grid, n, d)
    if svd == "full":
        U, s, V = full_svd(T)
        U, s, V = U[:, :m], s[:m], V[:, :m]
    else:
        r0 = min(2 * m, N)
        U0, V0 = power_start_blocks(seed, N, r0)
        U, s, V, *_ = block_power_svd(T, r0, U0, V0, kw.get("tol_power", 8 * EPS64),
                                      kw.get("tol_rank", N * EPS64), kw.get("max_iter", 50),
                                      fixed_rank=m)
    U, V, _ = canonicalize(U, V)
    return build_S([build_Tl(grid, n, d, l) for l in range(d)], U, s, V), s, U, V


def gram(t: np.ndarray, n: int) -> np.ndarray:
    """Vandermonde Gram conj(A) A^T (m x m), the normal-equation matrix of Eq. ls_probl."""
    A = vandermonde(t, n)
    return A.conj() @ A.T


def rhs(t: np.ndarray, f: np.ndarray, n: int) -> np.ndarray:
    """conj(A) f, the normal-equation right-hand side of Eq. ls_probl."""
    return vandermonde(t, n).conj() @ f


def expsum_grad(t, c, k, r):
    """Gradient of L(t, c) = sum_k |f(k; t, c) - y_k|^2 given residual r_k = f(k) - y_k.

    dL/dc_j (Wirtinger, conj) = sum_k conj(e_jk) r_k as the complex gradient 2*that,
    dL/dt_j(l) = 2 Re sum_k conj(r_k) c_j e_jk (-2 pi i k_l), with e_jk = exp(-2 pi i <t_j, k>).
    Returns (grad_t (m, d) real, grad_c (m,) complex with grad = dL/dRe + i dL/dIm)."""
    E = np.exp(-2j * np.pi * np.mod(k.astype(np.float64) @ t.T, 1.0))     # (K, m)
    gc = 2.0 * (E.conj().T @ r)
    gt = np.empty_like(t)
    for l in range(t.shape[1]):
        gt[:, l] = 2.0 * np.real((E * (-2j * np.pi * k[:, l:l + 1])).T @ r.conj() * c)
    return gt, gc


def refine_least_squares(t0, c0, k, y, max_nfev: int = 200):
    """argmin over (t, c) of L = sum_k |f(k; t, c) - y_k|^2 (Eq. 1 model), from (t0, c0).

    The paper fits c alone by least squares for fixed t (Eq. ls_probl); the refinement moves
    t as well.  Plain definition: scipy's Levenberg-Marquardt on the real residual vector
    [Re r; Im r] with the parameters (t_j(1..d), Re c_j, Im c_j) and its analytic Jacobian."""
    from scipy.optimize import least_squares
    m, d = t0.shape
    kf = k.astype(np.float64)

    def unpack(x):
        return x[:m * d].reshape(m, d), x[m * d:m * d + m] + 1j * x[m * d + m:]

    def resid(x):
        t, c = unpack(x)
        r = np.exp(-2j * np.pi * (kf @ t.T)) @ c - y
        return np.concatenate([r.real, r.imag])

    def jac(x):
        t, c = unpack(x)
        E = np.exp(-2j * np.pi * (kf @ t.T))                       # (K, m)
        cols = []
        Jt = (-2j * np.pi) * E[:, :, None] * kf[:, None, :] * c[None, :, None]   # (K, m, d)
        cols.append(Jt.reshape(len(kf), m * d))
        cols.append(E)
        cols.append(1j * E)
        J = np.concatenate(cols, axis=1)
        return np.concatenate([J.real, J.imag], axis=0)

    x0 = np.concatenate([t0.reshape(-1), c0.real, c0.imag])
    sol = least_squares(resid, x0, jac=jac, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=max_nfev)
    t, c = unpack(sol.x)
    return np.mod(t, 1.0), c, float(np.sum(sol.fun ** 2))
