"""GPU parity of the exponential-sum kernels and of the least-squares refinement.

  * forward f(k) (Eq. 1): complex64 results of FP32 exponentials of exactly reduced phases;
    |f_gpu - f| <= 1e-5 sum_j |c_j| per point.
  * backward (vector-Jacobian product behind torch.autograd): within 1e-4 relative (2-norm)
    of the FP64 oracle gradient, and of central finite differences of the FP64 loss.
  * Levenberg-Marquardt on the device: non-increasing loss, and the same minimiser as the
    FP64 oracle fit (scipy's Levenberg-Marquardt) from the same start: torus distance of t
    <= 1e-6, relative error of c <= 1e-5, loss within 1e-5 relative.
"""
import numpy as np
import pytest

import workloads as W
from oracle import prony_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_11430_gb300 import Context
    from paper_2012_11430_gb300.build import build
    build()
    c = Context(0)
    yield c
    c.close()


def _box(n, d):
    lo = [-n] * d
    length = [2 * n + 2] * d
    return lo, length, O.box_set(length, d) + np.array(lo)


def _noisy(d, n, m, seed, snr):
    return W.make_problem(f"refine-{d}-{n}-{m}-{seed}", d, n, m, seed, snr_db=snr)


def _dev(x, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("d,n,m", [(1, 20, 3), (2, 15, 5), (2, 63, 20), (3, 6, 4)])
def test_expsum_forward(ctx, d, n, m):
    import torch
    from paper_2012_11430_gb300.refine import expsum
    P = _noisy(d, n, m, 500 + n, 30.0)
    lo, length, k = _box(n, d)
    f = expsum(_dev(P.t, torch.float64), _dev(P.c, torch.complex64), ctx, lo, length).cpu().numpy()
    ref = O.expsum(P.t, P.c.astype(np.complex64).astype(np.complex128), k)
    assert np.max(np.abs(f - ref)) <= 1e-5 * np.sum(np.abs(P.c))


@pytest.mark.parametrize("d,n,m", [(2, 15, 5), (2, 63, 20), (3, 6, 4)])
def test_expsum_gradient(ctx, d, n, m):
    import torch
    from paper_2012_11430_gb300.refine import loss_fn
    P = _noisy(d, n, m, 600 + n, 20.0)
    lo, length, k = _box(n, d)
    y = P.grid.reshape(-1)
    rng = np.random.default_rng(3)
    t0 = np.mod(P.t + 1e-3 / n * rng.standard_normal(P.t.shape), 1.0)
    c0 = (P.c * (1 + 0.05 * rng.standard_normal(m))).astype(np.complex64).astype(np.complex128)
    t = _dev(t0, torch.float64).requires_grad_(True)
    c = _dev(c0, torch.complex64).requires_grad_(True)
    L = loss_fn(t, c, _dev(y, torch.complex64), ctx, lo, length)
    L.backward()
    gt, gc = t.grad.cpu().numpy(), c.grad.cpu().numpy()
    ot, oc = O.expsum_grad(t0, c0, k, O.expsum(t0, c0, k) - y)
    assert np.linalg.norm(gt - ot) <= 1e-4 * np.linalg.norm(ot)
    assert np.linalg.norm(gc - oc) <= 1e-4 * np.linalg.norm(oc)
    # central differences of the FP64 loss along the gradient direction
    loss = lambda tt, cc: float(np.sum(np.abs(O.expsum(tt, cc, k) - y) ** 2))  # noqa: E731
    h = 1e-7 / n
    vt, vc = ot / np.linalg.norm(ot), oc / np.linalg.norm(oc)
    fd_t = (loss(t0 + h * vt, c0) - loss(t0 - h * vt, c0)) / (2 * h)
    fd_c = (loss(t0, c0 + 1e-6 * vc) - loss(t0, c0 - 1e-6 * vc)) / 2e-6
    assert abs(np.sum(gt * vt) - fd_t) <= 1e-4 * abs(fd_t)
    assert abs(np.sum(gc.real * vc.real + gc.imag * vc.imag) - fd_c) <= 1e-4 * abs(fd_c)


@pytest.mark.parametrize("d,n,m,snr", [(2, 15, 5, 20.0), (2, 63, 20, 20.0), (1, 30, 4, 10.0), (3, 6, 3, 20.0)])
def test_lm_matches_oracle_fit(ctx, d, n, m, snr):
    import torch
    from paper_2012_11430_gb300.refine import refine_lm
    P = _noisy(d, n, m, 700 + n, snr)
    lo, length, k = _box(n, d)
    y = P.grid.reshape(-1)
    rng = np.random.default_rng(11)
    t0 = np.mod(P.t + 0.2 / n * rng.standard_normal(P.t.shape) / (2 * np.pi), 1.0)
    c0 = P.c * (1 + 0.05 * rng.standard_normal(m))
    to, co, Lo = O.refine_least_squares(t0, c0, k, y)
    t, c, losses = refine_lm(_dev(t0, torch.float64), _dev(c0, torch.complex128), _dev(y, torch.complex64),
                             ctx, lo, length, steps=40)
    t, c, losses = t.cpu().numpy(), c.cpu().numpy(), losses.cpu().numpy()
    assert np.all(np.diff(losses) <= 0.0)
    assert np.max(W.torus_dist(t, to)) <= 1e-6
    assert np.linalg.norm(c - co) <= 1e-5 * np.linalg.norm(co)
    Lg = float(np.sum(np.abs(O.expsum(t, c, k) - y) ** 2))
    assert Lg <= Lo * (1 + 1e-5)


def test_lm_graph_reuse_and_recapture(ctx):
    import torch
    from paper_2012_11430_gb300.refine import refine_lm
    P = _noisy(2, 15, 5, 801, 20.0)
    lo, length, _ = _box(15, 2)
    args = (_dev(P.t, torch.float64), _dev(P.c, torch.complex128), _dev(P.grid.reshape(-1), torch.complex64))
    a = refine_lm(*args, ctx, lo, length, steps=5)
    b = refine_lm(*args, ctx, lo, length, steps=5)       # same argument set except outputs: recaptured
    c = refine_lm(*args, ctx, lo, length, steps=7)
    for x, y in zip(a[:2], b[:2]):              # FP64 atomics: same result up to summation order
        assert torch.allclose(x, y, rtol=0, atol=1e-12)
    assert c[2][-1] <= a[2][-1]


def test_lm_same_buffers_replay(ctx):
    """Repeated calls on the same buffers replay the captured graph and continue the fit."""
    import torch
    P = _noisy(2, 15, 5, 802, 20.0)
    lo, length, _ = _box(15, 2)
    t = _dev(P.t, torch.float64)
    c = _dev(P.c, torch.complex128)
    y = _dev(P.grid.reshape(-1), torch.complex64)
    loss = torch.empty(4, dtype=torch.float64, device="cuda")
    ctx.refine_lm_dev(t, c, lo, length, y, 3, 1e-3, loss)
    first = loss.clone()
    ctx.refine_lm_dev(t, c, lo, length, y, 3, 1e-3, loss)
    assert loss[0] <= first[-1] * (1 + 1e-12) and loss[-1] <= loss[0]


def test_refine_rejects_bad_sizes(ctx):
    import torch
    from paper_2012_11430_gb300 import PronyError
    t = torch.zeros((60, 2), dtype=torch.float64, device="cuda")     # m (d + 2) = 240 > 160
    c = torch.zeros(60, dtype=torch.complex128, device="cuda")
    y = torch.zeros(64, dtype=torch.complex64, device="cuda")
    with pytest.raises(PronyError):
        ctx.refine_lm_dev(t, c, [0, 0], [8, 8], y, 2)


def test_adam_through_autograd_reduces_loss(ctx):
    import torch
    from paper_2012_11430_gb300.refine import refine_adam
    P = _noisy(2, 15, 5, 803, 20.0)
    lo, length, _ = _box(15, 2)
    rng = np.random.default_rng(2)
    t0 = np.mod(P.t + 2e-3 * rng.standard_normal(P.t.shape), 1.0)
    t, c, losses = refine_adam(_dev(t0, torch.float64), _dev(P.c, torch.complex64),
                               _dev(P.grid.reshape(-1), torch.complex64), ctx, lo, length, steps=50,
                               lr_t=2e-4, lr_c=1e-2)
    losses = losses.cpu().numpy()
    assert losses[-1] < 0.5 * losses[0]
