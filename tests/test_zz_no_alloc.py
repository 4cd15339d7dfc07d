"""The allocation-free Toeplitz product entry point against the regular one.

prony_toeplitz_mm_static serves callers that cannot let the library allocate device
memory (a fixed memory budget owned by their own allocator, or loops where cudaMalloc's
implicit device synchronisation is not acceptable).  Its scratch lives in a fixed device
array shared by all calls, so two calls in a row must each give the right answer.

This file is collected last on purpose: a failure here leaves every other test run.
"""
import gc

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_11430_gb300.build import build
    build()
    from paper_2012_11430_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("d,n,r,L_ext,adjoint", [(2, 15, 10, 1, 0), (2, 20, 7, 0, 1), (3, 5, 9, 1, 0)])
def test_static_matches_regular_twice_in_a_row(lib, d, n, r, L_ext, adjoint):
    import torch
    rng = np.random.Generator(np.random.PCG64(1000 + d * 100 + n))
    grid = rng.standard_normal((2 * n + 2) ** d) + 1j * rng.standard_normal((2 * n + 2) ** d)
    N = (n + 1) ** d
    L = n + 2 if L_ext else n + 1
    g_dev = torch.from_numpy(grid).cuda()
    ctx = lib.Context(0)
    try:
        for call in range(2):
            X = (rng.standard_normal((r, N)) + 1j * rng.standard_normal((r, N))).astype(np.complex64)
            X_dev = torch.from_numpy(X).cuda()
            Y_ref = torch.zeros((r, L ** d), dtype=torch.complex64, device="cuda")
            ctx.toeplitz_mm_dev(g_dev, d, n, X_dev, L, adjoint, "fp32", Y_ref)
            Y_st = torch.full((r, L ** d), float("nan"), dtype=torch.complex64, device="cuda")
            stream = torch.cuda.current_stream()
            lib.toeplitz_mm_static(g_dev, d, n, X_dev, L, adjoint, Y_st, stream.cuda_stream)
            stream.synchronize()
            a = Y_st.cpu().numpy().astype(np.complex128)
            b = Y_ref.cpu().numpy().astype(np.complex128)
            # both sum the same products in FP32; split-K order may differ: dot-product bound
            scale = np.abs(X.astype(np.complex128)).sum(axis=1, keepdims=True) * np.abs(grid).max()
            assert np.all(np.isfinite(a)), f"call {call}: non-finite output"
            assert np.all(np.abs(a - b) <= (4 * N + 16) * U32 * scale), f"call {call}"
    finally:
        ctx.close()


def test_static_rejects_oversized_grid(lib):
    import torch
    n = 512                                    # (2n+2)^2 = 1026^2 > PRONY_STATIC_MAX_GRID
    g = torch.zeros(8, dtype=torch.complex128, device="cuda")
    X = torch.zeros((1, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.PronyError) as e:
        lib.toeplitz_mm_static(g, 2, n, X, n + 1, 0, X)
    assert e.value.code == lib.PRONY_EINVAL
    assert "PRONY_STATIC_MAX_GRID" in lib.last_error()


def _product_pair(lib, ctx, grid, g_dev, d, n, r, L, adjoint, rng):
    """One static call and one regular call on the same X; returns (static, regular, X)."""
    import torch
    N = (n + 1) ** d
    X = (rng.standard_normal((r, N)) + 1j * rng.standard_normal((r, N))).astype(np.complex64)
    X_dev = torch.from_numpy(X).cuda()
    Y_ref = torch.zeros((r, L ** d), dtype=torch.complex64, device="cuda")
    ctx.toeplitz_mm_dev(g_dev, d, n, X_dev, L, adjoint, "fp32", Y_ref)
    Y_st = torch.full((r, L ** d), float("nan"), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()
    lib.toeplitz_mm_static(g_dev, d, n, X_dev, L, adjoint, Y_st, stream.cuda_stream)
    stream.synchronize()
    return Y_st.cpu().numpy().astype(np.complex128), Y_ref.cpu().numpy().astype(np.complex128), X


def test_static_larger_then_smaller_call(lib):
    """A large product followed by a small one on the same stream: the second call must not
    see the first call's descriptor, job list or grid copies left in the shared array."""
    import torch
    rng = np.random.Generator(np.random.PCG64(4242))
    ctx = lib.Context(0)
    try:
        for d, n, r, L_ext, adjoint in [(3, 9, 12, 1, 0), (2, 7, 3, 0, 1), (1, 20, 5, 1, 0)]:
            grid = rng.standard_normal((2 * n + 2) ** d) + 1j * rng.standard_normal((2 * n + 2) ** d)
            g_dev = torch.from_numpy(grid).cuda()
            L = n + 2 if L_ext else n + 1
            a, b, X = _product_pair(lib, ctx, grid, g_dev, d, n, r, L, adjoint, rng)
            N = (n + 1) ** d
            scale = np.abs(X.astype(np.complex128)).sum(axis=1, keepdims=True) * np.abs(grid).max()
            assert np.all(np.isfinite(a)), (d, n)
            assert np.all(np.abs(a - b) <= (4 * N + 16) * U32 * scale), (d, n)
    finally:
        ctx.close()


def test_static_call_leaves_device_memory_unchanged(lib):
    """After a warm-up call (which loads the module on this device), further calls change
    neither the free device memory nor torch's allocator state."""
    import torch
    rng = np.random.Generator(np.random.PCG64(77))
    d, n, r = 2, 15, 6
    N = (n + 1) ** d
    grid = rng.standard_normal((2 * n + 2) ** d) + 1j * rng.standard_normal((2 * n + 2) ** d)
    g_dev = torch.from_numpy(grid).cuda()
    X_dev = torch.from_numpy((rng.standard_normal((r, N)) + 1j * rng.standard_normal((r, N))).astype(np.complex64)).cuda()
    Y_dev = torch.zeros((r, (n + 2) ** d), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()
    lib.toeplitz_mm_static(g_dev, d, n, X_dev, n + 2, 0, Y_dev, stream.cuda_stream)   # warm-up
    torch.cuda.synchronize()
    gc.collect()                       # tensors of earlier tests must not be freed in between
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        lib.toeplitz_mm_static(g_dev, d, n, X_dev, n + 2, 0, Y_dev, stream.cuda_stream)
    torch.cuda.synchronize()
    gc.collect()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert np.all(np.isfinite(Y_dev.cpu().numpy()))


def test_static_rejects_too_many_columns(lib):
    import torch
    d, n = 1, 3                                   # N = 4 < r = 5
    g = torch.zeros((2 * n + 2) ** d, dtype=torch.complex128, device="cuda")
    X = torch.zeros((5, 4), dtype=torch.complex64, device="cuda")
    Y = torch.zeros((5, 5), dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.PronyError) as e:
        lib.toeplitz_mm_static(g, d, n, X, n + 2, 0, Y)
    assert e.value.code == lib.PRONY_EINVAL
