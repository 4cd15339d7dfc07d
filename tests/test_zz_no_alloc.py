"""The allocation-free Toeplitz product entry point against the regular one.

prony_toeplitz_mm_static serves callers that cannot let the library allocate device
memory (a fixed memory budget owned by their own allocator, or loops where cudaMalloc's
implicit device synchronisation is not acceptable).  Its scratch lives in a fixed device
array shared by all calls, so two calls in a row must each give the right answer.

This file is collected last on purpose: a failure here leaves every other test run.
"""
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
