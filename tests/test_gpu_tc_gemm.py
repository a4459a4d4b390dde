"""The tcgen05 GEMM (row-scaled fp16 hi/lo split, three products, TMA, tensor-memory
accumulator) against an FP64 product on the GPU.  Error bound:
|D - AB^T| <= tol * (|A| |B|^T)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2604_01342_gb300 import binding
    L = binding.lib()
    p = ctypes.c_void_p
    L.hawkes_test_tc_gemm.argtypes = [p, p, p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, p, p]
    L.hawkes_test_tc_gemm.restype = ctypes.c_int
    return L


@pytest.mark.parametrize("M,N,K,splits,signed", [
    (128, 256, 64, 1, False), (128, 256, 1024, 1, False), (300, 520, 1000, 1, True),
    (1024, 1024, 4096, 4, False), (96, 40, 200, 3, True), (1024, 2048, 1024, 1, False),
    (130, 70, 77, 2, True)])
def test_tc_gemm_matches_fp64(lib, M, N, K, splits, signed):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    lo = -1.0 if signed else 0.0
    A = (torch.rand(M, K, device="cuda", generator=g) * (1 - lo) + lo).float()
    B = (torch.rand(N, K, device="cuda", generator=g) * (1 - lo) + lo).float()
    A[0, :3] = torch.tensor([1e-6, 3.0e4, -2.5 if signed else 2.5], device="cuda")
    D = torch.full((M, N), float("nan"), device="cuda")
    ld = (K + 31) // 32 * 64                # halves per paired hi/lo row
    scratch = torch.empty((M + N) * ld * 2 + 4 * (M + N), dtype=torch.uint8, device="cuda")
    rc = lib.hawkes_test_tc_gemm(A.data_ptr(), B.data_ptr(), D.data_ptr(), M, N, K, splits,
                                 scratch.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    ref = A.double() @ B.double().T
    bound = A.double().abs() @ B.double().abs().T
    err = (D.double() - ref).abs()
    assert torch.isfinite(D).all()
    rel = float((err / bound.clamp_min(1e-30)).max())
    print(f"tc gemm M={M} N={N} K={K} splits={splits}: max bound-relative error {rel:.3e}")
    assert rel < 5e-6
