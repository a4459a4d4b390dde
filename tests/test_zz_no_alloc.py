"""The allocation-free entry point hawkes_loglik_grad_static.

It exists for callers that have no device allocator of their own or must not
make the blocking cudaMalloc call: it takes no workspace and runs on a fixed
scratch array inside the library.  These tests call it through the C ABI twice
in a row and compare each result with the workspace-based hawkes_loglik_grad on
the same inputs, within the tolerances the other GPU tests use, on each launch
sequence the scratch array has to hold: the state walk (per-source decays), the
chunk-GEMM path (one shared decay) and two decay kernels (two workspace slices).
One case is also compared with the FP64 oracle.  This file is collected last."""
import ctypes

import numpy as np
import pytest

from helpers import GRAD_RTOL, LL_RTOL, f32, maxnorm_rel, rel_err
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2604_01342_gb300 import binding
    binding.lib()
    return binding


def _tensors(t, c, mu, alpha, beta, dev):
    import torch
    return dict(
        t=torch.from_numpy(np.ascontiguousarray(t)).to(dev),
        c=torch.from_numpy(np.ascontiguousarray(c, dtype=np.int32)).to(dev),
        mu=torch.tensor(mu, dtype=torch.float32, device=dev),
        al=torch.tensor(alpha, dtype=torch.float32, device=dev),
        be=torch.tensor(beta, dtype=torch.float32, device=dev))


def _outputs(M, n_alpha, n_beta, dev):
    import torch
    return (torch.empty((), dtype=torch.float64, device=dev),
            torch.empty(M, dtype=torch.float32, device=dev),
            torch.empty(n_alpha, dtype=torch.float32, device=dev),
            torch.empty(n_beta, dtype=torch.float32, device=dev))


def _compare(B, x, N, T, M, n_alpha, n_beta, opts):
    """Workspace entry point once, then the static entry point twice in a row; returns
    the static entry point's last result."""
    import torch
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert 0 < B.hawkes_workspace_size(N, M, 1, True, opts) <= B.hawkes_static_scratch_bytes()
    n = B.hawkes_workspace_size(N, M, 1, True, opts)
    ws = torch.empty(n, dtype=torch.uint8, device=dev)
    ref = _outputs(M, n_alpha, n_beta, dev)
    B.hawkes_loglik_grad(x["t"].data_ptr(), x["c"].data_ptr(), N, T, M, x["mu"].data_ptr(),
                         x["al"].data_ptr(), x["be"].data_ptr(), opts, ws.data_ptr(), n,
                         *[o.data_ptr() for o in ref], stream)
    assert B.hawkes_last_device_status(ws.data_ptr(), stream) == 0
    ref = [o.cpu().numpy().astype(np.float64) for o in ref]
    got = None
    for _ in range(2):      # two calls in a row share the scratch array
        out = _outputs(M, n_alpha, n_beta, dev)
        B.hawkes_loglik_grad_static(x["t"].data_ptr(), x["c"].data_ptr(), N, T, M,
                                    x["mu"].data_ptr(), x["al"].data_ptr(), x["be"].data_ptr(),
                                    opts, *[o.data_ptr() for o in out], stream)
        torch.cuda.synchronize()
        got = [o.cpu().numpy().astype(np.float64) for o in out]
        assert np.isfinite(got[0])
        assert rel_err(float(got[0]), float(ref[0])) <= LL_RTOL
        for g, r in zip(got[1:], ref[1:]):
            assert maxnorm_rel(g, r) <= GRAD_RTOL
    return got


def test_static_entry_state_walk(B):
    import torch
    p = synth.random_problem(24, 30_000, 2024, False)
    x = _tensors(p.t, p.c, p.mu, p.alpha, p.beta, torch.device("cuda"))
    got = _compare(B, x, p.N, p.T, p.M, p.M * p.M, p.M, B.make_opts(False, 0, True, 0))
    # and against the FP64 oracle at the same tolerances
    import oracle
    ref = oracle.loglik_grad(p.t, p.c, p.T, f32(p.mu), f32(p.alpha), f32(p.beta))
    assert rel_err(float(got[0]), ref["ll"]) <= LL_RTOL
    assert maxnorm_rel(got[1], ref["dmu"]) <= GRAD_RTOL
    assert maxnorm_rel(got[2].reshape(p.M, p.M), ref["dalpha"]) <= GRAD_RTOL
    assert maxnorm_rel(got[3], ref["dbeta"]) <= GRAD_RTOL


def test_static_entry_chunk_gemm_path(B):
    import torch
    p = synth.random_problem(64, 40_000, 2025, True)
    x = _tensors(p.t, p.c, p.mu, p.alpha, p.beta[:1], torch.device("cuda"))
    _compare(B, x, p.N, p.T, p.M, p.M * p.M, 1, B.make_opts(True, 0, True, 2))


def test_static_entry_two_decay_kernels(B):
    import torch
    p = synth.random_problem_multi(48, 20_000, 2026, 2)
    x = _tensors(p.t, p.c, p.mu, p.alphas, p.betas, torch.device("cuda"))
    _compare(B, x, p.N, p.T, p.M, 2 * p.M * p.M, 2, B.make_opts(True, 0, True, 2, kernels=2))


def test_static_entry_rejects_oversized_problem(B):
    """A problem whose workspace exceeds the scratch array is rejected before any launch.
    The inputs are real device buffers of the full size, so nothing here depends on the
    order of the host-side checks."""
    import torch
    dev = torch.device("cuda")
    opts = B.make_opts(False, 0, True, 0)
    cap = B.hawkes_static_scratch_bytes()
    n_big, M = 10_000_000, 64
    assert B.hawkes_workspace_size(n_big, M, 1, True, opts) > cap
    t = torch.zeros(n_big, dtype=torch.float64, device=dev)
    c = torch.zeros(n_big, dtype=torch.int32, device=dev)
    prm = torch.ones(M * M + 2 * M, dtype=torch.float32, device=dev)
    outs = _outputs(M, M * M, M, dev)
    ptr = [o.data_ptr() for o in outs]
    lib = B.lib()
    rc = lib.hawkes_loglik_grad_static(t.data_ptr(), c.data_ptr(), n_big, 1.0, M, prm.data_ptr(),
                                       prm.data_ptr() + 4 * M, prm.data_ptr() + 4 * (M + M * M),
                                       ctypes.byref(opts), *ptr, None)
    assert rc == 7   # HAWKES_ERR_WORKSPACE
    # the same argument checks as hawkes_loglik_grad come first: a missing output is an
    # invalid argument whatever the size
    rc = lib.hawkes_loglik_grad_static(t.data_ptr(), c.data_ptr(), n_big, 1.0, M, prm.data_ptr(),
                                       prm.data_ptr() + 4 * M, prm.data_ptr() + 4 * (M + M * M),
                                       ctypes.byref(opts), ptr[0], ptr[1], None, ptr[3], None)
    assert rc == 1   # HAWKES_ERR_INVALID_ARG
    # and an unsupported configuration reports what hawkes_loglik_grad reports
    bad = B.make_opts(True, 5000, True, 2)       # chunk above the chunk-GEMM limit
    rc = lib.hawkes_loglik_grad_static(t.data_ptr(), c.data_ptr(), 1000, 1.0, M, prm.data_ptr(),
                                       prm.data_ptr() + 4 * M, prm.data_ptr() + 4 * (M + M * M),
                                       ctypes.byref(bad), *ptr, None)
    assert rc == 1
