"""The allocation-free entry point hawkes_loglik_grad_static.

It exists for callers that have no device allocator of their own or must not
make the blocking cudaMalloc call: it takes no workspace and runs on a fixed
scratch array inside the library.  This test calls it through the C ABI twice
in a row and compares each result with the workspace-based hawkes_loglik_grad
on the same inputs, within the tolerances the other GPU tests use.  It lives in
a file that pytest collects last."""
import ctypes

import numpy as np
import pytest

from helpers import GRAD_RTOL, LL_RTOL, maxnorm_rel, rel_err
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2604_01342_gb300 import binding
    binding.lib()
    return binding


def _tensors(p, dev):
    import torch
    return dict(
        t=torch.from_numpy(p.t).to(dev), c=torch.from_numpy(p.c).to(dev),
        mu=torch.tensor(p.mu, dtype=torch.float32, device=dev),
        al=torch.tensor(p.alpha, dtype=torch.float32, device=dev),
        be=torch.tensor(p.beta, dtype=torch.float32, device=dev))


def _outputs(M, dev):
    import torch
    return (torch.empty((), dtype=torch.float64, device=dev),
            torch.empty(M, dtype=torch.float32, device=dev),
            torch.empty(M, M, dtype=torch.float32, device=dev),
            torch.empty(M, dtype=torch.float32, device=dev))


def test_static_entry_matches_workspace_entry(B):
    import torch
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    p = synth.random_problem(24, 30_000, 2024, False)
    x = _tensors(p, dev)
    opts = B.make_opts(False, 0, True, 0)
    # reference: the workspace entry point
    n = B.hawkes_workspace_size(p.N, p.M, 1, True, opts)
    ws = torch.empty(n, dtype=torch.uint8, device=dev)
    ref = _outputs(p.M, dev)
    B.hawkes_loglik_grad(x["t"].data_ptr(), x["c"].data_ptr(), p.N, p.T, p.M, x["mu"].data_ptr(),
                         x["al"].data_ptr(), x["be"].data_ptr(), opts, ws.data_ptr(), n,
                         *[o.data_ptr() for o in ref], stream)
    assert B.hawkes_last_device_status(ws.data_ptr(), stream) == 0
    ref = [o.cpu().numpy().astype(np.float64) for o in ref]
    for _ in range(2):      # two calls in a row share the scratch array
        out = _outputs(p.M, dev)
        B.hawkes_loglik_grad_static(x["t"].data_ptr(), x["c"].data_ptr(), p.N, p.T, p.M,
                                    x["mu"].data_ptr(), x["al"].data_ptr(), x["be"].data_ptr(),
                                    opts, *[o.data_ptr() for o in out], stream)
        torch.cuda.synchronize()
        got = [o.cpu().numpy().astype(np.float64) for o in out]
        assert np.isfinite(got[0])
        assert rel_err(float(got[0]), float(ref[0])) <= LL_RTOL
        for g, r in zip(got[1:], ref[1:]):
            assert maxnorm_rel(g, r) <= GRAD_RTOL


def test_static_entry_rejects_oversized_problem(B):
    opts = B.make_opts(False, 0, True, 0)
    cap = B.hawkes_static_scratch_bytes()
    n_big = 10_000_000
    assert B.hawkes_workspace_size(n_big, 64, 1, True, opts) > cap
    fake = ctypes.c_void_p(256)   # never dereferenced: the size check comes first
    rc = B.lib().hawkes_loglik_grad_static(fake, fake, n_big, 1.0, 64, fake, fake, fake,
                                           ctypes.byref(opts), fake, fake, fake, fake, None)
    assert rc == 7   # HAWKES_ERR_WORKSPACE
