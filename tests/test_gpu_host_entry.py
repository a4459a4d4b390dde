"""The host-buffer entry point hawkes_loglik_grad_host: events copied to the device in
pieces of whole scan groups on a second stream while the checks and the scan's reduce pass
of the earlier pieces run.  Its results equal the device entry point's on the same inputs
(within the atomics' summation-order differences) on every path, with one piece and with
several (more than 2^21 events), and bad inputs in a late piece are still reported."""
import numpy as np
import pytest

from helpers import GRAD_RTOL, LL_RTOL, f32, gpu_run, maxnorm_rel, rel_err
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


def host_run(p, path=0, support=False, expect=0):
    import torch
    from paper_2604_01342_gb300 import binding as B
    opts = B.make_opts(p.shared_beta, 0, True, path, support=support)
    M, N = p.M, p.N
    nbytes = B.hawkes_workspace_size_host(N, M, opts)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    th = torch.from_numpy(np.ascontiguousarray(p.t)).pin_memory()
    ch = torch.from_numpy(np.ascontiguousarray(p.c, dtype=np.int32)).pin_memory()
    beta = p.beta[:1] if p.shared_beta else p.beta
    mu, al, be = (torch.tensor(f32(a), dtype=torch.float32).pin_memory() for a in (p.mu, p.alpha, beta))
    ll = torch.zeros((), dtype=torch.float64).pin_memory()
    dmu = torch.zeros(M, dtype=torch.float32).pin_memory()
    dal = torch.zeros(M, M, dtype=torch.float32).pin_memory()
    dbe = torch.zeros(be.numel(), dtype=torch.float32).pin_memory()
    rc = B.lib().hawkes_loglik_grad_host(th.data_ptr(), ch.data_ptr(), N, p.T, M, mu.data_ptr(),
                                         al.data_ptr(), be.data_ptr(), opts, ws.data_ptr(), nbytes,
                                         ll.data_ptr(), dmu.data_ptr(), dal.data_ptr(),
                                         dbe.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == expect
    return {"ll": float(ll.item()), "dmu": dmu.numpy().astype(np.float64),
            "dalpha": dal.numpy().astype(np.float64), "dbeta": dbe.numpy().astype(np.float64)}


def _same(a, b, what):
    assert rel_err(a["ll"], b["ll"]) <= 1e-8, what
    for k in ("dmu", "dalpha", "dbeta"):
        assert maxnorm_rel(a[k], b[k]) <= 1e-5, (what, k)


@pytest.mark.parametrize("n", [50_000, 5_000_000])
def test_host_entry_gemm_path(n):
    p = synth.workload(4, n_events=n)
    _same(host_run(p), gpu_run(p), f"gemm n={n}")


@pytest.mark.parametrize("n", [30_000, 4_500_000])
def test_host_entry_state_walk(n):
    p = synth.random_problem(24, n, 81, False)
    _same(host_run(p, path=1), gpu_run(p, path=1), f"walk n={n}")


def test_host_entry_mark_major():
    p = synth.random_problem(300, 2_200_000, 82, False, rho=0.6, density=0.05, beta_range=(0.3, 3.0))
    _same(host_run(p, path=3, support=True), gpu_run(p, path=3, support=True), "marks")


def test_host_entry_reports_a_bad_mark_in_a_late_piece():
    p = synth.random_problem(16, 4_400_000, 83, True)
    p.c = p.c.copy()
    p.c[-10] = 16                       # outside [0, M): in the last piece
    out = host_run(p, expect=3)
    assert np.isnan(out["ll"])
