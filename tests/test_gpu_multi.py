"""Several decay kernels on the GPU (chunk-GEMM path, one workspace slice per kernel)
against the FP64 oracle of several kernels, at the stated tolerances (relative L error
<= 1e-6, max-norm relative gradient error <= 1e-4 per block).

The log-likelihood and the decay gradient of each kernel are differences of large sums
that nearly cancel at the simulating parameters; the tests print their conditioning
(kappa = the oracle's sum of magnitudes of their terms over the result,
oracle.condition_multi) for information; the tolerances are the stated ones."""
import numpy as np
import pytest

from helpers import assert_close, f32
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(p):
    import torch
    dev = torch.device("cuda")
    return (torch.from_numpy(p.t).to(dev), torch.from_numpy(p.c.astype(np.int32)).to(dev), p.T,
            torch.tensor(p.mu, dtype=torch.float32, device=dev),
            torch.tensor(p.alphas, dtype=torch.float32, device=dev),
            torch.tensor(p.betas, dtype=torch.float32, device=dev))


def _oracle(p):
    import oracle
    return oracle.loglik_grad_multi(p.t, p.c, p.T, f32(p.mu), f32(p.alphas), f32(p.betas))


def _scales(p):
    import oracle
    cond = oracle.condition_multi(p.t, p.c, p.T, f32(p.mu), f32(p.alphas), f32(p.betas))
    return cond["ll"], cond["dbeta"].sum(axis=1)       # one decay per kernel


def _run(p, chunk=0, grad=True, validate=True):
    import torch
    from paper_2604_01342_gb300 import torch_api
    t, c, T, mu, al, be = _dev(p)
    r = torch_api.loglik_grad_multi(t, c, T, mu, al, be, chunk=chunk, grad=grad, validate=validate)
    torch.cuda.synchronize()
    if not grad:
        return {"ll": float(r.item())}
    ll, dmu, dal, dbe = r
    return {"ll": float(ll.item()), "dmu": dmu.cpu().numpy().astype(np.float64),
            "dalpha": dal.cpu().numpy().astype(np.float64),
            "dbeta": dbe.cpu().numpy().astype(np.float64)}


def _check(p, got, what):
    ref = _oracle(p)
    ref = dict(ref, dbeta=ref["dbeta"].sum(axis=1))      # one decay per kernel
    ll_scale, dbeta_scale = _scales(p)
    print(f"{what}: kappa of L {ll_scale / abs(ref['ll']):.0f}, of each dbeta "
          f"{np.round(dbeta_scale / np.abs(ref['dbeta']))} (information only)")
    assert_close(got, ref, what=what)


@pytest.mark.parametrize("m,n,k,chunk,seed", [(8, 3000, 2, 64, 51), (5, 2500, 3, 0, 52),
                                              (150, 20000, 3, 0, 53), (64, 9000, 4, 96, 54)])
def test_multi_kernel_matches_oracle(m, n, k, chunk, seed):
    p = synth.random_problem_multi(m, n, seed=seed, kernels=k)
    _check(p, _run(p, chunk=chunk), f"M={m} K={k} N={n}")


def test_multi_kernel_without_validation():
    p = synth.random_problem_multi(24, 6000, seed=62, kernels=2)
    _check(p, _run(p, validate=False), "unvalidated K=2")


def test_multi_kernel_loglik_only():
    p = synth.random_problem_multi(40, 5000, seed=55, kernels=2)
    got = _run(p, grad=False)
    ref = _oracle(p)
    assert abs(got["ll"] - ref["ll"]) <= 1e-6 * abs(ref["ll"])


def test_one_kernel_through_the_multi_api_equals_single_call():
    import torch
    from paper_2604_01342_gb300 import torch_api
    p = synth.random_problem(100, 8000, seed=56, shared_beta=True)
    dev = torch.device("cuda")
    t = torch.from_numpy(p.t).to(dev)
    c = torch.from_numpy(p.c.astype(np.int32)).to(dev)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    al = torch.tensor(p.alpha, dtype=torch.float32, device=dev)
    be = torch.tensor(p.beta[:1], dtype=torch.float32, device=dev)
    a = torch_api.loglik_grad_multi(t, c, p.T, mu, al[None], be, chunk=128)
    b = torch_api.loglik_grad(t, c, p.T, mu, al, be, beta_shared=True, chunk=128, path=2)
    torch.cuda.synchronize()
    assert abs(float(a[0]) - float(b[0])) <= 1e-9 * abs(float(b[0]))
    for x, y in zip(a[1:], b[1:]):
        x = x.cpu().numpy().reshape(-1)
        y = y.cpu().numpy().reshape(-1)
        assert float(np.max(np.abs(x - y))) <= 1e-6 * max(1.0, float(np.max(np.abs(y))))


def test_multi_kernel_large_prefix():
    """M = 1024, three kernels, 2e5 events (decays 0.3 .. 3)."""
    p = synth.random_problem_multi(1024, 200000, seed=57, kernels=3, rho=0.7)
    _check(p, _run(p), "M=1024 K=3 N=2e5")


def test_multi_kernel_autograd():
    import torch
    from paper_2604_01342_gb300 import torch_api
    p = synth.random_problem_multi(16, 4000, seed=58, kernels=2)
    t, c, T, mu, al, be = _dev(p)
    mu.requires_grad_(True); al.requires_grad_(True); be.requires_grad_(True)
    ll = torch_api.loglik_multi(t, c, T, mu, al, be)
    (-ll).backward()
    ref = _oracle(p)
    assert al.grad.shape == al.shape and be.grad.shape == be.shape
    np.testing.assert_allclose(-al.grad.cpu().numpy(), ref["dalpha"], rtol=0, atol=1e-4 * np.abs(ref["dalpha"]).max())
    np.testing.assert_allclose(-mu.grad.cpu().numpy(), ref["dmu"], rtol=0, atol=1e-4 * np.abs(ref["dmu"]).max())


def test_bad_decay_of_one_kernel_is_reported():
    import torch
    from paper_2604_01342_gb300 import binding, torch_api
    p = synth.random_problem_multi(8, 1000, seed=59, kernels=3)
    t, c, T, mu, al, be = _dev(p)
    be[1] = -1.0
    with pytest.raises(binding.HawkesError) as e:
        torch_api.loglik_grad_multi(t, c, T, mu, al, be)
    assert e.value.code == 5                          # HAWKES_ERR_PARAM_DOMAIN
    ll, dmu, dal, dbe = torch_api.loglik_grad_multi(t, c, T, mu, al, be, check=False)
    torch.cuda.synchronize()
    assert np.isnan(float(ll)) and np.isnan(dal.cpu().numpy()).all()


def test_multi_kernel_throughput():
    """Time of one call with three kernels on 1e6 events at M = 1024 (printed)."""
    import torch
    from paper_2604_01342_gb300 import torch_api
    p = synth.random_problem_multi(1024, 1_000_000, seed=60, kernels=3, rho=0.7)
    t, c, T, mu, al, be = _dev(p)
    for _ in range(2):
        torch_api.loglik_grad_multi(t, c, T, mu, al, be, check=False)
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(5):
        torch_api.loglik_grad_multi(t, c, T, mu, al, be, check=False)
    b.record(s)
    b.synchronize()
    ms = a.elapsed_time(b) / 5
    print(f"K=3, M=1024, N=1e6: {ms:.3f} ms per call = {1e6 / (ms * 1e-3):.3e} events/s")
