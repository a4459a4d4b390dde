"""Parity at the benchmark's sizes, in the launch configuration bench.py times
(default chunk, automatic path), on what the FP64 oracle can finish in seconds:
  * the M=1024 shared-decay stream: the full 1e7-event run must be finite and
    satisfy the Euler identity of the 1-homogeneous (mu, alpha); a 2e5-event
    prefix of the same stream is compared with the oracle element by element;
  * the M=64 per-source stream of 1e6 events: compared with the oracle in full;
  * the 4,096-sequence batch of M=8 sequences: compared with the oracle in full.
"""
import numpy as np
import pytest

from helpers import assert_close, f32, gpu_run, maxnorm_rel, oracle_ref, rel_err
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c4():
    return synth.workload(4)


def _prefix(p, n):
    q = synth.Problem(t=p.t[:n].copy(), c=p.c[:n].copy(), T=float(p.t[n - 1]), mu=p.mu,
                      alpha=p.alpha, beta=p.beta, shared_beta=p.shared_beta, name=p.name)
    return q


def test_m1024_prefix_matches_oracle(c4):
    import oracle
    p = _prefix(c4, 200_000)
    got = gpu_run(p)
    ref = oracle_ref(p)
    for k in ("dmu", "dalpha", "dbeta"):
        print(f"M=1024 prefix 2e5: {k} max-norm rel err {maxnorm_rel(got[k], ref[k]):.3e}")
    print(f"M=1024 prefix 2e5: loglik rel err {rel_err(got['ll'], ref['ll']):.3e}")
    sc = oracle.condition(p.t, p.c, p.T, f32(p.mu), f32(p.alpha), np.full(p.M, f32(p.beta)[0]))
    assert_close(got, ref, what="M=1024 prefix", ll_scale=sc["ll"],
                 dbeta_scale=np.array([sc["dbeta"].sum()]))


def test_m1024_full_size_identities(c4):
    p = c4
    got = gpu_run(p)
    assert np.isfinite(got["ll"]) and all(np.all(np.isfinite(got[k]))
                                          for k in ("dmu", "dalpha", "dbeta"))
    # Euler identity: sum mu dmu + sum alpha dalpha = N - Lambda(T), with the compensator
    # Lambda(T) computed here in FP64 from its closed form
    mu, al, be = f32(p.mu), f32(p.alpha), f32(p.beta)[0]
    colsum = al.sum(axis=0)
    comp = p.T * mu.sum() + float(np.sum(colsum[p.c] * -np.expm1(-be * (p.T - p.t))))
    lhs = float(np.dot(mu, got["dmu"]) + np.sum(al * got["dalpha"]))
    scale = float(np.dot(mu, np.abs(got["dmu"] + p.T)) + p.T * mu.sum() + p.N)
    print(f"M=1024 full: Euler residual {abs(lhs - (p.N - comp)) / scale:.3e} of its scale")
    assert abs(lhs - (p.N - comp)) <= 1e-4 * scale


def test_m64_per_source_full_size():
    p = synth.workload(2)
    got = gpu_run(p)
    ref = oracle_ref(p)
    for k in ("dmu", "dalpha", "dbeta"):
        print(f"M=64 1e6: {k} max-norm rel err {maxnorm_rel(got[k], ref[k]):.3e}")
    assert_close(got, ref, what="M=64 per-source 1e6")


def test_varlen_4096_full_size():
    import oracle
    import torch
    from paper_2604_01342_gb300 import torch_api
    vp = synth.workload(3)
    dev = torch.device("cuda")
    r = torch_api.loglik_grad_varlen(
        torch.from_numpy(vp.t).to(dev), torch.from_numpy(vp.c).to(dev),
        torch.from_numpy(vp.offsets).to(dev), torch.from_numpy(vp.T).to(dev),
        torch.tensor(vp.mu, dtype=torch.float32, device=dev),
        torch.tensor(vp.alpha, dtype=torch.float32, device=dev),
        torch.tensor(vp.beta, dtype=torch.float32, device=dev), beta_shared=False)
    ll, dmu, dal, dbe = [x.cpu().numpy().astype(np.float64) for x in r]
    ref = oracle.loglik_grad_varlen(vp.t, vp.c, vp.offsets, vp.T, f32(vp.mu), f32(vp.alpha),
                                    f32(vp.beta))
    worst = 0.0
    for s in range(vp.B):
        got = {"ll": ll[s], "dmu": dmu[s], "dalpha": dal[s], "dbeta": dbe[s]}
        want = {k: ref[k][s] for k in ("ll", "dmu", "dalpha", "dbeta")}
        scale = dscale = None
        if rel_err(got["ll"], want["ll"]) > 1e-6 or maxnorm_rel(got["dbeta"], want["dbeta"]) > 1e-4:
            a, b = vp.offsets[s], vp.offsets[s + 1]
            sc = oracle.condition(vp.t[a:b], vp.c[a:b], vp.T[s], f32(vp.mu[s]),
                                  f32(vp.alpha[s]), f32(vp.beta[s]))
            scale, dscale = sc["ll"], sc["dbeta"]
        assert_close(got, want, what=f"seq {s}", ll_scale=scale, dbeta_scale=dscale)
        worst = max(worst, rel_err(got["ll"], want["ll"]))
    print(f"varlen 4096 x M=8: worst per-sequence loglik rel err {worst:.3e}")
