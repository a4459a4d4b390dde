"""Maximum-likelihood fitting of the fifth workload (paper, Algorithm 1 with the Adam
optimizer of Section 4.3): M=4096 marks with one decay each, alpha 1% dense at spectral
radius 0.85, N=5e7 events on [0, T ~ 1e7].  The fit runs on the support of the simulating
alpha (the library's support option); it starts from the truth with every parameter
multiplied by U[0.8, 1.2] (seeded).

  * A 1e6-event prefix, 8 steps: the log-likelihood of every step and the gradient of the
    first and last step against the FP64 oracle (lazy per-component form), at the stated
    tolerances, evaluated at the FP32 parameters the GPU received.
  * The whole stream, 50 steps: the log-likelihood at steps 0, 10, 20, 30, 40 and 49 and the
    gradient at steps 0 and 49 against the oracle (a documented subset: one oracle
    evaluation takes tens of seconds on one host core; the six run in spawned processes
    after the fit), and the relative l2 error of mu, alpha (on its support) and beta against
    the simulating parameters at every step (the recovery measure of Section 4.3)."""
import multiprocessing as mp
import os
import tempfile
import time

import numpy as np
import pytest

from helpers import GRAD_RTOL, LL_RTOL, f32, maxnorm_rel, rel_err, support_oracle_from_files
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c5():
    return synth.workload(5)


def _start(p, dev, seed=5):
    import torch
    rng = np.random.default_rng(seed)
    f = lambda a: torch.tensor(a * rng.uniform(0.8, 1.2, size=np.shape(a)), device=dev)  # noqa
    return f(p.mu), f(p.alpha), f(p.beta)


def _fit(p, steps, record_at):
    """Runs Adam; returns per-step log-likelihoods, the FP32 parameters at the steps in
    record_at, recovery errors and the step times."""
    import torch
    from paper_2604_01342_gb300 import mle
    dev = torch.device("cuda")
    mu0, al0, be0 = _start(p, dev)
    t = torch.from_numpy(p.t).to(dev)
    c = torch.from_numpy(p.c).to(dev)
    fit = mle.AdamMLE(t, c, p.T, mu0, al0, be0, False, lr=0.05, support=True)
    sup = torch.from_numpy(p.alpha != 0).to(dev)
    truth = (torch.tensor(p.mu), torch.tensor(p.alpha[p.alpha != 0]), torch.tensor(p.beta))
    params, errs, ms = {}, [], []
    for k in range(steps):
        if k in record_at:
            params[k] = (fit.mu.float().cpu().numpy(), fit.alpha.float().cpu().numpy(),
                         fit.beta.float().cpu().numpy())
        errs.append((mle.relative_l2(fit.mu, truth[0]), mle.relative_l2(fit.alpha[sup], truth[1]),
                     mle.relative_l2(fit.beta, truth[2])))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fit.step()
        torch.cuda.synchronize()
        ms.append(1e3 * (time.perf_counter() - t0))
        if k in record_at:
            params[k] = params[k] + (fit.last_grads,)
    return fit, params, errs, ms


def _grads_of_step(fit_grads):
    return [g.double().cpu().numpy() for g in fit_grads]


def test_mle_workload5_prefix_every_step(c5):
    import oracle
    p0 = c5
    n = 1_000_000
    p = synth.Problem(t=p0.t[:n].copy(), c=p0.c[:n].copy(), T=float(p0.t[n - 1]), mu=p0.mu,
                      alpha=p0.alpha, beta=p0.beta, shared_beta=False)
    steps = 8
    fit, params, errs, _ = _fit(p, steps, set(range(steps)))
    for k in range(steps):
        mu, al, be, g = params[k]
        ref = oracle.loglik_grad_support(p.t, p.c, p.T, mu.astype(np.float64),
                                         al.astype(np.float64), be.astype(np.float64))
        assert rel_err(fit.state.loglik[k], ref["ll"]) <= LL_RTOL, k
        if k in (0, steps - 1):
            dmu, dal, dbe = _grads_of_step(g)
            assert maxnorm_rel(dmu, ref["dmu"]) <= GRAD_RTOL
            assert maxnorm_rel(dal, ref["dalpha"]) <= GRAD_RTOL
            assert maxnorm_rel(dbe, ref["dbeta"]) <= GRAD_RTOL
    assert fit.state.nll[-1] < fit.state.nll[0]


def test_mle_workload5_full_50_steps(c5):
    p = c5
    check = (0, 10, 20, 30, 40, 49)
    fit, params, errs, ms = _fit(p, 50, set(check))
    lines = [f"fifth workload: M={p.M}, N={p.N}, T={p.T:.6g}; 50 Adam steps (lr 0.05) on "
             f"alpha's support; median {np.median(ms):.1f} ms per step (one exact "
             f"log-likelihood + gradient call and the update)",
             "step  L (GPU)                  rel l2 error: mu      alpha(support)  beta"]
    for k in range(50):
        lines.append(f"{k:4d}  {fit.state.loglik[k]: .10e}  {errs[k][0]:.5f}  {errs[k][1]:.5f}  "
                     f"{errs[k][2]:.5f}")
    # oracle checks in spawned processes (this process holds a CUDA context)
    with tempfile.TemporaryDirectory() as d:
        np.save(os.path.join(d, "t.npy"), p.t)
        np.save(os.path.join(d, "c.npy"), p.c)
        np.save(os.path.join(d, "T.npy"), np.array(p.T))
        jobs = []
        for k in check:
            mu, al, be, _ = params[k]
            names = []
            for nm, a in (("mu", mu), ("al", al), ("be", be)):
                path = os.path.join(d, f"{nm}{k}.npy")
                np.save(path, a.astype(np.float64))
                names.append(path)
            jobs.append((os.path.join(d, "t.npy"), os.path.join(d, "c.npy"),
                         os.path.join(d, "T.npy"), *names))
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
            refs = pool.map(support_oracle_from_files, jobs)
        oracle_s = time.perf_counter() - t0
    lines.append(f"oracle checks ({len(check)} evaluations in spawned processes, "
                 f"{oracle_s:.0f} s):")
    ok = True
    for k, ref in zip(check, refs):
        e_ll = rel_err(fit.state.loglik[k], ref["ll"])
        msg = f"  step {k:2d}: L rel err {e_ll:.3e}"
        ok &= e_ll <= LL_RTOL
        if k in (0, 49):
            dmu, dal, dbe = _grads_of_step(params[k][3])
            e = (maxnorm_rel(dmu, ref["dmu"]), maxnorm_rel(dal, ref["dalpha"]),
                 maxnorm_rel(dbe, ref["dbeta"]))
            msg += f"; dmu {e[0]:.3e}, dalpha {e[1]:.3e}, dbeta {e[2]:.3e}"
            ok &= max(e) <= GRAD_RTOL
        lines.append(msg)
    print("\n".join(lines))
    assert ok
    assert fit.state.nll[-1] < fit.state.nll[0]
