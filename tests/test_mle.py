"""Adam maximum-likelihood loop (paper, Algorithm 1 with the Section 4.3 optimizer) on top
of the exact log-likelihood and gradient.  CPU: the FP64 oracle as the gradient backend
(test infrastructure).  GPU: the CUDA library, step-by-step against the oracle backend."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_01342_gb300 import mle, synth


def oracle_fn(t, c, T, mu, alpha, beta, shared):
    M = mu.shape[0]
    b = beta.double().reshape(-1).cpu().numpy()
    b = np.full(M, b[0]) if shared else b
    r = oracle.loglik_grad(t.cpu().numpy(), c.cpu().numpy(), T, mu.double().cpu().numpy(),
                           alpha.double().cpu().numpy(), b)
    db = np.array([r["dbeta"].sum()]) if shared else r["dbeta"]
    dev = mu.device
    return (torch.tensor(r["ll"], dtype=torch.float64, device=dev),
            torch.from_numpy(r["dmu"]).to(dev), torch.from_numpy(r["dalpha"]).to(dev),
            torch.from_numpy(db).to(dev))


def _start(p, shared, seed=0, dev="cpu"):
    rng = np.random.default_rng(seed)
    f = lambda a: torch.tensor(a * rng.uniform(0.8, 1.2, size=np.shape(a)), device=dev)  # noqa
    beta = p.beta[:1] if shared else p.beta
    return f(p.mu), f(p.alpha), f(beta)


@pytest.mark.parametrize("shared", [True, False])
def test_adam_decreases_nll_and_beats_truth(shared):
    p = synth.random_problem(3, 3000, 21, shared)
    mu0, al0, be0 = _start(p, shared)
    fit = mle.AdamMLE(torch.from_numpy(p.t), torch.from_numpy(p.c), p.T, mu0, al0, be0, shared,
                      lr=0.02, loglik_grad_fn=oracle_fn)
    st = fit.fit(200)
    assert st.nll[-1] < st.nll[0]
    truth = oracle.loglik(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    # the MLE is at least as likely as the simulating parameters
    assert st.loglik[-1] >= truth - 1e-3 * abs(truth)
    assert torch.all(fit.alpha >= 0) and torch.all(fit.mu > 0) and torch.all(fit.beta > 0)


def test_penalty_gradient_is_offdiagonal_hinge():
    p = synth.random_problem(3, 500, 22, True)
    mu0, al0, be0 = _start(p, True)
    al0 = al0.clone()
    al0[0, 1] = 0.01   # below the hinge
    al0[1, 1] = 0.01   # diagonal: not penalised
    fit = mle.AdamMLE(torch.from_numpy(p.t), torch.from_numpy(p.c), p.T, mu0, al0, be0, True,
                      lam1=0.5, h=0.05, loglik_grad_fn=oracle_fn)
    nll, ll, (g_mu, g_al, g_be) = fit.objective()
    fit0 = mle.AdamMLE(torch.from_numpy(p.t), torch.from_numpy(p.c), p.T, mu0, al0, be0, True,
                       lam1=0.0, loglik_grad_fn=oracle_fn)
    _, _, (_, g_al0, _) = fit0.objective()
    diff = (g_al - g_al0).numpy()
    assert diff[0, 1] == pytest.approx(0.5)
    assert diff[1, 1] == 0.0
    assert np.all(diff[np.asarray(al0) >= 0.05] == 0.0)


@pytest.mark.gpu
def test_gpu_adam_tracks_oracle_backend():
    p = synth.workload(1, n_events=10_000)
    dev = torch.device("cuda")
    mu0, al0, be0 = _start(p, True, dev=dev)
    t = torch.from_numpy(p.t).to(dev)
    c = torch.from_numpy(p.c).to(dev)
    g = mle.AdamMLE(t, c, p.T, mu0, al0, be0, True, lr=0.05)
    o = mle.AdamMLE(t, c, p.T, mu0, al0, be0, True, lr=0.05, loglik_grad_fn=oracle_fn)
    for _ in range(5):
        a, b = g.step(), o.step()
        assert a == pytest.approx(b, rel=1e-6)
    g.fit(295)
    # recovery on 1e4 events of the 4-node workload (truth: mu, alpha, beta of workload 1)
    err_mu = mle.relative_l2(g.mu, torch.tensor(p.mu))
    err_al = mle.relative_l2(g.alpha, torch.tensor(p.alpha))
    err_be = mle.relative_l2(g.beta, torch.tensor(p.beta[:1]))
    print(f"recovery after 300 steps: mu {err_mu:.3f}, alpha {err_al:.3f}, beta {err_be:.3f}")
    assert g.state.nll[-1] < g.state.nll[0]
    assert err_be < 0.2 and err_mu < 0.3 and err_al < 0.5
