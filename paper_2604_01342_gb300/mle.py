"""Maximum-likelihood fitting on top of the exact log-likelihood and gradient.

The paper's training loop (Algorithm 1, and Section 4.3: Adam with learning rate 0.05)
alternates one exact log-likelihood + gradient pass with one optimizer step on the
per-event objective of Section 2,

    NLL(mu, alpha, beta) = -L / N + lam1 * sum_{p != q} alpha_pq 1{alpha_pq < h},

with the l1-hinge penalty on the off-diagonal entries (the prose of Section 2; the
printed formula sums over all entries, the prose excludes self-influence).  With
``support=True`` the interactions are those of the starting alpha's support (a sparse
model): the library returns the gradient on that support and zero elsewhere, and the
support entries are optimised as log alpha (the paper does not say how it keeps alpha
non-negative; on a support of positive entries of very different sizes a log
parametrisation makes every Adam step a relative change).  Positivity is
kept by optimising log mu and log beta, and by projecting alpha onto alpha >= 0 after
each step.  The gradient pass is one call of the library (``torch_api.loglik_grad``);
the Adam update itself is a few elementwise tensor operations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from . import torch_api


@dataclass
class FitState:
    step: int = 0
    nll: list = field(default_factory=list)
    loglik: list = field(default_factory=list)


class AdamMLE:
    """Adam on (log mu, alpha, log beta) for one event sequence on one GPU.

    ``loglik_grad_fn(t, c, T, mu, alpha, beta, shared) -> (L, dmu, dalpha, dbeta)`` may be
    replaced (the tests pass an FP64 reference); the default is the CUDA library."""

    def __init__(self, t, c, T, mu0, alpha0, beta0, beta_shared: bool, lr: float = 0.05,
                 lam1: float = 0.0, h: float = 0.05, betas=(0.9, 0.999), eps: float = 1e-8,
                 loglik_grad_fn=None, support: bool = False):
        self.t, self.c, self.T = t, c, float(T)
        self.N = int(t.shape[0])
        self.shared = bool(beta_shared)
        dev = mu0.device
        self.log_mu = torch.log(mu0.detach().double().clone()).to(dev)
        self.alpha = alpha0.detach().double().clone().to(dev)
        self.log_beta = torch.log(beta0.detach().double().reshape(-1).clone()).to(dev)
        self.support = False
        self.lr, self.lam1, self.h = lr, lam1, h
        self.b1, self.b2 = betas
        self.eps = eps
        self.m = [torch.zeros_like(x) for x in self.params()]
        self.v = [torch.zeros_like(x) for x in self.params()]
        self.state = FitState()
        self.support = bool(support)
        self.fn = loglik_grad_fn or self._cuda_fn
        M = self.alpha.shape[0]
        self.offdiag = 1.0 - torch.eye(M, dtype=torch.float64, device=dev)
        if self.support:
            # a sparse model: the interactions are the entries of alpha0's support, all
            # positive, optimised in log space like mu and beta (an Adam step is then a
            # relative change of each entry, whatever its scale); entries outside the
            # support stay 0 and have no penalty
            self.mask = (self.alpha != 0)
            self.log_alpha = torch.where(self.mask, torch.log(torch.where(
                self.mask, self.alpha, torch.ones_like(self.alpha))), torch.zeros_like(self.alpha))
            self.offdiag = self.offdiag * self.mask.double()
            self.m = [torch.zeros_like(x) for x in self.params()]
            self.v = [torch.zeros_like(x) for x in self.params()]

    def _cuda_fn(self, t, c, T, mu, alpha, beta, shared):
        ll, dmu, dal, dbe = torch_api.loglik_grad(t, c, T, mu.float(), alpha.float(),
                                                  beta.float(), beta_shared=shared,
                                                  support=self.support)
        return ll.double(), dmu.double(), dal.double(), dbe.double()

    def params(self):
        if self.support:
            return [self.log_mu, self.log_alpha, self.log_beta]
        return [self.log_mu, self.alpha, self.log_beta]

    def _sync_alpha(self):
        if self.support:
            self.alpha = torch.where(self.mask, torch.exp(self.log_alpha),
                                     torch.zeros_like(self.log_alpha))

    @property
    def mu(self):
        return torch.exp(self.log_mu)

    @property
    def beta(self):
        return torch.exp(self.log_beta)

    def objective(self):
        """(NLL, L, gradients of NLL w.r.t. log mu, alpha, log beta) at the current point."""
        mu, beta = self.mu, self.beta
        ll, dmu, dal, dbe = self.fn(self.t, self.c, self.T, mu, self.alpha, beta, self.shared)
        self.last_loglik_grads = (dmu, dal, dbe)      # of L at this point, for inspection
        ll = ll.reshape(())
        pen_mask = (self.alpha < self.h).double() * self.offdiag
        nll = -ll / self.N + self.lam1 * torch.sum(self.alpha * pen_mask)
        g_logmu = -(dmu * mu) / self.N
        g_alpha = -dal / self.N + self.lam1 * pen_mask
        if self.support:
            g_alpha = torch.where(self.mask, g_alpha * self.alpha, torch.zeros_like(g_alpha))
        g_logbeta = -(dbe.reshape(-1) * beta) / self.N
        return nll, ll, [g_logmu, g_alpha, g_logbeta]

    def step(self):
        nll, ll, grads = self.objective()
        self.last_grads = self.last_loglik_grads
        self.state.step += 1
        k = self.state.step
        for x, g, m, v in zip(self.params(), grads, self.m, self.v):
            m.mul_(self.b1).add_(g, alpha=1 - self.b1)
            v.mul_(self.b2).addcmul_(g, g, value=1 - self.b2)
            mhat = m / (1 - self.b1 ** k)
            vhat = v / (1 - self.b2 ** k)
            x.sub_(self.lr * mhat / (torch.sqrt(vhat) + self.eps))
        if self.support:
            self._sync_alpha()
        else:
            self.alpha.clamp_(min=0.0)
        self.state.nll.append(float(nll))
        self.state.loglik.append(float(ll))
        return float(nll)

    def fit(self, steps: int):
        for _ in range(steps):
            self.step()
        return self.state


def relative_l2(est: torch.Tensor, truth: torch.Tensor) -> float:
    """||est - truth|| / ||truth|| (the parameter-recovery error of Section 4.3)."""
    est = est.double().reshape(-1)
    truth = truth.double().reshape(-1).to(est.device)
    n = float(torch.linalg.norm(truth))
    return float(torch.linalg.norm(est - truth)) / (n if n > 0 else 1.0) if not math.isnan(n) else n
