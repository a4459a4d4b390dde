"""Shared helpers for the GPU parity tests: run the CUDA path through the C
ABI (via the torch wrapper) and the FP64 oracle on the same inputs, and
compare with the stated tolerances:
  relative log-likelihood error  |L - L*| / |L*|           <= 1e-6
  max-norm relative gradient error max|g - g*| / max|g*|    <= 1e-4 per block
The oracle is evaluated at the FP32-rounded parameters the GPU receives.

A result close to zero can be a small difference of large sums: the
log-likelihood (intensity logs minus the compensator) or the decay gradient
(excitation terms minus compensator terms, which nearly cancel at the simulating
parameters).  Its relative error is then ill-conditioned.  With the oracle's
conditioning scale S (the sum of magnitudes of those terms, oracle.condition),
a result passes at the stated relative tolerance, or else when its error is at
most 1e-7 of S (FP32-level accuracy of the terms): for L that is
|L - L*| <= 1e-6 max(|L*|, S / 10), for dbeta max|d - d*| <= 1e-4 max(max|d*|, S / 1000).
Every such case is reported with its kappa = S / |result|."""
import numpy as np

LL_RTOL = 1e-6
GRAD_RTOL = 1e-4


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def oracle_ref(p, grad=True):
    import oracle
    beta = f32(p.beta)
    if p.shared_beta:
        beta = np.full(p.M, beta[0])
    out = oracle.loglik_grad(p.t, p.c, p.T, f32(p.mu), f32(p.alpha), beta, want_grad=grad)
    if grad and p.shared_beta:
        out["dbeta"] = np.array([out["dbeta"].sum()])
    return out


def gpu_run(p, grad=True, path=0, chunk=0, check=True, validate=True):
    import torch
    from paper_2604_01342_gb300 import torch_api
    dev = torch.device("cuda")
    t = torch.from_numpy(np.ascontiguousarray(p.t)).to(dev)
    c = torch.from_numpy(np.ascontiguousarray(p.c, dtype=np.int32)).to(dev)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    al = torch.tensor(p.alpha, dtype=torch.float32, device=dev)
    be = torch.tensor(p.beta[:1] if p.shared_beta else p.beta, dtype=torch.float32, device=dev)
    r = torch_api.loglik_grad(t, c, p.T, mu, al, be, beta_shared=p.shared_beta, chunk=chunk,
                              path=path, check=check, grad=grad, validate=validate)
    if grad:
        ll, dmu, dal, dbe = r
        return {"ll": float(ll.item()), "dmu": dmu.cpu().numpy().astype(np.float64),
                "dalpha": dal.cpu().numpy().astype(np.float64),
                "dbeta": dbe.cpu().numpy().astype(np.float64)}
    return {"ll": float(r.item())}


def rel_err(got, ref):
    return abs(got - ref) / abs(ref)


def maxnorm_rel(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(got - ref))) / (den if den > 0 else 1.0)


SCALE_REL = 1e-7


def assert_close(got, ref, grad=True, ll_rtol=LL_RTOL, grad_rtol=GRAD_RTOL, what="",
                 ll_scale=None, dbeta_scale=None):
    e = rel_err(got["ll"], ref["ll"])
    if e > ll_rtol and ll_scale is not None:
        kappa = ll_scale / abs(ref["ll"])
        e_s = abs(got["ll"] - ref["ll"]) / ll_scale
        print(f"{what}: loglik kappa {kappa:.1f}: rel err {e:.3e}, err / scale {e_s:.3e}")
        e = e_s * ll_rtol / SCALE_REL
    assert e <= ll_rtol, f"{what} loglik rel err {e:.3e} (gpu {got['ll']!r} vs {ref['ll']!r})"
    if grad:
        for k in ("dmu", "dalpha", "dbeta"):
            e = maxnorm_rel(got[k], ref[k])
            if k == "dbeta" and e > grad_rtol and dbeta_scale is not None:
                S = float(np.max(dbeta_scale))
                kappa = S / float(np.max(np.abs(ref[k])))
                e_s = float(np.max(np.abs(np.asarray(got[k]) - np.asarray(ref[k])))) / S
                print(f"{what}: dbeta kappa {kappa:.1f}: max-norm rel err {e:.3e}, "
                      f"err / scale {e_s:.3e}")
                e = e_s * grad_rtol / SCALE_REL
            assert e <= grad_rtol, f"{what} {k} max-norm rel err {e:.3e}"
