"""The precision options of the chunk-GEMM path, measured on the CUDA path against the FP64
oracle (the error of each choice, per result):
  * reduce = 0 (FP64 partial sums of the log-intensities), 1 (Kahan-compensated FP32), 2
    (plain FP32): L at the stated tolerance for 0 and 1 on a well-conditioned stream; the
    plain FP32 sum is measured, not asserted to pass;
  * fp32_times = 1 (an ablation: time differences of times rounded to FP32 first) against the
    default FP64 differences, on a stream whose times are near 1e7: the default meets the
    tolerances, the ablation is far off (the reason for FP64 differences).
Every other output is the same across reduce modes (the option only changes the log-sum)."""
import numpy as np
import pytest

from helpers import assert_close, f32, maxnorm_rel, oracle_ref, rel_err
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(p, **kw):
    import torch
    from paper_2604_01342_gb300 import torch_api
    dev = torch.device("cuda")
    r = torch_api.loglik_grad(torch.from_numpy(p.t).to(dev), torch.from_numpy(p.c).to(dev), p.T,
                              torch.tensor(p.mu, dtype=torch.float32, device=dev),
                              torch.tensor(p.alpha, dtype=torch.float32, device=dev),
                              torch.tensor(p.beta[:1], dtype=torch.float32, device=dev),
                              beta_shared=True, path=2, **kw)
    return {"ll": float(r[0].item()), "dmu": r[1].cpu().numpy().astype(np.float64),
            "dalpha": r[2].cpu().numpy().astype(np.float64),
            "dbeta": r[3].cpu().numpy().astype(np.float64)}


def _errs(got, ref):
    return {"ll": rel_err(got["ll"], ref["ll"]),
            **{k: maxnorm_rel(got[k], ref[k]) for k in ("dmu", "dalpha", "dbeta")}}


def test_reduce_modes():
    p = synth.workload(4, n_events=300_000)
    ref = oracle_ref(p)
    res = {m: _run(p, reduce=m) for m in (0, 1, 2)}
    for m in (0, 1, 2):
        print(f"reduce={m}: " + ", ".join(f"{k} {v:.3e}" for k, v in _errs(res[m], ref).items()))
    assert_close(res[0], ref, what="reduce=0")
    assert_close(res[1], ref, what="reduce=1")
    for m in (1, 2):                      # only the log-sum differs
        for k in ("dmu", "dalpha", "dbeta"):
            assert maxnorm_rel(res[m][k], res[0][k]) < 1e-5
    assert rel_err(res[1]["ll"], ref["ll"]) < rel_err(res[2]["ll"], ref["ll"]) or \
        rel_err(res[2]["ll"], ref["ll"]) < 1e-7


def test_fp32_times_ablation():
    p = synth.random_problem(64, 100_000, 77, True, rho=0.6, time_shift=1e7)
    ref = oracle_ref(p)
    good = _run(p)
    bad = _run(p, fp32_times=True)
    e_good, e_bad = _errs(good, ref), _errs(bad, ref)
    print("FP64 time differences: " + ", ".join(f"{k} {v:.3e}" for k, v in e_good.items()))
    print("FP32 times (ablation): " + ", ".join(f"{k} {v:.3e}" for k, v in e_bad.items()))
    assert_close(good, ref, what="FP64 differences, times near 1e7")
    assert e_bad["ll"] > 100 * max(e_good["ll"], 1e-9)


def test_precision_options_elsewhere_are_rejected():
    import ctypes
    from paper_2604_01342_gb300 import binding as B
    lib = B.lib()
    for opts in (B.make_opts(False, 0, True, 1, reduce=1), B.make_opts(True, 0, True, 1, fp32_times=True),
                 B.make_opts(True, 0, True, 2, kernels=2, reduce=1)):
        assert lib.hawkes_workspace_size(1000, 8, 1, 1, ctypes.byref(opts)) == 0
    assert lib.hawkes_workspace_size(1000, 8, 1, 1, ctypes.byref(B.make_opts(True, 0, True, 2, reduce=3))) == 0
