"""CUDA-graph replay of whole calls, and the chunk/path autotuner.

The graphed call must reproduce the direct call and the FP64 oracle (stated tolerances),
follow in-place changes of its inputs between replays, and the autotuner must return one
of its candidates, cache it per shape, and its choice must meet the oracle.  A timing of
the batched workload (4,096 sequences) as one graph replay is printed."""
import numpy as np
import pytest

from helpers import assert_close, f32, maxnorm_rel, oracle_ref
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev_varlen(vp):
    import torch
    dev = torch.device("cuda")
    return (torch.from_numpy(vp.t).to(dev), torch.from_numpy(vp.c.astype(np.int32)).to(dev),
            torch.from_numpy(vp.offsets).to(dev), torch.from_numpy(vp.T).to(dev),
            torch.tensor(vp.mu, dtype=torch.float32, device=dev),
            torch.tensor(vp.alpha, dtype=torch.float32, device=dev),
            torch.tensor(vp.beta, dtype=torch.float32, device=dev))


def _dev_single(p):
    import torch
    dev = torch.device("cuda")
    return (torch.from_numpy(p.t).to(dev), torch.from_numpy(p.c.astype(np.int32)).to(dev), p.T,
            torch.tensor(p.mu, dtype=torch.float32, device=dev),
            torch.tensor(p.alpha, dtype=torch.float32, device=dev),
            torch.tensor(p.beta[:1] if p.shared_beta else p.beta, dtype=torch.float32, device=dev))


def _varlen_oracle(vp, mu=None):
    import oracle
    return oracle.loglik_grad_varlen(vp.t, vp.c, vp.offsets, vp.T, f32(vp.mu if mu is None else mu),
                                     f32(vp.alpha), f32(vp.beta))


def _check_varlen(out, ref, B):
    ll, dmu, dal, dbe = [x.cpu().numpy().astype(np.float64) for x in out]
    for s in range(B):
        assert_close({"ll": ll[s], "dmu": dmu[s], "dalpha": dal[s], "dbeta": dbe[s]},
                     {"ll": ref["ll"][s], "dmu": ref["dmu"][s], "dalpha": ref["dalpha"][s],
                      "dbeta": ref["dbeta"][s]}, what=f"seq {s}")


def test_graph_varlen_matches_direct_and_oracle():
    import torch
    from paper_2604_01342_gb300 import torch_api
    from paper_2604_01342_gb300.graphs import GraphedLogLikGrad
    vp = synth.varlen_workload(np.random.default_rng(21), 48, m=8, median=150, lo=0, hi=3000)
    t, c, off, T, mu, al, be = _dev_varlen(vp)
    g = GraphedLogLikGrad.varlen(t, c, off, T, mu, al, be, beta_shared=False, chunk=64)
    out = g.replay()
    torch.cuda.synchronize()
    assert g.status() == 0
    direct = torch_api.loglik_grad_varlen(t, c, off, T, mu, al, be, beta_shared=False, chunk=64)
    # accumulation order differs between runs (atomics), so compare block max-norms
    for a, b in zip(out, direct):
        assert maxnorm_rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
    _check_varlen(out, _varlen_oracle(vp), vp.B)


def test_graph_replay_follows_input_changes():
    import torch
    from paper_2604_01342_gb300.graphs import GraphedLogLikGrad
    vp = synth.varlen_workload(np.random.default_rng(22), 16, m=4, median=200, lo=1, hi=2000)
    t, c, off, T, mu, al, be = _dev_varlen(vp)
    g = GraphedLogLikGrad.varlen(t, c, off, T, mu, al, be, beta_shared=False)
    g.replay()
    mu.mul_(1.25)                                   # same tensor, new contents
    out = g.replay()
    torch.cuda.synchronize()
    _check_varlen(out, _varlen_oracle(vp, mu=vp.mu * 1.25), vp.B)


def test_graph_single_gemm_path():
    import torch
    from paper_2604_01342_gb300.graphs import GraphedLogLikGrad
    p = synth.random_problem(200, 6000, seed=23, shared_beta=True)
    t, c, T, mu, al, be = _dev_single(p)
    g = GraphedLogLikGrad.single(t, c, T, mu, al, be, beta_shared=True, chunk=96, path=2)
    for _ in range(3):
        ll, dmu, dal, dbe = g.replay()
    torch.cuda.synchronize()
    assert g.status() == 0
    got = {"ll": float(ll.item()), "dmu": dmu.cpu().numpy().astype(np.float64),
           "dalpha": dal.cpu().numpy().astype(np.float64),
           "dbeta": dbe.cpu().numpy().astype(np.float64)}
    assert_close(got, oracle_ref(p), what="graphed gemm path")


def test_autotune_returns_cached_valid_choice(tmp_path):
    import torch
    from paper_2604_01342_gb300 import autotune, torch_api
    p = synth.random_problem(48, 20000, seed=24, shared_beta=True)
    t, c, T, mu, al, be = _dev_single(p)
    path = str(tmp_path / "tune.json")
    best = autotune.tune(t, c, T, mu, al, be, beta_shared=True, cache_path=path)
    print("autotune:", best)
    cands = autotune._candidates(48, True, 1)
    assert (best["path"], best["chunk"], best["walk_lanes"]) in cands
    assert autotune.tune(t, c, T, mu, al, be, beta_shared=True, cache_path=path) is best
    # a new process (an empty memory cache) finds it in the file
    autotune._cache.clear()
    again = autotune.tune(t, c, T, mu, al, be, beta_shared=True, cache_path=path)
    assert (again["path"], again["chunk"], again["walk_lanes"]) == \
        (best["path"], best["chunk"], best["walk_lanes"])
    ll, dmu, dal, dbe = torch_api.loglik_grad(t, c, T, mu, al, be, beta_shared=True,
                                              chunk=best["chunk"], path=best["path"],
                                              walk_lanes=best["walk_lanes"])
    torch.cuda.synchronize()
    got = {"ll": float(ll.item()), "dmu": dmu.cpu().numpy().astype(np.float64),
           "dalpha": dal.cpu().numpy().astype(np.float64),
           "dbeta": dbe.cpu().numpy().astype(np.float64)}
    assert_close(got, oracle_ref(p), what="autotuned")


def test_batched_workload_as_one_graph():
    """The 4,096-sequence batch: tuned chunk, one graph replay per evaluation (timed)."""
    import torch
    from paper_2604_01342_gb300 import autotune
    from paper_2604_01342_gb300.graphs import GraphedLogLikGrad
    vp = synth.workload(3)
    t, c, off, T, mu, al, be = _dev_varlen(vp)
    best = autotune.tune(t, c, T, mu, al, be, beta_shared=False, offsets=off, cache_path=None)
    assert best["walk_lanes"] in (8, 16, 32)        # the lanes of a walker are tuned too (M = 8)
    g = GraphedLogLikGrad.varlen(t, c, off, T, mu, al, be, beta_shared=False,
                                 chunk=best["chunk"], path=best["path"],
                                 walk_lanes=best["walk_lanes"])
    for _ in range(3):
        g.replay()
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(10):
        g.replay()
    b.record(s)
    b.synchronize()
    ms = a.elapsed_time(b) / 10
    print(f"batched workload: {vp.B} sequences, {vp.t.shape[0]} events, tuned {best}: "
          f"{ms:.3f} ms per graph replay = {vp.t.shape[0] / (ms * 1e-3):.3e} events/s")
    assert g.status() == 0
    ll = g.outputs[0].cpu().numpy()
    assert np.all(np.isfinite(ll))
