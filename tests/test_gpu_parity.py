"""CUDA path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

from helpers import assert_close, gpu_run, maxnorm_rel, oracle_ref, rel_err
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


# ----------------------------------------------------------- state-walk path
@pytest.mark.parametrize("m", [1, 3, 8, 31, 33, 64])
@pytest.mark.parametrize("shared", [False, True])
def test_walk_matches_oracle(m, shared):
    p = synth.random_problem(m, 3000 + 7 * m, 100 + m, shared)
    assert_close(gpu_run(p, path=1), oracle_ref(p), what=f"walk m={m}")


@pytest.mark.parametrize("chunk", [1, 7, 32, 33, 128, 1000])
def test_walk_chunk_sizes(chunk):
    p = synth.random_problem(12, 2500, 7, False)
    assert_close(gpu_run(p, path=1, chunk=chunk), oracle_ref(p), what=f"chunk {chunk}")


@pytest.mark.parametrize("m", [65, 100, 256])
def test_walk_forward_only_larger_m(m):
    p = synth.random_problem(m, 2000, 300 + m, False, rho=0.5)
    assert_close(gpu_run(p, path=1, grad=False), oracle_ref(p, grad=False), grad=False)


# ------------------------------------------------------------ chunk-GEMM path
# (300, 64), (1500, 192): several backward row blocks per mark block, the last one partial;
# (4096, 192): row blocks of 8 marks
@pytest.mark.parametrize("m,chunk", [(5, 16), (16, 64), (100, 32), (130, 64), (256, 128),
                                     (300, 64), (1500, 192), (4096, 192)])
def test_gemm_path_matches_oracle(m, chunk):
    p = synth.random_problem(m, 4000, 500 + m, True, rho=0.6)
    assert_close(gpu_run(p, path=2, chunk=chunk), oracle_ref(p), what=f"gemm m={m} C={chunk}")


def test_gemm_path_large_m():
    """M = 8192 (64 mark blocks): the scan and epilogue kernels opt in to more than 48 KB
    of shared memory per block."""
    p = synth.random_problem(8192, 4000, 63, True, rho=0.5)
    assert_close(gpu_run(p, path=2, chunk=128), oracle_ref(p), what="gemm path M=8192")


def test_gemm_path_forward_only():
    p = synth.random_problem(200, 3000, 9, True)
    assert_close(gpu_run(p, path=2, grad=False), oracle_ref(p, grad=False), grad=False)


def test_paths_agree():
    p = synth.random_problem(48, 5000, 11, True)
    a = gpu_run(p, path=1)
    b = gpu_run(p, path=2, chunk=64)
    assert rel_err(a["ll"], b["ll"]) < 1e-6
    for k in ("dmu", "dalpha", "dbeta"):
        assert maxnorm_rel(a[k], b[k]) < 1e-4


# --------------------------------------------------------------- edge cases
@pytest.mark.parametrize("path", [1, 2])
def test_empty_sequence(path):
    p = synth.random_problem(6, 10, 1, True)
    p.t = p.t[:0]; p.c = p.c[:0]; p.T = 3.5
    assert_close(gpu_run(p, path=path), oracle_ref(p))


@pytest.mark.parametrize("path", [1, 2])
def test_single_event(path):
    p = synth.random_problem(6, 1, 2, True)
    p.T = p.t[0] + 0.75
    assert_close(gpu_run(p, path=path), oracle_ref(p))


@pytest.mark.parametrize("path", [1, 2])
def test_ties(path):
    p = synth.random_problem(5, 600, 3, True)
    p.t = np.round(p.t, 1)           # many equal times
    assert_close(gpu_run(p, path=path, chunk=16), oracle_ref(p))


@pytest.mark.parametrize("path,shared", [(1, False), (1, True), (2, True)])
def test_large_absolute_times(path, shared):
    # FP64 differences of times near 1e7, as in long observation windows
    p = synth.random_problem(7, 3000, 4, shared, time_shift=1e7)
    assert_close(gpu_run(p, path=path, chunk=64), oracle_ref(p))


def test_long_gaps():
    p = synth.random_problem(4, 800, 5, False)
    p.t = p.t.copy()
    p.t[400:] += 500.0               # one long quiet period inside a chunk
    p.T += 500.0
    assert_close(gpu_run(p, path=1, chunk=512), oracle_ref(p))


@pytest.mark.parametrize("m,shared,mu_range", [(3, False, (0.1, 1.0)), (3, True, (0.1, 1.0)),
                                               (40, False, (0.01, 0.1)),
                                               (40, True, (0.006, 0.06))])
def test_walk_batches_past_the_factorised_limit(m, shared, mu_range):
    """Fast decays and sparse events: beta times the span of 32 events is above the limit
    of the factorised batch walk (64) for part of the batches, which are then walked event
    by event, mixed with factorised batches inside clusters."""
    p = synth.random_problem(m, 3000, 400 + m, shared, beta_range=(4.0, 12.0), mu_range=mu_range)
    beta = np.full(m, p.beta[0]) if shared else p.beta
    t = p.t
    span = np.array([t[min(i + 31, len(t) - 1)] - t[i] for i in range(0, len(t), 32)])
    wide = np.mean(float(beta.max()) * span > 64.0)
    assert 0.2 < wide < 0.9, wide                     # both forms occur
    assert_close(gpu_run(p, path=1, chunk=96), oracle_ref(p), what=f"walk past limit m={m}")


@pytest.mark.parametrize("path,shared", [(1, False), (2, True)])
def test_without_validation(path, shared):
    """validate=False skips the device checks and the mark counts: the chunk-GEMM path then
    centres nothing and counts the marks of its compensator in the epilogue."""
    p = synth.random_problem(40, 5000, 61, shared)
    assert_close(gpu_run(p, path=path, chunk=96, validate=False), oracle_ref(p),
                 what=f"unvalidated path {path}")


def test_chunk_invariance_gemm():
    p = synth.random_problem(64, 6000, 6, True)
    res = [gpu_run(p, path=2, chunk=C) for C in (8, 64, 256, 1024)]
    for r in res[1:]:
        assert rel_err(r["ll"], res[0]["ll"]) < 1e-6
        for k in ("dmu", "dalpha", "dbeta"):
            assert maxnorm_rel(r[k], res[0][k]) < 1e-4


# ------------------------------------------------------------ integer work
def test_mark_counts_bit_exact():
    import torch
    import oracle
    from paper_2604_01342_gb300 import binding, torch_api
    p = synth.random_problem(37, 5000, 8, False)
    gpu_run(p, path=1, chunk=64)
    torch.cuda.synchronize()
    ws = next(iter(torch_api._ws_cache.values()))
    off = binding.hawkes_mark_counts_ptr(ws.data_ptr()) - ws.data_ptr()
    got = ws[off: off + 8 * 37].view(torch.int64).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.mark_counts(p.c, 37))


def test_varlen_counts_bit_exact():
    import torch
    from paper_2604_01342_gb300 import binding, torch_api
    rng = np.random.default_rng(3)
    vp = synth.varlen_workload(rng, 9, m=5, median=200, lo=0, hi=2000)
    run_varlen(vp, chunk=64)
    torch.cuda.synchronize()
    ws = next(iter(torch_api._ws_cache.values()))
    off = binding.hawkes_mark_counts_ptr(ws.data_ptr()) - ws.data_ptr()
    got = ws[off: off + 8 * 9 * 5].view(torch.int64).cpu().numpy().reshape(9, 5)
    for s in range(9):
        a, b = vp.offsets[s], vp.offsets[s + 1]
        np.testing.assert_array_equal(got[s], np.bincount(vp.c[a:b], minlength=5))


# ------------------------------------------------------------------ varlen
def run_varlen(vp, chunk=0, grad=True):
    import torch
    from paper_2604_01342_gb300 import torch_api
    dev = torch.device("cuda")
    t = torch.from_numpy(vp.t).to(dev)
    c = torch.from_numpy(vp.c.astype(np.int32)).to(dev)
    off = torch.from_numpy(vp.offsets).to(dev)
    T = torch.from_numpy(vp.T).to(dev)
    mu = torch.tensor(vp.mu, dtype=torch.float32, device=dev)
    al = torch.tensor(vp.alpha, dtype=torch.float32, device=dev)
    be = torch.tensor(vp.beta, dtype=torch.float32, device=dev)
    r = torch_api.loglik_grad_varlen(t, c, off, T, mu, al, be, beta_shared=False, chunk=chunk,
                                     grad=grad)
    return [x.cpu().numpy().astype(np.float64) for x in r] if grad else [r.cpu().numpy()]


def varlen_ref(vp):
    import oracle
    from helpers import f32
    return oracle.loglik_grad_varlen(vp.t, vp.c, vp.offsets, vp.T, f32(vp.mu), f32(vp.alpha),
                                     f32(vp.beta))


@pytest.mark.parametrize("chunk", [16, 128])
def test_varlen_matches_oracle(chunk):
    rng = np.random.default_rng(12)
    vp = synth.varlen_workload(rng, 37, m=8, median=150, sigma=1.0, lo=0, hi=3000)
    ll, dmu, dal, dbe = run_varlen(vp, chunk=chunk)
    ref = varlen_ref(vp)
    for s in range(vp.B):
        got = {"ll": ll[s], "dmu": dmu[s], "dalpha": dal[s], "dbeta": dbe[s]}
        want = {"ll": ref["ll"][s], "dmu": ref["dmu"][s], "dalpha": ref["dalpha"][s],
                "dbeta": ref["dbeta"][s]}
        assert_close(got, want, what=f"seq {s} (n={vp.offsets[s+1]-vp.offsets[s]})")


def test_varlen_equals_single_calls():
    rng = np.random.default_rng(13)
    vp = synth.varlen_workload(rng, 5, m=3, median=300, lo=1, hi=2000)
    ll, dmu, dal, dbe = run_varlen(vp, chunk=64)
    for s in range(vp.B):
        a, b = vp.offsets[s], vp.offsets[s + 1]
        p = synth.Problem(t=vp.t[a:b], c=vp.c[a:b], T=float(vp.T[s]), mu=vp.mu[s],
                          alpha=vp.alpha[s], beta=vp.beta[s], shared_beta=False)
        one = gpu_run(p, path=1, chunk=64)
        assert rel_err(ll[s], one["ll"]) < 1e-7
        assert maxnorm_rel(dal[s], one["dalpha"]) < 1e-5


# ------------------------------------------------------------ error statuses
@pytest.mark.parametrize("case,code", [("unsorted", 2), ("mark", 3), ("time", 4),
                                       ("param", 5)])
def test_device_status(case, code):
    from paper_2604_01342_gb300 import binding
    p = synth.random_problem(4, 300, 9, False)
    if case == "unsorted":
        p.t = p.t.copy(); p.t[100], p.t[101] = p.t[101] + 0.5, p.t[100]
    elif case == "mark":
        p.c = p.c.copy(); p.c[50] = 4
    elif case == "time":
        p.T = float(p.t[-1]) * 0.5
    elif case == "param":
        p.alpha = p.alpha.copy(); p.alpha[1, 2] = -0.25
    with pytest.raises(binding.HawkesError) as ei:
        gpu_run(p, path=1)
    assert ei.value.code == code
    out = gpu_run(p, path=1, check=False)
    assert np.isnan(out["ll"]) and np.all(np.isnan(out["dalpha"]))


def test_host_errors():
    from paper_2604_01342_gb300 import binding
    opts = binding.make_opts(False, 0, True, 0)
    assert binding.lib().hawkes_workspace_size(10, 0, 1, 1, opts) == 0
    with pytest.raises(binding.HawkesError) as ei:
        binding.hawkes_loglik(None, None, 5, 1.0, 3, None, None, None, opts, None, 0, None, None)
    assert ei.value.code == 1


def test_gemm_path_fixed_point_overflow_falls_back():
    """One mark dominates and the decay is slow, so that a single cell of the backward pair
    tile collects far more than the fixed-point range of one block (every pair of a 1024-event
    chunk of that mark adds about w_max): the wrapping adds are detected and those blocks are
    recomputed in FP32; the result matches the oracle."""
    p = synth.random_problem(2, 20_000, 42, True, rho=0.5, beta_range=(0.02, 0.03),
                             mu_range=(0.5, 0.5))
    p.mu = np.array([5.0, 0.01])
    p = synth.Problem(t=p.t, c=np.where(np.arange(p.N) % 50 == 0, 1, 0).astype(np.int32),
                      T=p.T, mu=p.mu, alpha=p.alpha, beta=p.beta, shared_beta=True)
    assert_close(gpu_run(p, path=2, chunk=1024), oracle_ref(p), what="fixed-point overflow")
