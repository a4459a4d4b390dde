"""The mark-major walk (one decay per source, large M, alpha read through its support)
against the FP64 oracle at the stated tolerances, through the C ABI:
  * sparse alpha with the gradient on its support, against the oracle's lazy
    per-component form (itself pinned to the dense oracle on the support);
  * dense alpha (every entry a support entry), against the dense oracle, and equal to the
    state walk where both apply;
  * several segments with a ragged last tile, ties, times near 1e7, empty and one-event
    streams, rows too long for the walk (reported on the device);
  * its integer work (support rows, the (segment, mark) order, the FP32 time pairs) bit by
    bit against the oracle's integer passes;
  * the fifth workload (M=4096, per-source decays, alpha 1% dense, N=5e7, T about 1e7):
    a 1e6-event prefix and the whole stream, with the time per call."""
import ctypes
import threading

import numpy as np
import pytest

from helpers import assert_close, f32, gpu_run, maxnorm_rel, oracle_ref, rel_err
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


def support_ref(p):
    import oracle
    return oracle.loglik_grad_support(p.t, p.c, p.T, f32(p.mu), f32(p.alpha), f32(p.beta))


def sparse_problem(m, n, seed, density, time_shift=0.0, beta_range=(0.2, 5.0)):
    return synth.random_problem(m, n, seed, False, rho=0.7, density=density,
                                beta_range=beta_range, time_shift=time_shift)


@pytest.mark.parametrize("m,n,seed,density,chunk", [
    (40, 5000, 1, 0.15, 0), (300, 20_000, 2, 0.05, 0), (1000, 30_000, 3, 0.02, 0),
    (200, 70_001, 4, 0.08, 16384), (64, 50_000, 5, 0.3, 16384)])
def test_marks_sparse_matches_support_oracle(m, n, seed, density, chunk):
    p = sparse_problem(m, n, seed, density)
    got = gpu_run(p, path=3, chunk=chunk, support=True)
    assert_close(got, support_ref(p), what=f"marks m={m} n={n} d={density}")


@pytest.mark.parametrize("m,n,seed", [(100, 8000, 11), (128, 6000, 12), (3, 2000, 13)])
def test_marks_dense_matches_oracle(m, n, seed):
    p = synth.random_problem(m, n, seed, False, rho=0.6, beta_range=(0.3, 3.0))
    got = gpu_run(p, path=3)
    assert_close(got, oracle_ref(p), what=f"marks dense m={m}")


def test_marks_equals_state_walk():
    p = synth.random_problem(48, 9000, 14, False)
    a = gpu_run(p, path=3, chunk=16384)
    b = gpu_run(p, path=1)
    assert rel_err(a["ll"], b["ll"]) < 1e-6
    for k in ("dmu", "dalpha", "dbeta"):
        assert maxnorm_rel(a[k], b[k]) < 1e-4, k


def test_marks_support_option_on_other_paths():
    """support=True zeroes the entries outside alpha's support on every path."""
    p = sparse_problem(30, 4000, 15, 0.2)
    ref = support_ref(p)
    for path in (1, 3):
        assert_close(gpu_run(p, path=path, support=True), ref, what=f"support on path {path}")


def test_marks_ties_and_large_times():
    p = sparse_problem(80, 6000, 16, 0.1, time_shift=1e7)
    p.t = np.round(p.t, 1)
    p.T = float(max(p.T, p.t[-1]))
    assert_close(gpu_run(p, path=3, support=True), support_ref(p), what="marks ties near 1e7")


@pytest.mark.parametrize("n", [0, 1])
def test_marks_empty_and_single_event(n):
    p = sparse_problem(70, 1, 17, 0.2)
    if n == 0:
        p.t, p.c, p.T = p.t[:0], p.c[:0], 2.5
    else:
        p.T = float(p.t[0]) + 0.75
    assert_close(gpu_run(p, path=3, support=True), support_ref(p), what=f"marks n={n}")


def test_marks_rows_too_long_are_reported():
    from paper_2604_01342_gb300 import binding
    p = sparse_problem(200, 500, 18, 0.9)            # rows of ~180 support entries
    with pytest.raises(binding.HawkesError) as ei:
        gpu_run(p, path=3, support=True)
    assert ei.value.code == 8
    dense = binding.make_opts(False, 0, True, 3)        # every entry a support entry: M > 128
    assert binding.lib().hawkes_workspace_size(500, 200, 1, 1, ctypes.byref(dense)) == 0


def test_marks_integer_tables_bit_exact():
    import torch
    import oracle
    from paper_2604_01342_gb300 import binding as B, torch_api
    p = sparse_problem(150, 40_000, 19, 0.05)
    gpu_run(p, path=3, chunk=16384, support=True)
    torch.cuda.synchronize()
    ws = next(iter(torch_api._ws_cache.values()))
    tb = B.hawkes_integer_tables(ws.data_ptr(), p.N, p.M, 1, True,
                                 B.make_opts(False, 16384, True, 3, support=True))

    def view(ptr, count, dtype):
        off = ptr - ws.data_ptr()
        nbytes = count * np.dtype(dtype).itemsize
        assert 0 <= off and off + nbytes <= ws.numel()
        return ws[off: off + nbytes].cpu().numpy().view(dtype)

    row_ptr, col = oracle.support_rows(f32(p.alpha))
    np.testing.assert_array_equal(view(tb.support_row_ptr, p.M + 1, np.int32), row_ptr)
    np.testing.assert_array_equal(view(tb.support_col, int(row_ptr[-1]), np.int32), col)
    L = tb.segment_events
    assert L == 16384 and tb.segments == (p.N + L - 1) // L
    start, order = oracle.mark_sort(p.c, p.M, L)
    np.testing.assert_array_equal(view(tb.mark_start, tb.segments * p.M + 1, np.int32), start)
    slots = view(tb.mark_slots, 4 * p.N, np.uint32).reshape(p.N, 4)
    np.testing.assert_array_equal(slots[:, 2].astype(np.int32), order)
    np.testing.assert_array_equal(slots[:, 3].astype(np.int32), p.c[order])
    d = p.t[order] - p.t[(order // L) * L]
    hi = d.astype(np.float32)
    lo = (d - hi.astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(slots[:, 0], hi.view(np.uint32))
    np.testing.assert_array_equal(slots[:, 1], lo.view(np.uint32))


# ------------------------------------------------------------------ the fifth workload
@pytest.fixture(scope="module")
def c5():
    return synth.workload(5)


def _prefix(p, n):
    return synth.Problem(t=p.t[:n].copy(), c=p.c[:n].copy(), T=float(p.t[n - 1]), mu=p.mu,
                         alpha=p.alpha, beta=p.beta, shared_beta=False, name=p.name)


def _report(what, got, ref):
    print(f"{what}: loglik rel err {rel_err(got['ll'], ref['ll']):.3e}; " + ", ".join(
        f"{k} {maxnorm_rel(got[k], ref[k]):.3e}" for k in ("dmu", "dalpha", "dbeta")))


def test_workload5_prefix_matches_oracle(c5):
    p = _prefix(c5, 1_000_000)
    got = gpu_run(p, support=True)          # automatic path: per-source decays, M = 4096
    ref = support_ref(p)
    _report("M=4096 prefix 1e6", got, ref)
    assert_close(got, ref, what="M=4096 prefix 1e6")


def test_workload5_full_matches_oracle(c5):
    """The whole stream (5e7 events, T about 1e7), element by element, and the time per call
    (CUDA events, inputs resident, after one warm-up call)."""
    import torch
    from paper_2604_01342_gb300 import torch_api
    p = c5
    box = {}
    th = threading.Thread(target=lambda: box.setdefault("ref", support_ref(p)), daemon=True)
    th.start()
    dev = torch.device("cuda")
    t = torch.from_numpy(p.t).to(dev)
    c = torch.from_numpy(p.c).to(dev)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    al = torch.tensor(p.alpha, dtype=torch.float32, device=dev)
    be = torch.tensor(p.beta, dtype=torch.float32, device=dev)
    run = lambda: torch_api.loglik_grad(t, c, p.T, mu, al, be, beta_shared=False,  # noqa: E731
                                        support=True, check=False)
    run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    r = run()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    print(f"M=4096 per-source, 5e7 events: {ms:.2f} ms per call = {p.N / ms * 1e3:.3e} events/s")
    got = {"ll": float(r[0].item()), "dmu": r[1].cpu().numpy().astype(np.float64),
           "dalpha": r[2].cpu().numpy().astype(np.float64),
           "dbeta": r[3].cpu().numpy().astype(np.float64)}
    th.join()
    ref = box["ref"]
    _report("M=4096 full 5e7", got, ref)
    assert_close(got, ref, what="M=4096 full 5e7")
