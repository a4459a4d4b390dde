"""The library's integer work compared bit by bit with the oracle's integer passes:
per-(sequence, mark) counts, the chunk table (chunk bases of the sequences and the owner
of every chunk; empty and ragged sequences included) and, on the chunk-GEMM path, each
chunk's bucket offsets and the order of its events in the buckets.  The device tables
are read through hawkes_integer_tables after an ordinary call."""
import numpy as np
import pytest

import oracle
from helpers import f32
from paper_2604_01342_gb300 import synth

pytestmark = pytest.mark.gpu


def _view(ws, ptr, count, dtype):
    import torch
    off = ptr - ws.data_ptr()
    nbytes = count * np.dtype(dtype).itemsize
    assert 0 <= off and off + nbytes <= ws.numel()
    return ws[off: off + nbytes].cpu().numpy().view(dtype)


def _varlen_call(vp, chunk, path=0):
    import torch
    from paper_2604_01342_gb300 import binding as B
    dev = torch.device("cuda")
    opts = B.make_opts(False, chunk, True, path)
    N, M, Bn = int(vp.offsets[-1]), vp.M, vp.B
    nbytes = B.hawkes_workspace_size(N, M, Bn, True, opts)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    x = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (vp.t, vp.c, vp.offsets, vp.T)]
    prm = [torch.tensor(f32(a), dtype=torch.float32, device=dev) for a in (vp.mu, vp.alpha, vp.beta)]
    out = [torch.empty(Bn, dtype=torch.float64, device=dev),
           torch.empty(Bn * M, dtype=torch.float32, device=dev),
           torch.empty(Bn * M * M, dtype=torch.float32, device=dev),
           torch.empty(Bn * M, dtype=torch.float32, device=dev)]
    s = torch.cuda.current_stream().cuda_stream
    B.hawkes_loglik_grad_varlen(*[a.data_ptr() for a in x[:3]], Bn, N, x[3].data_ptr(), M,
                                *[a.data_ptr() for a in prm], opts, ws.data_ptr(), nbytes,
                                *[o.data_ptr() for o in out], s)
    assert B.hawkes_last_device_status(ws.data_ptr(), s) == 0
    return ws, B.hawkes_integer_tables(ws.data_ptr(), N, M, Bn, True, opts)


def _with_empty(vp, at):
    """The same batch with empty sequences inserted before the sequences listed in ``at``."""
    lens = list(np.diff(vp.offsets))
    mu, al, be, T = list(vp.mu), list(vp.alpha), list(vp.beta), list(vp.T)
    for k, i in enumerate(sorted(at)):
        j = i + k
        lens.insert(j, 0)
        mu.insert(j, mu[0]); al.insert(j, al[0]); be.insert(j, be[0]); T.insert(j, 2.5)
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return synth.VarlenProblem(t=vp.t, c=vp.c, offsets=offsets, T=np.array(T), mu=np.array(mu),
                               alpha=np.array(al), beta=np.array(be), shared_beta=False)


@pytest.mark.parametrize("chunk", [1, 16, 100])
def test_varlen_tables_bit_exact(chunk):
    rng = np.random.default_rng(31)
    vp = _with_empty(synth.varlen_workload(rng, 23, m=6, median=120, sigma=1.2, lo=1, hi=900),
                     (0, 7, 23))
    lens = np.diff(vp.offsets)
    assert (lens == 0).any() and (chunk == 1 or (lens % chunk != 0).any())   # empty, ragged
    ws, tb = _varlen_call(vp, chunk)
    assert tb.chunk == chunk and tb.mark_blocks == 0
    base, seq = oracle.chunk_table(vp.offsets, chunk)
    got_base = _view(ws, tb.chunk_base, vp.B + 1, np.int64)
    np.testing.assert_array_equal(got_base, base)
    np.testing.assert_array_equal(_view(ws, tb.chunk_seq, int(base[-1]), np.int32), seq)
    counts = _view(ws, tb.mark_counts, vp.B * vp.M, np.int64).reshape(vp.B, vp.M)
    for s in range(vp.B):
        a, b = vp.offsets[s], vp.offsets[s + 1]
        np.testing.assert_array_equal(counts[s], oracle.mark_counts(vp.c[a:b], vp.M))


@pytest.mark.parametrize("m,n,chunk", [(300, 5000, 192), (1024, 20_000, 0), (40, 777, 64)])
def test_gemm_path_buckets_bit_exact(m, n, chunk):
    import torch
    from helpers import gpu_run
    from paper_2604_01342_gb300 import binding as B, torch_api
    p = synth.random_problem(m, n, 700 + m, True, rho=0.5)
    gpu_run(p, path=2, chunk=chunk)
    torch.cuda.synchronize()
    ws = next(iter(torch_api._ws_cache.values()))
    opts = B.make_opts(True, chunk, True, 2)
    tb = B.hawkes_integer_tables(ws.data_ptr(), p.N, p.M, 1, True, opts)
    C, P = tb.chunk, tb.mark_blocks
    assert P >= 1
    base, seq = oracle.chunk_table(np.array([0, p.N]), C)
    nb = int(base[-1])
    np.testing.assert_array_equal(_view(ws, tb.chunk_base, 2, np.int64), base)
    np.testing.assert_array_equal(_view(ws, tb.chunk_seq, nb, np.int32), seq)
    np.testing.assert_array_equal(_view(ws, tb.mark_counts, p.M, np.int64),
                                  oracle.mark_counts(p.c, p.M))
    bs, order = oracle.bucket_order(p.c, p.M, C, P)
    np.testing.assert_array_equal(_view(ws, tb.bucket_start, nb * (P + 1), np.int32).reshape(nb, P + 1), bs)
    slots = _view(ws, tb.bucket_slots, 4 * p.N, np.uint32).reshape(p.N, 4)[:, 3]
    np.testing.assert_array_equal((slots >> 16).astype(np.int32), order)
    pos = (p.c[np.arange(p.N) // C * C + order] // P).astype(np.uint32)
    np.testing.assert_array_equal(slots & 0xffff, pos)
