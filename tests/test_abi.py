"""The C-ABI library loads and exports every symbol include/hawkes_gb300.h
declares; host-side checks work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2604_01342_gb300 import binding

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "hawkes_gb300.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hawkes_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return binding.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTED) == names


def test_status_strings(lib):
    for code in range(10):
        assert binding.hawkes_status_str(code)
    assert binding.hawkes_status_str(0) == "ok"


def test_default_opts(lib):
    o = lib.hawkes_default_opts()
    assert (o.beta_shared, o.chunk, o.validate, o.path) == (0, 0, 1, 0)


def test_workspace_sizes(lib):
    per = binding.make_opts(False)
    sh = binding.make_opts(True)
    n1 = binding.hawkes_workspace_size(1_000_000, 64, 1, True, per)
    n0 = binding.hawkes_workspace_size(1_000_000, 64, 1, False, per)
    assert n1 > n0 > 0 and n1 % 256 == 0
    # large shared-decay problems take the chunk-GEMM path; per-source large M is not built
    assert binding.hawkes_workspace_size(10_000_000, 1024, 1, True, sh) > 0
    assert lib.hawkes_workspace_size(1000, 1024, 1, 1, ctypes.byref(per)) == 0
    assert lib.hawkes_workspace_size(-1, 4, 1, 1, ctypes.byref(per)) == 0
    assert binding.hawkes_workspace_size_host(1000, 8, per) > binding.hawkes_workspace_size(
        1000, 8, 1, True, per)


def _cuda_visible():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_host_side_errors_need_no_gpu(lib):
    """Argument checks that return before anything is launched.  Pointers are NULL or
    real (host) buffers of the right sizes, never made-up addresses."""
    import numpy as np
    opts = binding.make_opts(False)
    rc = lib.hawkes_loglik(None, None, 5, 1.0, 3, None, None, None, ctypes.byref(opts), None, 0,
                           None, None)
    assert rc == 1   # null inputs
    rc = lib.hawkes_loglik_grad(None, None, 5, -1.0, 3, None, None, None, ctypes.byref(opts),
                                None, 0, None, None, None, None, None)
    assert rc == 1   # T < 0 (checked before the pointers)
    rc = lib.hawkes_loglik_grad(None, None, 0, 1.0, 0, None, None, None, ctypes.byref(opts),
                                None, 0, None, None, None, None, None)
    assert rc == 1   # M = 0


@pytest.mark.skipif(_cuda_visible(), reason="host-buffer pointers are for the no-GPU check only")
def test_missing_workspace_is_reported_without_a_gpu(lib):
    import numpy as np
    opts = binding.make_opts(False)
    t = np.linspace(0.0, 1.0, 5)
    c = np.zeros(5, np.int32)
    mu, al, be = np.ones(3, np.float32), np.ones(9, np.float32), np.ones(3, np.float32)
    ll = np.zeros(1)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    rc = lib.hawkes_loglik(ptr(t), ptr(c), 5, 1.0, 3, ptr(mu), ptr(al), ptr(be),
                           ctypes.byref(opts), None, 0, ptr(ll), None)
    assert rc == 7   # workspace missing


def test_walk_lanes_option_is_checked(lib):
    ok = binding.make_opts(False, 0, True, 1, walk_lanes=8)
    assert lib.hawkes_workspace_size(1000, 8, 1, 1, ctypes.byref(ok)) > 0
    for lanes, M in ((8, 9), (16, 17), (12, 4)):
        bad = binding.make_opts(False, 0, True, 1, walk_lanes=lanes)
        assert lib.hawkes_workspace_size(1000, M, 1, 1, ctypes.byref(bad)) == 0


def test_autotune_file_cache_round_trip(tmp_path):
    from paper_2604_01342_gb300 import autotune
    path = str(tmp_path / "sub" / "tune.json")
    autotune._store_file(path, "gpu|sms=152|N=10|B=1|M=4|shared=1", {"path": 1, "chunk": 64})
    autotune._store_file(path, "gpu|sms=152|N=20|B=1|M=4|shared=1", {"path": 2, "chunk": 192})
    data = autotune._load_file(path)
    assert data["gpu|sms=152|N=10|B=1|M=4|shared=1"]["chunk"] == 64
    assert len(data) == 2
    assert autotune._load_file(str(tmp_path / "missing.json")) == {}
    # candidates: lanes for small M on the walk, segment lengths on the mark-major path
    assert (1, 128, 8) in autotune._candidates(8, False, 1)
    assert (1, 128, 16) not in autotune._candidates(20, False, 1)
    assert all(p == 3 for p, _, _ in autotune._candidates(4096, False, 1))
