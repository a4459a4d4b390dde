"""CUDA-graph replay of one log-likelihood + gradient call.

A call of the library is a fixed sequence of kernel launches and asynchronous memsets on
one stream, with every size and pointer known on the host before the first launch, so it
can be captured once and replayed: the inputs keep their addresses (their contents may
change between replays), the workspace and the outputs belong to the graph object.  This
is the launch form for the batched varlen workload (many short sequences, where launch
overhead matters): one graph replay computes every sequence's log-likelihood and gradient.

    g = GraphedLogLikGrad.varlen(t, c, offsets, T, mu, alpha, beta)
    ll, dmu, dalpha, dbeta = g.replay()          # tensors owned by g, overwritten by each replay
    g.status()                                   # synchronises; 0 or a hawkes_status
"""
from __future__ import annotations

import torch

from . import binding as _b


def _need(x: torch.Tensor, dtype, name: str):
    if not x.is_cuda or x.dtype != dtype or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


class GraphedLogLikGrad:
    """Holds the captured graph, its workspace and its output tensors."""

    def __init__(self, launch, ws: torch.Tensor, outputs: tuple, device: torch.device):
        self._launch = launch
        self.ws = ws
        self.outputs = outputs
        self.device = device
        # one eager call first: it sets the kernels' shared-memory attributes and checks
        # the inputs, so that nothing but launches and memsets happens inside the capture
        launch(torch.cuda.current_stream(device).cuda_stream)
        rc = _b.hawkes_last_device_status(ws.data_ptr(), torch.cuda.current_stream(device).cuda_stream)
        if rc:
            raise _b.HawkesError(rc, "device check before capture")
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device)
        side.wait_stream(torch.cuda.current_stream(device))
        with torch.cuda.graph(self.graph, stream=side):
            launch(side.cuda_stream)
        torch.cuda.current_stream(device).wait_stream(side)

    def replay(self):
        self.graph.replay()
        return self.outputs

    def status(self) -> int:
        return _b.hawkes_last_device_status(self.ws.data_ptr(),
                                            torch.cuda.current_stream(self.device).cuda_stream)

    @classmethod
    def single(cls, t, c, T: float, mu, alpha, beta, beta_shared=None, chunk: int = 0,
               path: int = 0, walk_lanes: int = 0):
        """One sequence: t float64 [N], c int32 [N], mu [M], alpha [M,M], beta [1] or [M]."""
        for x, dt, n in ((t, torch.float64, "t"), (c, torch.int32, "c"), (mu, torch.float32, "mu"),
                         (alpha, torch.float32, "alpha"), (beta, torch.float32, "beta")):
            _need(x, dt, n)
        dev = t.device
        N, M = t.shape[0], mu.shape[0]
        shared = bool(beta_shared) if beta_shared is not None else (beta.numel() == 1 and M != 1)
        opts = _b.make_opts(shared, chunk, True, path, walk_lanes=walk_lanes)
        nbytes = _b.hawkes_workspace_size(N, M, 1, True, opts)
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        ll = torch.empty((), dtype=torch.float64, device=dev)
        dmu = torch.empty(M, dtype=torch.float32, device=dev)
        dal = torch.empty(M, M, dtype=torch.float32, device=dev)
        dbe = torch.empty(1 if shared else M, dtype=torch.float32, device=dev)

        def launch(stream):
            _b.hawkes_loglik_grad(t.data_ptr(), c.data_ptr(), N, float(T), M, mu.data_ptr(),
                                  alpha.data_ptr(), beta.data_ptr(), opts, ws.data_ptr(),
                                  ws.numel(), ll.data_ptr(), dmu.data_ptr(), dal.data_ptr(),
                                  dbe.data_ptr(), stream)
        return cls(launch, ws, (ll, dmu, dal, dbe), dev)

    @classmethod
    def varlen(cls, t, c, offsets, T, mu, alpha, beta, beta_shared=None, chunk: int = 0,
               path: int = 0, walk_lanes: int = 0):
        """B sequences: offsets int64 [B+1], T float64 [B], mu [B,M], alpha [B,M,M], beta [B] or [B,M]."""
        for x, dt, n in ((t, torch.float64, "t"), (c, torch.int32, "c"),
                         (offsets, torch.int64, "offsets"), (T, torch.float64, "T"),
                         (mu, torch.float32, "mu"), (alpha, torch.float32, "alpha"),
                         (beta, torch.float32, "beta")):
            _need(x, dt, n)
        dev = t.device
        B, N, M = offsets.shape[0] - 1, t.shape[0], mu.shape[-1]
        shared = bool(beta_shared) if beta_shared is not None else (beta.numel() == B and M != 1)
        opts = _b.make_opts(shared, chunk, True, path, walk_lanes=walk_lanes)
        nbytes = _b.hawkes_workspace_size(N, M, B, True, opts)
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        ll = torch.empty(B, dtype=torch.float64, device=dev)
        dmu = torch.empty(B, M, dtype=torch.float32, device=dev)
        dal = torch.empty(B, M, M, dtype=torch.float32, device=dev)
        dbe = torch.empty(B if shared else B * M, dtype=torch.float32, device=dev)
        if not shared:
            dbe = dbe.view(B, M)

        def launch(stream):
            _b.hawkes_loglik_grad_varlen(t.data_ptr(), c.data_ptr(), offsets.data_ptr(), B, N,
                                         T.data_ptr(), M, mu.data_ptr(), alpha.data_ptr(),
                                         beta.data_ptr(), opts, ws.data_ptr(), ws.numel(),
                                         ll.data_ptr(), dmu.data_ptr(), dal.data_ptr(),
                                         dbe.data_ptr(), stream)
        return cls(launch, ws, (ll, dmu, dal, dbe), dev)
