#!/usr/bin/env python
"""Benchmark: events/s of the exact log-likelihood + gradient.

Workload (default): M=1,024 marks, one shared decay beta=1, mu_i ~ (i+1)^-1.1
summing to 50, dense alpha U[0,1] at spectral radius 0.7, N=10,000,000 events
of a seeded cluster-process simulation (synthetic; no dataset).  One step is
one hawkes_loglik_grad call over the whole stream: validation and mark counts,
the inter-chunk scan, intensities, log-sum, compensator and all gradients.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  Inputs are resident in HBM before the timed
region; L2 is flushed (a 512 MB write) between timed steps and the steps are
timed with CUDA events on the launching stream.  ``e2e`` repeats the metric
through the host-buffer entry point (pinned inputs copied in, L and gradients
copied out, inside the timed region).  ``roofline`` reports the dominant
kernel's achieved rate from per-kernel CUDA events (a separate instrumented
pass over the same steps).  ``cpu_baseline`` times the FP64 oracle on a
bounded prefix of the same stream on one host core; ``precision`` compares, on
that prefix, the CUDA path's result under each precision option (the FP64 and
FP32 log-sums, and the FP32-times ablation) with that oracle result.
``workload5`` times the fifth workload (one decay per source, M=4096, N=5e7) on
the mark-major path.  ``--impl reference`` times the oracle itself as the
reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "events/s exact loglik+grad (M=1024,N=10M) vs plain FP64 scan; % roofline"
WORKLOAD = ("hawkes_m1024_shared_n10m: M=1024, shared beta=1, mu_i ~ (i+1)^-1.1 (sum 50), "
            "dense alpha U[0,1] at spectral radius 0.7, N=10,000,000 cluster-simulated "
            "events, seed 3")
CPU_SAMPLE_EVENTS = 1 << 19


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get(
            "bf16_tflops_sustained", d["bf16_tflops"])), float(d.get("sm_max_mhz", 2070.0)), \
            "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(n_events=None):
    from paper_2604_01342_gb300 import synth
    return synth.workload(4, n_events=n_events or None)


def time_oracle(p, n_sample=CPU_SAMPLE_EVENTS, want_result=False):
    """The FP64 oracle as it stands on one host core, on the first n_sample events."""
    import oracle
    n = min(n_sample, p.N)
    t, c = p.t[:n], p.c[:n]
    T = float(t[-1])
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731
    oracle.build()
    t0 = time.perf_counter()
    res = oracle.loglik_grad(t, c, T, f32(p.mu), f32(p.alpha), np.full(p.M, f32(p.beta[:1])[0]))
    dt = time.perf_counter() - t0
    line = {"value": n / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} events of the same stream (T = t of the last one), "
                      f"FP64 log-likelihood + gradient, single thread, {dt:.2f} s"}
    if want_result:
        res["dbeta"] = np.array([res["dbeta"].sum()])        # one shared decay
        return line, res
    return line


def precision_report(p, dev, ref, n_sample=CPU_SAMPLE_EVENTS):
    """Error of each precision option of the CUDA path against the FP64 oracle, per result,
    on the oracle's sample (the first n_sample events): the default (FP64 time differences,
    FP64 log-sum partials), Kahan-compensated FP32 and plain FP32 log-sums, and the FP32-times
    ablation."""
    import torch
    from paper_2604_01342_gb300 import torch_api
    n = min(n_sample, p.N)
    t = torch.from_numpy(p.t[:n]).to(dev)
    c = torch.from_numpy(p.c[:n]).to(dev)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    al = torch.tensor(p.alpha, dtype=torch.float32, device=dev)
    be = torch.tensor(p.beta[:1], dtype=torch.float32, device=dev)
    T = float(p.t[n - 1])
    out = {"sample": f"first {n} events of the workload, against the FP64 oracle: relative L "
                     f"error, max-norm relative error per gradient block"}
    for name, kw in (("default (FP64 dt, FP64 log-sum)", {}),
                     ("Kahan FP32 log-sum", {"reduce": 1}), ("plain FP32 log-sum", {"reduce": 2}),
                     ("FP32 times (ablation)", {"fp32_times": True})):
        r = torch_api.loglik_grad(t, c, T, mu, al, be, beta_shared=True, check=False, **kw)
        got = [float(r[0].item())] + [x.cpu().numpy().astype(np.float64) for x in r[1:]]
        den = lambda a: max(float(np.max(np.abs(a))), 1e-300)  # noqa: E731
        out[name] = {"ll": abs(got[0] - ref["ll"]) / abs(ref["ll"]),
                     "dmu": float(np.max(np.abs(got[1] - ref["dmu"]))) / den(ref["dmu"]),
                     "dalpha": float(np.max(np.abs(got[2] - ref["dalpha"]))) / den(ref["dalpha"]),
                     "dbeta": float(np.max(np.abs(got[3] - ref["dbeta"]))) / den(ref["dbeta"])}
    return out


def workload5_line(dev, steps=3, events=0):
    """The fifth workload (M=4096, one decay per source, alpha 1% dense, N=5e7, T ~ 1e7) on
    the mark-major path, gradient on alpha's support: events/s over `steps` calls after one
    warm-up call (inputs resident, L2 flushed between calls).  `events` > 0 takes only the
    first that many events of the stream (T = the last one's time; profiling runs)."""
    import torch
    from paper_2604_01342_gb300 import binding as B, synth
    p = synth.workload(5)
    if 0 < events < p.N:
        p = synth.Problem(t=p.t[:events].copy(), c=p.c[:events].copy(), T=float(p.t[events - 1]),
                          mu=p.mu, alpha=p.alpha, beta=p.beta, shared_beta=False, name=p.name)
    N, M = p.N, p.M
    opts = B.make_opts(False, 0, True, 0, support=True)
    t = torch.from_numpy(p.t).to(dev)
    c = torch.from_numpy(p.c).to(dev)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    al = torch.tensor(p.alpha, dtype=torch.float32, device=dev)
    be = torch.tensor(p.beta, dtype=torch.float32, device=dev)
    nb = B.hawkes_workspace_size(N, M, 1, True, opts)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    ll = torch.empty((), dtype=torch.float64, device=dev)
    dmu = torch.empty(M, dtype=torch.float32, device=dev)
    dal = torch.empty(M, M, dtype=torch.float32, device=dev)
    dbe = torch.empty(M, dtype=torch.float32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    sptr = torch.cuda.current_stream(dev).cuda_stream

    def call():
        B.hawkes_loglik_grad(t.data_ptr(), c.data_ptr(), N, p.T, M, mu.data_ptr(), al.data_ptr(),
                             be.data_ptr(), opts, ws.data_ptr(), nb, ll.data_ptr(), dmu.data_ptr(),
                             dal.data_ptr(), dbe.data_ptr(), sptr)

    call()
    rc = B.hawkes_last_device_status(ws.data_ptr(), sptr)
    if rc:
        raise B.HawkesError(rc, "workload 5")
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        call()
        b.record()
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(b))
    B.hawkes_profile_enable(True)
    call()
    kern = {k: round(v, 3) for k, v in B.hawkes_profile_read()}
    B.hawkes_profile_enable(False)
    m = sum(ms) / len(ms)
    return {"workload": "M=4096, beta_j ~ U[0.2,5] per source, alpha 1% dense at spectral "
                        "radius 0.85, N=50,000,000 on [0, T~1e7], seed 4; gradient on "
                        "alpha's support; mark-major path" +
                        (f"; first {N:,} events only" if N < 50_000_000 else ""),
            "value": N / (m * 1e-3), "unit": "events/s", "ms_per_step": m, "steps": steps,
            "loglik": float(ll.item()), "kernels_ms": kern}


# ------------------------------------------------------ plain FP64 scan (paper)
def _next_pow2(n):
    p = 1
    while p < n:
        p *= 2
    return p


def _blelloch_inclusive(s, v):
    """Inclusive prefix products P_i = M_i ... M_1 of the compressed transitions
    (s_i, v_i) with the paper's operator (Section 3):
        (s_A, v_A) (.) (s_B, v_B) = (s_A s_B, s_A v_B + v_A),  A the later factor,
    by the Blelloch up-sweep / down-sweep on a power-of-two padding (identity
    elements (1, 0) at the end).  Plain FP64 tensor ops, one level at a time."""
    import torch
    n, m = v.shape
    n2 = _next_pow2(max(n, 1))
    S = torch.ones(n2, dtype=torch.float64, device=v.device)
    V = torch.zeros(n2, m, dtype=torch.float64, device=v.device)
    S[:n] = s
    V[:n] = v
    d = 1
    while d < n2:                                     # up-sweep
        r = torch.arange(2 * d - 1, n2, 2 * d, device=v.device)
        lft = r - d
        V[r] = S[r, None] * V[lft] + V[r]
        S[r] = S[r] * S[lft]
        d *= 2
    S[n2 - 1] = 1.0
    V[n2 - 1] = 0.0
    d = n2 // 2
    while d >= 1:                                     # down-sweep (exclusive)
        r = torch.arange(2 * d - 1, n2, 2 * d, device=v.device)
        lft = r - d
        tS, tV = S[lft].clone(), V[lft].clone()
        S[lft], V[lft] = S[r], V[r]
        V[r] = tS[:, None] * V[r] + tV
        S[r] = tS * S[r]
        d //= 2
    Si = s * S[:n]                                    # inclusive = M_i (.) exclusive
    Vi = s[:, None] * V[:n] + v
    return Si, Vi


def fp64_scan_loglik(t, c, T, mu, alpha, gamma, batch=1 << 19):
    """The paper's forward pass (Algorithm 1 / Algorithm 2) as plain FP64 PyTorch
    ops, for comparison only: transitions (e^{-g dt_i}, e^{-g dt_i} alpha[:, m_{i-1}])
    (Eq. define_augmented_M), a Blelloch scan per batch of 2^19 events, the batch
    carry R_i = P_i R_carry (Section 3.3), lambda = mu + g R (Algorithm 1), and
    the closed-form compensator.  Returns L as a float."""
    import torch
    t = t.to(torch.float64)
    c = c.to(torch.int64)
    mu = mu.to(torch.float64)
    alpha = alpha.to(torch.float64)
    n, m = t.shape[0], mu.shape[0]
    R = torch.zeros(m, dtype=torch.float64, device=t.device)
    logsum = torch.zeros((), dtype=torch.float64, device=t.device)
    for b0 in range(0, n, batch):
        b1 = min(n, b0 + batch)
        tb = t[b0:b1]
        prev_t = t[b0 - 1:b1 - 1] if b0 > 0 else torch.cat([tb[:1], tb[:-1]])
        prev_c = c[b0 - 1:b1 - 1] if b0 > 0 else torch.cat([c[:1], c[b0:b1 - 1]])
        s = torch.exp(-gamma * (tb - prev_t))
        v = s[:, None] * alpha[:, prev_c].T
        if b0 == 0:
            s[0] = 1.0
            v[0] = 0.0
        Si, Vi = _blelloch_inclusive(s, v)
        Rb = Si[:, None] * R[None, :] + Vi
        cb = c[b0:b1]
        lam = mu[cb] + gamma * Rb.gather(1, cb[:, None])[:, 0]
        logsum = logsum + torch.log(lam).sum()
        R = Rb[-1]
    colsum = alpha.sum(0)
    comp = T * mu.sum() + (colsum[c] * (-torch.expm1(-gamma * (T - t)))).sum()
    return float((logsum - comp).item())


def time_fp64_scan(p, dev, steps=1):
    import torch
    t = torch.from_numpy(p.t).to(dev)
    c = torch.from_numpy(p.c).to(dev)
    f32 = lambda a: torch.tensor(np.asarray(a, np.float32).astype(np.float64), device=dev)  # noqa
    mu, al, g = f32(p.mu), f32(p.alpha), float(np.float32(p.beta[0]))
    fp64_scan_loglik(t[:4096], c[:4096], float(p.t[4095]), mu, al, g)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        ll = fp64_scan_loglik(t, c, p.T, mu, al, g)
    b.record()
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    return {"value": p.N / (ms * 1e-3), "unit": "events/s", "ms_per_step": ms, "loglik": ll,
            "kind": "paper's method as plain PyTorch FP64 ops on the same GPU: Blelloch scan "
                    "over (s, v) pairs, batches of 2^19 events, forward only (no gradient)"}


# --------------------------------------------------------------------- reference
def run_reference(args):
    world, rank, _ = dist_init()
    if rank != 0:
        return
    p = workload()
    for _ in range(args.warmup):        # untimed: the same bounded sample as a timed step
        time_oracle(p, CPU_SAMPLE_EVENTS // 4)
    times = []
    per = None
    for _ in range(args.steps):
        per = time_oracle(p, CPU_SAMPLE_EVENTS // 4)
        times.append(CPU_SAMPLE_EVENTS // 4 / per["value"])
    n = CPU_SAMPLE_EVENTS // 4
    value = n * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_events_per_step": n,
                       "parallelism": "single host core"},
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": 1, "kind": "oracle",
                             "sample": per["sample"]},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2604_01342_gb300 import binding as B

    world, rank, local = dist_init()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = workload(args.events)
    N, M = p.N, p.M
    opts = B.make_opts(True, args.chunk, True, 0)
    t = torch.from_numpy(p.t).to(dev)
    c = torch.from_numpy(p.c).to(dev)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    al = torch.tensor(p.alpha, dtype=torch.float32, device=dev)
    be = torch.tensor(p.beta[:1], dtype=torch.float32, device=dev)
    ws_bytes = B.hawkes_workspace_size(N, M, 1, True, opts)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    out_ll = torch.empty((), dtype=torch.float64, device=dev)
    dmu = torch.empty(M, dtype=torch.float32, device=dev)
    dal = torch.empty(M, M, dtype=torch.float32, device=dev)
    dbe = torch.empty(1, dtype=torch.float32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream

    def step():
        B.hawkes_loglik_grad(t.data_ptr(), c.data_ptr(), N, p.T, M, mu.data_ptr(), al.data_ptr(),
                             be.data_ptr(), opts, ws.data_ptr(), ws_bytes, out_ll.data_ptr(),
                             dmu.data_ptr(), dal.data_ptr(), dbe.data_ptr(), sptr)

    for _ in range(max(args.warmup, 3)):
        step()
    rc = B.hawkes_last_device_status(ws.data_ptr(), sptr)
    if rc:
        raise B.HawkesError(rc, "device status after warm-up")
    launches_per_step = B.hawkes_last_launch_count()

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        tt = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    value = world * N / (ms * 1e-3)
    ll_val = float(out_ll.item())

    # ---- per-kernel timing (instrumented pass, same steps)
    B.hawkes_profile_enable(True)
    kern = {}
    for i in range(args.steps):
        flush.zero_()
        step()
        for name, kms in B.hawkes_profile_read():
            kern.setdefault(name, []).append(kms)
    B.hawkes_profile_enable(False)
    kern_ms = {k: sum(v) / len(v) for k, v in kern.items()}

    # ---- end to end through the host-buffer entry point
    # every rank takes part (the max over ranks below is a collective)
    hb = B.hawkes_workspace_size_host(N, M, opts)
    wsh = torch.empty(hb, dtype=torch.uint8, device=dev)
    th = torch.from_numpy(p.t).pin_memory()
    ch = torch.from_numpy(p.c).pin_memory()
    muh = mu.cpu().pin_memory(); alh = al.cpu().pin_memory(); beh = be.cpu().pin_memory()
    llh = torch.empty((), dtype=torch.float64).pin_memory()
    dmuh = torch.empty(M, dtype=torch.float32).pin_memory()
    dalh = torch.empty(M, M, dtype=torch.float32).pin_memory()
    dbeh = torch.empty(1, dtype=torch.float32).pin_memory()

    def host_step():
        B.hawkes_loglik_grad_host(th.data_ptr(), ch.data_ptr(), N, p.T, M, muh.data_ptr(),
                                  alh.data_ptr(), beh.data_ptr(), opts, wsh.data_ptr(), hb,
                                  llh.data_ptr(), dmuh.data_ptr(), dalh.data_ptr(),
                                  dbeh.data_ptr(), sptr)

    for _ in range(2):
        host_step()
    e_ms = []
    for i in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        host_step()
        b.record(stream)
        torch.cuda.synchronize(dev)
        e_ms.append(a.elapsed_time(b))
    em = sum(e_ms) / len(e_ms)
    if world > 1:
        tt = torch.tensor([em], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        em = float(tt.item())
    h2d = N * 8 + N * 4 + 4 * (M + M * M + 1)
    d2h = 8 + 4 * (M + M * M + 1)
    e2e = {"value": world * N / (em * 1e-3), "unit": "events/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": em}
    del wsh

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    hbm, bf16, bf16_sus, sm_max, src = peaks()
    roof = roofline(kern_ms, N, M, args, hbm, bf16, bf16_sus, clk, src)
    path_roof = path_roofline(ms, N, M, hbm, clk, bf16)
    cpu, precision = None, None
    if world == 1 and not args.no_cpu:
        cpu, ref = time_oracle(p, want_result=True)
        precision = precision_report(p, dev, ref)
    fp64 = time_fp64_scan(p, dev) if (world == 1 and not args.no_fp64_scan) else None
    w5 = (workload5_line(dev, events=args.workload5_events)
          if (world == 1 and not args.no_workload5) else None)
    line = {"metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "events": N, "M": M, "beta": "shared",
                       "chunk": args.chunk or "default", "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "loglik": ll_val},
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "clocks": clk,
            "roofline": roof, "path_roofline": path_roof, "cpu_baseline": cpu,
            "fp64_scan_baseline": fp64, "precision": precision, "workload5": w5,
            "kernels_ms": {k: round(v, 4) for k, v in kern_ms.items()}}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# DRAM bytes per event of the pair kernels: dram__bytes_read.sum + dram__bytes_write.sum from
# one ncu capture on the first 2e6 events of the benchmark stream.  A launch processes every
# event of the step and the kernels' traffic grows in proportion to the events, so a launch
# moves N times this.
DRAM_BYTES_PER_EVENT = {"pairs_bwd": (50371584 + 5120256) / 2e6,
                        "pairs_fwd": (36649984 + 142592) / 2e6}


def kernel_work(name, N, M, C):
    """(bound, algorithmic work per launch) of each kernel of one step.

    HBM kernels count the bytes the algorithm must move; tensor kernels the flops of
    one product (the fp16 hi/lo split issues three); shared-memory kernels the bytes of
    shared memory the pairs must touch: per forward pair one 4-byte alpha gather plus its
    share of the broadcast 16-byte source record (32 lanes), per backward pair one 4-byte
    read and one 4-byte write of the dalpha tile; ALU kernels FP32 operations."""
    nb = (N + C - 1) // C
    pairs = N * (C - 1) / 2.0                  # pairs (k, l) inside chunks, l before k
    table = {
        "validate_events": ("hbm", 12.0 * N),
        "scan_reduce": ("hbm", 12.0 * N + 4.0 * N),             # t, c in; offsets out
        "scan_states": ("hbm", 8.0 * N + 8.0 * M * nb),         # offsets, c in; S^, G^ out
        "split_S": ("hbm", 4.0 * M * nb + 4.0 * M * nb),
        "split_G": ("hbm", 8.0 * M * nb + 4.0 * M * nb),         # S^, G^ in; S^ - beta G^ out
        "split_S_G": ("hbm", 8.0 * M * nb + 8.0 * M * nb),       # S^, G^ in; both splits out
        "bucket": ("hbm", 8.0 * N + 24.0 * N),                  # offsets, c in; records out
        "epilogue": ("hbm", 12.0 * N + 8.0 * N + 12.0 * N),
        "split_W": ("hbm", 4.0 * M * nb + 4.0 * M * nb),
        "transpose_S": ("hbm", 4.0 * M * nb + 4.0 * M * nb),
        "gemm_Y": ("tensor", 2.0 * M * M * nb),
        "gemm_Z": ("tensor", 2.0 * M * M * nb),
        "gemm_dalpha": ("tensor", 2.0 * M * M * nb),
        "pairs_fwd": ("smem", (4.0 + 16.0 / 32.0) * pairs),
        "pairs_bwd": ("smem", 8.0 * pairs),
        "walk": ("alu", 2.0 * 3.0 * N * M),
    }
    return table.get(name)


def roofline(kern_ms, N, M, args, hbm, bf16, bf16_sus, clk, src):
    """Dominant kernel's achieved rate against its bound (bytes, flops or FMAs per launch over
    the launch's CUDA-event time, against the peak of that bound)."""
    if not kern_ms:
        return None
    C = args.chunk or 192
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12      # TFLOP/s, FMA = 2 flops
    f16_peak = bf16                                       # dense FP16 = BF16 (nominal ratio 1)
    smem_peak = 152 * 128 * sm_max * 1e6 / 1e9            # GB/s: 128 B per clock per SM
    rows = {}
    for name, ms in kern_ms.items():
        w = kernel_work(name, N, M, C)
        if w is None or ms <= 0:
            continue
        bound, work = w
        if bound == "hbm":
            ach, peak, unit = work / (ms * 1e-3) / 1e9, hbm, "GB/s"
        elif bound == "tensor":
            ach, peak, unit = work / (ms * 1e-3) / 1e12, f16_peak, "TFLOP/s"
        elif bound == "smem":
            ach, peak, unit = work / (ms * 1e-3) / 1e9, smem_peak, "GB/s"
        else:
            ach, peak, unit = work / (ms * 1e-3) / 1e12, fp32_peak, "TFLOP/s"
        rows[name] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                      "frac": ach / peak, "ms": ms}
    name = max(kern_ms, key=kern_ms.get)
    dom = rows.get(name)
    if dom is None:
        return {"kernel": name, "bound": None, "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None}
    traffic = DRAM_BYTES_PER_EVENT.get(name)
    out = {"kernel": name, "bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"],
           "unit": dom["unit"], "frac": dom["frac"],
           "traffic": traffic * N if traffic is not None else None,
           "peak_source": {"hbm": f"{src} HBM copy bandwidth",
                           "tensor": f"{src} bf16 dense (= fp16 dense), burst",
                           "smem": "shared memory: 152 SMs x 128 B/clock x max SM clock",
                           "alu": "152 SMs x 128 FP32 lanes x 2 x max SM clock"}[dom["bound"]],
           "per_kernel": {k: {"frac": round(v["frac"], 4), "ms": round(v["ms"], 4),
                              "bound": v["bound"]} for k, v in rows.items()}}
    if dom["bound"] == "tensor":
        out["issued_frac"] = 3.0 * dom["frac"]
    return out


def path_roofline(ms_step, N, M, hbm, clk, bf16=None):
    """The metric's roofline of the whole step: the slower of the event bytes at HBM peak
    and 3 N M FMAs (intensity dot, dalpha row, dbeta dot) at the FP32 peak."""
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    t_hbm = 12.0 * N / (hbm * 1e9)
    t_alu = 3.0 * N * M / (152 * 128 * sm_max * 1e6)
    t_roof = max(t_hbm, t_alu)
    # the same 3 N M multiply-adds at the dense tensor rate (the literal reading, which
    # ignores that only the inter-chunk part is a contraction): printed, labelled
    t_tensor = max(t_hbm, 2.0 * 3.0 * N * M / (bf16 * 1e12)) if bf16 else None
    return {"t_roof_ms": 1e3 * t_roof, "bound": "alu" if t_alu >= t_hbm else "hbm",
            "frac": 1e3 * t_roof / ms_step,
            "note": "3 N M FP32 FMA at 152 SMs x 128 lanes x max clock vs 12 B/event at HBM",
            "tensor_reading": None if t_tensor is None else
            {"t_roof_ms": 1e3 * t_tensor, "frac": 1e3 * t_tensor / ms_step,
             "note": "3 N M multiply-adds at the measured dense bf16 rate vs 12 B/event at HBM"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--no-fp64-scan", action="store_true",
                    help="skip the plain FP64 scan comparison leg")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the CPU oracle timing leg (and the precision report that uses it)")
    ap.add_argument("--no-workload5", action="store_true",
                    help="skip the fifth workload (per-source decays, M=4096, N=5e7)")
    ap.add_argument("--events", type=int, default=0,
                    help="use only the first N events of the workload (profiling runs)")
    ap.add_argument("--only-workload5", action="store_true",
                    help="run only the fifth workload's leg and print its line (profiling runs)")
    ap.add_argument("--workload5-events", type=int, default=0,
                    help="use only the first N events of the fifth workload (profiling runs)")
    args = ap.parse_args()
    if args.only_workload5:
        import torch
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        print(json.dumps({"workload5": workload5_line(dev, steps=args.steps,
                                                      events=args.workload5_events)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
