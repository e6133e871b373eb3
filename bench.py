#!/usr/bin/env python
"""Throughput of the hard-sphere lattice Boltzmann step on one GB300.

Workload: a 512 x 512 x 192 slit, sigma = 12, eta = 0.25, tau = 0.7,
F_e = 5e-7 (bounce-back walls in z, periodic x, y), FP32 compute, populations
stored as FP32 non-equilibrium parts (``--storage f16`` for FP16). One step =
ball average + g2 -> shell force -> BGK collision + pull streaming + the next
moments. The populations (3.8 GB FP32) exceed the 129 MB L2, so no flush is
needed. Beside the headline line: the same slit with FP16 storage, the
packing-fraction sweep (0.10 timed; 0.40 and 0.45 run until the divergence
flag), the attractive-tail workload, the ensemble, the network and the warm
start.

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload instead.
Multi-GPU (torchrun): independent replicas, one slit per GPU (one slit is not
split across GPUs), max time over ranks, weak scaling.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS incl. Enskog force, % HBM roofline; time-to-steady-state warm vs cold"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index),
                                      "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([s.strip() for s in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 3 + k and s[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def bytes_alg(storage: int):
    """Algorithmic bytes per node per step: populations in and out once
    (2 x 19 x s_pop) plus the nonlocal fields written once and read once
    (n,u out 16, n in 4, g2 out 4, n,u,g2 in 20 = 44)."""
    s = 2 if storage == 1 else 4
    return 2 * 19 * s + 44


def kernel_bytes(storage: int):
    """Algorithmic bytes per node moved by each kernel class (each array element
    read or written once; stencil neighbours come from cache):
      ball_g2         dn in, dG out
      tail            dn in, F_tail out
      force           {dn,u} + dG in, F out
      collide_stream  19 populations in and out, {dn,u} and F in, the next
                      {dn,u} out (the pull pass)"""
    s = 2 if storage == 1 else 4
    return {"ball_g2": 8, "tail": 20, "force": 36, "collide_stream": 2 * 19 * s + 32 + 16}


# DRAM bytes per node of each step kernel (dram__bytes_read.sum + dram__bytes_write.sum of one
# ncu capture on the 128x128x192 sigma = 12 slit, default launch shapes, divided by its nodes;
# the same per-node traffic as the 256x256x192 capture of the pull pass, so it scales with the
# nodes of a launch). The ball kernel's dG writes stay in L2 at that size: read bytes only.
TRAFFIC_B_PER_NODE = {0: {"ball_g2": 5.8, "force": 40.9, "collide_stream": 209.7},
                      1: {"ball_g2": 5.8, "force": 40.9, "collide_stream": 157.5}}
# the in-place pull pass (FP32; the FP16 in-place populations of that capture,
# 120 MB, nearly fit in L2, so its DRAM figure does not scale and is left out)
TRAFFIC_INPLACE = {0: {"ball_g2": 5.8, "force": 40.9, "collide_stream": 197.1}}


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x over the ranks (the slowest rank's time), with a barrier
    after it; x itself on a single rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo, else lscpu), or 'unknown'."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_mlups(nx, ny, W, steps_hint, max_steps=20):
    import oracle

    o = oracle.Oracle(nx, ny, W.nz, W.sigma, W.eta, W.tau, body=W.body, seed=W.seed)
    t0 = time.perf_counter()
    o.step(1)
    per = time.perf_counter() - t0
    k = max(1, min(max_steps, int(steps_hint / max(per, 1e-3))))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    o.close()
    return nx * ny * W.nz * k / dt / 1e6, k, dt


def cpu_sample(steps_hint: float = 15.0):
    """Time the FP64 oracle on bounded samples of the workload: the sigma = 12
    slit at 64 x 64 x 192 on all host cores (the reported value), the same slit
    at 32 x 32 x 192 on one core, and the full 1000 steps of the 16 x 16 x 32
    sigma = 4 slit (eta 0.25) on all cores."""
    import oracle
    from paper_0712_2247_gb300.inputs import C0S, C2

    cores = oracle.threads()
    v, k, dt = _oracle_mlups(64, 64, C2, steps_hint)
    oracle.set_threads(1)
    try:
        v1, k1, dt1 = _oracle_mlups(32, 32, C2, steps_hint / 3, max_steps=10)
    finally:
        oracle.set_threads(cores)
    o = oracle.Oracle(C0S.nx, C0S.ny, C0S.nz, C0S.sigma, C0S.eta, C0S.tau, body=C0S.body, seed=C0S.seed)
    t0 = time.perf_counter()
    o.step(C0S.steps)
    dt0 = time.perf_counter() - t0
    o.close()
    return {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, 64x64x{C2.nz} slit of the same sigma/eta/tau/F_e, "
                      f"{k} steps after 1 untimed, {dt:.1f} s",
            "cpu_model": cpu_model(),
            "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1,
                              "sample": f"32x32x{C2.nz} slit, {k1} steps after 1 untimed, {dt1:.1f} s"},
            "c0s_full": {"value": C0S.nodes * C0S.steps / dt0 / 1e6, "unit": "MLUPS", "cores": cores,
                         "sample": f"{C0S.nx}x{C0S.ny}x{C0S.nz} sigma={C0S.sigma} eta={C0S.eta}, "
                                   f"{C0S.steps} steps, {dt0:.1f} s"}}, dt, k, 64 * 64 * C2.nz


def warm_start_leg(args):
    """Time to steady state, warm vs cold (reduced form of the learned warm
    start study): steady profiles of thin slits drawn from the ensemble
    distribution (training set, seed 4), the network trained on the tensor
    cores, then held-out 32x32xH slits (seed 5) run to the FP64 residual
    1e-8 from a cold uniform start and from the network's prediction."""
    import numpy as np
    import torch

    from paper_0712_2247_gb300 import inputs
    from paper_0712_2247_gb300 import surrogate as S
    from paper_0712_2247_gb300.mlp import MLP

    ptr = inputs.ensemble(args.ws_train, seed=4, nx=4, ny=4)
    n_z, ux_z, steps, res, gen_wall = S.steady_profiles(ptr)
    use = np.nonzero(steps != -2)[0]
    raw = S.raw_features(ptr.H, ptr.eta, ptr.F, ptr.tau, ptr.sigma)
    sc = S.Scaling.fit(raw[use])
    T, M = S.encode(n_z, ux_z, ptr)
    batch = 512
    net = MLP(S.NFEAT, 256, 3, 2 * S.HMAX, max_batch=1024, seed=4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = S.train(net, sc(raw[use]), T[use], M[use], steps=args.ws_adam, batch=batch)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # tensor-core work of one training step: forward and two backward products per layer
    flops = 3 * 2 * batch * sum(o * i for o, i in net.shapes)
    phe = inputs.ensemble(args.ws_heldout, seed=5)
    r = S.warm_vs_cold(net, sc, phe, 32, 32)
    net.close()
    return {
        "workload": f"train {args.ws_train} thin 4x4xH slits (H in [8,80], eta in [0.10,0.25], "
                    f"F log-uniform [1e-7,1e-5], tau in [0.6,1.2]); evaluate {args.ws_heldout} held-out "
                    f"32x32xH slits to residual 1e-8 (FP32)",
        "generation_s": gen_wall, "train_s": train_s, "adam_steps": args.ws_adam, "batch": batch,
        "loss_first": float(losses[0]), "loss_last": float(losses[-50:].mean()),
        "train_step_tflops": flops * args.ws_adam / train_s / 1e12,
        "cold_s": r["cold"]["wall_s"], "warm_s": r["warm"]["wall_s"], "wall_speedup": r["wall_speedup"],
        "steps_mean_cold": r["cold"]["steps_mean"], "steps_mean_warm": r["warm"]["steps_mean"],
        "floored_cold": r["cold"]["not_converged"], "floored_warm": r["warm"]["not_converged"],
        "final_profile_diff": r["final_profile_diff"], "prediction_error": r["prediction_error"],
    }


def ensemble_leg(args):
    """Throughput of the batched ensemble: 256 slits of 32x32xH (H in
    [8, 80], eta in [0.10, 0.25], F log-uniform in [1e-7, 1e-5], tau in
    [0.6, 1.2], SplitMix64 seed 3), FP16 population storage in place,
    advanced by the CUDA-graph runner (graphs of 100 steps, FP64 residual
    check after each) after the autotuner has picked the launch shapes. The
    tolerance is set below reach, so every slit runs all steps. The same
    ensemble with FP32 storage and with two population buffers is timed for
    comparison."""
    import numpy as np
    import torch

    from paper_0712_2247_gb300 import inputs, lbif

    p = inputs.ensemble(256, seed=3)
    e = lbif.Ensemble(p.H, p.eta, p.F, p.tau, p.sigma, p.nx, p.ny, storage=lbif.STORE_F16, seed=3, inplace=True)
    ball, group, staging = e.autotune(trials=3)
    e.run(tol=1e-300, max_steps=200, check_every=100)  # builds the graph
    steps = args.ens_steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e.run(tol=1e-300, max_steps=steps, check_every=100)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # the same kernels launched one by one, each timed with CUDA events: what
    # a single persistent launch could save at most is the graph's time per
    # step beyond the kernels' own (launch gaps and the residual checks)
    kms, nl = e.step_profiled(200)
    per = {k: kms[k] / nl[k] for k in kms if nl[k]}
    kern = sum(per.values())
    fluid = int(np.sum(p.H)) * p.nx * p.ny
    e.close()
    graph_ms = dt / steps * 1e3
    # the same ensemble with FP32 storage, and with two population buffers,
    # for comparison (same steps, graph)
    def other(storage, inplace):
        e2 = lbif.Ensemble(p.H, p.eta, p.F, p.tau, p.sigma, p.nx, p.ny, storage=storage, seed=3, inplace=inplace)
        e2.autotune(trials=3)
        e2.run(tol=1e-300, max_steps=200, check_every=100)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2.run(tol=1e-300, max_steps=steps, check_every=100)
        torch.cuda.synchronize()
        dt2 = time.perf_counter() - t0
        e2.close()
        return fluid * steps / dt2 / 1e6

    m32 = other(lbif.STORE_F32, True)
    m16_two = other(lbif.STORE_F16, False)
    return {"workload": "256 slits 32x32xH, sigma=4, FP16 storage in place, graph-captured steps",
            "fluid_nodes": fluid, "stacked_nodes": e.N, "steps": steps, "seconds": dt,
            "mlups_fluid": fluid * steps / dt / 1e6, "autotuned": {"ball_ctas": ball, "force_group": group,
                                                        "ball_staging": "tma" if staging else "loads"},
            "graph_ms_per_step": graph_ms, "kernel_ms_per_step": kern, "kernels_ms": per,
            "beyond_kernels_frac": (graph_ms - kern) / graph_ms,
            "mlups_fluid_fp32_storage": m32, "mlups_fluid_two_buffers": m16_two}


def mlp_leg(args):
    """Tensor-core throughput of the warm-start network's forward pass on a
    large batch (every layer one tcgen05 product with its fused epilogue),
    inputs and outputs resident on the device."""
    import torch

    from paper_0712_2247_gb300.mlp import MLP

    B = args.mlp_batch
    net = MLP(4, 256, 3, 160, max_batch=B, seed=1)
    X = torch.randn(B, 4, device="cuda", dtype=torch.float32)
    for _ in range(3):
        net.forward(X)
    torch.cuda.synchronize()
    reps = 20
    t0 = time.perf_counter()
    for _ in range(reps):
        net.forward(X)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    net.close()
    kpad = [16, 256, 256, 256]  # K of each product (the 4 inputs padded to 16)
    flops = 2 * B * sum(k * o for k, o in zip(kpad, [256, 256, 256, 160]))
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, kind = float(json.load(f)["bf16_tflops"]), "measured bf16_tflops (burst)"
    except Exception:
        peak, kind = 1900.0, "fallback"
    tf = flops / dt / 1e12
    return {"batch": B, "ms_per_forward": dt * 1e3, "tflops": tf, "peak_tflops": peak, "peak_kind": kind,
            "frac": tf / peak, "note": "4 products per forward, host-synchronised call (includes launch and sync)"}


def tail_leg(args):
    """The attractive-tail workload's shape: 256 x 256 x 128 slit, sigma = 8,
    LJ tail cut at 2.5 sigma, tau = 0.8, F_e = 1e-6, eta = 0.25, eps = 0.3.
    At kT = 1/3 a tail of eps = 1 puts the fluid inside its spinodal: a
    homogeneous start decomposes within ~30 steps (FP64 oracle, eta 0.25), and
    the kernels' divergence flags then add atomics to their times; eta = 0.40
    is beyond the scheme's stability at sigma = 8. The kernels' cost does not
    depend on eps or eta. Per-kernel CUDA-event times of 20 steps."""
    from paper_0712_2247_gb300 import lbif

    g = lbif.Slit(256, 256, 128, 8, 0.25, 0.8, body=(1e-6, 0, 0), tail=True, eps=0.3, rcut=2.5, seed=1)
    g.step(3)
    kms, nl = g.step_profiled(20)
    status = g.status()
    g.close()
    per = {k: kms[k] / nl[k] for k in kms if nl[k]}
    ms = sum(per.values())
    return {"workload": "slit 256x256x128 sigma=8 eta=0.25 tau=0.8 F_e=1e-6, LJ tail eps=0.3 rcut=2.5 sigma",
            "ms_per_step": ms, "mlups": 256 * 256 * 128 / (ms * 1e-3) / 1e6, "kernels_ms": per,
            "status": status}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    steps, warm = args.steps, args.warmup
    import oracle
    from paper_0712_2247_gb300.inputs import C2

    W = C2
    nx = ny = 32
    o = oracle.Oracle(nx, ny, W.nz, W.sigma, W.eta, W.tau, body=W.body, seed=W.seed)
    o.step(warm)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    nodes = nx * ny * W.nz
    v = nodes * steps / dt / 1e6
    cores = oracle.threads()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": dt / steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "slit 512x512x192 sigma=12 eta=0.25 tau=0.7 F_e=5e-7 "
                                   "(oracle sample 32x32x192 per step)", "storage": "f64"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{nx}x{ny}x{W.nz} slit per step, {steps} steps"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _slit(W, storage, seed, stream, inplace=False):
    from paper_0712_2247_gb300 import lbif

    return lbif.Slit(W.nx, W.ny, W.nz, W.sigma, W.eta, W.tau, body=W.body, storage=storage,
                     seed=seed, stream=stream, inplace=inplace)


def time_steps(g, steps, stream, storage, N, peak):
    """CUDA-event time of `steps` steps on the handle's stream, with every
    kernel class timed by the library between its launches; per-kernel
    milliseconds and algorithmic GB/s, the whole step's roofline fraction."""
    import torch

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    kms, nl = g.step_profiled(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    kb = kernel_bytes(storage)
    per_kernel = {k: {"ms": kms[k] / nl[k], "gbs_alg": kb[k] * N / (kms[k] / nl[k] * 1e-3) / 1e9}
                  for k in kms if nl[k]}
    mps = ms / steps
    return {"ms_per_step": mps, "mlups": N / (mps * 1e-3) / 1e6, "kernels": per_kernel,
            "bytes_alg_per_node": bytes_alg(storage),
            "step_roofline_frac": bytes_alg(storage) * N / (mps * 1e-3) / 1e9 / peak}, kms, nl, ms


def storage_leg(args, stream, peak, storage=1, inplace=False):
    """The benchmark slit with another population storage: FP16 (2^8 times
    the non-equilibrium parts) or one buffer in place: its own step time,
    kernels, roofline and device memory."""
    import torch

    from paper_0712_2247_gb300.inputs import c2

    W = c2(args.eta, storage)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    g = _slit(W, storage, W.seed, stream.cuda_stream, inplace=inplace)
    torch.cuda.synchronize()
    dev_bytes = free0 - torch.cuda.mem_get_info()[0]
    g.step(args.warmup)
    g.autotune(3)
    g.step(1)
    r, _, _, _ = time_steps(g, args.steps, stream, storage, W.nodes, peak)
    r["status"] = g.status()
    r["autotuned"] = g.shapes()
    r["pass"] = "pull, in place" if inplace else "pull"
    r["device_bytes"] = dev_bytes
    g.close()
    dom = max(r["kernels"], key=lambda k: r["kernels"][k]["ms"])
    r["roofline"] = {"kernel": dom, "achieved": r["kernels"][dom]["gbs_alg"], "peak": peak,
                     "frac": r["kernels"][dom]["gbs_alg"] / peak}
    return r


def eta_sweep_leg(args, stream, peak):
    """The benchmark slit's packing-fraction sweep: 0.10 timed like the
    headline (0.25); 0.40 and 0.45 stepped from the same seeded start until
    the device's divergence flag (non-finite or non-positive density, or a
    coarse-grained packing fraction reaching 1) is raised, checked every 5
    steps up to 100."""
    from paper_0712_2247_gb300.inputs import c2

    out = {}
    W = c2(0.10, 0)
    g = _slit(W, 0, W.seed, stream.cuda_stream)
    g.step(args.warmup)
    g.autotune(3)
    g.step(1)
    r, _, _, _ = time_steps(g, args.steps, stream, 0, W.nodes, peak)
    r["status"] = g.status()
    g.close()
    out["0.10"] = r
    for eta in (0.40, 0.45):
        W = c2(eta, 0)
        g = _slit(W, 0, W.seed, stream.cuda_stream)
        flagged = None
        for k in range(5, 101, 5):
            g.step(5)
            if g.status() != 0:
                flagged = k
                break
        out[f"{eta:.2f}"] = {"status": g.status(), "diverged_by_step": flagged,
                             "note": "beyond the explicit scheme's stability from a uniform start"}
        g.close()
    return out


def run_ours(args, world, rank, local):
    import torch

    torch.cuda.set_device(local)
    from paper_0712_2247_gb300 import build
    from paper_0712_2247_gb300.inputs import c2

    # one rank compiles (when the library is stale), the others wait for it
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
        if rank != 0:
            build.build()  # up to date now: returns at once
    storage = 1 if args.storage == "f16" else 0
    W = c2(args.eta, storage)
    if args.grid:
        nx, ny, nz = (int(v) for v in args.grid.lower().split("x"))
        W = W.with_(nx=nx, ny=ny, nz=nz)
    stream = torch.cuda.current_stream()
    g = _slit(W, storage, W.seed + rank, stream.cuda_stream, inplace=args.inplace)
    N = W.nodes
    peak, peak_kind = _peaks()
    # warm-up, then the launch shapes the library's autotuner picks on this
    # state (ball CTAs and staging, force tile group, pull segments and
    # gathers; results bit-identical), or its defaults (profiler captures,
    # whose timings would mislead the autotuner)
    g.step(args.warmup)
    if args.shapes == "auto":
        g.autotune(3)
    shapes = g.shapes()
    g.step(1)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        main, kms, nl, ms = time_steps(g, args.steps, stream, storage, N, peak)
    ms = max_over_ranks(ms, world)
    ms_per_step = ms / args.steps
    mlups = world * N / (ms_per_step * 1e-3) / 1e6
    status = g.status()

    # dominant kernel roofline, live CUDA-event timing of each launch class
    dom = max(kms, key=lambda k: kms[k])
    launches = sum(nl.values())
    kb = kernel_bytes(storage)
    dom_bytes = kb[dom] * N
    dom_ms = kms[dom] / max(nl[dom], 1)
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    step_gbs = bytes_alg(storage) * N / (ms_per_step * 1e-3) / 1e9
    tb = (TRAFFIC_INPLACE if args.inplace else TRAFFIC_B_PER_NODE).get(storage, {}).get(dom)

    # end to end through the C ABI's host-pointer path: per iteration the
    # density field goes from pinned host memory through lbif_set_fields
    # (on_device = 0: the library copies it in on the handle's stream and
    # starts the state from it), S steps run, and the FP64 profiles are read
    # back to the host (which synchronises every iteration)
    S = 10
    rho_h = torch.empty(W.nz * W.ny * W.nx, dtype=torch.float32, pin_memory=True)
    rho_h.fill_(float(g.n0))
    rho_np = rho_h.numpy().reshape(W.nz, W.ny, W.nx)
    iters = max(1, args.steps // S)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(iters):
        g.set_fields(rho_np)
        g.step(S)
        g.profiles(allow_diverged=True)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)  # the slowest replica
    e2e = {"value": world * N * S * iters / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": 4 * N / S, "d2h_bytes_per_step": 5 * 8 * W.nz / S,
           "note": f"per iteration: lbif_set_fields from {4 * N} B of pinned host memory (copied in "
                   f"on the handle's stream), {S} steps, FP64 profile readback"}
    g.close()

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu, _, _, _ = cpu_sample(args.cpu_seconds)

    def leg(enabled, fn, *a):
        if not enabled or world != 1:
            return None
        try:
            return fn(*a)
        except Exception as e:  # reported, never hides the throughput line
            return {"error": f"{type(e).__name__}: {e}"}

    f16 = leg(not args.no_sweep and storage == 0 and not args.inplace, storage_leg, args, stream, peak, 1, False)
    inpl = leg(not args.no_sweep and storage == 0 and not args.inplace, storage_leg, args, stream, peak, 0, True)
    f16_inpl = leg(not args.no_sweep and storage == 0 and not args.inplace, storage_leg, args, stream, peak, 1, True)
    sweep = leg(not args.no_sweep and storage == 0 and args.eta == 0.25, eta_sweep_leg, args, stream, peak)
    tail = leg(not args.no_tail, tail_leg, args)
    mlp = leg(not args.no_mlp, mlp_leg, args)
    ens = leg(not args.no_ensemble, ensemble_leg, args)
    warm = leg(not args.no_warm_start, warm_start_leg, args)
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"slit {W.nx}x{W.ny}x{W.nz} sigma={W.sigma} eta={W.eta} tau={W.tau} "
                               f"F_e={W.body[0]} bounce-back z, periodic x,y, seeded 1e-3 noise",
                   "storage": args.storage, "nodes": N,
                   "pass": "pull, in place" if args.inplace else "pull",
                   "autotuned": shapes, "parallelism": f"replicas x{world}",
                   "l2": "populations (>= 1.9 GB) exceed L2; no flush",
                   "bytes_alg_per_node": bytes_alg(storage),
                   "step_gbs_alg": step_gbs, "step_roofline_frac": step_gbs / peak,
                   "kernels": main["kernels"],
                   "status": status},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind + " hbm_gbs", "unit": "GB/s", "frac": achieved / peak,
                     "traffic": tb * N if tb else None,
                     "traffic_unit": "bytes per launch (ncu capture, scaled by nodes)",
                     "bytes_alg_per_launch": dom_bytes},
        "cpu_baseline": cpu,
        "storage_f16": f16,
        "storage_inplace": inpl,
        "storage_f16_inplace": f16_inpl,
        "eta_sweep": sweep,
        "ensemble": ens,
        "tail_workload": tail,
        "mlp_forward": mlp,
        "warm_start": warm,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["f32", "f16"], default="f32")
    ap.add_argument("--eta", type=float, default=0.25)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true", help="skip the warm vs cold study")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble throughput")
    ap.add_argument("--no-mlp", action="store_true", help="skip the tensor-core forward throughput")
    ap.add_argument("--no-tail", action="store_true", help="skip the attractive-tail workload")
    ap.add_argument("--mlp-batch", type=int, default=65536, help="rows of the tensor-core forward leg")
    ap.add_argument("--ens-steps", type=int, default=2000, help="timed steps of the ensemble leg")
    ap.add_argument("--ws-train", type=int, default=8192, help="training slits of the warm-start leg")
    ap.add_argument("--ws-adam", type=int, default=8000, help="Adam steps of the warm-start leg")
    ap.add_argument("--ws-heldout", type=int, default=128, help="held-out slits of the warm-start leg")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the FP16-storage record and the packing-fraction sweep")
    ap.add_argument("--inplace", action="store_true",
                    help="populations in one buffer (the main line's layout; default two buffers)")
    ap.add_argument("--shapes", choices=["auto", "default"], default="auto",
                    help="launch shapes: the autotuner's (auto) or the library defaults (profiler captures)")
    ap.add_argument("--grid", default=None,
                    help="override the slit extents NXxNYxNZ (profiling captures on a smaller case)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
