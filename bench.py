"""Benchmark of the fused coupled-LBM step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--storage fp32|fp16] [--impl ours|reference]
                [--flush] [--workload bubbles|ensemble|warmstart|unet|cpu]

One step = one pass of the whole hot path (moments, stencils, closures, forces,
the three collisions, streaming and boundary rules) over the 2048 x 512 bubble
channel (two bubbles, Poiseuille inlet, outflow, parabolic sigma(T)), with the
state resident in HBM.  The K timed steps run back to back between two CUDA events
on the lattice's stream: each step reads one 113 MB population buffer and writes
the other (plus 8 MB of (phi u)), 234 MB per step against the 126 MB L2, so a step
finds at most the tail of the previous step's writes in L2 (ncu: DRAM reads per
launch equal the algorithmic reads).  With --flush a 256 MiB write runs between
timed steps instead, outside per-step events (that write leaves up to the whole L2
dirty for the next step to write back).  Metric: lattice updates per second (MLUPS,
one update = one node through all three LBEs), whole job.  At N = 1 the line also
carries the metric's second half, `time_to_steady`: wall time to a steady-state
residual of 1e-8 from the cold start and from the learned warm start on the 20
held-out 512 x 128 channels (--no-steady skips it).  Prints one JSON line.

N > 1 (torchrun, one rank per GPU): independent replicas (the path has no
data-path exchange); value = all ranks' updates / max-over-ranks time.
--impl reference times the FP64 CPU oracle on this machine's host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 2048, 512
WORKLOAD = "bubbles_2048x512"
# algorithmic bytes per lattice update: every population read once and written once
# (27 x 2 x element size) plus the previous (phi u) read and written (2 x 2 x 4 B);
# FP16 storage adds each node's three 8-byte reference records (read and written)
ALG_BYTES = {"fp32": 27 * 2 * 4 + 16, "fp16": 27 * 2 * 2 + 16 + 48}
CPU_SAMPLE_SECONDS = 15.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def _kernel_hash():
    """Hash of the step kernel's sources (the files the ncu counters describe)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_11320_gb300", "csrc")
    for name in ("lattice.cuh", "step.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(storage):
    """DRAM bytes per step-kernel launch from the committed ncu summary, if it was
    taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "step_%s_%s.json" % (storage, WORKLOAD))
    try:
        with open(path) as fh:
            d = json.load(fh)
        if d.get("kernel_hash") == _kernel_hash():
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def max_over_ranks(x, world, device):
    """The largest value of x over all ranks (for times: the slowest rank's), or x
    itself when running alone.  All ranks must call it."""
    if world <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes, steps, world, seconds):
    """Whole-job rate in MLUPS: each of the `world` ranks advances its own replica of
    `nodes` nodes by `steps` steps within `seconds` (the slowest rank's time)."""
    return nodes * steps * world / seconds / 1e6


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_oracle_sample(seconds, threads=None):
    """Time the FP64 oracle on the bubble workload for about `seconds` of CPU work."""
    from oracle.oracle import OracleSim, num_threads, set_threads
    from paper_2306_11320_gb300 import workloads as WL

    if threads:
        set_threads(threads)
    params, fields, _ = WL.bubbles(nx=NX, ny=NY)
    sim = OracleSim(NX, NY, params)
    sim.init(**fields)
    sim.step(1)  # first touch of every buffer
    steps, t0 = 0, time.perf_counter()
    while True:
        sim.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds and steps >= 2:
            break
    return NX * NY * steps / el / 1e6, steps, el, num_threads()


def bench_reference(args, rank, world):
    if rank != 0:
        return
    # a bounded sample of the workload: about a minute of oracle steps, whatever --steps
    mlups, steps, el, cores = run_oracle_sample(60.0)
    line = {
        "metric": "coupled-LBM MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "l2": "inputs > L2 (CPU run)"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": "%d oracle steps of the %dx%d bubble channel" % (steps, NX, NY)},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# step cap of the time-to-steady runs: every cold and warm run of the 20 held-out channels
# converges within 1.47M steps, so the cap only guards against a run that never does
STEADY_MAX_STEPS = 2_000_000


def time_to_steady(instances=None, log=lambda m: None):
    """Cold against learned warm start on the held-out warm-start channels (512 x 128
    heated microchannel), wall time to max(r_u, r_T) < 1e-8 with r every RESID_K steps,
    at most STEADY_MAX_STEPS steps; returns (rows, summary) of warmstart.compare/summarize."""
    from paper_2306_11320_gb300 import warmstart as WS

    net, norm, meta = WS.load(WS.WEIGHTS)
    insts = WS.held_out(meta, instances)
    rows = WS.compare(net, norm, insts, tols=(1e-8,), max_steps=STEADY_MAX_STEPS, log=log)
    return rows, WS.summarize(rows, (1e-8,)), meta


def bench_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2306_11320_gb300 import workloads as WL
    from paper_2306_11320_gb300.tpflbm import STORAGE_FP16, STORAGE_FP32, Lattice

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    storage = STORAGE_FP16 if args.storage == "fp16" else STORAGE_FP32
    params, fields, _ = WL.bubbles(nx=NX, ny=NY)
    if storage == STORAGE_FP16:
        params.update(WL.fp16_scales(params))
    params["normal_law"] = 1 if args.normal == "local" else 0
    if args.collision == "trt":
        params.update(collision=1, trt_lambda=0.25)
    stream = torch.cuda.Stream(device=dev)
    lat = Lattice(NX, NY, params, storage=storage, stream=stream)
    f32 = {k: v.astype(np.float32) for k, v in fields.items()}
    lat.init(**f32)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev) if args.flush else None

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            lat.step(1)
            if args.flush:
                flush.fill_(1)
        barrier()
        with ClockSampler(local_rank) as clk:
            if args.flush:
                starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
                ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
                for k in range(args.steps):
                    starts[k].record(stream)
                    lat.step(1)
                    ends[k].record(stream)
                    flush.fill_(1)
                barrier()
                times = [a.elapsed_time(b) for a, b in zip(starts, ends)]  # ms
                step_ms = sum(times)
            else:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                # after the synchronisation the GPU is idle: an untimed spin (about 0.2 s, so
                # that the clock sampler also sees the GPU busy next to a short timed region)
                # keeps it busy while the start event and the K launches are queued, so the
                # events enclose the K steps' device time and not the first launch's latency
                torch.cuda._sleep(400_000_000)
                e0.record(stream)
                for _ in range(args.steps):
                    lat.step(1)
                e1.record(stream)
                barrier()
                step_ms = e0.elapsed_time(e1)
    total_ms = max_over_ranks(step_ms, world, dev)
    diag = lat.diagnostics()

    # end to end through the public API with host buffers: H2D of the initial fields
    # from pinned memory, then every step the step itself and a D2H read of its
    # outcome (tpflbm_status_async: the step kernels' 4-byte error flag copied to pinned
    # host memory on a second stream, so that the next step does not queue behind the
    # copy; the host checks step k's flag once it has landed, while step k + 1 already
    # runs), and D2H of the final fields
    host_in = {k: torch.from_numpy(v).pin_memory() for k, v in f32.items()}
    host_out = [torch.empty((NY, NX), dtype=torch.float32).pin_memory() for _ in range(5)]
    flags = torch.zeros(2, dtype=torch.int32).pin_memory()
    done_ev = [torch.cuda.Event(), torch.cuda.Event()]
    copy_stream = torch.cuda.Stream(device=dev)
    import ctypes

    def check_flag(k):
        done_ev[k % 2].synchronize()
        if int(flags[k % 2]) != 0:
            raise RuntimeError("step %d: a step kernel gave up waiting for its copies" % k)

    barrier()
    t0 = time.perf_counter()
    lat.init(**host_in)
    for k in range(args.steps):
        lat._check(lat.lib.tpflbm_step(lat.h, 1))
        lat._check(lat.lib.tpflbm_status_async(lat.h, ctypes.c_void_p(flags[k % 2].data_ptr()),
                                               ctypes.c_void_p(copy_stream.cuda_stream)))
        done_ev[k % 2].record(copy_stream)
        if k > 0:
            check_flag(k - 1)
    check_flag(args.steps - 1)
    lat._check(lat.lib.tpflbm_get_fields(lat.h, *[ctypes.c_void_p(t.data_ptr()) for t in host_out]))
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)

    if rank != 0:
        return
    units = NX * NY * args.steps * world
    value = job_mlups(NX * NY, args.steps, world, total_ms * 1e-3)
    per_launch_s = total_ms * 1e-3 / args.steps
    alg = ALG_BYTES[args.storage] * NX * NY
    peak, peak_kind = _peaks()
    achieved = alg / per_launch_s / 1e9
    cpu = None
    if world == 1 and not args.no_cpu:
        mlups, steps, el, cores = run_oracle_sample(CPU_SAMPLE_SECONDS)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": "%d FP64 oracle steps of the %dx%d bubble channel (%.1f s)" % (steps, NX, NY, el)}
    steady = None
    if world == 1 and not args.no_steady:
        # the metric's second half: time to steady state, plain against learned warm start
        rows, summ, meta = time_to_steady()
        agg = summ["aggregate_1e-08"]
        steady = {"workload": "warmstart_512x128", "instances": len(rows), "tol": 1e-8, "max_steps": STEADY_MAX_STEPS,
                  "cold_s": agg["cold_s"], "warm_s": agg["warm_s"], "ratio": agg["ratio"],
                  "cold_unconverged": agg["cold_unconverged"], "warm_unconverged": agg["warm_unconverged"],
                  "per_instance_median": summ["speedup_time_1e-08"]["median"], "target": ">= 3x",
                  "train_instances": meta["train"]}
    field_bytes = 5 * 4 * NX * NY
    line = {
        "metric": "coupled-LBM MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "storage": args.storage, "normal": args.normal, "collision": args.collision,
                   "l2": ("256 MiB L2 flush between timed steps" if args.flush else
                          "inputs > L2: 234 MB read+written per step vs 126 MB L2, steps back to back"),
                   "parallelism": "replicas"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": _traffic(args.storage),
                     "peak_source": peak_kind, "alg_bytes_per_launch": alg,
                     "kernel": "k_step"},
        "cpu_baseline": cpu,
        "e2e": {"value": units / e2e_s / 1e6, "unit": "MLUPS",
                "h2d_bytes_per_step": field_bytes / args.steps,
                "d2h_bytes_per_step": field_bytes / args.steps + 4},
        "gpu_launches": args.steps,
        "clocks": dict(clk.summary(), window="timed region and the 0.2 s untimed spin before it"),
        "check": {"nonfinite": diag["nonfinite"], "sum_phi": diag["sum_phi"]},
        "time_to_steady": steady,
    }
    print(json.dumps(line), flush=True)


def bench_ensemble(args, rank, world, local_rank):
    """256 independent lattices of 64x64 to 512x256 nodes (microchannel and drop,
    Ma 0.01-50, viscosity and conductivity ratios 0.1-10), one batched launch per
    step replayed from CUDA graphs, variant (tile shape, general or TMA-staged path)
    chosen by the autotuner.  Each rank
    runs its own copy of the ensemble."""
    import numpy as np
    import torch

    from paper_2306_11320_gb300 import workloads as WL
    from paper_2306_11320_gb300.tpflbm import STORAGE_FP16, STORAGE_FP32, Batch

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    storage = STORAGE_FP16 if args.storage == "fp16" else STORAGE_FP32
    members = WL.ensemble(n=256, seed=0)
    lats = []
    for p, f, m in members:
        if storage == STORAGE_FP16:
            p = dict(p, **WL.fp16_scales(p))
        lats.append((m["nx"], m["ny"], p))
    stream = torch.cuda.Stream(device=dev)
    b = Batch(lats, storage=storage, stream=stream)
    for k, (p, f, m) in enumerate(members):
        b.init(k, **{n: v.astype(np.float32) for n, v in f.items()})
    best, ms = b.tune(steps=10)
    nodes = sum(nx * ny for nx, ny, _ in lats)
    steps = max(2, args.steps - args.steps % 2)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        b.step(2 * max(2, args.warmup))
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            e0.record(stream)
            b.step(steps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        total_ms = e0.elapsed_time(e1)
    total_ms = max_over_ranks(total_ms, world, dev)
    d, rc = b.diagnostics()
    if rank != 0:
        return
    shapes = Batch.variants(b.lib)
    alg = ALG_BYTES[args.storage] * nodes
    peak, peak_kind = _peaks()
    achieved = alg / (total_ms * 1e-3 / steps) / 1e9
    line = {
        "metric": "coupled-LBM MLUPS", "value": job_mlups(nodes, steps, world, total_ms * 1e-3), "unit": "MLUPS",
        "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": total_ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ensemble_256", "lattices": len(lats), "nodes": nodes, "storage": args.storage,
                   "tile": "%dx%d" % shapes[best],
                   "tile_path": "tma" if best == Batch.tma_variant(b.lib) else "general", "tune_ms_per_step": ms,
                   "l2": "state %.0f MB > L2 (steps timed back to back)" % (2 * alg / 1e6)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                     "alg_bytes_per_launch": alg, "kernel": "k_step_batch"},
        "gpu_launches": steps,
        "clocks": clk.summary(),
        "check": {"nonfinite_lattices": int((d[:, 7] > 0).sum()), "rc": rc},
    }
    print(json.dumps(line), flush=True)


# the warm-start U-Net's 3x3 layers at batch 4 (512 x 128 input): N, H, W, Cin, Cout
UNET_LAYERS = [(4, 128, 512, 32, 32), (4, 64, 256, 64, 64), (4, 32, 128, 128, 128), (4, 16, 64, 256, 256),
               (4, 32, 128, 384, 128), (4, 64, 256, 192, 64), (4, 128, 512, 96, 32)]


def bench_unet(args, rank, world, local_rank):
    """The warm-start U-Net's tensor-core kernels: per 3x3 layer shape of the network
    (batch 4), the forward convolution (bias + ReLU), the data gradient and the weight
    gradient through tpfnet_* (CUDA events, --warmup untimed and min(--steps, 50) timed
    calls each; FLOP = 2 N H W 9 Cin Cout per call), which kernel each takes, and a whole
    training step (forward, MSE, backward, Adam) on random data.  The U-Net is off the
    lattice's measured path; this line documents its kernels."""
    import ctypes

    import numpy as np
    import torch

    from paper_2306_11320_gb300.unet import UNet, net_library

    torch.cuda.set_device(local_rank)
    lib = net_library()
    stream = torch.cuda.current_stream()
    s = ctypes.c_void_p(stream.cuda_stream)
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    peak, peak_kind = _bf16_peak()
    reps = max(1, min(args.steps, 50))  # calls timed per kernel and shape (the default --steps is for the lattice)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps  # us per call

    layers = []
    with ClockSampler(local_rank) as clk:
        for N, H, W, Cin, Cout in UNET_LAYERS:
            g = torch.Generator(device="cuda").manual_seed(N * H * W + Cin + Cout)
            x = torch.randn((N, H, W, Cin), device="cuda", generator=g).to(torch.bfloat16)
            wt = (torch.randn((9, Cout, Cin), device="cuda", generator=g) / (9 * Cin) ** 0.5).to(torch.bfloat16)
            b = torch.randn(Cout, device="cuda", generator=g)
            y = torch.empty((N, H, W, Cout), dtype=torch.bfloat16, device="cuda")
            dz = torch.randn((N, H, W, Cout), device="cuda", generator=g).to(torch.bfloat16)
            dx = torch.empty((N, H, W, Cin), dtype=torch.bfloat16, device="cuda")
            wf = torch.empty(9 * Cin * Cout, dtype=torch.bfloat16, device="cuda")
            dw = torch.zeros((9, Cout, Cin), device="cuda")
            db = torch.zeros(Cout, device="cuda")
            flop = 2.0 * N * H * W * 9 * Cin * Cout
            row = {"shape": [N, H, W, Cin, Cout],
                   "kernel": {"forward": "tcgen05 BN %d" % lib.tpfnet_conv3x3_tcgen05(N, H, W, Cin, Cout)
                              if lib.tpfnet_conv3x3_tcgen05(N, H, W, Cin, Cout) else "mma.sync",
                              "weight_gradient": "tcgen05" if lib.tpfnet_conv3x3_wgrad_tcgen05(N, H, W, Cin, Cout)
                              else "mma.sync"}}
            for name, fn in (
                    ("forward", lambda: lib.tpfnet_conv3x3(P(x), N, H, W, Cin, P(wt), P(b), Cout, 1, P(y), s)),
                    ("data_gradient", lambda: lib.tpfnet_conv3x3_dgrad(P(dz), N, H, W, Cout, P(wt), Cin, P(wf), P(dx), s)),
                    ("weight_gradient", lambda: lib.tpfnet_conv3x3_wgrad(P(x), P(dz), N, H, W, Cin, Cout, P(dw), P(db), s))):
                us = timed(fn)
                row[name] = {"us": round(us, 2), "tflops": round(flop / us / 1e6, 1),
                             "frac_of_bf16_peak": round(flop / us / 1e6 / peak, 4)}
            layers.append(row)
        net = UNet(4, 4, seed=1)
        rng = np.random.default_rng(0)
        xin = torch.from_numpy(rng.standard_normal((4, 128, 512, 32)).astype(np.float32)).to(torch.bfloat16).cuda()
        tgt = torch.from_numpy(rng.standard_normal((4, 128, 512, 4)).astype(np.float32)).cuda()
        for _ in range(3):
            net.train_step(xin, tgt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            net.train_step(xin, tgt)
        torch.cuda.synchronize()
        train_ms = (time.perf_counter() - t0) * 1e3 / reps
    if lib.tpfnet_status() != 0:
        raise RuntimeError("a tcgen05 kernel's bounded wait ran out")
    if rank != 0:
        return
    tot = {k: sum(r[k]["us"] for r in layers) for k in ("forward", "data_gradient", "weight_gradient")}
    flops = sum(2.0 * n * h * w * 9 * ci * co for n, h, w, ci, co in UNET_LAYERS)
    line = {
        "metric": "U-Net 3x3 convolution TFLOP/s (forward, the network's seven layer shapes)",
        "value": flops / tot["forward"] / 1e6, "unit": "TFLOP/s", "n_gpus": world, "steps": reps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic", "config": {"workload": "unet_warmstart_layers", "batch": 4},
        "roofline": {"bound": "tensor", "achieved": flops / tot["forward"] / 1e6, "peak": peak, "unit": "TFLOP/s",
                     "frac": flops / tot["forward"] / 1e6 / peak, "peak_source": peak_kind,
                     "kernel": "k_conv3x3_tc"},
        "totals_us": {k: round(v, 1) for k, v in tot.items()},
        "layers": layers,
        "train_step_ms": round(train_ms, 3),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def bench_warmstart(args, rank, world, local_rank):
    """Time to steady state of the 512 x 128 heated microchannel from the cold start
    and from the trained network's prediction (committed weights), on the held-out
    instances (all 20 by default), each on its own lattice and stream: wall time to
    max(r_u, r_T) < 1e-8 with r checked every RESID_K steps.  The warm time includes
    the network's input upload, inference, phase-field projection and initialisation.
    The target is a 3x shorter wall time; value is the aggregate ratio (total cold
    time over total warm time, a cold run that never converges counted at max_steps)."""
    import torch

    from paper_2306_11320_gb300 import warmstart as WS

    torch.cuda.set_device(local_rank)
    tol, max_steps = 1e-8, STEADY_MAX_STEPS
    with ClockSampler(local_rank) as clk:
        rows, summ, meta = time_to_steady(args.instances)
    insts = rows
    if rank != 0:
        return
    agg = summ["aggregate_1e-08"]
    line = {
        "metric": "time-to-steady speed-up (cold / learned warm start)", "value": agg["ratio"], "unit": "x",
        "n_gpus": world, "steps": None, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 LBM, bf16 network", "data": "synthetic",
        "config": {"workload": "warmstart_512x128", "instances": len(insts), "tol": tol, "residual_K": WS.RESID_K,
                   "max_steps": max_steps, "train_instances": meta["train"], "epochs": meta["epochs"]},
        "target": ">= 3x shorter wall time to r < 1e-8",
        "aggregate": agg, "per_instance_time": summ["speedup_time_1e-08"],
        "steps_median": summ["speedup_steps_1e-08"], "final_rel_l2_max": summ["final_rel_l2_max"],
        "rows": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items() if k != "final_rel_l2"}
                 for r in rows],
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def bench_cpu_table(args):
    """The FP64 oracle on this machine's host cores, at one thread and at all threads, on
    each workload configuration: the 128 x 32 microchannel, the 256 x 1024 drop, the
    2048 x 512 bubble channel and the 512 x 128 warm-start channel.  Each leg runs the
    configuration's first steps for about 20 s of CPU time (at most the step count the
    configuration names) and reports MLUPS.  The warm-start channel's cold start needs
    hundreds of thousands of steps to reach r < 1e-8; its CPU time to steady state is
    given as that step count (measured on the GPU path) over the oracle's rate."""
    import platform

    from oracle.oracle import OracleSim, num_threads, set_threads
    from paper_2306_11320_gb300 import warmstart as WS
    from paper_2306_11320_gb300 import workloads as WL

    cases = [
        ("microchannel_128x32", 128, 32, WL.microchannel()[:2], 20000),
        ("drop_256x1024", 256, 1024, WL.drop_migration(Ma=0.1)[:2], 2000),
        ("bubbles_2048x512", 2048, 512, WL.bubbles()[:2], 200),
        ("warmstart_channel_512x128", 512, 128, WS.channel(dict(lam_r=1.0, hr=1.0, k=1))[:2], 800000),
    ]
    all_threads = num_threads()
    rows = []
    for name, nx, ny, (params, fields), max_steps in cases:
        for threads in (1, all_threads):
            set_threads(threads)
            sim = OracleSim(nx, ny, params)
            sim.init(**fields)
            sim.step(1)
            steps, t0 = 0, time.perf_counter()
            chunk = max(1, int(2e6 // (nx * ny)))
            while steps < max_steps:
                n = min(chunk, max_steps - steps)
                sim.step(n)
                steps += n
                if time.perf_counter() - t0 >= 20.0:
                    break
            el = time.perf_counter() - t0
            rows.append({"workload": name, "threads": threads, "steps": steps, "seconds": round(el, 3),
                         "mlups": nx * ny * steps / el / 1e6})
    set_threads(all_threads)
    cpu = "unknown"
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                cpu = ln.split(":", 1)[1].strip()
                break
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                cpu = ln.split(":", 1)[1].strip()
    except Exception:
        pass
    print(json.dumps({"kind": "oracle", "cores": all_threads, "nproc": os.cpu_count(), "cpu": cpu,
                      "machine": platform.machine(), "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000,
                    help="timed steps (the default keeps the clock samples inside the timed region)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--storage", choices=("fp32", "fp16"), default="fp32")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-steady", action="store_true",
                    help="skip the time-to-steady comparison (cold against learned warm start) of the default line")
    ap.add_argument("--flush", action="store_true",
                    help="write 256 MiB between timed steps (per-step events) instead of timing steps back to back")
    ap.add_argument("--workload", choices=("bubbles", "ensemble", "warmstart", "unet", "cpu"), default="bubbles",
                    help="bubbles: the 2048x512 channel (the headline line); ensemble: the "
                         "256-lattice parameter sweep through the batched launch; warmstart: time to "
                         "steady state, cold vs learned warm start, on held-out microchannels; unet: the "
                         "warm-start network's tensor-core kernels per layer shape; cpu: the "
                         "FP64 oracle at one thread and at all threads on every workload configuration")
    ap.add_argument("--instances", type=int, default=20, help="warmstart: held-out instances to time")
    ap.add_argument("--collision", choices=("bgk", "trt"), default="bgk",
                    help="NS and thermal collision operator: BGK (the paper's) or two relaxation times")
    ap.add_argument("--normal", choices=("stencil", "local"), default="stencil",
                    help="interface normal of the Allen-Cahn source: stencil gradient or local recovery")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return bench_reference(args, rank, world)
    if args.workload == "cpu":
        return bench_cpu_table(args) if rank == 0 else None
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.workload == "ensemble":
            bench_ensemble(args, rank, world, local_rank)
        elif args.workload == "warmstart":
            bench_warmstart(args, rank, world, local_rank)
        elif args.workload == "unet":
            bench_unet(args, rank, world, local_rank)
        else:
            bench_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
