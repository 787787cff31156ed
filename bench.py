#!/usr/bin/env python
"""Benchmark: output audio samples/s of batched nonlinear string synthesis.

Default workload (one "step"): the batching workload, the largest that runs
on one GPU: 4096 strings of uneven N, 4 s at 48 kHz each (192,000 samples),
f0 log-uniform 30-2000 Hz, half with vibrato (5-7 Hz, +-20 cents), half with
glissando (+-1 octave), kappa U[0.5,3], alpha U[1,10], sigma0 U[0.1,2],
sigma1 U[1e-6,1e-4], excitation uniform over pluck / hammer / bow (seed 3).
Warps per CTA are autotuned once; each step replays one captured CUDA graph
of the prepared launch (one persistent kernel per class, concurrently) on
freshly created strings (inputs resident in device memory before the timed
region); L2 is flushed between timed steps.  `--workload mixed` times the
256-string batch (2 s, f0 40-1000 Hz, seed 2) with direct launches instead.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--workload modulated|mixed|serving|gradient|dataset|single]

Under torchrun each rank synthesizes its own batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.  `--impl
reference` times the FP64 CPU oracle (the only reference this method has)
on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
# A batch's kernel classes run concurrently, one stream each.  With the CUDA
# runtime's default of 8 hardware work queues, steps enqueued back to back
# (--enqueue-ahead) put two class kernels of a step behind one queue some of
# the time: measured on the 4096-string batch, a mean of 4.96 s per step with
# the default against 4.81 s with 32 queues (4.52 s with each step launched
# once the previous one ended, the timed loop's default).  The setting must
# precede CUDA's initialisation; a value the caller set is kept.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2311_18505_gb300 import workloads as W  # noqa: E402

METRIC = "output audio samples/s (all strings)"
UNIT = "samples/s"
FS = 48000.0
# nominal FP32 CUDA-core rate for context: SMs x 128 FP32 lanes x 2 flops (FMA) x clock
FP32_LANES_PER_SM = 128

# Algorithmic FLOPs per grid-point update (one exact step, no repeated
# sweeps): stencil right-hand side, matrix assembly, one exact tridiagonal
# factor + solve and the coupling terms; see the design notes for the count.
FLOP_U_LINEAR = 24.0      # RHS 19 + prefactored solve 5
FLOP_U_NONLINEAR = 75.0   # RHS 31 + assembly 8 + factor 4 + solve 5 + coupling 27
FLOP_Z = 20.0             # RHS 8 + spread 4 + prefactored solve 5 + interpolation 3
FLOP_EXCITATION = 30.0    # per string-step with a hammer or bow (scalar solve + update)
FLOP_RESPONSE_U = 10.0    # per transverse row for the unit-force response (nonlinear, forced)


# The minimal counts per update of the survey of the method (prefactored
# solves, no delta form): linear 17, nonlinear 40-55 (47.5 taken), longitudinal
# 20-30 (25 taken), 10 per forced string-step plus 9 per transverse row.
MINIMAL_COUNTS = (17.0, 47.5, 25.0, 10.0, 9.0)


def algorithmic_flops(strings, grids, select=None, counts=None) -> float:
    """Algorithmic FLOPs of one synthesis of `strings` (optionally only the
    indices in `select`), with this build's counts or `counts` = (linear u,
    nonlinear u, z, per forced step, per forced u row)."""
    lin_u, nl_u, z_row, exc, resp = counts or (FLOP_U_LINEAR, FLOP_U_NONLINEAR, FLOP_Z, FLOP_EXCITATION,
                                               FLOP_RESPONSE_U)
    tot = 0.0
    for idx, (d, (nt, nl)) in enumerate(zip(strings, grids)):
        if select is not None and idx not in select:
            continue
        n_u = nt - 1
        linear = d["alpha"] == 1.0
        n_z = 0 if linear else max(nl - 1, 0)
        per = n_u * (lin_u if linear else nl_u) + n_z * z_row
        if d["excitation"]["kind"] != "pluck":
            per += exc + (0.0 if linear else n_u * resp)
        tot += per * (d["n_samples"] - 2)
    return tot


KERNEL_SOURCES = ["sfd_kernel.cu", "sfd_df64.cuh", "sfd_device.cuh", "sfd_step_reg.cuh", "sfd_step_smem.cuh", "sfd_types.h"]


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2311_18505_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profile_figures(name: str) -> dict | None:
    """The "key: value" figures of a committed ncu summary (profiles/<name>),
    or None when it is missing or was taken on other kernel sources (its
    kernel_sources_sha256 line differs from the current sources)."""
    import re
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    figs = {}
    for m in re.finditer(r"^- ([a-z0-9_]+): ([0-9a-fA-F.e+-]+)\s*$", open(path).read(), re.M):
        figs[m.group(1)] = m.group(2)
    if figs.get("kernel_sources_sha256") != kernel_sources_hash():
        return None
    return figs


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ distributed

def dist_setup(n_gpus: int):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, value: float) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------ CPU oracle

def cpu_oracle_rate(strings, n_samples: int, threads: int = 0):
    """Time the FP64 oracle (OpenMP over strings) on `strings` x n_samples."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    _, used = oracle.run_batch(strings, n_samples=n_samples, threads=threads)
    dt = time.perf_counter() - t0
    return len(strings) * n_samples / dt, used, dt


def oracle_cost(d: dict, n_samples: int) -> float:
    """Grid-point updates of one string over n_samples (the oracle's work
    grows with the unknowns it solves for per step)."""
    import oracle
    nt, nl = oracle.grid(d)
    return ((nt - 1) + (0 if d["alpha"] == 1.0 else max(nl - 1, 0))) * float(n_samples)


def extrapolated_rate(strings, sample, n_sample: int, seconds: float) -> float:
    """Samples/s of the whole workload at the speed the oracle showed on a
    sample of it: the sample's grid-point updates per second, divided into
    the workload's grid-point updates, gives the time the workload takes."""
    upd_rate = sum(oracle_cost(d, n_sample) for d in sample) / seconds
    total_samples = sum(d["n_samples"] for d in strings)
    total_updates = sum(oracle_cost(d, d["n_samples"]) for d in strings)
    return total_samples / (total_updates / upd_rate)


WORKLOAD_NAME = ("256 strings x 2 s at 48 kHz: f0 log-U[40,1000] Hz, kappa U[0.5,3], alpha U[1,10], "
                 "sigma0 U[0.1,2], sigma1 U[1e-6,1e-4], pluck/hammer/bow uniform (seed 2)")
WORKLOAD_MODULATED = ("4096 strings x 4 s at 48 kHz, uneven N: f0 log-U[30,2000] Hz, half vibrato (5-7 Hz, "
                      "+-20 cents), half glissando (+-1 octave), parameters and excitations as the mixed batch "
                      "(seed 3); one CUDA-graph replay per step, autotuned warps per CTA")


def make_workload(args, rank):
    if args.workload == "gradient":
        base, _ = W.batch_gradient(64, seconds=0.5, seed=4 + 1000 * rank)
        return base, WORKLOAD_GRADIENT
    if args.workload == "serving":
        trace = W.serving_trace(args.rate, args.trace_seconds, seed=5 + 1000 * rank)
        return [d for _, d in trace], WORKLOAD_SERVING.format(rate=args.rate, secs=args.trace_seconds,
                                                              live=args.max_live)
    split = getattr(args, "partition", "none") == "lpt"
    seed_rank = 0 if split else rank   # a split batch is the same batch on every rank
    if args.workload == "modulated":
        strings = W.batch_modulated(args.strings or 4096, seconds=args.seconds or 4.0, seed=3 + 1000 * seed_rank)
        name = WORKLOAD_MODULATED
    else:
        strings = W.batch_mixed(args.strings or 256, seconds=args.seconds or 2.0, seed=2 + 1000 * seed_rank)
        name = WORKLOAD_NAME
    if split:
        from paper_2311_18505_gb300 import partition
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        args.batch_samples = sum(d["n_samples"] for d in strings)
        strings = [strings[i] for i in partition.shard(strings, rank, ws)]
        name += f"; split across {ws} ranks by cost (greedy longest processing time)"
    return strings, name


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    strings, workload_name = make_workload(args, 0)
    sample = strings[: args.ref_strings]
    n = args.ref_samples or (48000 if args.workload == "modulated" else 96000)
    for _ in range(args.warmup):
        cpu_oracle_rate(sample, n)
    rates, used, dts = [], 0, []
    for _ in range(args.steps):
        r, used, dt = cpu_oracle_rate(sample, n)
        rates.append(r)
        dts.append(dt)
    # the workload's samples/s at the oracle's measured speed on the sample
    value = extrapolated_rate(strings, sample, n, sum(dts) / len(dts))
    desc = (f"first {len(sample)} strings of the workload x their first {n} samples per step, "
            f"extrapolated to the whole workload by grid-point updates (sum over strings of "
            f"(N_t - 1 + N_l - 1) x samples)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(dts) / len(dts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name, "reference": "FP64 CPU oracle (OpenMP)",
                                        "sample_rate_measured": len(sample) * n * len(dts) / sum(dts)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ our arm

def run_ours(args, ws, rank, local):
    import torch
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    # roofline denominators, measured on this device (clocks sampled meanwhile)
    pclk = ClockSampler(local)
    pclk.start()
    peak_runs = [sfd.sfd_measure_peaks(local) for _ in range(3)]
    time.sleep(0.45)
    pclk_stats = pclk.stop()
    peaks = {k: max(r[k] for r in peak_runs) for k in peak_runs[0]}
    stream = torch.cuda.Stream(dev)            # the context's stream (also the capture stream)
    torch.cuda.set_stream(stream)
    strings, workload_name = make_workload(args, rank)
    # the device pool holds every prepared batch's strings and, for the
    # end-to-end leg, the whole step's output
    out_bytes = 4 * sum(d["n_samples"] for d in strings)
    pool = (256 << 20) + (0 if args.no_e2e else out_bytes) + (args.steps + 1) * len(strings) * (48 << 10)
    ctx = sfd.sfd_ctx_create(local, stream.cuda_stream, pool)
    sfd.sfd_ctx_set_warp_pairs(ctx, bool(args.warp_groups))
    graphed = args.workload == "modulated"
    ns = np.array([d["n_samples"] for d in strings], dtype=np.int64)
    offs = np.zeros(len(ns), dtype=np.int64)
    offs[1:] = np.cumsum(ns)[:-1]
    total = int(ns.sum())
    out = torch.empty(total, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 18, dtype=torch.float32, device=dev)   # 256 MiB > L2

    def make_batch():
        hs = [sfd.string_from_dict(ctx, d) for d in strings]
        return hs, sfd.sfd_batch_create(ctx, hs)

    def free_batch(hb):
        hs, b = hb
        sfd.sfd_batch_destroy(b)
        for h in hs:
            sfd.sfd_string_destroy(h)

    grids, classes = [], []   # grid sizes and kernel classes as the library derived them
    for d in strings:
        h = sfd.string_from_dict(ctx, d)
        nt, nl, _, _ = sfd.sfd_string_info(h)
        grids.append((nt, nl))
        classes.append(sfd.sfd_string_kernel_class(h))
        sfd.sfd_string_destroy(h)
    flops = algorithmic_flops(strings, grids)
    updates = sum(((nt - 1) + (0 if d["alpha"] == 1.0 else max(nl - 1, 0))) * (d["n_samples"] - 2)
                  for d, (nt, nl) in zip(strings, grids))

    wpc = args.warps_per_cta
    if not graphed:
        sfd.sfd_ctx_set_timing(ctx, True)
    if graphed and not wpc:   # autotune warps per CTA once, on throwaway copies
        hb = make_batch()
        wpc = sfd.sfd_batch_autotune(hb[1], 2048)
        free_batch(hb)

    def prepared_batch():
        """A fresh batch, its job table uploaded and (modulated workload) its
        launch captured as a CUDA graph."""
        hb = make_batch()
        if wpc:
            sfd.sfd_batch_set_warps_per_cta(hb[1], wpc)
        g = None
        if graphed:
            sfd.sfd_batch_prepare(hb[1], ns, out, offs)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                sfd.sfd_batch_launch(hb[1])
        return hb, g

    def run_step(hb, g):
        if g is not None:
            g.replay()
        else:
            sfd.sfd_batch_synthesize(hb[1], ns, out, offs)

    # warm-up
    for _ in range(args.warmup):
        hb, g = prepared_batch()
        run_step(hb, g)
        torch.cuda.synchronize(dev)
        del g
        free_batch(hb)
    # timed: inputs for every step created (and captured) before the region
    batches = [prepared_batch() for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    class_ms = [0.0] * sfd.SFD_KERNEL_CLASSES
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize(dev)
    launches = 0
    for i, (hb, g) in enumerate(batches):
        flush.zero_()
        ev[i][0].record(stream)
        run_step(hb, g)
        ev[i][1].record(stream)
        if not args.enqueue_ahead:
            # launched on an idle GPU, the class kernels start in launch order,
            # heaviest first; enqueued behind a running step they become ready
            # together and the GPU's dispatch order varies (4.5-5.5 s per
            # step on the 4096-string batch against 4.51-4.55 s this way)
            ev[i][1].synchronize()
        launches += len(set(classes)) if g is not None else sfd.sfd_last_launch_count(ctx)
        if g is None:
            # per-class kernel times, recorded with events on each kernel's own stream
            ms_k, _ = sfd.sfd_ctx_kernel_times(ctx)
            class_ms = [a + b for a, b in zip(class_ms, ms_k)]
    torch.cuda.synchronize(dev)
    barrier(ws)
    clk = clocks.stop()
    sfd.sfd_ctx_set_timing(ctx, False)
    times_ms = [a.elapsed_time(b) for a, b in ev]
    if rank == 0:
        print("step ms:", " ".join(f"{t:.1f}" for t in times_ms), file=sys.stderr)
    y = out[: min(total, 1 << 20)].float().cpu().numpy()
    finite = bool(np.all(np.isfinite(y)))
    for hb, g in batches:
        del g
        free_batch(hb)
    direct_ms = None
    if graphed:
        # after the timed region: one direct launch of the same prepared
        # batch with per-class kernel events (on each class's own stream),
        # which a graph replay does not record
        hb = make_batch()
        if wpc:
            sfd.sfd_batch_set_warps_per_cta(hb[1], wpc)
        sfd.sfd_ctx_set_timing(ctx, True)
        flush.zero_()
        sfd.sfd_batch_synthesize(hb[1], ns, out, offs)
        direct_ms, _ = sfd.sfd_ctx_kernel_times(ctx)
        sfd.sfd_ctx_set_timing(ctx, False)
        torch.cuda.synchronize(dev)
        free_batch(hb)
    t_total = max_over_ranks(ws, sum(times_ms) / 1e3)
    split = getattr(args, "partition", "none") == "lpt"
    value = (args.batch_samples if split else ws * total) * args.steps / t_total
    ms_step = 1e3 * t_total / args.steps

    # e2e through the public API with host buffers (create -> synthesize to
    # pinned host memory, which the kernels write directly -> destroy),
    # wall-clock per step
    e2e = None
    if not args.no_e2e:
        host_out = torch.empty(total, dtype=torch.float32).pin_memory()

        def e2e_step():
            hs = [sfd.string_from_dict(ctx, d) for d in strings]
            b = sfd.sfd_batch_create(ctx, hs)
            sfd.lib().sfd_batch_synthesize_host(
                b, ns.ctypes.data_as(sfd.ctypes.POINTER(sfd.ctypes.c_int64)), host_out.data_ptr(),
                offs.ctypes.data_as(sfd.ctypes.POINTER(sfd.ctypes.c_int64)), None)
            sfd.sfd_batch_destroy(b)
            for h in hs:
                sfd.sfd_string_destroy(h)

        e2e_step()   # untimed: first touch of the output buffer and the staging
        h0, d0 = sfd.sfd_ctx_transfer_bytes(ctx)
        barrier(ws)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize(dev)
        dt = max_over_ranks(ws, time.perf_counter() - t0)
        h1, d1 = sfd.sfd_ctx_transfer_bytes(ctx)
        e2e = {"value": (args.batch_samples if split else ws * total) * args.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": int((h1 - h0) / args.e2e_steps),
               "d2h_bytes_per_step": int((d1 - d0) / args.e2e_steps)}
    sfd.sfd_ctx_destroy(ctx)

    if rank != 0:
        return 0
    peak = peaks["fp32_tflops"]
    nominal = sm_count * FP32_LANES_PER_SM * 2 * (clk["sm_max_mhz"] if clk else 2070.0) * 1e6 / 1e12
    class_names = ["synth_kernel_reg1", "synth_kernel_reg3", "synth_kernel_reg5", "synth_kernel_reg7",
                   "synth_kernel_reg9", "synth_kernel_smem"]
    per_class = {}
    src_ms = class_ms if sum(class_ms) > 0 else (direct_ms or [0.0] * len(class_names))
    div = args.steps if sum(class_ms) > 0 else 1
    for k in range(len(class_names)):
        idx = {i for i, c in enumerate(classes) if c == k}
        if not idx or src_ms[k] <= 0:
            continue
        f = algorithmic_flops(strings, grids, idx)
        per_class[class_names[k]] = {"ms": src_ms[k] / div, "strings": len(idx),
                                     "tflops": f / (src_ms[k] / div / 1e3) / 1e12}
    if sum(class_ms) > 0:
        # dominant kernel: the class kernel with the largest average launch time
        dom = max(range(len(class_ms)), key=lambda k: class_ms[k])
        dom_ms = class_ms[dom] / args.steps
        dom_idx = {i for i, c in enumerate(classes) if c == dom}
        kernel = class_names[dom]
    else:
        # graph replays: the class kernels run concurrently in one replay,
        # timed together by the events around it on the capture stream
        dom_ms = sum(times_ms) / len(times_ms)
        dom_idx = set(range(len(strings)))
        kernel = "synth_kernel_* (all classes, concurrent in one graph replay)"
    achieved = algorithmic_flops(strings, grids, dom_idx) / (dom_ms / 1e3) / 1e12
    achieved_min = algorithmic_flops(strings, grids, dom_idx, MINIMAL_COUNTS) / (dom_ms / 1e3) / 1e12
    # DRAM traffic and ncu pipe / shared-memory fractions from the committed
    # summaries of this workload's kernels (None if taken on other sources)
    tr = profile_figures(f"synth_kernel_dram_{args.workload}.md") if ws == 1 else None
    traffic = None
    if tr and "dram_bytes_per_sample" in tr:
        traffic = float(tr["dram_bytes_per_sample"]) * sum(
            strings[i]["n_samples"] for i in dom_idx)
    dom_class = max(per_class, key=lambda k: per_class[k]["ms"]) if per_class else None
    sm_prof = profile_figures(f"{dom_class}_full_small.md") if dom_class else None
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        sample = strings[: args.cpu_strings or (128 if args.workload == "modulated" else 256)]
        n_cpu = args.cpu_samples or sample[0]["n_samples"]
        rate, used, dt = cpu_oracle_rate(sample, n_cpu)
        extrap = extrapolated_rate(strings, sample, n_cpu, dt)
        cpu = {"value": extrap, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": f"first {len(sample)} strings of the workload x {n_cpu} samples ({dt:.1f} s wall, "
                         f"{rate:.4g} samples/s on them), extrapolated to the whole workload by grid-point "
                         f"updates (sum over strings of (N_t - 1 + N_l - 1) x samples)"}
        # one thread, for comparison with a single-core figure (a bounded sample)
        one = strings[:16]
        r1, _, dt1 = cpu_oracle_rate(one, 24000, threads=1)
        cpu["single_thread"] = {"value": extrapolated_rate(strings, one, 24000, dt1), "unit": UNIT, "cores": 1,
                                "sample": f"first {len(one)} strings x 24000 samples ({dt1:.1f} s wall), "
                                          f"extrapolated likewise"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong" if split else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name, "strings": len(strings),
                   "seconds": float(strings[0]["n_samples"] / FS), "fs": FS,
                   "samples_per_step": total, "l2": "flushed between timed steps (256 MiB write)",
                   "launch": ("one CUDA-graph replay per step (concurrent class kernels), warps per CTA "
                              f"{'set' if args.warps_per_cta else 'autotuned'} to {wpc}") if graphed else
                             "one persistent kernel per class per step, one warp per string",
                   "step_issue": ("enqueued back to back" if args.enqueue_ahead else
                                  "each timed step launched once the previous one ended (host waits on its "
                                  "end event; the value sums the steps' event times)")},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "fp32_frac": achieved / peak,
                     "frac_minimal_counts": achieved_min / peak,
                     "smem_frac": (float(sm_prof["smem_pct_of_peak"]) / 100.0
                                   if sm_prof and "smem_pct_of_peak" in sm_prof else None),
                     "fma_pipe_frac": (float(sm_prof["fma_pipe_pct_of_peak"]) / 100.0
                                       if sm_prof and "fma_pipe_pct_of_peak" in sm_prof else None),
                     "pipe_source": (f"ncu, profiles/{dom_class}_full_small.md (kernel {dom_class}, small case)"
                                     if sm_prof else None),
                     "traffic": traffic,
                     "kernel": kernel, "kernel_ms": dom_ms, "kernel_strings": len(dom_idx),
                     "per_class": per_class,
                     "per_class_source": ("events around each class kernel in the timed steps" if sum(class_ms) > 0
                                          else "one direct launch of the same batch after the timed region, "
                                               "events around each class kernel on its own stream"),
                     "step_flops_total": flops,
                     "peak_note": ("of measured: FP32 FMA microbenchmark (sfd_measure_peaks, best of 3 x 5 "
                                   "launches) on this device; nominal SMs x 128 lanes x 2 x max clock = "
                                   f"{nominal:.1f} TFLOP/s"),
                     "measured_peaks": dict(peaks, sm_count=sm_count,
                                            sm_mhz_during=(pclk_stats or {}).get("sm_mhz"))},
        "grid_point_updates_per_s": ws * updates * args.steps / t_total,
        "realtime_factor": ws * total / FS * args.steps / t_total,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "outputs_finite": finite,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ serving

WORKLOAD_SERVING = ("serving: Poisson note requests at {rate:g}/s for {secs:g} s (seed 5), f0 log-U[40,1000] Hz, "
                    "duration U[0.25,4] s, params and excitations as the mixed batch, 1024-sample chunks, "
                    "admission by device memory, up to {live} live notes")


def run_serving(args, ws, rank, local):
    """Replay the arrival trace in real time through the serving API: submit
    each request at its arrival time, pump (admit, launch the next chunk,
    deliver the previous one) until every note has been delivered.  Reports
    delivered samples/s, first-chunk latency percentiles and the real-time
    factor (audio seconds delivered per wall second)."""
    import torch
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    secs = args.trace_seconds
    trace = W.serving_trace(args.rate, secs, seed=5 + 1000 * rank)
    ctx = sfd.sfd_ctx_create(local, stream.cuda_stream, 2 << 30)
    sfd.sfd_ctx_set_warp_pairs(ctx, bool(args.warp_groups))
    sv = sfd.sfd_server_create(ctx, 1024, args.max_live)
    reqs = [sfd.request_from_dict(d, i) for i, (_, d) in enumerate(trace)]   # marshalled before the clock starts

    def drained():
        st = sfd.sfd_server_stats_get(sv)
        return st.queued == 0 and st.live == 0 and st.in_flight == 0

    # warm-up: a burst of short notes through the same path
    for i, (_, d) in enumerate(W.serving_trace(args.rate, 0.05, seed=99)):
        sfd.sfd_server_submit(sv, sfd.request_from_dict(d, 10 ** 9 + i, n_samples=3000))
    while not drained():
        sfd.sfd_server_pump(sv, copy=False)

    barrier(ws)
    clocks = ClockSampler(local)
    clocks.start()
    t0 = sfd.sfd_server_clock(sv) + 0.01
    n, i = len(trace), 0
    lat, samples, notes_done, peak_queue, peak_live, pumps = [], 0, 0, 0, 0, 0
    while True:
        now = sfd.sfd_server_clock(sv)
        while i < n and t0 + trace[i][0] <= now:
            reqs[i].arrival_s = t0 + trace[i][0]
            sfd.sfd_server_submit(sv, reqs[i])
            i += 1
        st = sfd.sfd_server_stats_get(sv)
        peak_queue, peak_live = max(peak_queue, st.queued), max(peak_live, st.live)
        if st.queued == 0 and st.live == 0 and st.in_flight == 0:
            if i == n:
                break
            time.sleep(max(0.0, min(0.002, t0 + trace[i][0] - now)))
            continue
        for tag, first, cnt, last, status, ready, arrival in sfd.sfd_server_pump(sv, copy=False):
            if first == 0:
                lat.append(ready - arrival)
            samples += cnt
            notes_done += last
        pumps += 1
    t1 = sfd.sfd_server_clock(sv)
    clk = clocks.stop()
    h0, d0 = sfd.sfd_ctx_transfer_bytes(ctx)
    sfd.sfd_server_destroy(sv)
    sfd.sfd_ctx_destroy(ctx)
    wall = max_over_ranks(ws, t1 - t0)
    if rank != 0:
        return 0
    lat_ms = np.array(lat) * 1e3
    audio_s = samples / FS
    line = {
        "metric": METRIC, "value": ws * samples / wall, "unit": UNIT, "n_gpus": ws, "steps": 1, "warmup": 1,
        "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_SERVING.format(rate=args.rate, secs=secs, live=args.max_live),
                   "notes": n, "offered_audio_s": float(sum(d["n_samples"] for _, d in trace) / FS),
                   "l2": "not flushed (serving replay: state stays resident by design)"},
        "serving": {"first_chunk_latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                                               "p99": float(np.percentile(lat_ms, 99)),
                                               "max": float(lat_ms.max())},
                    "realtime_factor": ws * audio_s / wall, "notes_completed": notes_done,
                    "peak_live": peak_live, "peak_queued": peak_queue, "pumps": pumps,
                    "wall_s": wall, "trace_s": secs},
        "e2e": {"value": ws * samples / wall, "unit": UNIT, "h2d_bytes_per_step": int(h0), "d2h_bytes_per_step": int(d0)},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ gradients

WORKLOAD_GRADIENT = ("differentiation: 64 plucked or hammered strings x 0.5 s at 48 kHz (seed 4), loss = sum of "
                     "squared differences to targets rendered from parameters perturbed by up to 5 %, gradients "
                     "w.r.t. kappa, alpha, sigma0, sigma1, amplitude; checkpoint every 1024 steps; one step = "
                     "forward + adjoint")


def run_gradient(args, ws, rank, local):
    """Time forward synthesis plus the reverse sweep of the discrete adjoint
    (the forward records the trajectory when it fits, else each segment is
    replayed from its checkpoint; then the adjoint kernel) on the
    differentiation workload."""
    import torch
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    base, target = W.batch_gradient(64, seconds=0.5, seed=4 + 1000 * rank)
    n = base[0]["n_samples"]
    ctx = sfd.sfd_ctx_create(local, stream.cuda_stream, 1 << 30)
    sfd.sfd_ctx_set_warp_pairs(ctx, bool(args.warp_groups))
    # targets rendered by the same synthesis
    hs = [sfd.string_from_dict(ctx, d) for d in target]
    b = sfd.sfd_batch_create(ctx, hs)
    ys, _ = sfd.sfd_batch_synthesize_host(b, [n] * len(target))
    sfd.sfd_batch_destroy(b)
    for h in hs:
        sfd.sfd_string_destroy(h)
    tgt = torch.from_numpy(np.stack(ys)).to(dev)
    tape = sfd.sfd_tape_create(ctx, base, n, 1024)
    y = torch.empty(len(base), n, device=dev, dtype=torch.float32)

    def step():
        t0 = time.perf_counter()
        sfd.sfd_tape_forward(tape, y)
        t1 = time.perf_counter()
        dy = (2.0 * (y - tgt)).contiguous()
        torch.cuda.synchronize(dev)
        g = sfd.sfd_tape_backward(tape, dy, len(base))
        t2 = time.perf_counter()
        return g, t1 - t0, t2 - t1

    for _ in range(args.warmup):
        step()
    barrier(ws)
    clocks = ClockSampler(local)
    clocks.start()
    fw, bw, tot = [], [], []
    for _ in range(args.steps):
        torch.cuda.synchronize(dev)
        g, a, c = step()
        fw.append(a)
        bw.append(c)
        tot.append(a + c)
    clk = clocks.stop()
    sfd.sfd_tape_destroy(tape)
    sfd.sfd_ctx_destroy(ctx)
    t_step = max_over_ranks(ws, sum(tot) / len(tot))
    if rank != 0:
        return 0
    samples = len(base) * n
    line = {
        "metric": METRIC, "value": ws * samples / t_step, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (forward), double-float f32x2 (adjoint recursion)", "data": "synthetic",
        "config": {"workload": WORKLOAD_GRADIENT, "strings": len(base), "samples_per_string": n,
                   "checkpoint_every": 1024, "timing": "host wall clock around the two C-ABI calls (each "
                   "synchronises its stream)"},
        "gradient": {"forward_ms": 1e3 * statistics.median(fw), "backward_ms": 1e3 * statistics.median(bw),
                     "backward_over_forward": statistics.median(bw) / statistics.median(fw),
                     "grad_finite": bool(np.all(np.isfinite(g)))},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


WORKLOAD_DATASET = ("dataset generation: {count} items x {secs:g} s at 48 kHz drawn per item (seed 0) from the "
                    "default distribution (f0 log-U[40,1000] Hz, kappa U[0.5,3], alpha U[1,10], pluck/hammer/bow "
                    "with randomised friction a and eps, 25 % vibrato, 25 % glissando), {shard}-item shards "
                    "rendered as GPU batches and written to local disk (npz + jsonl)")


def run_dataset(args, ws, rank, local):
    """Time the dataset generator end to end: per-item draws, GPU batch
    rendering through the C-ABI and shard files on local disk (the writer
    thread overlaps the next shard's rendering)."""
    import shutil
    import tempfile
    import torch
    from paper_2311_18505_gb300 import dataset as D

    torch.cuda.set_device(local)
    count = args.strings or 1024
    secs = args.seconds or 1.0
    shard = 256
    dist = D.Distribution(seconds=secs)
    render = D.GpuRenderer(local)
    from paper_2311_18505_gb300 import sfd as _sfd
    _sfd.sfd_ctx_set_warp_pairs(render.ctx, bool(args.warp_groups))
    render_s = [0.0]

    def timed(dicts):
        t0 = time.perf_counter()
        out = render(dicts)
        render_s[0] += time.perf_counter() - t0
        return out

    root = tempfile.mkdtemp(prefix="sfd_dataset_")
    try:
        for w in range(args.warmup):
            D.generate(os.path.join(root, f"w{w}"), min(count, shard), dist, seed=0, shard_size=shard,
                       rank=rank, world=ws, render=timed)
            shutil.rmtree(os.path.join(root, f"w{w}"))
        barrier(ws)
        clocks = ClockSampler(local)
        clocks.start()
        walls = []
        render_s[0] = 0.0
        from paper_2311_18505_gb300 import sfd
        h2d0, d2h0 = sfd.sfd_ctx_transfer_bytes(render.ctx)
        for k in range(args.steps):
            out = os.path.join(root, f"s{k}")
            t0 = time.perf_counter()
            D.generate(out, count, dist, seed=0, shard_size=shard, rank=rank, world=ws, render=timed)
            walls.append(time.perf_counter() - t0)
            shutil.rmtree(out)
        clk = clocks.stop()
        h2d1, d2h1 = sfd.sfd_ctx_transfer_bytes(render.ctx)
    finally:
        render.close()
        shutil.rmtree(root, ignore_errors=True)
    t_step = max_over_ranks(ws, sum(walls) / len(walls))
    if rank != 0:
        return 0
    n_shards = len(D.shard_ranges(count, shard))
    mine = len(D.shards_of_rank(n_shards, 0, ws))
    samples = count * int(round(secs * FS))
    line = {
        "metric": METRIC, "value": samples / t_step, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_DATASET.format(count=count, secs=secs, shard=shard), "items": count,
                   "shards": n_shards, "shards_on_rank0": mine,
                   "timing": "host wall clock around generate() (draws, renders, writes)"},
        "dataset": {"render_s_per_step": render_s[0] / args.steps, "wall_s_per_step": t_step,
                    "bytes_written_per_step": samples * 4},
        "e2e": {"value": samples / t_step, "unit": UNIT, "h2d_bytes_per_step": (h2d1 - h2d0) // args.steps,
                "d2h_bytes_per_step": (d2h1 - d2h0) // args.steps},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


WORKLOAD_SINGLE = ("single string (config 1): f0 110 Hz, kappa 1, alpha {alpha:g}, sigma0 0.5, sigma1 1e-5, 1 mm "
                   "pluck at 0.3, pickup 0.7, 1 s at 48 kHz, one sfd_synthesize call per step")


def run_single(args, ws, rank, local):
    """Plain single-string stepping: one string per launch (one warp, or a
    warp group when its longitudinal grid is large), the form the batched,
    served and graph-replayed launches are compared with."""
    import torch
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = sfd.sfd_ctx_create(local, stream.cuda_stream, 256 << 20)
    sfd.sfd_ctx_set_warp_pairs(ctx, bool(args.warp_groups))
    alpha = args.alpha
    d = W.single_string(alpha=alpha, seconds=args.seconds or 1.0)
    n = d["n_samples"]
    out = torch.empty(n, dtype=torch.float32, device=dev)
    ms = []
    clocks = ClockSampler(local)
    for k in range(args.warmup + args.steps):
        h = sfd.string_from_dict(ctx, d)
        if k == args.warmup:
            barrier(ws)
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        sfd.sfd_synthesize(h, n, out)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            ms.append(e0.elapsed_time(e1))
        sfd.sfd_string_destroy(h)
    clk = clocks.stop()
    nt, nl = string_grid(d, sfd, ctx)
    sfd.sfd_ctx_destroy(ctx)
    t = max_over_ranks(ws, sum(ms) / len(ms) / 1e3)
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": ws * n / t, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_SINGLE.format(alpha=alpha), "strings": 1, "n_t": nt, "n_l": nl,
                   "timing": "CUDA events around sfd_synthesize on the context stream (device output)"},
        "grid_point_updates_per_s": (nt - 1 + (nl - 1 if alpha > 1 else 0)) * (n - 2) / t,
        "realtime_factor": (n / FS) / t,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def string_grid(d, sfd, ctx):
    """(N_t, N_l) of a string as the library sizes it."""
    h = sfd.string_from_dict(ctx, d)
    try:
        return tuple(sfd.sfd_string_info(h)[:2])
    finally:
        sfd.sfd_string_destroy(h)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="modulated", choices=["modulated", "mixed", "serving", "gradient",
                                                                 "dataset", "single"])
    ap.add_argument("--alpha", type=float, default=1.0, help="single: stiffness-to-tension ratio (1 or 3)")
    ap.add_argument("--partition", default="none", choices=["none", "lpt"],
                    help="N > 1, mixed/modulated: split one batch across the ranks by cost (strong scaling) "
                         "instead of one batch per rank (weak scaling)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: note requests per second")
    ap.add_argument("--trace-seconds", type=float, default=60.0, help="serving: length of the arrival trace")
    ap.add_argument("--max-live", type=int, default=8192, help="serving: live-note slots")
    ap.add_argument("--strings", type=int, default=0)
    ap.add_argument("--seconds", type=float, default=0.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--enqueue-ahead", action="store_true",
                    help="launch each timed step without waiting for the previous one to end")
    ap.add_argument("--warp-groups", type=int, default=1, choices=[0, 1],
                    help="1: large-grid strings may take 2 or 4 warps (sfd_ctx_set_warp_pairs)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--warps-per-cta", type=int, default=0, choices=[0, 1, 2, 4],
                    help="modulated: warps per CTA (0: autotuned once before the warm-up)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # oracle samples (0: per workload).  Baseline: the first 128 strings of
    # the 4096-string batch over their whole 4 s (~10 s on 16 cores), or the
    # whole 256-string mixed batch; reference arm: the first 128 strings
    # over their first second (modulated) or 2 s (mixed) per step
    ap.add_argument("--cpu-strings", type=int, default=0)
    ap.add_argument("--cpu-samples", type=int, default=0)
    ap.add_argument("--ref-strings", type=int, default=128)
    ap.add_argument("--ref-samples", type=int, default=0)
    return ap.parse_args(argv)


def main(argv=None):
    args = parse_args(argv)
    ws, rank, local = dist_setup(args.gpus)
    try:
        if args.impl == "reference":
            return run_reference(args, ws, rank)
        if args.workload == "serving":
            return run_serving(args, ws, rank, local)
        if args.workload == "gradient":
            return run_gradient(args, ws, rank, local)
        if args.workload == "dataset":
            return run_dataset(args, ws, rank, local)
        if args.workload == "single":
            return run_single(args, ws, rank, local)
        return run_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
