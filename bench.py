#!/usr/bin/env python3
"""Benchmark of the checkerboard local-update sweep on one GB300 (or N, as
independent replicas).

Workload (one "step" = one Metropolis sweep, with E and M measured, of every
chain): the multi-spin-coded 2D Ising batch L in {1024, 4096, 16384} x
beta in {0.30, 0.40, 0.4406868, 0.50, 0.60}, periodic, hot start, 15 chains;
rank r runs the same 15 lattices with its own chain ids (weak scaling, no
data-path collective: chains are independent).  value = attempted spin flips
per second over all ranks.  The SU(2) heat-bath on 32^4 at beta in
{1.5, 2.0, 2.3, 2.6} is timed in the same run and reported under "components".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

The reference arm times the CPU oracle (oracle/, plain C, one core) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Ising spin-flips/s, SU(2) link-updates/s, eff. samples/s at beta_c vs plain"
BETAS = [0.30, 0.40, 0.4406868, 0.50, 0.60]
SIZES = [1024, 4096, 16384]
SU2_BETAS = [1.5, 2.0, 2.3, 2.6]
SU2_L = 32
# The MSC half-sweep is bound by the integer multiplier: every attempted flip
# consumes one 32-bit Philox4x32-10 word, a quarter of a block of 10 rounds x 2
# (32 x 32 -> 64)-bit products = 10 32-bit multiplies (high and low halves).
MUL32_PER_FLIP = 10.0
MUL32_PER_BLOCK = 40.0
# Nominal 32-bit integer multiplies per SM and clock on compute capability
# 10.x, for the derived figure reported beside the measured peak.
MUL32_PER_SM_CLK = 64
# Algorithmic bytes per SU(2) link update: read + write of the link once per sweep.
SU2_BYTES_PER_UPDATE = 32.0
# Algorithmic instructions per SU(2) link update (one issue slot per thread
# instruction, FMA = 1): staple 12 quaternion products x 16 + 5 quaternion sums
# x 4 = 212; |W|, V, alpha 11; Kennedy-Pendleton 20 per try x 1.2 tries = 24;
# direction on S^2 18; X V, reprojection and store 26; 19 link loads; Philox
# 2.2 blocks x (20 wide multiplies + 20 xors) = 88  ->  ~400.
SU2_INSTR_PER_UPDATE = 400.0
# Thread instructions issued per SM and clock: 4 schedulers x 32 lanes.
ISSUE_PER_SM_CLK = 128
# DRAM bytes (read + write) per MSC half-sweep launch of this workload from one
# ncu capture (179.0 MB read: both colour planes once; 47.9 MB written: the
# changed words), valid only for the kernel sources it was captured from:
# reported when the SHA-256 of those files still matches, else null.
MSC_TRAFFIC = {"bytes_per_launch": 226.89e6, "captured": "2026-12-03 (GB300, 4 launches averaged)",
               "sources_sha256": "b28af9ee335484ab6a487e37c1bb41dfb71d84693f36ba11c3daf6a7269fb643"}
MSC_KERNEL_SOURCES = ["ising.cu", "ising_dev.cuh", "philox.cuh", "mc_internal.cuh", "fastdiv.cuh"]


def kernel_sources_sha256(names) -> str:
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_0903_3053_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measure_philox_peak(mc, torch, sms: int, reps: int = 5) -> dict:
    """Multiply ceiling measured in this run: the library's pure-Philox kernel
    (8 CTAs of 256 threads per SM, 2048 blocks per thread, nothing else),
    timed with CUDA events on the current stream; the best of `reps`."""
    blocks, threads, iters = sms * 8, 256, 2048
    out = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    mc.philox_rate(blocks, threads, iters, 1, out)
    torch.cuda.synchronize()
    best = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        e0.record(stream)
        mc.philox_rate(blocks, threads, iters, 1, out)
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, MUL32_PER_BLOCK * blocks * threads * iters / (e0.elapsed_time(e1) / 1e3))
    return {"mul32_per_s": best, "blocks": blocks, "threads": threads, "blocks_per_thread": iters}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- distributed
def dist_setup():
    from paper_0903_3053_gb300 import replicas
    world, rank, local = replicas.env_world()
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    from paper_0903_3053_gb300 import replicas
    replicas.barrier(world)


def max_over_ranks(x: float, world: int) -> float:
    from paper_0903_3053_gb300 import replicas
    return replicas.max_over_ranks(x, world, "cuda")


def cid(rank: int, index: int) -> int:
    from paper_0903_3053_gb300 import replicas
    return replicas.chain_id(rank, index)


# ----------------------------------------------------------------------------- workload
def ising_chains(rank: int):
    import paper_0903_3053_gb300 as mc
    out = []
    for i, L in enumerate(SIZES):
        for j, b in enumerate(BETAS):
            idx = i * len(BETAS) + j
            out.append(mc.ising(L, b, seed=1, chain_id=cid(rank, idx), hot=True))
    return out


def flips_per_step() -> int:
    return len(BETAS) * sum(L * L for L in SIZES)


def run_gb300(args):
    import torch

    import paper_0903_3053_gb300 as mc

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev_props = torch.cuda.get_device_properties(local)
    stream = torch.cuda.current_stream()
    K, W = args.steps, args.warmup

    # ---- device-resident timed region ------------------------------------------
    chains = ising_chains(rank)
    batch = mc.Batch(chains, layout=mc.MC_LAYOUT_MSC32, series_capacity=K + W + 8)
    batch.set_mode(mc.MC_MODE_GRID, args.threads)
    batch.sweep(W, 1)
    batch.read_series()
    sms = dev_props.multi_processor_count
    peak = measure_philox_peak(mc.mc, torch, sms)
    batch.profile(True)
    batch.profile_read()
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(K):
        batch.sweep(1, 1)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clock_info = clocks.stop()
    ms = t0.elapsed_time(t1)
    launches, kernel_ms = batch.profile_read()
    series = batch.read_series()
    assert series.shape[1] == K, series.shape
    batch.profile(False)
    ms_max = max_over_ranks(ms, world)
    flips = flips_per_step() * K * world
    value = flips / (ms_max / 1e3)
    # dominant kernel: the MSC half-sweep (launches = 2 per step)
    half_ms = kernel_ms / max(launches, 1)
    mul_per_launch = MUL32_PER_FLIP * flips_per_step() / 2
    achieved = mul_per_launch / (half_ms / 1e3)
    clk = clock_info.get("sm_mhz") or clock_info.get("sm_max_mhz")
    derived_peak = sms * MUL32_PER_SM_CLK * clk * 1e6 if clk else None
    sha = kernel_sources_sha256(MSC_KERNEL_SOURCES)
    traffic_ok = MSC_TRAFFIC["sources_sha256"] == sha
    batch.close()
    del batch
    torch.cuda.empty_cache()

    # ---- end to end through the C ABI, host buffers -----------------------------
    e2e = run_e2e(mc, torch, rank, min(K, args.e2e_steps), world)

    # ---- SU(2) and batched-chain components -------------------------------------------
    small = run_ising_64(mc, torch, rank, world)
    su2 = run_su2(mc, torch, rank, args.su2_steps, world, sms * ISSUE_PER_SM_CLK * (clk or 2070.0) * 1e6)
    batched = run_batched(mc, torch, rank, args.batch_steps, world)
    ess_cmp = run_ess(args) if not args.no_ess else None
    paper = run_paper_protocol(mc, torch) if not args.no_paper else None

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "spin-flips/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms_max / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {
            "workload": "2D Ising, multi-spin-coded uint32 (32 spins/word), L in {1024, 4096, 16384} x beta in "
                        "{0.30, 0.40, 0.4406868, 0.50, 0.60}, periodic, hot start seed 1, E/M every sweep",
            "chains_per_gpu": len(chains),
            "step": "one sweep of every chain (2 half-sweep launches + E/M reduction fused)",
            "l2": "inputs larger than L2: 170 MiB of spins per GPU (L2 = 129 MB)",
            "parallelism": f"replicas{world}",
            "threads_per_block": args.threads,
        },
        "roofline": {
            "bound": "alu",
            "achieved": achieved,
            "peak": peak["mul32_per_s"],
            "unit": "int32-mul/s",
            "frac": achieved / peak["mul32_per_s"],
            "traffic": MSC_TRAFFIC["bytes_per_launch"] if traffic_ok else None,
            "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, captured "
                               f"{MSC_TRAFFIC['captured']} from kernel sources sha256 {sha[:16]} (unchanged)")
                              if traffic_ok else f"null: the kernel sources (sha256 {sha[:16]}) differ from the "
                                                 "ones the stored ncu figure was captured from",
            "kernel": "k_half_sweep<C, MSC32> (Ising half-sweep)",
            "kernel_ms_per_launch": half_ms,
            "kernel_share_of_step": kernel_ms / ms if ms > 0 else None,
            "algorithmic": "10 int32 multiplies per attempted flip (1/4 Philox4x32-10 block)",
            "peak_source": "measured in this run: the library's pure-Philox kernel (mc_philox_rate), "
                           f"{peak['blocks']} CTAs x {peak['threads']} threads x {peak['blocks_per_thread']} blocks, "
                           "40 int32 multiplies per block, best of 5 (the measured peaks file has no integer figure)",
            "sm_count": sms,
            "derived_peak": derived_peak,
            "derived_peak_source": f"{sms} SMs (queried) x {MUL32_PER_SM_CLK} int32 multiplies/clk x {clk} MHz "
                                   "(median SM clock sampled during the timed region)",
        },
        "e2e": e2e,
        "gpu_launches": launches + K,  # 2 half-sweeps + 1 state-advance kernel per step
        "clocks": clock_info,
        "components": {"ising_64x64_int8": small, "su2": su2, "batched": batched, "ess_beta_c": ess_cmp,
                       "paper_protocol": paper},
        "device": dev_props.name,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_e2e(mc, torch, rank, K, world, n_ctx=3):
    """Per step: upload every chain's configuration from page-locked host memory,
    one sweep with measurement, read the step's records back to the host -- all
    through the C ABI.  Measured three ways:
      sequential -- one context, canonical bit rows; the layout-conversion
        kernel reads the page-locked rows in place (mc_set_config with a host
        pointer), and each step's upload waits for the previous sweep;
      canonical pipelined -- n_ctx contexts on their own streams take turns;
        a step's bit rows go host -> device by the copy engine into the
        context's device buffer and are converted there (mc_set_config with a
        device pointer), so that the next steps' uploads run while a step sweeps;
      native pipelined (the reported value) -- the same rotation, each chain's
        configuration held on the host in the storage format (MC_FMT_NATIVE,
        the same bytes as the bit rows) and copied by the copy engine straight
        into the lattice (mc_set_config with a host pointer): no conversion
        kernel competes with the sweeps for SMs or HBM.
    Every step carries its own upload and read-back in all three; a context's
    records are read back n_ctx - 1 steps after its sweep was enqueued."""
    chains = ising_chains(rank)
    streams = [torch.cuda.Stream() for _ in range(n_ctx)]
    batches = []
    for st in streams:
        b = mc.Batch(chains, layout=mc.MC_LAYOUT_MSC32, series_capacity=4, stream=st)
        b.set_mode(mc.MC_MODE_GRID, 256)
        batches.append(b)
    host, native, dev = [], [], [[] for _ in range(n_ctx)]
    h2d = h2d_native = 0
    for k, c in enumerate(chains):
        t = torch.from_numpy(batches[0].get_config(k, mc.MC_FMT_BITS).view(np.int32)).pin_memory()
        host.append(t)
        h2d += t.numel() * 4
        t = torch.from_numpy(batches[0].get_config(k, mc.MC_FMT_NATIVE).view(np.int32)).pin_memory()
        native.append(t)
        h2d_native += t.numel() * 4
        for i in range(n_ctx):
            dev[i].append(torch.empty_like(host[k], device="cuda"))
    assert h2d_native == h2d
    d2h = len(chains) * 48

    def enqueue_zero_copy(i):
        b = batches[i]
        for k in range(len(chains)):
            b.set_config_host_async(k, host[k], mc.MC_FMT_BITS)
        b.sweep(1, 1)

    def enqueue_dma(i):
        # all copies first: a conversion kernel between two copies would hold
        # the next copy back until it gets SMs, which another stream's sweep
        # occupies
        b = batches[i]
        with torch.cuda.stream(streams[i]):
            for k in range(len(chains)):
                dev[i][k].copy_(host[k], non_blocking=True)
            for k in range(len(chains)):
                b.set_config_device(k, dev[i][k], mc.MC_FMT_BITS)
        b.sweep(1, 1)

    def enqueue_native(i):
        b = batches[i]
        for k in range(len(chains)):
            b.set_config_host_async(k, native[k], mc.MC_FMT_NATIVE)
        b.sweep(1, 1)

    def timed(n, enqueue):
        for _ in range(2):
            for i in range(n):
                enqueue(i)
                batches[i].read_series()
        barrier(world)
        torch.cuda.synchronize()
        t = time.perf_counter()
        pending = []
        for step in range(K):
            i = step % n
            enqueue(i)
            pending.append(i)
            if len(pending) >= n:
                batches[pending.pop(0)].read_series()
        while pending:
            batches[pending.pop(0)].read_series()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        barrier(world)
        return max_over_ranks(dt, world)

    dt_seq = timed(1, enqueue_zero_copy)
    dt_dma = timed(n_ctx, enqueue_dma)
    dt = timed(n_ctx, enqueue_native)
    for b in batches:
        b.close()
    rate = flips_per_step() * K * world
    return {"value": rate / dt, "unit": "spin-flips/s", "h2d_bytes_per_step": h2d_native,
            "d2h_bytes_per_step": d2h, "steps": K,
            "pipeline": f"{n_ctx} contexts on {n_ctx} streams take turns; copy-engine upload of the storage-format "
                        "configurations straight into the next contexts' lattices overlaps the running sweep",
            "canonical_pipelined_value": rate / dt_dma, "sequential_value": rate / dt_seq}


def run_ising_64(mc, torch, rank, world, sweeps=1000) -> dict:
    """The parity workload: one 64 x 64 int8 chain at beta_c, hot start, E/M
    every sweep, 1000 sweeps per call (the resident kernel: the lattice in
    shared memory, all sweeps in one launch).  4096 sites: latency-bound, no
    roofline claimed."""
    b = mc.Batch([mc.ising(64, 0.4406868, seed=1, chain_id=cid(rank, 0))], series_capacity=sweeps)
    b.set_mode(mc.MC_MODE_AUTO)
    b.sweep(sweeps, 1)
    b.read_series()
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    b.sweep(sweeps, 1)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    b.read_series()
    b.close()
    return {"metric": "Ising spin-flips/s", "workload": "64x64 int8, beta_c, hot start, E/M every sweep",
            "sweeps": sweeps, "us_per_sweep": 1e3 * ms / sweeps, "value": 64 * 64 * sweeps * world / (ms / 1e3),
            "unit": "spin-flips/s", "bound": "latency (one CTA, 4096 sites)"}


def run_su2(mc, torch, rank, K, world, issue_peak):
    """SU(2) heat-bath on 4 x 32^4 with the plaquette measured every sweep.
    The timed loop replays CUDA graphs (sweep(1, 1) per step, inputs > L2); the
    phase-kernel time comes from a separate profiled pass (CUDA events around
    each launch, no graphs); then the same chains with one overrelaxation sweep
    per heat-bath sweep."""
    chains = [mc.su2(SU2_L, b, seed=1, chain_id=cid(rank, i), hot=True) for i, b in enumerate(SU2_BETAS)]
    batch = mc.Batch(chains, series_capacity=K + 64)
    batch.sweep(3, 1)
    batch.sweep(1, 1)  # graph capture
    batch.read_series()
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(K):
        batch.sweep(1, 1)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(t0.elapsed_time(t1), world)
    P = batch.read_series()["P"][:, -1].tolist()
    # phase-kernel time
    Kp = max(2, min(K, 8))
    batch.profile(True)
    batch.profile_read()
    batch.sweep(Kp, 1)
    torch.cuda.synchronize()
    launches, kernel_ms = batch.profile_read()
    batch.profile(False)
    batch.read_series()
    # heat-bath with overrelaxation (Sec. 2.4): one overrelaxation sweep per heat-bath sweep
    batch.set_overrelax(1)
    Kor = max(2, K // 4)
    batch.sweep(2, 1)
    batch.read_series()
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(Kor):
        batch.sweep(1, 1)
    t1.record(stream)
    torch.cuda.synchronize()
    ms_or = t0.elapsed_time(t1) / Kor
    batch.read_series()
    batch.close()
    # the small lattice of the workload: 8^4 at the same four beta, plaquette every sweep, in 1000-sweep
    # calls; 2048 links per phase and chain, so launch- and latency-bound: the resident mode (one
    # cluster per chain, one launch per call) against the grid mode (10 graph-replayed launches per sweep)
    ms_small = {}
    for mode, name in ((mc.MC_MODE_RESIDENT, "resident"), (mc.MC_MODE_GRID, "grid")):
        small = mc.Batch([mc.su2(8, b, seed=1, chain_id=cid(rank, i), hot=True) for i, b in enumerate(SU2_BETAS)],
                         series_capacity=1024)
        small.set_mode(mode)
        small.sweep(1000, 1)
        small.read_series()
        torch.cuda.synchronize()
        t0.record(stream)
        small.sweep(1000, 1)
        t1.record(stream)
        torch.cuda.synchronize()
        ms_small[name] = t0.elapsed_time(t1) / 1000
        small.read_series()
        small.close()
    updates = len(chains) * 4 * SU2_L ** 4 * K * world
    phase_ms = kernel_ms / max(launches, 1)
    per_launch_updates = len(chains) * 4 * SU2_L ** 4 * Kp / max(launches, 1)
    hbm = 6777.3e9
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] * 1e9
    except (OSError, KeyError, ValueError):
        pass
    achieved_bw = SU2_BYTES_PER_UPDATE * per_launch_updates / (phase_ms / 1e3)
    alu = SU2_INSTR_PER_UPDATE * per_launch_updates / (phase_ms / 1e3)
    return {"metric": "SU(2) link-updates/s", "value": updates / (ms / 1e3), "unit": "link-updates/s",
            "workload": f"4D SU(2) {SU2_L}^4, beta in {SU2_BETAS}, hot start, heat-bath (KP+Creutz), plaquette "
                        "every sweep", "steps": K, "ms_per_sweep": ms / K, "phase_kernel_ms": phase_ms,
            "last_plaquette": P,
            "lattice_8x4": {"ms_per_sweep": ms_small["resident"], "mode": "resident (the automatic choice)",
                            "link_updates_per_s": len(SU2_BETAS) * 4 * 8 ** 4 * world / (ms_small["resident"] / 1e3),
                            "grid_ms_per_sweep": ms_small["grid"],
                            "bound": "latency: 2048 links per phase and chain; resident: one cluster of 16 CTAs per "
                                     "chain, 8 cluster barriers per sweep"},
            "with_overrelaxation": {"n_or": 1, "ms_per_compound_sweep": ms_or,
                                    "overrelax_link_updates_per_s": len(chains) * 4 * SU2_L ** 4 / ((ms_or - ms / K) / 1e3)
                                    if ms_or > ms / K else None},
            "roofline_hbm": {"achieved": achieved_bw, "peak": hbm, "unit": "B/s", "frac": achieved_bw / hbm,
                             "bytes_per_update": SU2_BYTES_PER_UPDATE},
            "roofline_alu": {"bound": "alu", "achieved": alu, "peak": issue_peak, "unit": "thread-instr/s",
                             "frac": alu / issue_peak, "instr_per_update": SU2_INSTR_PER_UPDATE,
                             "peak_source": "SMs (queried) x 4 schedulers x 32 lanes x median sampled SM clock",
                             "note": "the slower bound: phase kernel at its algorithmic issue count"}}


def run_batched(mc, torch, rank, K, world, sweeps_per_call=10):
    """256 Ising + 64 SU(2) chains of uneven sizes in one persistent launch per
    call (autotuned launch shape); value = site/link updates per second."""
    from paper_0903_3053_gb300 import autotune, workloads
    spec = workloads.batched_chains(seed=0)
    def chain(d):
        f = mc.ising if d["kind"] == "ising" else mc.su2
        return f(d["L"], d["beta"], d["seed"], cid(rank, d["chain_id"]))

    i8 = [chain(d) for d in spec if d["kind"] == "ising" and d["L"] < 64]
    msc = [chain(d) for d in spec if d["kind"] == "ising" and d["L"] >= 64]
    s2 = [chain(d) for d in spec if d["kind"] == "su2"]
    cap = sweeps_per_call * (K + 2) + 64
    bs = [mc.Batch(i8, layout=mc.MC_LAYOUT_INT8, series_capacity=cap),
          mc.Batch(msc, layout=mc.MC_LAYOUT_MSC32, series_capacity=cap), mc.Batch(s2, series_capacity=cap)]
    g = mc.Group(bs)
    choice = autotune.tune_group(g, n_sweeps=sweeps_per_call, reps=2)
    for b in bs:
        b.read_series()
    g.sweep(sweeps_per_call, 1)
    stream = torch.cuda.current_stream()
    barrier(world)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(K):
        g.sweep(sweeps_per_call, 1)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(t0.elapsed_time(t1), world)
    nc, nr = g.schedule()
    for b in bs:
        b.read_series()
    g.close()
    per_sweep = sum(c.L[0] * c.L[1] for c in i8 + msc) + sum(4 * int(np.prod(c.L)) for c in s2)
    sweeps = K * sweeps_per_call
    return {"metric": "batched updates/s", "value": per_sweep * sweeps * world / (ms / 1e3),
            "unit": "site+link updates/s",
            "workload": "256 Ising chains L in {32..1024}, beta ~ U[0.35, 0.55] + 64 SU(2) chains L^4, "
                        "L in {4, 6, 8, 12, 16}, beta ~ U[1.8, 2.6] (numpy default_rng(0)); E/M and plaquette "
                        "every sweep", "launches_per_call": 1 + len(bs), "sweeps_per_call": sweeps_per_call,
            "ms_per_sweep": ms / sweeps, "clusters": nc, "rounds": nr,
            "autotuned": {k: choice[k] for k in ("cluster", "threads", "split", "cached")}}


# The paper's own workloads (Sec. 2.3 and Table 1), for a like-for-like table:
# its times are for an ATI HD 4850 and are context only.
PAPER_TABLE1_S = {(4, 8): 5.2, (4, 16): 17.9, (4, 24): 52.8, (4, 32): 120.6, (8, 16): 32.7, (8, 24): 102.3,
                  (8, 32): 397.4}
PAPER_ISING_S = {"sweep": 630.0, "sweep+measure": 730.0}  # 10^6 sweeps of 1024 x 512


def run_paper_protocol(mc, torch, ising_sweeps=20000) -> dict:
    """Ising 1024 x 512, one chain, sweeps with and without the E/M measurement
    (the paper's 10^6 sweeps projected from `ising_sweeps`); SU(2) L_t x L_s^3
    lattices of Table 1, one chain each at beta = 2.3, the paper's protocol of
    1000 thermalisation sweeps then 1000 measurements 5 sweeps apart, run in
    full, through the per-phase launches (grid) and the persistent launch
    (group); the faster is reported."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    out = {"ising_1024x512": {}, "su2_table1": []}
    for name, layout in (("msc32", mc.MC_LAYOUT_MSC32), ("int8", mc.MC_LAYOUT_INT8)):
        row = {}
        # per-colour launches from a CUDA graph; the persistent launch (one cluster for
        # one chain) measured 3x (MSC) to 37x (int8) slower on this lattice
        for mode in ("grid",):
            b = mc.Batch([mc.ising((1024, 512), 0.4406868, seed=1)], layout=layout, series_capacity=ising_sweeps + 16)
            g = mc.Group([b]) if mode == "group" else None
            run = (lambda n, every: g.sweep(n, every)) if g else (lambda n, every: b.sweep(n, every))
            run(200, 0)
            run(ising_sweeps, 0)
            t_sweep = timed(lambda: run(ising_sweeps, 0))
            run(ising_sweeps, 1)
            b.read_series()
            t_meas = timed(lambda: run(ising_sweeps, 1))
            b.read_series()
            if g:
                g.close()
            b.close()
            row[mode] = {"us_per_sweep": t_sweep * 1e6 / ising_sweeps, "us_per_sweep_measured": t_meas * 1e6 / ising_sweeps}
        best = min(row.values(), key=lambda r: r["us_per_sweep_measured"])
        proj = {"sweep": best["us_per_sweep"], "sweep+measure": best["us_per_sweep_measured"]}  # s per 10^6 sweeps
        row["projected_s_per_1e6_sweeps"] = proj
        row["speedup_vs_paper_gpu"] = {k: PAPER_ISING_S[k] / proj[k] for k in proj}
        out["ising_1024x512"][name] = row
    for (lt, ls), paper_s in PAPER_TABLE1_S.items():
        L = (lt, ls, ls, ls)
        row = {"lattice": f"{lt}x{ls}^3", "paper_gpu_s": paper_s}
        # the persistent launches (group: one cluster for the chain; resident: the SU(2) resident mode)
        # pay off only for the smallest lattices
        modes = ("grid",) + (("group",) if ls <= 16 and lt == 4 else ()) + (("resident",) if ls <= 8 else ())
        for mode in modes:
            b = mc.Batch([mc.su2(L, 2.3, seed=3, chain_id=0, hot=True)], series_capacity=1100)
            if mode == "group":
                g = mc.Group([b])
                run = lambda n, every: g.sweep(n, every)
            else:
                b.set_mode(mc.MC_MODE_GRID if mode == "grid" else mc.MC_MODE_RESIDENT)
                run = lambda n, every: b.sweep(n, every)
            run(5, 5)  # graph capture
            b.read_series()

            def protocol():
                run(1000, 0)
                run(5000, 5)

            t = timed(protocol)
            P = b.read_series()["P"][0]
            if mode == "group":
                g.close()
            b.close()
            row[mode + "_s"] = t
            row[mode + "_mean_P"] = float(P.mean())
        row["gb300_s"] = min(row.get("grid_s", 1e30), row.get("group_s", 1e30), row.get("resident_s", 1e30))
        row["speedup_vs_paper_gpu"] = paper_s / row["gb300_s"]
        out["su2_table1"].append(row)
    return out


def run_ess(args) -> dict:
    """Effective independent |M| samples per second at beta_c: plain
    checkerboard Metropolis (4096 chains in 32-spin words where L % 64 == 0, its fastest form)
    versus Metropolis interleaved 1:10 with the learned proposal (4096 int8
    chains, one proposal each per round; the network trained on ~2 x 10^5
    configurations of the plain chains, training time reported separately).
    L = 64 is the headline; L = 32 is the other lattice of the workload."""
    from paper_0903_3053_gb300 import ess, mc
    beta = 0.4406868
    out = {"metric": "eff. independent |M| samples/s at beta_c, L=64", "unit": "samples/s"}
    for L in (64, 32):
        layout = mc.MC_LAYOUT_MSC32 if L % 64 == 0 else mc.MC_LAYOUT_INT8
        plain = ess.plain_rate(L, beta, chains=4096, therm=5000, sweeps=args.ess_sweeps, every=4, layout=layout)
        # tau from a run of >= 1000 tau (fewer chains: the series must fit the ring buffer)
        long = ess.plain_tau_long(L, beta, chains=256, therm=5000, sweeps=args.ess_long_sweeps, every=8,
                                  layout=layout)
        plain["tau_long"] = long
        plain["ess_per_s"] = plain["chain_sweeps_per_s"] / (2.0 * long["tau_absM_sweeps"])
        plain["ess_tau_source"] = "tau_long"
        learned = ess.learned_rate(L, beta, chains=4096, therm=5000, data_snapshots=48, data_spacing=200,
                                   train_steps=args.ess_train_steps, train_batch=512,
                                   rounds=args.ess_rounds if L == 64 else 2 * args.ess_rounds, local_sweeps=10)
        res = {"plain": plain, "learned": learned, "learned_over_plain": learned["ess_per_s"] / plain["ess_per_s"]}
        if L == 64:
            out.update(res)
        else:
            out["L32"] = res
    return out


# ----------------------------------------------------------------------------- CPU oracle
def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_ising_rate(steps: int, warmup: int, threads: int, seconds: float | None = None):
    """The oracle as it stands on `threads` host cores: one independent 1024^2
    chain at beta_c per thread (chain id = thread index), E/M recorded every
    sweep.  The oracle is plain C without global state called through ctypes,
    which releases the GIL, so the threads run in parallel.  With `seconds`,
    `steps` is replaced by as many sweeps as fit in about that time.  Returns
    (spin-flips/s over all threads, timed seconds, steps)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.build()
    beta = 0.4406868
    lat = [oracle.ising_init(1024, seed=1, chain=i, hot=True) for i in range(threads)]

    def run(i, first, n):
        for k in range(n):
            oracle.ising_run(lat[i], beta, 1, i, first + k, 1)

    with ThreadPoolExecutor(threads) as ex:
        t = time.perf_counter()
        list(ex.map(lambda i: run(i, 0, max(1, warmup)), range(threads)))
        per_sweep = (time.perf_counter() - t) / max(1, warmup)
        if seconds is not None:
            steps = max(1, int(seconds / max(per_sweep, 1e-6)))
        t = time.perf_counter()
        list(ex.map(lambda i: run(i, max(1, warmup), steps), range(threads)))
        dt = time.perf_counter() - t
    return threads * 1024 * 1024 * steps / dt, dt, steps


def cpu_baseline(seconds: float) -> dict:
    """The oracle on all host cores, on a bounded sample of the workload."""
    threads = host_threads()
    value, dt, n = oracle_ising_rate(0, 2, threads, seconds)
    return {"value": value, "unit": "spin-flips/s", "cores": threads, "kind": "oracle",
            "sample": f"{threads} independent 1024x1024 chains at beta=0.4406868 (one per core), {n} sweeps each "
                      f"(int8 oracle, E/M every sweep), {dt:.1f} s"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # one step = one oracle sweep of a 1024^2 chain on every host core (a bounded sample of the workload)
    threads = host_threads()
    value, dt, _ = oracle_ising_rate(args.steps, args.warmup, threads)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "spin-flips/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i8", "data": "synthetic",
        "config": {"workload": "2D Ising 1024x1024 samples of the multi-spin-coded batch, beta=0.4406868, hot start, "
                               "E/M every sweep (CPU oracle, one chain per host core)"},
        "cpu_baseline": {"value": value, "unit": "spin-flips/s", "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} sweeps of {threads} independent 1024x1024 chains"},
        "e2e": {"value": value, "unit": "spin-flips/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--su2-steps", type=int, default=40)
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--ess-sweeps", type=int, default=20000)
    ap.add_argument("--ess-long-sweeps", type=int, default=200000)
    ap.add_argument("--ess-rounds", type=int, default=200)
    ap.add_argument("--ess-train-steps", type=int, default=1500)
    ap.add_argument("--no-ess", action="store_true")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper-protocol component")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
