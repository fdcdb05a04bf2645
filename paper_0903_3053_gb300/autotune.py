"""Autotuner for launch shapes.

Every launch shape gives bit-identical results (the Philox counters depend only
on seed, sweep, site and chain), so shapes can be chosen for speed alone.  The
tuner times candidate shapes with CUDA events and caches the winner in a JSON
file keyed by GPU name and workload signature (override the path with
MC_AUTOTUNE_CACHE).
"""
from __future__ import annotations

import json
import os
import time

from . import mc

CACHE = os.environ.get("MC_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "mc_gb300",
                                                          "autotune.json"))


def _load_cache() -> dict:
    try:
        return json.load(open(CACHE))
    except (OSError, ValueError):
        return {}


def _store_cache(d: dict):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}"
        json.dump(d, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _signature(batches) -> str:
    parts = []
    for b in batches:
        for c in b.chains:
            parts.append(f"{c.kind}:{b.layout}:{'x'.join(str(v) for v in c.L)}")
    return ",".join(sorted(parts))


def _time(fn, reps: int) -> float:
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()  # warm-up (graph capture)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0.record(s)
        fn()
        e1.record(s)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def group_candidates():
    for C in (1, 2, 4, 8, 16):
        for threads in (128, 256):
            for split in (-1.0, 0.0):
                if C == 1 and split == 0.0:
                    continue
                yield C, threads, split


def tune_group(group: "mc.Group", n_sweeps: int = 4, reps: int = 3, use_cache: bool = True, verbose=False) -> dict:
    """Pick (cluster size, threads, split cost) for a group; returns the choice
    with its time per sweep.  The group is left configured with it."""
    key = f"group|{_gpu_name()}|{_signature(group.batches)}|{n_sweeps}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        c = cache[key]
        group.configure(c["cluster"], c["threads"], c["split"])
        return dict(c, cached=True)
    results = []
    for C, threads, split in group_candidates():
        group.configure(C, threads, split)
        try:
            ms = _time(lambda: group.sweep(n_sweeps), reps) / n_sweeps
        except mc.MCError as err:  # e.g. a cluster size the device cannot co-schedule
            if verbose:
                print(f"  cluster {C} threads {threads} split {split}: unavailable ({err})", flush=True)
            continue
        results.append((ms, C, threads, split))
        if verbose:
            print(f"  cluster {C} threads {threads} split {split}: {ms:.3f} ms/sweep", flush=True)
    ms, C, threads, split = min(results)
    group.configure(C, threads, split)
    choice = {"cluster": C, "threads": threads, "split": split, "ms_per_sweep": ms,
              "tried": [list(r) for r in results], "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if use_cache:
        cache[key] = choice
        _store_cache(cache)
    return dict(choice, cached=False)


def tune_batch(batch: "mc.Batch", n_sweeps: int = 4, reps: int = 3, use_cache: bool = True) -> dict:
    """Pick execution mode and block size for one Batch."""
    key = f"batch|{_gpu_name()}|{_signature([batch])}|{n_sweeps}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        c = cache[key]
        batch.set_mode(c["mode"], c["threads"])
        return dict(c, cached=True)
    cands = [(mc.MC_MODE_GRID, t) for t in ((64, 128, 256, 512) if batch.kind == mc.MC_KIND_ISING
                                             else (64, 128, 256))]
    if batch.kind == mc.MC_KIND_ISING:
        cands += [(mc.MC_MODE_RESIDENT, t) for t in (256, 512, 1024)]
    results = []
    for mode, t in cands:
        try:
            batch.set_mode(mode, t)
        except mc.MCError:
            continue  # e.g. lattices too large for the resident mode
        ms = _time(lambda: batch.sweep(n_sweeps), reps) / n_sweeps
        results.append((ms, mode, t))
    ms, mode, t = min(results)
    batch.set_mode(mode, t)
    choice = {"mode": mode, "threads": t, "ms_per_sweep": ms, "tried": [list(r) for r in results],
              "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if use_cache:
        cache[key] = choice
        _store_cache(cache)
    return dict(choice, cached=False)
