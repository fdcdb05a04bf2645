"""Seeded synthetic workloads (no method arithmetic: only which chains to run).

The batched-chain workload: 256 Ising chains with L drawn uniformly from
{32, 64, 128, 256, 512, 1024} and beta uniform in [0.35, 0.55], plus 64 SU(2)
chains with L^4, L drawn from {4, 6, 8, 12, 16}, and beta uniform in
[1.8, 2.6]; drawn with numpy default_rng(seed); chain seed 1000 + index, hot
start.  The plain lists of the other benchmark configurations live here too.
"""
from __future__ import annotations

import numpy as np

ISING_BETAS = [0.30, 0.40, 0.4406868, 0.50, 0.60]
ISING_MSC_SIZES = [1024, 4096, 16384]
SU2_BETAS = [1.5, 2.0, 2.3, 2.6]
BETA_C = 0.4406868


def batched_chains(seed: int = 0, n_ising: int = 256, n_su2: int = 64):
    """List of dicts {kind, L, beta, seed, chain_id} for the batched workload."""
    rng = np.random.default_rng(seed)
    out = []
    Ls = rng.choice([32, 64, 128, 256, 512, 1024], size=n_ising)
    bs = rng.uniform(0.35, 0.55, size=n_ising)
    for i in range(n_ising):
        out.append({"kind": "ising", "L": int(Ls[i]), "beta": float(bs[i]), "seed": 1000 + i, "chain_id": i})
    Ls = rng.choice([4, 6, 8, 12, 16], size=n_su2)
    bs = rng.uniform(1.8, 2.6, size=n_su2)
    for j in range(n_su2):
        i = n_ising + j
        out.append({"kind": "su2", "L": int(Ls[j]), "beta": float(bs[j]), "seed": 1000 + i, "chain_id": i})
    return out
