"""Writes su2_plaquette_8x4_beta2.3.txt: the average plaquette <P> (Eqs.
(2)-(3)) of 4D SU(2) on an 8^4 periodic lattice at beta = 2.3, from the FP64
CPU oracle alone (oracle/mc_oracle.c: heat-bath of Eqs. (5)-(7), phase order
of Sec. 2.4), hot start.  Eight independent chains (seed 33, chain ids 0..7),
each 500 thermalisation sweeps then 5000 measured sweeps, one process per
chain; the 40,000 measurements are cut into 80 bins of 500 consecutive
sweeps of one chain (far longer than the plaquette's autocorrelation), and the
file holds the mean and the standard error of the bin means.

    python tests/golden/make_su2_plaquette_8x4.py   # ~1 minute on 8 cores
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
L = (8, 8, 8, 8)
BETA = 2.3
SEED = 33
CHAINS = 8
THERM = 500
MEAS = 5000
BIN = 500
OUT = os.path.join(HERE, "su2_plaquette_8x4_beta2.3.txt")


def run_chain(chain: int) -> np.ndarray:
    sys.path.insert(0, ROOT)
    import oracle
    q = oracle.su2_init(L, SEED, chain, True)
    P = np.empty(MEAS)
    for k in range(THERM + MEAS):
        oracle.su2_sweep(q, L, BETA, SEED, chain, k)
        if k >= THERM:
            P[k - THERM] = oracle.su2_plaquette(q, L)[0]
    return P


def main():
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(min(CHAINS, os.cpu_count() or 1)) as pool:
        series = pool.map(run_chain, range(CHAINS))
    bins = np.concatenate([s.reshape(-1, BIN).mean(axis=1) for s in series])
    mean = float(bins.mean())
    err = float(bins.std(ddof=1) / np.sqrt(len(bins)))
    with open(OUT, "w") as f:
        f.write(f"# <P> of 4D SU(2), 8^4 periodic, beta = {BETA}, hot start, FP64 CPU oracle\n")
        f.write("# written by: python tests/golden/make_su2_plaquette_8x4.py (calls oracle/ only)\n")
        f.write(f"# {CHAINS} chains (seed {SEED}, chain ids 0..{CHAINS - 1}), {THERM} thermalisation + {MEAS} "
                f"measured sweeps each; standard error from {len(bins)} bins of {BIN} sweeps\n")
        f.write(f"mean {mean:.9f}\nerr {err:.9f}\nsweeps {CHAINS * MEAS}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
