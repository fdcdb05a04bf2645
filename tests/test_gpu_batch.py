"""Many uneven chains in one persistent launch (mc_group_*): results must be
bit-identical to each context's own sweeps (and so to the oracle) for every
cluster size, block size and split policy the autotuner may pick."""
import numpy as np
import pytest

import oracle
import paper_0903_3053_gb300 as mc
from paper_0903_3053_gb300 import autotune, workloads

pytestmark = pytest.mark.gpu


def mixed_batches(cap=16):
    msc = [mc.ising(64, 0.40, seed=11, chain_id=0), mc.ising((128, 64), 0.44, seed=12, chain_id=1),
           mc.ising(256, 0.50, seed=13, chain_id=2), mc.ising((1024, 512), 0.44, seed=14, chain_id=3)]
    i8 = [mc.ising(32, 0.45, seed=21, chain_id=0), mc.ising((96, 64), 0.38, seed=22, chain_id=1),
          mc.ising((2, 6), 0.3, seed=23, chain_id=2)]
    s2 = [mc.su2((4, 4, 4, 4), 2.3, seed=31, chain_id=0), mc.su2((6, 6, 6, 6), 2.0, seed=32, chain_id=1),
          mc.su2((8, 8, 8, 8), 2.6, seed=33, chain_id=2), mc.su2((4, 6, 8, 4), 1.8, seed=34, chain_id=3)]
    return [mc.Batch(msc, layout=mc.MC_LAYOUT_MSC32, series_capacity=cap),
            mc.Batch(i8, layout=mc.MC_LAYOUT_INT8, series_capacity=cap),
            mc.Batch(s2, series_capacity=cap)]


def snapshot(batches):
    cfgs = [[b.get_config(k) for k in range(len(b.chains))] for b in batches]
    series = [b.read_series() for b in batches]
    return cfgs, series


def assert_same(a, b):
    for ca, cb in zip(a[0], b[0]):
        for x, y in zip(ca, cb):
            np.testing.assert_array_equal(x, y)
    for sa, sb in zip(a[1], b[1]):
        np.testing.assert_array_equal(sa, sb)


@pytest.fixture(scope="module")
def reference():
    bs = mixed_batches()
    for b in bs:
        b.set_mode(mc.MC_MODE_GRID, 256)
        b.sweep(4, 2)
        b.sweep(2, 2)
    return snapshot(bs)


@pytest.mark.parametrize("C,threads,split", [(1, 256, -1.0), (2, 128, -1.0), (4, 256, -1.0), (8, 256, 0.0),
                                             (4, 64, 1e300), (8, 128, -1.0), (16, 256, 0.0), (16, 128, -1.0)])
def test_group_matches_context_sweeps(reference, C, threads, split):
    bs = mixed_batches()
    g = mc.Group(bs)
    g.configure(C, threads, split)
    g.sweep(4, 2)
    g.sweep(2, 2)  # graph replay with device-side counters
    nc, nr = g.schedule()
    assert nc >= 1 and nr >= 1
    assert_same(snapshot(bs), reference)
    g.close()


def test_group_chains_against_oracle():
    chains = [mc.ising(32, 0.4406868, seed=5, chain_id=9), mc.ising((64, 32), 0.3, seed=6, chain_id=1)]
    msc = [mc.ising(128, 0.5, seed=7, chain_id=4), mc.ising((128, 64), 3.0, seed=8, chain_id=2),
           mc.ising(64, 6.0, seed=9, chain_id=3)]  # T4 = 0; T2 = T4 = 0
    b1 = mc.Batch(chains, layout=mc.MC_LAYOUT_INT8, series_capacity=8)
    b2 = mc.Batch(msc, layout=mc.MC_LAYOUT_MSC32, series_capacity=8)
    g = mc.Group([b1, b2])
    g.configure(2, 128, -1.0)
    g.sweep(10, 5)
    for b, cs in ((b1, chains), (b2, msc)):
        rec = b.read_series()
        for k, c in enumerate(cs):
            s = oracle.ising_init(c.L, c.seed, c.chain_id, True)
            E, M = oracle.ising_run(s, c.beta, c.seed, c.chain_id, 0, 10)
            np.testing.assert_array_equal(b.get_config(k), s)
            np.testing.assert_array_equal(rec["E"][k], E[4::5])
            np.testing.assert_array_equal(rec["M"][k], M[4::5])


def test_batched_workload_autotuned():
    """The 256 + 64 chain workload in one persistent launch, autotuned; a sample
    of chains checked against single-chain contexts run on their own."""
    spec = workloads.batched_chains(seed=0)
    i8 = [mc.ising(d["L"], d["beta"], d["seed"], d["chain_id"]) for d in spec if d["kind"] == "ising" and d["L"] < 64]
    msc = [mc.ising(d["L"], d["beta"], d["seed"], d["chain_id"]) for d in spec if d["kind"] == "ising" and d["L"] >= 64]
    s2 = [mc.su2(d["L"], d["beta"], d["seed"], d["chain_id"]) for d in spec if d["kind"] == "su2"]
    bs = [mc.Batch(i8, layout=mc.MC_LAYOUT_INT8, series_capacity=64),
          mc.Batch(msc, layout=mc.MC_LAYOUT_MSC32, series_capacity=64), mc.Batch(s2, series_capacity=64)]
    g = mc.Group(bs)
    choice = autotune.tune_group(g, n_sweeps=2, reps=2, use_cache=False)
    assert choice["ms_per_sweep"] > 0
    for b in bs:  # tuning advanced the chains; start the check from here
        b.read_series()
    g.sweep(3, 1)
    rng = np.random.default_rng(1)
    for b in bs:
        rec = b.read_series()
        assert rec.shape == (len(b.chains), 3)
        for k in rng.choice(len(b.chains), size=3, replace=False):
            c = b.chains[k]
            one = mc.Batch([c], layout=b.layout, series_capacity=4)  # same seed and chain id: same start
            one.sweep(b.sweeps_done, 0)
            np.testing.assert_array_equal(one.get_config(0), b.get_config(k))
            one.close()
    g.close()


def test_group_with_overrelaxation_matches_contexts():
    """SU(2) members with overrelaxation: the persistent launch gives the same
    links and plaquettes as the context's own compound sweeps, also after the
    count changes between calls."""
    def make():
        return mc.Batch([mc.su2((4, 4, 4, 4), 2.3, seed=41, chain_id=0), mc.su2((6, 4, 4, 8), 2.0, seed=42, chain_id=1)],
                        series_capacity=16)
    ref = make()
    ref.set_mode(mc.MC_MODE_GRID, 256)
    ref.set_overrelax(2)
    ref.sweep(3, 1)
    ref.set_overrelax(1)
    ref.sweep(2, 1)
    want = snapshot([ref])
    b = make()
    g = mc.Group([b])
    g.configure(4, 256, -1.0)
    b.set_overrelax(2)
    g.sweep(3, 1)
    b.set_overrelax(1)
    g.sweep(2, 1)
    assert_same(snapshot([b]), want)
    g.close()
