"""GPU parity of the SU(2) heat-bath (Eqs. (2)-(7), Sec. 2.4) through the C ABI.

FP32 quaternion links on the GPU against the FP64 2x2-matrix oracle: every link
within 1e-5 after a sweep; an accept decision that FP32 and FP64 take
differently is allowed only when it lies within 1e-6 of its threshold, and such
events are counted and reported."""
import numpy as np
import pytest

import oracle
import paper_0903_3053_gb300 as mc
from conftest import binned_mean_err

pytestmark = pytest.mark.gpu
TOL = 1e-5
EPS = 1e-6
# A decision FP32 and FP64 take differently needs its acceptance margin within
# the FP32 error of the test (a few 1e-7) of zero.  With ~1.2 tries per link and
# a margin density of order one near zero, the expected count is ~1e-7 per
# decision: ~0.002 per sweep of 8^4 x 4 links.  More than NEAR_MAX in one sweep
# would mean a systematic error in the FP32 heat-bath, not rounding.
NEAR_MAX = 3
NEAR_TALLY = {"near": 0, "decisions": 0}


def f32_roundtrip(q):
    return q.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 8, 2), (8, 8, 8, 8)])
def test_init_matches_oracle(L):
    for hot in (True, False):
        b = mc.Batch([mc.su2(L, 2.3, seed=17, chain_id=4, hot=hot)])
        g = b.get_config(0).astype(np.float64)
        o = oracle.su2_init(L, 17, 4, hot)
        assert np.abs(g - o).max() < 1e-6
        b.close()


@pytest.mark.parametrize("beta", [1.5, 2.0, 2.3, 2.6])
@pytest.mark.parametrize("L,hot", [((4, 4, 4, 4), True), ((6, 4, 8, 2), True), ((8, 8, 8, 8), True),
                                   ((8, 8, 8, 8), False)])
def test_one_sweep_per_link(beta, L, hot):
    """Same starting links on both sides (the oracle's start rounded to FP32),
    one sweep; the oracle follows the GPU's try indices only where its own FP64
    decision differs within EPS of the threshold."""
    q0 = f32_roundtrip(oracle.su2_init(L, 5, 0, hot))
    b = mc.Batch([mc.su2(L, beta, seed=5, chain_id=0, hot=hot)])
    b.set_config(0, q0.astype(np.float32))
    b.record_tries(True)
    b.sweep(1)
    g = b.get_config(0).astype(np.float64)
    tries = b.get_tries(0)
    q = q0.copy()
    _, fails, near, bad = oracle.su2_sweep(q, L, beta, 5, 0, 0, forced_tries=tries, eps=EPS)
    assert bad == 0, f"{bad} decisions differ by more than {EPS} from their thresholds"
    err = np.abs(g - q).max()
    assert err < TOL, err
    assert b.failed_updates() == fails
    assert near <= NEAR_MAX, f"{near} near-threshold decisions in one sweep"
    NEAR_TALLY["near"] += near
    NEAR_TALLY["decisions"] += tries.size
    print(f"near-threshold decisions: {near} of {tries.size} links "
          f"(all cases so far: {NEAR_TALLY['near']} of {NEAR_TALLY['decisions']})")
    b.close()


def test_multi_sweep_trajectory_follows_oracle():
    """Five sweeps re-synchronised per sweep: the per-link error stays at FP32
    round-off (no drift in the quaternion algebra)."""
    L = (4, 6, 4, 4)
    beta = 2.3
    q = f32_roundtrip(oracle.su2_init(L, 8, 2, True))
    b = mc.Batch([mc.su2(L, beta, seed=8, chain_id=2)])
    b.set_config(0, q.astype(np.float32))
    b.record_tries(True)
    for k in range(5):
        b.sweep(1)
        tries = b.get_tries(0)
        _, _, _, bad = oracle.su2_sweep(q, L, beta, 8, 2, k, forced_tries=tries, eps=EPS)
        assert bad == 0
        g = b.get_config(0).astype(np.float64)
        assert np.abs(g - q).max() < TOL
        q = g.copy()  # continue from the GPU's own FP32 state


def _random_links(L, seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(int(np.prod(L)), 4, 4))
    q /= np.linalg.norm(q, axis=2, keepdims=True)
    return f32_roundtrip(q)


# L1 = 2 makes the x1 pair of the measuring thread wrap onto itself; 8x6x4x6
# has 576 pairs, a ragged last block of the 128-pair measurement blocks.
@pytest.mark.parametrize("L", [(8, 6, 4, 6), (2, 2, 2, 2), (4, 2, 6, 2), (6, 10, 2, 4)])
def test_plaquette_on_fixed_configuration(L):
    q = _random_links(L, 1)
    b = mc.Batch([mc.su2(L, 2.0, seed=1)])
    b.set_config(0, q.astype(np.float32))
    m = b.measure(0)
    want = oracle.su2_plaquette(q, L)
    assert abs(m["P"] - want[0]) < 1e-6
    assert abs(m["Ps"] - want[1]) < 1e-6
    assert abs(m["Pt"] - want[2]) < 1e-6
    b.close()


def test_config_through_page_locked_host_memory():
    torch = pytest.importorskip("torch")
    L = (4, 6, 2, 4)
    q = _random_links(L, 3).astype(np.float32)
    b = mc.Batch([mc.su2(L, 2.0, seed=1)])
    b.set_config_host_async(0, torch.from_numpy(q.copy()).pin_memory())
    b.sync()
    np.testing.assert_array_equal(b.get_config(0), q)
    out = torch.zeros(q.shape, dtype=torch.float32).pin_memory()
    b.get_config_host(0, out)
    np.testing.assert_array_equal(out.numpy(), q)
    b.close()


def test_native_format_is_the_storage():
    """MC_FMT_NATIVE is float4 U[parity][mu][s >> 1] of the canonical links."""
    L = (4, 6, 2, 4)
    q = _random_links(L, 8).astype(np.float32)
    b = mc.Batch([mc.su2(L, 2.0, seed=1)])
    b.set_config(0, q)
    x0, x3, x2, x1 = np.meshgrid(*(np.arange(n) for n in (L[0], L[3], L[2], L[1])), indexing="ij")
    par = ((x0 + x1 + x2 + x3) & 1).reshape(-1)  # canonical order s = x1 + L1 (x2 + L2 (x3 + L3 x0))
    want = np.zeros((2, 4, q.shape[0] // 2, 4), dtype=np.float32)
    for p in range(2):
        idx = np.nonzero(par == p)[0]
        want[p][:, idx >> 1] = q[idx].transpose(1, 0, 2)
    got = b.get_config(0, mc.MC_FMT_NATIVE)
    np.testing.assert_array_equal(got, want)
    b.set_config(0, np.zeros_like(q))
    b.set_config(0, want, mc.MC_FMT_NATIVE)
    np.testing.assert_array_equal(b.get_config(0), q)
    b.close()


def test_plaquette_of_a_batch_of_shapes():
    """Several chains of different shapes in one measurement launch (per-chain
    block table of the pair kernel)."""
    shapes = [(4, 4, 4, 4), (2, 6, 2, 8), (6, 2, 4, 2), (8, 8, 6, 4)]
    qs = [_random_links(L, 10 + i) for i, L in enumerate(shapes)]
    b = mc.Batch([mc.su2(L, 2.0, seed=1, chain_id=i) for i, L in enumerate(shapes)], series_capacity=4)
    for i, q in enumerate(qs):
        b.set_config(i, q.astype(np.float32))
    for i, (L, q) in enumerate(zip(shapes, qs)):
        m = b.measure(i)
        want = oracle.su2_plaquette(q, L)
        assert abs(m["P"] - want[0]) < 1e-6 and abs(m["Ps"] - want[1]) < 1e-6 and abs(m["Pt"] - want[2]) < 1e-6
    b.close()


def test_unit_norm_and_series():
    L = (8, 8, 8, 8)
    b = mc.Batch([mc.su2(L, 2.3, seed=3)], series_capacity=64)
    b.sweep(40, 4)
    rec = b.read_series()
    assert rec.shape == (1, 10)
    np.testing.assert_array_equal(rec["sweep"][0], np.arange(3, 40, 4))
    g = b.get_config(0).astype(np.float64).reshape(-1, 4)
    assert np.abs(np.linalg.norm(g, axis=1) - 1).max() < 1e-6
    # the recorded P of the last sweep equals a fresh measurement of the state
    m = b.measure(0)
    assert abs(m["P"] - rec["P"][0, -1]) < 1e-12
    assert abs(m["P"] - (m["Ps"] + m["Pt"]) / 2) < 1e-12
    b.close()


def test_batch_of_uneven_chains():
    rng = np.random.default_rng(0)
    shapes = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 8), (4, 6, 8, 4)]
    chains = [mc.su2(s, float(rng.uniform(1.8, 2.6)), seed=1000 + k, chain_id=k, hot=bool(k % 2 == 0))
              for k, s in enumerate(shapes)]
    b = mc.Batch(chains)
    b.record_tries(True)
    starts = [b.get_config(k).astype(np.float64) for k in range(len(chains))]
    b.sweep(1)
    for k, c in enumerate(chains):
        q = starts[k].copy()
        tries = b.get_tries(k)
        _, _, _, bad = oracle.su2_sweep(q, c.L, c.beta, c.seed, c.chain_id, 0, forced_tries=tries, eps=EPS)
        assert bad == 0
        assert np.abs(b.get_config(k).astype(np.float64) - q).max() < TOL
    b.close()


@pytest.mark.parametrize("L", [(32, 32, 32, 32), (8, 32, 32, 32)])
def test_full_size_sampled_links(L):
    """Full-size lattice, benchmark launch configuration: 20k sampled links of
    one sweep recomputed in FP64 from the lattice each update saw."""
    beta = 2.3
    b = mc.Batch([mc.su2(L, beta, seed=1, chain_id=0)])
    b.sweep(2)
    pre = b.get_config(0).astype(np.float64)
    b.record_tries(True)
    b.sweep(1)
    post = b.get_config(0).astype(np.float64)
    tries = b.get_tries(0).reshape(-1)
    rng = np.random.default_rng(7)
    links = rng.choice(pre.shape[0] * 4, size=20_000, replace=False)
    want, _, near, bad = oracle.su2_check_links(pre, post, L, beta, 1, 0, 2, links, tries[links], eps=EPS)
    assert bad == 0
    got = post.reshape(-1, 4)[links]
    assert np.abs(got - want).max() < TOL
    assert np.abs(np.linalg.norm(post.reshape(-1, 4), axis=1) - 1).max() < 1e-6
    b.close()


def _golden_plaquette_8x4():
    """Mean and standard error of <P> at 8^4, beta = 2.3, from the stored
    40,000-sweep FP64 oracle run (tests/golden/make_su2_plaquette_8x4.py)."""
    import os
    vals = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "su2_plaquette_8x4_beta2.3.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals["mean"], vals["err"]


@pytest.mark.slow
def test_plaquette_average_8x4_long_run():
    """10^4 measured sweeps of 8^4 at beta = 2.3 on the GPU (after 1000
    thermalisation sweeps, the paper's protocol) against the stored
    independent 40,000-sweep FP64 oracle run: the averages agree within 3
    combined statistical sigma (binned errors; bins of 500 sweeps are far
    longer than the plaquette's autocorrelation), with no added slack."""
    L = (8, 8, 8, 8)
    beta = 2.3
    b = mc.Batch([mc.su2(L, beta, seed=21)], series_capacity=10_000)
    b.sweep(1000)
    b.read_series()
    b.sweep(10_000, 1)
    P = b.read_series()["P"][0]
    b.close()
    gm, ge = binned_mean_err(P, 20)
    om, oe = _golden_plaquette_8x4()
    print(f"<P> GPU {gm:.6f} +- {ge:.6f}  oracle {om:.6f} +- {oe:.6f}  "
          f"({(gm - om) / np.hypot(ge, oe):+.2f} sigma)")
    assert abs(gm - om) < 3 * np.hypot(ge, oe), (gm, ge, om, oe)


@pytest.mark.parametrize("n_or", [1, 3])
@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 8, 2)])
def test_overrelaxation_per_link(L, n_or):
    """One compound sweep (heat-bath + n_or overrelaxation sweeps) against the
    oracle's heat-bath sweep (following the GPU's tries, as above) and n_or
    oracle overrelaxation sweeps, from a thermalised start.  (On random links
    the staples can be short, and a reflection about a short staple magnifies
    FP32 round-off by ~1/|W| per sweep.)"""
    beta = 2.3
    q0 = oracle.su2_init(L, 9, 1, True)
    for k in range(20):
        oracle.su2_sweep(q0, L, beta, 9, 1, 1000 + k)
    q0 = f32_roundtrip(q0)
    b = mc.Batch([mc.su2(L, beta, seed=9, chain_id=1)])
    b.set_config(0, q0.astype(np.float32))
    b.set_overrelax(n_or)
    assert b.overrelax() == n_or
    b.record_tries(True)
    b.sweep(1)
    g = b.get_config(0).astype(np.float64)
    q = q0.copy()
    _, _, _, bad = oracle.su2_sweep(q, L, beta, 9, 1, 0, forced_tries=b.get_tries(0), eps=EPS)
    assert bad == 0
    for _ in range(n_or):
        oracle.su2_overrelax(q, L)
    err = np.abs(g - q).max()
    print(f"n_or={n_or}: max per-link deviation {err:.2e}")
    assert err < TOL
    assert b.sweeps_done == 1
    b.close()


def test_overrelaxation_strong_coupling_on_gpu():
    """Heat-bath + 2 overrelaxation sweeps still samples the Wilson measure:
    plaquette at beta = 0.2 equals I2(b)/I1(b) (closed form)."""
    from oracle import exact
    L, beta = (4, 4, 4, 4), 0.2
    b = mc.Batch([mc.su2(L, beta, seed=19, chain_id=k) for k in range(32)], series_capacity=2100)
    b.set_overrelax(2)
    b.sweep(200, 0)
    b.sweep(2000, 1)
    P = b.read_series()["P"]
    means = P.mean(axis=1)  # 32 independent chains
    mean, err = means.mean(), means.std(ddof=1) / np.sqrt(len(means))
    want = exact.strong_coupling_plaquette(beta)
    assert abs(mean - want) < 4.5 * err + 1e-4, (mean, want, err)
    b.close()


def test_overrelaxation_argument_checks():
    b = mc.Batch([mc.su2((4, 4, 4, 4), 2.0, seed=1)])
    for bad in (-1, 65):
        with pytest.raises(mc.MCError):
            b.set_overrelax(bad)
    b.close()
    i = mc.Batch([mc.ising(8, 0.4, seed=1)])
    with pytest.raises(mc.MCError):
        i.set_overrelax(1)
    i.close()


@pytest.mark.parametrize("L", [(4, 8, 8, 8), (2, 6, 4, 8), (8, 4, 4, 4)])
def test_polyakov_loop_matches_oracle(L):
    """GPU Polyakov loop of the same configuration as the oracle's: FP32 products
    of L0 quaternions, so within ~L0 x 1e-7; cold start gives exactly 1 (within
    the 2^-29 fixed-point quantum)."""
    b = mc.Batch([mc.su2(L, 2.3, seed=21, chain_id=0, hot=False), mc.su2(L, 2.3, seed=21, chain_id=1, hot=True)])
    assert abs(b.polyakov(0) - 1.0) < 1e-8
    b.sweep(5)
    for k in range(2):
        q = b.get_config(k).astype(np.float64)
        want = oracle.su2_polyakov(q, L)
        assert abs(b.polyakov(k) - want) < 2e-6, (b.polyakov(k), want)
    b.close()
    i = mc.Batch([mc.ising(8, 0.4, seed=1)])
    with pytest.raises(mc.MCError):
        i.polyakov(0)
    i.close()


def test_polyakov_loop_deconfinement_signal():
    """On an L_t = 2 lattice the loop is small in the confined phase (beta = 1.5)
    and large in the deconfined one (beta = 2.6, above the L_t = 2 transition at
    beta ~ 1.88): |<L>| averaged over chains, after thermalisation."""
    def absL(beta):
        b = mc.Batch([mc.su2((2, 8, 8, 8), beta, seed=30, chain_id=k, hot=False) for k in range(8)])
        b.set_overrelax(1)
        b.sweep(300, 0)
        vals = []
        for _ in range(20):
            b.sweep(5, 0)
            vals.append([abs(b.polyakov(k)) for k in range(8)])
        b.close()
        return float(np.mean(vals))
    low, high = absL(1.5), absL(2.6)
    print(f"|L| confined {low:.3f}, deconfined {high:.3f}")
    assert low < 0.2 and high > 2.5 * low, (low, high)


def _run_mode(chains, mode, n, every, n_or=0):
    cap = max(1, n // every) if every else 4
    b = mc.Batch(chains, series_capacity=cap)
    b.set_mode(mode)
    if n_or:
        b.set_overrelax(n_or)
    b.sweep(n, every)
    series = b.read_series() if every else None
    cfg = [b.get_config(k) for k in range(len(chains))]
    fails = b.failed_updates()
    b.close()
    return cfg, series, fails


@pytest.mark.parametrize("case", ["8x4_4beta", "table1_4x8x3_cold", "mixed_small", "12x4_multipass",
                                  "overrelax", "low_beta"])
def test_resident_mode_bit_identical_to_grid(case):
    """The single-launch SU(2) mode (one thread-block cluster per chain, all
    phases and sweeps of a call in one launch) gives bit-identical links,
    plaquette series and failure counts to the per-phase grid launches: the
    8^4 workload at its four beta, a Table 1 lattice from a cold start, uneven
    small shapes in one batch, a lattice needing several passes per phase,
    overrelaxation sweeps, and beta down to 0 (alpha = 0: Creutz only)."""
    n, every, n_or = 12, 1, 0
    if case == "8x4_4beta":
        chains = [mc.su2(8, b, seed=1, chain_id=i, hot=True) for i, b in enumerate([1.5, 2.0, 2.3, 2.6])]
    elif case == "table1_4x8x3_cold":
        chains = [mc.su2((4, 8, 8, 8), 2.3, seed=3, chain_id=0, hot=False)]
        n, every = 15, 5
    elif case == "mixed_small":
        chains = [mc.su2(L, 2.2, seed=5, chain_id=i, hot=True)
                  for i, L in enumerate([(2, 2, 2, 2), (6, 4, 8, 2), (4, 6, 2, 4), (8, 8, 6, 4)])]
    elif case == "12x4_multipass":
        chains = [mc.su2(12, 2.4, seed=7, chain_id=0, hot=True), mc.su2((4, 12, 12, 12), 1.9, seed=7, chain_id=1)]
        n, every = 6, 2
    elif case == "overrelax":
        chains = [mc.su2(8, 2.3, seed=9, chain_id=i, hot=True) for i in range(2)]
        n, every, n_or = 8, 2, 1
    else:
        chains = [mc.su2((4, 4, 6, 4), b, seed=11, chain_id=i, hot=True) for i, b in enumerate([0.0, 0.05, 0.3])]
        n, every = 10, 1
    ref = _run_mode(chains, mc.MC_MODE_GRID, n, every, n_or)
    got = _run_mode(chains, mc.MC_MODE_RESIDENT, n, every, n_or)
    for a, b_ in zip(ref[0], got[0]):
        np.testing.assert_array_equal(a, b_)
    for f in ("sweep", "P", "Ps", "Pt"):
        np.testing.assert_array_equal(ref[1][f], got[1][f])
    assert ref[2] == got[2]
    auto = _run_mode(chains, mc.MC_MODE_AUTO, n, every, n_or)
    for a, b_ in zip(ref[0], auto[0]):
        np.testing.assert_array_equal(a, b_)
