"""GPU parity of the Ising sweep (Eq. (1), Sec. 2.3): the CUDA path, called
through the C ABI, must reproduce the oracle bit for bit -- configurations and
the exact E/M series -- in every layout, execution mode and block size."""
import numpy as np
import pytest

import oracle
import paper_0903_3053_gb300 as mc

pytestmark = pytest.mark.gpu
BC = 0.4406868


def run_gpu(chains, layout, n, every=1, mode=mc.MC_MODE_AUTO, threads=0, cap=None):
    b = mc.Batch(chains, layout=layout, series_capacity=cap or max(1, n // max(every, 1)))
    if mode != mc.MC_MODE_AUTO or threads:
        b.set_mode(mode, threads)
    b.sweep(n, every)
    series = b.read_series() if every else None
    cfgs = [b.get_config(k) for k in range(len(chains))]
    b.close()
    return cfgs, series


def test_hot_and_cold_init_match_oracle():
    for layout in (mc.MC_LAYOUT_INT8, mc.MC_LAYOUT_MSC32):
        for hot in (True, False):
            b = mc.Batch([mc.ising((128, 64), 0.3, seed=77, chain_id=5, hot=hot)], layout=layout)
            np.testing.assert_array_equal(b.get_config(0), oracle.ising_init((128, 64), 77, 5, hot))
            b.close()


@pytest.mark.parametrize("mode", [mc.MC_MODE_RESIDENT, mc.MC_MODE_GRID])
def test_64x64_beta_c_1000_sweeps_bit_exact(mode):
    """64x64 periodic, J=1, h=0, beta=0.4406868, hot start seed 1, int8 spins,
    1000 sweeps with E and M measured after every sweep."""
    s = oracle.ising_init(64, seed=1, chain=0, hot=True)
    E, M = oracle.ising_run(s, BC, 1, 0, 0, 1000)
    cfgs, series = run_gpu([mc.ising(64, BC, seed=1)], mc.MC_LAYOUT_INT8, 1000, 1, mode)
    np.testing.assert_array_equal(cfgs[0], s)
    np.testing.assert_array_equal(series["E"][0], E)
    np.testing.assert_array_equal(series["M"][0], M)
    np.testing.assert_array_equal(series["sweep"][0], np.arange(1000))


@pytest.mark.parametrize("beta", [0.30, 0.40, BC, 0.50, 0.60])
def test_msc_1024_bit_exact(beta):
    """Multi-spin-coded L = 1024, hot start: configuration after 1, 2 and 10
    sweeps and the E/M series equal the oracle's."""
    s = oracle.ising_init(1024, seed=1, chain=2, hot=True)
    b = mc.Batch([mc.ising(1024, beta, seed=1, chain_id=2)], layout=mc.MC_LAYOUT_MSC32, series_capacity=16)
    done = 0
    for k in (1, 1, 8):
        E, M = oracle.ising_run(s, beta, 1, 2, done, k)
        b.sweep(k, 1)
        done += k
        rec = b.read_series()
        np.testing.assert_array_equal(b.get_config(0), s)
        np.testing.assert_array_equal(rec["E"][0], E)
        np.testing.assert_array_equal(rec["M"][0], M)
    b.close()


@pytest.mark.parametrize("layout", [mc.MC_LAYOUT_INT8, mc.MC_LAYOUT_MSC32])
@pytest.mark.parametrize("launch", ["grid", "auto", "group"])
def test_paper_lattice_1024x512_bit_exact(layout, launch):
    """The paper's Ising lattice (Sec. 2.3: 1024 x 512, the shape of its only
    Ising timing), hot start, beta_c: configuration and E/M series after 10
    sweeps equal the oracle's, through the per-colour launches, the mode the
    context picks for itself and the persistent group launch (the lattice is
    too large for the shared-memory resident mode)."""
    shape = (1024, 512)
    s = oracle.ising_init(shape, seed=1, chain=0, hot=True)
    E, M = oracle.ising_run(s, BC, 1, 0, 0, 10)
    b = mc.Batch([mc.ising(shape, BC, seed=1, chain_id=0)], layout=layout, series_capacity=16)
    if launch == "group":
        g = mc.Group([b])
        g.sweep(10, 1)
        g.close()
    else:
        b.set_mode(mc.MC_MODE_GRID if launch == "grid" else mc.MC_MODE_AUTO)
        b.sweep(10, 1)
    rec = b.read_series()
    np.testing.assert_array_equal(b.get_config(0), s)
    np.testing.assert_array_equal(rec["E"][0], E)
    np.testing.assert_array_equal(rec["M"][0], M)
    b.close()


@pytest.mark.parametrize("layout,shape", [
    (mc.MC_LAYOUT_INT8, (2, 2)), (mc.MC_LAYOUT_INT8, (2, 6)), (mc.MC_LAYOUT_INT8, (6, 2)),
    (mc.MC_LAYOUT_INT8, (10, 14)), (mc.MC_LAYOUT_INT8, (130, 66)),
    (mc.MC_LAYOUT_MSC32, (64, 2)), (mc.MC_LAYOUT_MSC32, (64, 6)), (mc.MC_LAYOUT_MSC32, (192, 34)),
    (mc.MC_LAYOUT_MSC32, (128, 320)),
])
@pytest.mark.parametrize("mode", [mc.MC_MODE_GRID, mc.MC_MODE_RESIDENT])
def test_ragged_and_degenerate_shapes(layout, shape, mode):
    """Rectangular, 2-wide (doubled bonds), one-word-per-row and ragged Philox
    groups; both execution modes."""
    s = oracle.ising_init(shape, seed=9, chain=1, hot=True)
    E, M = oracle.ising_run(s, 0.35, 9, 1, 0, 25)
    cfgs, series = run_gpu([mc.ising(shape, 0.35, seed=9, chain_id=1)], layout, 25, 5, mode)
    np.testing.assert_array_equal(cfgs[0], s)
    np.testing.assert_array_equal(series["E"][0], E[4::5])
    np.testing.assert_array_equal(series["M"][0], M[4::5])


@pytest.mark.parametrize("threads", [32, 64, 128, 512, 1024])
def test_block_size_invariance(threads):
    chains = [mc.ising((256, 128), 0.44, seed=3, chain_id=0)]
    ref, rs = run_gpu(chains, mc.MC_LAYOUT_MSC32, 12, 3, mc.MC_MODE_GRID, 256)
    got, gs = run_gpu(chains, mc.MC_LAYOUT_MSC32, 12, 3, mc.MC_MODE_GRID, threads)
    np.testing.assert_array_equal(ref[0], got[0])
    np.testing.assert_array_equal(rs, gs)
    got2, _ = run_gpu(chains, mc.MC_LAYOUT_MSC32, 12, 3, mc.MC_MODE_RESIDENT, threads)
    np.testing.assert_array_equal(ref[0], got2[0])


@pytest.mark.parametrize("layout,L,threads", [
    (mc.MC_LAYOUT_MSC32, 64, 0), (mc.MC_LAYOUT_MSC32, 64, 1024), (mc.MC_LAYOUT_INT8, 32, 0),
    (mc.MC_LAYOUT_INT8, 32, 64),
])
def test_resident_small_chains_more_ctas_than_sms(layout, L, threads):
    """Resident CTAs are sized to the chain's work (64^2 MSC32: 32 row pairs,
    one warp; 32^2 int8: 128 site groups), capped by the block size: 400
    chains in one launch equal grid mode chain by chain and the oracle on a
    sample of them."""
    chains = [mc.ising(L, 0.3 + 0.0005 * k, seed=21, chain_id=k, hot=bool(k % 2)) for k in range(400)]
    ref, rs = run_gpu(chains, layout, 16, 4, mc.MC_MODE_GRID)
    got, gs = run_gpu(chains, layout, 16, 4, mc.MC_MODE_RESIDENT, threads)
    for k in range(len(chains)):
        np.testing.assert_array_equal(got[k], ref[k])
    np.testing.assert_array_equal(gs, rs)
    for k in (0, 151, 399):
        c = chains[k]
        s = oracle.ising_init(L, 21, k, c.start == mc.MC_HOT)
        E, M = oracle.ising_run(s, c.beta, 21, k, 0, 16)
        np.testing.assert_array_equal(got[k], s)
        np.testing.assert_array_equal(gs["E"][k], E[3::4])
        np.testing.assert_array_equal(gs["M"][k], M[3::4])


@pytest.mark.parametrize("layout", [mc.MC_LAYOUT_INT8, mc.MC_LAYOUT_MSC32])
def test_batch_of_uneven_chains(layout):
    rng = np.random.default_rng(0)
    sizes = [64, 128, 64, 192, 256, 64]
    chains = []
    for k, L in enumerate(sizes):
        chains.append(mc.ising((L, sizes[-1 - k]), float(rng.uniform(0.35, 0.55)), seed=1000 + k, chain_id=k,
                               hot=bool(k % 3)))
    for mode in (mc.MC_MODE_GRID, mc.MC_MODE_RESIDENT):
        cfgs, series = run_gpu(chains, layout, 20, 2, mode)
        for k, c in enumerate(chains):
            s = oracle.ising_init(c.L, c.seed, c.chain_id, c.start == mc.MC_HOT)
            E, M = oracle.ising_run(s, c.beta, c.seed, c.chain_id, 0, 20)
            np.testing.assert_array_equal(cfgs[k], s)
            np.testing.assert_array_equal(series["E"][k], E[1::2])
            np.testing.assert_array_equal(series["M"][k], M[1::2])


def test_config_roundtrip_and_formats():
    rng = np.random.default_rng(4)
    s = np.where(rng.random((96, 128)) < 0.5, 1, -1).astype(np.int8)
    bits = np.packbits((s > 0).astype(np.uint8), axis=1, bitorder="little").view(np.uint32)
    for layout in (mc.MC_LAYOUT_INT8, mc.MC_LAYOUT_MSC32):
        b = mc.Batch([mc.ising((128, 96), 0.4, seed=1)], layout=layout)
        b.set_config(0, s)
        np.testing.assert_array_equal(b.get_config(0), s)
        np.testing.assert_array_equal(b.get_config(0, mc.MC_FMT_BITS), bits)
        b.set_config(0, -s)
        b.set_config(0, bits, mc.MC_FMT_BITS)
        np.testing.assert_array_equal(b.get_config(0), s)
        E, M = oracle.ising_observe(s)
        m = b.measure(0)
        assert (m["E"], m["M"]) == (E, M)
        b.close()


def _msc_planes(s):
    """uint32 plane[c][y][w] of the MSC32 storage, packed here from its
    definition: bit b of word w of row y in plane c is the site x = 2 (32 w + b)
    + ((y + c) & 1)."""
    Ly, Lx = s.shape
    out = np.zeros((2, Ly, Lx // 64), dtype=np.uint32)
    for c in range(2):
        for y in range(Ly):
            xs = 2 * np.arange(Lx // 2) + ((y + c) & 1)
            bits = (s[y, xs] > 0).astype(np.uint8)
            out[c, y] = np.packbits(bits, bitorder="little").view(np.uint32)
    return out


def test_native_format_is_the_storage():
    """MC_FMT_NATIVE returns the storage as documented (int8 rows; MSC32 colour
    planes) and a native checkpoint restores a chain bit-exactly."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    s = np.where(rng.random((64, 192)) < 0.5, 1, -1).astype(np.int8)
    for layout, want in ((mc.MC_LAYOUT_INT8, s), (mc.MC_LAYOUT_MSC32, _msc_planes(s))):
        c = mc.ising((192, 64), BC, seed=21)
        b = mc.Batch([c], layout=layout)
        assert b.config_bytes(0, mc.MC_FMT_NATIVE) == want.nbytes
        b.set_config(0, s)
        np.testing.assert_array_equal(b.get_config(0, mc.MC_FMT_NATIVE), want)
        b.sweep(9)
        ckpt, done = b.get_config(0, mc.MC_FMT_NATIVE), b.sweeps_done
        b.sweep(11)
        ref = b.get_config(0)
        r = mc.Batch([c], layout=layout)
        dev = torch.from_numpy(ckpt.copy()).cuda()
        r.set_config_device(0, dev, mc.MC_FMT_NATIVE)
        r.sweeps_done = done
        r.sweep(11)
        np.testing.assert_array_equal(r.get_config(0), ref)
        r.set_config(0, -s)
        r.set_config(0, want, mc.MC_FMT_NATIVE)
        np.testing.assert_array_equal(r.get_config(0), s)
        b.close()
        r.close()


def test_config_through_page_locked_host_memory():
    """Page-locked host buffers are read and written in place by the layout
    conversion kernels (no staging copy); results equal the staged path's."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    s = np.where(rng.random((64, 192)) < 0.5, 1, -1).astype(np.int8)
    bits = np.packbits((s > 0).astype(np.uint8), axis=1, bitorder="little").view(np.uint32)
    for layout in (mc.MC_LAYOUT_INT8, mc.MC_LAYOUT_MSC32):
        b = mc.Batch([mc.ising((192, 64), 0.4, seed=1)], layout=layout)
        b.set_config_host_async(0, torch.from_numpy(s.copy()).pin_memory())
        b.sync()
        np.testing.assert_array_equal(b.get_config(0), s)
        b.set_config(0, -s)
        hb = torch.from_numpy(bits.view(np.int32).copy()).pin_memory()
        b.set_config_host_async(0, hb, mc.MC_FMT_BITS)
        b.sync()
        np.testing.assert_array_equal(b.get_config(0), s)
        out_bits = torch.zeros(bits.shape, dtype=torch.int32).pin_memory()
        b.get_config_host(0, out_bits, mc.MC_FMT_BITS)
        np.testing.assert_array_equal(out_bits.numpy().view(np.uint32), bits)
        out8 = torch.zeros(s.shape, dtype=torch.int8).pin_memory()
        b.get_config_host(0, out8)
        np.testing.assert_array_equal(out8.numpy(), s)
        b.close()


def test_resume_is_bit_exact():
    """Checkpoint = configuration + sweep counter (counter-based stream)."""
    c = mc.ising(128, BC, seed=11)
    a = mc.Batch([c], layout=mc.MC_LAYOUT_MSC32)
    a.sweep(30)
    ref = a.get_config(0)
    b = mc.Batch([c], layout=mc.MC_LAYOUT_MSC32)
    b.sweep(13)
    cfg, done = b.get_config(0), b.sweeps_done
    b.close()
    r = mc.Batch([c], layout=mc.MC_LAYOUT_MSC32)
    r.set_config(0, cfg)
    r.sweeps_done = done
    r.sweep(17)
    np.testing.assert_array_equal(r.get_config(0), ref)


def test_graph_replay_and_ring_buffer():
    """Repeated calls replay one captured graph; device-side counters keep the
    stream and record positions advancing; the ring wraps."""
    c = mc.ising(64, 0.5, seed=2)
    s = oracle.ising_init(64, 2, 0, True)
    E, M = oracle.ising_run(s, 0.5, 2, 0, 0, 60)
    b = mc.Batch([c], layout=mc.MC_LAYOUT_INT8, series_capacity=7)
    got = []
    for _ in range(12):
        b.sweep(5, 1)
        got.append(b.read_series())
    got = np.concatenate(got, axis=1)
    np.testing.assert_array_equal(got["E"][0], E)
    np.testing.assert_array_equal(got["M"][0], M)
    with pytest.raises(mc.MCError):
        b.sweep(8, 1)  # 8 records > capacity 7
    b.close()


@pytest.mark.parametrize("L,layout", [(16384, mc.MC_LAYOUT_MSC32), (4096, mc.MC_LAYOUT_MSC32),
                                      (4096, mc.MC_LAYOUT_INT8)])
def test_full_size_sampled_sites(L, layout):
    """Full-size lattices in the benchmark's launch configuration: every one of
    200k sampled sites of one sweep is recomputed by the oracle from the
    configurations before and after; E/M of the final state checked exactly."""
    beta = BC
    b = mc.Batch([mc.ising(L, beta, seed=1, chain_id=3)], layout=layout, series_capacity=4)
    b.set_mode(mc.MC_MODE_GRID, 256)
    b.sweep(3)
    pre = b.get_config(0)
    b.sweep(1, 1)
    post = b.get_config(0)
    rec = b.read_series()
    rng = np.random.default_rng(L)
    sites = rng.integers(0, L * L, size=200_000)
    want = oracle.ising_check_sites(pre, post, beta, 1, 3, 3, sites)
    np.testing.assert_array_equal(post.reshape(-1)[sites], want)
    E, M = oracle.ising_observe(post)
    assert (int(rec["E"][0, 0]), int(rec["M"][0, 0])) == (E, M)
    assert (pre != post).any()
    b.close()


@pytest.mark.parametrize("beta", [3.0, 6.0])
@pytest.mark.parametrize("mode", [mc.MC_MODE_GRID, mc.MC_MODE_RESIDENT])
def test_msc_thresholds_rounding_to_zero(beta, mode):
    """Large beta: the dE = 8 threshold floor(e^{-8 beta} 2^32) is 0 at beta = 3
    and both are 0 at beta = 6, so no site with dE > 0 may flip (the multi-spin
    kernel treats a zero threshold apart from its carry-chain compare); the
    configurations and E/M series still equal the oracle's."""
    t2, t4 = (int(v) for v in oracle.ising_thresholds(beta))
    assert t4 == 0 and (t2 == 0) == (beta == 6.0)
    chains = [mc.ising((128, 64), beta, seed=11, chain_id=4), mc.ising((64, 128), beta, seed=12, chain_id=5)]
    cfgs, series = run_gpu(chains, mc.MC_LAYOUT_MSC32, 6, 1, mode)
    for k, c in enumerate(chains):
        s = oracle.ising_init(c.L, c.seed, c.chain_id, True)
        E, M = oracle.ising_run(s, beta, c.seed, c.chain_id, 0, 6)
        np.testing.assert_array_equal(cfgs[k], s)
        np.testing.assert_array_equal(series["E"][k], E)
        np.testing.assert_array_equal(series["M"][k], M)


def test_beta_zero_flips_everything_on_gpu():
    b = mc.Batch([mc.ising((256, 64), 0.0, seed=5)], layout=mc.MC_LAYOUT_MSC32)
    s0 = b.get_config(0)
    b.sweep(1)
    np.testing.assert_array_equal(b.get_config(0), -s0)
    b.close()


def test_philox_rate_probe_computes_philox():
    """The multiply-ceiling probe that bench.py times generates true Philox
    blocks: each thread's output is the xor of the words of its blocks
    (counter (thread id, i, 0x7F000000, 0)), recomputed with the oracle's
    Philox."""
    import torch
    blocks, threads, iters, seed = 3, 64, 5, 0x1234_5678_9ABC
    out = torch.zeros(blocks * threads, dtype=torch.int32, device="cuda")
    mc.mc.philox_rate(blocks, threads, iters, seed, out)
    got = out.cpu().numpy().view(np.uint32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for tid in (0, 1, 63, 64, 191):
        want = np.uint32(0)
        for i in range(iters):
            want ^= np.bitwise_xor.reduce(oracle.philox4x32_10([tid, i, 0x7F000000, 0], key))
        assert got[tid] == want, tid
