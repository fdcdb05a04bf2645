"""GPU parity of the learned proposal (BF16 tensor-core network, FP64 log q)
against the FP64 oracle (oracle/van.py), and exactness of its
Metropolis-Hastings correction against the Boltzmann distribution of Eq. (1).

Tolerances.  Weights are BF16-representable on both sides.  Against the oracle
run with BF16-rounded activations (the precision the task fixes), the GPU
differs only by FP32 accumulation order: log q to 1e-4 relative, gradients to
1e-3 relative per tensor.  Against the plain FP64 oracle the network itself is
a slightly different function -- each activation carries a relative rounding
of up to 2^-9 -- so log q agrees to 1e-2 relative, and a weight gradient, a sum
of ~10^3 terms of both signs, to cos > 0.995 and 10% relative (the measured
gap between the FP64 and BF16-activation oracles is cos 0.9984, rel 0.057 for
the test's network).  Normalisation (sum_s q(s) = 1) is structural and holds to
FP32 rounding."""
import numpy as np
import pytest
import torch
from scipy import stats

import oracle
import paper_0903_3053_gb300 as mc
from oracle import exact, van

pytestmark = pytest.mark.gpu


def bf16_params(depth=6, channels=32, seed=0, scale=1.0, bias=0.0):
    p = van.masked(van.init_params(depth, channels, seed=seed, scale=scale))
    rng = np.random.default_rng(seed + 100)
    out = []
    for W, b in p:
        Wb = torch.from_numpy(W).to(torch.bfloat16).to(torch.float64).numpy()
        bb = torch.from_numpy(b + bias * rng.normal(size=b.shape)).to(torch.bfloat16).to(torch.float64).numpy()
        out.append((Wb, bb))
    return out


def all_states(Lx, Ly):
    idx = np.arange(1 << (Lx * Ly))
    return (((idx[:, None] >> np.arange(Lx * Ly)) & 1) * 2 - 1).reshape(-1, Ly, Lx).astype(np.int8)


def test_log_prob_matches_oracle():
    L, n = 8, 32
    p = bf16_params(seed=1, bias=0.3)
    net = mc.VAN(L, batch=n, depth=6, seed=0)
    net.set_params(mc.mc.van_pack(p))
    rng = np.random.default_rng(2)
    s = np.where(rng.random((n, L, L)) < 0.5, 1, -1).astype(np.int8)
    g = net.log_prob(torch.from_numpy(s).cuda()).cpu().numpy()
    o = van.log_prob(p, s.astype(np.float64))
    assert np.max(np.abs(g - o) / np.abs(o)) < 1e-2, (g[:4], o[:4])
    ob = van.log_prob(p, s.astype(np.float64), act="bf16")
    assert np.max(np.abs(g - ob) / np.abs(ob)) < 1e-4, (g[:4], ob[:4])
    gn = net.log_prob(torch.from_numpy(s).cuda(), negate=True).cpu().numpy()
    on = van.log_prob(p, -s.astype(np.float64))
    assert np.max(np.abs(gn - on) / np.abs(on)) < 1e-2


def test_normalisation_4x4():
    """sum over all 2^16 states of q(s) = 1 (autoregressive structure)."""
    p = bf16_params(depth=6, seed=3, scale=1.5, bias=0.5)
    s = all_states(4, 4)
    net = mc.VAN(4, batch=len(s), depth=6, seed=0)
    net.set_params(mc.mc.van_pack(p))
    lq = net.log_prob(torch.from_numpy(s).cuda()).cpu().numpy()
    assert abs(np.exp(lq).sum() - 1.0) < 1e-4


def test_gradients_match_oracle():
    L, n = 8, 16
    p = bf16_params(seed=4, bias=0.2)
    net = mc.VAN(L, batch=n, depth=6, seed=0)
    net.set_params(mc.mc.van_pack(p))
    rng = np.random.default_rng(5)
    s = np.where(rng.random((n, L, L)) < 0.5, 1, -1).astype(np.int8)
    loss_g = net.train_step(torch.from_numpy(s).cuda(), lr=0.0, apply=False)
    _, gflat = net.get_params(grads=True)
    gg = mc.mc.van_unpack(gflat)
    for act, cos_min, rel_max in (("bf16", 1 - 1e-6, 1e-3), ("fp64", 0.995, 0.1)):
        loss_o, go = van.loss_and_grad(p, s.astype(np.float64), act=act)
        assert abs(loss_g - loss_o) / abs(loss_o) < (1e-5 if act == "bf16" else 1e-2)
        for l, ((gW, gb), (oW, ob)) in enumerate(zip(gg, go)):  # taps outside the masks are 0 on both sides
            a = np.concatenate([gW.ravel(), gb.ravel()])
            b = np.concatenate([oW.ravel(), ob.ravel()])
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert cos > cos_min and rel < rel_max, (act, l, cos, rel)


def test_training_step_is_deterministic():
    """Two identical training steps give bit-identical gradients: every
    reduction (weight gradients of all layers, loss) sums in a fixed order."""
    L, n = 16, 96
    net = mc.VAN(L, batch=n, depth=6, seed=4)
    net.set_params(mc.mc.van_pack(bf16_params(depth=6, seed=21)))
    g = torch.Generator().manual_seed(5)
    s = (torch.randint(0, 2, (n, L, L), generator=g) * 2 - 1).to(torch.int8).cuda()
    l1 = net.train_step(s, lr=0.0, apply=False)
    _, g1 = net.get_params(grads=True)
    l2 = net.train_step(s, lr=0.0, apply=False)
    _, g2 = net.get_params(grads=True)
    assert l1 == l2
    np.testing.assert_array_equal(g1, g2)


def test_sampler_follows_q():
    """Samples on a 4x4 lattice follow the network's own q (chi^2 over all
    states), and the sampler's log q equals a batched forward of its samples."""
    p = bf16_params(depth=4, seed=6, scale=1.5, bias=0.5)
    n = 8192
    net = mc.VAN(4, batch=65536, depth=4, seed=7)
    net.set_params(mc.mc.van_pack(p))
    samp, lq = net.sample(n, round=0)
    lq_fwd = net.log_prob(samp).cpu().numpy()
    assert np.max(np.abs(lq.cpu().numpy() - lq_fwd)) < 1e-3
    s = samp.cpu().numpy().reshape(n, -1)
    code = ((s > 0).astype(np.int64) << np.arange(16)).sum(axis=1)
    q = np.exp(net.log_prob(torch.from_numpy(all_states(4, 4)).cuda()).cpu().numpy())
    counts = np.bincount(code, minlength=1 << 16)
    e = q * n
    big = e >= 5
    obs = np.append(counts[big], counts[~big].sum())
    ex = np.append(e[big], e[~big].sum())
    chi2 = ((obs - ex) ** 2 / ex).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-4


def test_sampler_matches_oracle_sampler_statistics():
    """The same network sampled by the oracle (FP64) and by the GPU: the mean
    magnetisation and energy agree within their statistical errors."""
    L = 6
    p = bf16_params(depth=6, seed=8, scale=1.2, bias=0.4)
    net = mc.VAN(L, batch=4096, depth=6, seed=9)
    net.set_params(mc.mc.van_pack(p))
    g = net.sample(4096, round=3)[0].cpu().numpy().astype(np.float64)
    o = van.sample(p, 2000, L, np.random.default_rng(10).random((2000, L * L)))
    for f in (lambda s: s.mean(axis=(1, 2)), lambda s: van.ising_energy(s) / L ** 2):
        a, b = f(g), f(o)
        err = np.hypot(a.std() / np.sqrt(len(a)), b.std() / np.sqrt(len(b)))
        assert abs(a.mean() - b.mean()) < 4.5 * err


def test_mh_round_keeps_boltzmann_distribution():
    """Chains of a 4x4 torus started in the exact Boltzmann distribution stay in
    it under MH rounds with a deliberately poor network (exactness does not
    depend on training)."""
    beta, L, n = 0.4406868, 4, 4096
    en = exact.ising_enumerate(L, L, beta)
    chains = [mc.ising(L, beta, seed=3, chain_id=k) for k in range(n)]
    b = mc.Batch(chains, layout=mc.MC_LAYOUT_INT8)
    rng = np.random.default_rng(11)
    code = rng.choice(len(en["p"]), size=n, p=en["p"])
    start = (((code[:, None] >> np.arange(L * L)) & 1) * 2 - 1).reshape(n, L, L).astype(np.int8)
    mc.mc.ising_gather(b, torch.from_numpy(start).cuda(), back=True)
    net = mc.VAN(L, batch=n, depth=4, seed=12)
    net.set_params(mc.mc.van_pack(bf16_params(depth=4, seed=13, scale=2.0, bias=0.5)))
    acc = 0
    for _ in range(6):
        acc += net.mh_round(b)
    assert 0 < acc < 6 * n  # some accepted, some rejected
    s = mc.mc.ising_gather(b).cpu().numpy().reshape(n, -1)
    got = ((s > 0).astype(np.int64) << np.arange(L * L)).sum(axis=1)
    classes = {}
    for E, M, pr in zip(en["E_states"], en["M_states"], en["p"]):
        classes[(int(E), int(M))] = classes.get((int(E), int(M)), 0.0) + pr
    keys = sorted(classes)
    idx = {k: i for i, k in enumerate(keys)}
    counts = np.zeros(len(keys))
    for c in got:
        counts[idx[(int(en["E_states"][c]), int(en["M_states"][c]))]] += 1
    e = np.array([classes[k] for k in keys]) * n
    big = e >= 5
    obs = np.append(counts[big], counts[~big].sum()) if (~big).any() else counts[big]
    ex = np.append(e[big], e[~big].sum()) if (~big).any() else e[big]
    chi2 = ((obs - ex) ** 2 / ex).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-4


def test_training_lowers_loss_and_raises_acceptance():
    """Maximum-likelihood training on Metropolis configurations (8x8, beta_c)
    lowers -mean log q and raises the MH acceptance over the untrained network:
    what the network gains over the method without it."""
    beta, L = 0.4406868, 8
    nchain = 2048
    chains = [mc.ising(L, beta, seed=21, chain_id=k) for k in range(nchain)]
    b = mc.Batch(chains, layout=mc.MC_LAYOUT_INT8)
    b.sweep(200)
    data = [mc.mc.ising_gather(b).clone()]
    for _ in range(7):
        b.sweep(20)
        data.append(mc.mc.ising_gather(b).clone())
    data = torch.cat(data)
    net = mc.VAN(L, batch=nchain, depth=6, seed=22)
    net.set_params(mc.mc.van_pack(van.masked(van.init_params(6, 32, seed=23, scale=0.5))))
    acc0 = net.mh_round(b)
    gen = torch.Generator(device="cuda").manual_seed(0)
    first = last = None
    for step in range(300):
        idx = torch.randint(0, data.shape[0], (512,), device="cuda", generator=gen)
        loss = net.train_step(data[idx].contiguous(), lr=2e-3)
        first = loss if first is None else first
        last = loss
    assert last < first - 1.0, (first, last)
    acc1 = sum(net.mh_round(b) for _ in range(3)) / 3
    assert acc1 > 2 * max(acc0, 1), (acc0, acc1)


def test_full_size_L64_sampler_log_prob_and_gradients():
    """The benchmark's configuration, L = 64 with 4096 proposals: the sampler's
    FP64 log q equals the forward network's on what it sampled, and both equal
    the BF16-activation oracle on sampled configurations; one training step's
    loss and gradients at L = 64 (batch 32) match the oracle.  The gradient
    tolerance is looser than at L = 8: each weight gradient is a sum over
    32 x 4096 positions whose terms carry the 2^-16 relative error of the
    BF16 hi + lo split of dZ, and the sum cancels to ~1/100 of the sum of
    magnitudes, so 1e-2 relative (cos > 1 - 1e-5) is the arithmetic's bound."""
    L, n = 64, 4096
    p = bf16_params(seed=7, bias=0.2)
    net = mc.VAN(L, batch=n, depth=6, seed=3)
    net.set_params(mc.mc.van_pack(p))
    s, lq = net.sample(n, 0)
    lp = net.log_prob(s).cpu().numpy()
    lqs = lq.cpu().numpy()
    assert np.max(np.abs(lqs - lp) / np.abs(lp)) < 1e-5
    idx = [0, 1, 2047, n - 1]
    ob = van.log_prob(p, s[idx].cpu().numpy().astype(np.float64), act="bf16")
    assert np.max(np.abs(lp[idx] - ob) / np.abs(ob)) < 1e-4, (lp[idx], ob)
    # gradients on 32 of the sampled configurations
    sub = s[:32].contiguous()
    loss_g = net.train_step(sub, lr=0.0, apply=False)
    _, gflat = net.get_params(grads=True)
    gg = mc.mc.van_unpack(gflat)
    loss_o, go = van.loss_and_grad(p, sub.cpu().numpy().astype(np.float64), act="bf16")
    assert abs(loss_g - loss_o) / abs(loss_o) < 1e-5
    for l, ((gW, gb), (oW, ob_)) in enumerate(zip(gg, go)):
        a = np.concatenate([gW.ravel(), gb.ravel()])
        b = np.concatenate([oW.ravel(), ob_.ravel()])
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert cos > 1 - 1e-5 and rel < 1e-2, (l, cos, rel)
    net.close()


def test_sampler_prefetch_depths_and_coexisting_networks():
    """The sampler keeps up to three gathered hidden-layer tap tiles in flight
    (besides the output layer's), as many as shared memory allows and at most
    the D - 2 hidden layers: one at depth 3 and at depth 7 with L = 128, two at
    depth 4 and at depth 7 with L <= 96, three at depths 5 and 6.  For each, the
    sampler's FP64 log q equals the forward network's on what it sampled and
    the BF16-activation oracle's on two of the samples, and no bounded device
    wait gave up.  The networks are all created before any is sampled: creating
    a smaller network must not shrink the shared memory a larger one launches
    with."""
    cases = [(7, 96, 2), (3, 8, 64), (7, 8, 64), (6, 16, 64), (7, 128, 2), (4, 8, 40)]
    nets = []
    for depth, L, n in cases:
        p = bf16_params(depth=depth, seed=20 + depth, bias=0.2)
        net = mc.VAN(L, batch=n, depth=depth, seed=depth)
        net.set_params(mc.mc.van_pack(p))
        nets.append((net, p, L, n))
    for net, p, L, n in nets:
        s, lq = net.sample(n, round=5)
        net.sync()
        lp = net.log_prob(s).cpu().numpy()
        lqs = lq.cpu().numpy()
        assert np.max(np.abs(lqs - lp) / np.abs(lp)) < 1e-5, (L, lqs[:4], lp[:4])
        ob = van.log_prob(p, s[[0, n - 1]].cpu().numpy().astype(np.float64), act="bf16")
        assert np.max(np.abs(lp[[0, n - 1]] - ob) / np.abs(ob)) < 1e-4, (L, lp[[0, n - 1]], ob)
    for net, *_ in nets:
        net.close()


@pytest.mark.parametrize("L", [2, 6, 128])
def test_log_prob_extreme_lattice_sides(L):
    """The smallest lattices (one padded tile, rows past the lattice) and the
    largest side the network supports (several rows per tile item): log q of a
    few configurations against the BF16-activation oracle, and the gradient
    path runs."""
    n = 3
    p = bf16_params(seed=11, bias=0.2)
    net = mc.VAN(L, batch=n, depth=6, seed=0)
    net.set_params(mc.mc.van_pack(p))
    rng = np.random.default_rng(12)
    s = np.where(rng.random((n, L, L)) < 0.5, 1, -1).astype(np.int8)
    g = net.log_prob(torch.from_numpy(s).cuda()).cpu().numpy()
    ob = van.log_prob(p, s.astype(np.float64), act="bf16")
    assert np.max(np.abs(g - ob) / np.abs(ob)) < 1e-4, (g, ob)
    loss = net.train_step(torch.from_numpy(s).cuda(), lr=0.0, apply=False)
    assert np.isfinite(loss)
    net.close()


# --------------------------------------------------------------------------- element-wise parity
# Forward activations.  The GPU sums each hidden pre-activation in FP32 (tensor
# cores: exact BF16 products, FP32 accumulation of 13 taps x 32 channels + bias)
# and rounds its ReLU output to BF16; the oracle does the same in FP64.  Where
# the oracle's z lies within ACT_EPS x S of a BF16 rounding midpoint or of the
# ReLU kink (S = sum of |W| |x| + |b|, the scale of the FP32 sum's error; a
# typical FP32 sum of 417 terms errs by ~sqrt(417) 2^-24 S = 1.2e-6 S) the two
# may round differently: the oracle adopts the GPU's activation there and counts
# it (oracle.van.forward_following); any other difference fails.  Every hidden
# activation of every layer is checked this way.
ACT_EPS = 2.0 ** -17
# Gradients.  With the forward passes aligned, the backward passes differ only
# by (i) the FP32 logit and sigmoid of dF (relative ~2^-22), (ii) the BF16
# hi + lo hand-over of the upstream gradient between layers (relative <= 2^-17
# per hand-over, D - 1 hand-overs) and (iii) FP32 accumulation of <= 417 terms
# per output (<= 417 x 2^-24 of the sum of |terms| per layer).  Relative to
# oracle.van.grad_scale (every term in absolute value through the whole pass)
# that is <= (D - 1)(2^-17 + 417 x 2^-24) + 2^-22 ~ 1.6e-4 < 2^-12: GRAD_TOL.
# The propagated scale is loose for the early layers (their sums cancel
# through five layers of weights), so each element is also held to
# GRAD_TOL_DIRECT of the scale of its own sum (|upstream gradient| x
# |activation|), at which a wrong sign, a dropped or transposed tap shows in
# about 90% of the elements of every layer; this second bound is empirical
# (measured worst case 3.8e-3, an element that is a single term whose upstream
# gradient itself cancels to 1/600 of its terms; typical 1e-4 or less).
GRAD_TOL = 2.0 ** -12
GRAD_TOL_DIRECT = 2.0 ** -7
# Sampler.  The kernel compares its FP32 uniform with an FP32 sigmoid of a logit
# accumulated in FP32; the oracle compares the same uniform with the FP64
# conditional.  A draw may differ only where the two lie within SAMPLE_MARGIN.
SAMPLE_MARGIN = 1e-3
# MH.  The log ratio combines four FP64-accumulated log q values (each within
# 1e-4 relative of the oracle's, log q ~ -10 at L = 4) and an exact energy
# difference; a decision may differ only within MH_MARGIN of log u.
MH_MARGIN = 1e-2


def _grad_check(L, n, seed, depth=6):
    p = bf16_params(depth=depth, seed=seed, bias=0.2)
    net = mc.VAN(L, batch=n, depth=depth, seed=0)
    net.set_params(mc.mc.van_pack(p))
    rng = np.random.default_rng(seed + 1)
    s = np.where(rng.random((n, L, L)) < 0.5, 1, -1).astype(np.int8)
    loss_g = net.train_step(torch.from_numpy(s).cuda(), lr=0.0, apply=False)
    _, gflat = net.get_params(grads=True)
    acts = [net.get_activations(l, n) for l in range(depth - 1)]
    net.close()
    gg = mc.mc.van_unpack(gflat, depth=depth)
    loss_o, go, sp, sd, near, bad = van.loss_and_grad_following(p, s.astype(np.float64), acts, ACT_EPS)
    nact = sum(a.size for a in acts)
    assert bad == 0, f"{bad} activations differ away from any rounding boundary"
    assert near <= max(8, nact // 10000), (near, nact)
    assert abs(loss_g - loss_o) / abs(loss_o) < 1e-6
    worst, worst_d = 0.0, 0.0
    for l, ((gW, gb), (oW, ob), (sW, sb), (dW, db)) in enumerate(zip(gg, go, sp, sd)):
        for a, o, m, d, name in ((gW, oW, sW, dW, "W"), (gb, ob, sb, db, "b")):
            err = np.abs(a - o)
            live = m > 0
            # taps outside the masks, and parameters no term reaches: exactly zero on both sides
            assert np.all(a[~live] == 0.0) and np.all(o[~live] == 0.0), (l, name)
            r = err[live] / m[live]
            rd = err[live] / np.maximum(d[live], 1e-300)
            worst, worst_d = max(worst, float(r.max())), max(worst_d, float(rd.max()))
            i = np.argmax(r)
            assert r.max() <= GRAD_TOL, (l, name, np.argwhere(live)[i], a[live][i], o[live][i], m[live][i])
            i = np.argmax(rd)
            assert rd.max() <= GRAD_TOL_DIRECT, (l, name, np.argwhere(live)[i], a[live][i], o[live][i], d[live][i])
    print(f"L={L} n={n} seed={seed}: {near} of {nact} activations adopted near a boundary; max |g_gpu - g_oracle| "
          f"= {worst:.2g} of the propagated scale, {worst_d:.2g} of the direct scale")


@pytest.mark.parametrize("L,n,seed", [(8, 16, 4), (8, 16, 14), (6, 40, 24), (12, 3, 44), (14, 3, 44),
                                      (16, 16, 4), (16, 16, 44)])
def test_forward_activations_and_gradients_per_element(L, n, seed):
    """Every hidden activation of a training step's forward pass, and every
    weight and bias gradient of every layer, element by element against the
    BF16-activation oracle (which follows the GPU's activation only within
    ACT_EPS of a rounding boundary, counted)."""
    _grad_check(L, n, seed)


def test_full_size_L64_forward_and_gradients_per_element():
    """The same at the benchmark's lattice, L = 64 (a batch of 8)."""
    _grad_check(64, 8, 34)


@pytest.mark.parametrize("L,n,seed", [(2, 16, 66), (128, 1, 74)])
def test_extreme_sides_forward_and_gradients_per_element(L, n, seed):
    """The same at the smallest and the largest lattice side, where the
    tensor-core kernels' geometry changes: one padded row tile and a single
    16-position K step at L = 2; at L = 128 the forward convolution runs one
    CTA per SM (two would cost too many tiles) and the weight gradient's ring
    holds only two stages."""
    _grad_check(L, n, seed)


def _sampler_uniforms(seed, rnd, n, L):
    return van.sampler_uniforms(seed, rnd, range(n), L)


@pytest.mark.parametrize("L,n,depth", [(4, 64, 4), (6, 64, 6), (8, 32, 6)])
def test_sampler_draws_equal_oracle_on_the_kernel_stream(L, n, depth):
    """The oracle's sequential sampler fed the sampler's own Philox uniforms
    (the oracle's Philox in the same counter layout) draws the GPU's samples:
    sample by sample, equal up to the first position whose decision lies
    within SAMPLE_MARGIN of its threshold (counted; none expected)."""
    seed, rnd = 77, 5
    p = bf16_params(depth=depth, seed=40 + L, scale=1.3, bias=0.4)
    net = mc.VAN(L, batch=n, depth=depth, seed=seed)
    net.set_params(mc.mc.van_pack(p))
    g, _ = net.sample(n, round=rnd)
    net.close()
    g = g.cpu().numpy().astype(np.float64)
    u = _sampler_uniforms(seed, rnd, n, L)
    o = van.sample(p, n, L, u, act="bf16")
    pk = van.conditionals(p, o, act="bf16").reshape(n, -1)
    near = 0
    for b in range(n):
        diff = np.flatnonzero(g[b].ravel() != o[b].ravel())
        if len(diff):
            k = diff[0]
            assert abs(u[b, k] - pk[b, k]) < SAMPLE_MARGIN, (b, k, u[b, k], pk[b, k])
            near += 1
    print(f"L={L}: {near} of {n} samples diverge at a near-threshold draw")
    assert near <= max(1, n // 32)
    assert 0.1 < (g > 0).mean() < 0.9  # a non-trivial network


def test_full_size_L64_sampler_draws_per_position():
    """At L = 64 with 4096 proposals, every position of a sample of the GPU's
    draws is the oracle's decision u_k < p(s_k = +1 | s_<k) on the GPU's own
    prefix (the conditionals from one BF16-activation oracle forward pass),
    except within SAMPLE_MARGIN of the threshold (counted)."""
    L, n, seed, rnd = 64, 4096, 91, 2
    p = bf16_params(seed=7, bias=0.2)
    net = mc.VAN(L, batch=n, depth=6, seed=seed)
    net.set_params(mc.mc.van_pack(p))
    g, _ = net.sample(n, round=rnd)
    net.close()
    pick = [0, 1, 2047, 4095]
    gs = g[pick].cpu().numpy().astype(np.float64)
    u = van.sampler_uniforms(seed, rnd, pick, L)
    pk = van.conditionals(p, gs, act="bf16").reshape(len(pick), -1)
    want = np.where(u < pk, 1.0, -1.0)
    mism = want != gs.reshape(len(pick), -1)
    assert np.all(np.abs(u - pk)[mism] < SAMPLE_MARGIN), np.abs(u - pk)[mism]
    print(f"L=64: {int(mism.sum())} of {mism.size} draws at a near-threshold decision")
    assert mism.sum() <= 4


def test_mh_decisions_equal_oracle_per_chain():
    """One MH round on 4096 chains of a 4x4 torus (beta = 0.2, where an
    untrained network is accepted about half the time) with a poor network: the
    proposal (the sampler's draw for this round, possibly globally flipped by
    the chain's MH stream), the accept uniform and the decision of every chain
    against the oracle's log ratio (BF16-activation network, exact energies).
    Decisions may differ only within MH_MARGIN of log u (counted)."""
    beta, L, n, seed, rnd = 0.2, 4, 4096, 61, 9
    chains = [mc.ising(L, beta, seed=3, chain_id=k) for k in range(n)]
    b = mc.Batch(chains, layout=mc.MC_LAYOUT_INT8)
    b.sweep(5)
    p = bf16_params(depth=4, seed=13, scale=0.5, bias=0.2)
    net = mc.VAN(L, batch=n, depth=4, seed=seed)
    net.set_params(mc.mc.van_pack(p))
    cur = mc.mc.ising_gather(b).cpu().numpy().astype(np.float64)
    raw, _ = net.sample(n, round=rnd)
    raw = raw.cpu().numpy().astype(np.float64)
    net.set_round(rnd)
    acc = net.mh_round(b)
    new = mc.mc.ising_gather(b).cpu().numpy().astype(np.float64)
    net.close()
    b.close()
    u, flip = van.mh_draws(seed, rnd, range(n))
    prop = np.where(flip[:, None, None], -raw, raw)
    lr = van.mh_accept_logratio(p, beta, cur, prop, act="bf16")
    want = np.log(u) < lr
    got_accept = np.all(new == prop, axis=(1, 2))
    got_stay = np.all(new == cur, axis=(1, 2))
    assert np.all(got_accept | got_stay)  # each chain holds either its proposal or its old state
    ambiguous = got_accept & got_stay       # proposal equal to the current state
    got = np.where(ambiguous, want, got_accept)
    mism = got != want
    assert np.all(np.abs(np.log(u) - lr)[mism] < MH_MARGIN), np.abs(np.log(u) - lr)[mism]
    print(f"MH: {int(want.sum())} of {n} accepted; {int(mism.sum())} decisions at the threshold")
    assert mism.sum() <= 2
    assert abs(acc - int(got_accept.sum() - (ambiguous & ~want).sum())) <= int(mism.sum())
    assert 0.05 * n < want.sum() < 0.95 * n  # both outcomes well represented
