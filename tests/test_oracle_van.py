"""Pins of the learned-proposal oracle (oracle/van.py): exact normalisation of
the autoregressive distribution, the autoregressive mask, the backward pass
against finite differences, the sampler against q itself, and exactness of the
Metropolis-Hastings correction against the Boltzmann distribution of Eq. (1)."""
import numpy as np
import pytest
from scipy import stats

from oracle import exact, van


def all_states(Lx, Ly):
    idx = np.arange(1 << (Lx * Ly))
    return (((idx[:, None] >> np.arange(Lx * Ly)) & 1) * 2 - 1).reshape(-1, Ly, Lx).astype(np.float64)


def _merge_small(counts, expected, floor=5.0):
    """Pool the cells with expected count < floor into one (if there are any)."""
    big = expected >= floor
    obs, e = counts[big].astype(np.float64), expected[big]
    if (~big).any():
        obs = np.append(obs, counts[~big].sum())
        e = np.append(e, expected[~big].sum())
    return obs, e


def test_taps():
    assert len(van.taps("A")) == 12 and len(van.taps("B")) == 13
    assert (0, 0) not in van.taps("A") and (0, 0) in van.taps("B")
    assert all(dy < 0 or (dy == 0 and dx <= 0) for dy, dx in van.taps("B"))


def test_normalisation_by_enumeration():
    """sum_s q(s) = 1 exactly over all 2^16 states of a 4x4 lattice (any weights)."""
    p = van.masked(van.init_params(depth=4, channels=4, seed=3, scale=2.0))
    for a in range(2):
        p[1] = (p[1][0], p[1][1] + a)  # non-zero biases too
    q = np.exp(van.log_prob(p, all_states(4, 4)))
    assert abs(q.sum() - 1.0) < 1e-10


def test_autoregressive_mask():
    """f_k depends only on s_j for j < k in raster order."""
    rng = np.random.default_rng(1)
    p = van.masked(van.init_params(depth=6, channels=6, seed=1))
    L = 6
    s = np.where(rng.random((1, L, L)) < 0.5, 1.0, -1.0)
    f0, _ = van.forward(p, s)
    for j in [0, 7, 14, 20, 35]:
        s2 = s.copy()
        s2[0, j // L, j % L] *= -1
        f1, _ = van.forward(p, s2)
        d = np.abs(f1 - f0).reshape(-1)
        assert np.all(d[: j + 1] == 0.0), j
        if j < L * L - 1:
            assert d[j + 1:].max() > 0.0


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = van.masked(van.init_params(depth=6, channels=5, seed=2))
    p = [(W, b + 0.1 * rng.normal(size=b.shape)) for W, b in p]
    s = np.where(rng.random((3, 6, 6)) < 0.5, 1.0, -1.0)
    _, g = van.loss_and_grad(p, s)
    h = 1e-6
    for l in range(6):
        W, b = p[l]
        mask = "A" if l == 0 else "B"
        for _ in range(3):
            o = rng.integers(W.shape[0]); i = rng.integers(W.shape[1])
            dy, dx = van.taps(mask)[rng.integers(len(van.taps(mask)))]
            ix = (o, i, dy + 2, dx + 2)
            pp = [(w.copy(), bb.copy()) for w, bb in p]; pp[l][0][ix] += h
            pm = [(w.copy(), bb.copy()) for w, bb in p]; pm[l][0][ix] -= h
            fd = (van.loss_and_grad(pp, s)[0] - van.loss_and_grad(pm, s)[0]) / (2 * h)
            assert abs(g[l][0][ix] - fd) <= 1e-6 * max(1.0, abs(fd)), (l, ix, g[l][0][ix], fd)
        o = rng.integers(b.shape[0])
        pp = [(w.copy(), bb.copy()) for w, bb in p]; pp[l][1][o] += h
        pm = [(w.copy(), bb.copy()) for w, bb in p]; pm[l][1][o] -= h
        fd = (van.loss_and_grad(pp, s)[0] - van.loss_and_grad(pm, s)[0]) / (2 * h)
        assert abs(g[l][1][o] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_sampler_follows_q():
    """Chi-square of 20000 autoregressive samples on a 3x3 lattice against q."""
    p = van.masked(van.init_params(depth=4, channels=4, seed=5, scale=1.5))
    n = 20000
    u = np.random.default_rng(6).random((n, 9))
    s = van.sample(p, n, 3, u)
    states = all_states(3, 3)
    q = np.exp(van.log_prob(p, states))
    code = ((s.reshape(n, -1) > 0).astype(np.int64) << np.arange(9)).sum(axis=1)
    counts = np.bincount(code, minlength=512)
    obs, e = _merge_small(counts, q * n)
    chi2 = ((obs - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-4


def _mh_chain_histogram(correct: bool, n_chains=6000, steps=30, beta=0.4):
    """Independence-sampler chains on a 4x2 torus using only MH proposals from a
    deliberately poor (random) network, started in the exact Boltzmann
    distribution: an exact MH step keeps them there (stationarity), a wrong
    ratio drifts away."""
    Lx, Ly = 4, 2
    p = van.masked(van.init_params(depth=3, channels=4, seed=9, scale=2.0))
    rng = np.random.default_rng(10)
    en = exact.ising_enumerate(Lx, Ly, beta)
    code = rng.choice(len(en["p"]), size=n_chains, p=en["p"])
    s = (((code[:, None] >> np.arange(Lx * Ly)) & 1) * 2 - 1).reshape(-1, Ly, Lx).astype(np.float64)
    for _ in range(steps):
        # proposals from q_sym: sample from q, then flip globally with probability 1/2
        prop = _sample_rect(p, n_chains, Lx, Ly, rng)
        flip = rng.random(n_chains) < 0.5
        prop[flip] *= -1
        if correct:
            lr = (-beta * (van.ising_energy(prop) - van.ising_energy(s)) + van.log_prob_sym(p, s)
                  - van.log_prob_sym(p, prop))
        else:  # planted mistake: the proposal density left out of the ratio
            lr = -beta * (van.ising_energy(prop) - van.ising_energy(s))
        acc = np.log(rng.random(n_chains)) < lr
        s[acc] = prop[acc]
    return s


def _sample_rect(p, n, Lx, Ly, rng):
    s = np.zeros((n, Ly, Lx))
    for k in range(Lx * Ly):
        y, x = divmod(k, Lx)
        f, _ = van.forward(p, s)
        pr = 1.0 / (1.0 + np.exp(-f[:, y, x]))
        s[:, y, x] = np.where(rng.random(n) < pr, 1.0, -1.0)
    return s


@pytest.mark.parametrize("correct", [True, False])
def test_mh_correction_is_exact(correct):
    beta = 0.4
    s = _mh_chain_histogram(correct, beta=beta)
    en = exact.ising_enumerate(4, 2, beta)
    code = ((s.reshape(len(s), -1) > 0).astype(np.int64) << np.arange(8)).sum(axis=1)
    counts = np.bincount(code, minlength=256)
    obs, ex = _merge_small(counts, en["p"] * len(s))
    chi2 = ((obs - ex) ** 2 / ex).sum()
    pval = stats.chi2.sf(chi2, len(obs) - 1)
    if correct:
        assert pval > 1e-4, pval
    else:
        assert pval < 1e-6, pval  # the test has the power to see a wrong ratio


def test_bf16_rounding():
    """Round to nearest BF16, ties to even, against values worked out by hand."""
    # BF16 keeps 7 explicit significand bits: spacing 2^-7 at 1, halfway point 2^-8
    x = np.array([1.0, 1.0 + 2.0**-8, 1.0 + 3 * 2.0**-9, 1.0 + 2.0**-9 + 2.0**-20, 1.0 + 3 * 2.0**-8, -2.5,
                  3.14159265, 1.5 * 2.0**-100, 0.0])
    want = np.array([1.0, 1.0, 1.0 + 2.0**-7, 1.0, 1.0 + 2.0**-6, -2.5, 3.140625, 1.5 * 2.0**-100, 0.0])
    np.testing.assert_array_equal(van.round_bf16(x), want)
    r = van.round_bf16(np.linspace(-4, 4, 1001))
    assert np.all(np.abs(r - np.linspace(-4, 4, 1001)) <= 2.0**-8 * np.abs(np.linspace(-4, 4, 1001)) + 1e-45)


def test_bf16_activation_network_is_normalised():
    p = van.masked(van.init_params(depth=4, channels=4, seed=3, scale=2.0))
    q = np.exp(van.log_prob(p, all_states(4, 4), act="bf16"))
    assert abs(q.sum() - 1.0) < 1e-10


def test_philox_words_are_the_pinned_blocks():
    """The word-run helper the proposal's streams use returns, word for word,
    the Philox4x32-10 blocks pinned by the known-answer vectors."""
    import oracle
    seed = 0x0123456789ABCDEF
    w = oracle.philox_words(seed, 7, van.TAG_SAMPLE, 11, 22)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(22):
        blk = oracle.philox4x32_10([j >> 2, 7, van.TAG_SAMPLE, 11], key)
        assert w[j] == blk[j & 3]


def test_proposal_streams_are_uniform_and_distinct():
    u = van.sampler_uniforms(5, 3, range(64), 16)
    assert u.shape == (64, 256) and u.min() > 0.0 and u.max() <= 1.0
    assert stats.kstest(u.ravel(), "uniform").pvalue > 1e-4
    assert np.abs(np.corrcoef(u[:32].ravel(), u[32:].ravel())[0, 1]) < 0.02
    u2 = van.sampler_uniforms(5, 4, range(64), 16)  # another round
    assert np.abs(np.corrcoef(u.ravel(), u2.ravel())[0, 1]) < 0.02
    a, flip = van.mh_draws(5, 3, range(20000))
    assert a.min() > 0.0 and a.max() <= 1.0 and stats.kstest(a, "uniform").pvalue > 1e-4
    assert abs(flip.mean() - 0.5) < 4.0 * 0.5 / np.sqrt(len(flip))


@pytest.mark.parametrize("act", ["fp64", "bf16"])
def test_sample_takes_each_position_from_its_conditional(act):
    """The defining property of the autoregressive sampler: at every position,
    the drawn spin is +1 exactly when the position's uniform lies below
    p(s_k = +1 | s_<k) evaluated on the drawn prefix (one forward pass of the
    result gives every conditional at once)."""
    L, n = 5, 40
    p = van.masked(van.init_params(depth=4, channels=6, seed=12, scale=1.5))
    p[0] = (p[0][0], p[0][1] + 0.3)
    u = van.sampler_uniforms(9, 1, range(n), L)
    s = van.sample(p, n, L, u, act=act)
    pk = van.conditionals(p, s, act=act).reshape(n, -1)
    want = np.where(u < pk, 1.0, -1.0)
    np.testing.assert_array_equal(s.reshape(n, -1), want)
    # and the draws are not trivial: both spins occur, from a spread of probabilities
    assert 0.2 < (s > 0).mean() < 0.8 and pk.std() > 0.05


def test_grad_scale_bounds_every_gradient_element():
    """|gradient| <= scale element by element (triangle inequality), with
    equality when no sum cancels (non-negative weights, all spins +1: every
    term of every sum has the same sign)."""
    rng = np.random.default_rng(4)
    p = van.masked(van.init_params(depth=4, channels=5, seed=8))
    s = np.where(rng.random((6, 6, 6)) < 0.5, 1.0, -1.0)
    _, g = van.loss_and_grad(p, s)
    sc = van.grad_scale(p, s)
    for (gW, gb), (sW, sb) in zip(g, sc):
        assert np.all(np.abs(gW) <= sW * (1 + 1e-12) + 1e-300)
        assert np.all(np.abs(gb) <= sb * (1 + 1e-12) + 1e-300)
        assert (sW > 2 * np.abs(gW)).any()  # with mixed signs some sums do cancel
    # the direct scale (own sum only) lies between |gradient| and the propagated one
    for (gW, gb), (sW, sb), (dW, db) in zip(van.loss_and_grad(p, s)[1], van.grad_scale(p, s),
                                            van.grad_scale(p, s, propagate=False)):
        assert np.all(np.abs(gW) <= dW * (1 + 1e-12) + 1e-300) and np.all(dW <= sW * (1 + 1e-12) + 1e-300)
        assert np.all(np.abs(gb) <= db * (1 + 1e-12) + 1e-300) and np.all(db <= sb * (1 + 1e-12) + 1e-300)
    pos = [(np.abs(W), b) for W, b in p]
    ones = np.ones((3, 6, 6))
    _, g = van.loss_and_grad(pos, ones)
    sc = van.grad_scale(pos, ones)
    for (gW, gb), (sW, sb), (dW, db) in zip(g, sc, van.grad_scale(pos, ones, propagate=False)):
        np.testing.assert_allclose(np.abs(gW), sW, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(np.abs(gb), sb, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(np.abs(gW), dW, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(np.abs(gb), db, rtol=1e-12, atol=1e-300)


def test_forward_following_checks_and_adopts_activations():
    """forward_following / loss_and_grad_following: fed the oracle's own BF16
    activations it reproduces loss_and_grad(act="bf16") exactly with nothing
    near or bad; an activation moved by one BF16 step is 'bad' when no window
    is allowed and 'near' (adopted, and used downstream) when the window
    covers it; an activation the ReLU kept, set to zero, likewise -- and then
    its ReLU derivative is zero in the backward."""
    rng = np.random.default_rng(6)
    p = van.masked(van.init_params(depth=4, channels=5, seed=3))
    s = np.where(rng.random((3, 6, 6)) < 0.5, 1.0, -1.0)
    acts = van.hidden_activations(p, s)
    loss0, g0 = van.loss_and_grad(p, s, act="bf16")
    loss, g, sc, dr, near, bad = van.loss_and_grad_following(p, s, acts, eps_rel=0.0)
    assert (near, bad) == (0, 0) and loss == loss0
    for (a, b), (c, d) in zip(g, g0):
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(b, d)
    # one activation of the last hidden layer (so that no later activation is
    # rechecked against values computed from the old one), positive, moved up
    # by one BF16 step
    l = len(p) - 2
    pos = tuple(np.argwhere(acts[l] > 0.25)[0])
    v = acts[l][pos]
    step = 2.0 ** (np.floor(np.log2(v)) - 7)
    for new in (v + step, 0.0):
        other = [a.copy() for a in acts]
        other[l][pos] = new
        assert van.forward_following(p, s, other, eps_rel=0.0)[3:] == (0, 1)
        f, cache, masks, near, bad = van.forward_following(p, s, other, eps_rel=1.0)
        assert (near, bad) == (1, 0)
        b_, y_, x_, c_ = pos
        assert cache[l + 1][0][b_, c_, y_, x_] == new  # the next layer reads the adopted value
        assert masks[l][b_, c_, y_, x_] == (1.0 if new > 0 else 0.0)
        assert van.loss_and_grad_following(p, s, other, eps_rel=1.0)[0] != loss0
