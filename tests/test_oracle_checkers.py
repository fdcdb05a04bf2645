"""Pins of the oracle's sampled checkers, `orc_ising_check_sites` and
`orc_su2_check_links`, against the full-sweep oracle.

The checkers recompute single sites / links of one sweep from the
configurations before and after it, so that full-size GPU lattices can be
checked on a sample.  They restate the local rule and the phase order of the
sweep (Sec. 2.3: colour 0 then colour 1; Sec. 2.4: odd sites mu = 0..3, then
even sites mu = 0..3) separately from `orc_ising_sweep` / `orc_su2_sweep`,
which are pinned by exact enumeration, closed forms and invariants elsewhere.
Here every site and every link of one sweep, on several shapes, starts, beta
and sweep numbers, must come out of the checker exactly as the full sweep
produced it.  The second half of each test shows the check is not vacuous:
a wrong sweep number, or neighbours taken from the wrong side of the sweep,
changes the checker's answer."""
import numpy as np
import pytest

ISING_SHAPES = [(4, 4), (6, 10), (10, 6), (2, 2), (8, 2), (2, 8), (16, 16)]


@pytest.mark.parametrize("shape", ISING_SHAPES)
@pytest.mark.parametrize("hot", [True, False])
def test_ising_check_sites_reproduces_every_site(orc, shape, hot):
    Lx, Ly = shape
    for beta in (0.0, 0.3, 0.4406868, 0.6):
        for sweep, therm in ((0, 0), (7, 3), (123, 5)):
            s = orc.ising_init((Lx, Ly), seed=5, chain=2, hot=hot)
            if therm:
                orc.ising_run(s, beta, seed=5, chain=2, first_sweep=sweep - therm, n=therm, record=False)
            pre = s.copy()
            orc.ising_run(s, beta, seed=5, chain=2, first_sweep=sweep, n=1, record=False)
            sites = np.arange(Lx * Ly)
            got = orc.ising_check_sites(pre, s, beta, seed=5, chain=2, sweep=sweep, sites=sites)
            np.testing.assert_array_equal(got, s.ravel(), err_msg=f"{shape} hot={hot} beta={beta} sweep={sweep}")


def test_ising_check_sites_is_sensitive(orc):
    """A wrong sweep number, a wrong chain, or colour-1 sites reading the
    pre-sweep colour-0 spins each change some recomputed site."""
    Lx, Ly, beta = 16, 12, 0.4406868
    s = orc.ising_init((Lx, Ly), seed=9, chain=0, hot=True)
    orc.ising_run(s, beta, seed=9, chain=0, first_sweep=0, n=4, record=False)
    pre = s.copy()
    orc.ising_run(s, beta, seed=9, chain=0, first_sweep=4, n=1, record=False)
    sites = np.arange(Lx * Ly)
    good = orc.ising_check_sites(pre, s, beta, 9, 0, 4, sites)
    np.testing.assert_array_equal(good, s.ravel())
    assert (orc.ising_check_sites(pre, s, beta, 9, 0, 5, sites) != good).any()
    assert (orc.ising_check_sites(pre, s, beta, 9, 1, 4, sites) != good).any()
    # colour-1 sites must see the post-sweep colour-0 neighbours: with pre in both roles they differ
    assert (orc.ising_check_sites(pre, pre, beta, 9, 0, 4, sites) != good).any()


SU2_SHAPES = [(2, 2, 2, 2), (4, 4, 4, 4), (2, 4, 2, 4), (4, 2, 6, 2), (6, 4, 2, 2)]


@pytest.mark.parametrize("L", SU2_SHAPES)
@pytest.mark.parametrize("hot", [True, False])
def test_su2_check_links_reproduces_every_link(orc, L, hot):
    """Every link of one heat-bath sweep, recomputed by the checker from the
    lattice each phase saw, equals the full sweep's result to FP64 rounding;
    no decision is classified near or bad (nothing is forced) and the
    failure count agrees."""
    nlinks = 4 * int(np.prod(L))
    for beta in (0.5, 2.3):
        for sweep, therm in ((0, 0), (5, 2)):
            q = orc.su2_init(L, seed=4, chain=1, hot=hot)
            for k in range(therm):
                orc.su2_sweep(q, L, beta, seed=4, chain=1, sweep=sweep - therm + k)
            pre = q.copy()
            _, fails, _, _ = orc.su2_sweep(q, L, beta, seed=4, chain=1, sweep=sweep)
            out, cfails, near, bad = orc.su2_check_links(pre, q, L, beta, seed=4, chain=1, sweep=sweep,
                                                         links=np.arange(nlinks))
            assert near == 0 and bad == 0
            assert cfails == fails
            np.testing.assert_allclose(out, q.reshape(-1, 4), rtol=0, atol=1e-14,
                                       err_msg=f"L={L} hot={hot} beta={beta} sweep={sweep}")


def test_su2_check_links_is_sensitive(orc):
    """The phase order matters: treating no link as already updated (pre in
    both roles), a wrong sweep number or a wrong chain changes links; and a
    subset of links gives the same values as the full list."""
    L, beta = (4, 4, 4, 4), 2.3
    nlinks = 4 * int(np.prod(L))
    q = orc.su2_init(L, seed=8, chain=0, hot=True)
    orc.su2_sweep(q, L, beta, seed=8, chain=0, sweep=0)
    pre = q.copy()
    orc.su2_sweep(q, L, beta, seed=8, chain=0, sweep=1)
    links = np.arange(nlinks)
    good = orc.su2_check_links(pre, q, L, beta, 8, 0, 1, links)[0]
    np.testing.assert_allclose(good, q.reshape(-1, 4), atol=1e-14)
    for args in ((pre, pre, 8, 0, 1), (pre, q, 8, 0, 2), (pre, q, 8, 3, 1)):
        other = orc.su2_check_links(args[0], args[1], L, beta, args[2], args[3], args[4], links)[0]
        assert np.abs(other - good).max() > 1e-3, args
    # links of the first phase (odd sites, mu = 0) see only pre-sweep links: pre/pre gives them right
    pp = orc.su2_check_links(pre, pre, L, beta, 8, 0, 1, links)[0]
    s = links >> 2
    x1, x2, x3, x0 = s % 4, (s // 4) % 4, (s // 16) % 4, s // 64
    first = ((x0 + x1 + x2 + x3) % 2 == 1) & ((links & 3) == 0)
    np.testing.assert_allclose(pp[first], good[first], atol=1e-14)
    assert np.abs(pp[~first] - good[~first]).max() > 1e-3
    rng = np.random.default_rng(0)
    sub = np.sort(rng.choice(nlinks, size=97, replace=False))
    np.testing.assert_array_equal(orc.su2_check_links(pre, q, L, beta, 8, 0, 1, sub)[0], good[sub])
