"""Pins of the Ising oracle (Eq. (1), Metropolis on the checkerboard, Sec. 2.3)
against what the physics fixes: exact enumeration, Kaufman's finite-torus
partition function, Onsager/Yang, the Metropolis acceptance rule itself, and
exact special cases and symmetries."""
import math

import numpy as np
import pytest
from scipy import stats

from conftest import binned_mean_err
from oracle import exact

BC = 0.4406868


def test_kaufman_closed_form_matches_enumeration():
    """The closed form itself, pinned by brute force (including m != n)."""
    for (m, n) in [(4, 4), (4, 5), (5, 4), (2, 6)]:
        for beta in [0.1, 0.3, BC, 0.7]:
            en = exact.ising_enumerate(m, n, beta)
            assert exact.kaufman_lnZ(m, n, beta) == pytest.approx(en["lnZ"], rel=1e-12, abs=1e-12)
            assert exact.kaufman_energy(m, n, beta) == pytest.approx(en["e"], rel=1e-9, abs=1e-9)


def test_onsager_matches_kaufman_large_lattice():
    for beta in [0.3, 0.6]:
        assert exact.kaufman_energy(256, 256, beta) == pytest.approx(exact.onsager_energy(beta), abs=1e-10)
    assert exact.onsager_energy(exact.BETA_C) == pytest.approx(-math.sqrt(2.0), abs=1e-12)


def test_thresholds_special_values(orc):
    assert list(orc.ising_thresholds(0.0)) == [0xFFFFFFFF, 0xFFFFFFFF]
    assert list(orc.ising_thresholds(50.0)) == [0, 0]
    t2, t4 = (int(v) for v in orc.ising_thresholds(BC))
    assert abs(t2 / 2**32 - math.exp(-4 * BC)) < 2**-31
    assert abs(t4 / 2**32 - math.exp(-8 * BC)) < 2**-31


def test_metropolis_acceptance_per_energy_change(orc):
    """Colour-0 sites are updated first, against the initial colour-1 spins, so
    their flip rate per class of dE = 2 s h can be read off one sweep: 1 for
    dE <= 0, exp(-beta dE) otherwise (Metropolis min(1, e^{-beta dE}))."""
    beta, L = 0.2, 256
    s0 = orc.ising_init(L, seed=5, chain=0, hot=True)
    s = s0.copy()
    orc.ising_run(s, beta, seed=5, chain=0, first_sweep=0, n=1, record=False)
    h = np.roll(s0, 1, 0) + np.roll(s0, -1, 0) + np.roll(s0, 1, 1) + np.roll(s0, -1, 1)
    local = s0 * h
    yy, xx = np.indices(s0.shape)
    c0 = ((xx + yy) & 1) == 0
    flipped = (s != s0)
    for sl in (-4, -2, 0):
        sel = c0 & (local == sl)
        assert sel.sum() > 100
        assert flipped[sel].all()
    for sl in (2, 4):
        sel = c0 & (local == sl)
        k, n = int(flipped[sel].sum()), int(sel.sum())
        p = math.exp(-2 * beta * sl)
        z = (k - n * p) / math.sqrt(n * p * (1 - p))
        assert abs(z) < 4.5, (sl, k, n, p)


@pytest.mark.parametrize("beta", [0.3, BC, 0.6])
def test_4x4_moments_vs_enumeration(orc, beta):
    en = exact.ising_enumerate(4, 4, beta)
    s = orc.ising_init(4, seed=11, chain=3, hot=True)
    orc.ising_run(s, beta, 11, 3, 0, 1000, record=False)
    E, M = orc.ising_run(s, beta, 11, 3, 1000, 200_000)
    for series, want in [(E / 16, en["e"]), (np.abs(M) / 16, en["absm"]), (M.astype(float) ** 2, en["M2"])]:
        mean, err = binned_mean_err(series, 40)
        assert abs(mean - want) < 4.5 * err + 1e-12, (mean, want, err)


def test_4x4_stationary_distribution_chi2(orc):
    """Independent chains (different chain ids), each run well past its
    autocorrelation time; the final (E, M) class histogram must follow the exact
    Boltzmann weights."""
    beta = 0.35
    en = exact.ising_enumerate(4, 4, beta)
    classes = {}
    for E, M, p in zip(en["E_states"], en["M_states"], en["p"]):
        classes[(int(E), int(M))] = classes.get((int(E), int(M)), 0.0) + p
    keys = sorted(classes)
    index = {k: i for i, k in enumerate(keys)}
    n_chains = 12000
    counts = np.zeros(len(keys))
    for ch in range(n_chains):
        s = orc.ising_init(4, seed=21, chain=ch, hot=True)
        orc.ising_run(s, beta, 21, ch, 0, 30, record=False)
        E, M = orc.ising_observe(s)
        counts[index[(E, M)]] += 1
    expected = np.array([classes[k] for k in keys]) * n_chains
    big = expected >= 5
    obs = np.append(counts[big], counts[~big].sum())
    exp_ = np.append(expected[big], expected[~big].sum())
    chi2 = float(((obs - exp_) ** 2 / exp_).sum())
    p = stats.chi2.sf(chi2, len(obs) - 1)
    assert p > 1e-4, (chi2, len(obs), p)


@pytest.mark.parametrize("Lx,Ly,beta", [(32, 32, BC), (16, 8, 0.3), (8, 16, 0.6)])
def test_energy_vs_kaufman_finite_torus(orc, Lx, Ly, beta):
    """Rectangular lattices pin the Lx/Ly bookkeeping: Kaufman's m x n torus."""
    want = exact.kaufman_energy(Lx, Ly, beta)
    s = orc.ising_init((Lx, Ly), seed=3, chain=0, hot=True)
    orc.ising_run(s, beta, 3, 0, 0, 2000, record=False)
    E, _ = orc.ising_run(s, beta, 3, 0, 2000, 20_000)
    mean, err = binned_mean_err(E / (Lx * Ly), 20)
    assert abs(mean - want) < 4.5 * err, (mean, want, err)


@pytest.mark.parametrize("beta", [0.5, 0.6])
def test_spontaneous_magnetisation_onsager(orc, beta):
    """Deep in the ordered phase a 64^2 torus has <|m|> = m0 up to corrections
    of order exp(-L/xi) (xi of a few lattice spacings)."""
    want = exact.onsager_magnetisation(beta)
    s = orc.ising_init(64, seed=9, chain=1, hot=False)
    orc.ising_run(s, beta, 9, 1, 0, 200, record=False)
    _, M = orc.ising_run(s, beta, 9, 1, 200, 2000)
    mean, err = binned_mean_err(np.abs(M) / 4096.0, 20)
    assert abs(mean - want) < 4.5 * err + 2e-3, (mean, want, err)


def test_infinite_temperature_flips_every_spin(orc):
    """beta = 0: both thresholds clamp to 2^32 - 1, so every site flips unless its
    random word is exactly 2^32 - 1 (strict <)."""
    s0 = orc.ising_init((48, 32), seed=17, chain=2, hot=True)
    s = s0.copy()
    orc.ising_run(s, 0.0, 17, 2, 0, 1, record=False)
    assert (s == -s0).all()


def test_zero_temperature_never_raises_energy(orc):
    s = orc.ising_init(32, seed=2, chain=0, hot=False)
    orc.ising_run(s, 50.0, 2, 0, 0, 5, record=False)
    assert (s == 1).all()
    s = orc.ising_init(32, seed=2, chain=0, hot=True)
    E, _ = orc.ising_run(s, 50.0, 2, 0, 0, 50)
    assert (np.diff(E) <= 0).all()
    assert E[-1] < E[0]


def test_global_spin_flip_symmetry(orc):
    """s -> -s leaves s_i h_i unchanged, so with the same random words the
    trajectory from -s0 is exactly minus the trajectory from s0."""
    s0 = orc.ising_init((24, 40), seed=4, chain=7, hot=True)
    a = s0.copy()
    b = (-s0).copy()
    Ea, Ma = orc.ising_run(a, BC, 4, 7, 100, 60)
    Eb, Mb = orc.ising_run(b, BC, 4, 7, 100, 60)
    assert (b == -a).all()
    assert (Ea == Eb).all() and (Ma == -Mb).all()


def test_hot_start_is_fair_coin(orc):
    s = orc.ising_init(256, seed=1, chain=0, hot=True)
    n = s.size
    k = int((s == 1).sum())
    assert abs(k - n / 2) < 4.5 * math.sqrt(n / 4)
    # neighbouring spins uncorrelated
    corr = float((s * np.roll(s, 1, 1)).mean())
    assert abs(corr) < 4.5 / math.sqrt(n)


def test_observables_definition(orc):
    """E counts each of the 2 L^2 bonds once; all-up gives E = -2N, M = N; a
    checkerboard (antiferromagnet) gives E = +2N, M = 0."""
    s = np.ones((6, 8), dtype=np.int8)
    assert orc.ising_observe(s) == (-96, 48)
    yy, xx = np.indices((6, 8))
    s = np.where(((xx + yy) & 1) == 0, 1, -1).astype(np.int8)
    assert orc.ising_observe(s) == (96, 0)
