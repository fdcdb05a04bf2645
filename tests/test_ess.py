"""The integrated-autocorrelation estimator (Sokal windowing) against closed
forms, and a small end-to-end run of the plain and learned-proposal chains."""
import numpy as np
import pytest

from paper_0903_3053_gb300 import ess


@pytest.mark.parametrize("phi", [0.0, 0.5, 0.9])
def test_tau_int_of_ar1(phi):
    """AR(1) x_t = phi x_{t-1} + noise: rho(t) = phi^t, tau = (1 + phi) / (2 (1 - phi))."""
    rng = np.random.default_rng(3)
    n, chains = 20000, 16
    x = np.zeros((chains, n))
    e = rng.normal(size=(chains, n))
    for t in range(1, n):
        x[:, t] = phi * x[:, t - 1] + e[:, t]
    want = (1 + phi) / (2 * (1 - phi))
    assert ess.tau_int(x) == pytest.approx(want, rel=0.08)


def test_autocorrelation_of_constant_lag_structure():
    x = np.tile([1.0, -1.0], 500)[None, :]  # rho(t) = (-1)^t
    rho = ess.autocorrelation(x)
    assert rho[0] == pytest.approx(1.0) and rho[1] == pytest.approx(-1.0) and rho[2] == pytest.approx(1.0)


@pytest.mark.gpu
def test_small_ess_comparison_runs():
    p = ess.plain_rate(16, 0.4406868, chains=256, therm=500, sweeps=4000, every=2)
    assert p["tau_absM_sweeps"] > 1 and p["ess_per_s"] > 0 and 0.3 < p["mean_absm"] < 1.0
    q = ess.learned_rate(16, 0.4406868, chains=512, therm=300, data_snapshots=8, data_spacing=20, train_steps=150,
                         train_batch=256, rounds=60, local_sweeps=10)
    assert q["loss_last"] < q["loss_first"]
    assert 0.0 < q["acceptance"] <= 1.0 and q["ess_per_s"] > 0
    assert abs(q["mean_absm"] - p["mean_absm"]) < 0.08  # same Boltzmann distribution


def test_tau_error_estimates_cover_the_truth():
    """The Sokal variance formula and the spread over chain groups both give
    errors that cover the closed-form tau of AR(1) series ~4000 tau long, and
    agree with each other within a factor of three; a series shorter than its
    window is flagged.  (On much shorter series the windowed estimator also
    carries a bias of order W tau / n from the mean subtraction, which neither
    error estimate includes: one reason to run for >= 1000 tau.)"""
    rng = np.random.default_rng(11)
    phi, n, chains = 0.8, 20000, 32
    want = (1 + phi) / (2 * (1 - phi))
    x = np.zeros((chains, n))
    e = rng.normal(size=(chains, n))
    for t in range(1, n):
        x[:, t] = phi * x[:, t - 1] + e[:, t]
    r = ess.tau_int_with_error(x)
    assert r["closed"] and r["length_over_tau"] > 100
    assert abs(r["tau"] - want) < 4 * r["err_sokal"] and abs(r["tau"] - want) < 4 * r["err_groups"]
    assert 1 / 3 < r["err_sokal"] / r["err_groups"] < 3
    short = ess.tau_int_with_error(x[:, :20])
    assert not short["closed"]
