"""Effective sample rates: plain checkerboard Metropolis versus Metropolis
interleaved with the learned global proposal, for |M| at beta_c.

The integrated autocorrelation time is estimated with Sokal's automatic
windowing (A. D. Sokal, "Monte Carlo methods in statistical mechanics:
foundations and new algorithms", 1996): tau(W) = 1/2 + sum_{t=1}^{W} rho(t),
with W the smallest window such that W >= c tau(W), c = 6; the
autocorrelation function rho is averaged over chains.  An observable series of
n measurements then carries n / (2 tau) independent samples.  This is host-side
analysis of the recorded series (the paper's post-production step); every
sweep, sample and Metropolis-Hastings step runs in libmc's kernels.
"""
from __future__ import annotations

import time

import numpy as np


def autocorrelation(series: np.ndarray) -> np.ndarray:
    """Mean normalised autocorrelation function of chains x time (FFT, zero
    padded), each chain centred on the global mean."""
    x = np.atleast_2d(np.asarray(series, dtype=np.float64))
    x = x - x.mean()
    n = x.shape[1]
    f = np.fft.rfft(x, 2 * n, axis=1)
    acf = np.fft.irfft(f * np.conj(f), axis=1)[:, :n].mean(axis=0)
    acf /= np.arange(n, 0, -1)  # unbiased lag averages
    return acf / acf[0]


def tau_int_window(series: np.ndarray, c: float = 6.0):
    """(tau, W, closed): Sokal's windowed estimate, its window W and whether
    the window closed (W >= c tau) before the end of the series."""
    rho = autocorrelation(series)
    tau = 0.5
    for w in range(1, len(rho)):
        tau += rho[w]
        if w >= c * tau:
            return float(tau), w, True
    return float(tau), len(rho) - 1, False  # window never closed: the series is too short


def tau_int(series: np.ndarray, c: float = 6.0) -> float:
    return tau_int_window(series, c)[0]


def tau_int_with_error(series: np.ndarray, c: float = 6.0, groups: int = 8) -> dict:
    """tau with two error estimates: Sokal's variance formula
    var(tau) ~ 2 (2 W + 1) tau^2 / N over the N = chains x length measurements,
    and the spread of tau over `groups` disjoint groups of chains (standard
    error of their mean); the series is measured in units of one record."""
    x = np.atleast_2d(np.asarray(series, dtype=np.float64))
    tau, w, closed = tau_int_window(x, c)
    n = x.size
    err_sokal = tau * np.sqrt(2.0 * (2 * w + 1) / n)
    g = min(groups, x.shape[0])
    per = [tau_int(part, c) for part in np.array_split(x, g, axis=0)] if g >= 2 else [tau]
    err_groups = float(np.std(per, ddof=1) / np.sqrt(len(per))) if len(per) > 1 else float("nan")
    return {"tau": tau, "err_sokal": float(err_sokal), "err_groups": err_groups, "window": w, "closed": closed,
            "length_over_tau": x.shape[1] / tau}


def _cuda_time(fn):
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def plain_tau_long(L: int, beta: float, chains: int, therm: int, sweeps: int, every: int, seed: int = 1,
                   layout: int | None = None) -> dict:
    """tau of |M| (in sweeps, with its errors) from a long run of fewer chains:
    the full batch of the rate measurement would not fit a 1000-tau series in
    the ring buffer."""
    from . import mc
    layout = mc.MC_LAYOUT_INT8 if layout is None else layout
    b = mc.Batch([mc.ising(L, beta, seed, chain_id=100000 + k) for k in range(chains)], layout=layout,
                 series_capacity=sweeps // every + 4)
    b.sweep(therm)
    b.read_series()
    secs = _cuda_time(lambda: b.sweep(sweeps, every))
    absm = np.abs(b.read_series()["M"].astype(np.float64)) / (L * L)
    b.close()
    r = tau_int_with_error(absm)
    return {"tau_absM_sweeps": r["tau"] * every, "err_sokal": r["err_sokal"] * every,
            "err_chain_groups": r["err_groups"] * every, "run_over_tau": r["length_over_tau"],
            "window_closed": r["closed"], "chains": chains, "sweeps": sweeps, "every": every, "seconds": secs}


def plain_rate(L: int, beta: float, chains: int, therm: int, sweeps: int, every: int, seed: int = 1,
               layout: int | None = None) -> dict:
    """Plain Metropolis: chain-sweeps per second and tau of |M| in sweeps
    (int8 layout by default; the 32-spin words where L allows)."""
    from . import mc
    layout = mc.MC_LAYOUT_INT8 if layout is None else layout
    b = mc.Batch([mc.ising(L, beta, seed, chain_id=k) for k in range(chains)], layout=layout,
                 series_capacity=sweeps // every + 4)
    b.sweep(therm)
    b.sweep(every, every)  # graph warm-up
    b.read_series()
    secs = _cuda_time(lambda: b.sweep(sweeps, every))
    absm = np.abs(b.read_series()["M"].astype(np.float64)) / (L * L)
    r = tau_int_with_error(absm)
    tau = r["tau"] * every
    b.close()
    rate = chains * sweeps / secs
    return {"chain_sweeps_per_s": rate, "tau_absM_sweeps": tau, "tau_err_sokal": r["err_sokal"] * every,
            "tau_err_chain_groups": r["err_groups"] * every, "run_over_tau": r["length_over_tau"],
            "ess_per_s": rate / (2.0 * tau), "seconds": secs,
            "chains": chains, "sweeps": sweeps, "mean_absm": float(absm.mean()),
            "layout": "msc32" if layout == mc.MC_LAYOUT_MSC32 else "int8"}


def learned_rate(L: int, beta: float, chains: int, therm: int, data_snapshots: int, data_spacing: int,
                 train_steps: int, train_batch: int, rounds: int, local_sweeps: int = 10, lr: float = 2e-3,
                 seed: int = 2, depth: int = 6) -> dict:
    """Metropolis interleaved 1:local_sweeps with the learned proposal: train
    the network by maximum likelihood on configurations of plain chains, then
    time rounds of (MH proposal, local sweeps) and estimate tau of |M| in
    rounds."""
    import torch

    from . import mc
    b = mc.Batch([mc.ising(L, beta, seed, chain_id=k) for k in range(chains)], layout=mc.MC_LAYOUT_INT8,
                 series_capacity=rounds + 4)
    b.sweep(therm)
    # training data: snapshots of the plain chains, data_spacing sweeps apart
    t0 = time.perf_counter()
    data = []
    for _ in range(data_snapshots):
        b.sweep(data_spacing)
        data.append(mc.ising_gather(b).clone())
    data = torch.cat(data)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = mc.VAN(L, batch=max(chains, train_batch), depth=depth, seed=seed)
    net.set_params(_init_flat(depth, 32, seed, 0.5))
    gen = torch.Generator(device="cuda").manual_seed(seed)
    t0 = time.perf_counter()
    losses = []
    for step in range(train_steps):
        idx = torch.randint(0, data.shape[0], (train_batch,), device="cuda", generator=gen)
        want = step == 0 or step == train_steps - 1
        loss = net.train_step(data[idx].contiguous(), lr=lr, apply=True)  # synchronous: returns the loss
        if want:
            losses.append(loss)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    net.mh_round(b)  # warm-up round (and graph capture of the local sweeps)
    b.sweep(local_sweeps, local_sweeps)
    b.read_series()
    acc_total = 0

    def run():
        nonlocal acc_total
        for _ in range(rounds):
            acc_total += net.mh_round(b)
            b.sweep(local_sweeps, local_sweeps)

    secs = _cuda_time(run)
    absm = np.abs(b.read_series()["M"].astype(np.float64)) / (L * L)
    r = tau_int_with_error(absm)
    tau = r["tau"]
    # the sequential sampler alone: L^2 dependent steps through every layer
    t_sample = _cuda_time(lambda: net.sample(chains, 0x7FFFFFFF))
    net.close()
    b.close()
    rate = chains * rounds / secs
    return {"rounds_per_s": rounds / secs, "chain_rounds_per_s": rate, "tau_absM_rounds": tau,
            "tau_err_sokal": r["err_sokal"], "tau_err_chain_groups": r["err_groups"],
            "run_over_tau": r["length_over_tau"],
            "ess_per_s": rate / (2.0 * tau), "acceptance": acc_total / (chains * rounds), "seconds": secs,
            "local_sweeps_per_round": local_sweeps, "chains": chains, "rounds": rounds,
            "train_seconds": t_train, "data_seconds": t_data, "train_configs": int(data.shape[0]),
            "train_steps": train_steps, "loss_first": losses[0], "loss_last": losses[-1],
            "mean_absm": float(absm.mean()), "sample_ms": t_sample * 1e3,
            "sample_us_per_position": t_sample * 1e6 / (L * L)}


def _init_flat(depth: int, channels: int, seed: int, scale: float) -> np.ndarray:
    """He-style random initial weights (masked taps are ignored by the network)."""
    rng = np.random.default_rng(seed)
    out = []
    for l in range(depth):
        cin = 1 if l == 0 else channels
        cout = 1 if l == depth - 1 else channels
        ntap = 12 if l == 0 else 13
        out.append(rng.normal(0.0, scale * np.sqrt(2.0 / (cin * ntap)), size=cout * cin * 25))
        out.append(np.zeros(cout))
    return np.concatenate(out).astype(np.float32)
