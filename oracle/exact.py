"""Closed forms and brute-force references that pin the oracle (test
infrastructure; see the package docstring for who may import it).

* ``ising_enumerate``  -- every state of a small periodic lattice, Eq. (1).
* ``kaufman_*``        -- Kaufman's exact partition function of the finite
  periodic m x n torus (B. Kaufman, Phys. Rev. 76 (1949) 1232; in the form of
  A. E. Ferdinand & M. E. Fisher, Phys. Rev. 185 (1969) 832), evaluated in
  multiple precision with mpmath.
* ``onsager_*``        -- the infinite-lattice internal energy (Onsager 1944)
  and spontaneous magnetisation (Yang 1952).
* ``heatbath_*``       -- the SU(2) heat-bath density sqrt(1 - a^2) e^{alpha a}
  of the a0 component, its normaliser pi I1(alpha)/alpha and its mean
  I2(alpha)/I1(alpha) (the single-plaquette strong-coupling <P> at alpha=beta).
"""
from __future__ import annotations

import functools
import math

import mpmath
import numpy as np
from scipy import integrate, special

BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))


# --------------------------------------------------------------------------- Ising
@functools.lru_cache(maxsize=8)
def ising_all_states(Lx: int, Ly: int):
    """E and M of every one of the 2^(Lx*Ly) states of the periodic lattice,
    state bits read in row-major order (bit k -> site (k % Lx, k // Lx), 1 = +1).
    E counts each bond once exactly as Eq. (1): -sum s(x,y)[s(x+1,y)+s(x,y+1)]."""
    n = Lx * Ly
    assert n <= 24
    idx = np.arange(1 << n, dtype=np.int64)
    s = ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int8) * 2 - 1
    s = s.reshape(-1, Ly, Lx)
    E = -(s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)).astype(np.int64) \
        - (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2)).astype(np.int64)
    M = s.sum(axis=(1, 2)).astype(np.int64)
    return E, M


def ising_enumerate(Lx: int, Ly: int, beta: float):
    """Exact Boltzmann averages by brute force: dict with lnZ, <E>, <|M|>, <M^2>,
    per-site <e>, <|m|>, and the state probabilities."""
    E, M = ising_all_states(Lx, Ly)
    w = -beta * E.astype(np.float64)
    wmax = w.max()
    p = np.exp(w - wmax)
    Z = p.sum()
    p /= Z
    N = Lx * Ly
    return {
        "lnZ": float(np.log(Z) + wmax),
        "E": float((p * E).sum()),
        "absM": float((p * np.abs(M)).sum()),
        "M2": float((p * M.astype(np.float64) ** 2).sum()),
        "e": float((p * E).sum()) / N,
        "absm": float((p * np.abs(M)).sum()) / N,
        "p": p,
        "E_states": E,
        "M_states": M,
    }


def _kaufman_lnZ_mp(m: int, n: int, K):
    """ln Z of the m x n periodic Ising torus at coupling K (mpmath number),
    Kaufman's four-term form: Z = (1/2)(2 sinh 2K)^{mn/2} (Z1+Z2+Z3+Z4) with
    Z1 = prod_r 2cosh(m g_{2r+1}/2), Z2 = prod_r 2sinh(m g_{2r+1}/2),
    Z3 = prod_r 2cosh(m g_{2r}/2),   Z4 = prod_r 2sinh(m g_{2r}/2), r = 0..n-1,
    cosh g_l = cosh 2K cosh 2K* - sinh 2K sinh 2K* cos(pi l / n), tanh K* = e^{-2K},
    and g_0 = 2(K - K*) with its sign kept."""
    K = mpmath.mpf(K)
    Ks = mpmath.atanh(mpmath.e ** (-2 * K))
    c = mpmath.cosh(2 * K) * mpmath.cosh(2 * Ks)
    d = mpmath.sinh(2 * K) * mpmath.sinh(2 * Ks)

    def gamma(l):
        if l == 0:
            return 2 * (K - Ks)
        return mpmath.acosh(c - d * mpmath.cos(mpmath.pi * l / n))

    Z1 = Z2 = Z3 = Z4 = mpmath.mpf(1)
    for r in range(n):
        go = gamma(2 * r + 1)
        ge = gamma(2 * r)
        Z1 *= 2 * mpmath.cosh(m * go / 2)
        Z2 *= 2 * mpmath.sinh(m * go / 2)
        Z3 *= 2 * mpmath.cosh(m * ge / 2)
        Z4 *= 2 * mpmath.sinh(m * ge / 2)
    pref = mpmath.mpf(m * n) / 2 * mpmath.log(2 * mpmath.sinh(2 * K))
    return pref + mpmath.log((Z1 + Z2 + Z3 + Z4) / 2)


def kaufman_lnZ(m: int, n: int, beta: float, dps: int = 50) -> float:
    with mpmath.workdps(dps):
        return float(_kaufman_lnZ_mp(m, n, mpmath.mpf(beta)))


def kaufman_energy(m: int, n: int, beta: float, dps: int = 60) -> float:
    """Exact <E>/(m n) = -(1/mn) d lnZ / d beta on the finite torus."""
    with mpmath.workdps(dps):
        d = mpmath.diff(lambda b: _kaufman_lnZ_mp(m, n, b), mpmath.mpf(beta))
        return float(-d / (m * n))


def onsager_energy(beta: float) -> float:
    """Infinite-lattice energy per site u = -coth(2b)[1 + (2/pi)(2 tanh^2(2b) - 1) K(k)],
    k = 2 sinh(2b)/cosh^2(2b), K the complete elliptic integral of the first kind."""
    b2 = 2.0 * beta
    k = 2.0 * math.sinh(b2) / math.cosh(b2) ** 2
    coef = 2.0 * math.tanh(b2) ** 2 - 1.0
    if k >= 1.0 or coef == 0.0:
        # at beta_c the elliptic integral diverges only logarithmically while its
        # coefficient vanishes linearly: the product tends to 0
        return -1.0 / math.tanh(b2)
    Kk = special.ellipk(k * k)  # scipy uses the parameter m = k^2
    return -1.0 / math.tanh(b2) * (1.0 + (2.0 / math.pi) * coef * Kk)


def onsager_magnetisation(beta: float) -> float:
    """Spontaneous magnetisation per site (1 - sinh(2b)^-4)^(1/8) for b > b_c, else 0."""
    if beta <= BETA_C:
        return 0.0
    return (1.0 - math.sinh(2.0 * beta) ** -4) ** 0.125


# --------------------------------------------------------------------------- SU(2)
def heatbath_density(a, alpha: float):
    """Normalised density of a0: sqrt(1-a^2) e^{alpha a} / (pi I1(alpha)/alpha)."""
    a = np.asarray(a, dtype=np.float64)
    norm = math.pi * special.ive(1, alpha) / alpha  # times e^{alpha}, cancelled below
    return np.sqrt(np.clip(1.0 - a * a, 0.0, None)) * np.exp(alpha * (a - 1.0)) / norm


def heatbath_cdf(a: float, alpha: float) -> float:
    val, _ = integrate.quad(lambda t: heatbath_density(t, alpha), -1.0, a, limit=200, epsabs=1e-13)
    return float(val)


def heatbath_mean(alpha: float) -> float:
    """<a0> = I2(alpha)/I1(alpha)."""
    return float(special.ive(2, alpha) / special.ive(1, alpha))


def strong_coupling_plaquette(beta: float) -> float:
    """Single-plaquette (leading strong-coupling) value <P> = I2(beta)/I1(beta)."""
    return heatbath_mean(beta)


def heatbath_cdf_vec(a, alpha) -> np.ndarray:
    """Vectorised CDF of the a0 density at per-sample alpha.  With t = -cos(phi)
    the integrand sqrt(1-t^2) e^{alpha t} dt becomes the smooth
    sin^2(phi) e^{-alpha cos(phi)} dphi, integrated by 96-point Gauss-Legendre
    on [0, phi(a)] and normalised by the same rule on [0, pi]."""
    a = np.clip(np.asarray(a, dtype=np.float64), -1.0, 1.0)
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), a.shape)
    x, w = np.polynomial.legendre.leggauss(96)

    def integral(upper):
        phi = 0.5 * upper[..., None] * (x + 1.0)
        # scale by e^{-alpha} so large alpha does not overflow (cancels in the ratio)
        f = np.sin(phi) ** 2 * np.exp(-alpha[..., None] * (np.cos(phi) + 1.0))
        return 0.5 * upper * (f * w).sum(axis=-1)

    num = integral(np.arccos(-a))
    den = integral(np.full_like(a, math.pi))
    return num / den
