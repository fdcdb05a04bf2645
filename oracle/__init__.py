"""CPU oracle for the checkerboard local-update sweep of Demchik & Strelchenko,
"Monte Carlo simulations on Graphics Processing Units" (arXiv:0903.3053).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library in ``paper_0903_3053_gb300``
and never imports it.

``mc_oracle.c`` holds the method itself (Philox4x32-10, Ising Metropolis of
Eq. (1) / Sec. 2.3, SU(2) heat-bath of Eqs. (2)-(7) / Sec. 2.4) in plain FP64 C;
this module compiles it with gcc on first use and wraps it for NumPy arrays.
``exact`` holds closed forms that pin the oracle; ``van`` the FP64 masked
autoregressive network of the learned proposal.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "mc_oracle.c")
_lock = threading.Lock()
_lib = None

HB_FAILED = 255


def build(force: bool = False) -> str:
    """Compile mc_oracle.c into oracle/_build/liboracle.so (plain gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _u32p():
    return ctypes.POINTER(ctypes.c_uint32)


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            c = ctypes
            P = c.c_void_p
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_philox_words.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, c.c_long, P]
            L.orc_ising_thresholds.argtypes = [c.c_double, P]
            L.orc_ising_init.argtypes = [P, c.c_int, c.c_int, c.c_uint64, c.c_uint32, c.c_int]
            L.orc_ising_sweep.argtypes = [P, c.c_int, c.c_int, P, c.c_uint64, c.c_uint32, c.c_uint32]
            L.orc_ising_observe.argtypes = [P, c.c_int, c.c_int, P, P]
            L.orc_ising_run.argtypes = [P, c.c_int, c.c_int, c.c_double, c.c_uint64, c.c_uint32, c.c_uint32,
                                        c.c_int, P, P]
            L.orc_su2_init.argtypes = [P, P, c.c_uint64, c.c_uint32, c.c_int]
            L.orc_su2_sweep.argtypes = [P, P, c.c_double, c.c_uint64, c.c_uint32, c.c_uint32, P, P, c.c_double,
                                        P, P]
            L.orc_su2_sweep.restype = c.c_long
            L.orc_su2_plaquette.argtypes = [P, P, P]
            L.orc_su2_overrelax.argtypes = [P, P]
            L.orc_su2_polyakov.argtypes = [P, P]
            L.orc_su2_polyakov.restype = c.c_double
            L.orc_su2_action.argtypes = [P, P, c.c_double]
            L.orc_su2_action.restype = c.c_double
            L.orc_su2_staple.argtypes = [P, P, c.c_long, c.c_int, P]
            L.orc_su2_sample_a0.argtypes = [c.c_double, c.c_uint64, c.c_long, P, P]
            L.orc_su2_mul.argtypes = [P, P, P]
            L.orc_ising_check_sites.argtypes = [P, P, c.c_int, c.c_int, c.c_double, c.c_uint64, c.c_uint32,
                                                c.c_uint32, P, c.c_long, P]
            L.orc_su2_check_links.argtypes = [P, P, P, c.c_double, c.c_uint64, c.c_uint32, c.c_uint32, P, c.c_long,
                                              P, c.c_double, P, P, P]
            L.orc_su2_check_links.restype = c.c_long
            L.orc_su2_nlinks.argtypes = [P]
            L.orc_su2_nlinks.restype = c.c_long
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------- Philox
def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 uint32 counter words, 2 uint32 key words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_words(seed: int, c1: int, c2: int, c3: int, n: int) -> np.ndarray:
    """n consecutive words of one stream: word j is word j & 3 of the block
    with counter (j >> 2, c1, c2, c3), key (seed low, seed high)."""
    out = np.zeros(n, dtype=np.uint32)
    lib().orc_philox_words(seed & (2**64 - 1), c1 & 0xFFFFFFFF, c2 & 0xFFFFFFFF, c3 & 0xFFFFFFFF, int(n), _ptr(out))
    return out


def uniform01(r) -> np.ndarray:
    """Random words -> (0, 1]: ((r >> 8) + 1) 2^-24, the paper's 24-bit
    resolution (Sec. 2.2) shifted off zero."""
    r = np.asarray(r, dtype=np.uint32)
    return ((r >> 8).astype(np.float64) + 1.0) * 2.0 ** -24


# --------------------------------------------------------------------------- Ising
def ising_thresholds(beta: float) -> np.ndarray:
    """[T(dE=4), T(dE=8)] = floor(exp(-beta dE) 2^32), clamped to 2^32 - 1."""
    out = np.zeros(2, dtype=np.uint32)
    lib().orc_ising_thresholds(float(beta), _ptr(out))
    return out


def ising_init(L, seed: int, chain: int = 0, hot: bool = True) -> np.ndarray:
    """Initial spins, int8 array of shape (Ly, Lx); L = (Lx, Ly) or an int."""
    Lx, Ly = (L, L) if np.isscalar(L) else L
    s = np.zeros((Ly, Lx), dtype=np.int8)
    lib().orc_ising_init(_ptr(s), Lx, Ly, seed, chain, int(bool(hot)))
    return s


def ising_run(s: np.ndarray, beta: float, seed: int, chain: int, first_sweep: int, n: int,
              record: bool = True):
    """Advance spins `s` (modified in place) by n Metropolis sweeps numbered
    first_sweep..first_sweep+n-1; returns the (E, M) series when record."""
    Ly, Lx = s.shape
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"]
    if record:
        E = np.zeros(n, dtype=np.int64)
        M = np.zeros(n, dtype=np.int64)
        lib().orc_ising_run(_ptr(s), Lx, Ly, float(beta), seed, chain, first_sweep, n, _ptr(E), _ptr(M))
        return E, M
    lib().orc_ising_run(_ptr(s), Lx, Ly, float(beta), seed, chain, first_sweep, n, None, None)
    return None


def ising_observe(s: np.ndarray):
    Ly, Lx = s.shape
    E = np.zeros(1, dtype=np.int64)
    M = np.zeros(1, dtype=np.int64)
    lib().orc_ising_observe(_ptr(np.ascontiguousarray(s)), Lx, Ly, _ptr(E), _ptr(M))
    return int(E[0]), int(M[0])


# --------------------------------------------------------------------------- SU(2)
def _dims(L):
    d = np.ascontiguousarray(L, dtype=np.int32)
    assert d.shape == (4,)
    return d


def su2_init(L, seed: int, chain: int = 0, hot: bool = True) -> np.ndarray:
    """Links as quaternions (U0, U1, U2, U3) of Eq. (4), shape (nsites, 4, 4),
    site index s = x1 + L1 (x2 + L2 (x3 + L3 x0)), mu = 0 time."""
    d = _dims(L)
    ns = int(np.prod(d))
    q = np.zeros((ns, 4, 4), dtype=np.float64)
    lib().orc_su2_init(_ptr(q), _ptr(d), seed, chain, int(bool(hot)))
    return q


def su2_sweep(q: np.ndarray, L, beta: float, seed: int, chain: int, sweep: int,
              forced_tries: np.ndarray | None = None, eps: float = 1e-6):
    """One heat-bath sweep in place.  Returns (tries[nsites, 4] uint8, failures,
    n_near, n_bad); see orc_su2_sweep for forced_tries."""
    d = _dims(L)
    assert q.dtype == np.float64 and q.flags["C_CONTIGUOUS"]
    tries = np.zeros(q.shape[:2], dtype=np.uint8)
    near = ctypes.c_long(0)
    bad = ctypes.c_long(0)
    f = None
    if forced_tries is not None:
        forced_tries = np.ascontiguousarray(forced_tries, dtype=np.uint8).reshape(q.shape[:2])
        f = _ptr(forced_tries)
    fails = lib().orc_su2_sweep(_ptr(q), _ptr(d), float(beta), seed, chain, sweep, _ptr(tries), f, float(eps),
                                ctypes.byref(near), ctypes.byref(bad))
    return tries, int(fails), int(near.value), int(bad.value)


def su2_overrelax(q: np.ndarray, L) -> None:
    """One overrelaxation sweep in place (orc_su2_overrelax)."""
    d = _dims(L)
    assert q.dtype == np.float64 and q.flags["C_CONTIGUOUS"]
    lib().orc_su2_overrelax(_ptr(q), _ptr(d))


def su2_polyakov(q: np.ndarray, L) -> float:
    """Volume-averaged Polyakov loop (1/2) Tr prod_t U_0(t, x) (FP64)."""
    d = _dims(L)
    return float(lib().orc_su2_polyakov(_ptr(np.ascontiguousarray(q, dtype=np.float64)), _ptr(d)))


def su2_plaquette(q: np.ndarray, L) -> np.ndarray:
    """[P, P_spatial, P_temporal] (FP64)."""
    d = _dims(L)
    out = np.zeros(3, dtype=np.float64)
    lib().orc_su2_plaquette(_ptr(np.ascontiguousarray(q, dtype=np.float64)), _ptr(d), _ptr(out))
    return out


def su2_action(q: np.ndarray, L, beta: float) -> float:
    d = _dims(L)
    return float(lib().orc_su2_action(_ptr(np.ascontiguousarray(q, dtype=np.float64)), _ptr(d), float(beta)))


def su2_staple(q: np.ndarray, L, s: int, mu: int) -> np.ndarray:
    d = _dims(L)
    out = np.zeros(4, dtype=np.float64)
    lib().orc_su2_staple(_ptr(np.ascontiguousarray(q, dtype=np.float64)), _ptr(d), int(s), int(mu), _ptr(out))
    return out


def su2_sample_a0(alpha: float, seed: int, n: int):
    out = np.zeros(n, dtype=np.float64)
    tries = np.zeros(n, dtype=np.uint8)
    lib().orc_su2_sample_a0(float(alpha), seed, int(n), _ptr(out), _ptr(tries))
    return out, tries


def su2_mul(a, b) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(4, dtype=np.float64)
    lib().orc_su2_mul(_ptr(a), _ptr(b), _ptr(out))
    return out


# --------------------------------------------------------------------------- sampled checks
def ising_check_sites(pre: np.ndarray, post: np.ndarray, beta: float, seed: int, chain: int, sweep: int,
                      sites) -> np.ndarray:
    """Expected post-sweep spins of the listed sites (flat indices y*Lx + x)."""
    Ly, Lx = pre.shape
    pre = np.ascontiguousarray(pre, dtype=np.int8)
    post = np.ascontiguousarray(post, dtype=np.int8)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.zeros(len(sites), dtype=np.int8)
    lib().orc_ising_check_sites(_ptr(pre), _ptr(post), Lx, Ly, float(beta), seed, chain, sweep, _ptr(sites),
                                len(sites), _ptr(out))
    return out


def su2_check_links(pre: np.ndarray, post: np.ndarray, L, beta: float, seed: int, chain: int, sweep: int, links,
                    forced_tries=None, eps: float = 1e-6):
    """Expected post-sweep links (flat indices 4 s + mu) recomputed in FP64 from
    the lattice each update saw.  Returns (values[n, 4], failures, near, bad)."""
    d = _dims(L)
    pre = np.ascontiguousarray(pre, dtype=np.float64)
    post = np.ascontiguousarray(post, dtype=np.float64)
    links = np.ascontiguousarray(links, dtype=np.int64)
    out = np.zeros((len(links), 4), dtype=np.float64)
    f = None
    if forced_tries is not None:
        forced_tries = np.ascontiguousarray(forced_tries, dtype=np.uint8)
        f = _ptr(forced_tries)
    near = ctypes.c_long(0)
    bad = ctypes.c_long(0)
    fails = lib().orc_su2_check_links(_ptr(pre), _ptr(post), _ptr(d), float(beta), seed, chain, sweep, _ptr(links),
                                      len(links), f, float(eps), _ptr(out), ctypes.byref(near), ctypes.byref(bad))
    return out, int(fails), int(near.value), int(bad.value)
