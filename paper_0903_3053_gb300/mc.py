"""Thin ctypes binding of libmc.so (include/mc.h).

Argument marshalling only: every step of the sweep runs in the library's CUDA
kernels.  PyTorch supplies device memory (the workspace tensor) and the CUDA
stream.  There is no CPU fallback: if libmc.so cannot be loaded or no GPU is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MC_OK, MC_EINVAL, MC_ENOMEM, MC_ECUDA, MC_ETIMEOUT, MC_ESTATE, MC_EDEVICE = 0, -1, -2, -3, -4, -5, -6
MC_COLD, MC_HOT = 0, 1
MC_KIND_ISING, MC_KIND_SU2 = 1, 2
MC_LAYOUT_INT8, MC_LAYOUT_MSC32 = 0, 1
MC_FMT_INT8, MC_FMT_BITS, MC_FMT_F32, MC_FMT_NATIVE = 0, 1, 2, 3
MC_MODE_AUTO, MC_MODE_GRID, MC_MODE_RESIDENT = 0, 1, 2

#: every symbol include/mc.h declares (checked by the ABI test)
EXPORTS = [
    "mc_workspace_bytes", "mc_batch_init", "mc_ising_init", "mc_su2_init", "mc_sweep", "mc_set_mode", "mc_sync",
    "mc_measure", "mc_read_series", "mc_get_config", "mc_set_config", "mc_config_bytes", "mc_get_sweep",
    "mc_set_sweep", "mc_su2_record_tries", "mc_su2_get_tries", "mc_su2_failed_updates", "mc_su2_set_overrelax",
    "mc_su2_get_overrelax", "mc_su2_polyakov", "mc_destroy",
    "mc_last_error", "mc_version", "mc_profile_enable", "mc_profile_read", "mc_su2_plaquette_noalloc",
    "mc_philox_rate",
    "mc_group_workspace_bytes", "mc_group_create", "mc_group_configure", "mc_group_sweep", "mc_group_schedule",
    "mc_group_destroy",
]


class mc_chain_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("L", ctypes.c_int32 * 4), ("beta", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("chain_id", ctypes.c_uint32), ("start", ctypes.c_int32)]


class mc_record(ctypes.Structure):
    _fields_ = [("sweep", ctypes.c_int64), ("E", ctypes.c_int64), ("M", ctypes.c_int64), ("P", ctypes.c_double),
                ("Ps", ctypes.c_double), ("Pt", ctypes.c_double)]


RECORD_DTYPE = np.dtype([("sweep", "<i8"), ("E", "<i8"), ("M", "<i8"), ("P", "<f8"), ("Ps", "<f8"), ("Pt", "<f8")])
assert ctypes.sizeof(mc_chain_desc) == 48 and ctypes.sizeof(mc_record) == 48 == RECORD_DTYPE.itemsize


class MCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libmc status {status}: {msg}")
        self.status = status


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libmc.so (building it with nvcc first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libmc.so not found at {_build.LIB}; run paper_0903_3053_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    c, P = ctypes, ctypes.c_void_p
    st = c.c_int
    sig = {
        "mc_workspace_bytes": (c.c_size_t, [c.c_int32, P, c.c_int32, c.c_int64]),
        "mc_batch_init": (st, [P, c.c_int32, P, c.c_int32, c.c_int64, P, c.c_size_t, P]),
        "mc_ising_init": (st, [P, P, c.c_double, c.c_uint64, c.c_int32, c.c_int32, c.c_int64, P, c.c_size_t, P]),
        "mc_su2_init": (st, [P, P, c.c_double, c.c_uint64, c.c_int32, c.c_int64, P, c.c_size_t, P]),
        "mc_sweep": (st, [P, c.c_int64, c.c_int32]),
        "mc_set_mode": (st, [P, c.c_int32, c.c_int32]),
        "mc_sync": (st, [P]),
        "mc_measure": (st, [P, c.c_int32, P]),
        "mc_read_series": (st, [P, P, c.c_int64, P]),
        "mc_get_config": (st, [P, c.c_int32, c.c_int32, P, c.c_int32]),
        "mc_set_config": (st, [P, c.c_int32, c.c_int32, P, c.c_int32]),
        "mc_config_bytes": (c.c_size_t, [P, c.c_int32, c.c_int32]),
        "mc_get_sweep": (st, [P, P]),
        "mc_set_sweep": (st, [P, c.c_int64]),
        "mc_su2_record_tries": (st, [P, c.c_int32]),
        "mc_su2_get_tries": (st, [P, c.c_int32, P]),
        "mc_su2_failed_updates": (st, [P, P]),
        "mc_su2_set_overrelax": (st, [P, c.c_int32]),
        "mc_su2_get_overrelax": (st, [P, P]),
        "mc_su2_polyakov": (st, [P, c.c_int32, P]),
        "mc_destroy": (st, [P]),
        "mc_profile_enable": (st, [P, c.c_int32]),
        "mc_profile_read": (st, [P, P, P]),
        "mc_su2_plaquette_noalloc": (st, [P, P, P, P]),
        "mc_philox_rate": (st, [c.c_int32, c.c_int32, c.c_uint32, c.c_uint64, P, P]),
        "mc_group_workspace_bytes": (c.c_size_t, [c.c_int32, P]),
        "mc_group_create": (st, [P, c.c_int32, P, P, c.c_size_t, P]),
        "mc_group_configure": (st, [P, c.c_int32, c.c_int32, c.c_double]),
        "mc_group_sweep": (st, [P, c.c_int64, c.c_int32]),
        "mc_group_schedule": (st, [P, P, P]),
        "mc_group_destroy": (st, [P]),
        "mc_last_error": (c.c_char_p, []),
        "mc_version": (c.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != MC_OK:
        raise MCError(status, load().mc_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libmc needs a CUDA GPU; no CPU fallback exists")
    return torch


@dataclass
class Chain:
    """One Markov chain.  Ising: L = (Lx, Ly); SU(2): L = (L0, L1, L2, L3), mu = 0 time."""
    kind: int
    L: tuple
    beta: float
    seed: int
    chain_id: int = 0
    start: int = MC_HOT

    def desc(self) -> mc_chain_desc:
        d = mc_chain_desc()
        d.kind = self.kind
        L = list(self.L) + [1] * (4 - len(self.L))
        for i in range(4):
            d.L[i] = int(L[i])
        d.beta = float(self.beta)
        d.seed = int(self.seed) & 0xFFFFFFFFFFFFFFFF
        d.chain_id = int(self.chain_id) & 0xFFFFFFFF
        d.start = int(self.start)
        return d


def ising(L, beta, seed, chain_id=0, hot=True) -> Chain:
    L = (L, L) if np.isscalar(L) else tuple(L)
    return Chain(MC_KIND_ISING, L, beta, seed, chain_id, MC_HOT if hot else MC_COLD)


def su2(L, beta, seed, chain_id=0, hot=True) -> Chain:
    L = (L,) * 4 if np.isscalar(L) else tuple(L)
    return Chain(MC_KIND_SU2, L, beta, seed, chain_id, MC_HOT if hot else MC_COLD)


def mc_workspace_bytes(chains, layout=MC_LAYOUT_INT8, series_capacity=1024) -> int:
    arr = (mc_chain_desc * len(chains))(*[c.desc() for c in chains])
    n = load().mc_workspace_bytes(len(chains), arr, layout, series_capacity)
    if n == 0:
        raise MCError(MC_EINVAL, load().mc_last_error().decode())
    return int(n)


def philox_rate(blocks: int, threads: int, iters: int, seed: int, out, stream=None):
    """Launch the Philox multiply-ceiling kernel (see include/mc.h) into the
    uint32/int32 CUDA tensor `out` (blocks x threads entries), async."""
    torch = _torch()
    if not (out.is_cuda and out.dtype in (torch.int32,) and out.is_contiguous() and out.numel() >= blocks * threads):
        raise ValueError("philox_rate: out must be a contiguous int32 CUDA tensor of blocks x threads entries")
    st = stream if stream is not None else torch.cuda.current_stream(out.device)
    with torch.cuda.device(out.device):
        _check(load().mc_philox_rate(int(blocks), int(threads), int(iters) & 0xFFFFFFFF, int(seed) & (2**64 - 1),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream)))


def su2_plaquette_noalloc(links, L, out, stream=None):
    """{P, P_s, P_t} of a canonical-order float32 CUDA tensor `links` (shape
    (N, 4, 4)) into the float64 CUDA tensor `out` (3 entries), for callers
    that cannot let the library allocate: no context, no workspace, nothing
    allocated (see include/mc.h for the size limit and the shared scratch)."""
    torch = _torch()
    dims = [int(v) for v in L]
    if len(dims) != 4 or min(dims) < 1:
        raise ValueError(f"su2_plaquette_noalloc: L must be four positive extents, got {L}")
    if not (links.is_cuda and links.dtype == torch.float32 and links.is_contiguous()):
        raise ValueError("su2_plaquette_noalloc: links must be a contiguous float32 CUDA tensor")
    if links.numel() != 16 * int(np.prod(dims)):
        raise ValueError(f"su2_plaquette_noalloc: links holds {links.numel()} floats, the lattice {dims} needs "
                         f"{16 * int(np.prod(dims))}")
    if not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() >= 3):
        raise ValueError("su2_plaquette_noalloc: out must be a contiguous float64 CUDA tensor of >= 3 entries")
    if out.device != links.device:
        raise ValueError("su2_plaquette_noalloc: links and out must be on the same device")
    st = stream if stream is not None else torch.cuda.current_stream(links.device)
    if st.device != links.device:
        raise ValueError("su2_plaquette_noalloc: the stream must belong to the links' device")
    # the C side launches on, and takes the scratch of, the current device
    with torch.cuda.device(links.device):
        _check(load().mc_su2_plaquette_noalloc(ctypes.c_void_p(links.data_ptr()), (ctypes.c_int32 * 4)(*dims),
                                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream)))


class Batch:
    """A batch of chains of one kind, advanced together on one CUDA stream."""

    def __init__(self, chains, layout=MC_LAYOUT_INT8, series_capacity=1024, stream=None, device=None):
        torch = _torch()
        L = load()
        self.chains = list(chains)
        self.kind = self.chains[0].kind
        self.layout = layout
        self.cap = int(series_capacity)
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        arr = (mc_chain_desc * len(self.chains))(*[c.desc() for c in self.chains])
        nbytes = L.mc_workspace_bytes(len(self.chains), arr, layout, self.cap)
        if nbytes == 0:
            raise MCError(MC_EINVAL, L.mc_last_error().decode())
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        if self.workspace.data_ptr() % 256:
            raise RuntimeError("workspace tensor is not 256-byte aligned")
        self._ctx = ctypes.c_void_p()
        _check(L.mc_batch_init(ctypes.byref(self._ctx), len(self.chains), arr, layout, self.cap,
                               ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                               ctypes.c_void_p(self.stream.cuda_stream)))

    # -- sweeping ---------------------------------------------------------------
    def sweep(self, n: int, measure_every: int = 0):
        _check(load().mc_sweep(self._ctx, int(n), int(measure_every)))

    def set_mode(self, mode: int, threads_per_block: int = 0):
        _check(load().mc_set_mode(self._ctx, int(mode), int(threads_per_block)))

    def sync(self):
        _check(load().mc_sync(self._ctx))

    @property
    def sweeps_done(self) -> int:
        v = ctypes.c_int64()
        _check(load().mc_get_sweep(self._ctx, ctypes.byref(v)))
        return int(v.value)

    @sweeps_done.setter
    def sweeps_done(self, value: int):
        _check(load().mc_set_sweep(self._ctx, int(value)))

    # -- observables --------------------------------------------------------------
    def measure(self, chain: int = 0) -> dict:
        r = mc_record()
        _check(load().mc_measure(self._ctx, int(chain), ctypes.byref(r)))
        return {"sweep": r.sweep, "E": r.E, "M": r.M, "P": r.P, "Ps": r.Ps, "Pt": r.Pt}

    def read_series(self, max_per_chain: int | None = None) -> np.ndarray:
        """Unread records as a structured array of shape (n_chains, n)."""
        m = self.cap if max_per_chain is None else int(max_per_chain)
        out = np.zeros((len(self.chains), m), dtype=RECORD_DTYPE)
        n = ctypes.c_int64()
        _check(load().mc_read_series(self._ctx, ctypes.c_void_p(out.ctypes.data), m, ctypes.byref(n)))
        return out[:, : n.value].copy()

    # -- configurations ---------------------------------------------------------------
    def config_bytes(self, chain: int, fmt: int) -> int:
        return int(load().mc_config_bytes(self._ctx, int(chain), int(fmt)))

    def _shape(self, chain: int, fmt: int):
        c = self.chains[chain]
        if fmt == MC_FMT_NATIVE:  # the context's own storage (layouts in include/mc.h)
            if self.kind == MC_KIND_SU2:
                return (2, 4, int(np.prod(c.L)) // 2, 4), np.float32
            Lx, Ly = c.L[0], c.L[1]
            if self.layout == MC_LAYOUT_INT8:
                return (Ly, Lx), np.int8
            return (2, Ly, Lx // 64), np.uint32
        if self.kind == MC_KIND_ISING:
            Lx, Ly = c.L[0], c.L[1]
            return ((Ly, Lx), np.int8) if fmt == MC_FMT_INT8 else ((Ly, Lx // 32), np.uint32)
        n = int(np.prod(c.L))
        return (n, 4, 4), np.float32

    def _check_tensor(self, chain: int, fmt: int, t):
        shape, dt = self._shape(chain, fmt)
        need = int(np.prod(shape)) * np.dtype(dt).itemsize
        if not t.is_contiguous() or t.numel() * t.element_size() < need:
            raise ValueError(f"tensor must be contiguous and hold at least {need} bytes")

    def get_config(self, chain: int = 0, fmt: int | None = None) -> np.ndarray:
        fmt = self._default_fmt() if fmt is None else fmt
        shape, dt = self._shape(chain, fmt)
        out = np.zeros(shape, dtype=dt)
        _check(load().mc_get_config(self._ctx, int(chain), int(fmt), ctypes.c_void_p(out.ctypes.data), 0))
        return out

    def set_config(self, chain: int, data: np.ndarray, fmt: int | None = None):
        fmt = self._default_fmt() if fmt is None else fmt
        shape, dt = self._shape(chain, fmt)
        a = np.ascontiguousarray(data, dtype=dt).reshape(shape)
        _check(load().mc_set_config(self._ctx, int(chain), int(fmt), ctypes.c_void_p(a.ctypes.data), 0))
        self.sync()  # the host buffer `a` is released when this returns

    def get_config_device(self, chain: int, out_tensor, fmt: int | None = None):
        fmt = self._default_fmt() if fmt is None else fmt
        self._check_tensor(chain, fmt, out_tensor)
        _check(load().mc_get_config(self._ctx, int(chain), int(fmt), ctypes.c_void_p(out_tensor.data_ptr()), 1))

    def set_config_device(self, chain: int, tensor, fmt: int | None = None):
        fmt = self._default_fmt() if fmt is None else fmt
        self._check_tensor(chain, fmt, tensor)
        _check(load().mc_set_config(self._ctx, int(chain), int(fmt), ctypes.c_void_p(tensor.data_ptr()), 1))

    def set_config_host_async(self, chain: int, host_tensor, fmt: int | None = None):
        """Asynchronous upload from a page-locked host tensor (keep it unchanged
        until the next synchronising call)."""
        fmt = self._default_fmt() if fmt is None else fmt
        self._check_tensor(chain, fmt, host_tensor)
        _check(load().mc_set_config(self._ctx, int(chain), int(fmt), ctypes.c_void_p(host_tensor.data_ptr()), 0))

    def get_config_host(self, chain: int, host_tensor, fmt: int | None = None):
        """Synchronous download into a caller-owned host tensor (page-locked
        memory is written in place by the conversion kernel)."""
        fmt = self._default_fmt() if fmt is None else fmt
        self._check_tensor(chain, fmt, host_tensor)
        _check(load().mc_get_config(self._ctx, int(chain), int(fmt), ctypes.c_void_p(host_tensor.data_ptr()), 0))

    def _default_fmt(self):
        return MC_FMT_INT8 if self.kind == MC_KIND_ISING else MC_FMT_F32

    # -- SU(2) diagnostics --------------------------------------------------------------
    def record_tries(self, enable: bool = True):
        _check(load().mc_su2_record_tries(self._ctx, int(bool(enable))))

    def get_tries(self, chain: int = 0) -> np.ndarray:
        n = int(np.prod(self.chains[chain].L))
        out = np.zeros((n, 4), dtype=np.uint8)
        _check(load().mc_su2_get_tries(self._ctx, int(chain), ctypes.c_void_p(out.ctypes.data)))
        return out

    def failed_updates(self) -> int:
        v = ctypes.c_int64()
        _check(load().mc_su2_failed_updates(self._ctx, ctypes.byref(v)))
        return int(v.value)

    def polyakov(self, chain: int = 0) -> float:
        """SU(2): volume-averaged Polyakov loop of the chain's current links."""
        v = ctypes.c_double()
        _check(load().mc_su2_polyakov(self._ctx, int(chain), ctypes.byref(v)))
        return float(v.value)

    def set_overrelax(self, n_or: int):
        """SU(2): each sweep becomes one heat-bath sweep plus n_or overrelaxation sweeps."""
        _check(load().mc_su2_set_overrelax(self._ctx, int(n_or)))

    def overrelax(self) -> int:
        v = ctypes.c_int32()
        _check(load().mc_su2_get_overrelax(self._ctx, ctypes.byref(v)))
        return int(v.value)

    # -- kernel timing --------------------------------------------------------------
    def profile(self, enable: bool = True):
        _check(load().mc_profile_enable(self._ctx, int(bool(enable))))

    def profile_read(self):
        """(launches, summed duration in ms) of the sweep kernels since the last read."""
        n = ctypes.c_int64()
        t = ctypes.c_double()
        _check(load().mc_profile_read(self._ctx, ctypes.byref(n), ctypes.byref(t)))
        return int(n.value), float(t.value)

    # -- lifetime -----------------------------------------------------------------
    def close(self):
        if self._ctx:
            st = load().mc_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()
            _check(st)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Group:
    """Chains of several Batches advanced by one persistent launch per call."""

    def __init__(self, batches):
        torch = _torch()
        L = load()
        self.batches = list(batches)
        self.stream = self.batches[0].stream
        for b in self.batches:
            if b.stream.cuda_stream != self.stream.cuda_stream:
                raise ValueError("every batch of a group must use the same CUDA stream")
        arr = (ctypes.c_void_p * len(self.batches))(*[b._ctx.value for b in self.batches])
        self._arr = arr
        nbytes = L.mc_group_workspace_bytes(len(self.batches), arr)
        if nbytes == 0:
            raise MCError(MC_EINVAL, L.mc_last_error().decode())
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.batches[0].device)
        self._g = ctypes.c_void_p()
        _check(L.mc_group_create(ctypes.byref(self._g), len(self.batches), arr,
                                 ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                 ctypes.c_void_p(self.stream.cuda_stream)))

    def configure(self, cluster_size: int = 0, threads_per_block: int = 0, split_cost: float = -1.0):
        _check(load().mc_group_configure(self._g, int(cluster_size), int(threads_per_block), float(split_cost)))

    def sweep(self, n: int, measure_every: int = 0):
        _check(load().mc_group_sweep(self._g, int(n), int(measure_every)))

    def schedule(self):
        nc, nr = ctypes.c_int32(), ctypes.c_int32()
        _check(load().mc_group_schedule(self._g, ctypes.byref(nc), ctypes.byref(nr)))
        return int(nc.value), int(nr.value)

    def close(self):
        if self._g:
            st = load().mc_group_destroy(self._g)
            self._g = ctypes.c_void_p()
            _check(st)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _van_sigs(L):
    c, P = ctypes, ctypes.c_void_p
    st = c.c_int
    return {
        "mc_van_param_count": (c.c_size_t, [c.c_int32]),
        "mc_van_workspace_bytes": (c.c_size_t, [c.c_int32, c.c_int32, c.c_int32]),
        "mc_van_create": (st, [P, c.c_int32, c.c_int32, c.c_int32, c.c_uint64, P, c.c_size_t, P]),
        "mc_van_set_params": (st, [P, P, c.c_size_t]),
        "mc_van_get_params": (st, [P, P, c.c_size_t, P]),
        "mc_van_get_activations": (st, [P, c.c_int32, c.c_int32, P]),
        "mc_van_log_prob": (st, [P, P, c.c_int32, c.c_int32, P]),
        "mc_van_train_step": (st, [P, P, c.c_int32, c.c_float, c.c_int32, P]),
        "mc_van_sample": (st, [P, c.c_int32, c.c_uint32, P, P, P]),
        "mc_van_mh_round": (st, [P, P, P]),
        "mc_van_set_round": (st, [P, c.c_uint32]),
        "mc_van_sync": (st, [P]),
        "mc_van_destroy": (st, [P]),
        "mc_ising_gather": (st, [P, P, c.c_int32]),
    }


VAN_EXPORTS = list(_van_sigs(None))
EXPORTS += VAN_EXPORTS


def _load_van():
    L = load()
    if not getattr(L, "_van_ready", False):
        for name, (res, args) in _van_sigs(None).items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        L._van_ready = True
    return L


def van_param_count(depth: int = 6) -> int:
    return int(_load_van().mc_van_param_count(depth))


def van_pack(params) -> np.ndarray:
    """[(W[out][in][5][5], b[out]), ...] -> the flat FP32 order of the ABI."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32).ravel()])
                           for W, b in params]).astype(np.float32)


def van_unpack(flat: np.ndarray, depth: int = 6, channels: int = 32):
    out, off = [], 0
    for l in range(depth):
        cin = 1 if l == 0 else channels
        cout = 1 if l == depth - 1 else channels
        n = cout * cin * 25
        W = flat[off:off + n].reshape(cout, cin, 5, 5)
        off += n
        b = flat[off:off + cout]
        off += cout
        out.append((W, b))
    return out


class VAN:
    """The learned proposal network (see include/mc.h)."""

    def __init__(self, L: int, batch: int, depth: int = 6, seed: int = 0, stream=None):
        torch = _torch()
        lib = _load_van()
        self.L, self.batch, self.depth = int(L), int(batch), int(depth)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nbytes = lib.mc_van_workspace_bytes(self.L, self.batch, self.depth)
        if nbytes == 0:
            raise MCError(MC_EINVAL, lib.mc_last_error().decode())
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        self._w = ctypes.c_void_p()
        _check(lib.mc_van_create(ctypes.byref(self._w), self.L, self.batch, self.depth, int(seed) & (2**64 - 1),
                                 ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                 ctypes.c_void_p(self.stream.cuda_stream)))
        self.n_params = van_param_count(self.depth)

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(_load_van().mc_van_set_params(self._w, ctypes.c_void_p(a.ctypes.data), a.size))

    def get_params(self, grads: bool = False):
        p = np.zeros(self.n_params, np.float32)
        g = np.zeros(self.n_params, np.float32) if grads else None
        _check(_load_van().mc_van_get_params(self._w, ctypes.c_void_p(p.ctypes.data), p.size,
                                             ctypes.c_void_p(g.ctypes.data) if grads else None))
        return (p, g) if grads else p

    def get_activations(self, layer: int, n: int) -> np.ndarray:
        """BF16 output of hidden layer `layer` (0 .. depth-2) of the last forward
        pass for its first n configurations, as float64 [n][L][L][32]."""
        raw = np.zeros((n, self.L, self.L, 32), dtype=np.uint16)
        _check(_load_van().mc_van_get_activations(self._w, int(layer), int(n), ctypes.c_void_p(raw.ctypes.data)))
        return (raw.astype(np.uint32) << 16).view(np.float32).astype(np.float64)

    def log_prob(self, spins, negate: bool = False):
        import torch
        out = torch.empty(spins.shape[0], dtype=torch.float64, device="cuda")
        _check(_load_van().mc_van_log_prob(self._w, ctypes.c_void_p(spins.data_ptr()), int(spins.shape[0]),
                                           int(bool(negate)), ctypes.c_void_p(out.data_ptr())))
        return out

    def train_step(self, spins, lr: float = 1e-3, apply: bool = True) -> float:
        loss = ctypes.c_double()
        _check(_load_van().mc_van_train_step(self._w, ctypes.c_void_p(spins.data_ptr()), int(spins.shape[0]),
                                             float(lr), int(bool(apply)), ctypes.byref(loss)))
        return float(loss.value)

    def sample(self, n: int, round: int = 0, ids=None):
        import torch
        out = torch.empty((n, self.L, self.L), dtype=torch.int8, device="cuda")
        lq = torch.empty(n, dtype=torch.float64, device="cuda")
        _check(_load_van().mc_van_sample(self._w, int(n), int(round) & 0xFFFFFFFF,
                                         ctypes.c_void_p(ids.data_ptr()) if ids is not None else None,
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(lq.data_ptr())))
        return out, lq

    def mh_round(self, batch: "Batch") -> int:
        acc = ctypes.c_int32()
        _check(_load_van().mc_van_mh_round(self._w, batch._ctx, ctypes.byref(acc)))
        return int(acc.value)

    def set_round(self, r: int):
        _check(_load_van().mc_van_set_round(self._w, int(r) & 0xFFFFFFFF))

    def sync(self):
        """Wait for the network's stream; raises if a bounded device wait of an
        earlier call gave up."""
        _check(_load_van().mc_van_sync(self._w))

    def close(self):
        if self._w:
            st = _load_van().mc_van_destroy(self._w)
            self._w = ctypes.c_void_p()
            _check(st)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ising_gather(batch: "Batch", out=None, back: bool = False):
    """All chains of an int8-layout Ising Batch as one [n][L][L] int8 CUDA tensor
    (or write `out` back into the chains when back=True)."""
    import torch
    if out is None:
        c = batch.chains[0]
        out = torch.empty((len(batch.chains), c.L[1], c.L[0]), dtype=torch.int8, device="cuda")
    _check(_load_van().mc_ising_gather(batch._ctx, ctypes.c_void_p(out.data_ptr()), int(bool(back))))
    return out
