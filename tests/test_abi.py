"""The C-ABI library builds, loads without a GPU, exports every symbol that
include/mc.h declares, and validates arguments on the host (no compute calls)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def mc():
    import paper_0903_3053_gb300 as p
    p.load()
    return p


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^MC_API\s+[\w\s\*]*?\b(mc_\w+)\s*\(", text, flags=re.M)
    return names


def test_every_declared_symbol_is_exported(mc):
    lib = ctypes.CDLL(mc.mc.lib_path())
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(mc.mc.EXPORTS)


def test_version(mc):
    assert b"sm_103a" in mc.load().mc_version()


@pytest.mark.parametrize("chains,layout,msg", [
    ("odd", 0, "even"),
    ("msc64", 1, "Lx % 64"),
    ("negbeta", 0, "beta"),
    ("mixed", 0, "one kind"),
])
def test_workspace_validation(mc, chains, layout, msg):
    table = {
        "odd": [mc.ising((63, 64), 0.4, 1)],
        "msc64": [mc.ising((96, 64), 0.4, 1)],
        "negbeta": [mc.ising(64, -0.1, 1)],
        "mixed": [mc.ising(64, 0.4, 1), mc.su2(4, 2.0, 1)],
    }
    with pytest.raises(mc.MCError, match=msg):
        mc.mc_workspace_bytes(table[chains], layout, 16)


def test_workspace_sizes_scale(mc):
    a = mc.mc_workspace_bytes([mc.ising(1024, 0.4, 1)], 1, 16)
    b = mc.mc_workspace_bytes([mc.ising(1024, 0.4, 1)], 0, 16)
    assert b - a >= 1024 * 1024 - 1024 * 1024 // 8 - 4096  # int8 vs 1 bit per spin
    s = mc.mc_workspace_bytes([mc.su2((4, 6, 8, 10), 2.0, 1)], 0, 16)
    assert s >= 4 * 6 * 8 * 10 * 4 * 16


def test_null_and_bad_arguments_rejected(mc):
    L = mc.load()
    assert L.mc_sweep(None, 1, 0) == mc.mc.MC_EINVAL
    assert L.mc_sync(None) == mc.mc.MC_EINVAL
    assert L.mc_destroy(None) == 0
    out = ctypes.c_void_p()
    arr = (mc.mc.mc_chain_desc * 1)(mc.ising(64, 0.4, 1).desc())
    # a host pointer is not a device workspace (caught before any kernel)
    buf = ctypes.create_string_buffer(1 << 20)
    st = L.mc_batch_init(ctypes.byref(out), 1, arr, 0, 16, ctypes.c_void_p(ctypes.addressof(buf) + 0), 1 << 20, None)
    assert st != 0


@pytest.mark.parametrize("case,msg", [
    ("empty", "n_chains"),
    ("zero_extent", "even and >= 2"),
    ("su2_odd", "even and >= 2"),
    ("nan_beta", "finite"),
    ("too_big", "2\\^31"),
    ("no_ring", "series_capacity"),
])
def test_degenerate_inputs_rejected_on_the_host(mc, case, msg):
    """Empty batches, zero or odd extents, a NaN coupling, lattices past the
    32-bit site index and an empty ring are refused before anything reaches a
    GPU."""
    args = {
        "empty": ([], 0, 16),
        "zero_extent": ([mc.ising((0, 64), 0.4, 1)], 0, 16),
        "su2_odd": ([mc.su2((4, 4, 4, 3), 2.0, 1)], 0, 16),
        "nan_beta": ([mc.ising(64, float("nan"), 1)], 0, 16),
        "too_big": ([mc.ising(1 << 17, 0.4, 1)], 1, 16),
        "no_ring": ([mc.ising(64, 0.4, 1)], 0, 0),
    }[case]
    with pytest.raises(mc.MCError, match=msg):
        mc.mc_workspace_bytes(*args)
