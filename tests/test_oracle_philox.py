"""Pins of the oracle's Philox4x32-10 against things other than itself:
published known-answer vectors and an independent implementation (the header-only
engine shipped in PyTorch's C++ headers), compiled and run on the host."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from conftest import ROOT

KAT = os.path.join(ROOT, "tests", "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(KAT):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_known_answer_vectors(orc):
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = orc.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == want


_CPP = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char** argv) {
  unsigned long long seed = strtoull(argv[1], 0, 0);
  unsigned long long sub = strtoull(argv[2], 0, 0);
  unsigned long long off = strtoull(argv[3], 0, 0);
  at::Philox4_32 eng(seed, sub, off);
  for (int i = 0; i < 8; ++i) printf("%u\n", eng());
  return 0;
}
"""


def test_against_independent_implementation(orc):
    """PyTorch's at::Philox4_32 keys with (seed lo, seed hi) and counts with
    (offset lo, offset hi, subsequence lo, subsequence hi); its first four
    outputs are the block at that counter and the next four the block at
    offset + 1."""
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PyTorch C++ headers not installed")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.cpp")
        exe = os.path.join(d, "p")
        open(src, "w").write(_CPP)
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", inc, src, "-o", exe])
        rng = np.random.default_rng(7)
        for _ in range(6):
            seed = int(rng.integers(0, 2**63))
            sub = int(rng.integers(0, 2**63))
            off = int(rng.integers(0, 2**40))
            out = subprocess.check_output([exe, str(seed), str(sub), str(off)]).decode().split()
            got = [int(v) for v in out]
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for blk in range(2):
                o = off + blk
                ctr = [o & 0xFFFFFFFF, o >> 32, sub & 0xFFFFFFFF, sub >> 32]
                want = [int(v) for v in orc.philox4x32_10(ctr, key)]
                assert got[4 * blk: 4 * blk + 4] == want


def test_output_is_uniform(orc):
    """Chi-square of the top byte over a few thousand blocks (catches a stuck or
    truncated word)."""
    words = np.concatenate([orc.philox4x32_10([i, 3, 5, 7], [11, 13]) for i in range(4096)])
    counts = np.bincount((words >> 24).astype(np.int64), minlength=256)
    exp = len(words) / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 360  # 255 dof, p ~ 1e-5
