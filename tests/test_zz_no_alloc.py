"""The plaquette entry point for callers that cannot allocate device memory
(mc_su2_plaquette_noalloc): no context, no workspace, partial sums in a fixed
array inside libmc.so.  It must agree with the context-based measurement
(mc_measure) on the same links, on two calls in a row -- the second call
reuses the scratch the first one left behind -- on lattices from a few CTAs up
to exactly the largest the fixed scratch serves, and refuse a lattice one site
larger.  Kept in a file of its own, collected after every other test."""
import numpy as np
import pytest

import paper_0903_3053_gb300 as mc

pytestmark = pytest.mark.gpu
TOL = 1e-6  # the plaquette tolerance of the other SU(2) tests
MAX_SITES = 4194304  # the fixed scratch: 16384 CTAs of 256 sites


def _links(L, seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(int(np.prod(L)), 4, 4)).astype(np.float32)
    return q / np.linalg.norm(q, axis=2, keepdims=True)


def _check_against_context(L, seeds):
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for seed in seeds:  # consecutive calls share the scratch
        q = _links(L, seed)
        b = mc.Batch([mc.su2(L, 2.0, seed=seed)], series_capacity=4)
        b.set_config(0, q)
        want = b.measure(0)
        b.close()
        links = torch.from_numpy(q).cuda()
        mc.mc.su2_plaquette_noalloc(links, L, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - want["P"]) <= TOL, (L, seed, got, want)
        assert abs(got[1] - want["Ps"]) <= TOL, (L, seed, got, want)
        assert abs(got[2] - want["Pt"]) <= TOL, (L, seed, got, want)
        del links


def test_noalloc_plaquette_matches_context_measurement():
    _check_against_context((8, 6, 4, 6), (1, 2))


def test_noalloc_plaquette_many_blocks():
    """24^4: 1296 CTAs, so the final pass's strided loop runs over more
    partials than it has threads."""
    _check_against_context((24, 24, 24, 24), (3, 4))


def test_noalloc_plaquette_at_the_size_limit():
    """Exactly the largest lattice the scratch serves (32^3 x 128, 16384 CTAs)."""
    L = (128, 32, 32, 32)
    assert int(np.prod(L)) == MAX_SITES
    _check_against_context(L, (5, 6))


def test_noalloc_rejects_lattices_beyond_its_scratch():
    """One more row than the limit, with a correctly sized link buffer, so the
    refusal comes from the library's own size check and nothing can be read
    out of bounds even if that check were missing."""
    import torch
    L = (2, 2, 2, MAX_SITES // 8 + 1)
    links = torch.zeros(16 * int(np.prod(L)), dtype=torch.float32, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(mc.MCError, match="more than the fixed scratch"):
        mc.mc.su2_plaquette_noalloc(links, L, out)


def test_noalloc_wrapper_rejects_mismatched_buffers():
    import torch
    L = (4, 4, 4, 4)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    good = torch.zeros(16 * 256, dtype=torch.float32, device="cuda")
    for links, o in ((good[:-16], out), (good.double(), out), (good.cpu(), out), (good, out.float()),
                     (good, out[:2])):
        with pytest.raises(ValueError):
            mc.mc.su2_plaquette_noalloc(links, L, o)
