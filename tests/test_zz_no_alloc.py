"""The plaquette entry point for callers that cannot allocate device memory
(mc_su2_plaquette_noalloc): no context, no workspace, partial sums in a fixed
array inside libmc.so.  It must agree with the context-based measurement
(mc_measure) on the same links, on two calls in a row -- the second call
reuses the scratch the first one left behind -- and refuse lattices larger than
its fixed scratch.  Kept in a file of its own, collected after every other
test."""
import numpy as np
import pytest

import paper_0903_3053_gb300 as mc

pytestmark = pytest.mark.gpu
TOL = 1e-6  # the plaquette tolerance of the other SU(2) tests


def _links(L, seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(int(np.prod(L)), 4, 4))
    return (q / np.linalg.norm(q, axis=2, keepdims=True)).astype(np.float32)


def test_noalloc_plaquette_matches_context_measurement():
    import torch
    L = (8, 6, 4, 6)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for seed in (1, 2):  # two calls in a row
        q = _links(L, seed)
        b = mc.Batch([mc.su2(L, 2.0, seed=seed)])
        b.set_config(0, q)
        want = b.measure(0)
        b.close()
        links = torch.from_numpy(q).cuda()
        mc.mc.su2_plaquette_noalloc(links, L, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - want["P"]) <= TOL
        assert abs(got[1] - want["Ps"]) <= TOL
        assert abs(got[2] - want["Pt"]) <= TOL


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    links = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(mc.MCError, match="more than the fixed scratch"):
        mc.mc.su2_plaquette_noalloc(links, (48, 48, 48, 48), out)
