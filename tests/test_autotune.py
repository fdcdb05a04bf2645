"""Host logic of the autotuner (no GPU): candidates a device cannot run are
skipped, the fastest remaining shape is chosen and left configured, and the
choice is cached per device and workload signature."""
from paper_0903_3053_gb300 import autotune, mc


class _Chain:
    kind, L = mc.MC_KIND_SU2, (16, 16, 16, 16)


class _Batch:
    layout, chains = mc.MC_LAYOUT_INT8, [_Chain()]


class _Group:
    """Stands in for mc.Group: a cluster of 16 CTAs fails as on a device that
    cannot co-schedule it."""

    def __init__(self):
        self.batches = [_Batch()]
        self.cfg = None

    def configure(self, C, threads, split):
        self.cfg = (C, threads, split)

    def sweep(self, n):
        if self.cfg[0] == 16:
            raise mc.MCError(mc.MC_ECUDA, "cluster occupancy query failed")


def test_tune_group_skips_unavailable_shapes_and_caches(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "fake-device")
    g = _Group()
    timed = []

    def fake_time(fn, reps):
        fn()
        timed.append(g.cfg)
        C, threads, split = g.cfg
        return 100.0 / (C * threads) + (0.01 if split == 0.0 else 0.0)  # the larger shape is faster

    monkeypatch.setattr(autotune, "_time", fake_time)
    choice = autotune.tune_group(g, n_sweeps=2, reps=1)
    assert (choice["cluster"], choice["threads"], choice["split"]) == (8, 256, -1.0)
    assert not choice["cached"]
    assert all(cfg[0] != 16 for cfg in timed)  # the failing shape was never timed
    assert g.cfg == (8, 256, -1.0)             # left configured with the choice
    g.cfg = None
    again = autotune.tune_group(g, n_sweeps=2, reps=1)
    assert again["cached"] and g.cfg == (8, 256, -1.0)
