"""The benchmark's host-side legs without a GPU: the `config` object both arms
print, and the oracle timings of the rows outside the step on small CPU
tensors of the tiny geometry (the same code the GPU machine runs on the
ensemble's own buffers)."""
import sys

import numpy as np
import torch


def _bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench
    finally:
        sys.argv = argv
    return bench


def test_config_object_is_shared_by_both_arms():
    from synth import workload
    bench = _bench()
    w = workload("paper")
    c = bench.workload_config(w, w.n_frames, "fp32", 1)
    assert c["frames"] == 300 and c["n_tx"] == 8 and c["n_el"] == 128 and c["us"] == 2
    assert "RF 1.26 GB" in c["l2"] and "planes 4.92 GB" in c["l2"]
    assert c == bench.workload_config(w, w.n_frames, "fp32", 1)
    assert "RF 0.63 GB" in bench.workload_config(w, w.n_frames, "reduced", 1)["l2"]


def test_next_row_oracle_timings_on_cpu_tensors(tiny):
    from paper_2511_21647_gb300 import _lib as L
    bench = _bench()
    g = tiny.geom
    F = 16
    rng = np.random.default_rng(0)
    n = 200
    rec = np.zeros(n, dtype=L.LOC3D)
    rec["frame"] = np.sort(rng.integers(0, F, n))
    rec["x"] = rng.uniform(0, g.n_el - 1, n)
    rec["y"] = rng.uniform(0, g.n_el - 1, n)
    rec["z"] = rng.uniform(0, g.nz - 1, n)
    out3d = torch.from_numpy(rec.view(np.int32).reshape(-1, 10).copy())
    n3d = torch.tensor([n], dtype=torch.int32)
    gen = torch.Generator().manual_seed(1)
    planes = torch.randn((F, 2, 2, g.n_slab, g.nz, g.n_el, 2), generator=gen)
    slices = torch.randn((F, 2, g.nzs, g.n_el, 2), generator=gen)
    r = bench.cpu_next_rows(tiny, L, out3d, n3d, planes, slices, F)
    for k in ("tracking", "separation", "clutter_svd", "motion"):
        assert r[k]["ms_per_ensemble"] >= 0.0 and r[k]["sample"]
    assert r["cores"] >= 1
