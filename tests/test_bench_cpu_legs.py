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
    npx = planes.numel() // (2 * F)
    expect = {"tracking": 1.0, "separation": npx / 4096, "clutter_svd": slices.shape[1], "motion": F / 3}
    for k, scale in expect.items():
        e = r[k]
        assert e["measured_ms"] > 0.0 and e["ms_per_ensemble"] > 0.0, k
        assert abs(e["scale"] - scale) <= 1e-6 * scale, (k, e["scale"], scale)
        # both figures are rounded (0.1 ms and 1 us): allow those roundings only
        slack = 0.05 + 0.0005 * e["scale"] + 1e-6 * e["ms_per_ensemble"]
        assert abs(e["ms_per_ensemble"] - e["measured_ms"] * e["scale"]) <= slack, k
    assert f"{n} localisations" in r["tracking"]["sample"]
    assert f"{F} frames" in r["separation"]["sample"] and f"{F} frames" in r["clutter_svd"]["sample"]
    assert f"of {F} frames" in r["motion"]["sample"]
    assert r["cores"] >= 1


def test_cpu_baseline_times_one_thread_and_all_cores(tiny, tiny_rf):
    """best of 3 after a warm-up, once per thread setting, on a sample of the
    tiny ensemble; the all-core figure is the line's value"""
    bench = _bench()
    r = bench.cpu_baseline(tiny, tiny_rf.rf, 2)
    assert r["kind"] == "oracle" and r["cores"] >= 1
    assert r["value"] > 0 and r["one_thread"]["value"] > 0 and r["one_thread"]["threads"] == 1
    assert "best of 3" in r["sample"] and "2 of 64 frames" in r["sample"]
    assert "1 of 64 frames" in r["one_thread"]["sample"]


def test_reference_arm_reports_what_it_ran(capsys):
    """the reference line's steps, warm-up and time per step are those of the
    run itself; the per-ensemble extrapolation has its own key"""
    import argparse
    import json
    bench = _bench()
    args = argparse.Namespace(workload="tiny", steps=3, warmup=2, gpus=1, precision="fp32", impl="reference")
    bench.reference_arm(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 2
    assert line["ms_per_step"] > 0
    assert abs(line["value"] - 1e3 / line["ms_per_step"]) <= 0.01 * line["value"]
    assert abs(line["ms_per_ensemble_extrapolated"] - 64 * line["ms_per_step"]) <= 0.01 * line["ms_per_ensemble_extrapolated"]
    assert line["e2e"]["value"] == line["value"] and line["cpu_baseline"]["value"] == line["value"]
