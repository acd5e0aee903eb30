"""Benchmark: projection beamforming + NCC localisation of one 300-frame
paper-scale RCA ensemble per step (128 + 128 elements, 8 transmissions,
1024 samples, 250 x 128 planes, P = 8), on synthetic seeded channel data.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 runs N independent replicas (one
ensemble per rank; the path has no exchange step), launched by torchrun.
``--impl reference`` times the FP64 CPU oracle (the only reference this
method has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "projection frames/s & ms per 300-frame ensemble vs plain FP32; % HBM roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "reduced"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the tables' default Stage-1 / Stage-2 launch shapes (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-frames", type=int, default=4)
    ap.add_argument("--frames", type=int, default=0, help="override the ensemble length (profiling runs)")
    ap.add_argument("--no-forms", action="store_true", help="skip the reduced-precision / batched / learned forms")
    ap.add_argument("--no-next-rows", action="store_true", help="skip tracking, separation, motion estimation and the SVD filter")
    ap.add_argument("--cnn-profile", action="store_true",
                    help="profiling aid: the learned network (untrained weights) on the ensemble's planes only")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # the timed region starts once sampling runs (nvidia-smi takes a moment to start)
            t0 = time.time()
            while not self.samples and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.samples.clear()      # keep only samples taken during the timed region
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if len(s) > 8 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) > 8 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for n, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# distributed helpers (replicas only)
# ---------------------------------------------------------------------------
def dist_init(args=None):
    """Join the torchrun job (env:// rendezvous).  NCCL with one GPU per rank;
    gloo when CUDA is unavailable (the host-side logic is tested that way)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Largest value over the ranks (the slowest replica sets the job time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(frames_per_rank: int, steps: int, max_ms: float, world: int) -> float:
    """Whole-job frames/s: every rank processed frames_per_rank x steps frames
    and the job took the slowest rank's time."""
    return world * frames_per_rank * steps / (max_ms / 1e3)


def emit(line: dict, rank: int) -> None:
    """The one JSON line of a run, printed by rank 0 only."""
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# algorithmic work per launch
# ---------------------------------------------------------------------------
def stage1_terms(R, L, t, geom, F):
    """valid (pixel, element) interpolate-and-accumulate terms of Stage 1 for
    F frames: for every transmission k and slice row r, lateral distance d up
    to the aperture limit with the delay inside the record, times the number
    of (pixel, element) pairs at that distance (N for d = 0, 2 (N - d) else)."""
    import numpy as np
    txq = R.rca_tables_download(t, L.RCA_TAB_TX_Q16).astype(np.int64)     # [2K][nzs]
    rxq = R.rca_tables_download(t, L.RCA_TAB_RX_Q16).astype(np.int64)     # [nzs][N]
    dmax = R.rca_tables_download(t, L.RCA_TAB_DMAX)
    N = geom.n_el
    d = np.arange(N)
    pairs = np.where(d == 0, N, 2 * (N - d))
    qmax = (geom.ns - 1) << 16
    total = 0
    for k in range(txq.shape[0]):
        q = txq[k][:, None] + rxq                                          # [nzs][N]
        ok = (q >= 0) & (q <= qmax) & (d[None, :] <= dmax[:, None])
        total += int((ok * pairs[None, :]).sum())
    return total * F


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import numpy as np
    import torch

    rank, world, local = dist_init(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300 import rca as R
    from paper_2511_21647_gb300.pipeline import RcaSession, complex_buffer
    from synth import generate, quantize_int16, workload

    w = workload(args.workload, seed=workload(args.workload).seed + rank)
    if args.frames:
        w = workload(args.workload, seed=w.seed, n_frames=args.frames)
    g = w.geom
    F = w.n_frames
    t_gen = time.time()
    G = generate(w, device=str(dev), dtype=torch.float32, with_noise=True)
    rf = G.rf.contiguous()
    gen_s = time.time() - t_gen
    reduced = args.precision == "reduced"
    if reduced:
        rf_dev, scale = quantize_int16(rf)
        rf_dev = rf_dev.contiguous()
        scale = scale.contiguous()
        rf_t, iq_t, pl_t = L.RCA_I16, L.RCA_C16F, L.RCA_C16BF
    else:
        rf_dev, scale = rf, None
        rf_t, iq_t, pl_t = L.RCA_F32, L.RCA_C32, L.RCA_C32

    sess = RcaSession(g, device=local)
    stream = torch.cuda.current_stream(dev)
    R.rca_reserve(sess.h, sess.g, F)
    nt = 2 * g.K
    iq = complex_buffer((F, nt, g.ns, g.n_el), iq_t, dev)
    slices = complex_buffer((F, nt, g.nzs, g.n_el), L.RCA_C32, dev)
    planes = complex_buffer(sess.planes_shape(F), pl_t, dev)
    A = torch.empty(sess.a_shape(F), dtype=torch.float32, device=dev)
    M = torch.empty(F, dtype=torch.float32, device=dev)
    # list capacities sized to the workload: 256 detections per projection
    # plane (2D) and 64 per frame and slab (3D), several times what the method finds
    cap2d = min(1 << 22, max(1 << 12, 256 * F * 2 * g.n_slab))
    cap3d = min(1 << 19, max(1 << 12, 64 * F * g.n_slab))
    out2d, n2d, out3d, n3d = sess.loc_buffers(cap2d, cap3d)
    prm = R.make_ulm_params(d=w.ncc_d, sig_z=0.81, sig_lat=1.45, alpha=0.1, ncc_min=0.5)
    h, t = sess.h, sess.t

    stages = ["ingest", "stage1", "stage2", "enhance", "detect2d", "pair3d"]
    # kernels per call: mean + demodulation; detect + three scan passes + gather;
    # list offsets + match + flags + three scan passes + write
    launches = {"ingest": 2, "stage1": 1, "stage2": 1, "enhance": 1, "detect2d": 5, "pair3d": 7}

    def step(ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        R.rca_ingest(h, t, rf_dev, rf_t, scale, F, L.RCA_CLUTTER_MEAN, iq, iq_t)
        mark(1)
        R.rca_stage1(h, t, iq, iq_t, F, slices)
        mark(2)
        R.rca_stage2_project(h, t, slices, F, planes, pl_t)
        mark(3)
        R.ulm_enhance(h, t, planes, pl_t, F, L.ULM_ENH_XDOPPLER, A, M)
        mark(4)
        R.ulm_detect2d(h, t, A, M, F, prm, out2d, cap2d, n2d)
        mark(5)
        R.ulm_pair3d(h, t, out2d, n2d, cap2d, F, out3d, cap3d, n3d)
        mark(6)

    # Stage-1 (row tile x distance chunk) and Stage-2 (plane-row tile) launch
    # shapes timed on this ensemble's IQ by the library's autotuner (part of
    # the set-up, outside the timed region)
    shapes = None
    if not args.no_autotune:
        R.rca_ingest(h, t, rf_dev, rf_t, scale, F, L.RCA_CLUTTER_MEAN, iq, iq_t)
        zt_, dc_, zp_ = R.rca_autotune(h, t, iq, iq_t, F)
        shapes = {"stage1_row_tile": zt_, "stage1_distance_chunk": dc_, "stage2_plane_rows": zp_,
                  "source": "rca_autotune on this ensemble's IQ"}
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    dev_status = R.rca_sync_status(h)
    if args.cnn_profile:
        # the network's forward pass over every plane of the ensemble, twice
        # (untrained weights: the kernels' work does not depend on them)
        c = R.ulm_cnn_create(h, max_pixels=1 << 24, seed=1)
        fc = 16
        heat = torch.empty((fc * 2 * g.n_slab, 4 * g.nz, 4 * g.n_el), dtype=torch.float32, device=dev)
        for _ in range(2):
            for f0 in range(0, F - fc + 1, fc):
                R.ulm_cnn_forward(c, A[f0:f0 + fc], M[f0:f0 + fc], 2 * g.n_slab, fc * 2 * g.n_slab, g.nz, g.n_el, heat)
        torch.cuda.synchronize()
        R.ulm_cnn_destroy(c)
        emit({"cnn_profile": "done", "frames": F, "status": R.rca_sync_status(h)}, rank)
        sess.close()
        return

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(K)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(K):
            step(evs[k])
        torch.cuda.synchronize()
    barrier(world)
    per_stage = {s: [] for s in stages}
    totals = []
    for k in range(K):
        for i, s in enumerate(stages):
            per_stage[s].append(evs[k][i].elapsed_time(evs[k][i + 1]))
        totals.append(evs[k][0].elapsed_time(evs[k][6]))
    ms_total = sum(totals)
    ms_max = max_over_ranks(ms_total, world)
    ms_step = ms_max / K
    value = job_throughput(F, K, ms_max, world)
    stage_ms = {s: sum(v) / K for s, v in per_stage.items()}
    n2d_v, n3d_v = int(n2d.item()), int(n3d.item())

    fp32 = fp32_peak(R, h, dev, local)
    direct = direct_form(R, L, sess, iq, iq_t, F, stream, stage_ms) if rank == 0 and not reduced else None

    # -- roofline of the dominant kernel -----------------------------------
    import json as _json
    peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_derived_tflops = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    fp32_peak_tflops = fp32["tflops"]
    esz_rf = 2 if reduced else 4
    esz_iq = 4 if reduced else 8
    esz_pl = 4 if reduced else 8
    n_rf = F * nt * g.n_el * g.ns
    n_sl = F * nt * g.nzs * g.n_el
    n_pl = F * 4 * g.n_slab * g.nz * g.n_el
    n_a = F * 2 * g.n_slab * g.nz * g.n_el
    bytes_alg = {
        "ingest": 2 * n_rf * esz_rf + n_rf * esz_iq,
        "stage1": n_rf * esz_iq + n_sl * 8,
        "stage2": n_sl * 8 + n_pl * esz_pl,
        "enhance": n_pl * esz_pl + n_a * 4,
        "detect2d": n_a * 4 + n2d_v * 40,
        "pair3d": n2d_v * 40 + n3d_v * 40,
    }
    terms = stage1_terms(R, L, t, g, F)
    flops_stage1 = 14.0 * terms
    dominant = max(stage_ms, key=stage_ms.get)
    if dominant == "stage1":
        ach = flops_stage1 / (stage_ms["stage1"] / 1e3) / 1e12
        roof = {"kernel": "k_stage1", "bound": "alu", "achieved": round(ach, 2), "peak": round(fp32_peak_tflops, 1),
                "unit": "TFLOP/s", "frac": round(ach / fp32_peak_tflops, 4), "traffic": None,
                "peak_source": "measured in this run: rca_fp32_probe (the library's FP32 FMA issue probe, "
                               "best of scalar and packed, %.0f MHz median SM clock); derived 152 x 128 x 2 x "
                               "sm_max_mhz = %.1f" % (fp32["sm_mhz"] or 0, fp32_derived_tflops),
                "limiter": "shared-memory data path: each term reads two complex FP32 samples (16 B); "
                           "83 % of L1/shared throughput in profiles/stage1_paper_40frames.md"}
    else:
        ach = bytes_alg[dominant] / (stage_ms[dominant] / 1e3) / 1e9
        roof = {"kernel": dominant, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(ach / hbm_peak, 4), "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    # DRAM traffic of the dominant kernel from the committed ncu summary, only
    # while the kernel's source is the one that was profiled
    try:
        import hashlib
        prof = _json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        key = roof["kernel"].split("<")[0]
        ent = prof.get(key)
        if ent:
            src = open(os.path.join(ROOT, ent["source"]), "rb").read()
            if hashlib.sha256(src).hexdigest()[:16] == ent["source_sha256_16"]:
                roof["traffic"] = int(ent["dram_bytes_per_frame"] * F)
                roof["traffic_source"] = "profiles/traffic.json (" + ent.get("profile", "ncu capture") + "), scaled by frames"
    except (OSError, ValueError, KeyError):
        pass
    stage_roof = {}
    for s in stages:
        gbs = bytes_alg[s] / (stage_ms[s] / 1e3) / 1e9
        stage_roof[s] = {"ms": round(stage_ms[s], 4), "alg_GBps": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4)}
    stage_roof["stage1"]["alg_TFLOPs"] = round(flops_stage1 / (stage_ms["stage1"] / 1e3) / 1e12, 2)
    stage_roof["stage1"]["fp32_frac"] = round(flops_stage1 / (stage_ms["stage1"] / 1e3) / 1e12 / fp32_peak_tflops, 4)
    stage_roof["stage1"]["terms"] = terms

    # -- end to end through the public calls, host buffers -------------------
    # Every step copies its channel data from pinned host memory and reads its
    # 3D list (the whole capacity buffer, so no host sync is needed to size it)
    # and counts back to pinned host memory.  Steps are pipelined the way an
    # acquisition stream would run: the copy of step k+1 (copy stream, second
    # staging buffer) overlaps the compute of step k.
    e2e = None
    if not args.no_e2e:
        rf_host = rf_dev.cpu().pin_memory()
        scale_host = scale.cpu().pin_memory() if scale is not None else None
        rf_stage = [torch.empty_like(rf_dev) for _ in range(2)]
        sc_stage = [torch.empty_like(scale) for _ in range(2)] if scale is not None else [None, None]
        out_host = torch.empty((cap3d, 10), dtype=torch.int32).pin_memory()
        cnt_host = torch.empty(2, dtype=torch.int32).pin_memory()
        cnt_dev = torch.empty(2, dtype=torch.int32, device=dev)
        copy_stream = torch.cuda.Stream(dev)
        d2h_stream = torch.cuda.Stream(dev)
        ready = [torch.cuda.Event() for _ in range(2)]
        free = [torch.cuda.Event() for _ in range(2)]
        done = torch.cuda.Event()
        read = torch.cuda.Event()
        for ev in free:
            ev.record(stream)
        read.record(stream)

        def h2d(slot):
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(free[slot])
                rf_stage[slot].copy_(rf_host, non_blocking=True)
                if sc_stage[slot] is not None:
                    sc_stage[slot].copy_(scale_host, non_blocking=True)
                ready[slot].record(copy_stream)

        def compute(slot):
            stream.wait_event(ready[slot])
            R.rca_beamform_projections(h, t, rf_stage[slot], rf_t, sc_stage[slot], F, R.bf_params(iq_dtype=iq_t),
                                       planes, pl_t)
            free[slot].record(stream)
            stream.wait_event(read)            # the previous step's list has been read back
            R.ulm_localize(h, t, planes, pl_t, F, prm, out2d, cap2d, n2d, out3d, cap3d, n3d)
            cnt_dev[0:1].copy_(n2d)
            cnt_dev[1:2].copy_(n3d)
            done.record(stream)
            with torch.cuda.stream(d2h_stream):
                d2h_stream.wait_event(done)
                cnt_host.copy_(cnt_dev, non_blocking=True)
                out_host.copy_(out3d, non_blocking=True)
                read.record(d2h_stream)

        def run(nsteps):
            h2d(0)
            for k in range(nsteps):
                if k + 1 < nsteps:
                    h2d((k + 1) % 2)
                compute(k % 2)

        run(2)
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        copy_stream.wait_event(e0)
        run(K)
        stream.wait_event(read)                # the last step's results are on the host
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(e0.elapsed_time(e1), world)
        e2e = {"value": round(job_throughput(F, K, e_ms, world), 1), "unit": "frames/s",
               "ms_per_ensemble": round(e_ms / K, 3),
               "h2d_bytes_per_step": int(rf_dev.numel() * rf_dev.element_size() + (scale.numel() * 4 if scale is not None else 0)),
               "d2h_bytes_per_step": int(out_host.numel() * 4 + cnt_host.numel() * 4),
               "pipelined": "copy of step k+1 overlaps compute of step k (two staging buffers)",
               "n3d_last": int(cnt_host[1])}

    status_after = R.rca_sync_status(h)
    forms = None
    if rank == 0 and not args.no_forms and not reduced and not args.frames:
        forms = {}
        forms["reduced"] = reduced_form(R, L, sess, rf, F, prm, max(3, args.warmup), K, stream,
                                        autotune=not args.no_autotune)
        forms["batched"] = batched_form(R, L, dev, stream, K)
        forms["learned"] = learned_form(R, L, sess, planes, F, g, dev, stream, peaks)
    next_rows = rank == 0 and not args.no_next_rows and not reduced
    track = tracking_step(R, L, sess, out3d, n3d, cap3d, F, stream, K) if next_rows else None
    sep = separation_step(R, L, sess, w, planes, F, prm, cap2d, cap3d, stream, K) if next_rows else None
    motion = motion_step(R, L, sess, w, rf_dev, rf_t, scale, iq, iq_t, slices, F, stream, K) if next_rows else None
    svd = svd_step(R, sess, slices, F, stream, K) if next_rows else None
    pipe = pipeline_step(R, L, sess, w, rf_dev, rf_t, scale, iq, iq_t, slices, planes, F, prm, cap2d, cap3d,
                         stream, K) if next_rows else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, G.rf, args.cpu_sample_frames)
        if next_rows:
            cpu["next_rows"] = cpu_next_rows(w, L, out3d, n3d, planes, slices, F)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": round(value, 1),
            "unit": "frames/s",
            "n_gpus": world,
            "steps": K,
            "warmup": max(3, args.warmup),
            "ms_per_step": round(ms_step, 4),
            "ms_per_ensemble": round(ms_step, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "i16/f16/bf16+f32acc" if reduced else "f32",
            "data": "synthetic (seeded point scatterers; paper's in-vivo / Field II data unavailable)",
            "config": workload_config(w, F, args.precision, world),
            "launch_shapes": shapes,
            "stages": stage_roof,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "forms": forms,
            "fp32_peak": fp32,
            "direct_projection": direct,
            "tracking": track,
            "separation": sep,
            "motion": motion,
            "clutter_svd": svd,
            "pipeline": pipe,
            "gpu_launches": K * sum(launches.values()),
            "clocks": clk.summary(),
            "localisations": {"n2d": n2d_v, "n3d": n3d_v},
            "device_status": [dev_status, status_after],
            "generate_s": round(gen_s, 1),
        }
        emit(line, rank)
    sess.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def fp32_peak(R, h, dev, gpu_index, reps=25):
    """The FP32 roofline denominator, measured: the library's FMA issue probe
    (every SM full, 16 independent FMA chains per thread), scalar and packed
    f32x2, each timed with CUDA events as the best of `reps` launches after
    two warm-up launches, with the SM clock sampled meanwhile."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(8 * sms, device=dev)
    iters = 1 << 17
    res = {}
    with ClockSampler(gpu_index) as clk:
        for name, packed in (("scalar", 0), ("packed", 1)):
            for _ in range(2):
                flops = R.rca_fp32_probe(h, packed, iters, sink)
            best = None
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                R.rca_fp32_probe(h, packed, iters, sink)
                e1.record()
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            res[name] = round(flops / (best / 1e3) / 1e12, 2)
    c = clk.summary()
    return {"tflops": max(res.values()), "scalar_tflops": res["scalar"], "packed_tflops": res["packed"],
            "sm_mhz": c["sm_mhz"], "clock_reasons": c["reasons"],
            "method": f"rca_fp32_probe: {sms} SMs x 8 CTAs x 256 threads x 16 FMA chains x {iters} steps, "
                      f"best of {reps} launches (CUDA events)"}


def direct_form(R, L, sess, iq, iq_t, F, stream, stage_ms, n=4):
    """The work the two-stage method replaces (Sec. II-A1's conventional
    beamforming, compared in Sec. III): the exact full-3D DAS projected per
    plane pixel (RCA_MODE_DIRECT), timed on n frames of the ensemble's IQ and
    scaled to the ensemble, next to the two-stage Stage 1 + Stage 2 time."""
    import torch
    from paper_2511_21647_gb300.pipeline import complex_buffer
    h, t = sess.h, sess.t
    pl = complex_buffer(sess.planes_shape(n), L.RCA_C32, iq.device)
    R.rca_direct_project(h, t, iq[:n], iq_t, n, pl, L.RCA_C32)
    times = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R.rca_direct_project(h, t, iq[:n], iq_t, n, pl, L.RCA_C32)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = min(times) * F / n
    two = stage_ms["stage1"] + stage_ms["stage2"]
    return {"frames_timed": n, "ms_per_ensemble": round(ms, 2), "two_stage_ms_per_ensemble": round(two, 3),
            "direct_over_two_stage": round(ms / two, 1), "status": R.rca_sync_status(h),
            "what": "exact full-3D DAS volume, slab-projected per plane pixel (k_direct), best of 3, scaled by frames"}


def motion_step(R, L, sess, w, rf_dev, rf_t, scale, iq, iq_t, slices, F, stream, K):
    """Projection-based rigid motion estimation (Sec. II-A3) on the Stage-1
    slices of the same ensemble without clutter removal (the tissue carries
    the motion); timed beside the step, and compared with the generator's
    tissue displacement (a 0.2 mm 1 Hz axial sinusoid at 400 Hz)."""
    import math
    import torch
    R.rca_ingest(sess.h, sess.t, rf_dev, rf_t, scale, F, L.RCA_CLUTTER_NONE, iq, iq_t)
    R.rca_stage1(sess.h, sess.t, iq, iq_t, F, slices)
    motion = torch.zeros((F, 3), device=slices.device)

    def run():
        R.rca_motion_estimate(sess.h, sess.t, slices, F, motion)

    for _ in range(3):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    m = motion.cpu().numpy()
    t = [f / 400.0 for f in range(F)]
    truth = [w.tissue_motion_amp * math.sin(2 * math.pi * w.tissue_motion_hz * x) for x in t]
    err = [abs(float(a) - b) for a, b in zip(m[:, 2], truth)]
    return {"ms_per_ensemble": round(e0.elapsed_time(e1) / K, 4), "frames": F,
            "axial_rms_error_um": round(1e6 * math.sqrt(sum(e * e for e in err) / F), 3),
            "axial_max_error_um": round(1e6 * max(err), 3),
            "lateral_max_um": round(1e6 * float(abs(m[:, :2]).max()), 3),
            "truth": "tissue displacement 0.2 mm sin(2 pi 1 Hz t), t = frame / 400 Hz, axial",
            "kernels": 5 + 2 * ((F + 63) // 64), "status": R.rca_sync_status(sess.h)}


def svd_step(R, sess, slices, F, stream, K, rank=16, iters=30):
    """Eigen-based SVD clutter filter (Sec. II-A2) on the ensemble's unfiltered
    Stage-1 slices (as motion_step leaves them), in place; timed beside the
    step.  Work: the 2K frame covariances (F^2 P / 2 complex products each),
    the eigenspace iteration, the projection (2 F rank P complex products)."""
    import torch
    # the first call reports how well the removed subspace is determined on
    # the unfiltered slices (every later call filters the filtered slices)
    info = torch.zeros((slices.shape[1], 4), dtype=torch.float32, device=slices.device)
    R.rca_clutter_svd_info(sess.h, sess.t, slices, F, rank, iters, info)
    R.rca_clutter_svd(sess.h, sess.t, slices, F, rank, iters)
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    report = {"gap_over_lambda1": [round(float((a[1] - a[2]) / a[0]), 9) for a in inf],
              "invariance_residual": [round(float(a[3]), 5) for a in inf],
              "note": "(theta_rank - theta_rank+1) / theta_1 near the FP32 covariance's rounding (~1e-7) "
                      "leaves the vectors near the split undetermined (rca_clutter_svd_info)"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        R.rca_clutter_svd(sess.h, sess.t, slices, F, rank, iters)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    nt, P = slices.shape[1], slices.shape[2] * slices.shape[3]
    flops = nt * (F * F * P * 4.0 + 2 * F * rank * P * 8.0)
    return {"ms_per_ensemble": round(ms, 4), "rank": rank, "iterations": iters, "frames": F,
            "gflop": round(flops / 1e9, 1), "tflops": round(flops / (ms / 1e3) / 1e12, 2),
            "kernels": 4, "split": report, "status": R.rca_sync_status(sess.h)}


def separation_step(R, L, sess, w, planes, F, prm, cap2d, cap3d, stream, K, n_bands=3):
    """Microbubble separation (Sec. II-A5) of the step's FP32 planes into three
    equal speed bands over (0, 200] Hz x up / down, fused with each subset's
    XDoppler enhancement (ulm_separate_enhance), then each subset's detection
    and pairing (the paper's Up3 / Down3 localisation); timed beside the step.
    Algorithmic bytes: planes read once, six amplitude stacks written; work:
    one forward and six inverse F-point transforms per plane pixel
    (5 F log2 F flop each, the conventional FFT count)."""
    import math
    import torch
    g = w.geom
    sp = R.make_sep_params(w.frame_rate, n_bands)
    ns = 2 * n_bands
    A = torch.empty((ns,) + tuple(sess.a_shape(F)), dtype=torch.float32, device=planes.device)
    M = torch.empty((ns, F), dtype=torch.float32, device=planes.device)
    bufs = [sess.loc_buffers(cap2d, cap3d) for _ in range(ns)]

    def sep():
        R.ulm_separate_enhance(sess.h, sess.t, planes, L.RCA_C32, F, sp, L.ULM_ENH_XDOPPLER, A, M)

    def loc():
        for s in range(ns):
            out2d, n2d, out3d, n3d = bufs[s]
            R.ulm_detect2d(sess.h, sess.t, A[s], M[s], F, prm, out2d, cap2d, n2d)
            R.ulm_pair3d(sess.h, sess.t, out2d, n2d, cap2d, F, out3d, cap3d, n3d)

    for _ in range(2):
        sep()
        loc()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_sep = t_loc = 0.0
    for _ in range(K):
        ev[0].record(stream)
        sep()
        ev[1].record(stream)
        loc()
        ev[2].record(stream)
        torch.cuda.synchronize()
        t_sep += ev[0].elapsed_time(ev[1])
        t_loc += ev[1].elapsed_time(ev[2])
    ms_sep, ms_loc = t_sep / K, t_loc / K
    npx = planes.numel() // (2 * F)
    bytes_ = planes.numel() * planes.element_size() + A.numel() * 4
    flop = 7 * 5.0 * F * math.log2(F) * npx
    import json as _json
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = _json.load(open(pk)).get("hbm_gbs") if os.path.exists(pk) else None
    n2d = [int(b[1].item()) for b in bufs]
    n3d = [int(b[3].item()) for b in bufs]
    return {"ms_per_ensemble": round(ms_sep, 4), "subsets": ns, "bands_hz": [round(x, 3) for x in sp.edges_hz[:n_bands + 1]],
            "alg_GBps": round(bytes_ / (ms_sep / 1e3) / 1e9, 1),
            "hbm_frac": round(bytes_ / (ms_sep / 1e3) / 1e9 / peak, 4) if peak else None,
            "fft_TFLOPs": round(flop / (ms_sep / 1e3) / 1e12, 2),
            "localise_subsets_ms": round(ms_loc, 4), "n2d": n2d, "n3d": n3d,
            "kernels": 1, "status": R.rca_sync_status(sess.h)}


def pipeline_step(R, L, sess, w, rf_dev, rf_t, scale, iq, iq_t, slices, planes, F, prm, cap2d, cap3d, stream, K,
                  rank=16, iters=30, n_bands=3):
    """The paper's whole per-ensemble chain on the device-resident RF as one
    timed sequence: ingest without clutter removal, Stage 1, motion estimation
    on the unfiltered slices, the SVD clutter filter (rank 16, 30 subspace
    iterations), Stage 2 + projection, separation into three speeds x up /
    down fused with each subset's XDoppler, and per subset detection, pairing
    and tracking into one density grid and its velocity volumes (zeroed per
    ensemble).  Context for the
    paper's 0.52 s per 300-volume ensemble on its own GPU and data."""
    import torch
    h, t = sess.h, sess.t
    dev = planes.device
    motion = torch.zeros((F, 3), device=dev)
    sp = R.make_sep_params(w.frame_rate, n_bands)
    ns = 2 * n_bands
    A = torch.empty((ns,) + tuple(sess.a_shape(F)), dtype=torch.float32, device=dev)
    M = torch.empty((ns, F), dtype=torch.float32, device=dev)
    bufs = [sess.loc_buffers(cap2d, cap3d) for _ in range(ns)]
    tp = R.make_track_params()
    nx, ny, nz = R.ulm_density_shape(t, tp.voxel_m)
    grid = torch.zeros((nz, ny, nx), dtype=torch.int32, device=dev)
    vel = torch.zeros((2, nz, ny, nx), dtype=torch.int64, device=dev)
    trk = [torch.zeros((cap3d, L.TRACK.itemsize // 4), dtype=torch.int32, device=dev) for _ in range(ns)]
    ntr = [torch.zeros(1, dtype=torch.int32, device=dev) for _ in range(ns)]
    parts = ["stage1", "motion", "svd", "stage2", "separate", "localise_track"]

    def chain(ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        R.rca_ingest(h, t, rf_dev, rf_t, scale, F, L.RCA_CLUTTER_NONE, iq, iq_t)
        R.rca_stage1(h, t, iq, iq_t, F, slices)
        mark(1)
        R.rca_motion_estimate(h, t, slices, F, motion)
        mark(2)
        R.rca_clutter_svd(h, t, slices, F, rank, iters)
        mark(3)
        R.rca_stage2_project(h, t, slices, F, planes, L.RCA_C32)
        mark(4)
        R.ulm_separate_enhance(h, t, planes, L.RCA_C32, F, sp, L.ULM_ENH_XDOPPLER, A, M)
        mark(5)
        grid.zero_()
        vel.zero_()
        for s in range(ns):
            out2d, n2d, out3d, n3d = bufs[s]
            R.ulm_detect2d(h, t, A[s], M[s], F, prm, out2d, cap2d, n2d)
            R.ulm_pair3d(h, t, out2d, n2d, cap2d, F, out3d, cap3d, n3d)
            R.ulm_track(h, t, out3d, n3d, cap3d, F, tp, trk[s], cap3d, ntr[s], grid)
            R.ulm_track_velocity(h, t, trk[s], ntr[s], cap3d, tp, vel[0], vel[1])
        mark(6)

    for _ in range(2):
        chain()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(K)]
    for k in range(K):
        chain(evs[k])
    torch.cuda.synchronize()
    tot = sum(e[0].elapsed_time(e[6]) for e in evs) / K
    part_ms = {p: round(sum(e[i].elapsed_time(e[i + 1]) for e in evs) / K, 3) for i, p in enumerate(parts)}
    kept = 0
    for s in range(ns):
        k = min(int(ntr[s].item()), cap3d)
        kept += int(trk[s][:k].cpu().numpy().view(L.TRACK).reshape(-1)["accepted"].sum())
    return {"ms_per_ensemble": round(tot, 3), "volumes_per_s": round(F / (tot / 1e3), 1), "parts_ms": part_ms,
            "order": "ingest (no clutter removal) + Stage 1 | motion | SVD rank 16 | Stage 2 + projection | "
                     "separation x6 + XDoppler | per subset: detect, pair, track, density + velocity",
            "n3d_per_subset": [int(b[3].item()) for b in bufs], "tracks_kept": kept,
            "density_counts": int(grid.sum().item()),
            "paper_ms_per_ensemble_context": 520.0, "status": R.rca_sync_status(h)}


def tracking_step(R, L, sess, out3d, n3d, cap3d, F, stream, K):
    """Fixed-length tracking (Sec. II-A6) of the last step's 3D list: ten-point
    tracks, 150 um link radius, 45 degree / half-mean-speed rejection, 50 um
    density and velocity volumes; not part of the timed step (the paper's
    tracking follows the projection path)."""
    import torch
    prm = R.make_track_params()
    nx, ny, nz = R.ulm_density_shape(sess.t, prm.voxel_m)
    grid = torch.zeros((nz, ny, nx), dtype=torch.int32, device=out3d.device)
    speed = torch.zeros((nz, ny, nx), dtype=torch.int64, device=out3d.device)
    vz = torch.zeros_like(speed)
    cap_t = cap3d
    out = torch.zeros((cap_t, L.TRACK.itemsize // 4), dtype=torch.int32, device=out3d.device)
    nt = torch.zeros(1, dtype=torch.int32, device=out3d.device)

    def run():
        R.ulm_track(sess.h, sess.t, out3d, n3d, cap3d, F, prm, out, cap_t, nt, grid)
        R.ulm_track_velocity(sess.h, sess.t, out, nt, cap_t, prm, speed, vz)

    for _ in range(3):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    k = int(nt.item())
    rec = out[:min(k, cap_t)].cpu().numpy().view(L.TRACK).reshape(-1)
    return {"ms_per_ensemble": round(e0.elapsed_time(e1) / K, 4), "tracks": k,
            "accepted": int(rec["accepted"].sum()), "localisations": int(n3d.item()),
            "params": {"len": prm.len, "max_step_m": prm.max_step_m, "max_turn_deg": 45.0,
                       "max_speed_change": prm.max_speed_change, "voxel_m": prm.voxel_m, "substeps": prm.substeps},
            "density_grid": [nz, ny, nx], "velocity_volumes": "speed and axial sums, nm per frame, int64",
            "kernels": 7, "status": R.rca_sync_status(sess.h)}


def reduced_form(R, L, sess0, rf, F, prm, W, K, stream, autotune=True):
    """Same ensemble, int16 channel data + per-channel scale, FP16 IQ, BF16
    planes, FP32 accumulation: ms per ensemble through the public calls (own
    tables, launch shapes tuned on its FP16 IQ)."""
    import torch
    from paper_2511_21647_gb300.pipeline import RcaSession, complex_buffer
    from synth import quantize_int16
    q, scale = quantize_int16(rf)
    q, scale = q.contiguous(), scale.contiguous()
    sess = RcaSession(sess0.geom, device=rf.device.index or 0)
    R.rca_reserve(sess.h, sess.g, F)
    shapes = None
    if autotune:
        iq0 = complex_buffer(sess.iq_shape(F), L.RCA_C16F, rf.device)
        R.rca_ingest(sess.h, sess.t, q, L.RCA_I16, scale, F, L.RCA_CLUTTER_MEAN, iq0, L.RCA_C16F)
        shapes = R.rca_autotune(sess.h, sess.t, iq0, L.RCA_C16F, F)
        del iq0
    planes = complex_buffer(sess.planes_shape(F), L.RCA_C16BF, rf.device)
    cap2d, cap3d = 1 << 21, 1 << 19
    bufs = sess.loc_buffers(cap2d, cap3d)
    bp = R.bf_params(iq_dtype=L.RCA_C16F)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def step(timed=False):
        if timed:
            ev[0].record(stream)
        R.rca_beamform_projections(sess.h, sess.t, q, L.RCA_I16, scale, F, bp, planes, L.RCA_C16BF)
        if timed:
            ev[1].record(stream)
        R.ulm_localize(sess.h, sess.t, planes, L.RCA_C16BF, F, prm, bufs[0], cap2d, bufs[1], bufs[2], cap3d, bufs[3])
        if timed:
            ev[2].record(stream)

    for _ in range(W):
        step()
    torch.cuda.synchronize()
    bf, lo = [], []
    for _ in range(K):
        step(True)
        torch.cuda.synchronize()
        bf.append(ev[0].elapsed_time(ev[1]))
        lo.append(ev[1].elapsed_time(ev[2]))
    ms = (sum(bf) + sum(lo)) / K
    # the beamforming split by stage (stage-level calls on preallocated buffers)
    iq = complex_buffer(sess.iq_shape(F), L.RCA_C16F, rf.device)
    sl = complex_buffer(sess.slices_shape(F), L.RCA_C32, rf.device)
    se = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    st_ms = {"ingest": 0.0, "stage1": 0.0, "stage2": 0.0}
    for rep in range(K + 1):
        se[0].record(stream)
        R.rca_ingest(sess.h, sess.t, q, L.RCA_I16, scale, F, L.RCA_CLUTTER_MEAN, iq, L.RCA_C16F)
        se[1].record(stream)
        R.rca_stage1(sess.h, sess.t, iq, L.RCA_C16F, F, sl)
        se[2].record(stream)
        R.rca_stage2_project(sess.h, sess.t, sl, F, planes, L.RCA_C16BF)
        se[3].record(stream)
        torch.cuda.synchronize()
        if rep:
            for q_, name in enumerate(("ingest", "stage1", "stage2")):
                st_ms[name] += se[q_].elapsed_time(se[q_ + 1]) / K
    del iq, sl
    out = {"ms_per_ensemble": round(ms, 3), "value": round(F / (ms / 1e3), 1), "unit": "frames/s",
           "beamform_ms": round(sum(bf) / K, 3), "localise_ms": round(sum(lo) / K, 3),
           "stages_ms": {k: round(v, 3) for k, v in st_ms.items()},
           "launch_shapes": list(shapes) if shapes else None,
           "dtype": "int16 RF + per-channel scale, FP16 IQ, BF16 planes, FP32 accumulation",
           "n3d": int(bufs[3].item()), "status": R.rca_sync_status(sess.h)}
    sess.close()
    return out


def batched_form(R, L, dev, stream, K):
    """16 uneven ensembles of the tiny geometry (100..600 frames, 2K in
    {2, 4, 8}) beamformed in one batch (one persistent launch, or one launch
    per stage: both timed, the faster reported) and localised, replayed as a
    CUDA graph; compared with the same work issued ensemble by ensemble."""
    import torch
    from paper_2511_21647_gb300.pipeline import complex_buffer
    from synth import batch_workloads, generate
    ws = batch_workloads(16)
    h = R.rca_create(dev.index or 0)
    R.rca_set_stream(h, stream)
    prm = R.make_ulm_params(d=5, sig_z=0.807, sig_lat=1.4495, alpha=0.1, ncc_min=0.5)
    items, keep = [], []
    t_gen = time.time()
    for w in ws:
        g = w.geom
        geo = R.rca_geometry_create(h, g)
        t = R.rca_delay_tables(h, geo)
        rf = generate(w, device=str(dev), dtype=torch.float32, frame_batch=32).rf.contiguous()
        items.append(dict(tables=t, rf=rf, n_frames=w.n_frames,
                          planes=complex_buffer((w.n_frames, 2, 2, g.n_slab, g.nz, g.n_el), L.RCA_C32, dev),
                          out2d=torch.zeros((1 << 17, 10), dtype=torch.int32, device=dev), cap2d=1 << 17,
                          n2d=torch.zeros(1, dtype=torch.int32, device=dev),
                          out3d=torch.zeros((1 << 16, 10), dtype=torch.int32, device=dev), cap3d=1 << 16,
                          n3d=torch.zeros(1, dtype=torch.int32, device=dev)))
        keep.append((geo, t))
    gen_s = time.time() - t_gen
    frames = sum(w.n_frames for w in ws)
    # launch shapes tuned per ensemble on its own IQ (Stage-1 row tile x
    # distance chunk, Stage-2 plane-row tile), before the plan is built
    t_tune = time.time()
    shapes = {}
    for w, it in zip(ws, items):
        g = w.geom
        iq = complex_buffer((w.n_frames, g.n_tx, g.ns, g.n_el), L.RCA_C32, dev)
        R.rca_ingest(h, it["tables"], it["rf"], L.RCA_F32, None, w.n_frames, L.RCA_CLUTTER_MEAN, iq, L.RCA_C32)
        shapes.setdefault(g.n_tx, set()).add(R.rca_autotune(h, it["tables"], iq, L.RCA_C32, w.n_frames))
        del iq
    tune_s = time.time() - t_tune
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    b = R.rca_batch_create(h, items, L.RCA_F32, L.RCA_C32, L.RCA_C32, prm)
    ms_modes = {}
    for name, mode in (("persistent", L.RCA_BATCH_PERSISTENT), ("staged", L.RCA_BATCH_STAGED)):
        R.rca_batch_set_mode(b, mode)
        ms_modes[name] = timed(lambda: R.rca_batch_run(b, use_graph=True, h=h))
    best_mode = min(ms_modes, key=ms_modes.get)
    ms_batch = ms_modes[best_mode]
    st_batch = R.rca_sync_status(h)
    R.rca_batch_destroy(b)
    # the beamforming part alone, without the localisation branches
    b = R.rca_batch_create(h, items, L.RCA_F32, L.RCA_C32, L.RCA_C32, None)
    ms_modes_bf = {}
    for name, mode in (("persistent", L.RCA_BATCH_PERSISTENT), ("staged", L.RCA_BATCH_STAGED)):
        R.rca_batch_set_mode(b, mode)
        ms_modes_bf[name] = timed(lambda: R.rca_batch_run(b, use_graph=True, h=h))
    ms_batch_bf = min(ms_modes_bf.values())

    def seq_bf():
        for it in items:
            R.rca_beamform_projections(h, it["tables"], it["rf"], L.RCA_F32, None, it["n_frames"], R.bf_params(),
                                       it["planes"], L.RCA_C32)

    def sequential():
        for it in items:
            R.rca_beamform_projections(h, it["tables"], it["rf"], L.RCA_F32, None, it["n_frames"], R.bf_params(),
                                       it["planes"], L.RCA_C32)
            R.ulm_localize(h, it["tables"], it["planes"], L.RCA_C32, it["n_frames"], prm, it["out2d"], it["cap2d"],
                           it["n2d"], it["out3d"], it["cap3d"], it["n3d"])
    ms_seq = timed(sequential)
    ms_seq_bf = timed(seq_bf)
    R.rca_batch_destroy(b)
    for geo, t in keep:
        R.rca_tables_destroy(t)
        R.rca_geometry_destroy(geo)
    R.rca_destroy(h)
    return {"ensembles": len(ws), "frames": frames, "n_tx": sorted({w.geom.n_tx for w in ws}),
            "ms_per_batch": round(ms_batch, 3), "value": round(frames / (ms_batch / 1e3), 1), "unit": "frames/s",
            "mode": best_mode, "ms_per_batch_by_mode": {k: round(v, 3) for k, v in ms_modes.items()},
            "ms_per_300_frames": round(ms_batch * 300 / frames, 3),
            "sequential_ms_per_batch": round(ms_seq, 3), "speedup_vs_sequential": round(ms_seq / ms_batch, 3),
            "beamform_only": {"ms_per_batch": round(ms_batch_bf, 3), "sequential_ms": round(ms_seq_bf, 3),
                              "ms_per_batch_by_mode": {k: round(v, 3) for k, v in ms_modes_bf.items()},
                              "speedup_vs_sequential": round(ms_seq_bf / ms_batch_bf, 3)},
            "tuned_shapes": {str(k): sorted(v) for k, v in sorted(shapes.items())},
            "tuned_shapes_key": "n_tx: [(Stage-1 row tile, distance chunk, Stage-2 plane-row tile)]",
            "tune_s": round(tune_s, 1), "graph": True, "status": st_batch, "generate_s": round(gen_s, 1)}


def learned_form(R, L, sess, planes, F, g, dev, stream, peaks):
    """The learned localiser: trained on 20k planes of the tiny-geometry
    generator (BF16 tensor-core kernels), scored against the NCC path on
    held-out data, then timed on this paper-scale ensemble's planes (XDoppler
    amplitude -> CNN -> heatmap peaks -> pairing, in chunks of frames)."""
    import torch
    from dataclasses import replace
    from paper_2511_21647_gb300 import learned
    from synth import workload
    tg = workload("tiny").geom
    t0 = time.time()
    data = learned.build_dataset(tg, learned.training_workloads(40, frames=64))
    build_s = time.time() - t0
    n_train = data.n_planes
    h = sess.h
    c = R.ulm_cnn_create(h, max_pixels=1 << 24, seed=1)
    t0 = time.time()
    steps = 2000
    hist = learned.train(c, data, steps=steps, batch=64, log_every=500)
    train_s = time.time() - t0
    prm = R.make_ulm_params(d=5, sig_z=0.807, sig_lat=1.4495, alpha=0.1, ncc_min=0.5)
    ev = {}
    for n_mb, seed in ((20, 9100), (40, 9200)):
        res = learned.evaluate(tg, replace(workload("tiny"), n_mb=n_mb, seed=seed), c, prm)
        ev[str(res["density_per_mm3"])] = {"ncc": res["ncc"], "cnn": res["cnn"]}
    del data
    torch.cuda.empty_cache()
    # paper-scale inference on the bench ensemble's planes
    S = g.n_el // g.P
    A, M = sess.enhance(planes)
    fc = 16                                  # frames per chunk
    P = fc * 2 * S
    heat = torch.empty((P, 4 * g.nz, 4 * g.n_el), dtype=torch.float32, device=dev)
    cap = 1 << 18
    l2 = torch.zeros((cap, 10), dtype=torch.int32, device=dev)
    l3 = torch.zeros((cap, 10), dtype=torch.int32, device=dev)
    n2 = torch.zeros(1, dtype=torch.int32, device=dev)
    n3 = torch.zeros(1, dtype=torch.int32, device=dev)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    split = {"peaks_ms": 0.0, "pair_ms": 0.0, "n2d": 0}

    def infer(timing):
        cnn_ms = 0.0
        for f0 in range(0, F - fc + 1, fc):
            a = A[f0:f0 + fc]
            m = M[f0:f0 + fc]
            e[0].record(stream)
            R.ulm_cnn_forward(c, a, m, 2 * S, P, g.nz, g.n_el, heat)
            e[1].record(stream)
            R.ulm_detect_map(h, sess.t, heat, 4, a, m, fc, 0.3, 0.1, l2, cap, n2)
            e[2].record(stream)
            R.ulm_pair3d(h, sess.t, l2, n2, cap, fc, l3, cap, n3)
            e[3].record(stream)
            if timing:
                torch.cuda.synchronize()
                cnn_ms += e[0].elapsed_time(e[1])
                split["peaks_ms"] += e[1].elapsed_time(e[2])
                split["pair_ms"] += e[2].elapsed_time(e[3])
                split["n2d"] += int(n2.item())
        return cnn_ms

    infer(False)
    torch.cuda.synchronize()
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    infer(False)
    w1.record(stream)
    torch.cuda.synchronize()
    total_ms = w0.elapsed_time(w1)
    cnn_ms = infer(True)
    frames = (F // fc) * fc
    px = frames * 2 * S * g.nz * g.n_el
    flop = px * (2 * 9 * 32 + 2 * 2 * 288 * 32 + 2 * 288 * 16)
    tflops = flop / (cnn_ms / 1e3) / 1e12
    peak = peaks.get("bf16_tflops", 1900.0)
    # algorithmic bytes per plane pixel of the forward pass: input plane read, FP32
    # input written and read, three 32-channel BF16 activations written and read,
    # 16 FP32 heatmap values written -- 460 B against 46 656 FLOP (below the
    # FLOP/B ridge of this GPU: the network is bound by HBM)
    cnn_bytes = px * (4 + 4 + 4 + 3 * (64 + 64) + 64)
    cnn_gbs = cnn_bytes / (cnn_ms / 1e3) / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    R.ulm_cnn_destroy(c)
    return {"train_planes": n_train,
            "train_steps": steps, "batch": 64, "loss_first_last": [hist[0][1], hist[-1][1]],
            "dataset_s": round(build_s, 1), "train_s": round(train_s, 1), "eval_tiny": ev,
            "paper_frames": frames, "localise_ms_per_300_frames": round(total_ms * 300 / frames, 3),
            "heatmap_peaks_ms_per_300_frames": round(split["peaks_ms"] * 300 / frames, 3),
            "pairing_ms_per_300_frames": round(split["pair_ms"] * 300 / frames, 3),
            "n2d_per_300_frames": int(split["n2d"] * 300 / frames),
            "cnn_ms_per_300_frames": round(cnn_ms * 300 / frames, 3),
            "cnn_roofline": {"bound": "hbm", "achieved": round(cnn_gbs, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(cnn_gbs / hbm, 4), "bytes_per_pixel": 460,
                             "kernel": "k_conv_tc (tcgen05 BF16, TMEM accumulators) + k_conv1_fwd",
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                             "tensor": {"achieved": round(tflops, 1), "peak": peak, "unit": "TFLOP/s",
                                        "frac": round(tflops / peak, 4),
                                        "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)"}},
            "status": R.rca_sync_status(h)}


def _oracle_step(O, w, rf, frames):
    """one sample of the FP64 oracle's step: ensemble mean over all frames,
    demodulation, Stage 1, Stage 2 + projection of the listed frames, then
    XDoppler (window clipped at the sample's ends), NCC, peaks and pairing
    of those frames; returns its wall time in seconds"""
    g = w.geom
    t0 = time.perf_counter()
    planes = O.beamform_projections(g, rf, frames=frames)
    O.localize(planes, w.ncc_d, 0.81, 1.45, 0.1, 0.5, g.P)
    return time.perf_counter() - t0


def cpu_baseline(w, rf_tensor, n_frames):
    """The FP64 oracle as it stands on the host cores, best of 3 after one
    warm-up (time.perf_counter), once with every core and once with one
    thread (a smaller sample, the same per-frame work)."""
    import oracle as O
    rf = rf_tensor.cpu().numpy()
    cores = os.cpu_count() or 1
    res = {}
    for label, nth, nfr in (("all_cores", cores, n_frames), ("one_thread", 1, 1)):
        O.set_threads(nth)
        frames = list(range(1, 1 + nfr))
        _oracle_step(O, w, rf, frames)
        best = min(_oracle_step(O, w, rf, frames) for _ in range(3))
        res[label] = {"value": round(nfr / best, 3), "unit": "frames/s", "threads": nth,
                      "sample": f"{nfr} of {w.n_frames} frames (mean over all {w.n_frames}), best of 3 after one "
                                f"warm-up: {best:.2f} s"}
    O.set_threads(cores)
    a = res["all_cores"]
    return {"value": a["value"], "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": a["sample"],
            "one_thread": res["one_thread"],
            "parallel_speedup": round(a["value"] / res["one_thread"]["value"], 2)}


def _scaled(dt, scale, sample):
    """one oracle timing of a bounded sample and its figure for one ensemble"""
    return {"ms_per_ensemble": round(1e3 * dt * scale, 1), "measured_ms": round(1e3 * dt, 3),
            "scale": round(float(scale), 6), "sample": sample}


def cpu_next_rows(w, L, out3d, n3d, planes, slices, F):
    """The FP64 oracle of each row outside the step, timed as it stands on the
    host cores on a bounded sample and scaled to one 300-frame ensemble:
    tracking of the step's whole 3D list, separation of 4096 sampled pixels'
    slow-time signals, the SVD filter of one transmission, motion estimation of
    three frames against frame 0.  Inputs are the ensemble's own data."""
    import numpy as np
    import oracle as O
    from oracle import motion as OM
    from oracle import separation as OSep
    from oracle import svd_filter as OS
    g = w.geom
    out = {}
    n = int(n3d.item())
    rec = out3d[:n].cpu().numpy().view(L.LOC3D).reshape(-1)
    lst = np.zeros(n, dtype=O.LOC3D)
    lst["frame"] = rec["frame"]
    for f in ("x", "y", "z"):
        lst[f] = rec[f].astype(np.float64)
    t0 = time.perf_counter()
    O.track(g, lst, O.track_params())
    dt = time.perf_counter() - t0
    out["tracking"] = _scaled(dt, 1.0, f"the whole 3D list ({n} localisations)")
    rng = np.random.default_rng(0)
    npx = planes.numel() // (2 * F)
    sel = rng.choice(npx, 4096, replace=False)
    a = planes.reshape(F, npx, 2)[:, sel].cpu().numpy().astype(np.float64)
    xs = a[..., 0] + 1j * a[..., 1]
    t0 = time.perf_counter()
    OSep.separate(xs, w.frame_rate, OSep.default_edges(w.frame_rate, 3))
    dt = time.perf_counter() - t0
    out["separation"] = _scaled(dt, npx / 4096, f"4096 of {npx} plane pixels ({F} frames each)")
    b = slices[:, 0:1].cpu().numpy().astype(np.float64)
    sl = b[..., 0] + 1j * b[..., 1]
    t0 = time.perf_counter()
    OS.filter_slices(sl, 16)
    dt = time.perf_counter() - t0
    nt = slices.shape[1]
    out["clutter_svd"] = _scaled(dt, nt, f"1 of {nt} transmissions, {F} frames (rank 16, eigendecomposition)")
    c = slices[:4].cpu().numpy().astype(np.float64)
    sm = c[..., 0] + 1j * c[..., 1]
    t0 = time.perf_counter()
    OM.estimate(g, sm, frames=[1, 2, 3])
    dt = time.perf_counter() - t0
    out["motion"] = _scaled(dt, F / 3, f"3 of {F} frames against frame 0")
    out["cores"] = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return out


def workload_config(w, F, precision, world):
    """the `config` object of the bench line, the same for both arms"""
    g = w.geom
    nt = g.n_tx
    reduced = precision == "reduced"
    rf_gb = F * nt * g.n_el * g.ns * (2 if reduced else 4) / 1e9
    pl_gb = F * 4 * g.n_slab * g.nz * g.n_el * (4 if reduced else 8) / 1e9
    return {"workload": f"{w.name}: RCA {g.n_el}+{g.n_el} el, {nt} tx, {F} frames, {g.ns} samples, "
                        f"planes {g.nz}x{g.n_el}, P={g.P}, NCC d={w.ncc_d}",
            "frames": F, "n_el": g.n_el, "n_tx": nt, "ns": g.ns, "nz": g.nz, "us": g.us, "precision": precision,
            "l2": "inputs larger than L2 (RF %.2f GB, planes %.2f GB)" % (rf_gb, pl_gb),
            "parallelism": f"replicas x{world}"}


def reference_arm(args):
    """The FP64 CPU oracle timed on this host (the method has no other
    reference implementation); rank 0 only.  Every warm-up and timed step is
    one sample of the workload: the oracle's step on one frame of the
    ensemble (its ensemble mean over all frames included), frames taken in
    turn.  The line reports what ran; the per-ensemble figure that the
    sample implies is under its own key."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    import oracle as O
    from synth import generate, workload
    w = workload(args.workload)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    G = generate(w, device=dev, dtype=torch.float32 if dev == "cuda" else torch.float64)
    rf = G.rf.float().cpu().numpy()
    del G
    F = w.n_frames
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    for i in range(args.warmup):
        _oracle_step(O, w, rf, [1 + i % (F - 2)])
    times = [_oracle_step(O, w, rf, [1 + (args.warmup + i) % (F - 2)]) for i in range(args.steps)]
    total = sum(times)
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, F, args.precision, args.gpus),
            "step_unit": "one frame of the ensemble through the oracle's step (mean over all frames, demodulation, "
                         "Stage 1, Stage 2 + projection, XDoppler, NCC, peaks, pairing)",
            "ms_per_ensemble_extrapolated": round(1e3 * F / value, 1),
            "cpu_baseline": {"value": round(value, 3), "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed steps of one frame each after {args.warmup} warm-up "
                                       f"steps, {total:.1f} s"},
            "e2e": {"value": round(value, 3), "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line, rank)


if __name__ == "__main__":
    main()
