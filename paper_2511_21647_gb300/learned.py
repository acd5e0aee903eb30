"""Learned localiser: training data from simulated ensembles with known
microbubble positions, training on the GPU with librca's CNN kernels, and
evaluation against the NCC localiser (which stays the fallback and the
reference the localisation error is compared with).

Targets: every visible microbubble is projected onto the XZ plane of its
y-slab and the YZ plane of its x-slab (Sec. II-A4's sub-blocks) and drawn as
a unit Gaussian (sigma = 1 fine pixel) on the 4x grid, plane pixel centres
at fine coordinate 4 i + 1.5.  Input: XDoppler amplitude / frame maximum.
Only the input generation (synth) runs outside librca; the network's forward,
backward, loss, optimiser, targets, peak search and pairing are librca calls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np
import torch

from . import _lib as L
from . import rca as R
from .pipeline import RcaSession, list3d_numpy

UP = 4


def plane_points(w, fields, frames):
    """(plane, z4, x4) rows for the visible MBs of the given frames; plane
    index = (q * 2 + axis) * S + slab with q the frame's position in frames."""
    from synth.rca_sim import visible_mask
    g = w.geom
    u0 = -(g.n_el - 1) / 2.0 * g.pitch
    S = g.n_el // g.P
    vis = visible_mask(w, fields)
    rows = []
    for q, f in enumerate(frames):
        for m in np.nonzero(vis[f])[0]:
            x, y, z = fields.mb_pos[f, m]
            zp, xp, yp = (z - g.z0) / g.dz, (x - u0) / g.pitch, (y - u0) / g.pitch
            by = min(S - 1, max(0, int(round(yp)) // g.P))
            bx = min(S - 1, max(0, int(round(xp)) // g.P))
            rows.append(((q * 2 + 0) * S + by, UP * zp + 1.5, UP * xp + 1.5))
            rows.append(((q * 2 + 1) * S + bx, UP * zp + 1.5, UP * yp + 1.5))
    rows.sort(key=lambda r: r[0])
    return np.array(rows, dtype=np.float32).reshape(-1, 3)


@dataclass
class Dataset:
    A: torch.Tensor       # [P][H][W] amplitude planes
    M: torch.Tensor       # [P] per-plane normaliser (frame maximum)
    target: torch.Tensor  # [P][4H][4W]
    n_planes: int


def build_dataset(geom, workloads, device="cuda") -> Dataset:
    """Simulate, beamform and enhance each ensemble; Gaussian targets from the
    ground truth.  All ensembles must share the geometry."""
    from synth import generate
    As, Ms, Ts = [], [], []
    with RcaSession(geom) as s:
        S = geom.n_el // geom.P
        for w in workloads:
            G = generate(w, device=device, dtype=torch.float32, frame_batch=32)
            planes = s.beamform(G.rf.contiguous())
            A, M = s.enhance(planes)
            F = w.n_frames
            P = F * 2 * S
            pts = torch.from_numpy(plane_points(w, G.fields, range(F))).to(device)
            T = torch.zeros((P, UP * geom.nz, UP * geom.n_el), dtype=torch.float32, device=device)
            R.ulm_cnn_target(s.h, pts, pts.shape[0], P, UP * geom.nz, UP * geom.n_el, 1.0, T)
            As.append(A.reshape(P, geom.nz, geom.n_el))
            Ms.append(M.repeat_interleave(2 * S))
            Ts.append(T)
        torch.cuda.synchronize()
    A = torch.cat(As)
    return Dataset(A, torch.cat(Ms), torch.cat(Ts), A.shape[0])


def train(cnn, data: Dataset, steps: int, batch: int = 64, seed: int = 0, log_every: int = 0):
    """Adam steps on random mini-batches; returns the loss history (host)."""
    H, W = data.A.shape[1], data.A.shape[2]
    gen = torch.Generator(device="cpu").manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=data.A.device)
    hist = []
    for step in range(steps):
        idx = torch.randint(0, data.n_planes, (batch,), generator=gen).to(data.A.device)
        A = data.A.index_select(0, idx).contiguous()
        M = data.M.index_select(0, idx).contiguous()
        T = data.target.index_select(0, idx).contiguous()
        R.ulm_cnn_train_step(cnn, A, M, 1, batch, H, W, T, loss, True)
        if log_every and (step % log_every == 0 or step == steps - 1):
            hist.append((step, float(loss.item())))
    torch.cuda.synchronize()
    return hist


def match(w, fields, frames, L3, max_dist=0.2e-3):
    """Mutual nearest-neighbour matching of 3D detections to the visible
    ground truth within max_dist (per frame).  Returns (matches, detections,
    visible, squared errors)."""
    from synth.rca_sim import visible_mask
    g = w.geom
    u0 = -(g.n_el - 1) / 2.0 * g.pitch
    vis = visible_mask(w, fields)
    n_match, n_vis, sq = 0, 0, []
    for q, f in enumerate(frames):
        gt = fields.mb_pos[f][vis[f]]
        n_vis += len(gt)
        det = L3[L3["frame"] == q]
        if len(gt) == 0 or len(det) == 0:
            continue
        P = np.stack([u0 + det["x"] * g.pitch, u0 + det["y"] * g.pitch, g.z0 + det["z"] * g.dz], axis=1)
        d = np.linalg.norm(P[:, None, :] - gt[None, :, :], axis=2)
        a = d.argmin(axis=1)
        bmin = d.argmin(axis=0)
        for i, j in enumerate(a):
            if bmin[j] == i and d[i, j] <= max_dist:
                n_match += 1
                sq.append(d[i, j] ** 2)
    return n_match, len(L3), n_vis, sq


def evaluate(geom, w, cnn, ncc_prm, score_min=0.3, alpha=0.1, device="cuda"):
    """Localise one held-out ensemble with the NCC path and with the CNN
    heatmaps; compare both against the ground truth."""
    from synth import generate
    G = generate(w, device=device, dtype=torch.float32, frame_batch=32)
    F = w.n_frames
    S = geom.n_el // geom.P
    out = {}
    with RcaSession(geom) as s:
        planes = s.beamform(G.rf.contiguous())
        o2, n2, o3, n3 = s.localize(planes, ncc_prm)
        torch.cuda.synchronize()
        L3 = list3d_numpy(o3, int(n3.item()))
        out["ncc"] = _metrics(*match(w, G.fields, range(F), L3))
        A, M = s.enhance(planes)
        P = F * 2 * S
        heat = torch.empty((P, UP * geom.nz, UP * geom.n_el), dtype=torch.float32, device=device)
        R.ulm_cnn_forward(cnn, A, M, 2 * S, P, geom.nz, geom.n_el, heat)
        cap = 1 << 16
        l2 = torch.zeros((cap, 10), dtype=torch.int32, device=device)
        n2d = torch.zeros(1, dtype=torch.int32, device=device)
        R.ulm_detect_map(s.h, s.t, heat, UP, A, M, F, score_min, alpha, l2, cap, n2d)
        l3 = torch.zeros((cap, 10), dtype=torch.int32, device=device)
        n3d = torch.zeros(1, dtype=torch.int32, device=device)
        R.ulm_pair3d(s.h, s.t, l2, n2d, cap, F, l3, cap, n3d)
        torch.cuda.synchronize()
        out["cnn"] = _metrics(*match(w, G.fields, range(F), list3d_numpy(l3, int(n3d.item()))))
        out["status"] = s.sync_status()
    g = w.geom
    vol = g.nz * g.dz * (g.n_el * g.pitch) ** 2 * 1e9
    out["density_per_mm3"] = round(w.n_mb / vol, 4)
    return out


def _metrics(n_match, n_det, n_vis, sq):
    return {"matches": n_match, "detections": n_det, "visible": n_vis,
            "detection_accuracy": round(n_match / n_det, 4) if n_det else 0.0,
            "missing_rate": round(1 - n_match / n_vis, 4) if n_vis else 0.0,
            "rmse_um": round(1e6 * math.sqrt(np.mean(sq)), 2) if sq else None}


def training_workloads(n_ensembles: int, frames: int = 64, seed: int = 6000, mb_range=(10, 60)):
    """tiny-geometry ensembles (config-1 generator) with MB counts spread over
    mb_range (about 0.03 to 0.16 MB/mm^3)."""
    from synth import workload
    rng = np.random.default_rng(seed)
    base = workload("tiny")
    return [replace(base, name=f"train{q}", n_frames=frames, n_mb=int(rng.integers(*mb_range)), seed=seed + q)
            for q in range(n_ensembles)]
