"""Synthetic RCA point-scatterer channel data.

Acquisition model (stands in for the paper's Field II simulations and in-vivo
pig-kidney acquisitions, Sec. II-C and Sec. III-C, which are not available):

* Ideal row-column array of ``n_el`` rows and ``n_el`` columns, pitch ``p``.
  Element centres ``u_e = (e - (n_el-1)/2) p``; aperture ``L = n_el p``.
  Columns are strips parallel to y at x = u_e (they resolve x); rows are
  strips parallel to x at y = u_e (they resolve y).
* Transmissions 0..K-1 are RC (row transmit, column receive) steered by
  ``theta_k`` in the y-z plane; K..2K-1 are CR (column transmit, row receive)
  steered in the x-z plane (Sec. II-A1, Fig. 1h).
* RC echo delay of a point (x, y, z) on column e:
  ``(z cos th + y sin th + (L/2)|sin th|)/c + sqrt((x-u_e)^2 + z^2)/c``;
  CR swaps x and y.
* Pulse: Gaussian envelope at fc with 65 % -6 dB fractional bandwidth
  (Sec. II-C), truncated at 4 sigma.
* Sample times ``t_n = t0 + n/fs`` with ``t0 = 2 z0 / c``.
* Microbubbles move linearly between frames (frame rate 400 Hz, Sec. II-C)
  and respawn uniformly with a new id when they leave the volume; tissue is
  static (optionally a rigid axial sinusoid) and 40 dB brighter; white
  Gaussian noise at 30 dB SNR w.r.t. the MB-only signal.

Random numbers come from numpy's PCG64 (platform independent); the echo sum
runs in torch on any device so the paper-scale ensemble can be generated on the
GPU.  Nothing here beamforms or localises.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Dict, List, Optional, Tuple

import numpy as np
import torch

DEG = math.pi / 180.0


def tx_angles(k_per_family: int, single_rc: float = 3.0, single_cr: float = -3.0):
    """Steering angles (radians) for one family of K transmissions.

    K = 1 uses the tiny workload's single +3 deg (RC) / -3 deg (CR) pair;
    K >= 2 spreads K angles evenly over [-3 deg, +3 deg].
    Returns (ang_rc, ang_cr).
    """
    if k_per_family == 1:
        return (single_rc * DEG,), (single_cr * DEG,)
    a = tuple((-3.0 + 6.0 * j / (k_per_family - 1)) * DEG for j in range(k_per_family))
    return a, a


@dataclass(frozen=True)
class RcaGeometry:
    n_el: int
    pitch: float
    fc: float
    fs: float
    c: float
    z0: float
    dz: float
    nz: int
    ns: int
    fnum: float
    P: int
    ang_rc: Tuple[float, ...]
    ang_cr: Tuple[float, ...]
    us: int = 2          # Stage-1 slice rows per plane pixel (axial oversampling)

    @property
    def nzs(self) -> int:
        return (self.nz - 1) * self.us + 1

    @property
    def K(self) -> int:
        return len(self.ang_rc)

    @property
    def n_tx(self) -> int:
        return 2 * self.K

    @property
    def t0(self) -> float:
        return 2.0 * self.z0 / self.c

    @property
    def L(self) -> float:
        return self.n_el * self.pitch

    @property
    def n_slab(self) -> int:
        return self.n_el // self.P

    @property
    def angles(self) -> Tuple[float, ...]:
        return tuple(self.ang_rc) + tuple(self.ang_cr)

    def element_pos(self) -> np.ndarray:
        return (np.arange(self.n_el) - (self.n_el - 1) / 2.0) * self.pitch

    def pulse_sigma(self) -> float:
        # Gaussian envelope exp(-t^2/2s^2): -6 dB full bandwidth 0.65 fc.
        return math.sqrt(2.0 * math.log(2.0)) / (math.pi * 0.65 * self.fc)


@dataclass(frozen=True)
class RcaWorkload:
    name: str
    geom: RcaGeometry
    n_frames: int
    n_mb: int
    n_tissue: int
    seed: int
    frame_rate: float = 400.0
    mb_speed: Tuple[float, float] = (5e-3, 20e-3)
    mb_amp_db: float = 5.0
    tissue_amp: float = 100.0
    snr_db: float = 30.0
    tissue_motion_amp: float = 0.0
    tissue_motion_hz: float = 1.0
    ncc_d: int = 5

    @property
    def rf_shape(self):
        g = self.geom
        return (self.n_frames, g.n_tx, g.n_el, g.ns)

    @property
    def planes_shape(self):
        g = self.geom
        return (self.n_frames, 2, 2, g.n_slab, g.nz, g.n_el)


def _tiny_geom(K: int = 1) -> RcaGeometry:
    rc, cr = tx_angles(K)
    return RcaGeometry(n_el=32, pitch=0.214e-3, fc=7.8e6, fs=31.2e6, c=1540.0,
                       z0=5e-3, dz=0.1e-3, nz=80, ns=256, fnum=1.0, P=8,
                       ang_rc=rc, ang_cr=cr)


def _paper_geom() -> RcaGeometry:
    rc, cr = tx_angles(4)
    return RcaGeometry(n_el=128, pitch=0.214e-3, fc=7.8e6, fs=31.2e6, c=1540.0,
                       z0=20e-3, dz=0.1e-3, nz=250, ns=1024, fnum=1.0, P=8,
                       ang_rc=rc, ang_cr=cr)


WORKLOADS: Dict[str, RcaWorkload] = {
    # 32+32 elements, 2 tx (+3 RC / -3 CR), 64 frames, 256 samples, 80x32 planes,
    # 20 MBs + 200 static tissue scatterers, NCC d = 5.
    "tiny": RcaWorkload("tiny", _tiny_geom(1), n_frames=64, n_mb=20, n_tissue=200,
                        seed=1000, ncc_d=5),
    # 128+128 elements, 8 tx (4 RC + 4 CR over -3..+3 deg), 300 frames, 1024
    # samples, 250x128 planes, 500 MBs + 20k tissue with a 0.2 mm 1 Hz axial
    # sinusoid, NCC d = 11 (Sec. II-C).
    "paper": RcaWorkload("paper", _paper_geom(), n_frames=300, n_mb=500, n_tissue=20000,
                         seed=2000, tissue_motion_amp=0.2e-3, ncc_d=11),
}


def workload(name: str, **kw) -> RcaWorkload:
    w = WORKLOADS[name]
    return replace(w, **kw) if kw else w


def batch_workloads(n: int = 16, seed: int = 4000) -> List[RcaWorkload]:
    """Uneven ensembles for the batched form: tiny geometry, frames uniform in
    100..600, transmit count 2K in {2, 4, 8}, per-ensemble seeds."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        F = int(rng.integers(100, 601))
        n_tx = int(rng.choice([2, 4, 8]))
        g = _tiny_geom(n_tx // 2)
        out.append(RcaWorkload(f"batch{i}", g, n_frames=F, n_mb=20, n_tissue=200,
                               seed=seed + 1 + i, ncc_d=5))
    return out


# ---------------------------------------------------------------------------
# scatterer fields
# ---------------------------------------------------------------------------

@dataclass
class ScattererFields:
    """Per-frame scatterer positions (m) and amplitudes."""
    mb_pos: np.ndarray      # [F, n_mb, 3]
    mb_amp: np.ndarray      # [F, n_mb]
    mb_id: np.ndarray       # [F, n_mb]
    tissue_pos: np.ndarray  # [F, n_tissue, 3]
    tissue_amp: np.ndarray  # [n_tissue]


def _volume_bounds(g: RcaGeometry):
    h = g.L / 2.0
    return np.array([-h, -h, g.z0]), np.array([h, h, g.z0 + g.nz * g.dz])


def scatterer_fields(w: RcaWorkload) -> ScattererFields:
    g = w.geom
    rng = np.random.Generator(np.random.PCG64(w.seed))
    lo, hi = _volume_bounds(g)
    F, n = w.n_frames, w.n_mb

    def rand_pos(m):
        return lo + (hi - lo) * rng.random((m, 3))

    def rand_vel(m):
        d = rng.standard_normal((m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        s = rng.uniform(w.mb_speed[0], w.mb_speed[1], size=(m, 1))
        return d * s

    def rand_amp(m):
        return 10.0 ** (rng.uniform(-w.mb_amp_db, w.mb_amp_db, size=m) / 20.0)

    pos = rand_pos(n)
    vel = rand_vel(n)
    amp = rand_amp(n)
    ids = np.arange(n)
    next_id = n
    dt = 1.0 / w.frame_rate
    mb_pos = np.empty((F, n, 3))
    mb_amp = np.empty((F, n))
    mb_id = np.empty((F, n), dtype=np.int64)
    for f in range(F):
        if f > 0:
            pos = pos + vel * dt
            out = np.any((pos < lo) | (pos > hi), axis=1)
            m = int(out.sum())
            if m:
                pos[out] = rand_pos(m)
                vel[out] = rand_vel(m)
                amp[out] = rand_amp(m)
                ids = ids.copy()
                ids[out] = np.arange(next_id, next_id + m)
                next_id += m
        mb_pos[f] = pos
        mb_amp[f] = amp
        mb_id[f] = ids

    t_pos0 = rand_pos(w.n_tissue)
    t_amp = w.tissue_amp * rng.choice([-1.0, 1.0], size=w.n_tissue)
    t = np.arange(F) * dt
    dz = w.tissue_motion_amp * np.sin(2 * math.pi * w.tissue_motion_hz * t)
    tissue_pos = np.broadcast_to(t_pos0, (F, w.n_tissue, 3)).copy()
    tissue_pos[:, :, 2] += dz[:, None]
    return ScattererFields(mb_pos, mb_amp, mb_id, tissue_pos, t_amp)


# ---------------------------------------------------------------------------
# echo synthesis
# ---------------------------------------------------------------------------

def synth_rf(g: RcaGeometry, pos: torch.Tensor, amp: torch.Tensor, *,
             max_entries: Optional[int] = None) -> torch.Tensor:
    """Sum of pulse echoes for one batch of frames.

    pos: [F, S, 3] positions (m), amp: [F, S] (or [S]) amplitudes, on the
    target device and dtype.  Returns rf [F, 2K, n_el, ns].
    """
    dev, dt = pos.device, pos.dtype
    F, S, _ = pos.shape
    if amp.dim() == 1:
        amp = amp.expand(F, S)
    E, ns, nt = g.n_el, g.ns, g.n_tx
    u = torch.as_tensor(g.element_pos(), device=dev, dtype=dt)
    th = torch.as_tensor(np.array(g.angles), device=dev, dtype=dt)
    sig = g.pulse_sigma()
    half = 4.0 * sig
    W = int(math.floor(2 * half * g.fs)) + 2
    woff = torch.arange(W, device=dev, dtype=dt)
    rf = torch.zeros(F * nt * E * ns, device=dev, dtype=dt)
    cos_t, sin_t = torch.cos(th), torch.sin(th)
    if max_entries is None:
        max_entries = (1 << 25) if dev.type == "cuda" else (1 << 22)
    chunk = max(1, max_entries // (F * nt * E * W))
    is_cr = torch.arange(nt, device=dev) >= g.K
    base = (torch.arange(F, device=dev)[:, None, None] * nt
            + torch.arange(nt, device=dev)[None, :, None]) * E \
        + torch.arange(E, device=dev)[None, None, :]          # [F, nt, E]
    base = base * ns
    for s0 in range(0, S, chunk):
        p = pos[:, s0:s0 + chunk]                              # [F, s, 3]
        a = amp[:, s0:s0 + chunk]
        x, y, z = p[..., 0], p[..., 1], p[..., 2]
        trans = torch.where(is_cr[None, :, None], x[:, None, :], y[:, None, :])  # [F, nt, s]
        recv = torch.where(is_cr[None, :, None], y[:, None, :], x[:, None, :])
        zz = z[:, None, :]
        t_tx = (zz * cos_t[None, :, None] + trans * sin_t[None, :, None]
                + 0.5 * g.L * torch.abs(sin_t)[None, :, None]) / g.c      # [F, nt, s]
        lat = recv[:, :, None, :] - u[None, None, :, None]                  # [F, nt, E, s]
        t_rx = torch.sqrt(lat * lat + zz[:, :, None, :] ** 2) / g.c
        nc = (t_tx[:, :, None, :] + t_rx - g.t0) * g.fs                     # [F, nt, E, s]
        n_lo = torch.ceil(nc - half * g.fs)
        n = n_lo[..., None] + woff                                          # [F, nt, E, s, W]
        tt = (n - nc[..., None]) / g.fs
        val = torch.exp(-tt * tt / (2 * sig * sig)) * torch.cos(2 * math.pi * g.fc * tt)
        ok = (tt.abs() <= half) & (n >= 0) & (n <= ns - 1)
        val = torch.where(ok, val * a[:, None, None, :, None], torch.zeros((), device=dev, dtype=dt))
        idx = base[..., None, None] + torch.where(ok, n, torch.zeros((), device=dev, dtype=dt)).long()
        if dev.type == "cuda":
            # one scatterer per call: its windows never share a sample (entries outside
            # a window add zero), so the atomic adds of a call do not collide and the
            # sum does not depend on their order -- the same RF on every run
            for q in range(idx.shape[3]):
                rf.index_add_(0, idx[:, :, :, q].reshape(-1), val[:, :, :, q].reshape(-1))
        else:
            rf.index_add_(0, idx.reshape(-1), val.reshape(-1))
    return rf.view(F, nt, E, ns)


@dataclass
class Generated:
    workload: RcaWorkload
    rf: torch.Tensor            # [F, 2K, E, ns] float32
    fields: ScattererFields
    noise_sigma: float


def generate(w: RcaWorkload, device: str = "cpu", dtype=torch.float64,
             frame_batch: Optional[int] = None, with_tissue: bool = True,
             with_noise: bool = True, with_mb: bool = True) -> Generated:
    """Generate the ensemble's RF channel data (float32) for a workload."""
    g = w.geom
    fields = scatterer_fields(w)
    F = w.n_frames
    # frames per synthesis call: on the GPU 32 by default (the per-scatterer
    # accumulation there issues one call per scatterer and batch)
    fb = frame_batch or (32 if str(device).startswith("cuda") else 1)
    out = torch.empty((F, g.n_tx, g.n_el, g.ns), dtype=torch.float32, device=device)
    ss_mb = 0.0
    for f0 in range(0, F, fb):
        f1 = min(F, f0 + fb)
        acc = torch.zeros((f1 - f0, g.n_tx, g.n_el, g.ns), dtype=dtype, device=device)
        if with_mb and w.n_mb:
            mb = synth_rf(g, torch.as_tensor(fields.mb_pos[f0:f1], device=device, dtype=dtype),
                          torch.as_tensor(fields.mb_amp[f0:f1], device=device, dtype=dtype))
            ss_mb += float((mb.double() ** 2).sum())
            acc += mb
        if with_tissue and w.n_tissue:
            acc += synth_rf(g, torch.as_tensor(fields.tissue_pos[f0:f1], device=device, dtype=dtype),
                            torch.as_tensor(fields.tissue_amp, device=device, dtype=dtype))
        out[f0:f1] = acc.to(torch.float32)
    sigma = 0.0
    if with_noise:
        rms = math.sqrt(ss_mb / out.numel()) if ss_mb > 0 else 1.0
        sigma = rms / (10.0 ** (w.snr_db / 20.0))
        rng = np.random.Generator(np.random.PCG64(w.seed + 7919))
        per = g.n_tx * g.n_el * g.ns
        for f in range(F):
            nz = rng.standard_normal(per, dtype=np.float32) * np.float32(sigma)
            out[f] += torch.from_numpy(nz).view(g.n_tx, g.n_el, g.ns).to(device)
    return Generated(w, out, fields, sigma)


def quantize_int16(rf: torch.Tensor):
    """Per-channel int16 quantisation: scale[k, e] = max|rf[:, k, e, :]| / 32767,
    q = round-half-even(rf / scale).  Returns (q int16, scale float32 [2K, E])."""
    amax = rf.abs().amax(dim=(0, 3))
    scale = (amax / 32767.0).to(torch.float32)
    safe = torch.where(scale > 0, scale, torch.ones_like(scale))
    q = torch.round(rf / safe[None, :, :, None]).clamp_(-32767, 32767).to(torch.int16)
    return q, scale


def visible_mask(w: RcaWorkload, fields: ScattererFields) -> np.ndarray:
    """[F, n_mb] True where every transmission's nearest-element echo lies
    4 sigma inside the sample window."""
    g = w.geom
    sig = g.pulse_sigma()
    lo = g.t0 + 4 * sig
    hi = g.t0 + (g.ns - 1) / g.fs - 4 * sig
    x, y, z = fields.mb_pos[..., 0], fields.mb_pos[..., 1], fields.mb_pos[..., 2]
    ok = np.ones(x.shape, dtype=bool)
    for k, th in enumerate(g.angles):
        trans = y if k < g.K else x
        tau = (z * math.cos(th) + trans * math.sin(th) + 0.5 * g.L * abs(math.sin(th))) / g.c + z / g.c
        ok &= (tau >= lo) & (tau <= hi)
    return ok
