"""Seeded 3D localisation lists for the tracking step (Sec. II-A6 input).

A scene is a set of microbubbles moving along smooth paths (straight or
gently curved, speeds of a few mm/s at the frame rate), each seen in a run
of consecutive frames with localisation noise, plus spurious detections.  The
output is what the pairing step produces: a frame-major list of (frame, x,
y, z) in plane pixels (x, y lateral pixels, z depth rows), rounded to float32.
This module draws positions only; it holds none of the tracking arithmetic.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class TrackScene:
    frame: np.ndarray      # int32 [n]
    x: np.ndarray          # float32 [n] lateral pixel (x)
    y: np.ndarray          # float32 [n] lateral pixel (y)
    z: np.ndarray          # float32 [n] depth row
    truth: np.ndarray      # int32 [n]: index of the bubble that made the point (-1: spurious)


def track_scene(geom, n_frames: int, n_bubbles: int, seed: int, *, step_m=(20e-6, 60e-6), noise_m=5e-6,
                curvature=0.2, run=(8, 40), n_spurious_per_frame: int = 2) -> TrackScene:
    """Bubbles start at uniform positions inside the plane extent, move with a
    speed drawn from step_m (metres per frame) in a random direction that
    turns by up to `curvature` radians over their run, and are seen for a
    run of consecutive frames drawn from `run`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N, pitch, dz, z0, nz = geom.n_el, geom.pitch, geom.dz, geom.z0, geom.nz
    half = 0.5 * (N - 1)
    pts = []
    for b in range(n_bubbles):
        length = int(rng.integers(run[0], run[1] + 1))
        t0 = int(rng.integers(-length // 2, n_frames))
        p = np.array([rng.uniform(-half * pitch, half * pitch), rng.uniform(-half * pitch, half * pitch),
                      rng.uniform(z0, z0 + (nz - 1) * dz)])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        axis = rng.normal(size=3)
        axis -= axis.dot(d) * d
        axis /= np.linalg.norm(axis)
        speed = rng.uniform(*step_m)
        turn = rng.uniform(-curvature, curvature) / max(length - 1, 1)
        for k in range(length):
            t = t0 + k
            if 0 <= t < n_frames:
                q = p + rng.normal(scale=noise_m, size=3)
                pts.append((t, q[0] / pitch + half, q[1] / pitch + half, (q[2] - z0) / dz, b))
            p = p + speed * d
            # rotate the direction about `axis` by `turn`
            c, s = np.cos(turn), np.sin(turn)
            d, axis = c * d + s * np.cross(axis, d), axis
    for t in range(n_frames):
        for _ in range(n_spurious_per_frame):
            pts.append((t, rng.uniform(0, N - 1), rng.uniform(0, N - 1), rng.uniform(0, nz - 1), -1))
    pts.sort(key=lambda r: (r[0], r[1], r[2], r[3]))
    a = np.array(pts, dtype=np.float64).reshape(-1, 5)
    return TrackScene(a[:, 0].astype(np.int32), a[:, 1].astype(np.float32), a[:, 2].astype(np.float32),
                      a[:, 3].astype(np.float32), a[:, 4].astype(np.int32))
