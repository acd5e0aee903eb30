"""Seeded Stage-1 slice stacks of a rigidly moving scatterer field, the input
of projection-based motion estimation (Sec. II-A3).

Each scatterer is a complex Gaussian blob on the slice grid (rows at dz / us,
lateral pixels at one pitch); the whole field moves by a given displacement
per frame.  RC slices (transmissions 0 .. K-1) see the field's (x, z)
positions, CR slices (K .. 2K-1) its (y, z) positions.  This module draws
inputs only; it holds none of the motion-estimation arithmetic."""
import numpy as np


def moving_slices(geom, n_frames: int, K: int, displacement, seed: int, n_scat: int = 150,
                  sigma_rows: float = 2.0, sigma_px: float = 1.0, noise: float = 0.0) -> np.ndarray:
    """displacement: [n_frames][3] metres (x, y, z) of the field in each frame.
    Returns slices [F][2K][nzs][N] complex128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N, nzs = geom.n_el, geom.nzs
    row_m = geom.dz / geom.us
    half = 0.5 * (N - 1)
    # scatterers inside the central part of the slice so that the motion keeps them in view
    pos = np.stack([rng.uniform(-0.3 * N * geom.pitch, 0.3 * N * geom.pitch, n_scat),
                    rng.uniform(-0.3 * N * geom.pitch, 0.3 * N * geom.pitch, n_scat),
                    geom.z0 + rng.uniform(0.2, 0.8, n_scat) * (nzs - 1) * row_m], axis=1)
    amp = rng.normal(size=(2 * K, n_scat)) + 1j * rng.normal(size=(2 * K, n_scat))
    out = np.zeros((n_frames, 2 * K, nzs, N), dtype=np.complex128)
    disp = np.asarray(displacement, dtype=np.float64)
    hz, hx = int(np.ceil(5 * sigma_rows)), int(np.ceil(5 * sigma_px))   # blobs cut at 5 sigma
    for f in range(n_frames):
        p = pos + disp[f][None, :]
        for k in range(2 * K):
            lat = p[:, 0] if k < K else p[:, 1]
            lp = lat / geom.pitch + half
            zr = (p[:, 2] - geom.z0) / row_m
            acc = np.zeros((nzs, N), dtype=np.complex128)
            for s in range(n_scat):
                z0, x0 = int(np.floor(zr[s])), int(np.floor(lp[s]))
                za, zb = max(0, z0 - hz), min(nzs, z0 + hz + 2)
                xa, xb = max(0, x0 - hx), min(N, x0 + hx + 2)
                if za >= zb or xa >= xb:
                    continue
                zz = np.arange(za, zb)[:, None].astype(np.float64)
                xx = np.arange(xa, xb)[None, :].astype(np.float64)
                acc[za:zb, xa:xb] += amp[k, s] * np.exp(-(zz - zr[s]) ** 2 / (2 * sigma_rows ** 2)
                                                        - (xx - lp[s]) ** 2 / (2 * sigma_px ** 2))
            if noise > 0:
                acc += noise * (rng.normal(size=acc.shape) + 1j * rng.normal(size=acc.shape))
            out[f, k] = acc
    return out
