"""Gaussian PSF widths for the NCC kernel (Sec. II-A4: "Gaussian-fitted PSF";
the paper does not print its values).

A single scatterer at the volume centre is simulated, beamformed and
XDoppler-enhanced by the oracle; the second moments of A around its peak
(within +-3 pixels, background-subtracted) give sigma_z and sigma_lat in
pixels for the XZ and YZ planes.  ``python -m oracle.psf_fit`` rewrites
tests/golden/psf_sigma.json from the oracle alone.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

import oracle as O
from synth import workload
from synth.rca_sim import synth_rf

GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                      "psf_sigma.json")


def fit(name: str, depth_frac: float = 0.35):
    w = workload(name)
    g = w.geom
    # centre laterally between pixels, at a depth well inside the sample window
    pos = np.array([[[0.0, 0.0, g.z0 + depth_frac * g.nz * g.dz]]] * 3)
    rf = synth_rf(g, torch.tensor(pos), torch.ones(3, 1, dtype=torch.float64)).numpy()
    planes = O.beamform_projections(g, rf, remove_mean=False)
    A, _ = O.xdoppler(planes)
    out = {}
    for axis in (0, 1):
        a = A[1, axis].sum(axis=0)            # sum over slabs: the scatterer sits in one
        i, l = np.unravel_index(np.argmax(a), a.shape)
        win = a[i - 3:i + 4, l - 3:l + 4]
        win = np.clip(win - win.min(), 0, None)
        q = np.arange(-3, 4)
        wz = win.sum(axis=1)
        wl = win.sum(axis=0)
        mz = (wz * q).sum() / wz.sum()
        ml = (wl * q).sum() / wl.sum()
        sz = float(np.sqrt((wz * (q - mz) ** 2).sum() / wz.sum()))
        sl = float(np.sqrt((wl * (q - ml) ** 2).sum() / wl.sum()))
        out[f"axis{axis}"] = {"sig_z": sz, "sig_lat": sl}
    sz = float(np.mean([out["axis0"]["sig_z"], out["axis1"]["sig_z"]]))
    sl = float(np.mean([out["axis0"]["sig_lat"], out["axis1"]["sig_lat"]]))
    return {"sig_z": round(sz, 4), "sig_lat": round(sl, 4), "per_axis": out}


def main():
    res = {name: fit(name) for name in ("tiny",)}
    res["source"] = "oracle/psf_fit.py: moments of the oracle's XDoppler amplitude of one centred scatterer"
    os.makedirs(os.path.dirname(GOLDEN), exist_ok=True)
    with open(GOLDEN, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
