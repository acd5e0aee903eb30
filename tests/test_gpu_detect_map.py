"""Peaks of the learned localiser's heatmaps (ulm_detect_map): the GPU list
equals a plain numpy statement of the same rule on seeded random maps.  On
the fine grid (up x the plane), pixel (i, j) off the border is a candidate
when its score s >= score_min, the plane amplitude at (i // up, j // up) is
at least alpha M_t, and s is above every earlier 3 x 3 neighbour (the row
above and the left pixel) and at least every later one (raster tie rule);
positions are refined by a three-point parabola per axis (clipped to half a
pixel) and mapped back to plane pixels; entries come out by plane (frame,
axis, slab), then in raster order."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

UP = 4


def para(fm, f0, fp):
    den = np.float32(np.float32(fm - np.float32(2) * f0) + fp)
    if den >= 0:
        return np.float32(0)
    dl = np.float32(np.float32(fm - fp) / np.float32(np.float32(2) * den))
    return np.float32(min(np.float32(0.5), max(np.float32(-0.5), dl)))


def reference(heat, A, M, S, score_min, alpha):
    out = []
    P, H4, W4 = heat.shape
    N = W4 // UP
    half, inv = np.float32(0.5 * (UP - 1)), np.float32(1.0 / UP)
    for plane in range(P):
        t, axis, b = plane // (2 * S), (plane // S) % 2, plane % S
        hm, ap = heat[plane], A[plane]
        thr = np.float32(alpha) * M[t]
        for i in range(1, H4 - 1):
            row = hm[i]
            for j in np.nonzero(row[1:W4 - 1] >= score_min)[0] + 1:
                c = row[j]
                if not ap[i // UP, j // UP] >= thr:
                    continue
                nb = hm[i - 1:i + 2, j - 1:j + 2]
                if not (c > nb[0].max() and c > nb[1, 0] and c >= nb[1, 2] and c >= nb[2].max()):
                    continue
                z = np.float32(np.float32(np.float32(i) + para(hm[i - 1, j], c, hm[i + 1, j])) - half) * inv
                lat = np.float32(np.float32(np.float32(j) + para(row[j - 1], c, row[j + 1])) - half) * inv
                out.append((t, axis, b, i // UP, j // UP, float(z), float(lat), float(c), float(ap[i // UP, j // UP])))
    return out


@pytest.mark.parametrize("seed", [3, 4])
def test_detect_map_matches_numpy_rule(seed):
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import RcaSession, list2d_numpy
    from synth import workload
    g = workload("tiny").geom
    F, S = 3, g.n_el // g.P
    P, H4, W4 = F * 2 * S, g.nz * UP, g.n_el * UP
    rng = np.random.default_rng(seed)
    raw = rng.standard_normal((P, H4 + 4, W4 + 4)).astype(np.float32)
    # smoothed noise: isolated maxima plus plateaus of equal values (ties)
    heat = (raw[:, :-4, :-4] + raw[:, 2:-2, 2:-2] + raw[:, 4:, 4:] + raw[:, 1:-3, 3:-1]) / np.float32(4)
    heat[:, 40:44, 60:64] = np.float32(1.25)
    heat = np.ascontiguousarray(heat, dtype=np.float32)
    A = rng.uniform(0, 1, (P, g.nz, g.n_el)).astype(np.float32)
    M = np.ones(F, dtype=np.float32)
    score_min, alpha = 1.2, 0.3          # sparse enough to stay inside every strip's 96 slots
    ref = reference(heat, A, M, S, np.float32(score_min), alpha)
    assert 100 < len(ref) < 20000
    cap = 1 << 16
    with RcaSession(g) as s:
        out = torch.zeros((cap, 10), dtype=torch.int32, device="cuda")
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        rca.ulm_detect_map(s.h, s.t, torch.from_numpy(heat).cuda(), UP, torch.from_numpy(A).cuda(),
                           torch.from_numpy(M).cuda(), F, score_min, alpha, out, cap, n)
        torch.cuda.synchronize()
        assert s.sync_status() == 0
        got = list2d_numpy(out, int(n.item()))
    assert len(got) == len(ref)
    for r, e in zip(got, ref):
        assert (int(r["frame"]), int(r["axis"]), int(r["slab"]), int(r["iz"]), int(r["ilat"])) == e[:5]
        assert abs(float(r["z"]) - e[5]) < 1e-5 and abs(float(r["lat"]) - e[6]) < 1e-5
        assert float(r["ncc"]) == e[7] and float(r["amp"]) == e[8]
