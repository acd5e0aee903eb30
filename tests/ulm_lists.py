"""Comparison of the GPU's 2D and 3D localisation lists with the oracle's,
shared by the GPU parity tests (Sec. II-A4: regional NCC peaks of the
projection planes, paired across the XZ and YZ planes into 3D).

A discrete decision may go either way only where its margin, measured on the
oracle's own FP64 values, is below the float32 error of the quantities it
compares:
  - a pixel's candidate decision (NCC >= ncc_min, A >= alpha M_t, strict /
    non-strict 3x3 regional maximum) within eps_ncc of the NCC threshold or
    of a neighbour's NCC, or within eps_amp M_t of the amplitude threshold;
  - a pairing decision (|z_xz - z_yz| <= 1 px, intensity ratio in
    [0.9, 1.11], mutual minimum of max(I) / min(I)) within tz of the axial
    tolerance, within tr (relative) of a ratio bound, or between two costs
    within tr of each other.
Every other decision must be identical: the 2D key lists are equal outside
the near-tie pixels, and the 3D pairs (as key pairs) are equal in every
(frame, x sub-block, y sub-block) group that holds no differing 2D entry and
no near-tie pairing decision.  When the 2D lists are identical and no group
is excluded, this is the bit-exact comparison of the pair indices."""
import numpy as np

import oracle as O


def key2(r):
    return (int(r["frame"]), int(r["axis"]), int(r["slab"]), int(r["iz"]), int(r["ilat"]))


def group_of(r, P):
    """pairing group (frame, b_x, b_y) of a 2D entry: an XZ entry (axis 0) lies
    in y-slab `slab` at lateral x index ilat, a YZ entry in x-slab `slab` at
    lateral y index ilat"""
    if int(r["axis"]) == 0:
        return (int(r["frame"]), int(r["ilat"]) // P, int(r["slab"]))
    return (int(r["frame"]), int(r["slab"]), int(r["ilat"]) // P)


def near_ties(A, M, prm, eps_ncc, eps_amp, frame_offset=0):
    """(frame, axis, slab, iz, ilat) of the pixels of A [F][2][S][nz][N] whose
    candidate decision is within the margins, from the oracle's NCC"""
    amb = set()
    F, _, S, nz, N = A.shape
    for t in range(F):
        Mt = float(M[t])
        thr = prm["alpha"] * Mt
        for axis in range(2):
            for b in range(S):
                a = np.asarray(A[t, axis, b], dtype=np.float64)
                n = O.ncc_plane(a, prm["d"], prm["sig_z"], prm["sig_lat"], Mt)
                c = n[1:-1, 1:-1]
                ai = a[1:-1, 1:-1]
                nbd = np.full(c.shape, np.inf)
                for di in (-1, 0, 1):
                    for dl in (-1, 0, 1):
                        if di or dl:
                            nb = n[1 + di:nz - 1 + di, 1 + dl:N - 1 + dl]
                            nbd = np.minimum(nbd, np.abs(nb - c))
                maybe = (c >= prm["ncc_min"] - eps_ncc) & (ai >= thr - eps_amp * Mt)
                close = (np.abs(c - prm["ncc_min"]) < eps_ncc) | (np.abs(ai - thr) < eps_amp * Mt) | (nbd < eps_ncc)
                for i, l in zip(*np.nonzero(maybe & close)):
                    amb.add((t + frame_offset, axis, b, int(i) + 1, int(l) + 1))
    return amb


def pair_margin_groups(L, P, tz, tr):
    """groups of the oracle's 2D list L with a pairing decision within the
    margins"""
    groups = {}
    for q, r in enumerate(L):
        g = groups.setdefault(group_of(r, P), ([], []))
        g[int(r["axis"])].append(q)
    bad = set()
    for gk, (xs, ys) in groups.items():
        if not xs or not ys:
            continue
        costs_x = {a: [] for a in xs}
        costs_y = {b: [] for b in ys}
        for a in xs:
            for b in ys:
                dz = abs(float(L[a]["z"]) - float(L[b]["z"]))
                ia, ib = float(L[a]["amp"]), float(L[b]["amp"])
                r = ia / ib
                if abs(dz - 1.0) < tz or abs(r - 0.9) < tr * 0.9 or abs(r - 1.11) < tr * 1.11:
                    bad.add(gk)
                if dz <= 1.0 and 0.9 <= r <= 1.11:
                    c = max(ia, ib) / min(ia, ib)
                    costs_x[a].append(c)
                    costs_y[b].append(c)
        for cs in list(costs_x.values()) + list(costs_y.values()):
            cs.sort()
            if len(cs) > 1 and cs[1] - cs[0] < tr * cs[0]:
                bad.add(gk)
    return bad


def compare(L2o, L3o, L2g, L3g, amb2d, P, pos_tol, ncc_tol, amp_rtol, tz, tr):
    """assert the comparison the module docstring states; returns counts"""
    ko = [key2(r) for r in L2o]
    kg = [key2(r) for r in L2g]
    assert kg == sorted(kg), "GPU 2D list not in (frame, axis, slab, iz, ilat) order"
    assert ko == sorted(ko)
    diff = set(ko) ^ set(kg)
    assert diff <= amb2d, sorted(diff - amb2d)[:10]
    io = {k: q for q, k in enumerate(ko)}
    ig = {k: q for q, k in enumerate(kg)}
    common = set(ko) & set(kg)
    for k in common:
        a, b = L2o[io[k]], L2g[ig[k]]
        assert abs(float(a["z"]) - float(b["z"])) < pos_tol, (k, float(a["z"]), float(b["z"]))
        assert abs(float(a["lat"]) - float(b["lat"])) < pos_tol, (k, float(a["lat"]), float(b["lat"]))
        assert abs(float(a["ncc"]) - float(b["ncc"])) < ncc_tol, (k, float(a["ncc"]), float(b["ncc"]))
        assert abs(float(a["amp"]) - float(b["amp"])) <= amp_rtol * abs(float(a["amp"])), k
    excluded = {group_of(L2o[io[k]], P) for k in diff if k in io}
    excluded |= {group_of(L2g[ig[k]], P) for k in diff if k in ig}
    excluded |= pair_margin_groups(L2o, P, tz, tr)

    def pairs(L2, L3, keys):
        out = []
        for r in L3:
            x, y = L2[int(r["i_xz"])], L2[int(r["i_yz"])]
            assert int(x["axis"]) == 0 and int(y["axis"]) == 1 and group_of(x, P) == group_of(y, P)
            if group_of(x, P) not in excluded:
                out.append((keys[int(r["i_xz"])], keys[int(r["i_yz"])], r))
        return out

    po = pairs(L2o, L3o, ko)
    pg = pairs(L2g, L3g, kg)
    assert [p[:2] for p in po] == [p[:2] for p in pg], "3D pairs differ outside the excluded groups"
    for (_, _, ro), (_, _, rg) in zip(po, pg):
        for f in ("x", "y", "z"):
            assert abs(float(ro[f]) - float(rg[f])) < pos_tol, (f, float(ro[f]), float(rg[f]))
    if not diff and not excluded:
        assert [(int(r["i_xz"]), int(r["i_yz"])) for r in L3g] == [(int(r["i_xz"]), int(r["i_yz"])) for r in L3o]
    return {"n2d": len(ko), "n3d": len(L3o), "n3d_gpu": len(L3g), "diff2d": len(diff), "near_tie_px": len(amb2d),
            "excluded_groups": len(excluded), "pairs_compared": len(po)}
