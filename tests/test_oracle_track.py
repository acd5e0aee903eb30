"""Pins of the oracle's fixed-length tracking (Sec. II-A6): the least-squares
quadratic against numpy's polynomial fit and exact quadratic paths, the
pairing against brute-force optimal assignment on sparse scenes, the
rejection rules on paths whose turn and speed change are known in closed
form, the density accumulation on a path whose voxel counts are known, and
the velocity sums on constant-velocity and accelerating paths."""
import math

import numpy as np
import pytest

import oracle as O

LEN = 10


def _geom(tiny):
    return tiny.geom


def _to_list(g, frames, pos_m):
    """frames [n], positions [n][3] in metres -> oracle 3D list (pixel units)"""
    half = 0.5 * (g.n_el - 1)
    L = np.zeros(len(frames), dtype=O.LOC3D)
    L["frame"] = frames
    L["x"] = pos_m[:, 0] / g.pitch + half
    L["y"] = pos_m[:, 1] / g.pitch + half
    L["z"] = (pos_m[:, 2] - g.z0) / g.dz
    return L


def _smoothed(tr, tau):
    m, q = 0.5 * (LEN - 1), (LEN * LEN - 1) / 12.0
    f1 = tau - m
    f2 = f1 * f1 - q
    return np.stack([tr["a"][ax, 0] + tr["a"][ax, 1] * f1 + tr["a"][ax, 2] * f2 for ax in range(3)], axis=-1)


def _path(p0, v, acc, tau):
    return p0[None, :] + v[None, :] * tau[:, None] + acc[None, :] * tau[:, None] ** 2


def test_quadratic_fit_matches_polyfit_and_reproduces_quadratics(tiny):
    g = _geom(tiny)
    tau = np.arange(LEN, dtype=np.float64)
    rng = np.random.default_rng(5)
    prm = O.track_params(max_step=1e-3)
    for noisy in (False, True):
        p = _path(np.array([1e-3, -0.5e-3, 7e-3]), np.array([30e-6, -20e-6, 10e-6]), np.array([1e-6, 2e-6, -1.5e-6]), tau)
        if noisy:
            p = p + rng.normal(scale=4e-6, size=p.shape)
        L = _to_list(g, np.arange(LEN), p)
        _, tr, _ = O.track(g, L, prm)
        assert len(tr) == 1 and tr[0]["first"] == 0 and tr[0]["frame0"] == 0
        got = _smoothed(tr[0], tau)
        # the positions the oracle saw (pixel round trip) fitted by numpy
        pm = np.stack([(L["x"] - 0.5 * (g.n_el - 1)) * g.pitch, (L["y"] - 0.5 * (g.n_el - 1)) * g.pitch,
                       g.z0 + L["z"] * g.dz], axis=1)
        ref = np.stack([np.polyval(np.polyfit(tau, pm[:, ax], 2), tau) for ax in range(3)], axis=1)
        assert np.max(np.abs(got - ref)) < 1e-12
        if not noisy:
            assert np.max(np.abs(got - p)) < 1e-12


def test_separated_bubbles_keep_their_identity_and_short_runs_make_no_track(tiny):
    g = _geom(tiny)
    tau = np.arange(14, dtype=np.float64)
    a = _path(np.array([-2e-3, 0.0, 6e-3]), np.array([40e-6, 0, 0]), np.zeros(3), tau)        # 14 frames
    b = _path(np.array([2e-3, 1e-3, 9e-3]), np.array([0, -30e-6, 20e-6]), np.zeros(3), tau)   # 14 frames
    c = _path(np.array([0.0, -2e-3, 8e-3]), np.array([25e-6, 25e-6, 0]), np.zeros(3), tau[:6])  # 6 frames
    rows = [(t, 0, a[t]) for t in range(14)] + [(t, 1, b[t]) for t in range(14)] + [(t, 2, c[t]) for t in range(6)]
    rows.sort(key=lambda r: (r[0], r[1]))
    frames = np.array([r[0] for r in rows])
    who = np.array([r[1] for r in rows])
    L = _to_list(g, frames, np.array([r[2] for r in rows]))
    succ, tr, _ = O.track(g, L, O.track_params())
    # every link joins the same bubble in consecutive frames
    for i, j in enumerate(succ):
        if j >= 0:
            assert who[j] == who[i] and frames[j] == frames[i] + 1
    assert np.sum(succ >= 0) == 13 + 13 + 5
    # bubbles a and b start 14 - 10 + 1 = 5 tracks each; c (6 frames) none
    assert len(tr) == 10
    assert sorted(set(who[tr["first"]])) == [0, 1]
    assert np.all(tr["accepted"] == 1)
    assert np.allclose(tr["mean_speed"][who[tr["first"]] == 0], 40e-6, rtol=1e-9)


def test_link_radius_and_mutual_nearest_rule(tiny):
    g = _geom(tiny)
    r = 150e-6
    # frame 0: A at 0, B at 100 um; frame 1: C at 60 um (nearest to A is C, nearest to C is B)
    pos = np.array([[0.0, 0, 6e-3], [100e-6, 0, 6e-3], [60e-6, 0, 6e-3], [2e-3, 0, 6e-3], [2e-3 + r * 1.01, 0, 6e-3]])
    L = _to_list(g, np.array([0, 0, 1, 0, 1]), pos)
    order = np.argsort(L["frame"], kind="stable")
    L = L[order]                                   # frame-major: A, B, D, C, E
    succ = O.track_link(g, L, r)
    idx = {k: int(np.where(order == k)[0][0]) for k in range(5)}
    assert succ[idx[1]] == idx[2]                  # B -> C (mutual)
    assert succ[idx[0]] == -1                      # A's nearest C prefers B
    assert succ[idx[3]] == -1                      # D -> E is 1.01 x the radius away


def test_pairing_equals_optimal_assignment_on_sparse_scenes(tiny):
    """Where bubbles are far apart compared with their step, the mutual
    nearest-neighbour pairing is the minimum-cost bipartite matching."""
    opt = pytest.importorskip("scipy.optimize")
    from synth import track_scene
    g = _geom(tiny)
    sc = track_scene(g, 12, 25, seed=11, step_m=(20e-6, 40e-6), noise_m=2e-6, n_spurious_per_frame=0)
    L = np.zeros(len(sc.frame), dtype=O.LOC3D)
    L["frame"], L["x"], L["y"], L["z"] = sc.frame, sc.x, sc.y, sc.z
    r = 150e-6
    succ = O.track_link(g, L, r)
    half = 0.5 * (g.n_el - 1)
    P = np.stack([(L["x"] - half) * g.pitch, (L["y"] - half) * g.pitch, g.z0 + L["z"] * g.dz], axis=1)
    checked = 0
    for t in range(11):
        a, b = np.where(L["frame"] == t)[0], np.where(L["frame"] == t + 1)[0]
        if len(a) == 0 or len(b) == 0:
            continue
        D = np.linalg.norm(P[a][:, None, :] - P[b][None, :, :], axis=2)
        near = np.sort(D, axis=None)
        if np.sum(D <= r) != np.sum(D <= 3 * r):   # not sparse at this frame pair
            continue
        cost = np.where(D <= r, D, 1e3)
        ri, ci = opt.linear_sum_assignment(cost)
        pairs = {(int(a[i]), int(b[j])) for i, j in zip(ri, ci) if cost[i, j] < 1e3}
        mine = {(int(i), int(succ[i])) for i in a if succ[i] >= 0}
        assert mine == pairs, t
        checked += 1
        del near
    assert checked >= 5


@pytest.mark.parametrize("acc_frac,turn_ok,speed_ok", [(1 / 10, False, False), (1 / 40, True, True)])
def test_turn_rule_closed_form(tiny, acc_frac, turn_ok, speed_ok):
    """p(tau) = (v tau, a tau^2, 0): segment s is (v, a (2 s + 1)); the first and
    last are (v, a) and (v, 17 a)."""
    g = _geom(tiny)
    v = 40e-6
    a = v * acc_frac
    tau = np.arange(LEN, dtype=np.float64)
    p = np.array([0.0, -1e-3, 6e-3])[None, :] + np.stack([v * tau, a * tau ** 2, 0 * tau], axis=1)
    _, tr, _ = O.track(g, _to_list(g, np.arange(LEN), p), O.track_params())
    cos_ref = (v * v + 17 * a * a) / (math.hypot(v, a) * math.hypot(v, 17 * a))
    assert len(tr) == 1 and abs(tr[0]["cos_turn"] - cos_ref) < 1e-9
    speeds = [math.hypot(v, a * (2 * s + 1)) for s in range(LEN - 1)]
    assert abs(tr[0]["mean_speed"] - np.mean(speeds)) < 1e-12
    assert abs(tr[0]["speed_range"] - (max(speeds) - min(speeds))) < 1e-12
    assert bool(tr[0]["accepted"]) == (turn_ok and speed_ok)
    assert (cos_ref >= math.cos(math.radians(45))) == turn_ok


def test_speed_rule_closed_form(tiny):
    """p(tau) = (v tau + a tau^2, 0, 0): speeds v + a (2 s + 1), range 16 a,
    mean v + 9 a; kept iff 16 a <= (v + 9 a) / 2, i.e. a <= v / 23."""
    g = _geom(tiny)
    v = 40e-6
    tau = np.arange(LEN, dtype=np.float64)
    for a, keep in ((v / 20, False), (v / 26, True)):
        p = np.array([-1e-3, 0.0, 6e-3])[None, :] + np.stack([v * tau + a * tau ** 2, 0 * tau, 0 * tau], axis=1)
        _, tr, _ = O.track(g, _to_list(g, np.arange(LEN), p), O.track_params())
        assert abs(tr[0]["speed_range"] - 16 * a) < 1e-12
        assert abs(tr[0]["mean_speed"] - (v + 9 * a)) < 1e-12
        assert bool(tr[0]["accepted"]) == keep
    # a bubble that does not move has no direction: dropped
    p = np.tile(np.array([[0.0, 0.0, 6e-3]]), (LEN, 1))
    _, tr, grid = O.track(g, _to_list(g, np.arange(LEN), p), O.track_params())
    assert len(tr) == 1 and tr[0]["accepted"] == 0 and tr[0]["mean_speed"] == 0.0 and grid.sum() == 0


def test_density_counts_closed_form(tiny):
    """One voxel per frame along x from 0.05 voxel inside the grid edge, ten
    samples per frame: voxels 0..8 get 10 counts, voxel 9 gets 1."""
    g = _geom(tiny)
    prm = O.track_params(substeps=10, voxel=50e-6)
    vox = prm.voxel
    lo = np.array([-0.5 * g.n_el * g.pitch, -0.5 * g.n_el * g.pitch, g.z0 - 0.5 * g.dz])
    tau = np.arange(LEN, dtype=np.float64)
    p0 = lo + np.array([0.05, 10.5, 20.5]) * vox
    p = p0[None, :] + np.stack([vox * tau, 0 * tau, 0 * tau], axis=1)
    _, tr, grid = O.track(g, _to_list(g, np.arange(LEN), p), prm)
    assert len(tr) == 1 and tr[0]["accepted"] == 1
    nx, ny, nz = O.track_grid(g, vox)
    assert grid.shape == (nz, ny, nx)
    assert nx == math.ceil(g.n_el * g.pitch / vox) and nz == math.ceil(g.nz * g.dz / vox)
    row = grid[20, 10]
    assert list(row[:10]) == [10] * 9 + [1] and row[10:].sum() == 0
    assert grid.sum() == (LEN - 1) * prm.substeps + 1
    # a track wholly outside the grid adds nothing
    p_out = p + np.array([0.0, 0.0, -5e-3])[None, :]
    _, tr2, grid2 = O.track(g, _to_list(g, np.arange(LEN), p_out), prm)
    assert tr2[0]["accepted"] == 1 and grid2.sum() == 0


@pytest.mark.parametrize("v", [(0.0, 0.0, 25e-6), (0.0, 0.0, -25e-6), (30e-6, 40e-6, 0.0), (-12e-6, 0.0, 16e-6)])
def test_velocity_sums_constant_velocity(tiny, v):
    """A straight path at v metres per frame: every accumulation sample adds |v|
    and v_z in whole nanometres per frame to its voxel (|v| = 25, 25, 50, 20 um)."""
    g = _geom(tiny)
    prm = O.track_params(substeps=10, voxel=50e-6)
    vox = prm.voxel
    lo = np.array([-0.5 * g.n_el * g.pitch, -0.5 * g.n_el * g.pitch, g.z0 - 0.5 * g.dz])
    tau = np.arange(LEN, dtype=np.float64)
    p0 = lo + np.array([60.5, 60.5, 60.5]) * vox
    p = p0[None, :] + np.asarray(v)[None, :] * tau[:, None]
    _, tr, grid = O.track(g, _to_list(g, np.arange(LEN), p), prm)
    assert len(tr) == 1 and tr[0]["accepted"] == 1
    speed, vz = O.track_velocity(g, tr, prm)
    sp_nm = round(1e9 * math.sqrt(sum(x * x for x in v)))
    vz_nm = round(1e9 * v[2])
    assert grid.sum() == (LEN - 1) * prm.substeps + 1
    assert np.array_equal(speed, grid.astype(np.int64) * sp_nm)
    assert np.array_equal(vz, grid.astype(np.int64) * vz_nm)


def test_velocity_sums_accelerating_path(tiny):
    """z = z0 + u tau + w tau^2 with u = 20 um and w = 0.25 um per frame^2: the
    smoothed velocity at sample s (tau = s / 10) is u + 2 w tau = 20 000 + 50 s
    nanometres per frame, positive (deeper); a track wholly outside the grid
    adds nothing."""
    g = _geom(tiny)
    prm = O.track_params(substeps=10, voxel=50e-6)
    vox = prm.voxel
    lo = np.array([-0.5 * g.n_el * g.pitch, -0.5 * g.n_el * g.pitch, g.z0 - 0.5 * g.dz])
    tau = np.arange(LEN, dtype=np.float64)
    p = _path(lo + np.array([30.5, 30.5, 3.5]) * vox, np.array([0.0, 0.0, 20e-6]), np.array([0.0, 0.0, 0.25e-6]), tau)
    _, tr, grid = O.track(g, _to_list(g, np.arange(LEN), p), prm)
    assert len(tr) == 1 and tr[0]["accepted"] == 1
    speed, vz = O.track_velocity(g, tr, prm)
    ns = (LEN - 1) * prm.substeps + 1
    want = sum(20000 + 50 * s for s in range(ns))
    assert grid.sum() == ns and vz.sum() == want and speed.sum() == want
    assert np.all(speed[grid == 0] == 0)
    p_out = p + np.array([0.0, 0.0, -5e-3])[None, :]
    _, tr2, _ = O.track(g, _to_list(g, np.arange(LEN), p_out), prm)
    s2, v2 = O.track_velocity(g, tr2, prm)
    assert tr2[0]["accepted"] == 1 and not s2.any() and not v2.any()

