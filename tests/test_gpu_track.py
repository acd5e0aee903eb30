"""GPU parity of fixed-length tracking (Sec. II-A6) against the FP64 oracle:
track ids, acceptance and every double-precision coefficient bit-exact, and
the density counts identical, on the same float32 3D lists (the record the
GPU reads).  Lists: seeded synthetic scenes at oracle size and at the paper
workload's size (300 frames), and the oracle's own 3D list of the tiny
ensemble."""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _gpu_list(frame, x, y, z):
    from paper_2511_21647_gb300 import _lib
    rec = np.zeros(len(frame), dtype=_lib.LOC3D)
    rec["frame"], rec["x"], rec["y"], rec["z"] = frame, x, y, z
    return rec


def _oracle_list(rec):
    L = np.zeros(len(rec), dtype=O.LOC3D)
    L["frame"] = rec["frame"]
    for f in ("x", "y", "z"):
        L[f] = rec[f].astype(np.float64)
    return L


def run_gpu(s, rec, F, prm, cap_tracks=1 << 16, density=True, grid=None):
    from paper_2511_21647_gb300 import _lib, rca
    n = len(rec)
    dev = torch.from_numpy(rec.view(np.int32).reshape(-1, 10).copy()).cuda() if n else \
        torch.zeros((1, 10), dtype=torch.int32, device="cuda")
    n3d = torch.tensor([n], dtype=torch.int32, device="cuda")
    out = torch.zeros((max(cap_tracks, 1), _lib.TRACK.itemsize // 4), dtype=torch.int32, device="cuda")
    nt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    if density and grid is None:
        nx, ny, nz = rca.ulm_density_shape(s.t, prm.voxel_m)
        grid = torch.zeros((nz, ny, nx), dtype=torch.int32, device="cuda")
    rca.ulm_track(s.h, s.t, dev, n3d, max(n, 1), F, prm, out, cap_tracks, nt, grid if density else None)
    torch.cuda.synchronize()
    k = int(nt.item())
    tracks = out[:min(k, cap_tracks)].cpu().numpy().view(_lib.TRACK).reshape(-1)
    return k, tracks, (grid.cpu().numpy().view(np.uint32) if density else None), grid


def oracle_prm(prm):
    return O.TrackParams(prm.len, prm.substeps, prm.max_step_m, prm.cos_max_turn, prm.max_speed_change, prm.voxel_m)


def assert_same(tr_g, tr_o):
    assert len(tr_g) == len(tr_o)
    assert np.array_equal(tr_g["first"], tr_o["first"])
    assert np.array_equal(tr_g["frame0"], tr_o["frame0"])
    assert np.array_equal(tr_g["accepted"], tr_o["accepted"])
    for f in ("a", "mean_speed", "cos_turn", "speed_range"):
        assert np.array_equal(tr_g[f], tr_o[f]), f


@pytest.fixture(scope="module")
def S(tiny):
    from paper_2511_21647_gb300.pipeline import RcaSession
    s = RcaSession(tiny.geom)
    yield s
    s.close()


@pytest.mark.parametrize("seed,n_bub", [(21, 40), (22, 120)])
def test_tracks_and_density_bit_exact_on_synthetic_scenes(S, tiny, seed, n_bub):
    from paper_2511_21647_gb300 import rca
    from synth import track_scene
    g = tiny.geom
    F = 64
    sc = track_scene(g, F, n_bub, seed=seed)
    rec = _gpu_list(sc.frame, sc.x, sc.y, sc.z)
    prm = rca.make_track_params()
    k, tr_g, grid_g, _ = run_gpu(S, rec, F, prm)
    assert S.sync_status() == 0
    succ, tr_o, grid_o = O.track(g, _oracle_list(rec), oracle_prm(prm))
    assert k == len(tr_o) and k > 20
    assert_same(tr_g, tr_o)
    assert np.array_equal(grid_g, grid_o) and grid_o.sum() > 0
    # most tracks follow one bubble
    same = [len({int(sc.truth[i])} | {int(sc.truth[j]) for j in _chain(succ, int(i))}) == 1 for i in tr_o["first"]]
    assert np.mean(same) > 0.9


@pytest.mark.parametrize("seed,n_bub", [(23, 120)])
def test_velocity_sums_bit_exact(S, tiny, seed, n_bub):
    """velocity volumes of the GPU's own tracks (ulm_track_velocity on the
    records ulm_track wrote) equal the oracle's sums on the oracle's tracks"""
    from paper_2511_21647_gb300 import _lib, rca
    from synth import track_scene
    g = tiny.geom
    F = 64
    sc = track_scene(g, F, n_bub, seed=seed)
    rec = _gpu_list(sc.frame, sc.x, sc.y, sc.z)
    prm = rca.make_track_params()
    n = len(rec)
    dev = torch.from_numpy(rec.view(np.int32).reshape(-1, 10).copy()).cuda()
    n3d = torch.tensor([n], dtype=torch.int32, device="cuda")
    cap = 1 << 14
    out = torch.zeros((cap, _lib.TRACK.itemsize // 4), dtype=torch.int32, device="cuda")
    nt = torch.zeros(1, dtype=torch.int32, device="cuda")
    nx, ny, nz = rca.ulm_density_shape(S.t, prm.voxel_m)
    dens = torch.zeros((nz, ny, nx), dtype=torch.int32, device="cuda")
    rca.ulm_track(S.h, S.t, dev, n3d, n, F, prm, out, cap, nt, dens)
    speed = torch.zeros((nz, ny, nx), dtype=torch.int64, device="cuda")
    vz = torch.zeros_like(speed)
    rca.ulm_track_velocity(S.h, S.t, out, nt, cap, prm, speed, vz)
    torch.cuda.synchronize()
    assert S.sync_status() == 0
    _, tr_o, grid_o = O.track(g, _oracle_list(rec), oracle_prm(prm))
    sp_o, vz_o = O.track_velocity(g, tr_o, oracle_prm(prm))
    assert np.array_equal(dens.cpu().numpy().view(np.uint32), grid_o)
    assert np.array_equal(speed.cpu().numpy(), sp_o) and np.array_equal(vz.cpu().numpy(), vz_o)
    assert sp_o.sum() > 0 and (vz_o > 0).any() and (vz_o < 0).any()
    # mean speed where counted: positive and within the scene's speeds (per frame at 400 Hz)
    m = grid_o > 0
    mean_mps = sp_o[m] / grid_o[m] * 1e-9 * 400.0
    print(f"\nvelocity volumes: {int(m.sum())} voxels, mean speed {mean_mps.mean() * 1e3:.2f} mm/s")
    assert mean_mps.min() > 0
    with pytest.raises(rca.RcaError) as e:
        bad = rca.make_track_params(voxel_m=0.0)
        rca.ulm_track_velocity(S.h, S.t, out, nt, cap, bad, speed, vz)
    assert e.value.status == _lib.RCA_ERR_INVALID_ARG


def _chain(succ, i, n=10):
    out = []
    for _ in range(n - 1):
        i = int(succ[i])
        out.append(i)
    return out


def test_tracks_on_the_oracle_localisations_of_the_tiny_ensemble(S, tiny, tiny_rf):
    """the oracle's planes -> the oracle's 3D list (float32, as ulm_pair3d
    stores it) -> GPU and oracle tracking"""
    from paper_2511_21647_gb300 import rca
    g = tiny.geom
    psf = json.load(open(os.path.join(HERE, "golden", "psf_sigma.json")))["tiny"]
    planes = O.beamform_projections(g, tiny_rf.rf.numpy()).astype(np.complex64).astype(np.complex128)
    _, _, _, L3 = O.localize(planes, 5, psf["sig_z"], psf["sig_lat"], 0.1, 0.5, g.P)
    rec = _gpu_list(L3["frame"], L3["x"].astype(np.float32), L3["y"].astype(np.float32), L3["z"].astype(np.float32))
    F = tiny.n_frames
    # NCC finds a bubble in about half of the frames at this density, so runs of
    # ten detections are rare: four-point tracks exercise the same path
    prm = rca.make_track_params(length=4, max_step_m=200e-6)
    k, tr_g, grid_g, _ = run_gpu(S, rec, F, prm)
    _, tr_o, grid_o = O.track(g, _oracle_list(rec), oracle_prm(prm))
    print(f"\ntiny ensemble: {len(rec)} 3D localisations, {k} tracks, {int(tr_o['accepted'].sum())} accepted")
    assert k == len(tr_o) and k > 0
    assert_same(tr_g, tr_o)
    assert np.array_equal(grid_g, grid_o)


def test_paper_scale_scene_bit_exact(tiny):
    """300 frames, about 100 localisations per frame, the paper geometry"""
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import RcaSession
    from synth import track_scene, workload
    w = workload("paper")
    g, F = w.geom, w.n_frames
    sc = track_scene(g, F, 1000, seed=31, run=(8, 60))
    rec = _gpu_list(sc.frame, sc.x, sc.y, sc.z)
    prm = rca.make_track_params()
    with RcaSession(g) as s:
        k, tr_g, grid_g, _ = run_gpu(s, rec, F, prm, cap_tracks=1 << 17)
        assert s.sync_status() == 0
    _, tr_o, grid_o = O.track(g, _oracle_list(rec), oracle_prm(prm))
    print(f"\npaper-size scene: {len(rec)} localisations, {k} tracks, {int(tr_o['accepted'].sum())} accepted")
    assert k == len(tr_o) and k > 1000
    assert_same(tr_g, tr_o)
    assert np.array_equal(grid_g, grid_o)


def test_density_accumulates_capacity_and_empty(S, tiny):
    from paper_2511_21647_gb300 import _lib, rca
    from synth import track_scene
    g = tiny.geom
    sc = track_scene(g, 40, 60, seed=23)
    rec = _gpu_list(sc.frame, sc.x, sc.y, sc.z)
    prm = rca.make_track_params()
    k, tr, grid1, gdev = run_gpu(S, rec, 40, prm)
    assert S.sync_status() == 0 and k > 4
    # a second call adds into the same grid
    _, _, grid2, _ = run_gpu(S, rec, 40, prm, grid=gdev)
    assert np.array_equal(grid2, 2 * grid1)
    # capacity: true count, first entries written, CAPACITY in the status word
    k2, tr2, _, _ = run_gpu(S, rec, 40, prm, cap_tracks=3, density=False)
    assert k2 == k and S.sync_status() == _lib.RCA_ERR_CAPACITY
    assert np.array_equal(tr2["first"], tr["first"][:3])
    # empty list
    k3, _, grid3, _ = run_gpu(S, rec[:0], 40, prm)
    assert k3 == 0 and grid3.sum() == 0 and S.sync_status() == 0


def test_host_side_parameter_errors(S):
    from paper_2511_21647_gb300 import _lib, rca
    rec = _gpu_list(np.zeros(1, np.int32), np.zeros(1, np.float32), np.zeros(1, np.float32), np.zeros(1, np.float32))
    for kw in (dict(length=1), dict(length=_lib.ULM_TRACK_MAX_LEN + 1), dict(substeps=0), dict(max_step_m=0.0),
               dict(voxel_m=-1.0)):
        with pytest.raises(rca.RcaError) as e:
            run_gpu(S, rec, 4, rca.make_track_params(**kw))
        assert e.value.status == _lib.RCA_ERR_INVALID_ARG
