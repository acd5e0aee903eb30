"""GPU parity of the localisation path (XDoppler + frame max, separable NCC,
sub-pixel peaks, XZ/YZ pairing) against the FP64 oracle.

Inputs of every stage come from the oracle (its planes, its A, its 2D
lists, rounded to float32), never from the CUDA path.  Discrete outputs must
be identical; where a decision's margin is within the float32 error of the
quantities it compares (listed in the test), either outcome is accepted and
the rest must still agree."""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
PSF = json.load(open(os.path.join(HERE, "golden", "psf_sigma.json")))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def S(tiny):
    from paper_2511_21647_gb300.pipeline import RcaSession
    s = RcaSession(tiny.geom)
    yield s
    s.close()


@pytest.fixture(scope="module")
def prm_tiny():
    return dict(d=5, sig_z=PSF["tiny"]["sig_z"], sig_lat=PSF["tiny"]["sig_lat"], alpha=0.1, ncc_min=0.5)


@pytest.fixture(scope="module")
def oracle_planes(tiny, tiny_rf):
    """oracle planes of the tiny ensemble, rounded to complex64 (the GPU input)"""
    pl = O.beamform_projections(tiny.geom, tiny_rf.rf.numpy())
    return pl.astype(np.complex64)


def c64(x):
    a = np.stack([x.real, x.imag], axis=-1).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def ulm(prm, **kw):
    from paper_2511_21647_gb300 import rca
    p = dict(prm)
    p.update(kw)
    return rca.make_ulm_params(**p)


def test_xdoppler_amplitude_and_frame_max(S, oracle_planes):
    A_o, M_o = O.xdoppler(oracle_planes.astype(np.complex128))
    A, M = S.enhance(c64(oracle_planes))
    assert rel(A.cpu().numpy(), A_o) < 2e-6
    assert np.allclose(M.cpu().numpy(), M_o, rtol=2e-6, atol=0)


@pytest.mark.parametrize("F", [1, 2, 3])
def test_xdoppler_window_clipped_at_ensemble_ends(S, oracle_planes, F):
    pl = oracle_planes[:F]
    A_o, M_o = O.xdoppler(pl.astype(np.complex128))
    A, M = S.enhance(c64(pl))
    assert rel(A.cpu().numpy(), A_o) < 2e-6


@pytest.fixture(scope="module")
def oracle_A(oracle_planes):
    A_o, M_o = O.xdoppler(oracle_planes.astype(np.complex128))
    return A_o.astype(np.float32), M_o.astype(np.float32)


def test_separable_ncc_matches_brute_2d(S, oracle_A, prm_tiny):
    A32, M32 = oracle_A
    A = torch.from_numpy(A32).cuda()
    M = torch.from_numpy(M32).cuda()
    _, _, ncc = S.detect2d(A, M, ulm(prm_tiny), want_ncc=True)
    ncc = ncc.cpu().numpy()
    worst = 0.0
    for t in (0, 20, 63):
        for axis in (0, 1):
            for b in range(A32.shape[2]):
                ref = O.ncc_plane(A32[t, axis, b].astype(np.float64), prm_tiny["d"], prm_tiny["sig_z"],
                                  prm_tiny["sig_lat"], float(M32[t]))
                worst = max(worst, float(np.max(np.abs(ncc[t, axis, b] - ref))))
    assert worst < 2e-5, worst


def _key(L2):
    return [(int(r["frame"]), int(r["axis"]), int(r["slab"]), int(r["iz"]), int(r["ilat"])) for r in L2]


def test_peaks_match_oracle_lists(S, oracle_A, prm_tiny):
    """detection on the oracle's float32 amplitudes: keys equal outside the
    oracle's near-tie pixels (3e-5 in NCC, 1e-6 M_t in amplitude: the same
    float32 input on both sides), fields within the stated tolerances"""
    import ulm_lists as UL
    A32, M32 = oracle_A
    L_o = O.localize2d(A32.astype(np.float64), M32.astype(np.float64), prm_tiny["d"], prm_tiny["sig_z"],
                       prm_tiny["sig_lat"], prm_tiny["alpha"], prm_tiny["ncc_min"])
    from paper_2511_21647_gb300.pipeline import list2d_numpy
    out, n2d, _ = S.detect2d(torch.from_numpy(A32).cuda(), torch.from_numpy(M32).cuda(), ulm(prm_tiny))
    n = int(n2d.item())
    L_g = list2d_numpy(out, n)
    assert S.sync_status() == 0
    ko, kg = _key(L_o), _key(L_g)
    assert kg == sorted(kg), "GPU list not in (frame, axis, slab, iz, ilat) order"
    diff = set(ko) ^ set(kg)
    amb = UL.near_ties(A32, M32, prm_tiny, eps_ncc=3e-5, eps_amp=1e-6)
    assert diff <= amb, sorted(diff - amb)[:10]
    print(f"\npeaks: {len(ko)} oracle entries, {len(diff)} differing, {len(amb)} near-tie pixels")
    io = {k: q for q, k in enumerate(ko)}
    ig = {k: q for q, k in enumerate(kg)}
    for k in sorted(set(ko) & set(kg)):
        a, b = L_o[io[k]], L_g[ig[k]]
        assert abs(a["z"] - b["z"]) < 1e-3 and abs(a["lat"] - b["lat"]) < 1e-3
        assert abs(a["ncc"] - b["ncc"]) < 2e-5
        assert a["amp"] == b["amp"]          # A at the peak pixel, same float32 input
    assert len(ko) > 20


def _to_gpu_list(L_o):
    """oracle 2D list -> librca ulm_loc2d records (float32 positions)"""
    from paper_2511_21647_gb300 import _lib
    rec = np.zeros(len(L_o), dtype=_lib.LOC2D)
    for f in ("frame", "axis", "slab", "iz", "ilat"):
        rec[f] = L_o[f]
    for f in ("z", "lat", "ncc", "amp"):
        rec[f] = L_o[f].astype(np.float32)
    return rec


def _f32_list(L_o):
    """the same list, float fields rounded to float32, back in the oracle's format"""
    L = L_o.copy()
    for f in ("z", "lat", "ncc", "amp"):
        L[f] = L_o[f].astype(np.float32).astype(np.float64)
    return L


def test_pairing_bit_exact_on_oracle_lists(S, oracle_A, prm_tiny, tiny):
    A32, M32 = oracle_A
    L_o = _f32_list(O.localize2d(A32.astype(np.float64), M32.astype(np.float64), prm_tiny["d"],
                                 prm_tiny["sig_z"], prm_tiny["sig_lat"], prm_tiny["alpha"], prm_tiny["ncc_min"]))
    P3_o = O.pair3d(L_o, tiny.geom.P)
    rec = _to_gpu_list(L_o)
    dev = torch.from_numpy(rec.view(np.int32).reshape(-1, 10).copy()).cuda()
    n2d = torch.tensor([len(rec)], dtype=torch.int32, device="cuda")
    out, n3d = S.pair3d(dev, n2d, len(rec), A32.shape[0])
    from paper_2511_21647_gb300.pipeline import list3d_numpy
    P3 = list3d_numpy(out, int(n3d.item()))
    assert [(int(r["i_xz"]), int(r["i_yz"])) for r in P3] == [(int(r["i_xz"]), int(r["i_yz"])) for r in P3_o]
    assert len(P3_o) > 5
    assert np.array_equal(P3["x"], P3_o["x"].astype(np.float32))
    assert np.array_equal(P3["y"], P3_o["y"].astype(np.float32))
    assert np.allclose(P3["z"], P3_o["z"], atol=1e-5, rtol=0)


def test_pairing_hand_built_rules(S, tiny):
    from paper_2511_21647_gb300 import _lib
    from paper_2511_21647_gb300.pipeline import list3d_numpy
    rows = [  # frame axis slab iz ilat z lat ncc amp
        (0, 0, 1, 20, 10, 20.0, 10.2, 0.9, 1.00),
        (0, 0, 1, 21, 11, 21.0, 11.0, 0.9, 1.2),
        (0, 1, 1, 21, 12, 21.0, 12.1, 0.9, 1.00),
        (0, 1, 1, 22, 13, 22.0000019, 13.0, 0.9, 1.00),
        (1, 0, 0, 5, 1, 5.0, 1.0, 0.9, 0.95),
        (1, 1, 0, 5, 2, 5.0, 2.0, 0.9, 1.0),
    ]
    rec = np.zeros(len(rows), dtype=_lib.LOC2D)
    for q, r in enumerate(rows):
        rec[q] = r + (0,)
    dev = torch.from_numpy(rec.view(np.int32).reshape(-1, 10).copy()).cuda()
    n2d = torch.tensor([len(rec)], dtype=torch.int32, device="cuda")
    out, n3d = S.pair3d(dev, n2d, len(rec), 2)
    P3 = list3d_numpy(out, int(n3d.item()))
    L_o = np.zeros(len(rows), dtype=O.LOC2D)
    for q, r in enumerate(rows):
        L_o[q] = (r[0], r[1], r[2], r[3], r[4], np.float32(r[5]), np.float32(r[6]), np.float32(r[7]), np.float32(r[8]))
    P3_o = O.pair3d(L_o, tiny.geom.P)
    assert [(int(r["i_xz"]), int(r["i_yz"])) for r in P3] == [(int(r["i_xz"]), int(r["i_yz"])) for r in P3_o]
    assert [(int(r["i_xz"]), int(r["i_yz"])) for r in P3] == [(0, 2), (4, 5)]


def test_localize_end_to_end_on_oracle_planes(S, oracle_planes, prm_tiny, tiny):
    """The public ulm_localize call on the oracle's planes vs the oracle's
    localiser on the same (complex64-rounded) planes: the 2D key lists equal
    outside the oracle's near-tie pixels, the 3D pairs equal in every
    sub-block group without a differing entry or a near-tie pairing decision
    (tests/ulm_lists.py).  The GPU's amplitude is its own (FP32 XDoppler of
    the planes, within 2e-6 of the oracle's), so the candidate margins are
    3e-5 in NCC and 1e-5 M_t in amplitude."""
    import ulm_lists as UL
    from paper_2511_21647_gb300.pipeline import list2d_numpy, list3d_numpy
    A_o, M_o, L2_o, L3_o = O.localize(oracle_planes.astype(np.complex128), prm_tiny["d"], prm_tiny["sig_z"],
                                      prm_tiny["sig_lat"], prm_tiny["alpha"], prm_tiny["ncc_min"], tiny.geom.P)
    out2d, n2d, out3d, n3d = S.localize(c64(oracle_planes), ulm(prm_tiny))
    assert S.sync_status() == 0
    L2 = list2d_numpy(out2d, int(n2d.item()))
    L3 = list3d_numpy(out3d, int(n3d.item()))
    amb = UL.near_ties(A_o, M_o, prm_tiny, eps_ncc=3e-5, eps_amp=1e-5)
    st = UL.compare(L2_o, L3_o, L2, L3, amb, tiny.geom.P, pos_tol=1e-3, ncc_tol=5e-5, amp_rtol=1e-5, tz=2e-3, tr=2e-5)
    print(f"\nend to end (tiny): {st}")
    assert st["n2d"] > 20 and st["n3d"] > 5


def test_empty_input_gives_empty_lists(S, prm_tiny, tiny):
    g = tiny.geom
    pl = torch.zeros(S.planes_shape(4) + (2,), device="cuda")
    out2d, n2d, out3d, n3d = S.localize(pl, ulm(prm_tiny))
    assert int(n2d.item()) == 0 and int(n3d.item()) == 0
    assert S.sync_status() == 0


def test_capacity_overflow_reports_true_count(S, oracle_planes, prm_tiny):
    from paper_2511_21647_gb300 import _lib
    full = S.localize(c64(oracle_planes), ulm(prm_tiny))
    n_full = int(full[1].item())
    assert S.sync_status() == 0 and n_full > 8
    out2d, n2d, out3d, n3d = S.localize(c64(oracle_planes), ulm(prm_tiny), cap2d=8, cap3d=2)
    assert int(n2d.item()) == n_full
    assert S.sync_status() == _lib.RCA_ERR_CAPACITY
    assert S.sync_status() == 0          # read-and-clear


def test_coherent_enhancement_option(S, oracle_planes):
    from paper_2511_21647_gb300 import _lib
    A, _ = S.enhance(c64(oracle_planes[:3]), enh=_lib.ULM_ENH_COHERENT)
    pl = oracle_planes[:3].astype(np.complex128)
    ref = np.abs(pl[:, :, 0] + pl[:, :, 1])
    assert rel(A.cpu().numpy(), ref) < 2e-6
