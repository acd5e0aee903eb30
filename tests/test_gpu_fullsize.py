"""Full-size parity and the paired-pixel Stage 1.

Paper scale: the 128 + 128 element, 4 + 4 transmission, 300-frame ensemble
of 1024 samples per channel (250 x 128 planes per slab, NCC d = 11), run
through the same calls, dtypes and launch shapes as the benchmark, compared
with the FP64 oracle on sampled frames that the oracle computes one by one
(the clutter filter's mean is always taken over all 300 frames).  The
localisation checks feed the oracle's own planes / amplitudes of a sampled
frame, placed in an otherwise empty 300-frame ensemble, to the GPU calls.

Oracle sizes: geometries with 64 and 128 elements, whose Stage 1 runs the
paired-pixel kernel (a lane owns pixel l and its mirror N - 1 - l), which the
32-element parity cases do not reach; FP32, FP16 and BF16 IQ."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
TOL_REDUCED = 2e-3
SAMPLED = (0, 150, 299)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def as_c128(t):
    from paper_2511_21647_gb300.pipeline import to_complex128
    return to_complex128(t)


def c_tensor(x, dtype=torch.float32):
    """complex numpy -> interleaved [..., 2] cuda tensor of the given real dtype"""
    a = np.stack([x.real, x.imag], axis=-1).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def per_plane(a, b):
    n = np.linalg.norm(b.reshape(-1, b.shape[-2] * b.shape[-1]), axis=1)
    e = np.linalg.norm((a - b).reshape(n.size, -1), axis=1)
    big = n > 1e-3 * n.max()
    return e[big] / n[big]


# --- paired-pixel Stage 1 at oracle sizes ---------------------------------------------

@pytest.fixture(scope="module", params=[64, 128])
def paired(request, tiny):
    """n_el = 64 / 128, a ragged depth (89 slice rows: several row tiles and a
    partial one), 3 frames; oracle IQ, slices and planes of every frame."""
    from synth.rca_sim import RcaWorkload, generate
    from paper_2511_21647_gb300.pipeline import RcaSession
    n_el = request.param
    g = dataclasses.replace(tiny.geom, n_el=n_el, nz=45, ns=320)
    w = RcaWorkload(f"paired{n_el}", g, n_frames=3, n_mb=8, n_tissue=40, seed=90 + n_el)
    rf = generate(w).rf
    pl_o, sl_o = O.beamform_projections(g, rf.numpy(), return_slices=True)
    iq_o = O.demod(g, rf.numpy())
    s = RcaSession(g)
    yield g, s, rf, iq_o, sl_o, pl_o
    s.close()


def test_paired_stage1_fp32(paired):
    g, s, _, iq_o, sl_o, _ = paired
    sl = as_c128(s.stage1(c_tensor(iq_o.transpose(0, 1, 3, 2))))
    assert s.sync_status() == 0
    for f in range(sl.shape[0]):
        assert rel(sl[f], sl_o[f]) < 1e-5, f
    # both halves of the lateral axis (pixel l and its mirror) on every transmission
    h = g.n_el // 2
    for k in range(sl.shape[1]):
        assert rel(sl[:, k, :, :h], sl_o[:, k, :, :h]) < 1e-5
        assert rel(sl[:, k, :, h:], sl_o[:, k, :, h:]) < 1e-5


@pytest.mark.parametrize("iq_name,tdt,tol", [("C16F", torch.float16, TOL_REDUCED), ("C16BF", torch.bfloat16, 1e-5)])
def test_paired_stage1_half_iq(paired, iq_name, tdt, tol):
    """FP16 / BF16 IQ: the oracle runs on the same rounded IQ, so the only
    error left is the kernel's (FP16 weights for FP16 samples; FP32 weights
    and FP32 products for BF16 samples)."""
    from paper_2511_21647_gb300 import _lib as L
    g, s, _, iq_o, _, _ = paired
    iq_t = c_tensor(iq_o.transpose(0, 1, 3, 2), tdt)
    r = iq_t.float().cpu().numpy()
    iq_r = (r[..., 0] + 1j * r[..., 1]).transpose(0, 1, 3, 2)           # back to [F][2K][E][ns]
    ref = np.stack([O.stage1(g, iq_r[f]) for f in range(iq_r.shape[0])])
    sl = as_c128(s.stage1(iq_t, iq_dtype=getattr(L, "RCA_" + iq_name)))
    assert s.sync_status() == 0
    assert rel(sl, ref) < tol


def test_paired_beamform_end_to_end(paired):
    """Whole ensemble and per frame at 1e-4.  Per plane, the FP32 error is a
    floor of the same absolute size in every plane (about 5e-6 of the largest
    plane's norm): the clutter filter subtracts an ensemble mean 40 dB above
    the moving scatterers, so the rounding of the tissue-scale RF and IQ
    values sets it, not the plane's own content (Stage 2 alone on FP32-rounded
    oracle slices stays near 1e-7 of each plane's norm).  Each plane's error
    is therefore measured against the larger of its norm and 10 % of the
    largest plane's."""
    g, s, rf, _, _, pl_o = paired
    pl = as_c128(s.beamform(rf.cuda()))
    assert s.sync_status() == 0
    assert rel(pl, pl_o) < TOL_FP32
    for f in range(pl.shape[0]):
        assert rel(pl[f], pl_o[f]) < TOL_FP32, f
    n = np.linalg.norm(pl_o.reshape(-1, pl_o.shape[-2] * pl_o.shape[-1]), axis=1)
    e = np.linalg.norm((pl - pl_o).reshape(n.size, -1), axis=1)
    ratio = e / np.maximum(n, 0.1 * n.max())
    q = int(np.argmax(ratio))
    print(f"\nn_el {g.n_el}: worst plane error {ratio[q]:.2e} (plane norm {n[q] / n.max():.1e} of the largest)")
    _plane_report(n, e)
    assert ratio.max() < TOL_FP32


def _plane_report(n, e):
    """per-plane absolute error against the largest plane norm, by plane size"""
    o = np.argsort(n)
    ea = e / n.max()
    for lab, sel in (("smallest", o[:8]), ("largest", o[-8:])):
        print(f"  {lab:8s} planes: norm/max {np.array2string(n[sel] / n.max(), precision=1)}")
        print(f"  {'':8s}   err/max {np.array2string(ea[sel], precision=1)}")
    print(f"  err/max over all planes: median {np.median(ea):.1e}, max {ea.max():.1e} (plane {int(np.argmax(ea))})")


def test_paired_stage2_on_oracle_slices(paired):
    """Stage 2 + projection alone at 64 / 128 elements, on the oracle's slices
    rounded to complex64, against the oracle's projection of the same slices."""
    g, s, _, _, sl_o, _ = paired
    sl32 = sl_o.astype(np.complex64)
    ref = np.stack([O.stage2_project(g, sl32[f].astype(np.complex128)) for f in range(sl32.shape[0])])
    pl = as_c128(s.stage2(c_tensor(sl32)))
    assert s.sync_status() == 0
    assert rel(pl, ref) < 1e-5
    n = np.linalg.norm(ref.reshape(-1, ref.shape[-2] * ref.shape[-1]), axis=1)
    e = np.linalg.norm((pl - ref).reshape(n.size, -1), axis=1)
    print(f"\nStage 2 alone, n_el {g.n_el}:")
    _plane_report(n, e)
    big = n > 1e-3 * n.max()
    assert np.all(e[big] / n[big] < 1e-5)


# --- paper scale, sampled frames ---------------------------------------------------------

@pytest.fixture(scope="module")
def paper():
    """The benchmark's input: the paper-scale ensemble generated on the device
    (seeded), plus the oracle's IQ, slices and planes of the sampled frames."""
    from synth import generate, workload
    from paper_2511_21647_gb300.pipeline import RcaSession
    w = workload("paper")
    rf = generate(w, device="cuda", dtype=torch.float32, frame_batch=32).rf.contiguous()
    rf_h = rf.cpu().numpy()
    pl_o, sl_o = O.beamform_projections(w.geom, rf_h, frames=SAMPLED, return_slices=True)
    iq_o = O.demod(w.geom, rf_h, frames=SAMPLED)
    s = RcaSession(w.geom)
    yield w, s, rf, rf_h, iq_o, sl_o, pl_o
    s.close()


def test_paper_scale_fp32_chain_on_sampled_frames(paper):
    """ingest -> Stage 1 -> Stage 2 + projection as separate calls, and the
    public one-call beamformer the benchmark times, at full size."""
    w, s, rf, _, iq_o, sl_o, pl_o = paper
    F = w.n_frames
    iq = s.ingest(rf)
    sl = s.stage1(iq)
    assert s.sync_status() == 0
    idx = list(SAMPLED)
    iq_s = as_c128(iq[idx]).transpose(0, 1, 3, 2)
    assert rel(iq_s, iq_o) < 1e-5
    del iq
    sl_s = as_c128(sl[idx])
    for q in range(len(idx)):
        assert rel(sl_s[q], sl_o[q]) < TOL_FP32, idx[q]
    del sl
    pl = s.beamform(rf)
    assert s.sync_status() == 0 and pl.shape[0] == F
    pl_s = as_c128(pl[idx])
    for q in range(len(idx)):
        assert rel(pl_s[q], pl_o[q]) < TOL_FP32, idx[q]
    assert np.all(per_plane(pl_s, pl_o) < TOL_FP32)


def test_paper_scale_reduced_precision_on_sampled_frames(paper, record_property):
    """int16 RF with per-channel scale, FP16 IQ, BF16 planes (the benchmark's
    reduced form) vs the oracle on the same dequantised int16 input."""
    from synth import quantize_int16
    from paper_2511_21647_gb300 import _lib as L
    w, s, rf, _, _, _, _ = paper
    q, scale = quantize_int16(rf)
    deq = (q.double() * scale.double()[None, :, :, None]).float().cpu().numpy()
    ref = O.beamform_projections(w.geom, deq, frames=SAMPLED)
    del deq
    pl = s.beamform(q, rf_dtype=L.RCA_I16, scale=scale, iq_dtype=L.RCA_C16F, planes_dtype=L.RCA_C16BF)
    assert s.sync_status() == 0
    got = as_c128(pl[list(SAMPLED)])
    e = rel(got, ref)
    pp = per_plane(got, ref)
    record_property("rel_l2_vs_dequantised", e)
    record_property("per_plane_max", float(pp.max()))
    print(f"\npaper scale, FP16 IQ / BF16 planes: rel-L2 {e:.2e}, per-plane max {pp.max():.2e}")
    assert e < TOL_REDUCED
    assert pp.max() < 2.5 * TOL_REDUCED


def _near_ties(A, M, prm, eps=3e-5):
    """(axis, slab, iz, ilat) of one frame's pixels whose candidate decision is
    within eps of flipping (oracle NCC on the float32 amplitudes)"""
    amb = set()
    _, S_, nz, N = A.shape
    for axis in range(2):
        for b in range(S_):
            n = O.ncc_plane(A[axis, b].astype(np.float64), prm["d"], prm["sig_z"], prm["sig_lat"], float(M))
            c = n[1:-1, 1:-1]
            nbd = np.full(c.shape, np.inf)
            for di in (-1, 0, 1):
                for dl in (-1, 0, 1):
                    if di or dl:
                        nb = n[1 + di:nz - 1 + di, 1 + dl:N - 1 + dl]
                        nbd = np.minimum(nbd, np.abs(nb - c))
            close = (c >= prm["ncc_min"] - eps) & ((np.abs(c - prm["ncc_min"]) < eps) | (nbd < eps))
            for i, l in zip(*np.nonzero(close)):
                amb.add((axis, b, int(i) + 1, int(l) + 1))
    return amb


def test_paper_scale_localisation_on_oracle_frame(paper):
    """XDoppler, NCC detection and pairing at full size on the oracle's planes
    of frames 149..151 (the window of frame 150), in a 300-frame ensemble that
    is otherwise empty, against the oracle's localiser on the same inputs."""
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import list2d_numpy, list3d_numpy
    w, s, _, rf_h, _, _, _ = paper
    g, F, f = w.geom, w.n_frames, 150
    prm = dict(d=w.ncc_d, sig_z=0.81, sig_lat=1.45, alpha=0.1, ncc_min=0.5)
    win = O.beamform_projections(g, rf_h, frames=(f - 1, f, f + 1)).astype(np.complex64)
    A_o, M_o = O.xdoppler(win.astype(np.complex128))
    # enhancement over the whole ensemble; frame f's window is complete
    planes = torch.zeros(s.planes_shape(F) + (2,), device="cuda")
    planes[f - 1:f + 2] = c_tensor(win)
    A, M = s.enhance(planes)
    del planes
    assert rel(A[f].cpu().numpy(), A_o[1]) < 2e-6
    assert abs(float(M[f]) - M_o[1]) <= 2e-6 * M_o[1]
    # detection on the oracle's amplitudes (float32) of frame f
    A32 = A_o[1].astype(np.float32)
    M32 = np.float32(M_o[1])
    A_in = torch.zeros(s.a_shape(F), device="cuda")
    A_in[f] = torch.from_numpy(A32).cuda()
    M_in = torch.zeros(F, device="cuda")
    M_in[f] = float(M32)
    p = rca.make_ulm_params(**prm)
    out, n2d, ncc = s.detect2d(A_in, M_in, p, cap2d=1 << 16, want_ncc=True)
    assert s.sync_status() == 0
    # the separable NCC with the paper's 11-tap kernels against the oracle's brute 2D form
    ncc_f = ncc[f].cpu().numpy()
    del ncc
    worst = 0.0
    for ax in range(2):
        for sb in (0, 7, 15):
            ref = O.ncc_plane(A32[ax, sb].astype(np.float64), prm["d"], prm["sig_z"], prm["sig_lat"], float(M32))
            worst = max(worst, float(np.max(np.abs(ncc_f[ax, sb] - ref))))
    assert worst < 2e-5, worst
    L_g = list2d_numpy(out, int(n2d.item()))
    assert np.all(L_g["frame"] == f)
    L_o = O.localize2d(A32[None].astype(np.float64), np.array([float(M32)]), prm["d"], prm["sig_z"],
                       prm["sig_lat"], prm["alpha"], prm["ncc_min"])
    key = lambda L2: [(int(r["axis"]), int(r["slab"]), int(r["iz"]), int(r["ilat"])) for r in L2]
    ko, kg = key(L_o), key(L_g)
    assert len(ko) > 100
    diff = set(ko) ^ set(kg)
    if diff:
        amb = _near_ties(A32, M32, prm)
        assert diff <= amb, sorted(diff - amb)[:10]
    io = {k: q for q, k in enumerate(ko)}
    ig = {k: q for q, k in enumerate(kg)}
    for k in set(ko) & set(kg):
        a, b = L_o[io[k]], L_g[ig[k]]
        assert abs(a["z"] - b["z"]) < 1e-3 and abs(a["lat"] - b["lat"]) < 1e-3
        assert a["amp"] == b["amp"]
    # pairing on the oracle's list (float fields rounded to float32), bit-exact
    from paper_2511_21647_gb300 import _lib
    L_o32 = L_o.copy()
    for fld in ("z", "lat", "ncc", "amp"):
        L_o32[fld] = L_o[fld].astype(np.float32).astype(np.float64)
    L_o32["frame"] = f
    P3_o = O.pair3d(L_o32, g.P)
    rec = np.zeros(len(L_o32), dtype=_lib.LOC2D)
    for fld in ("frame", "axis", "slab", "iz", "ilat"):
        rec[fld] = L_o32[fld]
    for fld in ("z", "lat", "ncc", "amp"):
        rec[fld] = L_o32[fld].astype(np.float32)
    dev = torch.from_numpy(rec.view(np.int32).reshape(-1, 10).copy()).cuda()
    n_in = torch.tensor([len(rec)], dtype=torch.int32, device="cuda")
    out3, n3 = s.pair3d(dev, n_in, len(rec), F)
    P3 = list3d_numpy(out3, int(n3.item()))
    assert len(P3_o) > 20
    assert [(int(r["i_xz"]), int(r["i_yz"])) for r in P3] == [(int(r["i_xz"]), int(r["i_yz"])) for r in P3_o]
    assert np.array_equal(P3["x"], P3_o["x"].astype(np.float32))
    assert np.array_equal(P3["y"], P3_o["y"].astype(np.float32))


def test_paper_scale_localize_end_to_end_on_oracle_frames(paper):
    """The public ulm_localize call at full size (300 frames, 16 slabs, d = 11)
    on the oracle's planes of frames 149..151 in an otherwise empty ensemble:
    its lists for frames 148..152 (every frame whose XDoppler window meets a
    non-zero frame) against the oracle's localiser on the same five frames,
    2D keys equal outside the near-tie pixels and 3D pairs equal outside the
    excluded sub-block groups (tests/ulm_lists.py); no other frame detects."""
    import ulm_lists as UL
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import list2d_numpy, list3d_numpy
    w, s, _, rf_h, _, _, _ = paper
    g, F, f0 = w.geom, w.n_frames, 148
    prm = dict(d=w.ncc_d, sig_z=0.81, sig_lat=1.45, alpha=0.1, ncc_min=0.5)
    win = O.beamform_projections(g, rf_h, frames=(149, 150, 151)).astype(np.complex64)
    five = np.zeros((5,) + win.shape[1:], dtype=np.complex64)
    five[1:4] = win
    A_o, M_o, L2_o, L3_o = O.localize(five.astype(np.complex128), prm["d"], prm["sig_z"], prm["sig_lat"],
                                      prm["alpha"], prm["ncc_min"], g.P)
    L2_o = L2_o.copy()
    L3_o = L3_o.copy()
    L2_o["frame"] += f0
    L3_o["frame"] += f0
    planes = torch.zeros(s.planes_shape(F) + (2,), device="cuda")
    planes[f0:f0 + 5] = c_tensor(five)
    out2d, n2d, out3d, n3d = s.localize(planes, rca.make_ulm_params(**prm), cap2d=1 << 18, cap3d=1 << 16)
    assert s.sync_status() == 0
    del planes
    L2 = list2d_numpy(out2d, int(n2d.item()))
    L3 = list3d_numpy(out3d, int(n3d.item()))
    assert np.all((L2["frame"] >= f0) & (L2["frame"] < f0 + 5))
    amb = UL.near_ties(A_o, M_o, prm, eps_ncc=3e-5, eps_amp=1e-5, frame_offset=f0)
    st = UL.compare(L2_o, L3_o, L2, L3, amb, g.P, pos_tol=1e-3, ncc_tol=5e-5, amp_rtol=1e-5, tz=2e-3, tr=2e-5)
    print(f"\nend to end (paper scale, frames 148-152): {st}")
    assert st["n2d"] > 300 and st["n3d"] > 20
