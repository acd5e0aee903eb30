"""GPU parity of microbubble separation (Sec. II-A5) against the numpy FP64
oracle on the same complex64 planes: the complex subsets of `ulm_separate`
and the fused per-subset XDoppler amplitude and frame maxima of
`ulm_separate_enhance`.

Tolerances: the FP32 transforms round at the scale of the whole slow-time
signal, so each subset's error is bounded against the input's norm
(rel-L2 <= 1e-5 of ||planes||), and against the subset's own norm (1e-4)
where it holds at least 1 % of the energy.  The amplitudes follow the
enhancement test: rel-L2 <= 2e-5 of the oracle's per-subset A, maxima 2e-5."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import separation as OSep

pytestmark = pytest.mark.gpu


def c64(x):
    a = np.stack([x.real, x.imag], axis=-1).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_c(t):
    a = t.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def S(tiny):
    from paper_2511_21647_gb300.pipeline import RcaSession
    s = RcaSession(tiny.geom)
    yield s
    s.close()


@pytest.fixture(scope="module")
def tiny_planes(tiny, tiny_rf):
    """the oracle's planes of the tiny ensemble (64 frames), as complex64"""
    return O.beamform_projections(tiny.geom, tiny_rf.rf.numpy()).astype(np.complex64)


def check_subsets(got, ref, x, label):
    nx = np.linalg.norm(x)
    etot = sum(np.linalg.norm(r) ** 2 for r in ref)
    worst = 0.0
    for s in range(ref.shape[0]):
        e = np.linalg.norm(got[s] - ref[s])
        worst = max(worst, e / nx)
        assert e <= 1e-5 * nx, (label, s, e / nx)
        if np.linalg.norm(ref[s]) ** 2 >= 0.01 * etot:
            assert e <= 1e-4 * np.linalg.norm(ref[s]), (label, s, e / np.linalg.norm(ref[s]))
    return worst


def test_subsets_match_oracle_on_tiny_ensemble(S, tiny, tiny_planes):
    from paper_2511_21647_gb300 import rca
    prm = rca.make_sep_params(tiny.frame_rate, 3)
    got = to_c(S.separate(c64(tiny_planes), prm))
    torch.cuda.synchronize()
    assert S.sync_status() == 0
    ref = OSep.separate(tiny_planes.astype(np.complex128), tiny.frame_rate, np.array(prm.edges_hz[:4]))
    w = check_subsets(got, ref, tiny_planes, "tiny")
    print(f"\ntiny ensemble, 6 subsets: worst error {w:.2e} of the input")


@pytest.mark.parametrize("F", [1, 2, 5, 30, 60, 100, 128, 150, 300, 320, 480, 512])
def test_subsets_match_oracle_frame_counts(S, tiny, F):
    """random planes of the tiny geometry with every radix plan the library
    uses (2 .. 20, one to three passes) and the 1-frame degenerate case;
    uneven band edges with a low cut"""
    from paper_2511_21647_gb300 import rca
    rng = np.random.default_rng(F)
    shape = S.planes_shape(F)
    x = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    prf = 400.0
    edges = [5.0, 30.0, 90.0, 200.0]
    prm = rca.make_sep_params(prf, 3, edges)
    got = to_c(S.separate(c64(x), prm))
    torch.cuda.synchronize()
    assert S.sync_status() == 0
    ref = OSep.separate(x.astype(np.complex128), prf, np.array(edges))
    if F == 1:
        assert np.all(got == 0)
    else:
        check_subsets(got, ref, x, F)


@pytest.mark.parametrize("n_bands", [1, 2, 3, 4])
def test_band_counts(S, tiny, tiny_planes, n_bands):
    from paper_2511_21647_gb300 import rca
    prm = rca.make_sep_params(tiny.frame_rate, n_bands)
    got = to_c(S.separate(c64(tiny_planes), prm))
    ref = OSep.separate(tiny_planes.astype(np.complex128), tiny.frame_rate, np.array(prm.edges_hz[:n_bands + 1]))
    assert got.shape[0] == 2 * n_bands
    check_subsets(got, ref, tiny_planes, n_bands)


@pytest.mark.parametrize("enh", [0, 1])
def test_fused_enhancement_matches_oracle(S, tiny, tiny_planes, enh):
    from paper_2511_21647_gb300 import _lib as L, rca
    prm = rca.make_sep_params(tiny.frame_rate, 3)
    A, M = S.separate_enhance(c64(tiny_planes), prm, enh=enh)
    torch.cuda.synchronize()
    assert S.sync_status() == 0
    edges = np.array(prm.edges_hz[:4])
    subs = OSep.separate(tiny_planes.astype(np.complex128), tiny.frame_rate, edges)
    A, M = A.cpu().numpy(), M.cpu().numpy()
    for s in range(6):
        if enh == L.ULM_ENH_XDOPPLER:
            A_o, M_o = O.xdoppler(subs[s])
        else:
            A_o = np.abs(subs[s][:, :, 0] + subs[s][:, :, 1])
            M_o = A_o.reshape(A_o.shape[0], -1).max(axis=1)
        assert rel(A[s], A_o) < 2e-5, (s, rel(A[s], A_o))
        assert np.allclose(M[s], M_o, rtol=2e-5, atol=0), s
    # the same as separating, then enhancing each subset with ulm_enhance (the
    # fused kernel's square roots are the approximate ones, 2^-23 relative)
    sub_dev = S.separate(c64(tiny_planes), prm)
    for s in range(6):
        A2, M2 = S.enhance(sub_dev[s].contiguous(), enh=enh)
        assert rel(A[s], A2.cpu().numpy()) < 2e-6
        assert np.allclose(M[s], M2.cpu().numpy(), rtol=2e-6, atol=0)


@pytest.mark.parametrize("F", [64, 300])
@pytest.mark.parametrize("enh", [0, 1])
def test_fused_enhancement_random_planes(S, F, enh):
    """both amplitude modes on the generic plan (64 frames) and the 300-frame
    compile-time plan, random planes of the tiny geometry"""
    from paper_2511_21647_gb300 import _lib as L, rca
    rng = np.random.default_rng(100 + F + enh)
    shape = S.planes_shape(F)
    x = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    prm = rca.make_sep_params(400.0, 3)
    A, M = S.separate_enhance(c64(x), prm, enh=enh)
    torch.cuda.synchronize()
    assert S.sync_status() == 0
    subs = OSep.separate(x.astype(np.complex128), 400.0, np.array(prm.edges_hz[:4]))
    A, M = A.cpu().numpy(), M.cpu().numpy()
    for s in range(6):
        if enh == L.ULM_ENH_XDOPPLER:
            A_o, M_o = O.xdoppler(subs[s])
        else:
            A_o = np.abs(subs[s][:, :, 0] + subs[s][:, :, 1])
            M_o = A_o.reshape(F, -1).max(axis=1)
        assert rel(A[s], A_o) < 2e-5, (s, rel(A[s], A_o))
        assert np.allclose(M[s], M_o, rtol=2e-5, atol=0), s


def test_subset_localisation_runs_on_fused_output(S, tiny, tiny_planes):
    """each subset's A / M slice feeds ulm_detect2d and ulm_pair3d as they
    are; the 2D and 3D lists equal the oracle's localiser on the oracle's
    XDoppler of that subset outside the near-tie pixels and groups
    (tests/ulm_lists.py).  The fused amplitudes carry the FP32 transforms'
    error (rel-L2 <= 2e-5 above), so the candidate margins are 2e-4 in NCC and
    2e-5 M_t in amplitude, positions 2e-3 px, intensities 1e-4."""
    import json
    import os
    import ulm_lists as UL
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import list2d_numpy, list3d_numpy
    here = os.path.dirname(os.path.abspath(__file__))
    psf = json.load(open(os.path.join(here, "golden", "psf_sigma.json")))["tiny"]
    prm = rca.make_sep_params(tiny.frame_rate, 3)
    p = dict(d=5, sig_z=psf["sig_z"], sig_lat=psf["sig_lat"], alpha=0.1, ncc_min=0.5)
    ulm = rca.make_ulm_params(**p)
    A, M = S.separate_enhance(c64(tiny_planes), prm)
    subs = OSep.separate(tiny_planes.astype(np.complex128), tiny.frame_rate, np.array(prm.edges_hz[:4]))
    total = 0
    for s in range(6):
        out, n2d, _ = S.detect2d(A[s], M[s], ulm)
        out3, n3d = S.pair3d(out, n2d, out.shape[0], tiny.n_frames)
        L2 = list2d_numpy(out, int(n2d.item()))
        L3 = list3d_numpy(out3, int(n3d.item()))
        A_o, M_o = O.xdoppler(subs[s])
        L2_o = O.localize2d(A_o, M_o, 5, psf["sig_z"], psf["sig_lat"], 0.1, 0.5)
        L3_o = O.pair3d(L2_o, tiny.geom.P)
        amb = UL.near_ties(A_o, M_o, p, eps_ncc=2e-4, eps_amp=2e-5)
        st = UL.compare(L2_o, L3_o, L2, L3, amb, tiny.geom.P, pos_tol=2e-3, ncc_tol=2e-4, amp_rtol=1e-4, tz=4e-3,
                        tr=2e-4)
        print(f"\nsubset {s}: {st}")
        total += st["n2d"]
    assert S.sync_status() == 0
    assert total > 0


def test_paper_geometry_300_frames_sampled_pixels():
    """the paper's plane stack (300 frames, 2 x 2 x 16 x 250 x 128) of seeded
    random values; the oracle on 4000 sampled pixels' slow-time signals"""
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import RcaSession
    from synth import workload
    w = workload("paper")
    with RcaSession(w.geom) as s:
        F = w.n_frames
        shape = s.planes_shape(F)
        gen = torch.Generator(device="cuda").manual_seed(11)
        x = torch.randn(shape + (2,), device="cuda", generator=gen)
        prm = rca.make_sep_params(w.frame_rate, 3)
        A, M = s.separate_enhance(x, prm)
        sub = s.separate(x, prm)
        torch.cuda.synchronize()
        assert s.sync_status() == 0
        rng = np.random.default_rng(12)
        npx = int(np.prod(shape[1:]))
        idx = torch.from_numpy(rng.choice(npx, 4000, replace=False)).cuda()
        xs = to_c(x.reshape(F, npx, 2)[:, idx])
        gs = to_c(sub.reshape(6, F, npx, 2)[:, :, idx])
        del sub
        ref = OSep.separate(xs.astype(np.complex128), w.frame_rate, np.array(prm.edges_hz[:4]))
        w_err = check_subsets(gs, ref, xs, "paper")
        # fused amplitude at sampled (axis, slab, z, lat) pixels: RC and CR of each
        a_px = int(np.prod(shape[3:]))
        sel = rng.choice(2 * a_px, 2000, replace=False)
        axis, rest = sel // a_px, sel % a_px
        fam_idx = lambda fam: axis * 2 * a_px + fam * a_px + rest
        xr = to_c(x.reshape(F, npx, 2)[:, torch.from_numpy(fam_idx(0)).cuda()])
        xc = to_c(x.reshape(F, npx, 2)[:, torch.from_numpy(fam_idx(1)).cuda()])
        edges = np.array(prm.edges_hz[:4])
        sr = OSep.separate(xr.astype(np.complex128), w.frame_rate, edges)
        scr = OSep.separate(xc.astype(np.complex128), w.frame_rate, edges)
        As = A.reshape(6, F, 2 * a_px)[:, :, torch.from_numpy(sel).cuda()].cpu().numpy()
        for k in range(6):
            q = sr[k] * scr[k].conj()
            qs = q.copy()
            qs[1:] += q[:-1]
            qs[:-1] += q[1:]
            A_o = np.sqrt(np.abs(qs))
            assert rel(As[k], A_o) < 2e-5, (k, rel(As[k], A_o))
        assert np.all(M.cpu().numpy() >= As.max(axis=2) * (1 - 1e-6))
    print(f"\npaper geometry, 300 frames: worst subset error {w_err:.2e} of the input")


def test_argument_errors(S, tiny):
    from paper_2511_21647_gb300 import _lib as L, rca
    x = torch.zeros(S.planes_shape(8) + (2,), device="cuda")
    bad = [rca.make_sep_params(0.0, 3), rca.make_sep_params(400.0, 3, [10.0, 5.0, 100.0, 200.0]),
           rca.make_sep_params(400.0, 3, [-1.0, 50.0, 100.0, 200.0])]
    p = rca.make_sep_params(400.0, 3)
    p.n_bands = 5
    bad.append(p)
    p = rca.make_sep_params(400.0, 1)
    p.n_bands = 0
    bad.append(p)
    for prm in bad:
        with pytest.raises(rca.RcaError) as e:
            S.separate(x, prm)
        assert e.value.status == L.RCA_ERR_INVALID_ARG
    with pytest.raises(rca.RcaError) as e:
        S.separate_enhance(x, rca.make_sep_params(400.0, 3), enh=7)
    assert e.value.status == L.RCA_ERR_INVALID_ARG
    for F in (7, 1024):
        y = torch.zeros(S.planes_shape(F) + (2,), device="cuda")
        with pytest.raises(rca.RcaError) as e:
            S.separate(y, rca.make_sep_params(400.0, 3))
        assert e.value.status == L.RCA_ERR_UNSUPPORTED
