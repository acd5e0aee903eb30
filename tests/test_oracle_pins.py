"""Pins for the FP64 oracle: closed forms, invariants, library cross-checks and
special cases that a dropped term, a wrong sign or a transposed index would
break.  CPU only."""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle as O
from synth import workload
from synth.rca_sim import synth_rf

LAM = 1540.0 / 7.8e6  # wavelength of the synthetic workloads


def point_rf(g, pos_m, n_frames=1, amp=1.0):
    pos = torch.tensor(np.array([[pos_m]] * n_frames), dtype=torch.float64)
    a = torch.full((n_frames, 1), amp, dtype=torch.float64)
    return synth_rf(g, pos, a).numpy()


# --- geometry definitions -------------------------------------------------------

def test_geometry_closed_forms(tiny):
    g = tiny.geom
    c = g.c
    assert O.tau_rx(g, 3e-3, 4e-3) == pytest.approx(5e-3 / c, rel=1e-15)
    g0 = dataclasses.replace(g, ang_rc=(0.0,), ang_cr=(0.0,))
    assert O.tau_tx(g0, 0, 1.234e-3, 7e-3) == pytest.approx(7e-3 / c, rel=1e-15)
    # steered plane wave: a unit step in the transverse direction costs sin(th)/c
    th = g.angles[0]
    d = O.tau_tx(g, 0, 1e-3, 6e-3) - O.tau_tx(g, 0, 0.0, 6e-3)
    assert d == pytest.approx(1e-3 * math.sin(th) / c, rel=1e-9)
    # Stage-2 shift = u tan(th/2)
    for k, th in enumerate(g.angles):
        assert O.shift_dz(g, k, 2e-3) == pytest.approx(2e-3 * math.tan(th / 2), rel=1e-13)
    # Hann apodisation over a = z/F#
    z = 8e-3
    a = z / g.fnum
    assert O.apod(g, 0.0, z) == 1.0
    assert O.apod(g, a / 4, z) == pytest.approx(0.5, abs=1e-15)
    assert O.apod(g, a / 2 * 1.0000001, z) == 0.0
    # element centres are symmetric about 0 with pitch spacing
    assert O.elem_pos(g, 0) == pytest.approx(-O.elem_pos(g, g.n_el - 1), abs=1e-18)
    assert O.elem_pos(g, 1) - O.elem_pos(g, 0) == pytest.approx(g.pitch, rel=1e-12)
    assert O.slice_depth(g, 2 * g.us) == pytest.approx(O.depth(g, 2), rel=1e-15)


# --- IQ demodulation ------------------------------------------------------------

def test_fir_is_half_band_and_matches_windowed_sinc_shape():
    from scipy.signal import firwin
    h = O.fir_taps()
    assert h[15] == 0.5
    m = np.arange(-15, 16)
    assert np.all(h[(m % 2 == 0) & (m != 0)] == 0.0)
    assert np.allclose(h, h[::-1], atol=0)
    assert h.sum() == pytest.approx(1.0, abs=1e-15)
    assert (h * (-1.0) ** m).sum() == pytest.approx(0.0, abs=1e-15)
    ref = firwin(31, 0.5, window="hamming")          # cut-off fs/4, Hamming
    odd = m % 2 != 0
    ratio = h[odd] / ref[odd]
    assert np.allclose(ratio, ratio[0], rtol=1e-12)


def test_demod_pure_tone_gives_its_complex_amplitude(tiny):
    g = tiny.geom
    assert g.fs == 4 * g.fc
    A, phi = 2.5, 0.7
    t = O.t0(g) + np.arange(g.ns) / g.fs
    rf = np.broadcast_to(A * np.cos(2 * np.pi * g.fc * t + phi), (1, g.n_tx, g.n_el, g.ns)).astype(np.float32)
    iq = O.demod(g, rf, remove_mean=False)
    inner = iq[..., 15:g.ns - 15]
    # the float32 rounding of the input tone (~2e-7 relative) is the only error
    assert np.max(np.abs(inner - A * np.exp(1j * phi))) < 5e-6


def test_mean_removal_cancels_static_signal(tiny):
    g = tiny.geom
    rng = np.random.default_rng(3)
    one = (rng.standard_normal((1, g.n_tx, g.n_el, g.ns)) * 100).astype(np.float32)
    iq = O.demod(g, np.repeat(one, 4, axis=0), remove_mean=True)
    assert np.max(np.abs(iq)) < 1e-11
    # frame selection returns the same rows as the full run
    rf = rng.standard_normal((5, g.n_tx, g.n_el, g.ns)).astype(np.float32)
    full = O.demod(g, rf)
    assert np.array_equal(O.demod(g, rf, frames=[3, 1]), full[[3, 1]])


# --- beamforming ----------------------------------------------------------------

def _peak3(V, g):
    """integer argmax of |V| plus parabolic refinement along each axis (m)."""
    a = np.abs(V)
    j, m, i = np.unravel_index(np.argmax(a), a.shape)

    def para(fm, f0, fp):
        den = fm - 2 * f0 + fp
        return 0.0 if den >= 0 else (fm - fp) / (2 * den)
    x = O.elem_pos(g, j) + g.pitch * para(a[j - 1, m, i], a[j, m, i], a[j + 1, m, i])
    y = O.elem_pos(g, m) + g.pitch * para(a[j, m - 1, i], a[j, m, i], a[j, m + 1, i])
    z = O.depth(g, i) + g.dz * para(a[j, m, i - 1], a[j, m, i], a[j, m, i + 1])
    return np.array([x, y, z])


def _rc_cr_focus(V_rc, V_cr):
    """RC resolves x and z, CR resolves y and z (no transmit focusing): the
    point is where the two cross, i.e. the peak of sqrt|V_RC conj(V_CR)|."""
    return np.sqrt(np.abs(V_rc * np.conj(V_cr)))


@pytest.mark.parametrize("truth", [(0.61e-3, -0.93e-3, 8.04e-3), (-1.7e-3, 0.4e-3, 6.47e-3)])
def test_point_scatterer_focuses_full_3d(tiny, truth):
    g = tiny.geom
    truth = np.array(truth)
    iq = O.demod(g, point_rf(g, truth), remove_mean=False)
    V = _rc_cr_focus(O.das_volume(g, iq[0], 0), O.das_volume(g, iq[0], 1))
    err = np.abs(_peak3(V, g) - truth)
    assert np.all(err < LAM / 4), err


def test_point_scatterer_focuses_two_stage_steered(tiny):
    """10 deg steering and a 2.5 mm transverse offset: a wrong sign of the
    Stage-2 shift would put the focus 2 * 2.5 mm * tan(5 deg) = 0.44 mm deep."""
    g = dataclasses.replace(tiny.geom, ang_rc=(10 * math.pi / 180,), ang_cr=(10 * math.pi / 180,))
    truth = np.array([2.5e-3, 2.5e-3, 8.02e-3])
    iq = O.demod(g, point_rf(g, truth), remove_mean=False)
    S = O.stage1(g, iq[0])
    V = _rc_cr_focus(O.stage2_volume(g, S, 0), O.stage2_volume(g, S, 1))
    err = np.abs(_peak3(V, g) - truth)
    assert np.all(err < LAM / 4), err


@pytest.fixture(scope="module")
def mb_frame(tiny_rf):
    g = tiny_rf.workload.geom
    return O.demod(g, tiny_rf.rf.numpy()[:3], remove_mean=True)[1]


def test_two_stage_equals_full_3d_at_zero_steering(tiny, mb_frame):
    g = dataclasses.replace(tiny.geom, ang_rc=(0.0,), ang_cr=(0.0,))
    S = O.stage1(g, mb_frame)
    for fam in (0, 1):
        V = O.das_volume(g, mb_frame, fam)
        V2 = O.stage2_volume(g, S, fam)
        assert np.linalg.norm(V2 - V) / np.linalg.norm(V) < 1e-12


def test_two_stage_error_vs_full_3d_is_bounded(tiny, mb_frame):
    """Steered (+-3 deg) two-stage vs conventional 3D, relative L2 over the
    volume.  Measured 0.080 (RC) and 0.086 (CR) with 2x axial slice
    oversampling; bound fixed at 0.10."""
    g = tiny.geom
    S = O.stage1(g, mb_frame)
    for fam in (0, 1):
        V = O.das_volume(g, mb_frame, fam)
        V2 = O.stage2_volume(g, S, fam)
        rel = np.linalg.norm(V2 - V) / np.linalg.norm(V)
        assert rel < 0.10, (fam, rel)


def test_projection_direct_equals_slab_sum_of_volume(tiny, mb_frame):
    g = tiny.geom
    pv = np.zeros((2, 2, g.n_slab, g.nz, g.n_el), complex)
    pd = np.zeros_like(pv)
    for fam in (0, 1):
        O.project_volume(g, O.das_volume(g, mb_frame, fam), fam, pv)
        O.project_direct(g, mb_frame, fam, pd)
    assert np.linalg.norm(pd - pv) / np.linalg.norm(pv) < 1e-12
    # the XZ planes of slab b are the y-sums of the volume over that slab
    V = O.das_volume(g, mb_frame, 0)
    b = 2
    assert np.allclose(pv[0, 0, b], V[:, b * g.P:(b + 1) * g.P, :].sum(axis=1).T, rtol=0, atol=1e-12)
    assert np.allclose(pv[1, 0, b], V[b * g.P:(b + 1) * g.P, :, :].sum(axis=0).T, rtol=0, atol=1e-12)


def test_per_depth_totals_agree_across_axes(tiny, mb_frame):
    g = tiny.geom
    S = O.stage1(g, mb_frame)
    P = O.stage2_project(g, S)
    for fam in (0, 1):
        xz = P[0, fam].sum(axis=(0, 2))
        yz = P[1, fam].sum(axis=(0, 2))
        assert np.allclose(xz, yz, rtol=0, atol=1e-10 * np.abs(xz).max())


def test_beamforming_is_linear(tiny, tiny_rf):
    """BF(a x + b y) = a BF(x) + b BF(y).  Integer-valued float32 inputs keep
    the combination exact in the oracle's float32 input format."""
    g = tiny.geom
    x = np.round(tiny_rf.rf.numpy()[:3]).astype(np.float32)
    rng = np.random.default_rng(5)
    y = rng.integers(-100, 101, size=x.shape).astype(np.float32)
    a, b = 3.0, -2.0
    P1 = O.beamform_projections(g, x, frames=[1])
    P2 = O.beamform_projections(g, y, frames=[1])
    P12 = O.beamform_projections(g, (a * x + b * y).astype(np.float32), frames=[1])
    assert np.linalg.norm(P12 - (a * P1 + b * P2)) / np.linalg.norm(P12) < 1e-12


# --- XDoppler, NCC, peaks, pairing ----------------------------------------------

def test_xdoppler_constant_planes():
    F, S, nz, N = 4, 2, 6, 5
    planes = np.zeros((F, 2, 2, S, nz, N), complex)
    planes[:, :, 0] = 2.0 + 1.0j
    planes[:, :, 1] = 2.0 + 1.0j      # |P_RC conj(P_CR)| = 5 per frame
    A, M = O.xdoppler(planes)
    assert np.allclose(A[0], math.sqrt(10.0), rtol=1e-15)
    assert np.allclose(A[1:3], math.sqrt(15.0), rtol=1e-15)
    assert np.allclose(A[3], math.sqrt(10.0), rtol=1e-15)
    assert np.allclose(M, [math.sqrt(10), math.sqrt(15), math.sqrt(15), math.sqrt(10)])
    # cross-family conjugation: P_CR = conj(P_RC) gives |P_RC^2|, not |P_RC|^2 phase-free
    planes[:, :, 1] = np.conj(planes[:, :, 0])
    A2, _ = O.xdoppler(planes)
    assert np.allclose(A2[1], math.sqrt(3 * abs((2 + 1j) ** 2)))


def _gauss2(d, sz, sl):
    h = (d - 1) // 2
    q = np.arange(-h, h + 1)
    return np.exp(-q[:, None] ** 2 / (2 * sz * sz)) * np.exp(-q[None, :] ** 2 / (2 * sl * sl))


def test_ncc_is_one_on_the_kernel_and_affine_invariant():
    d, sz, sl = 5, 0.9, 1.3
    A = np.zeros((15, 17))
    A[5:10, 6:11] = _gauss2(d, sz, sl)
    n = O.ncc_plane(A, d, sz, sl, 1.0)
    assert n[7, 8] == pytest.approx(1.0, abs=1e-14)
    assert np.all(np.abs(n) <= 1 + 1e-12)
    rng = np.random.default_rng(1)
    B = rng.random((15, 17))
    n1 = O.ncc_plane(B, d, sz, sl, B.max())
    n2 = O.ncc_plane(3.0 * B + 0.25, d, sz, sl, (3.0 * B + 0.25).max())
    assert np.allclose(n1, n2, atol=1e-12)
    h = 2
    assert np.all(n1[:h] == 0) and np.all(n1[:, :h] == 0) and np.all(n1[-h:] == 0) and np.all(n1[:, -h:] == 0)


def test_ncc_brute_equals_separable_library_form():
    """Fig. 1g: the 2D NCC decomposes into successive 1D correlations.  The
    separable form here is built from scipy.ndimage 1D correlations."""
    from scipy.ndimage import correlate1d
    d, sz, sl = 7, 1.1, 0.8
    h = (d - 1) // 2
    rng = np.random.default_rng(2)
    A = rng.random((30, 24)) ** 3
    G = _gauss2(d, sz, sl)
    q = np.arange(-h, h + 1)
    gz = np.exp(-q ** 2 / (2 * sz * sz))
    gl = np.exp(-q ** 2 / (2 * sl * sl))
    box = np.ones(d)

    def sep(X, kz, kl):
        return correlate1d(correlate1d(X, kz, axis=0, mode="constant"), kl, axis=1, mode="constant")
    s1 = sep(A, box, box)
    s2 = sep(A * A, box, box)
    sg = sep(A, gz, gl)
    muG = G.mean()
    num = sg - muG * s1
    ssA = s2 - s1 * s1 / d ** 2
    ssG = ((G - muG) ** 2).sum()
    ref = num / np.sqrt(ssA * ssG)
    n = O.ncc_plane(A, d, sz, sl, A.max())
    inner = (slice(h, -h), slice(h, -h))
    assert np.allclose(n[inner], ref[inner], rtol=0, atol=1e-10)


def test_peak_subpixel_recovers_parabola_vertex():
    nz, N = 9, 9
    z0, l0 = 4.3, 3.8
    ii, ll = np.meshgrid(np.arange(nz), np.arange(N), indexing="ij")
    ncc = 0.95 - 0.02 * (ii - z0) ** 2 - 0.03 * (ll - l0) ** 2
    A = np.ones((nz, N))
    out = O.peaks_plane(A, ncc, 1.0, 0.1, 0.5)
    assert len(out) == 1
    assert (out[0]["iz"], out[0]["ilat"]) == (4, 4)
    assert out[0]["z"] == pytest.approx(z0, abs=1e-12)
    assert out[0]["lat"] == pytest.approx(l0, abs=1e-12)


def test_peak_ties_go_to_earlier_raster_pixel_and_thresholds_are_inclusive():
    ncc = np.zeros((6, 6))
    ncc[2, 2] = ncc[2, 3] = 0.8          # equal neighbours in one row
    ncc[4, 4] = 0.5                      # exactly ncc_min
    A = np.ones((6, 6))
    A[4, 4] = 0.1                        # exactly alpha * Mt
    out = O.peaks_plane(A, ncc, 1.0, 0.1, 0.5)
    assert [(int(o["iz"]), int(o["ilat"])) for o in out] == [(2, 2), (4, 4)]
    A[4, 4] = np.nextafter(0.1, 0.0)
    out = O.peaks_plane(A, ncc, 1.0, 0.1, 0.5)
    assert [(int(o["iz"]), int(o["ilat"])) for o in out] == [(2, 2)]
    ncc[3, 2] = 0.8                      # equal neighbour in a later row: earlier still wins
    out = O.peaks_plane(np.ones((6, 6)), ncc, 1.0, 0.1, 0.5)
    assert [(int(o["iz"]), int(o["ilat"])) for o in out][0] == (2, 2)
    assert (3, 2) not in [(int(o["iz"]), int(o["ilat"])) for o in out]


def _l2(rows):
    L = np.zeros(len(rows), dtype=O.LOC2D)
    for q, (frame, axis, slab, iz, ilat, z, lat, amp) in enumerate(rows):
        L[q] = (frame, axis, slab, iz, ilat, z, lat, 0.9, amp)
    return L


def test_pairing_rules():
    P = 8
    # XZ (axis 0) in y-slab 1 at x pixel 10 -> sub-block (1, 1);
    # YZ (axis 1) in x-slab 1 at y pixel 12 -> sub-block (1, 1).
    L = _l2([
        (0, 0, 1, 20, 10, 20.0, 10.2, 1.00),   # 0 XZ
        (0, 1, 1, 21, 12, 21.0, 12.1, 1.00),   # 1 YZ  |dz| = 1.0 -> eligible
        (0, 1, 1, 22, 13, 21.0000001, 13.0, 1.00),  # 2 YZ  |dz| > 1 -> not
    ])
    L3 = O.pair3d(L, P)
    assert [(r["i_xz"], r["i_yz"]) for r in L3] == [(0, 1)]
    assert L3[0]["x"] == 10.2 and L3[0]["y"] == 12.1 and L3[0]["z"] == 20.5
    # ratio window is inclusive at 0.9 and 1.11
    L = _l2([(0, 0, 1, 20, 10, 20.0, 10.0, 0.9), (0, 1, 1, 20, 12, 20.0, 12.0, 1.0)])
    assert len(O.pair3d(L, P)) == 1
    L = _l2([(0, 0, 1, 20, 10, 20.0, 10.0, 1.11), (0, 1, 1, 20, 12, 20.0, 12.0, 1.0)])
    assert len(O.pair3d(L, P)) == 1
    L = _l2([(0, 0, 1, 20, 10, 20.0, 10.0, 1.12), (0, 1, 1, 20, 12, 20.0, 12.0, 1.0)])
    assert len(O.pair3d(L, P)) == 0
    # different sub-block or different frame -> never paired
    L = _l2([(0, 0, 1, 20, 10, 20.0, 10.0, 1.0), (0, 1, 2, 20, 12, 20.0, 12.0, 1.0)])
    assert len(O.pair3d(L, P)) == 0
    L = _l2([(0, 0, 1, 20, 10, 20.0, 10.0, 1.0), (1, 1, 1, 20, 12, 20.0, 12.0, 1.0)])
    assert len(O.pair3d(L, P)) == 0


def test_pairing_mutual_minimum_ratio():
    P = 8
    L = _l2([
        (0, 0, 0, 5, 1, 5.0, 1.0, 1.00),   # 0 XZ
        (0, 0, 0, 5, 3, 5.0, 3.0, 1.05),   # 1 XZ
        (0, 1, 0, 5, 2, 5.0, 2.0, 1.04),   # 2 YZ: closest to XZ1 (ratio 1.0096)
        (0, 1, 0, 5, 6, 5.5, 6.0, 0.98),   # 3 YZ: closest to XZ0 (1.0204)
    ])
    L3 = O.pair3d(L, P)
    assert sorted((int(r["i_xz"]), int(r["i_yz"])) for r in L3) == [(0, 3), (1, 2)]
    # a YZ preferred by two XZs goes to the cheaper one; the other stays unpaired
    L = _l2([
        (0, 0, 0, 5, 1, 5.0, 1.0, 1.00),
        (0, 0, 0, 5, 3, 5.0, 3.0, 1.02),
        (0, 1, 0, 5, 2, 5.0, 2.0, 1.01),
    ])
    L3 = O.pair3d(L, P)
    assert [(int(r["i_xz"]), int(r["i_yz"])) for r in L3] == [(1, 2)]
    # exact tie in cost goes to the lower list index
    L = _l2([
        (0, 0, 0, 5, 1, 5.0, 1.0, 1.00),
        (0, 0, 0, 5, 3, 5.0, 3.0, 1.00),
        (0, 1, 0, 5, 2, 5.0, 2.0, 1.00),
    ])
    L3 = O.pair3d(L, P)
    assert [(int(r["i_xz"]), int(r["i_yz"])) for r in L3] == [(0, 2)]


def test_end_to_end_tiny_localises_simulated_mbs(tiny, tiny_rf):
    """Seeded tiny ensemble: detections paired into 3D lie near visible MBs."""
    from synth.rca_sim import visible_mask
    g = tiny.geom
    frames = range(20, 26)
    planes = O.beamform_projections(g, tiny_rf.rf.numpy(), frames=frames)
    A, M, L2, L3 = O.localize(planes, d=5, sig_z=1.0, sig_l=1.0, alpha=0.1, ncc_min=0.5, P=g.P)
    assert len(L2) > 0 and len(L3) > 0
    vis = visible_mask(tiny, tiny_rf.fields)
    hits = 0
    for r in L3:
        f = frames[0] + int(r["frame"])
        x = O.elem_pos(g, 0) + r["x"] * g.pitch
        y = O.elem_pos(g, 0) + r["y"] * g.pitch
        z = g.z0 + r["z"] * g.dz
        d = np.linalg.norm(tiny_rf.fields.mb_pos[f][vis[f]] - np.array([x, y, z]), axis=1)
        hits += int(d.size > 0 and d.min() < 0.3e-3)
    assert hits >= 0.5 * len(L3), (hits, len(L3))
