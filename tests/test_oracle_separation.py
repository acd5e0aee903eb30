"""Pins of the oracle's microbubble separation (Sec. II-A5): a pure slow-time
tone lands whole in the subset its frequency selects (band edges inclusive
above, exclusive below); the subsets plus the DC and Nyquist components add
back to the input; each subset equals a brute-force inverse DFT over its bins;
a real signal's up and down subsets are complex conjugates; and, through the
oracle's beamformer, a scatterer moving toward the array lands in the up subset
of the speed band that its Doppler shift 2 v fc / c selects (and away from it,
in the down subset)."""
import numpy as np
import pytest
import torch

from oracle import separation as OSep


def test_bin_table_closed_form():
    prf = 400.0
    e = OSep.default_edges(prf, 3)
    assert np.allclose(e, [0.0, 200.0 / 3, 400.0 / 3, 200.0])
    sub = OSep.bin_subsets(300, prf, e)
    # 300 frames at 400 Hz: bin width 4/3 Hz, bands of 50 bins each way
    assert sub[0] == -1 and sub[150] == -1
    assert np.all(sub[1:51] == 0) and np.all(sub[51:101] == 1) and np.all(sub[101:150] == 2)
    assert np.all(sub[250:300] == 3) and np.all(sub[200:250] == 4) and np.all(sub[151:200] == 5)
    # odd F: no Nyquist bin, the top bin pair is in the last band
    sub = OSep.bin_subsets(7, 7.0, OSep.default_edges(7.0, 1))
    assert list(sub) == [-1, 0, 0, 0, 1, 1, 1]


def test_tone_lands_in_its_subset_and_edges():
    F, prf = 60, 60.0  # 1 Hz bins
    edges = np.array([2.0, 10.0, 20.0, 30.0])  # band 0 = (2, 10], bins 1, 2 in no band
    t = np.arange(F)
    for k in (-29, -20, -11, -10, -3, -2, -1, 0, 1, 2, 3, 10, 11, 20, 21, 29, 30):
        x = np.exp(2j * np.pi * k * t / F)[:, None] * np.array([1.0, 2.0 - 1.0j])[None, :]
        subs = OSep.separate(x, prf, edges)
        f = abs(k)
        band = next((b for b in range(3) if edges[b] < f <= edges[b + 1]), None)
        if k == 0 or abs(k) == F // 2 or band is None:
            want = None
        else:
            want = (0 if k > 0 else 1) * 3 + band
        for s in range(6):
            ref = x if s == want else np.zeros_like(x)
            assert np.abs(subs[s] - ref).max() < 1e-12, (k, s)


def test_subsets_add_back_and_match_brute_force_dft():
    rng = np.random.default_rng(7)
    for F in (1, 2, 9, 16, 30):
        x = rng.normal(size=(F, 3, 2)) + 1j * rng.normal(size=(F, 3, 2))
        prf = 400.0
        edges = OSep.default_edges(prf, 3)
        subs = OSep.separate(x, prf, edges)
        # DC + Nyquist complete the decomposition
        rest = np.broadcast_to(x.mean(axis=0), x.shape).copy()
        if F % 2 == 0:
            alt = (-1.0) ** np.arange(F)
            rest += alt[:, None, None] * (alt[:, None, None] * x).mean(axis=0)[None]
        assert np.abs(subs.sum(axis=0) + rest - x).max() < 1e-12
        # each subset = (1/F) sum over its bins of X[j] exp(+2 pi i j t / F), X by a brute-force DFT
        W = np.exp(-2j * np.pi * np.outer(np.arange(F), np.arange(F)) / F)
        X = np.einsum("jt,tab->jab", W, x)
        sub = OSep.bin_subsets(F, prf, edges)
        for s in range(6):
            sel = sub == s
            y = np.einsum("tj,jab->tab", W.conj()[:, sel], X[sel]) / F
            assert np.abs(subs[s] - y).max() < 1e-12, (F, s)


def test_real_signal_up_and_down_are_conjugate():
    rng = np.random.default_rng(8)
    x = rng.normal(size=(40, 5))
    subs = OSep.separate(x, 400.0, OSep.default_edges(400.0, 2))
    for b in range(2):
        assert np.abs(subs[b] - subs[2 + b].conj()).max() < 1e-12


@pytest.mark.parametrize("v_z, want", [(-3.3e-3, 0), (-9.9e-3, 1), (-16.5e-3, 2),
                                       (3.3e-3, 3), (9.9e-3, 4), (16.5e-3, 5)])
def test_moving_scatterer_lands_in_its_speed_and_direction(tiny, v_z, want):
    """A single scatterer on the array axis moving with axial velocity v_z
    (negative = toward the array) at the frame rate 400 Hz: its Doppler shift
    -2 v_z fc / c (33, 100, 167 Hz, the centres of the three equal bands over
    (0, 200] Hz) decides the subset; the oracle beamforms 64 frames without
    clutter removal and the subset holding the energy is checked.  The echo's
    bandwidth (65 % of fc) spreads the shift by about a third either way, so
    the lower two bands hold nearly all of it; the top band loses part to the
    band below and, past prf / 2, wraps into the opposite direction."""
    import oracle as O
    from synth import synth_rf
    g = tiny.geom
    F, prf = 64, tiny.frame_rate
    z0 = g.z0 + 0.5 * g.nz * g.dz
    t = np.arange(F) / prf
    pos = np.zeros((F, 1, 3))
    pos[:, 0, 2] = z0 + v_z * t
    rf = synth_rf(g, torch.as_tensor(pos), torch.ones(1, dtype=torch.float64)).to(torch.float32)
    planes = O.beamform_projections(g, rf.numpy(), remove_mean=False)
    fd = -2.0 * v_z * g.fc / g.c
    edges = OSep.default_edges(prf, 3)
    band = next(b for b in range(3) if edges[b] < abs(fd) <= edges[b + 1])
    assert (0 if fd > 0 else 1) * 3 + band == want
    subs = OSep.separate(planes, prf, edges)
    energy = np.array([np.sum(np.abs(s) ** 2) for s in subs])
    frac = energy / energy.sum()
    opposite = [s for s in range(6) if (s < 3) != (want < 3)]
    print(f"\nv_z {v_z * 1e3:+.1f} mm/s, fd {fd:+.1f} Hz: subset energy fractions {np.round(frac, 3)}")
    assert int(np.argmax(frac)) == want
    if want % 3 < 2:
        assert frac[want] > 0.85 and frac[opposite].sum() < 0.02
    else:
        assert frac[want] > 0.6 and frac[opposite].sum() < 0.1
