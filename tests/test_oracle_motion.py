"""Pins of the oracle's projection-based motion estimation (Sec. II-A3): exact
recovery of integer circular shifts (positive, negative, wrapping), the
reference frame at zero shift with NCC 1, sub-pixel shifts of a blob field
within the parabolic estimator's bias, and the RC / CR combination on a
rigidly moving field with a known 3D displacement."""
import numpy as np

from oracle import motion as OM


def test_integer_circular_shifts_are_recovered_exactly(tiny):
    g = tiny.geom
    rng = np.random.default_rng(3)
    nzs, N = g.nzs, g.n_el
    s0 = np.zeros((nzs, N), dtype=np.complex128)
    s0[30:nzs - 30] = rng.normal(size=(nzs - 60, N)) + 1j * rng.normal(size=(nzs - 60, N))
    for dz, dx in ((0, 0), (7, 3), (-12, -5), (20, 15), (-3, 16)):
        sf = np.roll(np.roll(s0, dz, axis=0), dx, axis=1)
        pk, (sz, sx), ncc, _ = OM.correlate(sf, s0)
        zp, xp = OM.padded_shape(nzs, N)
        want_x = dx if dx < xp // 2 else dx - xp
        assert pk == (dz, want_x)
        assert abs(sz - dz) < 1e-9 and abs(sx - want_x) < 1e-9
        assert abs(ncc - 1.0) < 1e-12


def test_subpixel_shift_of_a_blob_field(tiny):
    from synth import moving_slices
    g = tiny.geom
    row_m = g.dz / g.us
    true_rows, true_px = 2.3, -0.6
    disp = np.array([[0.0, 0.0, 0.0], [true_px * g.pitch, -true_px * g.pitch, true_rows * row_m]])
    sl = moving_slices(g, 2, 1, disp, seed=5, sigma_rows=2.5, sigma_px=1.2)
    shifts, peaks, motion = OM.estimate(g, sl)
    assert np.allclose(shifts[0, :, :2], 0.0) and np.allclose(shifts[0, :, 2], 1.0)
    assert tuple(peaks[1, 0]) == (2, -1) and tuple(peaks[1, 1]) == (2, 1)
    # parabolic refinement of a Gaussian correlation peak: within 0.1 pixel
    assert abs(shifts[1, 0, 0] - true_rows) < 0.1 and abs(shifts[1, 0, 1] - true_px) < 0.1
    assert abs(shifts[1, 1, 0] - true_rows) < 0.1 and abs(shifts[1, 1, 1] + true_px) < 0.1


def test_rc_cr_combination_recovers_a_3d_displacement(tiny):
    from synth import moving_slices
    g = tiny.geom
    K = 2
    F = 4
    disp = np.array([[0, 0, 0], [40e-6, -25e-6, 30e-6], [-90e-6, 60e-6, -55e-6], [214e-6, 0.0, 100e-6]])
    sl = moving_slices(g, F, K, disp, seed=9, sigma_rows=2.5, sigma_px=1.2)
    shifts, peaks, motion = OM.estimate(g, sl)
    # within a tenth of a pixel on each axis (21 um lateral, 5 um axial)
    assert np.all(np.abs(motion[:, 0] - disp[:, 0]) < 0.1 * g.pitch)
    assert np.all(np.abs(motion[:, 1] - disp[:, 1]) < 0.1 * g.pitch)
    assert np.all(np.abs(motion[:, 2] - disp[:, 2]) < 0.1 * g.dz / g.us)
    assert np.all(shifts[:, :, 2] > 0.9)
