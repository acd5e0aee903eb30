"""GPU parity of projection-based motion estimation (Sec. II-A3) against the
numpy FP64 oracle on the same seeded slice stacks: integer correlation peaks
identical (a peak whose runner-up is within the FP32 error of the FFTs may go
either way and is listed), sub-pixel shifts, NCC and the 3D displacement
within the FP32 error of a 2D FFT of the slice's size.  Tiny geometry (all
frames) and the paper geometry at the benchmark's 300 frames (sampled
frames)."""
import numpy as np
import pytest
import torch

from oracle import motion as OM

pytestmark = pytest.mark.gpu


def c_tensor(x):
    a = np.stack([x.real, x.imag], axis=-1).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_gpu(s, sl, F, nt):
    from paper_2511_21647_gb300 import rca
    motion = torch.zeros((F, 3), device="cuda")
    shifts = torch.zeros((F, nt, 3), device="cuda")
    peaks = torch.full((F, nt, 2), -999, dtype=torch.int32, device="cuda")
    rca.rca_motion_estimate(s.h, s.t, sl, F, motion, shifts, peaks)
    torch.cuda.synchronize()
    assert s.sync_status() == 0
    return motion.cpu().numpy(), shifts.cpu().numpy(), peaks.cpu().numpy()


def near_tie(s_f, s_0, rel=1e-5):
    """the oracle's |R| has a runner-up within rel of its peak"""
    _, _, _, mag = OM.correlate(s_f, s_0)
    top = np.sort(mag, axis=None)[-2:]
    return top[1] - top[0] <= rel * top[1]


def compare(g, sl, frames, motion, shifts, peaks):
    sh_o, pk_o, mo_o = OM.estimate(g, sl, frames)
    amb = 0
    for q, f in enumerate(frames):
        for k in range(sl.shape[1]):
            if tuple(peaks[f, k]) != tuple(pk_o[q, k]):
                assert near_tie(sl[f, k], sl[0, k]), (f, k, peaks[f, k], pk_o[q, k])
                amb += 1
                continue
            assert abs(shifts[f, k, 0] - sh_o[q, k, 0]) < 2e-3, (f, k)
            assert abs(shifts[f, k, 1] - sh_o[q, k, 1]) < 2e-3, (f, k)
            assert abs(shifts[f, k, 2] - sh_o[q, k, 2]) < 1e-4, (f, k)
    if amb == 0:
        row_m = g.dz / g.us
        assert np.all(np.abs(motion[list(frames), :2] - mo_o[:, :2]) < 2e-3 * g.pitch)
        assert np.all(np.abs(motion[list(frames), 2] - mo_o[:, 2]) < 2e-3 * row_m)
    return sh_o, mo_o


def test_motion_matches_oracle_tiny(tiny):
    from paper_2511_21647_gb300.pipeline import RcaSession
    from synth import moving_slices
    g = tiny.geom
    F, K = 12, len(g.ang_rc)
    rng = np.random.default_rng(8)
    disp = np.concatenate([np.zeros((1, 3)), rng.uniform(-250e-6, 250e-6, size=(F - 1, 3))])
    sl = moving_slices(g, F, K, disp, seed=12, sigma_rows=2.5, sigma_px=1.2)
    with RcaSession(g) as s:
        motion, shifts, peaks = run_gpu(s, c_tensor(sl), F, 2 * K)
    compare(g, sl, range(F), motion, shifts, peaks)
    # the reference frame correlates with itself
    assert np.all(peaks[0] == 0) and np.allclose(shifts[0, :, 2], 1.0, atol=1e-5)
    # and the displacements follow the field's (a tenth of a pixel)
    assert np.all(np.abs(motion[:, 0] - disp[:, 0]) < 0.1 * g.pitch)
    assert np.all(np.abs(motion[:, 2] - disp[:, 2]) < 0.1 * g.dz / g.us)


def test_motion_paper_geometry_300_frames_sampled(tiny):
    """the paper workload's geometry and frame count, a 0.2 mm 1 Hz axial
    sinusoid at 400 Hz (the tissue motion of the paper-scale workload) plus a
    small lateral drift"""
    from paper_2511_21647_gb300.pipeline import RcaSession
    from synth import moving_slices, workload
    w = workload("paper")
    g, F = w.geom, w.n_frames
    K = len(g.ang_rc)
    t = np.arange(F) / 400.0
    disp = np.stack([20e-6 * t / t[-1], -30e-6 * t / t[-1], 0.2e-3 * np.sin(2 * np.pi * t)], axis=1)
    sl = moving_slices(g, F, K, disp, seed=13, sigma_rows=2.5, sigma_px=1.2)
    with RcaSession(g) as s:
        motion, shifts, peaks = run_gpu(s, c_tensor(sl), F, 2 * K)
    frames = (0, 1, 100, 150, 299)
    compare(g, sl, frames, motion, shifts, peaks)
    err = np.abs(motion[:, 2] - disp[:, 2])
    print(f"\npaper geometry, 300 frames: axial error max {err.max() * 1e6:.2f} um, "
          f"lateral x {np.abs(motion[:, 0] - disp[:, 0]).max() * 1e6:.2f} um")
    assert err.max() < 0.1 * g.dz / g.us


def test_single_frame_and_unsupported_width(tiny):
    import dataclasses
    from paper_2511_21647_gb300 import _lib, rca
    from paper_2511_21647_gb300.pipeline import RcaSession
    from synth import moving_slices
    g = tiny.geom
    K = len(g.ang_rc)
    sl = moving_slices(g, 1, K, np.zeros((1, 3)), seed=2)
    with RcaSession(g) as s:
        motion, shifts, peaks = run_gpu(s, c_tensor(sl), 1, 2 * K)
    assert np.all(peaks == 0) and np.allclose(motion, 0.0)
    g24 = dataclasses.replace(g, n_el=24)
    with RcaSession(g24) as s:
        sl24 = torch.zeros((2, 2 * K, g24.nzs, 24, 2), device="cuda")
        with pytest.raises(rca.RcaError) as e:
            rca.rca_motion_estimate(s.h, s.t, sl24, 2, torch.zeros((2, 3), device="cuda"))
        assert e.value.status == _lib.RCA_ERR_UNSUPPORTED
