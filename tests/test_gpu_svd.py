"""GPU parity of the eigen-based SVD clutter filter (Sec. II-A2) against the
numpy FP64 oracle on the same FP32 slices.  The scenes are exact SVDs: a
tissue component of the filter's rank, 40 to 60 dB above the blood, with
orthonormal spatial and temporal bases, so the dominant eigenspace is well
separated and both sides must remove the same subspace.  The FP32 error is
measured against the unfiltered slices' norm (the covariance and the
projection round at the tissue's scale) and reported against the blood's."""
import numpy as np
import pytest
import torch

from oracle import svd_filter as OS

pytestmark = pytest.mark.gpu


def exact_svd_scene(rng, F, nt, nzs, N, rank, amp):
    P = nzs * N
    tissue = np.zeros((F, nt, nzs, N), dtype=np.complex128)
    blood = np.zeros_like(tissue)
    for k in range(nt):
        Q, _ = np.linalg.qr(rng.normal(size=(F, F)) + 1j * rng.normal(size=(F, F)))
        U, _ = np.linalg.qr(rng.normal(size=(P, F)) + 1j * rng.normal(size=(P, F)))
        st = amp * np.geomspace(4.0, 1.0, rank)
        sb = rng.uniform(0.3, 1.0, F - rank)
        T = (U[:, :rank] * st[None, :]) @ Q[:, :rank].conj().T
        B = (U[:, rank:] * sb[None, :]) @ Q[:, rank:].conj().T
        tissue[:, k] = T.T.reshape(F, nzs, N)
        blood[:, k] = B.T.reshape(F, nzs, N)
    return tissue, blood


def c_tensor(x):
    a = np.stack([x.real, x.imag], axis=-1).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(s, sl32, F, rank, iters=30):
    from paper_2511_21647_gb300 import rca
    t = c_tensor(sl32)
    rca.rca_clutter_svd(s.h, s.t, t, F, rank, iters)
    torch.cuda.synchronize()
    assert s.sync_status() == 0
    r = t.cpu().numpy()
    return r[..., 0] + 1j * r[..., 1]


def check(g_out, sl32, blood, rank, tol):
    ref = OS.filter_slices(sl32.astype(np.complex128), rank)
    e_all = np.linalg.norm(g_out - ref) / np.linalg.norm(sl32)
    e_blood = np.linalg.norm(g_out - ref) / np.linalg.norm(blood)
    e_truth = np.linalg.norm(ref - blood) / np.linalg.norm(blood)
    print(f"\nrank {rank}: error vs oracle {e_all:.2e} of the input, {e_blood:.2e} of the blood "
          f"(oracle vs the constructed blood {e_truth:.2e})")
    assert e_all < tol
    return e_all, e_blood


def test_filter_matches_oracle_tiny_geometry(tiny):
    from paper_2511_21647_gb300.pipeline import RcaSession
    g = tiny.geom
    F, nt = 64, 2 * len(g.ang_rc)
    rng = np.random.default_rng(4)
    tissue, blood = exact_svd_scene(rng, F, nt, g.nzs, g.n_el, rank=4, amp=100.0)
    sl32 = (tissue + blood).astype(np.complex64)
    with RcaSession(g) as s:
        out = run(s, sl32, F, 4)
        same = run(s, sl32, F, 0)
    assert np.array_equal(same, sl32)
    check(out, sl32, blood, 4, 1e-5)


def test_filter_matches_oracle_paper_geometry_300_frames(tiny):
    from paper_2511_21647_gb300.pipeline import RcaSession
    from synth import workload
    g = workload("paper").geom
    F, nt = 300, 2 * len(g.ang_rc)
    rng = np.random.default_rng(5)
    tissue, blood = exact_svd_scene(rng, F, nt, g.nzs, g.n_el, rank=16, amp=1000.0)
    sl32 = (tissue + blood).astype(np.complex64)
    del tissue
    with RcaSession(g) as s:
        out = run(s, sl32, F, 16)
    check(out, sl32, blood, 16, 1e-5)


def test_argument_errors(tiny):
    from paper_2511_21647_gb300 import _lib, rca
    from paper_2511_21647_gb300.pipeline import RcaSession
    g = tiny.geom
    F, nt = 8, 2 * len(g.ang_rc)
    with RcaSession(g) as s:
        t = torch.zeros((F, nt, g.nzs, g.n_el, 2), device="cuda")
        for rank, iters in ((33, 10), (8, 10), (-1, 10), (2, 0)):
            with pytest.raises(rca.RcaError) as e:
                rca.rca_clutter_svd(s.h, s.t, t, F, rank, iters)
            assert e.value.status == _lib.RCA_ERR_INVALID_ARG


@pytest.mark.parametrize("rank", [1])
def test_beamform_with_svd_clutter_filter_end_to_end(tiny, tiny_rf, rank):
    """channel data -> IQ without clutter removal -> Stage 1 -> SVD filter ->
    Stage 2 + projection, through the one-call beamformer, against the oracle
    chained the same way (its filter on its own FP64 slices).  The tiny
    ensemble's tissue is static: one eigenvalue, then the blood and noise at
    1e-6 of it, whose next ratios (0.82, 0.93) are within FP32's resolution of
    a covariance that size, so only the rank-1 subspace is determined in FP32."""
    import oracle as O
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300.pipeline import RcaSession, to_complex128
    g = tiny.geom
    rf = tiny_rf.rf.numpy()
    iq = O.demod(g, rf, remove_mean=False)
    sl = np.stack([O.stage1(g, iq[f]) for f in range(rf.shape[0])])
    flt = OS.filter_slices(sl, rank)
    ref = np.stack([O.stage2_project(g, flt[f]) for f in range(rf.shape[0])])
    with RcaSession(g) as s:
        pl = to_complex128(s.beamform(tiny_rf.rf.cuda(), clutter=L.RCA_CLUTTER_SVD, svd_rank=rank))
        assert s.sync_status() == 0
        with pytest.raises(Exception):
            s.beamform(tiny_rf.rf.cuda(), mode=L.RCA_MODE_DIRECT, clutter=L.RCA_CLUTTER_SVD, svd_rank=rank)
    e = np.linalg.norm(pl - ref) / np.linalg.norm(ref)
    print(f"\nSVD rank {rank} through the beamformer: planes rel-L2 {e:.2e}, top eigenvalue ratios "
          f"{OS.spectrum(sl, 0)[:rank + 2] / OS.spectrum(sl, 0)[0]}")
    assert e < 1e-4
