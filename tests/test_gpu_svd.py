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


# --- the benchmark's setting: the paper ensemble's own slices, rank 16 ---------------

@pytest.fixture(scope="module")
def paper_slices():
    """The paper-scale ensemble (300 frames, moving tissue 40 dB above the
    microbubbles) as the generator makes it for the benchmark; the oracle's
    Stage-1 slices without clutter removal of one RC and one CR transmission
    (k = 0 and 4, the -3 deg transmissions), rounded to complex64 -- the
    input of both filters -- and the oracle's eigendecomposition of each
    transmission's frame covariance."""
    import dataclasses
    import oracle as O
    from synth import generate, workload
    w = workload("paper")
    g = w.geom
    g1 = dataclasses.replace(g, ang_rc=(g.ang_rc[0],), ang_cr=(g.ang_cr[0],))
    rf = generate(w, device="cuda", dtype=torch.float32, frame_batch=32).rf
    rf2 = rf[:, [0, len(g.ang_rc)]].contiguous().cpu().numpy()
    del rf
    F = rf2.shape[0]
    sl = np.zeros((F, 2, g1.nzs, g1.n_el), dtype=np.complex64)
    for f0 in range(0, F, 30):
        fr = list(range(f0, min(F, f0 + 30)))
        iq = O.demod(g1, rf2, remove_mean=False, frames=fr)
        for q, f in enumerate(fr):
            sl[f] = O.stage1(g1, iq[q]).astype(np.complex64)
    eig = []
    for k in range(2):
        X = OS.casorati(sl.astype(np.complex128), k)
        lam, V = np.linalg.eigh(X.conj().T @ X)
        o = np.argsort(lam)[::-1]
        eig.append((lam[o], V[:, o]))
    return g1, sl, eig


def _removed_basis(X, Xf, r):
    """orthonormal frame-space basis of the subspace a filter removed:
    the r leading right singular vectors of X - Xf"""
    _, _, Vh = np.linalg.svd(X - Xf, full_matrices=False)
    return Vh[:r].conj().T


def _angles_deg(A, B):
    """principal angles (degrees) between span(A) and span(B), A and B orthonormal"""
    c = np.linalg.svd(A.conj().T @ B, compute_uv=False)
    return np.degrees(np.arccos(np.clip(c, 0.0, 1.0)))


def _run_info(g1, sl, rank, iters):
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import RcaSession
    F = sl.shape[0]
    with RcaSession(g1) as s:
        t = c_tensor(sl)
        info = torch.zeros((2, 4), dtype=torch.float32, device="cuda")
        rca.rca_clutter_svd_info(s.h, s.t, t, F, rank, iters, info)
        torch.cuda.synchronize()
        assert s.sync_status() == 0
        r = t.cpu().numpy()
    return r[..., 0] + 1j * r[..., 1], info.cpu().numpy()


def test_paper_ensemble_rank16_30_iterations(paper_slices):
    """Rank 16, 30 iterations, as the benchmark runs the filter.  On this
    ensemble the tissue's eigenvalues fall smoothly from lambda_1 through the
    rank: lambda_16 - lambda_17 is about 2e-7 lambda_1, the size of the FP32
    covariance's own rounding, so FP32 arithmetic does not determine which
    vectors near the split are removed (any FP32 implementation, the paper's
    batched FP32 eigensolver included).  What is unique is checked exactly
    and the rest for validity:
      - the leading subspace the FP32 covariance resolves (every split m <= 16
        with (lambda_m - lambda_{m+1}) / lambda_1 >= 1e-4) lies inside the
        removed subspace: principal angles below 0.5 deg;
      - the removed energy ||X Q||^2 lies between the energy of the exact top
        16 minus the eigenvalues the split leaves undetermined and that of the
        exact top 16, to 1e-5 of lambda_1;
      - the report (rca_clutter_svd_info) shows it: the largest Rayleigh
        quotient equals lambda_1 to 1e-4, the smallest lies in the band of
        eigenvalues the split leaves undetermined, and the invariance residual
        is far above that of a resolved split.
    The principal angles at the split and the filtered outputs' difference are
    printed."""
    g1, sl, eig = paper_slices
    rank = 16
    out, info = _run_info(g1, sl, rank, 30)
    for k in range(2):
        lam, V = eig[k]
        X = OS.casorati(sl.astype(np.complex128), k)
        Xf = OS.casorati(out, k)
        ref = X - (X @ V[:, :rank]) @ V[:, :rank].conj().T
        Q = _removed_basis(X, Xf, rank)
        gaps = (lam[:rank] - lam[1:rank + 1]) / lam[0]
        m = max(j + 1 for j in range(rank) if gaps[j] >= 1e-4)
        ang_m = _angles_deg(V[:, :m], Q).max()
        ang_all = _angles_deg(V[:, :rank], Q).max()
        removed = float(np.linalg.norm(X @ Q) ** 2)
        undetermined = lam[np.abs(lam - lam[rank - 1]) <= 20 * (lam[rank - 1] - lam[rank])]
        lo = lam[:rank].sum() - undetermined.sum()
        e_f = np.linalg.norm(Xf - ref) / np.linalg.norm(ref)
        e_in = np.linalg.norm(Xf - ref) / np.linalg.norm(X)
        print(f"\ntx {k}: lambda_16/17 gap {gaps[rank - 1]:.2e} of lambda_1; resolved leading rank {m} "
              f"(angle {ang_m:.3g} deg), angle at rank {rank} {ang_all:.3g} deg; filtered difference "
              f"{e_f:.3g} of the filtered norm, {e_in:.3g} of the input; removed energy "
              f"{removed / lam[0]:.8f} vs exact {lam[:rank].sum() / lam[0]:.8f} (lambda_1); info "
              f"{info[k] / np.array([lam[0], lam[0], lam[0], 1.0])} (eigenvalues over lambda_1)")
        assert m >= 8
        assert ang_m < 0.5, ang_m
        assert lo - 1e-5 * lam[0] <= removed <= lam[:rank].sum() + 1e-5 * lam[0]
        assert abs(info[k, 0] - lam[0]) <= 1e-4 * lam[0]
        assert undetermined.min() - 1e-5 * lam[0] <= info[k, 1] <= undetermined.max() + 1e-5 * lam[0]
        assert info[k, 3] > 1e-2


def test_paper_ensemble_resolved_rank(paper_slices):
    """The same ensemble and call at the largest rank m <= 16 whose split the
    covariance resolves ((lambda_m - lambda_{m+1}) / lambda_1 >= 1e-4; m = 9
    here).  The tensor-core covariance (TF32 hi / lo products, FP32 TMEM
    accumulation over 1024-pixel splits) is accurate to about 1e-6 lambda_1
    (its largest Rayleigh quotient sits 1.3e-5 below lambda_1), so the m-th
    eigenvector's angle is bounded by 2e-6 lambda_1 / (lambda_m -
    lambda_{m+1}) radians; the filtered output is then within 2e-4 of the
    input's norm (2e-2 of the filtered output's) of the oracle's, and the
    report says the split is resolved: invariance residual below 1e-2 of
    lambda_m, quotients equal to lambda_1, lambda_m and lambda_{m+1} to 1e-4
    of lambda_1."""
    g1, sl, eig = paper_slices
    lam0 = eig[0][0]
    gaps = (lam0[:16] - lam0[1:17]) / lam0[0]
    rank = max(j + 1 for j in range(16) if gaps[j] >= 1e-4)
    out, info = _run_info(g1, sl, rank, 30)
    for k in range(2):
        lam, V = eig[k]
        X = OS.casorati(sl.astype(np.complex128), k)
        Xf = OS.casorati(out, k)
        ref = X - (X @ V[:, :rank]) @ V[:, :rank].conj().T
        ang = _angles_deg(V[:, :rank], _removed_basis(X, Xf, rank)).max()
        e_f = np.linalg.norm(Xf - ref) / np.linalg.norm(ref)
        e_in = np.linalg.norm(Xf - ref) / np.linalg.norm(X)
        print(f"\ntx {k}, rank {rank} (gap {(lam[rank - 1] - lam[rank]) / lam[0]:.2e} of lambda_1): angle "
              f"{ang:.3g} deg, filtered difference {e_f:.3g} of the filtered norm, {e_in:.3g} of the input, "
              f"info {info[k] / np.array([lam[0], lam[0], lam[0], 1.0])}")
        bound = np.degrees(2e-6 * lam[0] / (lam[rank - 1] - lam[rank]))
        assert ang < bound, (ang, bound)
        assert e_f < 2e-2 and e_in < 2e-4, (e_f, e_in)
        assert abs(info[k, 0] - lam[0]) <= 1e-4 * lam[0]
        assert abs(info[k, 1] - lam[rank - 1]) <= 1e-4 * lam[0]
        assert abs(info[k, 2] - lam[rank]) <= 1e-4 * lam[0]
        assert info[k, 3] < 1e-2
