"""Pins of the oracle's eigen-based SVD clutter filter (Sec. II-A2): a tissue
component of rank n_c whose temporal subspace is orthogonal to the blood's
is removed exactly and the blood kept; the filter equals subtracting the
n_c leading terms of numpy's singular value decomposition; n_c = 0 is the
identity; the filtered data are orthogonal to the removed subspace."""
import numpy as np

from oracle import svd_filter as OS


def _scene(rng, F=40, nt=2, nzs=12, N=8, rank=3, amp=1e3):
    """X_k = [U_t U_b] diag(S_t, S_b) [Q_t Q_b]^H with orthonormal spatial and
    temporal bases and every tissue singular value above every blood one: an
    exact SVD, so the n_c = rank leading temporal vectors are Q_t"""
    P = nzs * N
    tissue = np.zeros((nt, P, F), dtype=np.complex128)
    blood = np.zeros((nt, P, F), dtype=np.complex128)
    for k in range(nt):
        Q, _ = np.linalg.qr(rng.normal(size=(F, F)) + 1j * rng.normal(size=(F, F)))
        U, _ = np.linalg.qr(rng.normal(size=(P, F)) + 1j * rng.normal(size=(P, F)))
        st = amp * np.linspace(3, 1, rank)
        sb = rng.uniform(0.5, 2.0, F - rank)
        tissue[k] = (U[:, :rank] * st[None, :]) @ Q[:, :rank].conj().T
        blood[k] = (U[:, rank:] * sb[None, :]) @ Q[:, rank:].conj().T
    def to_slices(X):
        return np.stack([X[k].T.reshape(F, nzs, N) for k in range(nt)], axis=1)
    return to_slices(tissue), to_slices(blood)


def test_low_rank_tissue_removed_and_blood_kept():
    rng = np.random.default_rng(1)
    tissue, blood = _scene(rng)
    out = OS.filter_slices(tissue + blood, 3)
    assert np.linalg.norm(out - blood) < 1e-9 * np.linalg.norm(tissue)


def test_filter_equals_truncated_svd_and_identity_at_rank_zero():
    rng = np.random.default_rng(2)
    tissue, blood = _scene(rng, rank=4)
    sl = tissue + 3.0 * blood
    for n_c in (0, 2, 4, 7):
        out = OS.filter_slices(sl, n_c)
        for k in range(sl.shape[1]):
            X = OS.casorati(sl, k)
            U, s, Vh = np.linalg.svd(X, full_matrices=False)
            ref = X - (U[:, :n_c] * s[:n_c]) @ Vh[:n_c]
            got = OS.casorati(out, k)
            assert np.linalg.norm(got - ref) < 1e-9 * np.linalg.norm(X), (n_c, k)
            if n_c == 0:
                assert np.array_equal(got, X)
            else:
                # orthogonal to the removed temporal subspace
                assert np.linalg.norm(got @ Vh[:n_c].conj().T) < 1e-9 * np.linalg.norm(X)


def test_covariance_is_the_frame_gram_matrix():
    rng = np.random.default_rng(3)
    sl = rng.normal(size=(6, 2, 5, 4)) + 1j * rng.normal(size=(6, 2, 5, 4))
    C = OS.covariance(sl, 1)
    for a in range(6):
        for b in range(6):
            assert abs(C[a, b] - np.vdot(sl[a, 1], sl[b, 1])) < 1e-12
