"""Eigen-based SVD clutter filter on the Stage-1 slices (Sec. II-A2) in
numpy FP64.

TEST INFRASTRUCTURE ONLY: only the test-suite and the benchmark's CPU legs
may load this module; it shares nothing with the CUDA library.

For each transmission k the frames' slices form the Casorati matrix X_k
(pixels x frames, one column per frame).  The filter computes the frame
covariance C_k = X_k^H X_k, its eigendecomposition, and removes the
subspace of the n_c largest eigenvalues (the tissue):
    X_k,filtered = X_k - X_k V V^H,   V = the n_c leading eigenvectors.
The paper gives no rank or threshold; n_c is a parameter.  The library
matrix product and Hermitian eigensolver are the only library steps."""
import numpy as np


def casorati(slices: np.ndarray, k: int) -> np.ndarray:
    """slices [F][2K][nzs][N] -> X_k [nzs N][F]"""
    F = slices.shape[0]
    return slices[:, k].reshape(F, -1).T


def covariance(slices: np.ndarray, k: int) -> np.ndarray:
    X = casorati(slices, k)
    return X.conj().T @ X


def tissue_basis(C: np.ndarray, n_c: int) -> np.ndarray:
    """the n_c eigenvectors of the largest eigenvalues, [F][n_c]"""
    w, V = np.linalg.eigh(C)
    order = np.argsort(w)[::-1]
    return V[:, order[:n_c]]


def filter_slices(slices: np.ndarray, n_c: int) -> np.ndarray:
    """slices [F][2K][nzs][N] complex -> filtered slices, same shape"""
    slices = np.asarray(slices, dtype=np.complex128)
    F, nt = slices.shape[:2]
    out = np.empty_like(slices)
    for k in range(nt):
        X = casorati(slices, k)
        V = tissue_basis(X.conj().T @ X, n_c)
        Xf = X - (X @ V) @ V.conj().T
        out[:, k] = Xf.T.reshape(slices.shape[0], *slices.shape[2:])
    return out


def spectrum(slices: np.ndarray, k: int) -> np.ndarray:
    """eigenvalues of C_k, largest first"""
    return np.sort(np.linalg.eigvalsh(covariance(slices, k)))[::-1]
