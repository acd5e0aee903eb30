"""Microbubble separation on the projection planes (Sec. II-A5) in numpy FP64.

TEST INFRASTRUCTURE ONLY: only the test-suite and the benchmark's CPU legs
may load this module; it shares nothing with the CUDA library.

Each plane pixel's slow-time signal x[t], t = 0..F-1, is Fourier transformed
over the F frames, multiplied by one rectangular band-pass mask per subset and
transformed back (Sec. II-A5: temporal FFT per pixel, band-pass filters for
speed ranges, inverse FFT; subsets of upward and downward flow).  The paper
prints no band edges, so they are parameters:

  bin j of the F-point DFT has the signed index k = j (2 j < F) or j - F
  (2 j > F) and the Doppler frequency k * prf / F;
  DC (k = 0) and, for even F, the Nyquist bin (2 j = F) carry no direction and
  belong to no subset;
  speed band b (b = 0 .. nb-1) holds the bins with
      edges[b] < |k| * prf / F <= edges[b + 1];
  direction: k > 0 is flow toward the array (decreasing depth, "up") -- the
  planes carry the phase 2 pi fc (tau_pixel - tau_echo), which grows as the
  echo delay shrinks; k < 0 is "down";
  subset index = direction * nb + b (up bands first, then down bands).

The library FFT (numpy.fft.fft / ifft) is the only library step."""
import numpy as np

UP, DOWN = 0, 1


def default_edges(prf: float, n_bands: int) -> np.ndarray:
    """n_bands equal-width speed bands over (0, prf / 2]"""
    return np.array([i * prf / (2.0 * n_bands) for i in range(n_bands + 1)], dtype=np.float64)


def bin_subsets(F: int, prf: float, edges) -> np.ndarray:
    """subset index of each DFT bin j (int, -1 where the bin is in no subset)"""
    edges = np.asarray(edges, dtype=np.float64)
    nb = len(edges) - 1
    out = np.full(F, -1, dtype=np.int64)
    for j in range(F):
        if 2 * j == F or j == 0:
            continue
        k = j if 2 * j < F else j - F
        f = abs(k) * prf / F
        for b in range(nb):
            if edges[b] < f <= edges[b + 1]:
                out[j] = (UP if k > 0 else DOWN) * nb + b
                break
    return out


def separate(planes: np.ndarray, prf: float, edges) -> np.ndarray:
    """planes [F][...] complex -> subsets [2 nb][F][...] complex128"""
    planes = np.asarray(planes, dtype=np.complex128)
    F = planes.shape[0]
    nb = len(edges) - 1
    sub = bin_subsets(F, prf, edges)
    X = np.fft.fft(planes, axis=0)
    out = np.zeros((2 * nb,) + planes.shape, dtype=np.complex128)
    for s in range(2 * nb):
        mask = (sub == s).astype(np.float64).reshape((F,) + (1,) * (planes.ndim - 1))
        out[s] = np.fft.ifft(X * mask, axis=0)
    return out


def separate_xdoppler(planes: np.ndarray, prf: float, edges, xdoppler):
    """Each subset's XDoppler amplitude and frame maxima, as the localisation
    of a separated subset consumes them: (A [2 nb][F][2][S][nz][N],
    M [2 nb][F]).  `xdoppler` is the oracle's enhancement (planes -> (A, M))."""
    subs = separate(planes, prf, edges)
    A, M = zip(*(xdoppler(subs[s]) for s in range(subs.shape[0])))
    return np.stack(A), np.stack(M)
