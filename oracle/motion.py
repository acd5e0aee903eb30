"""Projection-based rigid motion estimation (Sec. II-A3, Fig. 1d) in numpy FP64.

TEST INFRASTRUCTURE ONLY: only the test-suite and the benchmark's CPU legs
may load this module; it shares nothing with the CUDA library.

Each frame's Stage-1 slices are compared with those of the reference frame
(frame 0) by Fourier-domain cross-correlation: the slices are zero-padded to
Zp x Xp (Zp the next power of two >= the slice rows, Xp = N, a power of two),
R = IFFT2(FFT2(S_f) conj(FFT2(S_0))) is the circular cross-correlation
R[dz, dx] = sum_p S_f[p + (dz, dx)] conj(S_0[p]), and the displacement is the
peak of |R| (first in row-major order on ties), refined per axis by a
3-point parabola through |R| at the peak and its two circular neighbours
(clamped to +-1/2, none when not concave).  Indices at or beyond half the
padded size are negative shifts.  The normalised peak |R| / (||S_f|| ||S_0||)
is the NCC.  RC slices (transmissions 0 .. K-1) resolve (x, z), CR slices
(K .. 2K-1) resolve (y, z); each family's shifts are averaged over its K
transmissions and the two are combined into one 3D displacement per frame:
(x_RC, y_CR, (z_RC + z_CR) / 2), in metres (lateral pixel = pitch, slice row =
dz / us).  The library FFT is the only library step."""
import numpy as np


def padded_shape(nzs: int, n: int):
    zp = 1
    while zp < nzs:
        zp *= 2
    assert n & (n - 1) == 0, "the lateral size must be a power of two"
    return zp, n


def _parabola(m_minus, m0, m_plus):
    den = m_minus - 2.0 * m0 + m_plus
    if den >= 0.0:
        return 0.0
    return float(min(0.5, max(-0.5, (m_minus - m_plus) / (2.0 * den))))


def correlate(s_f: np.ndarray, s_0: np.ndarray):
    """one slice pair [nzs][N] complex -> (dz, dx) integer peak, (sub_z, sub_x) refined shifts, ncc, |R|"""
    nzs, n = s_f.shape
    zp, xp = padded_shape(nzs, n)
    a = np.zeros((zp, xp), dtype=np.complex128)
    b = np.zeros((zp, xp), dtype=np.complex128)
    a[:nzs] = s_f
    b[:nzs] = s_0
    R = np.fft.ifft2(np.fft.fft2(a) * np.conj(np.fft.fft2(b)))
    mag = np.abs(R)
    k = int(np.argmax(mag))
    iz, ix = divmod(k, xp)
    dz = iz if iz < zp // 2 else iz - zp
    dx = ix if ix < xp // 2 else ix - xp
    sz = dz + _parabola(mag[(iz - 1) % zp, ix], mag[iz, ix], mag[(iz + 1) % zp, ix])
    sx = dx + _parabola(mag[iz, (ix - 1) % xp], mag[iz, ix], mag[iz, (ix + 1) % xp])
    den = np.sqrt(np.sum(np.abs(s_f) ** 2)) * np.sqrt(np.sum(np.abs(s_0) ** 2))
    ncc = float(mag[iz, ix] / den) if den > 0 else 0.0
    return (dz, dx), (sz, sx), ncc, mag


def estimate(g, slices: np.ndarray, frames=None):
    """slices [F][2K][nzs][N] complex -> (shifts [F'][2K][3] = (z, x, ncc) in slice pixels,
    peaks [F'][2K][2] integer, motion [F'][3] metres) for the listed frames (all by default)"""
    F, nt = slices.shape[:2]
    K = nt // 2
    frames = range(F) if frames is None else list(frames)
    shifts = np.zeros((len(frames), nt, 3))
    peaks = np.zeros((len(frames), nt, 2), dtype=np.int64)
    motion = np.zeros((len(frames), 3))
    for q, f in enumerate(frames):
        for k in range(nt):
            pk, (sz, sx), ncc, _ = correlate(slices[f, k], slices[0, k])
            shifts[q, k] = (sz, sx, ncc)
            peaks[q, k] = pk
        z_rc, x_rc = shifts[q, :K, 0].mean(), shifts[q, :K, 1].mean()
        z_cr, y_cr = shifts[q, K:, 0].mean(), shifts[q, K:, 1].mean()
        motion[q] = (x_rc * g.pitch, y_cr * g.pitch, 0.5 * (z_rc + z_cr) * g.dz / g.us)
    return shifts, peaks, motion
