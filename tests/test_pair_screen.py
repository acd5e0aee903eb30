"""The pairing test's FP32 screens (Sec. II-A4 pairing: |z_xz - z_yz| <= 1 px and
intensity ratio in [0.9, 1.11]) give the FP64 decision on FP32 inputs: the same
screen written here with numpy's IEEE float32 arithmetic, against FP64, on
random values and on values packed around every bound (one ulp either side)."""
import numpy as np


def fp64_ok(z1, z2, a1, a2):
    if abs(np.float64(z1) - np.float64(z2)) > 1.0:
        return False
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.float64(a1) / np.float64(a2)
    return bool(r >= 0.9 and r <= 1.11)


def screened_ok(z1, z2, a1, a2):
    dz = np.float32(abs(np.float32(z1) - np.float32(z2)))
    if dz > np.float32(1.0):
        return False
    if dz == np.float32(1.0) and abs(np.float64(z1) - np.float64(z2)) > 1.0:
        return False
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        r32 = np.float32(a1) / np.float32(a2)
    if r32 <= np.float32(0.89) or r32 >= np.float32(1.12) or r32 != r32:
        return False
    if not (r32 >= np.float32(0.91) and r32 <= np.float32(1.10)):
        r = np.float64(a1) / np.float64(a2)
        if not (r >= 0.9 and r <= 1.11):
            return False
    return True


def near(v, n=3):
    v = np.float32(v)
    out = [v]
    lo = hi = v
    for _ in range(n):
        lo = np.nextafter(lo, np.float32(-np.inf))
        hi = np.nextafter(hi, np.float32(np.inf))
        out += [lo, hi]
    return out


def test_screen_equals_fp64_random_and_at_bounds():
    rng = np.random.default_rng(0)
    cases = []
    for _ in range(20000):
        z1 = np.float32(rng.uniform(0, 250))
        z2 = np.float32(z1 + rng.uniform(-1.5, 1.5))
        a1 = np.float32(rng.lognormal(0, 1))
        a2 = np.float32(a1 * rng.uniform(0.85, 1.15))
        cases.append((z1, z2, a1, a2))
    # axial difference at exactly one pixel and one ulp around it, at several depths
    for z in (0.25, 1.0, 3.5, 77.75, 249.0):
        for z2 in near(np.float32(z) + np.float32(1.0)):
            cases.append((np.float32(z), z2, np.float32(1), np.float32(1)))
    # ratios at the bounds: a1 chosen so that a1 / a2 lands on 0.9 and 1.11 and next to them
    for a2 in (np.float32(0.37), np.float32(1.0), np.float32(3.3e3)):
        for b in (0.9, 1.11, 0.89, 0.91, 1.10, 1.12):
            for a1 in near(np.float32(b * float(a2)), 4):
                cases.append((np.float32(10), np.float32(10.5), a1, a2))
    # degenerate amplitudes
    for a1, a2 in ((0, 0), (1, 0), (0, 1), (np.inf, 1), (np.nan, 1)):
        cases.append((np.float32(5), np.float32(5), np.float32(a1), np.float32(a2)))
    bad = [c for c in cases if screened_ok(*c) != fp64_ok(*c)]
    assert not bad, bad[:5]
