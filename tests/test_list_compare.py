"""The list comparison the GPU parity tests use (tests/ulm_lists.py), pinned
on the CPU: the oracle's own lists compare equal to themselves, and a planted
mistake in a copy (a dropped detection, a moved position, a changed pair)
fails it."""
import json
import os

import numpy as np
import pytest

import oracle as O
import ulm_lists as UL

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lists(tiny, tiny_rf):
    psf = json.load(open(os.path.join(HERE, "golden", "psf_sigma.json")))["tiny"]
    prm = dict(d=5, sig_z=psf["sig_z"], sig_lat=psf["sig_lat"], alpha=0.1, ncc_min=0.5)
    planes = O.beamform_projections(tiny.geom, tiny_rf.rf.numpy(), frames=range(8))
    A, M, L2, L3 = O.localize(planes, prm["d"], prm["sig_z"], prm["sig_lat"], prm["alpha"], prm["ncc_min"],
                              tiny.geom.P)
    amb = UL.near_ties(A, M, prm, eps_ncc=3e-5, eps_amp=1e-5)
    return L2, L3, amb, tiny.geom.P


def run(L2, L3, L2g, L3g, amb, P):
    return UL.compare(L2, L3, L2g, L3g, amb, P, pos_tol=1e-3, ncc_tol=5e-5, amp_rtol=1e-5, tz=2e-3, tr=2e-5)


def test_identical_lists_compare_equal(lists):
    L2, L3, amb, P = lists
    st = run(L2, L3, L2.copy(), L3.copy(), amb, P)
    assert st["diff2d"] == 0 and st["n3d"] > 0 and st["pairs_compared"] > 0


def test_dropped_detection_fails(lists):
    L2, L3, amb, P = lists
    keys = [UL.key2(r) for r in L2]
    q = next(i for i, k in enumerate(keys) if k not in amb)
    L2g = np.delete(L2, q)
    L3g = L3.copy()
    L3g = L3g[(L3g["i_xz"] != q) & (L3g["i_yz"] != q)]
    L3g["i_xz"] -= (L3g["i_xz"] > q)
    L3g["i_yz"] -= (L3g["i_yz"] > q)
    with pytest.raises(AssertionError):
        run(L2, L3, L2g, L3g, amb, P)


def test_moved_position_fails(lists):
    L2, L3, amb, P = lists
    L2g = L2.copy()
    L2g["z"][0] += 0.01
    with pytest.raises(AssertionError):
        run(L2, L3, L2g, L3.copy(), amb, P)


def test_changed_pair_fails(lists):
    L2, L3, amb, P = lists
    L3g = L3.copy()
    # re-pair the first 3D entry with another YZ entry of the same frame, or drop it
    r = L3g[0]
    ys = [q for q in range(len(L2)) if L2[q]["axis"] == 1 and L2[q]["frame"] == r["frame"] and q != r["i_yz"]]
    if ys:
        L3g["i_yz"][0] = ys[0]
    else:
        L3g = L3g[1:]
    with pytest.raises(AssertionError):
        run(L2, L3, L2.copy(), L3g, amb, P)
