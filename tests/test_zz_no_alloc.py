"""ulm_pair3d_noalloc (pairing on the library's fixed per-device scratch,
no allocation) against ulm_pair3d, both called through the C ABI on the
same 2D lists.  The two share their kernels, so the 3D lists must agree
byte for byte, as the pairing parity tests require of ulm_pair3d against
the oracle.  Two no-alloc calls run in a row on different lists (the
second shorter and over fewer planes, so stale scratch from the first
would show), and the oracle's pairing of the same lists is checked too.

Named so that pytest collects it last: it must pass both on its own in a
fresh process and after every other test."""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lists(tiny, tiny_rf):
    """tiny ensemble -> 2D lists (beamforming, enhancement and detection on the GPU)"""
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import RcaSession
    psf = json.load(open(os.path.join(HERE, "golden", "psf_sigma.json")))["tiny"]
    prm = rca.make_ulm_params(d=5, sig_z=psf["sig_z"], sig_lat=psf["sig_lat"], alpha=0.1, ncc_min=0.5)
    s = RcaSession(tiny.geom)
    planes = s.beamform(tiny_rf.rf.cuda().contiguous())
    A, M = s.enhance(planes)
    out2d, n2d, _ = s.detect2d(A, M, prm)
    torch.cuda.synchronize()
    yield s, out2d, n2d, tiny.n_frames
    s.close()


def _pair(fn, s, L2, n2d, cap2d, F, cap3d=1 << 14):
    out = torch.full((cap3d, 10), -7, dtype=torch.int32, device="cuda")
    n3d = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    fn(s.h, s.t, L2, n2d, cap2d, F, out, cap3d, n3d)
    torch.cuda.synchronize()
    n = int(n3d.item())
    assert 0 <= n <= cap3d
    return out[:n].cpu().numpy().copy(), n


def _oracle_pairs(L2, n, P):
    from paper_2511_21647_gb300.pipeline import list2d_numpy
    g = list2d_numpy(L2, n)
    L_o = np.zeros(n, dtype=O.LOC2D)
    for name in O.LOC2D.names:
        L_o[name] = g[name]
    return [(int(r["i_xz"]), int(r["i_yz"])) for r in O.pair3d(L_o, P)]


def test_noalloc_pairing_matches_ulm_pair3d_twice_in_a_row(lists, tiny):
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import list2d_numpy, list3d_numpy
    s, out2d, n2d, F = lists
    n_all = int(n2d.item())
    cap2d = out2d.shape[0]
    assert 0 < n_all <= cap2d
    frames = list2d_numpy(out2d, n_all)["frame"]
    # second input: the entries of the first F2 frames (the list is frame-major)
    F2 = F // 3
    n_part = int(np.sum(frames < F2))
    assert 0 < n_part < n_all
    n2d_part = torch.tensor([n_part], dtype=torch.int32, device="cuda")

    cases = [(n2d, cap2d, F, n_all), (n2d_part, n_part, F2, n_part)]
    for q, (cnt, cap, nf, n) in enumerate(cases):
        ref, n_ref = _pair(rca.ulm_pair3d, s, out2d, cnt, cap, nf)
        got, n_got = _pair(rca.ulm_pair3d_noalloc, s, out2d, cnt, cap, nf)
        assert s.sync_status() == 0
        assert n_got == n_ref and n_ref > 5, (q, n_got, n_ref)
        assert np.array_equal(got, ref), q
        P3 = list3d_numpy(torch.from_numpy(got), n_got)
        assert [(int(r["i_xz"]), int(r["i_yz"])) for r in P3] == _oracle_pairs(out2d, n, tiny.geom.P), q
        assert np.all(P3["frame"] < nf)


def test_noalloc_rejects_sizes_beyond_its_scratch(lists):
    from paper_2511_21647_gb300 import _lib, rca
    s, out2d, n2d, F = lists
    out = torch.zeros((4, 10), dtype=torch.int32, device="cuda")
    n3d = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(rca.RcaError) as e:
        rca.ulm_pair3d_noalloc(s.h, s.t, out2d, n2d, _lib.ULM_PAIR3D_NOALLOC_MAX_2D + 1, F, out, 4, n3d)
    assert e.value.status == _lib.RCA_ERR_UNSUPPORTED and "cap2d" in str(e.value)
    too_many_frames = _lib.ULM_PAIR3D_NOALLOC_MAX_PLANES // (2 * s.S) + 1
    with pytest.raises(rca.RcaError) as e:
        rca.ulm_pair3d_noalloc(s.h, s.t, out2d, n2d, out2d.shape[0], too_many_frames, out, 4, n3d)
    assert e.value.status == _lib.RCA_ERR_UNSUPPORTED and "planes" in str(e.value)
    torch.cuda.synchronize()
    assert int(n3d.item()) == -7          # rejected before anything was enqueued
    assert s.sync_status() == 0


def test_zero_capacity_after_a_full_call_gives_no_pairs(lists):
    """cap2d = 0 with a non-zero count: no list entry may be read, so both
    entry points report zero pairs, even right after a call that left a
    matched first entry in the scratch."""
    from paper_2511_21647_gb300 import rca
    s, out2d, n2d, F = lists
    cap2d = out2d.shape[0]
    for fn in (rca.ulm_pair3d, rca.ulm_pair3d_noalloc):
        _, n_full = _pair(fn, s, out2d, n2d, cap2d, F)
        assert n_full > 0
        _, n_zero = _pair(fn, s, out2d, n2d, 0, F)
        assert n_zero == 0, fn.__name__
        assert s.sync_status() == 0
