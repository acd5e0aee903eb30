"""Reduced-precision form: int16 channel data with a per-channel scale,
FP16 / BF16 IQ and interpolation, FP16 / BF16 planes, FP32 accumulation,
FP64-computed tables stored as FP32 / Q16.

Parity (relative L2 <= 2e-3 for the reduced path) is against the FP64 oracle
run on the same dequantised int16 input; the error against the oracle on the
original FP32 channel data (which adds the int16 quantisation itself) is
reported, per projection and pooled."""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

TOL_REDUCED = 2e-3
HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def quant(tiny_rf):
    from synth import quantize_int16
    q, scale = quantize_int16(tiny_rf.rf)
    deq = (q.double() * scale.double()[None, :, :, None]).float()
    return q, scale, deq


@pytest.fixture(scope="module")
def oracle_refs(tiny, tiny_rf, quant):
    g = tiny.geom
    ref_fp32 = O.beamform_projections(g, tiny_rf.rf.numpy())
    ref_deq = O.beamform_projections(g, quant[2].numpy())
    return ref_fp32, ref_deq


@pytest.fixture(scope="module")
def S(tiny):
    from paper_2511_21647_gb300.pipeline import RcaSession
    s = RcaSession(tiny.geom)
    yield s
    s.close()


def run(S, q, scale, iq_t, pl_t):
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300.pipeline import to_complex128
    pl = S.beamform(q.cuda(), rf_dtype=L.RCA_I16, scale=scale.cuda(), iq_dtype=iq_t, planes_dtype=pl_t)
    assert S.sync_status() == 0
    return to_complex128(pl)


def per_plane(a, b):
    n = np.linalg.norm(b.reshape(-1, b.shape[-2] * b.shape[-1]), axis=1)
    e = np.linalg.norm((a - b).reshape(n.size, -1), axis=1)
    big = n > 1e-3 * n.max()
    return e[big] / n[big]


def test_int16_input_fp32_path_matches_dequantised_oracle(S, quant, oracle_refs):
    from paper_2511_21647_gb300 import _lib as L
    q, scale, _ = quant
    got = run(S, q, scale, L.RCA_C32, L.RCA_C32)
    assert rel(got, oracle_refs[1]) < 1e-4


@pytest.mark.parametrize("iq_name,pl_name,tol", [
    ("C16F", "C16F", TOL_REDUCED),
    ("C16F", "C16BF", TOL_REDUCED),
    ("C16BF", "C16BF", 4e-3),
])
def test_reduced_precision_planes(S, quant, oracle_refs, iq_name, pl_name, tol, record_property):
    from paper_2511_21647_gb300 import _lib as L
    q, scale, _ = quant
    iq_t, pl_t = getattr(L, "RCA_" + iq_name), getattr(L, "RCA_" + pl_name)
    got = run(S, q, scale, iq_t, pl_t)
    e_deq = rel(got, oracle_refs[1])
    e_fp32 = rel(got, oracle_refs[0])
    pp = per_plane(got, oracle_refs[1])
    record_property("rel_l2_vs_dequantised", e_deq)
    record_property("rel_l2_vs_fp32_rf", e_fp32)
    record_property("per_plane_max", float(pp.max()))
    print(f"\n{iq_name} IQ / {pl_name} planes: rel-L2 {e_deq:.2e} vs dequantised-int16 oracle, "
          f"{e_fp32:.2e} vs FP32-RF oracle, per-plane max {pp.max():.2e}")
    assert e_deq < tol
    assert pp.max() < 2.5 * tol


def test_fp16_channel_data_input(S, tiny, tiny_rf):
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300.pipeline import to_complex128
    rf16 = tiny_rf.rf.half()
    ref = O.beamform_projections(tiny.geom, rf16.float().numpy())
    got = to_complex128(S.beamform(rf16.cuda(), rf_dtype=L.RCA_F16))
    assert rel(got, ref) < 1e-4


def test_reduced_precision_localisation_error(S, tiny, tiny_rf, quant, oracle_refs):
    """MB positions from reduced-precision planes vs the FP64 oracle's
    localisation on the FP32 planes: the paired 3D detections are matched by
    nearest neighbour within 1 pixel and their RMS offset is reported."""
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import list3d_numpy
    psf = json.load(open(os.path.join(HERE, "golden", "psf_sigma.json")))["tiny"]
    prm = dict(d=5, sig_z=psf["sig_z"], sig_lat=psf["sig_lat"], alpha=0.1, ncc_min=0.5)
    _, _, _, L3_o = O.localize(oracle_refs[0], prm["d"], prm["sig_z"], prm["sig_lat"], prm["alpha"],
                               prm["ncc_min"], tiny.geom.P)
    q, scale, _ = quant
    pl = S.beamform(q.cuda(), rf_dtype=L.RCA_I16, scale=scale.cuda(), iq_dtype=L.RCA_C16F,
                    planes_dtype=L.RCA_C16BF)
    out2d, n2d, out3d, n3d = S.localize(pl, rca.make_ulm_params(**prm), planes_dtype=L.RCA_C16BF)
    L3 = list3d_numpy(out3d, int(n3d.item()))
    assert len(L3) > 0.8 * len(L3_o)
    d2 = []
    for r in L3:
        same = L3_o[L3_o["frame"] == r["frame"]]
        if len(same) == 0:
            continue
        dd = np.sqrt((same["x"] - r["x"]) ** 2 + (same["y"] - r["y"]) ** 2 + (same["z"] - r["z"]) ** 2)
        if dd.min() < 1.0:
            d2.append(dd.min() ** 2)
    rmse = float(np.sqrt(np.mean(d2)))
    print(f"\nreduced-precision MB positions: {len(d2)} matched of {len(L3)}, RMSE {rmse:.3f} px vs FP64 oracle")
    assert len(d2) >= 0.8 * len(L3_o)
    assert rmse < 0.1
