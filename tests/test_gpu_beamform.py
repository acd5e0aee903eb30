"""GPU parity of the beamforming path (tables, ingest, Stage 1, Stage 2 +
projection, direct conventional projection) against the FP64 oracle on the
same seeded inputs.  FP32 path tolerance: relative L2 <= 1e-4."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def R():
    from paper_2511_21647_gb300 import rca
    return rca


@pytest.fixture(scope="module")
def L():
    from paper_2511_21647_gb300 import _lib
    return _lib


@pytest.fixture(scope="module")
def S(tiny):
    from paper_2511_21647_gb300.pipeline import RcaSession
    s = RcaSession(tiny.geom)
    yield s
    s.close()


@pytest.fixture(scope="module")
def oracle_tiny(tiny, tiny_rf):
    """Oracle IQ, slices and planes of every frame of the tiny ensemble."""
    g = tiny.geom
    rf = tiny_rf.rf.numpy()
    iq = O.demod(g, rf)
    slices = np.stack([O.stage1(g, iq[f]) for f in range(rf.shape[0])])
    planes = np.stack([O.stage2_project(g, slices[f]) for f in range(rf.shape[0])])
    return iq, slices, planes


def c64(x):
    """complex numpy -> [..., 2] float32 cuda tensor"""
    a = np.stack([x.real, x.imag], axis=-1).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def as_c128(t):
    from paper_2511_21647_gb300.pipeline import to_complex128
    return to_complex128(t)


# --- tables ------------------------------------------------------------------------

def test_delay_tables_bit_exact(S, R, L, tiny):
    g = tiny.geom
    t0 = O.t0(g)
    tx = R.rca_tables_download(S.t, L.RCA_TAB_TX_F64)
    exp_tx = np.array([[(O.tau_tx(g, k, 0.0, O.slice_depth(g, r)) - t0) * g.fs for r in range(g.nzs)]
                       for k in range(g.n_tx)])
    assert np.array_equal(tx, exp_tx)
    rx = R.rca_tables_download(S.t, L.RCA_TAB_RX_F64)
    exp_rx = np.array([[O.tau_rx(g, d * g.pitch, O.slice_depth(g, r)) * g.fs for r in range(g.nzs)]
                       for d in range(g.n_el)])
    assert np.array_equal(rx, exp_rx)
    assert np.array_equal(R.rca_tables_download(S.t, L.RCA_TAB_TX_Q16), np.rint(exp_tx * 65536).astype(np.int32))
    assert np.array_equal(R.rca_tables_download(S.t, L.RCA_TAB_RX_Q16), np.rint(exp_rx.T * 65536).astype(np.int32))
    dmax = R.rca_tables_download(S.t, L.RCA_TAB_DMAX)
    exp_dm = [max(d for d in range(g.n_el) if not (d * g.pitch > 0.5 * (O.slice_depth(g, r) / g.fnum)))
              for r in range(g.nzs)]
    assert np.array_equal(dmax, exp_dm)
    sh = R.rca_tables_download(S.t, L.RCA_TAB_S2_SHIFT)
    exp_sh = np.array([[O.shift_dz(g, k, O.elem_pos(g, m)) * g.us / g.dz for m in range(g.n_el)]
                       for k in range(g.n_tx)])
    assert np.array_equal(sh, exp_sh)


def test_weight_tables_within_fp32_rounding(S, R, L, tiny):
    g = tiny.geom
    W = R.rca_tables_download(S.t, L.RCA_TAB_W)
    exp = np.zeros(W.shape, complex)
    for r in range(g.nzs):
        z = O.slice_depth(g, r)
        for d in range(g.n_el):
            trx = O.tau_rx(g, d * g.pitch, z)
            exp[r, d] = O.apod(g, d * g.pitch, z) * np.exp(2j * np.pi * g.fc * (trx - z / g.c))
    assert np.all(np.abs(W - exp) <= 1.5e-7 * np.abs(exp) + 1e-30)
    ec = R.rca_tables_download(S.t, L.RCA_TAB_S2_EC)
    exp_ec = np.array([[np.exp(2j * np.pi * g.fc * O.tau_c(g, k, O.depth(g, i))) for i in range(g.nz)]
                       for k in range(g.n_tx)])
    assert np.max(np.abs(ec - exp_ec)) < 2e-7


# --- stages ------------------------------------------------------------------------

def test_ingest_matches_oracle_demod(S, tiny, tiny_rf, oracle_tiny):
    iq_o = oracle_tiny[0]
    iq = S.ingest(tiny_rf.rf.cuda())
    got = as_c128(iq).transpose(0, 1, 3, 2)          # [F][2K][ns][E] -> [F][2K][E][ns]
    assert rel(got, iq_o) < 1e-5


def test_stage1_matches_oracle(S, oracle_tiny):
    iq_o, sl_o, _ = oracle_tiny
    iq_in = c64(iq_o.transpose(0, 1, 3, 2).copy())
    sl = as_c128(S.stage1(iq_in))
    assert rel(sl, sl_o) < 1e-5
    for f in (0, 31, 63):
        assert rel(sl[f], sl_o[f]) < 1e-5


def test_stage2_projection_matches_oracle(S, oracle_tiny):
    _, sl_o, pl_o = oracle_tiny
    pl = as_c128(S.stage2(c64(sl_o)))
    assert rel(pl, pl_o) < 1e-5


def test_beamform_projections_end_to_end(S, tiny_rf, oracle_tiny):
    """RF -> planes through the public call, FP32 path, vs the oracle."""
    pl_o = oracle_tiny[2]
    pl = as_c128(S.beamform(tiny_rf.rf.cuda()))
    assert rel(pl, pl_o) < TOL_FP32
    # per projection plane (frame, axis, family, slab) on the planes that hold signal
    norms = np.linalg.norm(pl_o.reshape(-1, pl_o.shape[-2] * pl_o.shape[-1]), axis=1)
    errs = np.linalg.norm((pl - pl_o).reshape(norms.size, -1), axis=1)
    big = norms > 1e-3 * norms.max()
    assert np.all(errs[big] / norms[big] < TOL_FP32)


def test_direct_projection_matches_oracle(S, L, tiny, tiny_rf):
    g = tiny.geom
    rf = tiny_rf.rf.numpy()
    frames = [0, 17, 63]
    pl_o = O.beamform_projections(g, rf, mode="direct", frames=frames)
    pl = as_c128(S.beamform(tiny_rf.rf.cuda(), mode=L.RCA_MODE_DIRECT))
    assert rel(pl[frames], pl_o) < TOL_FP32


def test_direct_and_two_stage_agree_at_zero_steering(L, tiny, tiny_rf):
    """theta = 0: the two-stage planes equal the exact conventional ones."""
    import dataclasses
    from paper_2511_21647_gb300.pipeline import RcaSession
    g0 = dataclasses.replace(tiny.geom, ang_rc=(0.0,), ang_cr=(0.0,))
    with RcaSession(g0) as s:
        rf = tiny_rf.rf[:4].cuda()
        a = as_c128(s.beamform(rf))
        b = as_c128(s.beamform(rf, mode=L.RCA_MODE_DIRECT))
    assert rel(a, b) < 1e-5


def test_clutter_none_and_static_input(S, L, tiny):
    """Identical frames + mean removal -> zero planes exactly (static tissue)."""
    g = tiny.geom
    one = torch.randn(1, g.n_tx, g.n_el, g.ns) * 100
    rf = one.repeat(8, 1, 1, 1).contiguous().cuda()
    pl = S.beamform(rf)
    assert float(pl.abs().max()) < 1e-3 * 100
    pl2 = S.beamform(rf, clutter=L.RCA_CLUTTER_NONE)
    assert float(pl2.abs().max()) > 1.0


def test_single_frame_and_ragged_sizes(L, tiny):
    """F = 1, a lateral count that is not a multiple of 32 and a ragged depth."""
    import dataclasses
    from paper_2511_21647_gb300.pipeline import RcaSession
    from synth.rca_sim import RcaWorkload, generate
    g = dataclasses.replace(tiny.geom, n_el=24, nz=37, ns=200)
    w = RcaWorkload("ragged", g, n_frames=3, n_mb=6, n_tissue=0, seed=77)
    G = generate(w)
    pl_o = O.beamform_projections(g, G.rf.numpy())
    with RcaSession(g) as s:
        pl = as_c128(s.beamform(G.rf.cuda()))
        one = as_c128(s.beamform(G.rf[:1].cuda(), clutter=L.RCA_CLUTTER_NONE))
    assert rel(pl, pl_o) < TOL_FP32
    pl1 = O.beamform_projections(g, G.rf.numpy()[:1], remove_mean=False)
    assert rel(one, pl1) < TOL_FP32


def test_host_side_argument_errors(S, R, L, tiny):
    rf = torch.zeros((2, tiny.geom.n_tx, tiny.geom.n_el, tiny.geom.ns), device="cuda")
    pl = torch.zeros(S.planes_shape(2) + (2,), device="cuda")
    with pytest.raises(R.RcaError) as e:
        R.rca_beamform_projections(S.h, S.t, rf, L.RCA_C32, None, 2, R.bf_params(), pl, L.RCA_C32)
    assert e.value.status == L.RCA_ERR_UNSUPPORTED
    with pytest.raises(R.RcaError) as e:
        R.rca_beamform_projections(S.h, S.t, rf, L.RCA_I16, None, 2, R.bf_params(), pl, L.RCA_C32)
    assert e.value.status == L.RCA_ERR_INVALID_ARG
    with pytest.raises(R.RcaError) as e:
        R.rca_beamform_projections(S.h, S.t, rf, L.RCA_F32, None, 0, R.bf_params(), pl, L.RCA_C32)
    assert e.value.status == L.RCA_ERR_SHAPE
    import dataclasses
    bad = dataclasses.replace(tiny.geom, P=7)
    with pytest.raises(R.RcaError) as e:
        R.rca_geometry_create(S.h, bad)
    assert e.value.status == L.RCA_ERR_INVALID_ARG
    assert R.rca_sync_status(S.h) == L.RCA_OK
