"""Batched form: uneven ensembles (frame counts, 2K in {2, 4, 8}) in one
persistent launch or one launch per stage, optionally replayed as a CUDA
graph; the launch-shape
autotuner; and the bounded-wait failure path of the persistent queue (a
host-built dependency that never completes must end the launch with
RCA_ERR_TIMEOUT, and the handle must stay usable)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ensembles():
    """five small uneven ensembles of the tiny geometry (seeded)"""
    from synth import generate
    from synth.rca_sim import RcaWorkload, _tiny_geom
    spec = [(7, 1), (23, 2), (40, 4), (11, 1), (18, 2)]   # (frames, K per family)
    out = []
    for q, (F, K) in enumerate(spec):
        w = RcaWorkload(f"b{q}", _tiny_geom(K), n_frames=F, n_mb=20, n_tissue=200, seed=4100 + q)
        out.append((w, generate(w)))
    return out


@pytest.fixture(scope="module")
def handle():
    from paper_2511_21647_gb300 import rca
    h = rca.rca_create(0)
    rca.rca_set_stream(h, torch.cuda.current_stream())
    yield h
    rca.rca_destroy(h)


def make_items(handle, ensembles, with_loc=False):
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import complex_buffer
    items, keep = [], []
    for w, G in ensembles:
        g = w.geom
        geo = rca.rca_geometry_create(handle, g)
        t = rca.rca_delay_tables(handle, geo)
        rf = G.rf.cuda()
        pl = complex_buffer((w.n_frames, 2, 2, g.n_slab, g.nz, g.n_el), 3, "cuda")
        it = dict(tables=t, rf=rf, n_frames=w.n_frames, planes=pl)
        if with_loc:
            it.update(out2d=torch.zeros((4096, 10), dtype=torch.int32, device="cuda"), cap2d=4096,
                      n2d=torch.zeros(1, dtype=torch.int32, device="cuda"),
                      out3d=torch.zeros((4096, 10), dtype=torch.int32, device="cuda"), cap3d=4096,
                      n3d=torch.zeros(1, dtype=torch.int32, device="cuda"))
        items.append(it)
        keep.append((geo, t))
    return items, keep


def free(keep):
    from paper_2511_21647_gb300 import rca
    for geo, t in keep:
        rca.rca_tables_destroy(t)
        rca.rca_geometry_destroy(geo)


def test_persistent_batch_matches_oracle_and_single_calls(handle, ensembles):
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import to_complex128
    items, keep = make_items(handle, ensembles)
    b = rca.rca_batch_create(handle, items, L.RCA_F32, L.RCA_C32, L.RCA_C32)
    try:
        rca.rca_batch_run(b, use_graph=False, h=handle)
        assert rca.rca_sync_status(handle) == L.RCA_OK
        for (w, G), it in zip(ensembles, items):
            got = to_complex128(it["planes"])
            ref = O.beamform_projections(w.geom, G.rf.numpy())
            assert rel(got, ref) < 1e-4, w.name
            single = torch.empty_like(it["planes"])
            rca.rca_beamform_projections(handle, it["tables"], it["rf"], L.RCA_F32, None, w.n_frames,
                                         rca.bf_params(), single, L.RCA_C32)
            torch.cuda.synchronize()
            assert torch.equal(single, it["planes"]), w.name   # same bodies, same order: bit-identical
    finally:
        rca.rca_batch_destroy(b)
        free(keep)


def test_staged_mode_equals_persistent_launch(handle, ensembles):
    """one launch per stage (no dependency waits) gives the persistent
    launch's planes bit for bit, plain and replayed as a graph"""
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300 import rca
    items, keep = make_items(handle, ensembles)
    b = rca.rca_batch_create(handle, items, L.RCA_F32, L.RCA_C32, L.RCA_C32)
    try:
        rca.rca_batch_run(b, use_graph=False, h=handle)
        torch.cuda.synchronize()
        ref = [it["planes"].clone() for it in items]
        for use_graph in (False, True, True):
            rca.rca_batch_set_mode(b, L.RCA_BATCH_STAGED)
            for it in items:
                it["planes"].zero_()
            rca.rca_batch_run(b, use_graph=use_graph, h=handle)
            torch.cuda.synchronize()
            assert rca.rca_sync_status(handle) == L.RCA_OK
            for q, it in enumerate(items):
                assert torch.equal(ref[q], it["planes"]), (use_graph, q)
        with pytest.raises(rca.RcaError):
            rca.rca_batch_set_mode(b, 7)
    finally:
        rca.rca_batch_destroy(b)
        free(keep)


def test_one_shot_batched_call_equals_the_plan(handle, ensembles):
    """rca_beamform_projections_batched (plan, run, synchronise, free) gives
    the plan's planes and lists bit for bit"""
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300 import rca
    items, keep = make_items(handle, ensembles, with_loc=True)
    prm = rca.make_ulm_params(d=5, sig_z=0.807, sig_lat=1.4495, alpha=0.1, ncc_min=0.5)
    try:
        rca.rca_beamform_projections_batched(handle, items, L.RCA_F32, L.RCA_C32, prm)
        first = [(it["planes"].clone(), int(it["n2d"].item()), int(it["n3d"].item())) for it in items]
        b = rca.rca_batch_create(handle, items, L.RCA_F32, L.RCA_C32, L.RCA_C32, prm)
        try:
            for it in items:
                it["planes"].zero_()
                it["n2d"].zero_()
                it["n3d"].zero_()
            rca.rca_batch_run(b, use_graph=False, h=handle)
            assert rca.rca_sync_status(handle) == L.RCA_OK
            for (pl, n2, n3), it in zip(first, items):
                assert torch.equal(pl, it["planes"])
                assert (n2, n3) == (int(it["n2d"].item()), int(it["n3d"].item()))
        finally:
            rca.rca_batch_destroy(b)
    finally:
        free(keep)


def test_batch_graph_replay_and_localisation(handle, ensembles):
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import list2d_numpy
    items, keep = make_items(handle, ensembles, with_loc=True)
    prm = rca.make_ulm_params(d=5, sig_z=0.807, sig_lat=1.4495, alpha=0.1, ncc_min=0.5)
    b = rca.rca_batch_create(handle, items, L.RCA_F32, L.RCA_C32, L.RCA_C32, prm)
    try:
        rca.rca_batch_run(b, use_graph=True, h=handle)      # plain run + capture
        torch.cuda.synchronize()
        first = [it["planes"].clone() for it in items]
        counts = [(int(it["n2d"].item()), int(it["n3d"].item())) for it in items]
        for it in items:
            it["planes"].zero_()
            it["n2d"].zero_()
        rca.rca_batch_run(b, use_graph=True, h=handle)      # graph launch
        torch.cuda.synchronize()
        assert rca.rca_sync_status(handle) == L.RCA_OK
        for q, it in enumerate(items):
            assert torch.equal(first[q], it["planes"])
            assert (int(it["n2d"].item()), int(it["n3d"].item())) == counts[q]
        # localisation of each ensemble equals the single-call localiser on its planes
        from paper_2511_21647_gb300.pipeline import RcaSession
        for (w, G), it in zip(ensembles, items):
            with RcaSession(w.geom) as s:
                o2, n2, o3, n3 = s.localize(it["planes"], prm)
                torch.cuda.synchronize()
                assert int(n2.item()) == int(it["n2d"].item())
                assert np.array_equal(list2d_numpy(o2, int(n2.item())), list2d_numpy(it["out2d"], int(n2.item())))
                assert int(n3.item()) == int(it["n3d"].item())
    finally:
        rca.rca_batch_destroy(b)
        free(keep)


def test_impossible_queue_times_out_and_handle_recovers(handle, ensembles):
    """Ensemble 1's Stage-1 units wait for a demodulation unit that is never
    queued; with a ~10 ms wait bound the persistent launch must end with
    RCA_ERR_TIMEOUT instead of hanging, and later work must still run."""
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import to_complex128
    items, keep = make_items(handle, ensembles[:3])
    b = rca.rca_batch_create(handle, items, L.RCA_F32, L.RCA_C32, L.RCA_C32)
    try:
        rca.rca_batch_set_wait_limit(b, 20_000_000, block_ensemble=1)
        rca.rca_batch_run(b, use_graph=False, h=handle)
        assert rca.rca_sync_status(handle) == L.RCA_ERR_TIMEOUT
        assert rca.rca_sync_status(handle) == L.RCA_OK
        w, G = ensembles[0]
        pl = torch.empty_like(items[0]["planes"])
        rca.rca_beamform_projections(handle, items[0]["tables"], items[0]["rf"], L.RCA_F32, None, w.n_frames,
                                     rca.bf_params(), pl, L.RCA_C32)
        assert rca.rca_sync_status(handle) == L.RCA_OK
        assert rel(to_complex128(pl), O.beamform_projections(w.geom, G.rf.numpy())) < 1e-4
    finally:
        rca.rca_batch_destroy(b)
        free(keep)


def test_autotune_keeps_results(tiny, tiny_rf):
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300 import rca
    from paper_2511_21647_gb300.pipeline import RcaSession, to_complex128
    with RcaSession(tiny.geom) as s:
        iq = s.ingest(tiny_rf.rf.cuda())
        zt, dc, zp = rca.rca_autotune(s.h, s.t, iq, L.RCA_C32, iq.shape[0])
        assert zt in (4, 8, 16, 32) and dc in (4, 8, 16) and zp in (1, 2, 4, 8, 16)
        got = to_complex128(s.beamform(tiny_rf.rf.cuda()))
    ref = O.beamform_projections(tiny.geom, tiny_rf.rf.numpy())
    assert rel(got, ref) < 1e-4
