"""The bounds-checked build (librca_checked.so, compiled with -DRCA_CHECKED):
its kernels check every shared-memory ring slot and record block of Stage 1,
every staged window row of Stage 2, the strip rows, flag and bitmap indexes
of the NCC detection and the pixels its gather reads, and every queue segment
and counter index of the persistent batched launch, and record RCA_ERR_BOUNDS in the status
word instead of trapping.  On the tiny ensemble (one-call beamformer with
the paired and unpaired Stage-1 kernels at 32, 64 and 128 elements,
localisation) and on a batch of
uneven ensembles (persistent launch, also as a CUDA graph) every call must
return RCA_OK with a clean status word and outputs bit-identical to the
release build's.  Each build runs in a fresh process (RCA_LIBRARY selects
the library)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import dataclasses, json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from synth import generate, workload
from synth.rca_sim import RcaWorkload, _tiny_geom
from paper_2511_21647_gb300 import _lib as L, rca
from paper_2511_21647_gb300.pipeline import RcaSession, complex_buffer
out, status = {}, []
w = workload("tiny")
G = generate(w)
prm = rca.make_ulm_params(d=5, sig_z=0.807, sig_lat=1.4495, alpha=0.1, ncc_min=0.5)
for n_el in (32, 64, 128):
    g = dataclasses.replace(w.geom, n_el=n_el) if n_el != 32 else w.geom
    ww = dataclasses.replace(w, geom=g, n_frames=16)
    rf = generate(ww).rf.cuda() if n_el != 32 else G.rf.cuda()
    with RcaSession(g) as s:
        pl = s.beamform(rf)
        o2, n2, o3, n3 = s.localize(pl, prm)
        torch.cuda.synchronize()
        status.append(s.sync_status())
        out[f"planes{n_el}"] = pl.cpu().numpy()
        out[f"l2_{n_el}"] = o2[: int(n2.item())].cpu().numpy()
        out[f"l3_{n_el}"] = o3[: int(n3.item())].cpu().numpy()
h = rca.rca_create(0)
rca.rca_set_stream(h, torch.cuda.current_stream())
items, keep = [], []
for q, (F, K) in enumerate([(7, 1), (23, 2), (40, 4), (11, 1)]):
    wq = RcaWorkload(f"c{q}", _tiny_geom(K), n_frames=F, n_mb=20, n_tissue=200, seed=4500 + q)
    gq = wq.geom
    geo = rca.rca_geometry_create(h, gq)
    t = rca.rca_delay_tables(h, geo)
    pl = complex_buffer((F, 2, 2, gq.n_slab, gq.nz, gq.n_el), L.RCA_C32, "cuda")
    items.append(dict(tables=t, rf=generate(wq).rf.cuda(), n_frames=F, planes=pl))
    keep.append((geo, t))
b = rca.rca_batch_create(h, items, L.RCA_F32, L.RCA_C32, L.RCA_C32)
for use_graph in (False, True):
    for it in items:
        it["planes"].zero_()
    rca.rca_batch_run(b, use_graph=use_graph, h=h)
    status.append(rca.rca_sync_status(h))
    for q, it in enumerate(items):
        out[f"batch{int(use_graph)}_{q}"] = it["planes"].cpu().numpy()
rca.rca_batch_destroy(b)
for geo, t in keep:
    rca.rca_tables_destroy(t)
    rca.rca_geometry_destroy(geo)
rca.rca_destroy(h)
np.savez(sys.argv[2], status=np.array(status), **out)
"""


def run(lib, path):
    env = dict(os.environ, RCA_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, str(path)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(str(path) + ".npz" if not str(path).endswith(".npz") else str(path))


def test_checked_build_matches_release_bit_for_bit(tmp_path):
    from paper_2511_21647_gb300 import _lib as L
    from paper_2511_21647_gb300.build import LIB_CHECKED
    assert os.path.exists(LIB_CHECKED), "the checked build is made by __graft_entry__.build()"
    rel = run("release", tmp_path / "release.npz")
    chk = run("checked", tmp_path / "checked.npz")
    assert list(chk["status"]) == [L.RCA_OK] * len(chk["status"]), list(chk["status"])
    assert list(rel["status"]) == [L.RCA_OK] * len(rel["status"])
    assert sorted(chk.files) == sorted(rel.files)
    for k in rel.files:
        if k == "status":
            continue
        assert rel[k].shape == chk[k].shape and np.array_equal(rel[k].view(np.uint8), chk[k].view(np.uint8)), k
    assert rel["l3_32"].shape[0] > 0 and rel["l3_64"].shape[0] >= 0
