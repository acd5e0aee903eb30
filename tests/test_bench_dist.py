"""Host-side logic of the multi-GPU bench path (independent replicas, no
exchange step) on two gloo ranks over 127.0.0.1: rendezvous, barrier, the
job time taken as the slowest rank's, the whole-job throughput, exactly one
JSON line (from rank 0), and the reference arm's other ranks leaving without
work.  CUDA is hidden from the ranks, so this runs on any host."""
import json
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = textwrap.dedent("""
    import contextlib, io, json, os, sys
    sys.path.insert(0, {root!r})
    import bench
    rank, world, local = bench.dist_init()
    assert world == 2 and local == rank
    bench.barrier(world)
    ms = 10.0 + 5.0 * rank                 # rank 1 is the slower replica
    mx = bench.max_over_ranks(ms, world)
    value = bench.job_throughput(300, 4, mx, world)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.emit({{"value": value, "n_gpus": world}}, rank)
    class A:  # the reference arm returns before reading its options on rank > 0
        pass
    ref = io.StringIO()
    if rank > 0:
        with contextlib.redirect_stdout(ref):
            bench.reference_arm(A())
    bench.barrier(world)
    import torch.distributed as dist
    dist.destroy_process_group()
    with open(os.path.join({out!r}, "rank%d.json" % rank), "w") as f:
        json.dump({{"max_ms": mx, "value": value, "printed": buf.getvalue(), "ref_printed": ref.getvalue()}}, f)
""")


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_replica_aggregation(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(RANK_SCRIPT.format(root=ROOT, out=str(tmp_path)))
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(r),
                   LOCAL_RANK=str(r), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        outs.append((p.returncode, o, e))
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    # both ranks see the slowest replica's time; throughput counts both replicas' frames
    assert res[0]["max_ms"] == res[1]["max_ms"] == 15.0
    expected = 2 * 300 * 4 / 0.015
    assert abs(res[0]["value"] - expected) < 1e-6 and abs(res[1]["value"] - expected) < 1e-6
    # one line in total, from rank 0
    line = json.loads(res[0]["printed"])
    assert line == {"value": expected, "n_gpus": 2}
    assert res[1]["printed"] == ""
    # the reference arm does no work on rank 1
    assert res[1]["ref_printed"] == ""


def test_single_rank_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert abs(bench.job_throughput(300, 10, 20.0, 1) - 150000.0) < 1e-9
