"""The multi-process path of bench.py on CPU (gloo, world size 2): each
rank builds its own set (replicas, weak scaling), the step time is the
maximum over ranks, the job rate counts every rank's cells, and only rank 0
prints (the reference arm included). No GPU and no oracle work."""
import json
import os
import socket
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = textwrap.dedent('''
    import json, os, sys
    sys.path.insert(0, os.environ["ROOT"])
    import torch.distributed as dist
    import bench
    ws, rank, local = bench.dist_env()
    dist.init_process_group("gloo", init_method="env://")
    # per-rank step times: the slowest rank sets the job time
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    rate = bench.job_rate(1000, ws, ms)
    # independent point sets per rank
    x0 = bench.make_workload("uniform10k", rank)[0]
    dist.barrier()
    print(json.dumps({"rank": rank, "ws": ws, "ms": ms, "rate": rate, "first": [float(v) for v in x0[0]]}))
    dist.destroy_process_group()
''')


def _launch(script, extra_env=None, nproc=2):
    port = _free_port()
    procs = []
    for r in range(nproc):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(nproc),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen(script, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                      cwd=ROOT))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_two_ranks_max_time_and_job_rate():
    outs = _launch([sys.executable, "-c", WORKER])
    rows = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert {r["rank"] for r in rows} == {0, 1}
    for r in rows:
        assert r["ws"] == 2
        assert r["ms"] == 15.0  # the maximum over ranks, on every rank
        assert r["rate"] == pytest.approx(1000 * 2 / 15e-3 / 1e6)
    assert rows[0]["first"] != rows[1]["first"]  # each rank has its own point set


def test_reference_arm_prints_on_rank_zero_only(tmp_path):
    # the reference arm times the oracle; a tiny sample keeps this cheap
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "uniform10k",
           "--steps", "1", "--warmup", "0", "--cpu-sample", "300", "--gpus", "2"]
    outs = _launch(cmd)
    lines = [[l for l in o.splitlines() if l.startswith("{")] for o in outs]
    by_rank = dict(zip((0, 1), lines))
    assert len(by_rank[0]) == 1 and by_rank[1] == []
    d = json.loads(by_rank[0][0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
