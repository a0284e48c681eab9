"""Multi-process paths on CPU (gloo, world size 2): the bench's bookkeeping
(the step time is the maximum over ranks, the job rate counts every rank's
cells, only rank 0 prints, the reference arm included), and the partition of
one diagram's cells over ranks (each rank's part from the oracle, gathered
into the whole diagram; each rank's partial gradient, all-reduced into the
whole gradient). No GPU."""
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
    prate = bench.partition_rate(1000, ms)  # one diagram of 1000 cells split over the ranks
    # independent point sets per rank
    x0 = bench.make_workload("uniform10k", rank)[0]
    dist.barrier()
    print(json.dumps({"rank": rank, "ws": ws, "ms": ms, "rate": rate, "prate": prate,
                      "first": [float(v) for v in x0[0]]}))
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
        assert r["prate"] == pytest.approx(1000 / 15e-3 / 1e6)
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


PARTITION_WORKER = textwrap.dedent('''
    import json, os, sys
    sys.path.insert(0, os.environ["ROOT"])
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2605_06408_gb300 import partition
    from paper_2605_06408_gb300 import workloads as W
    dist.init_process_group("gloo", init_method="env://")
    ws, rank = dist.get_world_size(), dist.get_rank()
    n = 3000
    x = W.mixture(n, 5)
    w = W.power_weights(x, 6)
    # this rank's cells: its contiguous range of a Morton order of the sites
    q = np.minimum((x * 1024).astype(np.int64), 1023)
    key = np.zeros(n, np.int64)
    for b in range(10):
        for a in range(3):
            key |= ((q[:, a] >> b) & 1) << (3 * b + a)
    order = np.argsort(key, kind="stable")
    lo, hi = partition.part_range(n, rank, ws)
    mine = np.sort(order[lo:hi])
    ref = oracle.cells(x, w, cells=mine, threads=2)
    counts = np.zeros(n, np.int64)
    counts[mine] = ref["counts"]
    off = torch.from_numpy(np.concatenate([[0], np.cumsum(counts)]).astype(np.int32))
    vol = torch.zeros(n, dtype=torch.float64)
    vol[mine] = torch.from_numpy(ref["vol"])
    cen = torch.zeros(n, 3, dtype=torch.float64)
    cen[mine] = torch.from_numpy(ref["cen"])
    go, gn, gv, gc = partition.gather(off, torch.from_numpy(ref["indices"]), vol, cen)
    full = oracle.cells(x, w, threads=2)
    ok_rows = bool(np.array_equal(go.numpy(), full["offsets"]) and np.array_equal(gn.numpy(), full["indices"]))
    ok_geo = bool(np.array_equal(gv.numpy(), full["vol"]) and np.array_equal(gc.numpy(), full["cen"]))
    # gradients: each rank's cells only, then one sum over ranks
    c, d = W.loss_coefficients(n, 7)
    gp, gw, _ = oracle.grad(x, w, W.UNIT_BOX, c, d, cells=mine, threads=2)
    ogp, ogw, _ = oracle.grad(x, w, W.UNIT_BOX, c, d, threads=2)
    part_only = float(np.abs(gp - ogp).max() / np.abs(ogp).max())
    tp, tw = torch.from_numpy(gp.copy()), torch.from_numpy(gw.copy())
    partition.allreduce_gradients(tp, tw)
    ep = float(np.abs(tp.numpy() - ogp).max() / np.abs(ogp).max())
    ew = float(np.abs(tw.numpy() - ogw).max() / np.abs(ogw).max())
    print(json.dumps({"rank": rank, "cells": len(mine), "rows": ok_rows, "geometry": ok_geo, "ep": ep, "ew": ew,
                      "part_only": part_only, "empty": int(np.sum(full["vol"] == 0))}))
    dist.destroy_process_group()
''')


def test_partition_of_one_diagram_gather_and_gradient_sum():
    outs = _launch([sys.executable, "-c", PARTITION_WORKER])
    rows = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(r["rank"] for r in rows) == [0, 1]
    assert sum(r["cells"] for r in rows) == 3000
    for r in rows:
        assert r["rows"] and r["geometry"]  # every rank holds the whole diagram
        assert r["ep"] < 1e-12 and r["ew"] < 1e-12  # the summed gradient is the whole gradient
        assert r["part_only"] > 1e-3  # one part alone is not
        assert r["empty"] > 0  # the power set has empty cells
