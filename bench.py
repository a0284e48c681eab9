#!/usr/bin/env python
"""Throughput of the Voronoi / power-cell build on GB300.

One step = one forward build of the whole point set (Morton keys, radix
sort, LBVH, fused traversal + cull + clip kernel, large-cell pass, CSR
compaction) with the sites already resident in device memory; the reported
value is Mcells/s. The default workload is the largest configuration that
fits one GPU: 20,000,000 sites in nested Gaussian shells around random
surfaces, forward and forward+backward. Forward+backward throughput, the
end-to-end number through the C ABI from pinned host buffers, the roofline
of the fused kernel (and, beside it, of the large-cell pass) and the FP64 CPU
oracle on the host cores are reported in the same JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle, same workload

Under torchrun (N > 1), by default (--mode partition) the ranks split one
diagram's cells: every rank holds all sites and builds the whole LBVH, then
makes the cells of its contiguous Morton-order range (vd_set_partition); the
forward's outputs stay sharded and the forward+backward step ends with one
NCCL all-reduce of the gradients (strong scaling: value = the diagram's
cells / the slowest rank's time). --mode replicas gives every rank its own
independent point set instead (weak scaling, no collective on the data
path). The step time is the maximum over ranks either way.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcells/s forward and forward+backward on 1 GB300 at oracle-exact neighbours; % of roofline"

WORKLOADS = {
    "mixture1M": "Voronoi of 1,000,000 sites from 64 anisotropic Gaussians (per-axis sigma log-uniform in "
                 "[1e-3,1e-1]) + 10% uniform background, unit box, float32, seed 1",
    "power1M": "power diagram of the mixture1M sites with w = r^2, r = 0.2 nn exp(N(0,1)), seed 2",
    "uniform10k": "Voronoi of 10,000 uniform sites in the unit cube, seed 0",
    "mixture200k": "Voronoi of 200,000 sites of the mixture1M distribution (seed 1); the small case used for "
                   "full ncu captures",
    "surfaces20M": "Voronoi of 20,000,000 sites in nested Gaussian shells (sigma 1e-2..1e-5) around 32 "
                   "random surfaces + 1% background, seed 4",
    "surfaces2M": "Voronoi of 2,000,000 sites of the surfaces20M distribution (seed 4); the smaller case of "
                  "that distribution used for ncu captures",
    "power200k": "power diagram of 200,000 mixture sites (seed 1) with the power1M weight law (seed 2); the "
                 "small case used for ncu captures of the large-cell kernel",
    "uniform1M": "Voronoi of 1,000,000 uniform sites (the paper's white-noise case, Sec. 5.1), seed 5",
    "gradient1M": "Voronoi of 1,000,000 sites with density linear in x (the paper's gradient case), seed 5",
    "clustered1M_K10": "Voronoi of 1,000,000 sites in 10 isotropic Gaussian clusters, sigma = 0.005 of the box "
                       "(the paper's K=10, sigma=0.1 in [-10,10]^3), clamped to the box, seed 6",
    "clustered1M_K5": "as clustered1M_K10 with 5 clusters",
    "gaussw_uniform1M": "power diagram of uniform1M with the paper's weights w ~ N(0, (d_nn^2/3)^2), seed 7",
    "uniform1M_wratio": "power diagram of uniform1M with w ~ N(0, (r d_nn^2)^2), r = --weight-ratio (the paper's "
                        "weight-ratio sweep, on uniform sites), seed 7",
    "batched256": "256 independent sets, sizes log-uniform in [1e3, 2e5] (~9M sites), odd sets power "
                  "(w = r^2, r = 0.2 nn exp(N(0,1))), uniform or mixture per set, seed 3; one build_batched "
                  "per step, replayed from a CUDA graph",
}

# algorithmic FP32 work per counted event:
# one vertex/plane sign test = 3 FMA; one new vertex = three cross products,
# a determinant, three 3-term numerators and a reciprocal (51 flop); one leaf
# candidate = its plane and support test (30 flop); one BVH child = its
# distance, radius and bound (40 flop).
FLOP_VTEST, FLOP_NEWV, FLOP_CAND, FLOP_NODE = 6, 51, 30, 40


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="surfaces20M", choices=sorted(WORKLOADS))
    p.add_argument("--no-backward", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample", type=int, default=300_000, help="cells in the oracle's timed sample")
    p.add_argument("--config", default="", help="JSON dict of libvd config overrides")
    p.add_argument("--no-autotune", action="store_true", help="skip vd_autotune before the timed steps")
    p.add_argument("--no-forms", action="store_true", help="skip the plain-FP32 and per-set comparisons")
    p.add_argument("--accuracy-sample", type=int, default=20_000, help="cells checked against the oracle")
    p.add_argument("--weight-ratio", type=float, default=1.0 / 3.0, help="r of the uniform1M_wratio workload")
    p.add_argument("--mode", default="partition", choices=["partition", "replicas"],
                   help="N > 1: split one diagram's cells over the ranks, or one independent diagram per rank")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(v, dist, device):
    """The maximum of v over all ranks (None and single-process: v)."""
    if dist is None or v is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(cells_per_rank: int, world_size: int, ms: float) -> float:
    """Whole-job Mcells/s: every rank builds its own set of cells_per_rank
    sites (replicas, weak scaling), timed by the slowest rank."""
    return cells_per_rank * world_size / (ms * 1e-3) / 1e6


def partition_rate(cells: int, ms: float) -> float:
    """Whole-job Mcells/s when the ranks split one diagram of `cells` cells,
    timed by the slowest rank (strong scaling)."""
    return cells / (ms * 1e-3) / 1e6


def make_workload(name: str, rank: int):
    """(xyz, weights or None, box, batch) where batch = (set offsets, boxes,
    weighted flags) for batched workloads, else None."""
    from paper_2605_06408_gb300 import workloads as W

    seed_shift = 1000 * rank  # independent point sets per rank
    if name == "batched256":
        X, Wt, offs, flags = W.batched(3 + seed_shift)
        return X, Wt, W.UNIT_BOX, (offs, [W.UNIT_BOX] * (len(offs) - 1), flags)
    x, w, box = _single_workload(name, seed_shift)
    return x, w, box, None


WEIGHT_RATIO = 1.0 / 3.0


def _single_workload(name: str, seed_shift: int):
    from paper_2605_06408_gb300 import workloads as W

    if name == "mixture1M":
        return W.mixture(1_000_000, 1 + seed_shift), None, W.UNIT_BOX
    if name == "power1M":
        x = W.mixture(1_000_000, 1 + seed_shift)
        return x, W.power_weights(x, 2 + seed_shift), W.UNIT_BOX
    if name == "uniform10k":
        return W.uniform(10_000, 0 + seed_shift), None, W.UNIT_BOX
    if name == "mixture200k":
        return W.mixture(200_000, 1 + seed_shift), None, W.UNIT_BOX
    if name == "surfaces20M":
        return W.surfaces(20_000_000, 4 + seed_shift), None, W.UNIT_BOX
    if name == "surfaces2M":
        return W.surfaces(2_000_000, 4 + seed_shift), None, W.UNIT_BOX
    if name == "power200k":
        x = W.mixture(200_000, 1 + seed_shift)
        return x, W.power_weights(x, 2 + seed_shift), W.UNIT_BOX
    if name == "uniform1M":
        return W.uniform(1_000_000, 5 + seed_shift), None, W.UNIT_BOX
    if name == "gradient1M":
        return W.gradient(1_000_000, 5 + seed_shift), None, W.UNIT_BOX
    if name in ("clustered1M_K10", "clustered1M_K5"):
        return W.clustered(1_000_000, 10 if name.endswith("K10") else 5, 6 + seed_shift), None, W.UNIT_BOX
    if name == "gaussw_uniform1M":
        x = W.uniform(1_000_000, 5 + seed_shift)
        return x, W.gaussian_weights(x, 7 + seed_shift), W.UNIT_BOX
    if name == "uniform1M_wratio":
        x = W.uniform(1_000_000, 5 + seed_shift)
        return x, W.gaussian_weights(x, 7 + seed_shift, ratio=WEIGHT_RATIO), W.UNIT_BOX
    raise KeyError(name)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle

def cpu_oracle_rate(sess, n: int, sample: int, seed: int = 7):
    """The FP64 oracle (k-d tree mode, OpenMP over all host cores) on a
    seeded sample of the workload's cells, from an oracle session already set
    up over all n sites. Returns (Mcells/s, cores, s, cells)."""
    from paper_2605_06408_gb300 import workloads as W

    rng = W.rng_for(seed)
    m = min(sample, n)
    cells = np.sort(rng.choice(n, m, replace=False))
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    sess.cells(cells, threads=cores)
    dt = time.perf_counter() - t0
    return m / dt / 1e6, cores, dt, m


def cpu_oracle_rate_1core(sess, n: int, sample: int, seed: int = 8):
    """The same oracle on one host thread (a smaller seeded sample).
    Returns (Mcells/s, cells)."""
    from paper_2605_06408_gb300 import workloads as W

    rng = W.rng_for(seed)
    m = min(max(2000, sample // 50), n)
    cells = np.sort(rng.choice(n, m, replace=False))
    t0 = time.perf_counter()
    sess.cells(cells, threads=1)
    return m / (time.perf_counter() - t0) / 1e6, m


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    x, w, box, batch = make_workload(args.workload, 0)
    if batch is not None:  # the oracle builds each set on its own: sample the largest set
        offs = batch[0]
        s = int(np.argmax(np.diff(offs)))
        x, w = x[offs[s]:offs[s + 1]], (w[offs[s]:offs[s + 1]] if batch[2][s] else None)
    import oracle

    sample = min(args.cpu_sample // 3, len(x))
    t0 = time.perf_counter()
    sess = oracle.Session(x, w, box)  # duplicate marks + k-d tree over all sites, once
    setup_s = time.perf_counter() - t0
    for k in range(args.warmup):
        cpu_oracle_rate(sess, len(x), min(sample, 20_000), seed=200 + k)
    rates, times = [], []
    for k in range(args.steps):
        r, cores, dt, m = cpu_oracle_rate(sess, len(x), sample, seed=100 + k)
        rates.append(r)
        times.append(dt)
    sess.close()
    value = len(rates) * sample / sum(times) / 1e6
    cb = {"value": value, "unit": "Mcells/s", "cores": cores, "kind": "oracle",
          "sample": f"{sample} seeded cells of {args.workload} per step (FP64 k-d tree oracle, all host cores; "
                    f"its set-up over all sites, {setup_s:.1f} s, done once before the steps)"}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mcells/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "n": len(x)},
           "cpu_baseline": cb, "e2e": {"value": value, "unit": "Mcells/s", "h2d_bytes_per_step": 0,
                                       "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------- GPU

def fused_traffic_from_profiles(src_hash: str, workload: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary for this workload (profiles/cells_kernel_<workload>.md; a
    capture of a smaller case of the same distribution, scaled by the cells
    one launch processes), if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"cells_kernel_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    h = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if h and b and h.group(1) == src_hash:
        return float(b.group(1))
    return None


def kernel_source_hash() -> str:
    import hashlib

    hsh = hashlib.sha256()
    for f in ("vd_cells.cu", "vd_big.cuh", "vd_clip.cuh", "vd_internal.cuh"):
        hsh.update(open(os.path.join(ROOT, "paper_2605_06408_gb300", "csrc", f), "rb").read())
    return hsh.hexdigest()[:16]


def accuracy_sample(sess, n: int, sample: int, seed: int = 11):
    """(cells, oracle result) for `sample` seeded cells of a set of n sites."""
    from paper_2605_06408_gb300 import workloads as W

    m = min(sample, n)
    cells = np.sort(W.rng_for(seed).choice(n, m, replace=False))
    return cells, sess.cells(cells)


def accuracy(res, cells, ref, base: int = 0):
    """Neighbour lists, volumes and centroids of the sampled cells of one set
    (rows base + i of res) against the FP64 oracle's result for them."""
    m = len(cells)
    off = res.offsets.cpu().numpy().astype(np.int64)
    nb = res.neighbors.cpu().numpy()
    vol = res.volume.cpu().numpy().astype(np.float64)[base + cells]
    cen = res.centroid.cpu().numpy().astype(np.float64)[base + cells]
    bad = sum(not np.array_equal(nb[off[base + i]:off[base + i + 1]], ref["nbrs"][q]) for q, i in enumerate(cells))
    rv = ref["vol"]
    nz = rv > 0
    ve = float(np.max(np.abs(vol[nz] - rv[nz]) / rv[nz])) if nz.any() else 0.0
    ce = float(np.max(np.linalg.norm(cen - ref["cen"], axis=1) / np.linalg.norm(ref["cen"], axis=1)))
    return {"cells": int(m), "neighbour_lists_differing": int(bad), "max_volume_rel_err": ve,
            "max_centroid_rel_err": ce, "oracle_degenerate_predicates": int(ref["stats"]["degenerate"])}


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        dist = None
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2605_06408_gb300 import vd

    split = ws > 1 and args.mode == "partition"
    # one diagram split over the ranks, or an independent diagram per rank
    x, w, box, batch = make_workload(args.workload, 0 if split else rank)
    n = len(x)
    cfg = {"timing": 1}
    if args.config:
        cfg.update(json.loads(args.config))

    def new_ctx(c):
        k = vd.Context(local, c)
        if split:
            k.set_partition(rank, ws)
        return k

    ctx = new_ctx(cfg)
    sites = torch.from_numpy(x).to(dev)
    weights = None if w is None else torch.from_numpy(w).to(dev)
    flush = torch.empty(256 * 2**20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def build(c, xs, wts, cap=None, sync=True):
        if batch is None:
            return c.build(xs, wts, box, nnz_capacity=cap, sync=sync)
        return c.build_batched(xs, wts, batch[0], batch[1], batch[2], nnz_capacity=cap, sync=sync)

    # autotune (outside the timed region): the configuration the steps use
    tune_s = None
    if not args.no_autotune:
        t0 = time.time()
        if batch is None:
            ctx.autotune(sites, weights, box)
        else:
            ctx.autotune_batched(sites, weights, batch[0], batch[1], batch[2])
        tune_s = time.time() - t0
    cfg = dict(ctx.config)

    # warm-up (also sizes the workspace and the neighbour buffer)
    res = None
    for _ in range(max(args.warmup, 1)):
        res = build(ctx, sites, weights)
    nnz = res.nnz
    cap = nnz + 1024
    st = ctx.status()

    # algorithmic work of one build, from a separate counting run
    cctx = new_ctx(dict(cfg, counters=1))
    build(cctx, sites, weights)
    cnt = cctx.status()
    # the main pass (fused kernel) and the large-cell pass are counted apart
    flop = (FLOP_VTEST * cnt["vertex_tests"] + FLOP_NEWV * cnt["new_vertices"] + FLOP_CAND * cnt["candidates"]
            + FLOP_NODE * cnt["nodes"])
    flop_large = (FLOP_VTEST * cnt["large_vertex_tests"] + FLOP_NEWV * cnt["large_new_vertices"]
                  + FLOP_CAND * cnt["large_candidates"] + FLOP_NODE * cnt["large_nodes"])
    del cctx

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- timed forward steps
    sampler = ClockSampler(local)
    step_ms, cells_ms, large_ms, launches = [], [], [], 0
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    graph = None
    if batch is not None or n <= 100_000:
        # batched and small builds replay one captured launch sequence
        # (vd_build / vd_build_batched enqueue kernels, async copies and
        # memsets only): the launch cost of a small build is paid once
        gctx = new_ctx(dict(cfg, timing=0))  # the tuned configuration
        gctx.reserve(n, weights is not None)
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            build(gctx, sites, weights, cap, sync=False)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            build(gctx, sites, weights, cap, sync=False)
        graph.replay()
        torch.cuda.synchronize()
        g_launches = gctx.timings()["launches"]
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if graph is not None:
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            launches += g_launches
            continue
        e0.record(stream)
        build(ctx, sites, weights, cap, sync=False)
        e1.record(stream)
        t = ctx.timings()  # synchronises the stream
        step_ms.append(e0.elapsed_time(e1))
        cells_ms.append(t["cells_ms"])
        large_ms.append(t["overflow_ms"])
        launches += t["launches"]
    if graph is not None:  # the kernels' times from eager builds with events
        for _ in range(2):
            flush.zero_()
            build(ctx, sites, weights, cap, sync=False)
            t = ctx.timings()
            cells_ms.append(t["cells_ms"])
            large_ms.append(t["overflow_ms"])
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = statistics.mean(step_ms)
    ms_min = min(step_ms)

    # the set the oracle samples: the whole input, or the largest set of a
    # batch (the oracle builds each set on its own); one oracle session (its
    # k-d tree built once) serves the accuracy sample and the CPU baseline
    if batch is None:
        ax, aw, abase = x, w, 0
    else:
        offs = batch[0]
        s_big = int(np.argmax(np.diff(offs)))
        abase = int(offs[s_big])
        ax = x[offs[s_big]:offs[s_big + 1]]
        aw = w[offs[s_big]:offs[s_big + 1]] if batch[2][s_big] else None
    sess_box = []

    def oracle_session():
        if not sess_box:
            import oracle

            t0 = time.perf_counter()
            sess_box.append(oracle.Session(ax, aw, box))
            sess_box.append(time.perf_counter() - t0)
        return sess_box[0]

    # ---- the same build in plain FP32, and (batched) as one build per set
    forms = None
    if not args.no_forms and rank == 0 and not split:
        def timed(fn, reps=3):
            out = fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                out = fn()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            return statistics.mean(ts), out

        f32 = vd.Context(local, dict(cfg, timing=0, precision=1))
        # plain FP32 derails on ill-conditioned cells and can be much slower:
        # one timed build after the warm-up on large inputs
        f32_ms, r32 = timed(lambda: build(f32, sites, weights, cap * 2, sync=False), reps=3 if n <= 2_000_000 else 1)
        torch.cuda.synchronize()
        if f32.status()["error"] != 0:  # (a neighbour-capacity error would leave rows unwritten)
            r32 = build(f32, sites, weights)
        sess = oracle_session()
        acells, aref = accuracy_sample(sess, len(ax), args.accuracy_sample)
        forms = {
            "mixed_fp32_fp64": {"mcells_s": n / (ms * 1e-3) / 1e6, "accuracy": accuracy(res, acells, aref, abase)},
            "plain_fp32": {"mcells_s": n / (f32_ms * 1e-3) / 1e6, "ms_per_step": f32_ms,
                           "accuracy": accuracy(r32, acells, aref, abase)},
        }
        del f32, r32
        if batch is not None:
            offs = batch[0]
            per = vd.Context(local, dict(cfg, timing=0))
            views = []
            for s in range(len(offs) - 1):
                a, b = int(offs[s]), int(offs[s + 1])
                views.append((sites[a:b], None if (weights is None or not batch[2][s]) else weights[a:b],
                              batch[1][s]))

            def per_set():
                for xs, wt, bx in views:
                    per.build(xs, wt, bx, sync=False)

            per_ms, _ = timed(per_set, reps=2)
            forms["per_set_builds"] = {"mcells_s": n / (per_ms * 1e-3) / 1e6, "ms_per_step": per_ms,
                                       "builds": len(views), "note": "one vd_build per set, same stream"}
            del per

    # ---- forward + backward
    fb_ms = None
    if not args.no_backward:
        from paper_2605_06408_gb300 import workloads as W

        c, d = W.loss_coefficients(n, 4)
        gv = torch.from_numpy(c).float().to(dev)
        gc = torch.from_numpy(d).float().to(dev)
        # a backward follows each build: the context keeps the forward's cells
        bctx = new_ctx(dict(cfg, tape=1))
        build(bctx, sites, weights, cap, sync=False)
        bctx.backward(gv, gc, want_weights=weights is not None)
        torch.cuda.synchronize()
        fb = []
        barrier()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            build(bctx, sites, weights, cap, sync=False)
            gp, gw = bctx.backward(gv, gc, want_weights=weights is not None)
            if split:  # each rank's adjoint covered its own cells: sum over ranks
                from paper_2605_06408_gb300 import partition

                partition.allreduce_gradients(gp, gw)
            e1.record(stream)
            e1.synchronize()
            fb.append(e0.elapsed_time(e1))
        barrier()
        fb_ms = statistics.mean(fb)
        del bctx

    # ---- end to end through the C ABI from pinned host buffers
    h_sites = torch.from_numpy(x).pin_memory()
    h_w = None if w is None else torch.from_numpy(w).pin_memory()
    d_sites = torch.empty_like(sites)
    d_w = None if w is None else torch.empty_like(weights)
    h_off = torch.empty(n + 1, dtype=torch.int32).pin_memory()
    h_nb = torch.empty(nnz, dtype=torch.int32).pin_memory()
    h_vol = torch.empty(n, dtype=torch.float32).pin_memory()
    h_cen = torch.empty(n, 3, dtype=torch.float32).pin_memory()
    e2e = []
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vd.copy_(d_sites, h_sites)
        if d_w is not None:
            vd.copy_(d_w, h_w)
        r = build(ctx, d_sites, d_w, cap, sync=False)
        vd.copy_(h_off, r.offsets)
        vd.copy_(h_nb, r.neighbors[:nnz])
        vd.copy_(h_vol, r.volume)
        vd.copy_(h_cen, r.centroid)
        e1.record(stream)
        e1.synchronize()
        e2e.append(e0.elapsed_time(e1))
    barrier()
    e2e_ms = statistics.mean(e2e)
    h2d = 12 * n + (4 * n if w is not None else 0)
    d2h = 4 * (n + 1) + 4 * nnz + 16 * n

    ms = max_over_ranks(ms, dist, dev)
    fb_ms = max_over_ranks(fb_ms, dist, dev)
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    def job_value(t_ms):
        """Whole-job Mcells/s for a step of t_ms (the slowest rank's)."""
        return partition_rate(n, t_ms) if split else job_rate(n, ws, t_ms)

    props = torch.cuda.get_device_properties(dev)
    sm_max = 2070.0
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        sm_max = float(json.load(open(peaks_path)).get("sm_max_mhz", sm_max))
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6  # FP32 lanes x FMA x clock
    cms = statistics.mean(cells_ms)
    lms = statistics.mean(large_ms) if large_ms else 0.0
    achieved = flop / (cms * 1e-3)
    achieved_large = flop_large / (lms * 1e-3) if lms > 0 else 0.0
    src_hash = kernel_source_hash()
    traffic = fused_traffic_from_profiles(src_hash, args.workload)

    cpu = None
    if not args.no_cpu_baseline:
        sess = oracle_session()
        rate, cores, dt, m = cpu_oracle_rate(sess, len(ax), args.cpu_sample)
        rate1, m1 = cpu_oracle_rate_1core(sess, len(ax), args.cpu_sample)
        cpu = {"value": rate, "unit": "Mcells/s", "cores": cores, "kind": "oracle",
               "sample": f"{m} seeded cells of {args.workload}"
                         + (" (its largest set)" if batch is not None else "")
                         + f" ({dt:.1f} s, FP64 k-d tree oracle, all host cores; its set-up over all "
                         f"{len(ax)} sites, {sess_box[1]:.1f} s, done once and not included)",
               "value_1core": rate1, "sample_1core": f"{m1} seeded cells, one host thread",
               "setup_s": sess_box[1]}
    if sess_box:
        sess_box[0].close()

    out = {
        "metric": METRIC,
        "value": job_value(ms),
        "unit": "Mcells/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "ms_per_step_min": ms_min,
        "higher_is_better": True,
        "scaling": "strong" if split else "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "n": n,
                   "weighted": w is not None, "l2": "flushed between timed steps (256 MiB write)",
                   "timed_step": "CUDA graph replay" if graph is not None else "eager vd_build",
                   "multi_gpu": (f"one diagram split over {ws} ranks (Morton-order cell ranges, LBVH replicated; "
                                 "gradients all-reduced)") if split else (
                                 f"{ws} independent diagrams" if ws > 1 else None),
                   "libvd": {k: v for k, v in ctx.config.items()},
                   "autotuned": not args.no_autotune, "autotune_s": tune_s,
                   "weight_ratio": args.weight_ratio if args.workload == "uniform1M_wratio" else None},
        "fwd_bwd_mcells_s": None if fb_ms is None else job_value(fb_ms),
        "fwd_bwd_config": "the timed configuration with tape = 1 (the forward keeps its cells for the adjoint)",
        "fwd_bwd_ms_per_step": fb_ms,
        "e2e": {"value": job_value(e2e_ms), "unit": "Mcells/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "transfers": "vd_copy (SM copies over NVLink-C2C) from and to pinned host buffers"},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": {"bound": "alu", "kernel": "cells_kernel (fused traversal + cull + clip)",
                     "achieved": achieved / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": traffic,
                     "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz",
                     "flop_per_launch": flop, "cells_ms": cms,
                     "flop_source": "main-pass counters of a separate counting build (counters = 1)",
                     "large_cell_pass": {"kernel": "big_cells_kernel", "achieved": achieved_large / 1e12,
                                         "frac": achieved_large / fp32_peak, "flop_per_launch": flop_large,
                                         "ms": lms}},
        "phase_ms": {k: v for k, v in ctx.timings().items() if k.endswith("_ms")},
        "nnz": nnz,
        "counters": {k: cnt[k] for k in ("candidates", "clips", "nodes", "vertex_tests", "new_vertices",
                                         "large_candidates", "large_clips", "large_nodes", "large_vertex_tests",
                                         "large_new_vertices")},
        "status": {k: st[k] for k in ("empty_cells", "overflow_cells", "failed_cells", "fp64_fallbacks",
                                      "fp64_ambiguous", "ambiguous_cells")},
        "cpu_baseline": cpu,
        "forms": forms,
    }
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def main():
    global WEIGHT_RATIO
    args = parse()
    WEIGHT_RATIO = args.weight_ratio
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
