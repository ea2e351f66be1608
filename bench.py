#!/usr/bin/env python
"""Benchmark: weighted-Hamming nearest-neighbour queries/s at 10M descriptors.

Workloads (synthetic, seeded; QUICCI-like 64x64-bit images, 512 B each, see
the generator in paper_2107_03368_gb300/csrc/synth.c):
  main step (tree at scale): 10,000,000 descriptors (10,000 objects x 1,000)
    and 10,000 queries (database descriptors with 30% of their set bits
    cleared and 0.5% of all bits flipped); one step = one Dissimilarity Tree
    search (dt_search, the batched traversal) of the whole batch for the
    top-10 by Eq. 1, against a tree built once beforehand.  Beside it: top-1,
    the per-query traversal, and the GPU brute force (popcount and
    tensor-core kernels) over the same batch.
  partial retrieval: 400 objects x 25,000 descriptors, 1,000 uneven partial
    queries (5.6M query descriptors); votes with threshold 0 (every
    descriptor, one call replayed from a CUDA graph) and threshold 10.
  tensor brute force: 65,536 queries x 20,000,000 descriptors, top-10.
  learned proposal: encoder trained on 2,000,000 (query, exact nearest
    neighbour) pairs over the 20,000,000-descriptor database, inverted file,
    exact rerank; 10,000 queries; recall@1 and queries/s against dt_search.
Plus QUICCI generation on synthetic meshes and insertion into the tree.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (a bounded sample of queries per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "weighted-Hamming NN queries/s @10M descriptors: tree & learned vs GPU brute force"
SEED = 210703368 + 1


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=10_000_000, help="database descriptors")
    p.add_argument("--per-object", type=int, default=1000)
    p.add_argument("--nq", type=int, default=10_000, help="queries per step")
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--cpu-sample", type=int, default=32, help="queries the oracle times")
    p.add_argument("--ref-sample", type=int, default=16,
                   help="queries per step of the reference arm (the CPU oracle)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--bf-steps", type=int, default=1, help="timed brute-force passes")
    p.add_argument("--no-votes", action="store_true", help="skip the partial-retrieval leg")
    p.add_argument("--votes-queries", type=int, default=1000)
    p.add_argument("--no-tensor", action="store_true", help="skip the 65,536 x 20M brute force")
    p.add_argument("--tc-n", type=int, default=20_000_000)
    p.add_argument("--tc-nq", type=int, default=65_536)
    p.add_argument("--tc-steps", type=int, default=2)
    p.add_argument("--no-learned", action="store_true", help="skip the learned proposal leg")
    p.add_argument("--learned-n", type=int, default=20_000_000)
    p.add_argument("--train-pairs", type=int, default=2_000_000,
                   help="(query, exact NN) training pairs, each used once")
    p.add_argument("--train-batch", type=int, default=256)
    p.add_argument("--n-lists", type=int, default=4096, help="inverted-file lists")
    p.add_argument("--target-recall", type=float, default=0.99)
    p.add_argument("--untrained-baseline", type=int, default=1,
                   help="also probe the encoder at its initial weights (1/0)")
    p.add_argument("--insert-n", type=int, default=100_000,
                   help="descriptors of new objects inserted into the tree (0: skip)")
    p.add_argument("--quicci-objects", type=int, default=16,
                   help="synthetic meshes for the QUICCI generation leg (0: skip)")
    p.add_argument("--quicci-subdiv", type=int, default=5,
                   help="mesh resolution: 5 = 10,242 vertices, 20,480 triangles")
    return p.parse_args(argv)


def workload_name(a):
    return ("Dissimilarity Tree search, %d descriptors (%d objects x %d), %d queries, top-%d"
            % (a.n, a.n // a.per_object, a.per_object, a.nq, a.k))


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; queries are sharded, no collective
# on the data path: each rank searches its own batch against its own replica)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, backend):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as td
            td.init_process_group(backend=backend)
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class nvtx:
    """A named NVTX range around a timed call (lets a profiler capture
    exactly that call; free when no profiler is attached)."""

    def __init__(self, name):
        self.name = name

    def __enter__(self):
        import torch
        torch.cuda.nvtx.range_push(self.name)

    def __exit__(self, *exc):
        import torch
        torch.cuda.nvtx.range_pop()
        return False


def aggregate(per_rank_ms, units_per_rank, world):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (per_rank_ms / 1000.0)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "dt_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    """Roofline denominators: the measured copy bandwidth and cuBLAS bf16
    rates (burst, and sustained over seconds) of this GPU type, else the
    stated fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "kind": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0, "kind": "fallback"}


def fp8_peak(sustained):
    """FP8 dense tensor peak: twice the bf16 figure (the nominal ratio); the
    sustained figure for a kernel timed inside seconds-long steps."""
    pk = peaks()
    bf16 = pk["bf16_tflops_sustained"] if sustained else pk["bf16_tflops"]
    return 2.0 * bf16, "FP8 = 2 x %s bf16 %s %.1f TFLOP/s (nominal ratio)" % (
        pk["kind"], "sustained" if sustained else "burst", bf16)


# DRAM traffic of the batched tree search's scan kernel, from one ncu
# capture of a smaller case (the command is in
# profiles/tree_scan_1M_10k.md): at a fixed query batch every split of the
# database is streamed by the CTAs of its wave, so the bytes grow with the
# database rows; scaled to a launch by n.  (109.93 GB read + 0.203 GB written
# at 1M rows; recapture when the scan kernel or its launch shape changes.)
TREE_SCAN_TRAFFIC = {"bytes_per_row": 110135.0, "rows": 1_000_000, "queries": 10_000, "k": 10}


def tree_scan_traffic(a):
    t = TREE_SCAN_TRAFFIC
    if t["bytes_per_row"] is None or (a.nq, a.k) != (t["queries"], t["k"]):
        return None, None
    return t["bytes_per_row"] * a.n, ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                      "tree_scan launch at %d rows x %d queries, top-%d, scaled "
                                      "by rows" % (t["rows"], t["queries"], t["k"]))


# ---------------------------------------------------------------------------
# CPU oracle leg (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_tree_leg(db, q, k, sample, nthreads):
    """Build the oracle's tree (untimed), then time its best-first search on
    `sample` queries.  Returns (queries/s, per-query best-first stats)."""
    import oracle
    tree = oracle.build(db, 32, nthreads=nthreads)
    qs = q[:sample]
    t0 = time.perf_counter()
    _, _, _, st = oracle.tree_search(db, tree, qs, k, nthreads=nthreads)
    dt_s = time.perf_counter() - t0
    return sample / dt_s, st, tree


def cpu_cores():
    return os.cpu_count() or 1


def run_reference(a, dist):
    """The CPU oracle as the reference arm: best-first tree search of a
    bounded sample of the same queries per step, on the host cores."""
    if dist.rank != 0:
        return 0
    from paper_2107_03368_gb300 import synth
    import oracle
    db, _ = synth.database(SEED, a.n, per_object=a.per_object, nthreads=cpu_cores())
    q, _ = synth.queries(SEED, db, max(a.nq, a.cpu_sample))
    nt = cpu_cores()
    tree = oracle.build(db, 32, nthreads=nt)
    per_step = max(1, min(a.ref_sample, a.nq))
    times = []
    for step in range(a.warmup + a.steps):
        lo = (step * per_step) % max(1, q.shape[0] - per_step + 1)
        t0 = time.perf_counter()
        oracle.tree_search(db, tree, q[lo:lo + per_step], a.k, nthreads=nt)
        if step >= a.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    qps = per_step / (ms / 1000.0)
    sample = ("%d queries per step (of the %d-query batch), best-first oracle tree search, "
              "tree built untimed" % (per_step, a.nq))
    line = {
        "impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": workload_name(a), "n_db": a.n, "n_queries": a.nq, "k": a.k,
                   "leaf_size": 32},
        "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": nt, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def timed_steps(fn, steps, warmup, stream, dist, clocks=True):
    """W untimed calls, then K calls bracketed by a barrier and device
    synchronisation, each between CUDA events on `stream`; returns (mean ms
    per call, max over ranks; clock record or None)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    sampler = ClockSampler(dist.local) if clocks else None
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    for i in range(steps):
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    rec = sampler.stop() if sampler else None
    ms = dist.max(sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)) / steps)
    return ms, rec


def run_ours(a, dist):
    import torch
    from paper_2107_03368_gb300 import dt, synth

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    stream = torch.cuda.current_stream(dev)
    nt = cpu_cores()

    db, _ = synth.database(SEED, a.n, per_object=a.per_object, nthreads=nt)
    q_all, _ = synth.queries(SEED + 1000 * dist.rank, db, a.nq, nthreads=nt)
    d_db = torch.from_numpy(db.view(np.int64)).to(dev)
    d_q = torch.from_numpy(q_all.view(np.int64)).to(dev)
    torch.cuda.synchronize()

    t0 = time.perf_counter()
    ix = dt.dt_build(d_db)
    build_s = time.perf_counter() - t0
    info = ix.info()
    # part of the index, like the tree: the tree-ordered rows kept widened
    # for the tensor cores (4 KB per descriptor), built once, untimed
    t0 = time.perf_counter()
    dt.dt_keep_widened(ix, True)
    widen_s = time.perf_counter() - t0

    k = a.k
    out = (torch.empty((a.nq, k), dtype=torch.int32, device=dev),
           torch.empty((a.nq, k), dtype=torch.float32, device=dev), None)

    def step():
        with nvtx("tree_step"):
            dt.dt_search(ix, d_q, k, out=out)

    # the timed steps; the library's own events time its kernels meanwhile
    for _ in range(a.warmup):
        step()
    dt.dt_kernel_timing(True)
    ms, clocks = timed_steps(step, a.steps, 0, stream, dist)
    kern = {name: dt.dt_kernel_time(name) for name in ("tree_scan", "tree_bound", "prewiden")}
    dt.dt_kernel_timing(False)
    dt.dt_sync_status()
    value = aggregate(ms, a.nq, dist.world)
    tree_idx = out[0].clone()

    # traversal statistics of the GPU search (one untimed run)
    _, _, _, gst = dt.dt_search(ix, d_q, k, stats=True)

    # end to end: pinned host queries in, results out, every step
    h_q = torch.from_numpy(q_all.view(np.int64)).pin_memory()
    h_idx = torch.empty((a.nq, k), dtype=torch.int32).pin_memory()
    h_score = torch.empty((a.nq, k), dtype=torch.float32).pin_memory()
    d_qe = torch.empty_like(d_q)

    def e2e_step():
        d_qe.copy_(h_q, non_blocking=True)
        idx_e, score_e, _, _ = dt.dt_search(ix, d_qe, k, out=out)
        h_idx.copy_(idx_e, non_blocking=True)
        h_score.copy_(score_e, non_blocking=True)

    e2e_ms, _ = timed_steps(e2e_step, min(a.steps, 5), 1, stream, dist, clocks=False)
    e2e_value = aggregate(e2e_ms, a.nq, dist.world)

    # the same step captured once in a CUDA graph and replayed
    graph = graph_replay_leg(lambda: dt.dt_search(ix, d_q, k, out=out), out[0], tree_idx, stream)

    # GPU brute force on the same batch (the method's sequential search), both
    # kernels: popcount (path 1) and the tcgen05 overlap contraction (path 2)
    bf = {}
    for name, path in (("popc", 1), ("tensor", 2)):
        ms_bf, same = time_bf(dt, d_db, d_q, k, path, a.bf_steps, stream, tree_idx)
        bf[name] = {"queries_per_s": a.nq / (ms_bf / 1000.0), "ms": ms_bf,
                    "descriptors_scanned_per_s": a.nq * a.n / (ms_bf / 1000.0),
                    "same_indices_as_tree": same}
    bf_best = max(v["queries_per_s"] for v in bf.values())
    pk = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    popc_peak = sms * 16 * pk["sm_max_mhz"] * 1e6 / 1e12            # tera-POPC/s
    popc_ach = a.nq * a.n * 128 / (bf["popc"]["ms"] / 1e3) / 1e12
    bf["popc"]["roofline"] = {"bound": "alu", "achieved": popc_ach, "peak": popc_peak,
                              "unit": "TPOPC32/s", "frac": popc_ach / popc_peak,
                              "peak_kind": "%d SMs x 16 POPC/clk x %.0f MHz" % (sms, pk["sm_max_mhz"])}
    tc_ach = 2.0 * a.nq * a.n * 4096 / (bf["tensor"]["ms"] / 1e3) / 1e12
    tc_peak, tc_kind = fp8_peak(sustained=False)
    bf["tensor"]["roofline"] = {"bound": "tensor", "achieved": tc_ach, "peak": tc_peak,
                                "unit": "TFLOP/s", "frac": tc_ach / tc_peak, "peak_kind": tc_kind,
                                "note": "2 x 4096 FLOP per (query, descriptor); whole call"}

    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": dist.world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "e4m3", "data": "synthetic",
        "config": {"workload": workload_name(a), "n_db": a.n, "n_queries": a.nq, "k": a.k,
                   "leaf_size": 32, "tree_nodes": info["n_nodes"], "tree_depth": info["depth"],
                   "traversal": "batched (pairs of 128-query tiles on CTA pairs x steps of 256 tree-ordered rows)",
                   "l2": "inputs larger than L2 (%.2f GB database)" % (a.n * 512 / 1e9),
                   "parallelism": "queries sharded, tree replicated" if dist.world > 1
                   else "single GPU",
                   "index_widened_copy": "tree-ordered rows kept as FP8 stage images in the index "
                                         "(%.1f GB, built once in %.2f s with the index, untimed)"
                                         % (a.n * 4096 / 1e9, widen_s)},
        "gpu_launches": LAUNCHES_PER_TREE_SEARCH * a.steps,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "queries/s",
                "h2d_bytes_per_step": int(a.nq * 512),
                "d2h_bytes_per_step": int(a.nq * k * 8)},
        "bf_search": bf,
        "tree_vs_bf_speedup": value / dist.world / bf_best,
        "build_s": build_s,
        "graph_replay": graph,
        "gpu_traversal_per_query": {kk: v / a.nq for kk, v in gst.items()},
        "kernels_ms_per_step": {name: v[0] / a.steps for name, v in kern.items()},
        "kernel_launches_per_step": {name: v[1] / a.steps for name, v in kern.items()},
    }
    line["top1"] = top1_leg(a, dt, ix, d_db, d_q, stream)
    line["per_query_traversal"] = per_query_leg(a, dt, ix, d_q, tree_idx, stream)

    # roofline of the dominant kernel, the tree scan: algorithmic work per
    # query = 2 x 4096 FLOP for every descriptor scanned and every node bound
    # of the oracle's best-first search (the method's own work), over the
    # scan kernel's mean launch time measured by the library's events
    scan_ms = kern["tree_scan"][0] / a.steps          # per call (one launch per 96 query tiles)
    peak, peak_kind = fp8_peak(sustained=True)
    traffic, traffic_note = tree_scan_traffic(a)
    roof = {"bound": "tensor", "achieved": None, "peak": peak, "unit": "TFLOP/s", "frac": None,
            "traffic": traffic, "traffic_scaled_from": traffic_note, "peak_kind": peak_kind,
            "kernel": "bf_tc_kernel<MODE_TREE> (tree_scan)", "kernel_ms_per_step": scan_ms}
    if dist.rank == 0 and not a.no_cpu_baseline:
        sample = min(a.cpu_sample, a.nq)
        cpu_qps, ost, _ = oracle_tree_leg(db, q_all, k, sample, nt)
        work_q = float(np.mean(ost[:, 3] + ost[:, 2]))
        flops = 2.0 * 4096 * work_q * a.nq
        achieved = flops / (scan_ms / 1e3) / 1e12
        executed = 2.0 * 4096 * gst["descs_scanned"] / (scan_ms / 1e3) / 1e12
        roof.update(achieved=achieved, frac=achieved / peak, algorithmic_flops=flops,
                    oracle_pairs_per_query=work_q, oracle_sample=sample,
                    executed_upper_tflops=executed)
        line["cpu_baseline"] = {
            "value": cpu_qps, "unit": "queries/s", "cores": nt, "kind": "oracle",
            "sample": "%d of the %d queries, best-first oracle tree search (tree built untimed)"
                      % (sample, a.nq)}
        line["oracle_best_first_per_query"] = {
            "nodes_popped": float(np.mean(ost[:, 0])), "leaves": float(np.mean(ost[:, 1])),
            "descs_scanned": float(np.mean(ost[:, 2])), "bounds": float(np.mean(ost[:, 3]))}
    line["roofline"] = roof
    dt.dt_keep_widened(ix, False)     # the legs below time other work

    if not a.no_votes:
        line["votes"] = votes_leg(a, dev, stream, nt)
    if a.quicci_objects > 0 and dist.rank == 0:
        line["quicci"] = quicci_leg(a, dev, stream, nt)
    if a.insert_n > 0:                # it grows the index
        line["insert"] = insert_leg(a, ix, d_db, d_q, build_s, stream, nt)
    ix.free()
    del d_db, d_q, d_qe
    torch.cuda.empty_cache()
    big = None
    if not a.no_tensor:
        line["tensor_bf"], big = tensor_leg(a, dist, dev, stream, nt)
    if not a.no_learned:
        line["learned"] = learned_leg(a, dist, dev, stream, nt, big)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# kernels of this library launched by one batched dt_search call (one
# batch of query tiles): descent, 3 radix passes x 3 kernels, slots, query
# widening, bound pass, scan, merge; the database widening (2 more) is not
# launched when the index keeps its widened copy, as the headline leg's does
LAUNCHES_PER_TREE_SEARCH = 15


def top1_leg(a, dt, ix, d_db, d_q, stream):
    """Config 1's other k: top-1 of the same batch by the tree and by the
    tensor-core brute force, same indices required."""
    import torch
    out_t = (torch.empty((a.nq, 1), dtype=torch.int32, device=d_q.device),
             torch.empty((a.nq, 1), dtype=torch.float32, device=d_q.device), None)
    out_b = (torch.empty_like(out_t[0]), torch.empty_like(out_t[1]), None)

    def run(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for _ in range(reps):
            fn()
        e.record(stream)
        torch.cuda.synchronize()
        return s.elapsed_time(e) / reps

    ms_t = run(lambda: dt.dt_search(ix, d_q, 1, out=out_t))
    ms_b = run(lambda: dt.bf_search(d_db, d_q, 1, path=2, out=out_b))
    _, _, _, st = dt.dt_search(ix, d_q, 1, stats=True)
    return {"k": 1, "tree_queries_per_s": a.nq / (ms_t / 1e3), "tree_ms": ms_t,
            "bf_tensor_queries_per_s": a.nq / (ms_b / 1e3), "bf_tensor_ms": ms_b,
            "tree_vs_bf_speedup": ms_b / ms_t, "same_indices": bool(torch.equal(out_t[0], out_b[0])),
            "scanned_pairs_frac": st["descs_scanned"] / (a.nq * float(ix.info()["n"]))}


def per_query_leg(a, dt, ix, d_q, tree_idx, stream):
    """The per-query traversal (one warp per query, depth first) on the
    same batch: one pass, same indices required."""
    import torch
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    idx, _, _, _ = dt.dt_search_path(ix, d_q, a.k, 1)
    e.record(stream)
    torch.cuda.synchronize()
    ms = s.elapsed_time(e)
    _, _, _, st = dt.dt_search_path(ix, d_q, a.k, 1, stats=True)
    return {"queries_per_s": a.nq / (ms / 1e3), "ms": ms,
            "same_indices": bool(torch.equal(idx, tree_idx)),
            "per_query": {kk: v / a.nq for kk, v in st.items()}}


def quicci_leg(a, dev, stream, nt):
    """Descriptor generation from meshes (§2.2, §5) and the paper's pipeline
    on its output: QUICCI of every vertex of complete synthetic objects,
    modified QUICCI of every vertex of partial views (triangles facing a
    random direction), a tree over the former, nearest neighbours and votes
    of the latter; the partial views' original QUICCI for comparison."""
    import torch
    import oracle
    from paper_2107_03368_gb300 import dt, synth

    R = 100.0
    n_obj = a.quicci_objects
    meshes = [synth.mesh_object(SEED + 500 + o, a.quicci_subdiv) for o in range(n_obj)]
    parts = [synth.mesh_partial(SEED + 900 + o, m[0], m[1])[:3] for o, m in enumerate(meshes)]
    f32 = lambda x: torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(dev)
    i32 = lambda x: torch.from_numpy(np.ascontiguousarray(x, np.int32)).to(dev)
    d_full = [(f32(v), i32(t), f32(n)) for v, t, n in meshes]
    d_part = [(f32(v), i32(t), f32(n)) for v, t, n in parts]

    def run(dm, modified):
        outs = [torch.empty((v.shape[0], 64), dtype=torch.int64, device=dev) for v, _, _ in dm]
        dt.quicci(dm[0][0], dm[0][1], dm[0][0], dm[0][2], R, modified, out=outs[0])   # warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        with nvtx("quicci_%s" % ("modified" if modified else "full")):
            for (v, t, n), o in zip(dm, outs):
                dt.quicci(v, t, v, n, R, modified, out=o)
        e1.record(stream)
        torch.cuda.synchronize()
        return outs, e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0

    full, s_full, w_full = run(d_full, False)
    part, s_part, w_part = run(d_part, True)
    part_orig, _, _ = run(d_part, False)
    n_full = sum(v.shape[0] for v, _, _ in meshes)
    pairs_full = sum(v.shape[0] * t.shape[0] for v, t, _ in meshes)
    n_part = sum(v.shape[0] for v, _, _ in parts)

    db = torch.cat(full)
    obj = torch.cat([torch.full((v.shape[0],), o, dtype=torch.int32, device=dev)
                     for o, (v, _, _) in enumerate(meshes)])
    off = torch.tensor(np.concatenate([[0], np.cumsum([v.shape[0] for v, _, _ in parts])]),
                       dtype=torch.int64, device=dev)
    ix = dt.dt_build(db)
    truth = torch.arange(n_obj, dtype=torch.int32, device=dev)
    src = torch.cat([torch.full((v.shape[0],), o, dtype=torch.int32, device=dev)
                     for o, (v, _, _) in enumerate(parts)])
    pipeline = {}
    for name, q in (("modified", part), ("original", part_orig)):
        qd = torch.cat(q)
        _, winner, _ = dt.retrieve_objects(ix, obj, n_obj, qd, off, 0, 1)
        nn, _, _ = dt.bf_search(db, qd, 1, path=2)
        nn_obj = obj[nn[:, 0].long()]
        pipeline[name] = {"objects_identified": int((winner == truth).sum()),
                          "nn_from_source_object": float((nn_obj == src).float().mean())}
    ix.free()

    # the oracle on a bounded sample: 48 vertices of the first object
    v0, t0_, n0 = meshes[0]
    pick = np.linspace(0, v0.shape[0] - 1, 48).astype(np.int64)
    c0 = time.perf_counter()
    ref = oracle.quicci(v0, t0_, v0[pick], n0[pick], R, False, nthreads=nt)
    cpu_s = time.perf_counter() - c0
    same = int((full[0][pick].cpu().numpy().view(np.uint64) == ref).all(axis=1).sum())

    # roofline on the method's own arithmetic: every triangle whose bounding
    # sphere reaches a point's support cylinder is moved into the point's
    # frame (27 FP32 operations) and every layer segment is cut and measured
    # (53: two interpolations, three distances, the closest point, the circle
    # indices); the culling that finds them is not counted.  Counts per point
    # are taken from 32 points of each of the first 4 objects (numpy
    # geometry of the input, not the method's result); peak = FP32 lanes x
    # clock, an FMA counted as one operation
    srng = np.random.default_rng(SEED)
    zl = -R + (2 * np.arange(64) + 1) * R / 64
    per_point = []
    for v, t, n in meshes[:4]:
        tri = v[t].astype(np.float64)
        cen = tri.mean(1)
        rad = np.sqrt(((tri - cen[:, None, :]) ** 2).sum(-1)).max(1)
        for j in srng.integers(0, v.shape[0], 32):
            pp, nn = v[j].astype(np.float64), n[j] / np.linalg.norm(n[j])
            rc = cen - pp
            zc = rc @ nn
            rr = np.linalg.norm(rc - zc[:, None] * nn[None, :], axis=1) - rad
            reach = (np.abs(zc) - rad <= R) & (rr <= R)
            z = (tri[reach] - pp) @ nn
            segs = ((z.min(1)[:, None] < zl[None, :]) & (z.max(1)[:, None] >= zl[None, :])).sum()
            per_point.append(27.0 * reach.sum() + 53.0 * segs)
    ops_per_desc = float(np.mean(per_point))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pk = peaks()
    fp32_peak = sms * 128 * pk["sm_max_mhz"] * 1e6
    achieved = n_full * ops_per_desc / s_full
    return {"objects": n_obj, "vertices_per_object": int(meshes[0][0].shape[0]),
            "triangles_per_object": int(meshes[0][1].shape[0]), "support_radius": R,
            "complete": {"descriptors": n_full, "seconds": s_full, "wall_s": w_full,
                         "descriptors_per_s": n_full / s_full,
                         "point_triangle_pairs_per_s": pairs_full / s_full},
            "partial_modified": {"descriptors": n_part, "seconds": s_part, "wall_s": w_part,
                                 "descriptors_per_s": n_part / s_part},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak / 1e12,
                         "unit": "TFLOP/s (FP32, FMA = 1)", "frac": achieved / fp32_peak,
                         "fp32_ops_per_descriptor": ops_per_desc,
                         "peak_kind": "%d SMs x 128 FP32 lanes x %.0f MHz" % (sms, pk["sm_max_mhz"])},
            "pipeline": pipeline,
            "cpu_baseline": {"value": 48 / cpu_s, "unit": "descriptors/s", "cores": nt,
                             "kind": "oracle", "sample": "48 vertices of the first object",
                             "identical_descriptors": same}}


def insert_leg(a, ix, d_db, d_q, build_s, stream, nt):
    """Incremental insertion: descriptors of new objects go into the built
    tree.  A slice of the batch's queries is searched before and after (the
    same queries), and the result after is checked against the tensor-core
    brute force over all descriptors."""
    import torch
    from paper_2107_03368_gb300 import dt, synth

    nq = min(a.nq, 2000)
    k = a.k
    dq = d_q[:nq].contiguous()

    def timed_search():
        dt.dt_search(ix, dq, k)             # warm-up
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        idx, score, _, _ = dt.dt_search(ix, dq, k)
        s1.record(stream)
        torch.cuda.synchronize()
        return nq / (s0.elapsed_time(s1) / 1e3), idx, score

    qps_before, _, _ = timed_search()
    new, _ = synth.database(SEED + 77, a.insert_n, per_object=a.per_object, nthreads=nt)
    d_new = torch.from_numpy(new.view(np.int64)).to(d_db.device)
    before = ix.info()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    with nvtx("insert"):
        dt.dt_insert(ix, d_new)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ev_s = e0.elapsed_time(e1) / 1e3
    after = ix.info()

    qps_after, t_idx, t_score = timed_search()
    d_all = torch.cat([d_db, d_new])
    c_idx, c_score, _ = dt.bf_search(d_all, dq, k, path=2)
    same = bool(torch.equal(t_idx, c_idx) and torch.equal(t_score, c_score))
    del d_all
    rows_moved = before["n"] + a.insert_n
    return {"inserted": a.insert_n, "n_before": before["n"], "n_after": after["n"],
            "seconds": wall, "seconds_cuda_events": ev_s,
            "descriptors_per_s": a.insert_n / wall,
            "full_build_s_before": build_s, "vs_full_build": wall / build_s,
            "nodes_before": before["n_nodes"], "nodes_after": after["n_nodes"],
            "depth_before": before["depth"], "depth_after": after["depth"],
            "tree_bytes_moved_per_s": rows_moved * 516 * 2 / wall,
            "search": {"queries": nq, "queries_per_s_before": qps_before,
                       "queries_per_s_after": qps_after,
                       "after_same_as_tensor_bf_over_all": same}}


def graph_replay_leg(fn, result, ref, stream):
    """Capture fn (stream-ordered, scratch from the stream-ordered allocator)
    in a CUDA graph, replay it, and time one replay against the direct call's
    result."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        fn()
    result.fill_(-1)
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    with nvtx("graph_replay"):
        g.replay()
    e.record(stream)
    torch.cuda.synchronize()
    same = bool(torch.equal(result, ref))
    del g
    return {"ms": s.elapsed_time(e), "same_indices_as_direct": same}


def time_bf(dt, d_db, d_q, k, path, steps, stream, ref_idx):
    """Mean CUDA-event time of one bf_search pass over the batch, and whether
    its indices equal ref_idx."""
    import torch
    out = (torch.empty_like(ref_idx), torch.empty(ref_idx.shape, dtype=torch.float32,
                                                  device=ref_idx.device), None)
    dt.bf_search(d_db, d_q, k, out=out, path=path)          # warm
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    with nvtx("bf_path%d" % path):
        for _ in range(steps):
            dt.bf_search(d_db, d_q, k, out=out, path=path)
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e) / steps, bool(torch.equal(out[0], ref_idx))


def learned_leg(a, dist, dev, stream, nt, big):
    """Learned proposal on the 20,000,000-descriptor database: train the
    encoder on (query, exact nearest neighbour) pairs from the GPU brute
    force, each pair used once; build the inverted file; find the fewest
    probed lists whose exactly reranked top-1 reaches the target recall@1
    against the exact top-1 and time the search there; compare with the
    plain tree search and the tensor-core brute force, and run the exact
    mode: the proposal's answers as the warm start of the batched tree
    search (identical results to the exact search)."""
    import torch
    import oracle
    from paper_2107_03368_gb300 import dt, learned, synth
    n = a.learned_n
    if big is not None and big["n"] == n:
        db, d_db, seed = big["db"], big["d_db"], big["seed"]
    else:
        seed = SEED + 2
        db, _ = synth.database(seed, n, per_object=a.per_object, nthreads=nt)
        d_db = torch.from_numpy(db.view(np.int64)).to(dev)
    q, _ = synth.queries(seed + 7 + 1000 * dist.rank, db, a.nq, nthreads=nt)
    d_q = torch.from_numpy(q.view(np.int64)).to(dev)
    nq = a.nq

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for _ in range(reps):
            r = fn()
        e.record(stream)
        torch.cuda.synchronize()
        return s.elapsed_time(e) / reps, r

    ms_bf, (exact, _, _) = timed(lambda: dt.bf_search(d_db, d_q, 1, path=2))
    exact = exact[:, 0].clone()
    ix = dt.dt_build(d_db)
    dt.dt_keep_widened(ix, True)       # as in the headline leg; released during training
    ms_tree, (t_idx, _, _, _) = timed(lambda: dt.dt_search(ix, d_q, 1))
    tree_same = bool(torch.equal(t_idx[:, 0], exact))
    dt.dt_keep_widened(ix, False)

    enc = learned.Encoder(seed=1)
    round_q = 16384

    def make_queries(r):            # training queries: disjoint seeds from the timed batch
        return synth.queries(seed + 5_000_000 + 1000 * dist.rank + r, db, round_q, nthreads=nt)[0]

    steps = max(1, a.train_pairs // a.train_batch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = learned.train(enc, d_db, make_queries, steps=steps, batch=a.train_batch, lr=1e-3,
                         tau=0.05, epochs_per_round=1)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ivf = learned.IVF(enc, d_db, n_lists=a.n_lists, iters=4)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0

    def run(probe, reps):
        return timed(lambda: ivf.search(d_q, 1, probe, with_scanned=True), reps)

    sweep, chosen = [], None
    for probe in [p for p in (1, 2, 4, 8, 16, 24, 32, 48, 64, 96, 128, 192, 256) if p <= a.n_lists]:
        ms, (idx, _, scanned) = run(probe, 1)
        rec = float((idx[:, 0] == exact).float().mean().item())
        sweep.append({"n_probe": probe, "recall_at_1": rec, "ms": ms,
                      "scanned_per_query": float(scanned.float().mean().item())})
        if rec >= a.target_recall:
            chosen = probe
            break
    out = {"workload": "%d descriptors, %d queries, top-1" % (n, nq),
           "train_pairs": steps * a.train_batch, "train_steps": steps,
           "train_s": train_s, "loss_first": hist[0][1], "loss_last": hist[-1][1],
           "ivf_build_s": build_s, "n_lists": a.n_lists, "sweep": sweep,
           "target_recall_at_1": a.target_recall,
           "plain_tree": {"queries_per_s": nq / (ms_tree / 1e3), "ms": ms_tree,
                          "same_indices_as_brute_force": tree_same},
           "bf_tensor": {"queries_per_s": nq / (ms_bf / 1e3), "ms": ms_bf}}
    if chosen is not None:
        ms, (idx, _, scanned) = run(chosen, 3)
        rec = float((idx[:, 0] == exact).float().mean().item())
        scanned = float(scanned.float().mean().item())
        qps = nq / (ms / 1e3)
        peak, peak_kind = fp8_peak(sustained=False)
        tf = 2.0 * 4096 * scanned * nq / (ms / 1e3) / 1e12
        out.update(n_probe=chosen, recall_at_1=rec, queries_per_s=qps, ms=ms,
                   scanned_per_query=scanned, speedup_vs_tree=qps / (nq / (ms_tree / 1e3)),
                   speedup_vs_bf=qps / (nq / (ms_bf / 1e3)),
                   scan_roofline={"bound": "tensor", "achieved": tf, "peak": peak,
                                  "unit": "TFLOP/s", "frac": tf / peak, "peak_kind": peak_kind,
                                  "traffic": None,
                                  "note": "2 x 4096 FLOP per (query, scanned row); time of the "
                                          "whole search call (embedding, probing, scan, merge)"})
        if a.untrained_baseline:
            enc0 = learned.Encoder(seed=1)
            ivf0 = learned.IVF(enc0, d_db, n_lists=a.n_lists, iters=4)
            idx0, _, _ = ivf0.search(d_q, 1, chosen)
            out["untrained_recall_at_1_same_probes"] = float((idx0[:, 0] == exact).float().mean().item())
            ivf0.free()
            enc0.free()
    # exact mode: the proposal's top-1 at a few probes caps the batched tree
    # search of every query from the start; the result is the exact one
    seeds, _, _ = ivf.search(d_q, 1, 8)
    dt.dt_keep_widened(ix, True)
    ms_ex, (e_idx, _, _, _) = timed(lambda: dt.dt_search_seeded(ix, d_q, 1, seeds), 3)
    _, _, _, est = dt.dt_search_seeded(ix, d_q, 1, seeds, stats=True)
    _, _, _, pst = dt.dt_search(ix, d_q, 1, stats=True)
    dt.dt_keep_widened(ix, False)
    out["exact_mode"] = {"n_probe_for_caps": 8, "queries_per_s": nq / (ms_ex / 1e3), "ms": ms_ex,
                         "same_indices_as_brute_force": bool(torch.equal(e_idx[:, 0], exact)),
                         "speedup_vs_bf": ms_bf / ms_ex, "speedup_vs_plain_tree": ms_tree / ms_ex,
                         "scanned_pairs_frac": est["descs_scanned"] / (nq * float(n)),
                         "plain_tree_scanned_pairs_frac": pst["descs_scanned"] / (nq * float(n))}
    if dist.rank == 0 and not a.no_cpu_baseline:
        sample = 4
        t0 = time.perf_counter()
        o_idx, _, _ = oracle.bf_topk(db, q[:sample], 1, nthreads=nt)
        cpu_s = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": sample / cpu_s, "unit": "queries/s", "cores": nt,
                               "kind": "oracle",
                               "sample": "%d of the %d queries, oracle exact top-1 (brute force), "
                                         "the answer the proposal must reach" % (sample, nq)}
        out["oracle_check_same_nn"] = bool(np.array_equal(
            exact[:sample].cpu().numpy().view(np.uint32).astype(np.int64), o_idx[:, 0]))
    ivf.free()
    enc.free()
    ix.free()
    return out


def votes_leg(a, dev, stream, nt):
    """Batched partial-object retrieval (§3): 400 objects x 25,000
    descriptors, 1,000 uneven partial queries (contiguous 5-40% of one
    object, clamped to 500-10,000 descriptors).  Threshold 10 (the paper's)
    over all queries in one call; threshold 0 (every descriptor votes) over
    all queries in one call captured in a CUDA graph and replayed."""
    import torch
    import oracle
    from paper_2107_03368_gb300 import dt, synth
    seed = SEED + 1                      # the partial-retrieval workload's own seed
    n_obj, per = 400, 25_000
    db, obj = synth.database(seed, n_obj * per, per_object=per, nthreads=nt)
    qd, off, qobj = synth.partial_queries(seed, db, n_obj, per, a.votes_queries, nthreads=nt)
    d_db = torch.from_numpy(db.view(np.int64)).to(dev)
    ix = dt.dt_build(d_db)
    d_obj = torch.from_numpy(obj.view(np.int32)).to(dev)
    d_qd = torch.from_numpy(qd.view(np.int64)).to(dev)
    d_off = torch.from_numpy(off).to(dev)
    nq, total = a.votes_queries, int(qd.shape[0])
    out = {"workload": "%d objects x %d descriptors, %d partial queries, %d query descriptors"
                       % (n_obj, per, nq, total), "engine": "0 (automatic / autotuned)"}

    def timed(fn):
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        r = fn()
        e.record(stream)
        torch.cuda.synchronize()
        return s.elapsed_time(e), r

    with nvtx("votes_t10"):
        ms, (votes, winner, consumed) = timed(lambda: dt.retrieve_objects(
            ix, d_obj, n_obj, d_qd, d_off, 10, seed))
    w = winner.cpu().numpy()
    out["threshold_10"] = {
        "ms": ms, "partial_queries_per_s": nq / (ms / 1e3),
        "descriptors_consumed": int(consumed.sum().item()),
        "winner_is_source_object": float(np.mean(w == qobj))}

    # autotune the threshold-0 call on one partial query (engine, engine 1's
    # resident blocks, the batched search's launch); engine 0 then uses it
    t0 = time.perf_counter()
    tune = dt.dt_autotune_retrieve(ix, d_obj, n_obj, d_qd[: int(off[1])], d_off[:2].contiguous(), 0)
    out["autotune_threshold_0"] = {"sample": "1 partial query (%d descriptors)" % int(off[1]),
                                   "seconds": time.perf_counter() - t0,
                                   "engine": tune["retrieve_engine"],
                                   "engine1_blocks_per_sm": tune["retrieve_blocks_per_sm"],
                                   "batched_splits": tune["tree_tc_splits"],
                                   "batched_prewiden": tune["tree_tc_prewiden"],
                                   "candidates_timed": tune["candidates_timed"]}

    # threshold 0: one call over all queries, captured and replayed once
    vo = (torch.empty((nq, n_obj), dtype=torch.int32, device=dev),
          torch.empty(nq, dtype=torch.int32, device=dev),
          torch.empty(nq, dtype=torch.int64, device=dev))
    call = lambda: dt.retrieve_objects(ix, d_obj, n_obj, d_qd, d_off, 0, seed, out=vo)
    small = d_off[:2].contiguous()                    # warm the code paths, not timed
    dt.retrieve_objects(ix, d_obj, n_obj, d_qd[: int(off[1])], small, 0, seed)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        call()
    with nvtx("votes_t0_graph"):
        ms0, _ = timed(g.replay)
    dt.dt_sync_status()
    del g
    v0 = vo[0].cpu().numpy().view(np.uint32)
    sizes = np.diff(off)
    checks = {"every_descriptor_voted": bool(np.array_equal(v0.sum(1), sizes)),
              "winner_is_source_object": float(np.mean(vo[1].cpu().numpy() == qobj))}
    same = True
    for j in (0, nq // 2, nq - 1):       # sampled queries against brute-force neighbours
        nn_j = dt.bf_search(d_db, d_qd[int(off[j]):int(off[j + 1])], 1, path=2)[0]
        nn_j = nn_j.cpu().numpy().view(np.uint32).astype(np.int64)[:, 0]
        same = same and bool(np.array_equal(v0[j], np.bincount(obj[nn_j], minlength=n_obj)))
    checks["sampled_votes_equal_brute_force"] = same
    out["threshold_0"] = {"ms": ms0, "graph_replay": True,
                          "partial_queries_per_s": nq / (ms0 / 1e3),
                          "descriptor_nn_per_s": total / (ms0 / 1e3), "checks": checks}
    # algorithmic work: the oracle's best-first search (top-1) of a sample of
    # query descriptors, per descriptor; CPU baseline from the same sample
    m = 16
    pick = np.linspace(0, total - 1, m).astype(np.int64)
    otree = oracle.build(db, 32, nthreads=nt)
    t0 = time.perf_counter()
    o_idx, _, _, ost = oracle.tree_search(db, otree, qd[pick], 1, nthreads=nt)
    cpu_s = time.perf_counter() - t0
    work_d = float(np.mean(ost[:, 2] + ost[:, 3]))
    peak, peak_kind = fp8_peak(sustained=True)
    ach = 2.0 * 4096 * work_d * total / (ms0 / 1e3) / 1e12
    out["threshold_0"]["roofline"] = {
        "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
        "peak_kind": peak_kind, "traffic": None,
        "note": "2 x 4096 FLOP per descriptor scanned or node bounded by the oracle's best-first "
                "top-1 search (%.0f per query descriptor, %d-descriptor sample), over the whole "
                "replayed call" % (work_d, m)}
    out["threshold_0"]["cpu_baseline"] = {
        "value": m / cpu_s, "unit": "descriptor NN/s", "cores": nt, "kind": "oracle",
        "sample": "%d query descriptors spread over the batch, best-first oracle tree search, "
                  "top-1 (tree built untimed)" % m}
    g_nn = dt.dt_search(ix, d_qd[torch.from_numpy(pick).to(dev)].contiguous(), 1)[0]
    out["threshold_0"]["oracle_sample_same_nn"] = bool(np.array_equal(
        g_nn.cpu().numpy().view(np.uint32).astype(np.int64)[:, 0], o_idx[:, 0]))
    del otree

    # object distance scores (§6.4) of 20 query objects against every object
    m = 20
    sub_off = d_off[: m + 1].contiguous()
    n_desc = int(off[m])
    torch.cuda.synchronize()
    ms_s, sc = timed(lambda: dt.object_scores(d_db, d_obj, n_obj, d_qd[:n_desc], sub_off))
    best = sc.argmin(dim=1).cpu().numpy()
    out["object_scores_sample"] = {
        "partial_queries": m, "query_descriptors": n_desc, "objects": n_obj, "ms": ms_s,
        "pairs_per_s": n_desc * (n_obj * per) / (ms_s / 1e3),
        "best_object_is_source": float(np.mean(best == qobj[:m]))}
    ix.free()
    return out


def tensor_leg(a, dist, dev, stream, nt):
    """Large-batch brute force: 65,536 queries against 20,000,000 descriptors
    on the tensor cores (bf_search path 2), the popcount kernel on a sample
    of the queries, both checked against each other and, on a few queries,
    the oracle.  Returns (the leg's record, the database for the learned
    leg)."""
    import torch
    import oracle
    from paper_2107_03368_gb300 import dt, synth
    seed = SEED + 2                              # the 20M workloads' own seed
    n, nq, k = a.tc_n, a.tc_nq, a.k
    db, _ = synth.database(seed, n, per_object=a.per_object, nthreads=nt)
    q, _ = synth.queries(seed + 1000 * dist.rank, db, nq, nthreads=nt)
    d_db = torch.from_numpy(db.view(np.int64)).to(dev)
    d_q = torch.from_numpy(q.view(np.int64)).to(dev)
    out = (torch.empty((nq, k), dtype=torch.int32, device=dev),
           torch.empty((nq, k), dtype=torch.float32, device=dev), None)

    def step():
        with nvtx("bf_path2_large"):
            dt.bf_search(d_db, d_q, k, out=out, path=2)

    step()
    dt.dt_kernel_timing(True)
    ms, clocks = timed_steps(step, a.tc_steps, 0, stream, dist)
    scan_ms, scan_n = dt.dt_kernel_time("tc_scan")
    pre_ms, pre_n = dt.dt_kernel_time("prewiden")
    dt.dt_kernel_timing(False)
    dt.dt_sync_status()

    # popcount kernel on a sample of the queries; same indices as the tensor kernel
    m = min(2048, nq)
    p_out = (torch.empty((m, k), dtype=torch.int32, device=dev),
             torch.empty((m, k), dtype=torch.float32, device=dev), None)
    dt.bf_search(d_db, d_q[:m], k, out=p_out, path=1)
    torch.cuda.synchronize()
    ps, pe = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ps.record(stream)
    dt.bf_search(d_db, d_q[:m], k, out=p_out, path=1)
    pe.record(stream)
    torch.cuda.synchronize()
    popc_ms = ps.elapsed_time(pe)

    peak, peak_kind = fp8_peak(sustained=True)
    kern_ms = scan_ms / a.tc_steps                    # per pass (one launch per 96 query tiles)
    tf = 2.0 * nq * n * 4096 / (kern_ms / 1e3) / 1e12
    rec = {"workload": "tensor-core brute force, %d descriptors x %d queries, top-%d" % (n, nq, k),
           "queries_per_s": aggregate(ms, nq, dist.world), "ms_per_pass": ms, "passes": a.tc_steps,
           "clocks": clocks, "dtype": "e4m3",
           "l2": "inputs larger than L2 (%.2f GB database)" % (n * 512 / 1e9),
           "kernels_ms_per_pass": {"tc_scan": kern_ms, "prewiden": pre_ms / a.tc_steps},
           "tc_scan_launches_per_pass": scan_n / a.tc_steps,
           "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                        "frac": tf / peak, "traffic": None, "peak_kind": peak_kind,
                        "kernel": "bf_tc_kernel<MODE_PLAIN> (tc_scan)",
                        "note": "2 x 4096 FLOP per (query, descriptor) over the scan kernel's "
                                "event time"},
           "popc_sample": {"queries": m, "ms": popc_ms, "queries_per_s": m / (popc_ms / 1e3),
                           "same_indices_as_tensor": bool(torch.equal(p_out[0], out[0][:m]))}}
    if dist.rank == 0 and not a.no_cpu_baseline:
        sample = 4
        t0 = time.perf_counter()
        o_idx, o_score, _ = oracle.bf_topk(db, q[:sample], k, nthreads=nt)
        cpu_s = time.perf_counter() - t0
        g_idx = out[0][:sample].cpu().numpy().view(np.uint32).astype(np.int64)
        g_score = out[1][:sample].cpu().numpy().astype(np.float64)
        rec["oracle_check"] = {
            "queries": sample, "same_indices": bool(np.array_equal(g_idx, o_idx)),
            "max_score_rel_err": float(np.max(np.abs(g_score - o_score) / np.maximum(o_score, 1e-300)))}
        rec["cpu_baseline"] = {"value": sample / cpu_s, "unit": "queries/s", "cores": nt,
                               "kind": "oracle",
                               "sample": "%d of the %d queries, oracle brute force" % (sample, nq)}
    del d_q, out
    return rec, {"n": n, "db": db, "d_db": d_db, "seed": seed}


def main(argv=None):
    a = parse_args(argv)
    if a.impl == "reference":
        dist = Dist("gloo")
        try:
            return run_reference(a, dist)
        finally:
            dist.close()
    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    dist = Dist("nccl")
    try:
        return run_ours(a, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    sys.exit(main())
