#!/usr/bin/env python
"""Benchmark: weighted-Hamming nearest-neighbour queries/s at 10M descriptors.

Workload (synthetic, seeded): 10,000,000 QUICCI-like descriptors (64x64 bits,
512 B each; 10,000 objects x 1,000 descriptors drawn from 50 curve sets per
object) and 10,000 queries made from database descriptors with 30% of their
set bits cleared and 0.5% of all bits flipped.  One step = one Dissimilarity
Tree search (dt_search) of the whole 10,000-query batch for the top-10 by
Eq. 1, against a tree built once beforehand.  Beside it: the GPU brute force
(bf_search, popcount and tensor-core kernels) over the same batch, and the
learned proposal (encoder trained on the GPU, inverted file, exact rerank)
at the fewest probed lists that reach recall@1 >= 0.99.

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
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=10_000_000, help="database descriptors")
    p.add_argument("--per-object", type=int, default=1000)
    p.add_argument("--nq", type=int, default=10_000, help="queries per step")
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--cpu-sample", type=int, default=32, help="queries the oracle times")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--bf-steps", type=int, default=1, help="timed brute-force passes")
    p.add_argument("--no-learned", action="store_true", help="skip the learned proposal leg")
    p.add_argument("--no-votes", action="store_true", help="skip the partial-retrieval leg")
    p.add_argument("--votes-queries", type=int, default=1000)
    p.add_argument("--votes-sample", type=int, default=20,
                   help="partial queries counted in full (threshold 0)")
    p.add_argument("--train-steps", type=int, default=4000, help="encoder training steps")
    p.add_argument("--train-epochs", type=int, default=2,
                   help="passes over each round of 16,384 (query, exact NN) pairs")
    p.add_argument("--train-batch", type=int, default=256)
    p.add_argument("--n-lists", type=int, default=4096, help="inverted-file lists")
    p.add_argument("--target-recall", type=float, default=0.99)
    p.add_argument("--untrained-baseline", type=int, default=1,
                   help="also sweep the encoder at its initial weights (1/0)")
    p.add_argument("--insert-n", type=int, default=100_000,
                   help="descriptors of new objects inserted into the tree (0: skip)")
    p.add_argument("--quicci-objects", type=int, default=16,
                   help="synthetic meshes for the QUICCI generation leg (0: skip)")
    p.add_argument("--quicci-subdiv", type=int, default=5,
                   help="mesh resolution: 5 = 10,242 vertices, 20,480 triangles")
    p.add_argument("--workload", choices=["tree", "tensor-bf"], default="tree",
                   help="tree: the tree-search step (default); tensor-bf: the large-batch "
                        "brute force, 65,536 queries x 20,000,000 descriptors")
    p.add_argument("--tc-n", type=int, default=20_000_000)
    p.add_argument("--tc-nq", type=int, default=65_536)
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
    rate of this GPU type, else the stated fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "kind": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0,
                "kind": "fallback"}


# DRAM traffic of one dt_search launch on this workload (10M descriptors,
# 10,000 queries, top-10), dram__bytes_read.sum + dram__bytes_write.sum from
# one ncu capture of this script's timed launch.  It describes the kernel
# source it was captured from; any change to that source voids it.
DT_SEARCH_TRAFFIC = {"bytes": 51.47e12 + 0.955e12,
                     "sources_sha1": "7acd789514359f3e9a9bb4cd41b0d652a5257a52"}
DT_SEARCH_SOURCES = ("paper_2107_03368_gb300/csrc/dt_search.cu",
                     "paper_2107_03368_gb300/csrc/dt_traverse.cuh")


def dt_search_sources_sha1():
    import hashlib
    h = hashlib.sha1()
    for rel in DT_SEARCH_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def dt_search_traffic(a):
    """Captured traffic per launch, or None when it does not apply."""
    if (a.n, a.nq, a.k) != (10_000_000, 10_000, 10) or DT_SEARCH_TRAFFIC["bytes"] is None:
        return None
    if DT_SEARCH_TRAFFIC["sources_sha1"] != dt_search_sources_sha1():
        return None
    return DT_SEARCH_TRAFFIC["bytes"]


def measured_peaks():
    p = peaks()
    return p["hbm_gbs"], p["kind"]


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
    per_step = max(1, min(a.cpu_sample, a.nq))
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

    k = a.k
    out = (torch.empty((a.nq, k), dtype=torch.int32, device=dev),
           torch.empty((a.nq, k), dtype=torch.float32, device=dev), None)

    def step():
        dt.dt_search(ix, d_q, k, out=out)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(dist.local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for i in range(a.steps):
        starts[i].record(stream)
        with nvtx("tree_step"):
            step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    dt.dt_sync_status()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = dist.max(sum(step_ms) / len(step_ms))
    value = aggregate(ms, a.nq, dist.world)
    tree_idx = out[0].clone()

    # traversal statistics of the GPU search (one untimed run)
    _, _, _, gst = dt.dt_search(ix, d_q, k, stats=True)

    # end to end: pinned host queries in, results out, every step
    h_q = torch.from_numpy(q_all.view(np.int64)).pin_memory()
    h_idx = torch.empty((a.nq, k), dtype=torch.int32).pin_memory()
    h_score = torch.empty((a.nq, k), dtype=torch.float32).pin_memory()
    d_qe = torch.empty_like(d_q)
    e_s = torch.cuda.Event(enable_timing=True)
    e_e = torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    e_s.record(stream)
    for _ in range(a.steps):
        d_qe.copy_(h_q, non_blocking=True)
        idx_e, score_e, _, _ = dt.dt_search(ix, d_qe, k, out=out)
        h_idx.copy_(idx_e, non_blocking=True)
        h_score.copy_(score_e, non_blocking=True)
    e_e.record(stream)
    torch.cuda.synchronize()
    e2e_ms = dist.max(e_s.elapsed_time(e_e) / a.steps)
    e2e_value = aggregate(e2e_ms, a.nq, dist.world)

    # the same step captured once in a CUDA graph and replayed
    graph = graph_replay_leg(lambda: dt.dt_search(ix, d_q, k, out=out), out[0], tree_idx,
                             stream)

    # GPU brute force on the same batch (the method's sequential search), both
    # kernels: popcount (path 1) and the tcgen05 overlap contraction (path 2)
    bf = {}
    for name, path in (("popc", 1), ("tensor", 2)):
        ms_bf, same = time_bf(dt, d_db, d_q, k, path, a.bf_steps, stream, tree_idx)
        bf[name] = {"queries_per_s": a.nq / (ms_bf / 1000.0), "ms": ms_bf,
                    "descriptors_scanned_per_s": a.nq * a.n / (ms_bf / 1000.0),
                    "same_indices_as_tree": same}
    bf_best = max(v["queries_per_s"] for v in bf.values())
    # their own rooflines: the popcount kernel is bound by the POPC pipe
    # (16 POPC per SM per clock), the tensor kernel by the FP8 tensor rate
    pk = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    popc_peak = sms * 16 * pk["sm_max_mhz"] * 1e6 / 1e12            # tera-POPC/s
    popc_ach = a.nq * a.n * 128 / (bf["popc"]["ms"] / 1e3) / 1e12
    bf["popc"]["roofline"] = {"bound": "alu", "achieved": popc_ach, "peak": popc_peak,
                              "unit": "TPOPC32/s", "frac": popc_ach / popc_peak,
                              "peak_kind": "%d SMs x 16 POPC/clk x %.0f MHz" % (sms, pk["sm_max_mhz"])}
    tc_ach = 2.0 * a.nq * a.n * 4096 / (bf["tensor"]["ms"] / 1e3) / 1e12
    tc_peak = 2.0 * pk["bf16_tflops"]
    bf["tensor"]["roofline"] = {"bound": "tensor", "achieved": tc_ach, "peak": tc_peak,
                                "unit": "TFLOP/s", "frac": tc_ach / tc_peak,
                                "peak_kind": "FP8 = 2 x %s bf16 %.1f TFLOP/s (nominal ratio)"
                                             % (pk["kind"], pk["bf16_tflops"])}

    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": dist.world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(a), "n_db": a.n, "n_queries": a.nq, "k": a.k,
                   "leaf_size": 32, "tree_nodes": info["n_nodes"], "tree_depth": info["depth"],
                   "l2": "inputs larger than L2 (%.2f GB database)" % (a.n * 512 / 1e9),
                   "parallelism": "queries sharded, tree replicated" if dist.world > 1
                   else "single GPU"},
        "gpu_launches": a.steps,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "queries/s",
                "h2d_bytes_per_step": int(a.nq * 512),
                "d2h_bytes_per_step": int(a.nq * k * 8)},
        "bf_search": bf,
        "tree_vs_bf_speedup": value / dist.world / bf_best,
        "build_s": build_s,
        "graph_replay": graph,
        "gpu_traversal_per_query": {kk: v / a.nq for kk, v in gst.items()},
        "descriptors_scanned_per_s": gst["descs_scanned"] / (ms / 1000.0) * dist.world,
    }

    if not a.no_votes:
        line["votes"] = votes_leg(a, dev, stream, nt)
    if not a.no_learned:
        line["learned"] = learned_leg(a, dist, d_db, d_q, db, value / dist.world, bf_best, stream,
                                      ix, tree_idx)
    if a.quicci_objects > 0 and dist.rank == 0:
        line["quicci"] = quicci_leg(a, dev, stream, nt)
    if a.insert_n > 0:                # last: it grows the index
        line["insert"] = insert_leg(a, ix, d_db, d_q, build_s, stream, nt)

    # roofline of the dominant kernel (dt_search): algorithmic bytes per query =
    # 512 B x (bounds evaluated + descriptors scanned) of the oracle's best-first
    # search, measured on the cpu_baseline sample
    peak, peak_kind = measured_peaks()
    roof = {"bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
            "traffic": dt_search_traffic(a), "peak_kind": peak_kind}
    if dist.rank == 0 and not a.no_cpu_baseline:
        sample = min(a.cpu_sample, a.nq)
        cpu_qps, ost, _ = oracle_tree_leg(db, q_all, k, sample, nt)
        bytes_per_q = 512.0 * float(np.mean(ost[:, 3] + ost[:, 2]))
        achieved = bytes_per_q * a.nq / (ms / 1000.0) / 1e9
        roof.update(achieved=achieved, frac=achieved / peak,
                    bytes_per_query=bytes_per_q, oracle_sample=sample)
        line["cpu_baseline"] = {
            "value": cpu_qps, "unit": "queries/s", "cores": nt, "kind": "oracle",
            "sample": "%d of the %d queries, best-first oracle tree search (tree built untimed)"
                      % (sample, a.nq)}
        line["oracle_best_first_per_query"] = {
            "nodes_popped": float(np.mean(ost[:, 0])), "leaves": float(np.mean(ost[:, 1])),
            "descs_scanned": float(np.mean(ost[:, 2])), "bounds": float(np.mean(ost[:, 3]))}
    line["roofline"] = roof
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    ix.free()
    return 0


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


def warm_start_leg(a, ix, d_q, seeds, tree_idx, stream, probe):
    """dt_search_seeded over the batch (exact; same indices as the plain
    tree search), timed like the main step, with its traversal counts."""
    import torch
    from paper_2107_03368_gb300 import dt
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    idx, _, _, _ = dt.dt_search_seeded(ix, d_q, a.k, seeds)
    e.record(stream)
    torch.cuda.synchronize()
    ms = s.elapsed_time(e)
    _, _, _, st = dt.dt_search_seeded(ix, d_q, a.k, seeds, stats=True)
    return {"n_probe": probe, "queries_per_s": a.nq / (ms / 1000.0), "ms": ms,
            "same_indices_as_tree": bool(torch.equal(idx, tree_idx)),
            "per_query": {kk: v / a.nq for kk, v in st.items()}}


def learned_leg(a, dist, d_db, d_q, db, tree_qps, bf_qps, stream, ix, tree_idx):
    """Learned proposal on the same database and queries: train the encoder on
    (query, exact nearest neighbour) pairs from the GPU brute force, build the
    inverted file, then find the fewest probed lists whose exact-reranked
    top-1 reaches the target recall against the exact top-1, and time the
    search there."""
    import torch
    from paper_2107_03368_gb300 import dt, learned, synth

    exact = dt.bf_search(d_db, d_q, 1, path=2)[0][:, 0].clone()
    enc = learned.Encoder(seed=1)

    def make_queries(r):            # training queries: disjoint seeds from the timed batch
        return synth.queries(SEED + 5_000_000 + 1000 * dist.rank + r, db, 16384)[0]

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = learned.train(enc, d_db, make_queries, steps=a.train_steps, batch=a.train_batch,
                         lr=1e-3, tau=0.05, epochs_per_round=a.train_epochs)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ivf = learned.IVF(enc, d_db, n_lists=a.n_lists, iters=4)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0

    def run(probe, reps):
        ivf.search(d_q, 1, probe)
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        with nvtx("learned_search_p%d" % probe):
            for _ in range(reps):
                idx, _, scanned = ivf.search(d_q, 1, probe, with_scanned=True)
        e.record(stream)
        torch.cuda.synchronize()
        rec = float((idx[:, 0] == exact).float().mean().item())
        return s.elapsed_time(e) / reps, rec, float(scanned.float().mean().item())

    sweep = []
    chosen = None
    probes = [p for p in (1, 2, 4, 8, 16, 24, 32, 48, 64, 96, 128, 192, 256) if p <= a.n_lists]
    for probe in probes:
        ms, rec, scanned = run(probe, 1)
        sweep.append({"n_probe": probe, "recall_at_1": rec, "ms": ms,
                      "scanned_per_query": scanned})
        if rec >= a.target_recall:
            chosen = probe
            break
    out = {"train_steps": a.train_steps, "train_epochs_per_round": a.train_epochs,
           "train_pairs": a.train_steps * a.train_batch // a.train_epochs,
           "train_s": train_s, "loss_first": hist[0][1], "loss_last": hist[-1][1],
           "ivf_build_s": build_s, "n_lists": a.n_lists, "sweep": sweep,
           "target_recall_at_1": a.target_recall}
    # the same network at its initial weights (what training adds)
    if a.untrained_baseline:
        enc0 = learned.Encoder(seed=1)
        ivf0 = learned.IVF(enc0, d_db, n_lists=a.n_lists, iters=4)
        un = []
        for row in sweep:
            idx0, _, _ = ivf0.search(d_q, 1, row["n_probe"])
            un.append({"n_probe": row["n_probe"],
                       "recall_at_1": float((idx0[:, 0] == exact).float().mean().item())})
        out["untrained_sweep"] = un
        ivf0.free()
        enc0.free()
    # warm start: the proposal's top-k (few probes) seeds the exact tree search
    ws_probe = 8
    seeds, _, _ = ivf.search(d_q, a.k, ws_probe)
    out["warm_start"] = warm_start_leg(a, ix, d_q, seeds, tree_idx, stream, ws_probe)
    if chosen is not None:
        # the per-query CUDA-core scan at the same setting, for comparison
        ivf.search(d_q, 1, chosen, path=1)
        torch.cuda.synchronize()
        s1 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        s1.record(stream)
        ivf.search(d_q, 1, chosen, path=1)
        e1.record(stream)
        torch.cuda.synchronize()
        out["per_query_cuda_core_path_ms"] = s1.elapsed_time(e1)
        ms, rec, scanned = run(chosen, 3)
        qps = a.nq / (ms / 1000.0)
        # the exact rerank is an overlap contraction over the probed rows
        tf = 2.0 * 4096 * scanned * a.nq / (ms / 1e3) / 1e12
        tc_peak = 2.0 * peaks()["bf16_tflops"]
        out.update(n_probe=chosen, recall_at_1=rec, queries_per_s=qps, ms=ms,
                   scanned_per_query=scanned, descriptors_scanned_per_s=qps * scanned,
                   speedup_vs_tree=qps / tree_qps,
                   speedup_vs_bf=qps / bf_qps,
                   scan_roofline={"bound": "tensor", "achieved": tf, "peak": tc_peak,
                                  "unit": "TFLOP/s", "frac": tf / tc_peak,
                                  "note": "2 x 4096 FLOP per (query, scanned row); time of the "
                                          "whole search call (embedding, probing, scan, merge)"})
    ivf.free()
    enc.free()
    return out


def votes_leg(a, dev, stream, nt):
    """Batched partial-object retrieval: 400 objects x 25,000 descriptors,
    1,000 uneven partial queries (contiguous 5-40% of one object, clamped to
    500-10,000 descriptors), all in one retrieve_objects call.  Threshold 10
    (the paper's vote threshold) over all queries, and threshold 0 (count
    every descriptor) over a sample of queries."""
    import torch
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
    out = {"workload": "%d objects x %d descriptors, %d partial queries, %d query descriptors"
                       % (n_obj, per, a.votes_queries, qd.shape[0])}

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
            ix, d_obj, n_obj, d_qd, d_off, 10, seed, engine=2))
    w = winner.cpu().numpy()
    out["threshold_10"] = {
        "engine": "tensor rounds", "ms": ms, "partial_queries_per_s": a.votes_queries / (ms / 1e3),
        "descriptors_consumed": int(consumed.sum().item()),
        "winner_is_source_object": float(np.mean(w == qobj))}
    m = a.votes_sample
    sub_off = d_off[: m + 1].contiguous()
    n_desc = int(off[m])
    ms0, _ = timed(lambda: dt.retrieve_objects(ix, d_obj, n_obj, d_qd[:n_desc], sub_off, 0, seed,
                                               engine=2))
    out["threshold_0_sample"] = {
        "engine": "tensor", "partial_queries": m, "query_descriptors": n_desc, "ms": ms0,
        "descriptor_nn_per_s": n_desc / (ms0 / 1e3)}
    # the same call (all its uneven queries in one call) captured once in a
    # CUDA graph and replayed
    vo = (torch.empty((m, n_obj), dtype=torch.int32, device=dev),
          torch.empty(m, dtype=torch.int32, device=dev),
          torch.empty(m, dtype=torch.int64, device=dev))
    q_sub = d_qd[:n_desc]
    ref_votes, _, _ = dt.retrieve_objects(ix, d_obj, n_obj, q_sub, sub_off, 0, seed, engine=2)
    torch.cuda.synchronize()
    # object distance scores (§6.4) of the same sample against every object
    torch.cuda.synchronize()
    s_ev = torch.cuda.Event(enable_timing=True)
    e_ev = torch.cuda.Event(enable_timing=True)
    s_ev.record(stream)
    with nvtx("object_scores"):
        sc = dt.object_scores(d_db, d_obj, n_obj, q_sub, sub_off)
    e_ev.record(stream)
    torch.cuda.synchronize()
    ms_s = s_ev.elapsed_time(e_ev)
    best = sc.argmin(dim=1).cpu().numpy()
    out["object_scores_sample"] = {
        "partial_queries": m, "query_descriptors": n_desc, "objects": n_obj, "ms": ms_s,
        "pairs_per_s": n_desc * (n_obj * per) / (ms_s / 1e3),
        "best_object_is_source": float(np.mean(best == qobj[:m]))}
    out["threshold_0_sample"]["graph_replay"] = graph_replay_leg(
        lambda: dt.retrieve_objects(ix, d_obj, n_obj, q_sub, sub_off, 0, seed, engine=2, out=vo),
        vo[0], ref_votes, stream)
    ix.free()
    return out


def run_tensor_workload(a, dist):
    """Large-batch brute force: every query against every descriptor on the
    tensor cores (bf_search path 2), the popcount kernel timed on a sample,
    both checked against each other and, on a few queries, the oracle."""
    import torch
    import oracle
    from paper_2107_03368_gb300 import dt, synth

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    stream = torch.cuda.current_stream(dev)
    nt = cpu_cores()
    seed = SEED + 2                              # the tensor workload's own seed
    n, nq, k = a.tc_n, a.tc_nq, a.k
    db, _ = synth.database(seed, n, per_object=a.per_object, nthreads=nt)
    q, _ = synth.queries(seed + 1000 * dist.rank, db, nq, nthreads=nt)
    d_db = torch.from_numpy(db.view(np.int64)).to(dev)
    d_q = torch.from_numpy(q.view(np.int64)).to(dev)
    out = (torch.empty((nq, k), dtype=torch.int32, device=dev),
           torch.empty((nq, k), dtype=torch.float32, device=dev), None)

    def step():
        dt.bf_search(d_db, d_q, k, out=out, path=2)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(dist.local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for i in range(a.steps):
        starts[i].record(stream)
        with nvtx("bf_path2_large"):
            step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    dt.dt_sync_status()
    ms = dist.max(sum(st.elapsed_time(e) for st, e in zip(starts, ends)) / a.steps)
    value = aggregate(ms, nq, dist.world)

    # popcount kernel on a sample of the queries; same indices as the tensor kernel
    m = min(2048, nq)
    p_out = (torch.empty((m, k), dtype=torch.int32, device=dev),
             torch.empty((m, k), dtype=torch.float32, device=dev), None)
    dt.bf_search(d_db, d_q[:m], k, out=p_out, path=1)
    torch.cuda.synchronize()
    ps = torch.cuda.Event(enable_timing=True)
    pe = torch.cuda.Event(enable_timing=True)
    ps.record(stream)
    dt.bf_search(d_db, d_q[:m], k, out=p_out, path=1)
    pe.record(stream)
    torch.cuda.synchronize()
    popc_ms = ps.elapsed_time(pe)
    same_popc = bool(torch.equal(p_out[0], out[0][:m]))

    pk = peaks()
    tf = 2.0 * nq * n * 4096 / (ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": dist.world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "e4m3", "data": "synthetic",
        "config": {"workload": "tensor-core brute force, %d descriptors x %d queries, top-%d"
                               % (n, nq, k), "n_db": n, "n_queries": nq, "k": k,
                   "l2": "inputs larger than L2 (%.2f GB database)" % (n * 512 / 1e9)},
        "gpu_launches": 3 * a.steps,
        "clocks": clocks,
        "roofline": {"bound": "tensor", "achieved": tf, "peak": 2.0 * pk["bf16_tflops"],
                     "unit": "TFLOP/s", "frac": tf / (2.0 * pk["bf16_tflops"]), "traffic": None,
                     "peak_kind": "FP8 = 2 x %s bf16 (nominal ratio)" % pk["kind"]},
        "popc_sample": {"queries": m, "ms": popc_ms, "queries_per_s": m / (popc_ms / 1e3),
                        "same_indices_as_tensor": same_popc},
    }
    if dist.rank == 0 and not a.no_cpu_baseline:
        sample = 4
        t0 = time.perf_counter()
        o_idx, o_score, _ = oracle.bf_topk(db, q[:sample], k, nthreads=nt)
        cpu_s = time.perf_counter() - t0
        g_idx = out[0][:sample].cpu().numpy().view(np.uint32).astype(np.int64)
        g_score = out[1][:sample].cpu().numpy().astype(np.float64)
        line["oracle_check"] = {
            "queries": sample, "same_indices": bool(np.array_equal(g_idx, o_idx)),
            "max_score_rel_err": float(np.max(np.abs(g_score - o_score) / np.maximum(o_score, 1e-300)))}
        line["cpu_baseline"] = {"value": sample / cpu_s, "unit": "queries/s", "cores": nt,
                                "kind": "oracle",
                                "sample": "%d of the %d queries, oracle brute force" % (sample, nq)}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    return 0


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
        if a.workload == "tensor-bf":
            return run_tensor_workload(a, dist)
        return run_ours(a, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    sys.exit(main())
