#!/usr/bin/env python3
"""Benchmark: stroke expansion throughput (input segments/s) on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

A step is one pass of the whole hot path -- tag-monoid scan, plan (subdivision),
pieces, primitive scan, emit -- over the map-like workload (50,000 open stroked paths, ~1.68M input
segments, tolerance 0.1, line output) with the encoded scene resident in HBM.
Between timed steps a 512 MB buffer is written to flush L2 (outside the timed
interval).  Prints one JSON line (rank 0).  N > 1 (torchrun) runs independent
replicas, one per GPU: the path shards by path, so there is no collective.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input segments/sec expanded"
UNIT = "segments/s"
TOL = 0.1
WORKLOAD = "map-like"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------- oracle (CPU)

def _oracle_chunk(args):
    verbs, pts, voff, hw, jn, cp, ml, dfi, dco, dof, dle, tol, arcs = args
    import numpy as np
    import oracle
    import workloads as W
    sc = W.Scene(verbs, pts, voff, hw, jn, cp, ml, dfi, dco, dof, dle)
    t = time.perf_counter()
    r = oracle.stroke(sc, tol, arcs=arcs)
    return time.perf_counter() - t, int(r["prim"].shape[0])


def oracle_jobs(scene, tol, arcs, chunks=64):
    import numpy as np
    n = scene.n_paths
    bounds = np.linspace(0, n, min(chunks, n) + 1).astype(int)
    jobs = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        s = scene.subset(range(a, b))
        jobs.append((s.verbs, s.pts, s.path_verb_off, s.half_width, s.join, s.cap, s.miter_limit, s.dash_first,
                     s.dash_count, s.dash_offset, s.dash_len, tol, arcs))
    return jobs


def oracle_pool(cores):
    """A pool of spawned worker processes (never forked from a CUDA process)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    pool = mp.get_context("spawn").Pool(cores)
    pool.map(_oracle_chunk, oracle_jobs(__import__("workloads").hand_cases(), 0.25, False, chunks=cores))
    return pool


def oracle_timed(pool, jobs):
    """Wall time of the FP64 oracle over the jobs on the pool."""
    t = time.perf_counter()
    res = pool.map(_oracle_chunk, jobs)
    return time.perf_counter() - t, sum(r[1] for r in res)


# --------------------------------------------------------------------------- clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons, n = [], [], set(), 0
        for line in self.file:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            n += 1
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": n}


def max_over_ranks(x, torch, device):
    """The largest of every rank's x (x itself on a single process)."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms):
    """Whole-job throughput: every rank expands its own replica of the workload
    (weak scaling), timed by the slowest rank."""
    return world * units_per_rank / (ms * 1e-3)


def _gpu_id(torch, dev):
    try:
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
    except Exception:
        return None


# --------------------------------------------------------------------------- main

def measure_batched(ex, P, B, W, torch, dev, stream, flush):
    """Batched workload: 4,096 independent documents (segments per document
    ceil(lognormal(ln 300, 1.5)) clipped to [1, 200,000]), map-like geometry and
    styles, tol 0.1, lines.  One CUDA-graph launch of the whole batch (launch
    shapes from the autotuner) against one launch sequence per document."""
    scenes = W.documents()
    n_seg = sum(s.n_segments for s in scenes)
    docs = [ex.upload(P.encode(s)) for s in scenes]
    params = P.make_params(TOL)
    default = B.se_get_tuning(ex.ctx)
    batch = P.Batch(ex, docs)
    batch.prepare(TOL)
    tuning = B.se_autotune(ex.ctx, B.se_batch_scene(batch.handle), params, batch.desc, reps=2)
    # the count above sized the context for the batch; capture after tuning
    batch.capture()
    for _ in range(3):
        batch.launch()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    for a, b in ev:
        flush.fill_(3.0)
        a.record(stream)
        batch.launch()
        b.record(stream)
    torch.cuda.synchronize(dev)
    graph_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    code, n_batch = B.se_sync(ex.ctx)
    assert code == B.SE_OK, code
    batch.close()
    # one launch sequence per document, each into its own slice of one buffer
    counts = [ex.count(ds, TOL) for ds in docs]
    total = int(sum(counts))
    assert total == n_batch, (total, n_batch)
    prims = torch.empty((max(total, 1), 4), dtype=torch.float32, device=dev)
    descs, off = [], 0
    for n in counts:
        descs.append(B.se_outline_dev(prims.data_ptr() + 16 * off, 0, 0, 0, 0, int(n)))
        off += int(n)
    for ds, d in zip(docs, descs):
        ex.expand_async(ds, params, d)
    torch.cuda.synchronize(dev)
    per_doc = []
    for _ in range(2):
        flush.fill_(4.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for ds, d in zip(docs, descs):
            ex.expand_async(ds, params, d)
        b.record(stream)
        torch.cuda.synchronize(dev)
        per_doc.append(a.elapsed_time(b))
    B.se_set_tuning(ex.ctx, **default)
    per_doc_ms = statistics.mean(per_doc)
    return {"workload": f"batched: {len(scenes)} documents, {n_seg} segments (lognormal median 300, sigma 1.5, "
                        f"clipped to [1, 200000]), map-like styles, tol 0.1, lines",
            "value": n_seg / (graph_ms * 1e-3), "unit": UNIT, "ms_per_step": graph_ms, "output_prims": total,
            "per_document": {"value": n_seg / (per_doc_ms * 1e-3), "ms_per_step": per_doc_ms,
                             "launch_sequences": len(docs)},
            "speedup_vs_per_document": per_doc_ms / graph_ms, "tuning": tuning}


def measure_served(ex, P, B, W, torch, dev, seconds=6.0):
    """Served workload: requests for documents of 1e3..5e6 segments (log-uniform;
    24 distinct documents, map-like styles, 30% of paths dashed) arrive as a Poisson
    stream; the library's serving loop (4 slots, continuous batching, 100 GB HBM
    budget) against one expansion per request (1 slot, batches of 1).  The offered
    2,000 requests/s exceeds what one GPU sustains, so the capacity is measured
    first (all requests queued at once) and the latency stream runs at 70% of it."""
    import math
    scenes = W.serving_pool()
    docs = [ex.upload(P.encode(s)) for s in scenes]
    segs = [s.n_segments for s in scenes]
    rng = np.random.default_rng(5)
    budget = 100 << 30

    def run(server, arrivals, picks):
        t0 = time.perf_counter()
        pending, done = [], []
        i = 0
        while i < len(arrivals) or pending:
            now = time.perf_counter() - t0
            while i < len(arrivals) and arrivals[i] <= now:
                pending.append((server.submit(docs[picks[i]], TOL), picks[i]))
                i += 1
            still = []
            for rid, k in pending:
                r = server.poll(rid)
                if r["done"]:
                    assert r["status"] == 0, (r["status"], server.last_error())
                    done.append((r["t_submit_ns"], r["t_done_ns"], segs[k], r["batch_docs"]))
                    server.release(rid)
                else:
                    still.append((rid, k))
            pending = still
            if i < len(arrivals):
                time.sleep(max(0.0, min(0.0005, arrivals[i] - (time.perf_counter() - t0))))
            else:
                time.sleep(0.0002)
        lat = np.array([(b - a) * 1e-6 for a, b, _, _ in done])
        span = (max(b for _, b, _, _ in done) - min(a for a, _, _, _ in done)) * 1e-9
        return {"requests": len(done), "segments": int(sum(s for _, _, s, _ in done)),
                "value": sum(s for _, _, s, _ in done) / span, "unit": UNIT,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_batch_docs": float(np.mean([b for _, _, _, b in done]))}

    served = P.Server(0, slots=4, max_batch_docs=64, max_batch_tags=1 << 23, hbm_budget=budget)
    n_sat = 96
    picks = rng.integers(0, len(docs), n_sat)
    cap = run(served, np.zeros(n_sat), picks)
    rate = min(2000.0, 0.7 * cap["value"] / float(np.mean(segs)))
    n_req = int(rate * seconds)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    picks = rng.integers(0, len(docs), n_req)
    stream_res = run(served, arrivals, picks)
    st = served.stats()
    served.close()
    single = P.Server(0, slots=1, max_batch_docs=1, max_batch_tags=0, hbm_budget=budget)
    per_doc = run(single, arrivals, picks)
    single.close()
    return {"workload": f"served: Poisson requests for {len(docs)} documents of 1e3..5e6 segments (log-uniform, "
                        f"mean {int(np.mean(segs))}), 30% of paths dashed, tol 0.1, lines, 100 GB budget",
            "offered_rate_req_s": 2000.0, "capacity": cap, "rate_req_s": rate,
            "continuous_batching": {**stream_res, "slots": 4, "max_concurrent": st["max_concurrent"],
                                    "bytes_peak": st["bytes_peak"]},
            "one_per_request": per_doc}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paths", type=int, default=50_000,
                    help="map-like paths (profiling runs use a smaller case of the same workload)")
    ap.add_argument("--lite", action="store_true", help="device stages only: no arcs, e2e or CPU baseline legs")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and served legs")
    ap.add_argument("--workload", default="map-like", choices=["map-like", "curvature"],
                    help="scene of the main measurement (profiling runs; the reported metric is map-like)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    import numpy as np
    import workloads as W

    global TOL
    if args.workload == "curvature":
        TOL = 0.25
        scene = W.curvature_stress(n_paths=min(args.paths, 100_000))
    else:
        scene = W.map_like(n_paths=args.paths)
    n_seg = scene.n_segments
    wname = WORKLOAD if args.workload == "map-like" else "curvature stress (dashed)"
    config = {"workload": f"{wname}: {scene.n_paths} open stroked paths, {n_seg} input segments, "
                          f"tol {TOL}, line output", "n_paths": scene.n_paths, "n_segments": n_seg, "tol": TOL,
              "output": "lines", "l2": "flushed between timed steps (512 MB write, untimed)",
              "parallelism": f"replicas x{args.gpus}"}

    if args.impl == "reference":
        if rank != 0:
            return 0
        cores = os.cpu_count() or 1
        # bounded sample per step: every 16th path (~105k segments)
        sample = scene.subset(range(0, scene.n_paths, 16))
        jobs = oracle_jobs(sample, TOL, False, chunks=4 * cores)
        pool = oracle_pool(cores)
        for _ in range(args.warmup):
            oracle_timed(pool, jobs)
        times = []
        for _ in range(args.steps):
            wall, _ = oracle_timed(pool, jobs)
            times.append(wall)
        pool.close()
        v = sample.n_segments / statistics.mean(times)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"every 16th path of the workload ({sample.n_segments} segments) per step"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    # CPU baseline first (spawned pool, before any GPU work)
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.lite:
        cores = os.cpu_count() or 1
        pool = oracle_pool(cores)
        wall, _ = oracle_timed(pool, oracle_jobs(scene, TOL, False, chunks=4 * cores))
        pool.close()
        # the same oracle on one host thread, in this process, on every 8th path
        one = scene.subset(range(0, scene.n_paths, 8))
        wall1, _ = _oracle_chunk(oracle_jobs(one, TOL, False, chunks=1)[0])
        cpu_baseline = {"value": n_seg / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                        "sample": f"the whole workload ({n_seg} segments) once, {cores} spawned worker processes",
                        "one_thread": {"value": one.n_segments / wall1, "unit": UNIT, "cores": 1,
                                       "sample": f"every 8th path ({one.n_segments} segments) once, in-process"}}

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2405_00127_gb300 import build
    build.build()
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B

    t0 = time.perf_counter()
    enc = P.encode(scene)
    encode_ms = 1e3 * (time.perf_counter() - t0)
    stream = torch.cuda.current_stream(dev)
    ex = P.StrokeExpander(local, stream)
    ds = ex.upload(enc)
    params = P.make_params(TOL)
    n_prims = ex.count(ds, TOL)
    bufs = ex.alloc(ds, n_prims, False, ex.expanded_tags(ds))
    desc = ex.outline_desc(bufs, n_prims)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    B.se_profile_enable(ex.ctx, True)
    for _ in range(args.warmup):
        ex.expand_async(ds, params, desc)
    code, n_check = B.se_sync(ex.ctx)
    assert code == B.SE_OK and n_check == n_prims, (code, n_check, n_prims)

    clocks = Clocks(_gpu_id(torch, dev) if rank == 0 else None)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage = []
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        ex.expand_async(ds, params, desc)
        ev[k][1].record(stream)
        stage.append(B.se_profile_read(ex.ctx))
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(step_ms)
    if world > 1:
        ms = max_over_ranks(ms, torch, dev)
    code, _ = B.se_sync(ex.ctx)
    assert code == B.SE_OK, code

    names = ("tag_scan", "plan", "pieces", "prim_scan", "emit", "dash")
    stage_ms = {nm: statistics.mean(s_[k] for s_ in stage) for k, nm in enumerate(names)}
    emit_ms = stage_ms["emit"]
    stats = B.se_ctx_stats(ex.ctx)
    n_tags = int(stats["n_tags"])
    n_words = int(enc.points.size)
    n_items = int(stats["n_items"])
    n_pieces = n_items - n_tags
    # bytes the emit stage must move: every primitive written (16 B geometry + 4 B path id);
    # per piece its record plus its item, count, offset and owner (24 B); per tag its join /
    # cap record plus its tail item's base, count and offset and its path id (24 B)
    emit_bytes = n_prims * (16 + 4) + n_pieces * (stats["piece_bytes"] + 24) + n_tags * (stats["tail_bytes"] + 24)
    peak, peak_kind = _peaks()
    achieved = emit_bytes / (emit_ms * 1e-3) / 1e9
    # DRAM traffic of the emit stage per primitive, from an ncu capture (dram__bytes_read.sum +
    # dram__bytes_write.sum) of both emit kernels on the 10,000-path map-like case (424.8 MB for
    # 6,126,892 line primitives), scaled by the primitives of this launch; reset to None whenever
    # the emit kernels change until they are captured again
    traffic = 425.054e6 / 6126892 * n_prims if args.workload == "map-like" else None
    roofline = {"bound": "hbm", "kernel": "emit stage (emit_pieces_kernel + emit_tails_kernel)", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
                "algorithmic_bytes_per_launch": emit_bytes,
                "units": {"prims": n_prims, "items": n_items, "pieces": n_pieces, "tags": n_tags}}

    if args.lite:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": job_value(n_seg, world, ms), "unit": UNIT,
                              "ms_per_step": ms, "stage_ms": stage_ms, "roofline": roofline, "config": config,
                              "lite": True}), flush=True)
        ex.close()
        return 0

    # arcs, same scene (reported alongside)
    params_a = P.make_params(TOL, arcs=True)
    n_arcs = ex.count(ds, TOL, arcs=True)
    bufs_a = ex.alloc(ds, n_arcs, True)
    desc_a = ex.outline_desc(bufs_a, n_arcs)
    for _ in range(3):
        ex.expand_async(ds, params_a, desc_a)
    torch.cuda.synchronize(dev)
    ea = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for a, b in ea:
        flush.fill_(1.0)
        a.record(stream)
        ex.expand_async(ds, params_a, desc_a)
        b.record(stream)
    torch.cuda.synchronize(dev)
    arcs_ms = statistics.mean(a.elapsed_time(b) for a, b in ea)

    # refined line output (exact-integral counts, Newton-refined vertices), same scene
    params_r = P.make_params(TOL, refine=True)
    n_ref = ex.count(ds, TOL, refine=True)
    bufs_r = ex.alloc(ds, n_ref, False, ex.expanded_tags(ds))
    desc_r = ex.outline_desc(bufs_r, n_ref)
    for _ in range(3):
        ex.expand_async(ds, params_r, desc_r)
    torch.cuda.synchronize(dev)
    er = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    ref_stage = []
    for a, b in er:
        flush.fill_(3.0)
        a.record(stream)
        ex.expand_async(ds, params_r, desc_r)
        b.record(stream)
        ref_stage.append(B.se_profile_read(ex.ctx))
    torch.cuda.synchronize(dev)
    code, n_chk = B.se_sync(ex.ctx)
    assert code == B.SE_OK and n_chk == n_ref, (code, n_chk, n_ref)
    ref_ms = statistics.mean(a.elapsed_time(b) for a, b in er)
    refined = {"value": n_seg / (ref_ms * 1e-3), "unit": UNIT, "ms_per_step": ref_ms, "output_prims": n_ref,
               "output_prims_vs_fast": n_ref / n_prims,
               "stage_ms": {nm: statistics.mean(s_[k] for s_ in ref_stage) for k, nm in enumerate(names)}}
    del bufs_r

    # curvature stress (100,000 dashed single-cubic paths, tol 0.25), reported alongside
    cs = W.curvature_stress()
    cs_enc = P.encode(cs)
    cs_ds = ex.upload(cs_enc)
    cs_params = P.make_params(0.25)
    cs_n = ex.count(cs_ds, 0.25)
    cs_bufs = ex.alloc(cs_ds, cs_n, False, ex.expanded_tags(cs_ds))
    cs_desc = ex.outline_desc(cs_bufs, cs_n)
    for _ in range(3):
        ex.expand_async(cs_ds, cs_params, cs_desc)
    torch.cuda.synchronize(dev)
    ec = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    cs_stage = []
    for a, b in ec:
        flush.fill_(2.0)
        a.record(stream)
        ex.expand_async(cs_ds, cs_params, cs_desc)
        b.record(stream)
        cs_stage.append(B.se_profile_read(ex.ctx))
    torch.cuda.synchronize(dev)
    code, _ = B.se_sync(ex.ctx)
    assert code == B.SE_OK, code
    cs_ms = statistics.mean(a.elapsed_time(b) for a, b in ec)
    cs_st = B.se_ctx_stats(ex.ctx)
    curvature = {"workload": f"curvature stress: {cs.n_paths} dashed single-cubic paths [10, 5], tol 0.25, lines",
                 "value": cs.n_segments / (cs_ms * 1e-3), "unit": UNIT, "ms_per_step": cs_ms,
                 "output_prims": cs_n, "dashed_tags": int(cs_st["n_tags"]),
                 "stage_ms": {nm: statistics.mean(s_[k] for s_ in cs_stage) for k, nm in enumerate(names)}}
    del cs_bufs, cs_ds

    # MotionMark-like scene (lines, quadratics and cubics under one scaling transform, tol 0.25), alongside
    mm = W.mmark_like(n_paths=60_000)
    mm_ds = ex.upload(P.encode(mm))
    mm_n = ex.count(mm_ds, 0.25)
    mm_bufs = ex.alloc(mm_ds, mm_n, False)
    mm_desc = ex.outline_desc(mm_bufs, mm_n)
    mm_params = P.make_params(0.25)
    for _ in range(3):
        ex.expand_async(mm_ds, mm_params, mm_desc)
    torch.cuda.synchronize(dev)
    em = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    mm_stage = []
    for a, b in em:
        flush.fill_(4.0)
        a.record(stream)
        ex.expand_async(mm_ds, mm_params, mm_desc)
        b.record(stream)
        mm_stage.append(B.se_profile_read(ex.ctx))
    torch.cuda.synchronize(dev)
    code, n_chk = B.se_sync(ex.ctx)
    assert code == B.SE_OK and n_chk == mm_n, (code, n_chk, mm_n)
    mm_ms = statistics.mean(a.elapsed_time(b) for a, b in em)
    mmark = {"workload": f"MotionMark-like: {mm.n_paths} paths, {mm.n_segments} line/quadratic/cubic segments, "
                         f"scaled x2.61 by a transform, tol 0.25, lines",
             "value": mm.n_segments / (mm_ms * 1e-3), "unit": UNIT, "ms_per_step": mm_ms, "output_prims": mm_n,
             "stage_ms": {nm: statistics.mean(s_[k] for s_ in mm_stage) for k, nm in enumerate(names)}}
    del mm_bufs, mm_ds

    # nonzero coverage of the map-like outline on a 4096 x 4096 grid (the downstream use of the line soup)
    out_m = P.Outline(bufs[0][:n_prims], None, bufs[2][:n_prims], bufs[3], bufs[4], n_prims, 0)
    P.coverage(ex, out_m, scene.n_paths, 4096, 4096)          # warm-up (allocator, first launch)
    cov_ms = []
    for _ in range(3):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        cnt, area = P.coverage(ex, out_m, scene.n_paths, 4096, 4096)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        cov_ms.append(c0.elapsed_time(c1))
    cov = {"workload": f"nonzero coverage of the map-like outline ({n_prims} lines, {scene.n_paths} paths) "
                       f"on a 4096 x 4096 pixel grid", "ms": statistics.mean(cov_ms),
           "prims_per_s": n_prims / (statistics.mean(cov_ms) * 1e-3),
           "covered_pixel_path_pairs": int(area.sum().item()), "pixels_covered": int((cnt > 0).sum().item())}
    del cnt, area

    # primitive counts against tolerance, lines and arcs (the count experiment of Section 9.1 on the
    # synthetic scenes): one count pass each
    sweep = {"tol": [1.0, 0.5, 0.25, 0.1, 0.05, 0.025, 0.01, 0.005, 0.001]}
    for wn, sds in (("map_like", ds), ("mmark_like", ex.upload(P.encode(mm)))):
        sweep[wn] = {"lines": [ex.count(sds, t) for t in sweep["tol"]],
                     "arcs": [ex.count(sds, t, arcs=True) for t in sweep["tol"]]}

    batched = None if args.no_extra else measure_batched(ex, P, B, W, torch, dev, stream, flush)
    served = None if args.no_extra else measure_served(ex, P, B, W, torch, dev)

    # end to end through the C ABI on pinned host buffers
    h_tags = torch.from_numpy(enc.tags).pin_memory().numpy()
    h_pts = torch.from_numpy(enc.points.view(np.int32)).pin_memory().numpy().view(np.uint32)
    h_sty = torch.from_numpy(enc.styles.view(np.uint8)).pin_memory().numpy().view(P.STYLE_DTYPE)
    h_out = torch.empty((n_prims, 4), dtype=torch.float32).pin_memory().numpy()
    e2e = []
    for k in range(args.e2e_steps + 1):
        t = time.perf_counter()
        code, n = B.se_expand_host(ex.ctx, h_tags, h_pts, h_sty, enc.n_paths, None, params, h_out, None, n_prims)
        dt = time.perf_counter() - t
        assert code == B.SE_OK and n == n_prims, (code, n)
        if k:
            e2e.append(dt)
    e2e_s = statistics.mean(e2e)
    if world > 1:
        e2e_s = max_over_ranks(e2e_s, torch, dev)
    h2d = n_tags + n_words * 4 + enc.styles.size * 24
    d2h = n_prims * 16 + 16

    if rank == 0:
        line = {"metric": METRIC, "value": job_value(n_seg, world, ms), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
                "output_prims": n_prims, "output_prims_per_s": world * n_prims / (ms * 1e-3),
                "stage_ms": stage_ms,
                "arcs": {"value": n_seg / (arcs_ms * 1e-3), "ms_per_step": arcs_ms, "output_prims": n_arcs},
                "refined": refined,
                "curvature_stress": curvature,
                "mmark_like": mmark,
                "count_vs_tolerance": sweep,
                "coverage": cov,
                "batched": batched,
                "served": served,
                "host_encode_ms": encode_ms,
                "roofline": roofline,
                "e2e": {"value": world * n_seg / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s},
                "gpu_launches": 8 * args.steps,
                "clocks": clk,
                "cpu_baseline": cpu_baseline}
        print(json.dumps(line), flush=True)
    ex.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
