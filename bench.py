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


# --------------------------------------------------------------------------- roofline (SURVEY 8(d) units)

# Arithmetic per unit of work, from the measurement plan's accounting of the
# method (FP32 instructions, an FMA counting once, and special-function ops):
# one cubic -> Euler-spiral fit attempt (cubic point and derivative, two atan2
# and three sine/cosine, the Appendix A polynomials, the error terms), and one
# output vertex (density-integral inverse, spiral position, normal offset).
FIT_FP32, FIT_SFU = 110, 8
VERT_FP32, VERT_SFU = 70, 4
# Issue rates per SM per clock on the GB300 (152 SMs at up to 2070 MHz): 128
# FP32 lanes, 16 special-function lanes.
FP32_LANES, SFU_LANES = 128, 16


def alu_peaks(n_sms, sm_mhz):
    """FP32 instructions/s and SFU ops/s of the whole GPU at sm_mhz."""
    hz = sm_mhz * 1e6
    return n_sms * FP32_LANES * hz, n_sms * SFU_LANES * hz


def algo_bytes(n_tags, n_words, n_styles, n_paths, n_prims, arcs, n_input_tags=None, n_dashes=0, n_xforms=0):
    """Algorithmic HBM bytes of one expansion: the encoded input read
    once (tags, path data words, styles, dashes, transforms), the tag-scan results
    written and read once (17 B per tag), the outline written once (20 B a line,
    24 B an arc: geometry, path id, curvature), and the per-tag and per-path
    offsets (8 B each).  Per stage: tag scan (tags in, scan results out), count
    (scan results and control points in), primitive scan (offsets out), emit
    (outline out)."""
    n_in = n_tags if n_input_tags is None else n_input_tags
    inp = n_in + 4 * n_words + 24 * n_styles + 4 * n_dashes + 24 * n_xforms
    soa = 17 * n_tags
    out = (24 if arcs else 20) * n_prims
    offs = 8 * (n_tags + 1) + 8 * (n_paths + 1)
    stages = {"tag_scan": n_in + soa, "count": soa + 4 * n_words + 24 * n_styles, "prim_scan": offs, "emit": out}
    return {"total": inp + 2 * soa + out + offs, "input": inp, "scan_soa": 2 * soa, "outline": out, "offsets": offs,
            "stages": stages}


def roofline_of(bytes_total, fits, verts, ms, hbm_gbs, n_sms, sm_mhz, stage_ms=None, stage_bytes=None,
                traffic=None):
    """The step against the slower of its HBM, FP32 and SFU bounds (all three
    times are reported; frac = bound time / measured time)."""
    fp32_peak, sfu_peak = alu_peaks(n_sms, sm_mhz)
    t_hbm = bytes_total / (hbm_gbs * 1e9)
    fp32 = FIT_FP32 * fits + VERT_FP32 * verts
    sfu = FIT_SFU * fits + VERT_SFU * verts
    t_fp32, t_sfu = fp32 / fp32_peak, sfu / sfu_peak
    bound = max(("hbm", t_hbm), ("alu", t_fp32), ("sfu", t_sfu), key=lambda x: x[1])
    t = ms * 1e-3
    r = {"bound": "hbm" if bound[0] == "hbm" else "alu", "bound_detail": bound[0],
         "achieved": bytes_total / t / 1e9, "peak": hbm_gbs, "unit": "GB/s", "frac": bound[1] / t,
         "traffic": traffic, "algorithmic_bytes": bytes_total, "time_at_bounds_ms":
         {"hbm": 1e3 * t_hbm, "fp32": 1e3 * t_fp32, "sfu": 1e3 * t_sfu}, "measured_ms": ms,
         "fp32_instr": fp32, "sfu_ops": sfu, "fits": fits, "vertices": verts,
         "fp32_peak_instr_s": fp32_peak, "sfu_peak_ops_s": sfu_peak, "peak_source": "measured (HBM copy); "
         f"ALU from {n_sms} SMs x {FP32_LANES} FP32 / {SFU_LANES} SFU lanes x {sm_mhz:.0f} MHz"}
    if r["bound"] == "alu":
        r.update(achieved=fp32 / t / 1e12, peak=fp32_peak / 1e12, unit="T FP32 instr/s")
    if stage_ms and stage_bytes:
        r["stages"] = {k: {"ms": stage_ms.get(k), "bytes": b,
                           "frac_hbm": (b / (hbm_gbs * 1e9)) / (stage_ms[k] * 1e-3) if stage_ms.get(k) else None}
                       for k, b in stage_bytes.items()}
    return r


def traffic_from_profiles(kernel_file, n_units):
    """DRAM bytes per launch from a committed ncu summary (the line
    'traffic-per-unit: <bytes> ... sources <sha>'), scaled by the units of this
    launch; None when the kernel sources changed since the capture."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", kernel_file)
    if not os.path.exists(path):
        return None
    m = re.search(r"traffic-per-unit: ([0-9.eE+-]+) .*sources ([0-9a-f]{16})", open(path).read())
    if not m:
        return None
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_2405_00127_gb300", "csrc"))):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(ROOT, "paper_2405_00127_gb300", "csrc", f), "rb").read())
    if h.hexdigest()[:16] != m.group(2):
        return None
    return float(m.group(1)) * n_units


# --------------------------------------------------------------------------- oracle (CPU)

def _oracle_chunk(args):
    """Time the oracle on one chunk of paths; (seconds, primitives, fit attempts, vertices)."""
    verbs, pts, voff, hw, jn, cp, ml, dfi, dco, dof, dle, tol, arcs = args
    import numpy as np
    import oracle
    import workloads as W
    sc = W.Scene(verbs, pts, voff, hw, jn, cp, ml, dfi, dco, dof, dle)
    t = time.perf_counter()
    r = oracle.stroke(sc, tol, arcs=arcs)
    return time.perf_counter() - t, int(r["prim"].shape[0]), r["n_fit"], r["n_vert"]


def _oracle_reference(job):
    """The oracle's full result for a sample scene (the CPU-baseline leg's reference
    for the error statistics and the work counters of a configuration)."""
    name, scene, tol, arcs, refine = job
    import oracle
    return name, oracle.stroke(scene, tol, arcs=arcs, refine=refine)


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
    """Wall time of the FP64 oracle over the jobs on the pool, with its primitive,
    fit-attempt and vertex totals."""
    t = time.perf_counter()
    res = pool.map(_oracle_chunk, jobs)
    return time.perf_counter() - t, sum(r[1] for r in res), sum(r[2] for r in res), sum(r[3] for r in res)


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

def measure_batched(ex, P, B, W, torch, dev, stream, flush, scenes):
    """Batched workload: 4,096 independent documents (segments per document
    ceil(lognormal(ln 300, 1.5)) clipped to [1, 200,000]), map-like geometry and
    styles, tol 0.1, lines.  One CUDA-graph launch of the whole batch (launch
    shapes from the autotuner) against one launch sequence per document (each
    sequence's grids sized to its document)."""
    n_seg = sum(s.n_segments for s in scenes)
    encs = [P.encode(s) for s in scenes]
    docs = [ex.upload(e) for e in encs]
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
            "speedup_vs_per_document": per_doc_ms / graph_ms, "tuning": tuning,
            "sizes": enc_sizes(encs, total, n_seg)}


def enc_sizes(encs, n_prims, n_seg):
    """Encoded input sizes of one or more scenes (for the algorithmic bytes)."""
    return {"n_input_tags": int(sum(e.tags.size for e in encs)), "n_words": int(sum(e.points.size for e in encs)),
            "n_styles": int(sum(e.styles.size for e in encs)), "n_paths": int(sum(e.n_paths for e in encs)),
            "n_dashes": int(sum(e.dashes.size for e in encs)),
            "n_xforms": int(sum(0 if e.transforms is None else e.transforms.shape[0] for e in encs)),
            "n_prims": int(n_prims), "n_segments": int(n_seg)}


def measure_served(ex, P, B, W, torch, dev, scenes, seconds=6.0):
    """Served workload: requests for documents of 1e3..5e6 segments (log-uniform;
    24 distinct documents, map-like styles, 30% of paths dashed) arrive as a Poisson
    stream; the library's serving loop (4 slots, continuous batching, 100 GB HBM
    budget) against one expansion per request (1 slot, batches of 1).  The offered
    2,000 requests/s exceeds what one GPU sustains, so the capacity is measured
    first (all requests queued at once) and the latency stream runs at 70% of it."""
    import math
    encs = [P.encode(s) for s in scenes]
    docs = [ex.upload(e) for e in encs]
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
    counts, tags = [], []
    for d in docs:                        # sizes of every pool document (for the algorithmic bytes)
        counts.append(ex.count(d, TOL))
        tags.append(ex.expanded_tags(d))
    sizes = enc_sizes(encs, sum(counts), sum(segs))
    sizes["n_tags"] = int(sum(tags))
    # the same documents as one scene, one launch sequence (device time): the rate
    # the serving loop's capacity is compared with
    batch = P.Batch(ex, docs)
    batch.prepare(TOL)
    for _ in range(2):
        batch.expand_async()
    torch.cuda.synchronize(dev)
    st0, st1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    one = []
    for _ in range(3):
        st0.record(ex.stream)
        batch.expand_async()
        st1.record(ex.stream)
        torch.cuda.synchronize(dev)
        one.append(st0.elapsed_time(st1))
    batch.close()
    one_ms = statistics.mean(one)
    one_batch = {"value": sum(segs) / (one_ms * 1e-3), "unit": UNIT, "ms": one_ms,
                 "what": "all pool documents gathered into one scene, one launch sequence (device time)"}
    return {"workload": f"served: Poisson requests for {len(docs)} documents of 1e3..5e6 segments (log-uniform, "
                        f"mean {int(np.mean(segs))}), 30% of paths dashed, tol 0.1, lines, 100 GB budget",
            "sizes": sizes, "pool_as_one_scene": one_batch,
            "capacity_vs_one_scene": cap["value"] / one_batch["value"],
            "offered_rate_req_s": 2000.0, "capacity": cap, "rate_req_s": rate,
            "continuous_batching": {**stream_res, "slots": 4, "max_concurrent": st["max_concurrent"],
                                    "bytes_peak": st["bytes_peak"]},
            "one_per_request": per_doc}




STAGES = ("tag_scan", "plan", "pieces", "prim_scan", "emit", "dash")


def timed_expansions(ex, B, ds, params, desc, steps, stream, flush, torch, dev, counted=False):
    """Mean device time of `steps` expansions (CUDA events on the launching stream,
    L2 flushed by a 512 MB write before each, outside the timed interval) and the
    mean stage times the library's own events measured."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stage = []
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        ex.expand_async(ds, params, desc)
        ev[k][1].record(stream)
        stage.append(B.se_profile_read(ex.ctx))
    torch.cuda.synchronize(dev)
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    return ms, {nm: statistics.mean(s_[k] for s_ in stage) for k, nm in enumerate(STAGES)}


def stage_bytes_ms(ab, stage_ms):
    """Stage times grouped like the algorithmic bytes (count = plan + pieces)."""
    ms = {"tag_scan": stage_ms["tag_scan"], "count": stage_ms["plan"] + stage_ms["pieces"],
          "prim_scan": stage_ms["prim_scan"], "emit": stage_ms["emit"]}
    return ms, ab["stages"]


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
            wall = oracle_timed(pool, jobs)[0]
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

    full = rank == 0 and world == 1 and not args.lite
    extra = full and not args.no_extra
    # the other workloads (generated once: the oracle samples and the GPU legs share them)
    cs = W.curvature_stress() if full else None
    mm = W.mmark_like(n_paths=60_000) if full else None
    pr1 = W.concat([W.hand_cases(), W.pr1()]) if full else None
    doc_scenes = W.documents() if extra else None
    pool_scenes = W.serving_pool() if extra else None

    # CPU baseline first (spawned pool, before any GPU work): the oracle timed on the
    # whole workload, on one thread, and its results on a bounded sample of every
    # configuration (work counters for the arithmetic roofline, references for the
    # error statistics of the GPU outline)
    cpu_baseline, refs, work = None, {}, {}
    if full and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        pool = oracle_pool(cores)
        wall, _, fits, verts = oracle_timed(pool, oracle_jobs(scene, TOL, False, chunks=4 * cores))
        work["map_like"] = (fits, verts, n_seg)
        # the same oracle on one host thread, in this process, on every 8th path
        one = scene.subset(range(0, scene.n_paths, 8))
        wall1 = _oracle_chunk(oracle_jobs(one, TOL, False, chunks=1)[0])[0]
        samples = {"map_like": (scene.subset(range(0, scene.n_paths, 16)), TOL, False, False),
                   "map_like_arcs": (scene.subset(range(0, scene.n_paths, 16)), TOL, True, False),
                   "map_like_refined": (scene.subset(range(0, scene.n_paths, 16)), TOL, False, True),
                   "curvature_stress": (cs.subset(range(0, cs.n_paths, 50)), 0.25, False, False),
                   "mmark_like": (mm.subset(range(0, mm.n_paths, 10)), 0.25, False, False),
                   "pr1": (pr1, 0.25, False, False)}
        if extra:
            samples["batched"] = (W.concat(doc_scenes[::32]), TOL, False, False)
            samples["served"] = (W.concat([d.subset(range(0, d.n_paths, 64)) for d in pool_scenes]), TOL, False, False)
        jobs = [(k, v[0], v[1], v[2], v[3]) for k, v in samples.items()]
        for name, r in pool.map(_oracle_reference, jobs):
            refs[name] = r
        pool.close()
        for k, (sc_, _, _, _) in samples.items():
            work.setdefault(k, (refs[k]["n_fit"], refs[k]["n_vert"], sc_.n_segments))
        cpu_baseline = {"value": n_seg / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                        "sample": f"the whole workload ({n_seg} segments) once, {cores} spawned worker processes",
                        "one_thread": {"value": one.n_segments / wall1, "unit": UNIT, "cores": 1,
                                       "sample": f"every 8th path ({one.n_segments} segments) once, in-process"}}

    def scaled_work(name, segs):
        """Fit attempts and vertices of a configuration, from the oracle's counters on
        its sample scaled by segments."""
        if name not in work:
            return None, None
        f, v, s_ = work[name]
        return f * segs / s_, v * segs / s_

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count

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
    ms, stage_ms = timed_expansions(ex, B, ds, params, desc, args.steps, stream, flush, torch, dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    if world > 1:
        ms = max_over_ranks(ms, torch, dev)
    code, _ = B.se_sync(ex.ctx)
    assert code == B.SE_OK, code

    stats = B.se_ctx_stats(ex.ctx)
    n_tags = int(stats["n_tags"])
    n_words = int(enc.points.size)
    n_items = int(stats["n_items"])
    hbm, peak_kind = _peaks()
    sm_mhz = 2070.0   # the GB300's maximum SM clock: the ALU peaks are the hardware's

    def sizes_of(e, prims, tags):
        return dict(n_tags=tags, n_words=int(e.points.size), n_styles=int(e.styles.size), n_paths=int(e.n_paths),
                    n_prims=int(prims), n_input_tags=int(e.tags.size), n_dashes=int(e.dashes.size),
                    n_xforms=0 if e.transforms is None else int(e.transforms.shape[0]))

    def roofline_cfg(name, sz, ms_, arcs=False, stage_ms_=None, segs=None, traffic=None):
        ab = algo_bytes(sz["n_tags"], sz["n_words"], sz["n_styles"], sz["n_paths"], sz["n_prims"], arcs,
                        sz.get("n_input_tags"), sz.get("n_dashes", 0), sz.get("n_xforms", 0))
        fits, verts = scaled_work(name, segs)
        sm_, sb_ = stage_bytes_ms(ab, stage_ms_) if stage_ms_ else (None, None)
        return roofline_of(ab["total"], fits or 0.0, verts or 0.0, ms_, hbm, n_sms, sm_mhz, sm_, sb_, traffic)

    main_sz = sizes_of(enc, n_prims, n_tags)
    roof_step = roofline_cfg("map_like", main_sz, ms, False, stage_ms, n_seg)
    # the dominant kernel stage (the emit): its algorithmic bytes are the outline it
    # writes, its arithmetic the output vertices
    emit_ms = stage_ms["emit"]
    _, verts_m = scaled_work("map_like", n_seg)
    emit_bytes = 20 * n_prims
    traffic = traffic_from_profiles("emit_kernels_map_like_20k_tol0.1_lines.md", n_prims)
    roofline = roofline_of(emit_bytes, 0.0, verts_m or 0.0, emit_ms, hbm, n_sms, sm_mhz, traffic=traffic)
    roofline["kernel"] = "emit stage (emit_pieces_kernel + emit_tails_kernel), map-like lines"
    roofline["peak_source"] = peak_kind + " HBM copy (MEASURED_PEAKS.json); " + roofline["peak_source"].split("; ")[1]
    roofline["units"] = {"prims": n_prims, "items": n_items, "pieces": n_items - n_tags, "tags": n_tags}

    if args.lite:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": job_value(n_seg, world, ms), "unit": UNIT,
                              "ms_per_step": ms, "stage_ms": stage_ms, "roofline": roofline,
                              "roofline_step": roof_step, "config": config, "lite": True}), flush=True)
        ex.close()
        return 0

    def gpu_outline(scene_, tol, arcs=False, refine=False):
        """The GPU outline of a sample scene: primitives and per-tag offsets (host)."""
        o = ex.expand(ex.upload(P.encode(scene_)), tol, arcs, refine=refine)
        return o.prims.cpu().numpy(), o.tag_offset.cpu().numpy()

    def oracle_error(name, scene_, tol, arcs=False, refine=False):
        if name not in refs:
            return None
        from oracle.parity import outline_error
        g, toff = gpu_outline(scene_, tol, arcs, refine)
        e = outline_error(refs[name], g, toff, tol, scene_)
        e["sample"] = f"{scene_.n_paths} paths, {scene_.n_segments} segments"
        return e

    configs = {}

    def time_scene(name, sc_, tol, arcs=False, refine=False, steps=20):
        e_ = P.encode(sc_)
        d_ = ex.upload(e_)
        p_ = P.make_params(tol, arcs=arcs, refine=refine)
        n_ = ex.count(d_, tol, arcs=arcs, refine=refine)
        t_ = ex.expanded_tags(d_)
        b_ = ex.alloc(d_, n_, arcs, t_)
        de_ = ex.outline_desc(b_, n_)
        for _ in range(3):
            ex.expand_async(d_, p_, de_)
        torch.cuda.synchronize(dev)
        ms_, st_ = timed_expansions(ex, B, d_, p_, de_, steps, stream, flush, torch, dev)
        code_, n_chk = B.se_sync(ex.ctx)
        assert code_ == B.SE_OK and n_chk == n_, (code_, n_chk, n_)
        return {"value": sc_.n_segments / (ms_ * 1e-3), "unit": UNIT, "ms_per_step": ms_, "output_prims": n_,
                "stage_ms": st_, "sizes": sizes_of(e_, n_, t_)}

    # map-like: lines (the headline), arcs and the refined mode
    configs["map_like"] = {"workload": config["workload"], "value": n_seg / (ms * 1e-3), "unit": UNIT,
                           "ms_per_step": ms, "output_prims": n_prims, "stage_ms": stage_ms, "roofline": roof_step,
                           "oracle_error": None}
    sample_map = scene.subset(range(0, scene.n_paths, 16))
    c = time_scene("map_like_arcs", scene, TOL, arcs=True)
    c.update(workload=config["workload"].replace("line output", "arc output"),
             roofline=roofline_cfg("map_like_arcs", c["sizes"], c["ms_per_step"], True, c["stage_ms"], n_seg),
             oracle_error=oracle_error("map_like_arcs", sample_map, TOL, arcs=True))
    configs["map_like_arcs"] = c
    c = time_scene("map_like_refined", scene, TOL, refine=True)
    c.update(workload=config["workload"].replace("line output", "refined line output (Section 4.2)"),
             output_prims_vs_fast=c["output_prims"] / n_prims,
             roofline=roofline_cfg("map_like_refined", c["sizes"], c["ms_per_step"], False, c["stage_ms"], n_seg),
             oracle_error=oracle_error("map_like_refined", sample_map, TOL, refine=True))
    configs["map_like_refined"] = c
    configs["map_like"]["oracle_error"] = oracle_error("map_like", sample_map, TOL)
    # curvature stress (100,000 dashed single cubics, tol 0.25), MotionMark-like, PR1 + hand cases
    c = time_scene("curvature_stress", cs, 0.25, steps=10)
    c.update(workload=f"curvature stress: {cs.n_paths} dashed single-cubic paths [10, 5], tol 0.25, lines",
             roofline=roofline_cfg("curvature_stress", c["sizes"], c["ms_per_step"], False, c["stage_ms"],
                                   cs.n_segments),
             oracle_error=oracle_error("curvature_stress", cs.subset(range(0, cs.n_paths, 50)), 0.25))
    configs["curvature_stress"] = c
    c = time_scene("mmark_like", mm, 0.25)
    c.update(workload=f"MotionMark-like: {mm.n_paths} paths, {mm.n_segments} line/quadratic/cubic segments, "
                      f"scaled x2.61 by a transform, tol 0.25, lines",
             roofline=roofline_cfg("mmark_like", c["sizes"], c["ms_per_step"], False, c["stage_ms"], mm.n_segments),
             oracle_error=oracle_error("mmark_like", mm.subset(range(0, mm.n_paths, 10)), 0.25))
    configs["mmark_like"] = c
    c = time_scene("pr1", pr1, 0.25)
    c.update(workload=f"PR1: 200 open stroked paths of 8-32 cubics and the 20 hand cases ({pr1.n_segments} "
                      f"segments), tol 0.25, lines (latency-bound: a parity configuration)",
             roofline=roofline_cfg("pr1", c["sizes"], c["ms_per_step"], False, c["stage_ms"], pr1.n_segments),
             oracle_error=oracle_error("pr1", pr1, 0.25))
    configs["pr1"] = c

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

    batched = served = None
    if extra:
        batched = measure_batched(ex, P, B, W, torch, dev, stream, flush, doc_scenes)
        bsz = dict(batched["sizes"])
        bsz["n_tags"] = bsz["n_input_tags"]
        batched["roofline"] = roofline_cfg("batched", bsz, batched["ms_per_step"], False, None,
                                           bsz["n_segments"])
        batched["oracle_error"] = oracle_error("batched", W.concat(doc_scenes[::32]), TOL)
        served = measure_served(ex, P, B, W, torch, dev, pool_scenes)
        # the served capacity against the bounds of the pool's mean request
        ssz = served["sizes"]
        seg_s = served["capacity"]["value"]
        served["roofline"] = roofline_cfg("served", ssz, 1e3 * ssz["n_segments"] / seg_s, False, None,
                                          ssz["n_segments"])
        served["roofline"]["note"] = "the pool's documents once each at the capacity rate"
        served["oracle_error"] = oracle_error(
            "served", W.concat([d.subset(range(0, d.n_paths, 64)) for d in pool_scenes]), TOL)

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
                "roofline": roofline,
                "roofline_step": roof_step,
                "configs": configs,
                "count_vs_tolerance": sweep,
                "coverage": cov,
                "batched": batched,
                "served": served,
                "host_encode_ms": encode_ms,
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
