"""The serving loop (C ABI se_server_*) on the GPU: continuous batching of
requests over several slots under an HBM budget.  Every request's result must be
the same as expanding its document alone (bit-identical: the batch steps are per
segment and the only cross-segment sums are integer scans), whatever batch it
ran in and whatever ran beside it."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00127_gb300 import build
    build.build()
    import paper_2405_00127_gb300 as P
    e = P.StrokeExpander(0)
    yield e
    e.close()


@pytest.fixture(scope="module")
def pool(ex):
    import paper_2405_00127_gb300 as P
    scenes = W.documents(seed=61, n_docs=40, median=400.0, sigma=1.5, max_segs=30_000, dash_frac=0.3)
    return [ex.upload(P.encode(s)) for s in scenes]


def _alone(ex, ds, tol, arcs=False):
    out = ex.expand(ds, tol, arcs)
    return out.prims.cpu().numpy(), (out.curvature.cpu().numpy() if arcs else None)


def test_results_in_the_mix_equal_alone(ex, pool):
    import paper_2405_00127_gb300 as P
    srv = P.Server(0, slots=3, max_batch_docs=8, hbm_budget=8 << 30)
    try:
        rids = [srv.submit(ds, 0.1) for ds in pool]
        for rid, ds in zip(rids, pool):
            res = srv.poll(rid, wait=True)
            assert res["done"] and res["status"] == 0
            got = srv.prims(res).cpu().numpy()
            ref, _ = _alone(ex, ds, 0.1)
            assert np.array_equal(got, ref)
            assert res["t_submit_ns"] <= res["t_start_ns"] <= res["t_done_ns"]
            srv.release(rid)
        st = srv.stats()
        assert st["completed"] == len(pool) and st["failed"] == 0
        assert st["batches"] < len(pool)          # requests were batched
        assert st["max_concurrent"] >= 2          # batches overlapped on the device
        assert st["bytes_in_use"] == 0
    finally:
        srv.close()


def test_mixed_parameters_and_arcs(ex, pool):
    import paper_2405_00127_gb300 as P
    srv = P.Server(0, slots=2, max_batch_docs=16, hbm_budget=8 << 30)
    try:
        jobs = []
        for i, ds in enumerate(pool[:24]):
            tol, arcs = [(0.1, False), (0.25, False), (0.1, True)][i % 3]
            jobs.append((srv.submit(ds, tol, arcs), ds, tol, arcs))
        for rid, ds, tol, arcs in jobs:
            res = srv.poll(rid, wait=True)
            assert res["status"] == 0
            ref, ref_k = _alone(ex, ds, tol, arcs)
            assert np.array_equal(srv.prims(res).cpu().numpy(), ref)
            if arcs:
                assert np.array_equal(srv.curvature(res).cpu().numpy(), ref_k)
            srv.release(rid)
    finally:
        srv.close()


def test_budget_admission(ex, pool):
    """With a budget a little above the largest single request, requests still all
    complete, but never more than the budget is held; a budget below a request's
    own size rejects that request."""
    import paper_2405_00127_gb300 as P
    sizes = []
    for ds in pool[:12]:
        n = ex.count(ds, 0.1)
        sizes.append(n * 16 + ds.n_tags * 12 + 4096)
    budget = int(max(sizes) * 1.6) + (1 << 20)
    srv = P.Server(0, slots=3, max_batch_docs=4, hbm_budget=budget)
    try:
        rids = [srv.submit(ds, 0.1) for ds in pool[:12]]
        for rid, ds in zip(rids, pool[:12]):
            res = srv.poll(rid, wait=True)
            assert res["status"] == 0
            ref, _ = _alone(ex, ds, 0.1)
            assert np.array_equal(srv.prims(res).cpu().numpy(), ref)
            srv.release(rid)
        st = srv.stats()
        assert st["bytes_peak"] <= budget and st["bytes_in_use"] == 0
        assert srv.last_error() == ""
    finally:
        srv.close()
    big = max(range(len(pool)), key=lambda i: pool[i].n_tags)
    srv = P.Server(0, slots=1, max_batch_docs=4, hbm_budget=1 << 16)
    try:
        rid = srv.submit(pool[big], 0.1)
        res = srv.poll(rid, wait=True)
        from paper_2405_00127_gb300 import binding as B
        assert res["status"] == B.SE_ERR_BUDGET and res["n_prims"] == 0
        assert "budget" in srv.last_error()
        srv.release(rid)
    finally:
        srv.close()


def test_requests_arriving_while_others_run(ex, pool):
    """Requests submitted over time (not all at once) are picked up by free slots
    while earlier batches run; all complete with correct results."""
    import paper_2405_00127_gb300 as P
    srv = P.Server(0, slots=2, max_batch_docs=8, hbm_budget=8 << 30)
    try:
        rids = []
        for ds in pool:
            rids.append(srv.submit(ds, 0.1))
            time.sleep(0.0005)
        for rid, ds in zip(rids, pool):
            res = srv.poll(rid, wait=True)
            ref, _ = _alone(ex, ds, 0.1)
            assert res["status"] == 0 and np.array_equal(srv.prims(res).cpu().numpy(), ref)
            srv.release(rid)
        assert srv.stats()["completed"] == len(pool)
    finally:
        srv.close()


_FIRST_LAUNCHES = r"""
import sys
sys.path.insert(0, sys.argv[1])
import workloads as W
import paper_2405_00127_gb300 as P
ex = P.StrokeExpander(0)
docs = [ex.upload(P.encode(W.map_like(seed=40 + k, n_paths=200))) for k in range(32)]
srv = P.Server(0, slots=8, max_batch_docs=2)
rids = [srv.submit(d, 0.1) for d in docs] + [srv.submit(d, 0.1, arcs=True) for d in docs]
bad = []
for rid in rids:
    r = srv.poll(rid, wait=True)
    if r["status"] != 0:
        bad.append((r["status"], srv.last_error()))
    srv.release(rid)
srv.close()
print("FAILED" if bad else "OK", bad[:3])
"""


def test_concurrent_first_launches():
    """A fresh process whose first expansions all start at once on eight worker
    threads: the emit grids' launch shape is set up once per device and kernel,
    never read half-written (such a read launched empty grids: an invalid
    argument on a batch)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", _FIRST_LAUNCHES, root], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0 and "OK" in r.stdout, (r.stdout[-800:], r.stderr[-800:])
