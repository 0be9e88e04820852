"""GPU parity of the device dash pass (SVG dash semantics; the paper dashes on the
CPU, Section 9.3): the dashed scene expanded through the C ABI against the FP64
oracle's dashing, segment by segment.  Paths whose dash structure FP32 cannot
decide (a pattern boundary within the arc-length resolution of a segment end)
are left out of the scene before either side runs, so the logical segments of
both sides line up one to one."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import FRAGILE, closed_per_path, compare, prim_tolerance, run_gpu

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


def dash_robust(sc, tol, arcs=False):
    """The scene without its dash-fragile paths, and the oracle's result for it."""
    r = oracle.stroke(sc, tol, arcs=arcs)
    dm = np.full(sc.n_paths, np.inf)
    np.minimum.at(dm, r["seg_path"], r["seg_dash_margin"])
    keep = np.nonzero(dm >= FRAGILE)[0]
    assert keep.size >= 0.97 * sc.n_paths, (sc.n_paths - keep.size)
    sub = sc.subset(keep)
    return sub, oracle.stroke(sub, tol, arcs=arcs)


def hand_dashes():
    b = W._Builder()
    b.path([W.M(0, 0), W.L(100, 0)], 2, cap=W.CAP_BUTT, dash=[10, 5], dash_offset=0.5)
    b.path([W.M(0, 10), W.L(100, 10)], 2, cap=W.CAP_SQUARE, dash=[10, 5], dash_offset=12)
    b.path([W.M(0, 20), W.C(30, 40, 60, 0, 100, 20), W.L(120, 60), W.Z], 2, cap=W.CAP_ROUND,
           join=W.JOIN_MITER, dash=[7, 3, 2], dash_offset=1)
    b.path([W.M(0, 90), W.L(50, 90)], 3, cap=W.CAP_ROUND, dash=[0, 10], dash_offset=0.25)   # dots
    b.path([W.M(0, 99), W.L(5, 99)], 3, dash=[10, 5], dash_offset=11)       # entirely in a gap
    b.path([W.M(0, 120), W.L(40, 120), W.L(40, 160)], 2, join=W.JOIN_ROUND)  # solid among dashed
    b.path([W.M(5, 5)], 2, dash=[3, 1], dash_offset=0)                      # empty path
    b.path([W.M(0, 200), W.C(100, 300, -50, 300, 60, 200)], 4, cap=W.CAP_ROUND, dash=[4, 2.5, 1],
           dash_offset=-3.5)                                                  # negative offset
    b.path([W.M(0, 260), W.L(1, 260)], 2, cap=W.CAP_ROUND, dash=[0, 0])      # zero period: nothing
    return b.build()


@pytest.mark.parametrize("arcs", [False, True])
def test_hand_dashes(ex, oracle_mod, arcs):
    sc, r = dash_robust(hand_dashes(), 0.25, arcs)
    rep, g, _ = compare(ex, sc, 0.25, arcs, ref=r)
    assert closed_per_path(g) == []
    print(rep)


def test_curvature_stress_dashed(ex, oracle_mod):
    sc, r = dash_robust(W.curvature_stress(seed=13, n_paths=400, dashed=True), 0.25)
    rep, g, _ = compare(ex, sc, 0.25, False, ref=r)
    assert closed_per_path(g) == []
    assert rep["fragile"] <= 0.05 * rep["n_seg"]
    print(rep)


@pytest.mark.parametrize("arcs", [False, True])
def test_map_like_partly_dashed(ex, oracle_mod, arcs):
    # ~10k input tags (three scan tiles and a ragged tail), 30% of the paths dashed
    sc, r = dash_robust(W.map_like(seed=12, n_paths=300, dash_frac=0.3), 0.1, arcs)
    rep, g, _ = compare(ex, sc, 0.1, arcs, ref=r)
    assert closed_per_path(g) == []
    print(rep)


def test_dash_rewrite_counts_and_layout(ex, oracle_mod):
    """One tag per logical segment of the oracle; the path offsets cover every path."""
    sc = W.map_like(seed=5, n_paths=1000, dash_frac=1.0)
    g = run_gpu(ex, sc, 0.1)
    po = g["path_offset"]
    assert po[0] == 0 and po[-1] == g["n"] and np.all(np.diff(po) >= 0)
    assert np.array_equal(g["path_id"], np.repeat(np.arange(sc.n_paths), np.diff(po)))
    assert g["tag_offset"][-1] == g["n"]


def test_dashed_deterministic(ex):
    import paper_2405_00127_gb300 as P
    sc = W.curvature_stress(seed=9, n_paths=3000, dashed=True)
    ds = ex.upload(P.encode(sc))
    a = ex.expand(ds, 0.25)
    b = ex.expand(ds, 0.25)
    assert a.n == b.n and bool((a.prims == b.prims).all())


def test_dash_workspace_grows(ex):
    """An expansion enqueued before any count of a heavily dashed scene reports
    SE_ERR_WORKSPACE without writing; after se_count the same call succeeds."""
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    b = W._Builder()
    for k in range(64):
        b.path([W.M(0, 3 * k), W.L(4000, 3 * k)], 0.5, dash=[0.5, 0.5], dash_offset=0)
    sc = b.build()
    fresh = P.StrokeExpander(0)
    try:
        ds = fresh.upload(P.encode(sc))
        bufs = fresh.alloc(ds, 1 << 20, False, n_tags=1 << 20)
        fresh.expand_async(ds, P.make_params(0.25), fresh.outline_desc(bufs, 1 << 20))
        code, _ = B.se_sync(fresh.ctx)
        assert code == B.SE_ERR_WORKSPACE
        out = fresh.expand(ds, 0.25)
        assert out.status == B.SE_OK and out.n > 64 * 4000
    finally:
        fresh.close()


def test_curvature_stress_full_size_sampled(ex, oracle_mod):
    """The full curvature-stress workload (100,000 dashed single-cubic paths) in
    one launch sequence; a seeded sample of its paths against the oracle run on
    those paths alone."""
    sc = W.curvature_stress()
    g = run_gpu(ex, sc, 0.25)
    po = g["path_offset"]
    assert po[-1] == g["n"]
    rng = np.random.default_rng(31)
    sample = np.sort(rng.choice(sc.n_paths, 150, replace=False))
    sub = sc.subset(sample)
    r = oracle.stroke(sub, 0.25)
    robust = np.ones(sample.size, bool)
    np.logical_and.at(robust, r["seg_path"], (~oracle.fragility(r)["any"]) & (r["seg_dash_margin"] >= FRAGILE))
    op = np.concatenate([[0], np.cumsum(np.bincount(np.repeat(r["seg_path"], r["seg_count"]), minlength=sample.size))])
    tolv = prim_tolerance(r, sub)
    checked = 0
    for j, p in enumerate(sample):
        if not robust[j]:
            continue
        gp = g["prims"][po[p]:po[p + 1]]
        o = r["prim"][op[j]:op[j + 1]]
        assert gp.shape[0] == o.shape[0], p
        assert np.all(np.abs(gp[:, :4] - o[:, :4]) <= tolv[op[j]:op[j + 1]]), p
        checked += 1
    assert checked >= 100


def test_dash_parts_below_fp32_resolution_stay_finite(ex, oracle_mod):
    """Two dashed paths of the serving pool whose dash parts are ~1e-4 long at
    coordinates near 2000 (FP32 resolution 2.4e-4): their rewritten end points
    coincide in FP32.  Such a part is one degenerate piece -- not 2^16 halvings
    of a zero chord -- and every vertex is finite."""
    pool = W.serving_pool()
    sample = W.concat([d.subset(range(0, d.n_paths, 64)) for d in pool])
    sc = sample.subset([5887, 6536])
    g = run_gpu(ex, sc, 0.1)
    assert np.isfinite(g["prims"]).all()
    r = oracle.stroke(sc, 0.1)
    # the oracle (FP64 parts, all of nonzero length) and the GPU differ only on the
    # dash-fragile parts; the outline stays the same size
    assert g["n"] < 2 * r["prim"].shape[0]
    assert closed_per_path(g) == []
