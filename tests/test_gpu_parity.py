"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, segment by
segment, on seeded synthetic scenes spanning several scan tiles and ragged tails."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import closed_per_path, compare, prim_tolerance, run_gpu

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


@pytest.mark.parametrize("arcs", [False, True])
def test_hand_cases(ex, oracle_mod, arcs):
    rep, g, _ = compare(ex, W.hand_cases(), 0.25, arcs)
    assert closed_per_path(g) == []
    print(rep)


@pytest.mark.parametrize("arcs", [False, True])
def test_pr1(ex, oracle_mod, arcs):
    sc = W.pr1()
    rep, g, r = compare(ex, sc, 0.25, arcs)
    assert rep["fragile"] <= 0.03 * rep["n_seg"]
    assert closed_per_path(g) == []
    # path ids and path offsets agree with the per-tag layout
    po = g["path_offset"]
    assert po[0] == 0 and po[-1] == g["n"]
    assert np.array_equal(g["path_id"], np.repeat(np.arange(sc.n_paths), np.diff(po)))
    print(rep)


@pytest.mark.parametrize("arcs", [False, True])
def test_map_like_small(ex, oracle_mod, arcs):
    # ~9k tags: spans three 4096-tag scan tiles with a ragged tail
    sc = W.map_like(seed=12, n_paths=300)
    rep, g, _ = compare(ex, sc, 0.1, arcs)
    assert closed_per_path(g) == []
    print(rep)


def test_curvature_stress_solid(ex, oracle_mod):
    sc = W.curvature_stress(seed=13, n_paths=400, dashed=False)
    rep, g, _ = compare(ex, sc, 0.25, False)
    assert closed_per_path(g) == []
    print(rep)


def test_map_like_full_size_sampled(ex, oracle_mod):
    """The bench workload (50,000 paths, tol 0.1) in one launch sequence; a seeded
    sample of its paths is checked against the oracle run on those paths alone:
    robust segments by count and per vertex, fragile ones by the exact-geometry gate."""
    from exact_gate import gate_segments, logical_sources, pieces_by_seg
    sc = W.map_like()
    g = run_gpu(ex, sc, 0.1)
    po = g["path_offset"]
    assert po[-1] == g["n"]
    last_tag = np.nonzero(g["enc"].tags & 0x10)[0]          # SE_TAG_PATH: last tag of a path
    first_tag = np.concatenate([[0], last_tag[:-1] + 1])
    toff = g["tag_offset"]
    rng = np.random.default_rng(99)
    sample = np.sort(rng.choice(sc.n_paths, 200, replace=False))
    sub = sc.subset(sample)
    r = oracle.stroke(sub, 0.1)
    tolv = prim_tolerance(r, sub)
    lsrc, pieces = logical_sources(sub, r), pieces_by_seg(r)
    robust = ~oracle.fragility(r)["any"]
    n_robust = n_gated = 0
    worst = 0.0
    for j, p in enumerate(sample):
        segs = np.nonzero(r["seg_path"] == j)[0]
        assert segs.size == last_tag[p] - first_tag[p] + 1, p
        for k, i in enumerate(segs):
            t = first_tag[p] + k
            gp = g["prims"][toff[t]:toff[t + 1]]
            if robust[i]:
                o = r["prim"][r["seg_first_prim"][i]:r["seg_first_prim"][i] + r["seg_count"][i]]
                assert gp.shape[0] == o.shape[0], (p, k)
                tv = tolv[r["seg_first_prim"][i]:r["seg_first_prim"][i] + r["seg_count"][i]]
                assert np.all(np.abs(gp[:, :4] - o[:, :4]) <= tv), (p, k)
                n_robust += 1
            else:
                _, _, w, _ = gate_segments(sub, r, g["prims"], toff, [i], 0.1, tag_base=t, r_seg_base=i,
                                           lsrc=lsrc, pieces=pieces)
                worst = max(worst, w)
                n_gated += 1
    assert worst <= 0.1 + 1e-3, worst
    assert n_robust + n_gated == r["seg_kind"].size
    print(f"robust segments compared {n_robust}, fragile segments gated {n_gated}, worst gate distance {worst:.3g}")


def test_edge_cases(ex, oracle_mod):
    b = W._Builder()
    b.path([W.M(5, 5)], 2)                                   # empty path
    b.path([W.M(1, 1), W.L(1, 1)], 3, cap=W.CAP_ROUND)       # dot
    b.path([W.M(1, 1), W.L(1, 1)], 3, cap=W.CAP_SQUARE)      # square dot
    b.path([W.M(1, 1), W.L(1, 1)], 3, cap=W.CAP_BUTT)        # butt dot: nothing
    b.path([W.M(0, 0), W.L(0.001, 0)], 50, cap=W.CAP_ROUND)  # tiny segment, huge width
    b.path([W.M(0, 0), W.C(1e4, 0, -1e4, 1, 1, 1)], 0.5)     # extreme handles
    rep, g, _ = compare(ex, b.build(), 0.25, False)
    assert closed_per_path(g) == []


def test_capacity_and_empty_scene(ex):
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    sc = W.hand_cases()
    ds = ex.upload(P.encode(sc))
    n = ex.count(ds, 0.25)
    bufs = ex.alloc(ds, n - 1, False)
    ex.expand_async(ds, P.make_params(0.25), ex.outline_desc(bufs, n - 1))
    code, total = B.se_sync(ex.ctx)
    assert code == B.SE_ERR_CAPACITY and total == n
    # the same context recovers
    out = ex.expand(ds, 0.25)
    assert out.n == n and out.status == B.SE_OK
    empty = W._Builder().build()
    ds0 = ex.upload(P.encode(empty))
    assert ex.count(ds0, 0.25) == 0


def test_malformed_tags_are_reported(ex):
    """A tag stream whose last marker is replaced by a cubic whose control points run
    past the point stream is rejected on the device without any out-of-bounds access
    (every index is checked first)."""
    import torch
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    enc = P.encode(W.hand_cases())
    tags = enc.tags.copy()
    tags[-1] = 0x08 | 0x03 | 0x10   # a cubic (3 new points) where the marker's 2 points end the stream
    enc2 = P.Encoded(tags, enc.points, enc.styles, enc.n_paths, enc.dashes)
    ds = ex.upload(enc2)
    code, _ = B.se_count(ex.ctx, ds.desc, P.make_params(0.25))
    assert code == B.SE_ERR_INVALID_INPUT


def test_deterministic(ex):
    import paper_2405_00127_gb300 as P
    sc = W.map_like(seed=5, n_paths=2000)
    ds = ex.upload(P.encode(sc))
    a = ex.expand(ds, 0.1)
    b = ex.expand(ds, 0.1)
    assert a.n == b.n
    assert bool((a.prims == b.prims).all())


@pytest.mark.parametrize("arcs", [False, True])
def test_host_entry_pipelined_download(ex, arcs):
    """se_expand_host on a scene large enough to emit in tag ranges while earlier
    ranges download: the host outline equals the device expansion bit for bit, and a
    short buffer reports SE_ERR_CAPACITY with the needed count."""
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    sc = W.map_like(seed=44, n_paths=3000, dash_frac=0.2)
    enc = P.encode(sc)
    assert enc.tags.size >= 65536
    ref = ex.expand(ex.upload(enc), 0.1, arcs)
    n = ref.n
    prims = np.zeros((n, 4), np.float32)
    curv = np.zeros(n, np.float32) if arcs else None
    code, got = B.se_expand_host(ex.ctx, enc.tags, enc.points, enc.styles, enc.n_paths, enc.dashes,
                                 P.make_params(0.1, arcs), prims, curv, n)
    assert code == B.SE_OK and got == n
    assert np.array_equal(prims, ref.prims.cpu().numpy())
    if arcs:
        assert np.array_equal(curv, ref.curvature.cpu().numpy())
    small = np.zeros((n // 2, 4), np.float32)
    code, got = B.se_expand_host(ex.ctx, enc.tags, enc.points, enc.styles, enc.n_paths, enc.dashes,
                                 P.make_params(0.1, arcs), small, np.zeros(n // 2, np.float32) if arcs else None, n // 2)
    assert code == B.SE_ERR_CAPACITY and got == n
