"""Batched expansion (C ABI se_batch_*) and launch tuning on the GPU.

A batch must give every document exactly the primitives that expanding it alone
gives (the steps are per segment and the only cross-segment sums are integer
scans), whether it runs as one launch sequence or from a captured CUDA graph;
the launch shapes chosen by the autotuner must not change any result."""
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


def _docs(ex, n, dash_frac, seed=41):
    import paper_2405_00127_gb300 as P
    scenes = W.documents(seed=seed, n_docs=n, median=150.0, sigma=1.5, max_segs=20_000, dash_frac=dash_frac)
    empty = W._Builder()
    empty.path([W.M(1, 1)], 2)                        # a document with nothing to draw
    scenes.insert(3, empty.build())
    return scenes, [ex.upload(P.encode(s)) for s in scenes]


@pytest.mark.parametrize("dash_frac,arcs", [(0.0, False), (0.3, False), (0.3, True)])
def test_batch_matches_documents_alone(ex, dash_frac, arcs):
    import paper_2405_00127_gb300 as P
    scenes, docs = _docs(ex, 48, dash_frac)
    b = P.Batch(ex, docs)
    b.prepare(0.1, arcs)
    b.expand_async()
    out = b.result()
    assert out.n == b.capacity
    prims = out.prims.cpu().numpy()
    curv = out.curvature.cpu().numpy() if arcs else None
    for d, ds in enumerate(docs):
        lo, hi = b.doc_range(out, d)
        alone = ex.expand(ds, 0.1, arcs)
        assert hi - lo == alone.n, d
        assert np.array_equal(prims[lo:hi], alone.prims.cpu().numpy()), d
        if arcs:
            assert np.array_equal(curv[lo:hi], alone.curvature.cpu().numpy()), d
    b.close()


def test_graph_replay_and_in_place_update(ex):
    import torch
    import paper_2405_00127_gb300 as P
    scenes, docs = _docs(ex, 32, 0.3, seed=43)
    b = P.Batch(ex, docs)
    b.prepare(0.1)
    b.expand_async()
    ref = b.result().prims.clone()
    b.capture()
    for _ in range(2):
        b.launch()
        out = b.result()
        assert torch.equal(out.prims, ref)
    # move one document by a power of two in place (same sizes): the replay sees it
    d = 5
    docs[d].points.view(torch.float32).add_(64.0)    # a 32-bit stream: the words are the coordinates
    b.launch()
    out = b.result()
    lo, hi = b.doc_range(out, d)
    alone = ex.expand(docs[d], 0.1)
    assert hi - lo == alone.n
    assert torch.equal(out.prims[lo:hi], alone.prims)
    b.close()


def test_autotune_keeps_results(ex):
    import torch
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    sc = W.map_like(seed=44, n_paths=1500, dash_frac=0.2)
    ds = ex.upload(P.encode(sc))
    n = ex.count(ds, 0.1)
    bufs = ex.alloc(ds, n, False, ex.expanded_tags(ds))
    desc = ex.outline_desc(bufs, n)
    params = P.make_params(0.1)
    ref = ex.expand(ds, 0.1).prims.clone()
    chosen = B.se_autotune(ex.ctx, ds.desc, params, desc, reps=2)
    assert chosen["emit_block"] in (64, 128) and chosen["plan_block"] in (64, 128, 256)
    assert chosen["piece_block"] in (64, 128, 256) and chosen["emit_blocks_per_sm"] <= 4
    for t in ({"emit_block": 64, "emit_blocks_per_sm": 1, "piece_block": 64, "plan_block": 256},
              {"emit_block": 128, "emit_blocks_per_sm": 0, "piece_block": 256, "plan_block": 64}, chosen):
        B.se_set_tuning(ex.ctx, **t)
        out = ex.expand(ds, 0.1)
        assert torch.equal(out.prims, ref), t
    with pytest.raises(B.SeError):
        B.se_set_tuning(ex.ctx, emit_block=96)
    B.se_set_tuning(ex.ctx, **chosen)


def test_capture_needs_a_counted_workspace(ex):
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    fresh = P.StrokeExpander(0)
    try:
        scenes, docs = _docs(fresh, 8, 0.0, seed=45)
        b = P.Batch(fresh, docs)
        b.params = P.make_params(0.1)
        t = fresh.torch
        prims = t.empty((1 << 16, 4), dtype=t.float32, device=fresh.device)
        b.desc = B.se_outline_dev(prims.data_ptr(), 0, 0, 0, 0, 1 << 16)
        with pytest.raises(B.SeError) as ei:
            b.capture()
        assert ei.value.code == B.SE_ERR_WORKSPACE
        b.close()
    finally:
        fresh.close()
