"""The object form of the boundary (library-owned scenes and outlines): a scene
built path by path, or from encoded streams, expands to exactly what the
caller-buffer entry points give; batches of scenes share one buffer."""
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


def _scene():
    sc = W.concat([W.hand_cases(), W.pr1(seed=3, n_paths=30), W.map_like(seed=6, n_paths=80, dash_frac=0.3)])
    return sc.as_fill(np.arange(sc.n_paths) % 7 == 3)


@pytest.mark.parametrize("arcs", [False, True])
def test_builder_scene_matches_caller_buffers(ex, arcs):
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    sc = _scene()
    ref = ex.expand(ex.upload(P.encode(sc)), 0.25, arcs)
    h = B.scene_from_verbs(ex.ctx, sc)
    o = B.se_scene_expand(ex.ctx, h, 0.25, arcs)
    code, n, npaths = B.se_outline_sync(o)
    assert code == B.SE_OK and n == ref.n and npaths == sc.n_paths
    prims, curv, poff = B.se_outline_copy(o, n, npaths, arcs)
    assert np.array_equal(prims, ref.prims.cpu().numpy())
    if arcs:
        assert np.array_equal(curv, ref.curvature.cpu().numpy())
    assert np.array_equal(poff, ref.path_offset.cpu().numpy().astype(np.uint64))
    dp, dc, dpo = B.se_outline_device(o)
    assert dp and dpo and (bool(dc) == arcs)
    B.se_outline_destroy(o)
    B.se_scene_destroy(h)


def test_scene_from_streams_and_batches(ex):
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    docs = [W.map_like(seed=20 + k, n_paths=15 + 10 * k, dash_frac=0.2) for k in range(6)]
    handles, refs = [], []
    for d in docs:
        enc = P.encode(d)
        handles.append(B.se_scene_from_streams(ex.ctx, enc.tags, enc.points, enc.styles, enc.n_paths, enc.dashes))
        refs.append(ex.expand(ex.upload(enc), 0.1).prims.cpu().numpy())
    outs = B.se_expand_batch(ex.ctx, handles, 0.1)
    for o, d, ref in zip(outs, docs, refs):
        code, n, npaths = B.se_outline_sync(o)
        assert code == B.SE_OK and npaths == d.n_paths and n == ref.shape[0]
        prims, _, poff = B.se_outline_copy(o, n, npaths)
        assert np.array_equal(prims, ref) and poff[0] == 0 and poff[-1] == n
    for o in outs:
        B.se_outline_destroy(o)
    for h in handles:
        B.se_scene_destroy(h)


def test_builder_errors(ex):
    from paper_2405_00127_gb300 import binding as B
    h = B.se_scene_begin(ex.ctx)
    with pytest.raises(B.SeError):
        B.se_move_to(h, 0, 0)                 # no open path
    st = np.zeros(1, B.STYLE_DTYPE)
    st["half_width"] = 1.0
    st["miter_limit"] = 4.0
    B.se_path_begin(h, st)
    with pytest.raises(B.SeError):
        B.se_line_to(h, 1, 1)                 # a path starts with move_to
    with pytest.raises(B.SeError):
        B.se_move_to(h, float("nan"), 0)
    B.se_move_to(h, 0, 0)
    B.se_line_to(h, 5, 0)
    B.se_path_end(h)
    with pytest.raises(B.SeError):
        B.se_path_end(h)                      # no open path
    o = B.se_scene_expand(ex.ctx, h, 0.25)
    code, n, npaths = B.se_outline_sync(o)
    assert code == B.SE_OK and npaths == 1 and n > 0
    with pytest.raises(B.SeError):
        B.se_line_to(h, 1, 1)                 # uploaded: no longer being built
    B.se_outline_destroy(o)
    B.se_scene_destroy(h)


def test_served_scene(ex):
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    sc = W.map_like(seed=31, n_paths=60, dash_frac=0.3)
    ref = ex.expand(ex.upload(P.encode(sc)), 0.1).prims.cpu().numpy()
    h = B.scene_from_verbs(ex.ctx, sc)
    srv = P.Server(0, slots=2, max_batch_docs=4, hbm_budget=1 << 30)
    try:
        rid = B.se_server_submit_scene(srv.handle, h, 0.1)
        res = srv.poll(rid, wait=True)
        assert res["status"] == 0
        assert np.array_equal(srv.prims(res).cpu().numpy(), ref)
        srv.release(rid)
    finally:
        srv.close()
        B.se_scene_destroy(h)


def test_outlines_in_flight_on_one_context(ex):
    """A second expansion on the context settles the first outline's read-back."""
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    scs = [W.map_like(seed=41, n_paths=40, dash_frac=0.5), W.pr1(seed=42, n_paths=25)]
    refs = [ex.expand(ex.upload(P.encode(s)), 0.2).prims.cpu().numpy() for s in scs]
    hs = [B.scene_from_verbs(ex.ctx, s) for s in scs]
    outs = [B.se_scene_expand(ex.ctx, h, 0.2) for h in hs]
    for o, s, ref in zip(reversed(outs), reversed(scs), reversed(refs)):
        code, n, npaths = B.se_outline_sync(o)
        assert code == B.SE_OK and n == ref.shape[0] and npaths == s.n_paths
        prims, _, _ = B.se_outline_copy(o, n, npaths)
        assert np.array_equal(prims, ref)
    for o in outs:
        B.se_outline_destroy(o)
    for h in hs:
        B.se_scene_destroy(h)
