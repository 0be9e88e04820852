"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and compare
it with the FP64 oracle segment by segment."""
from __future__ import annotations

import numpy as np

import oracle
from exact_gate import gate_applies, gate_segments
from oracle.parity import prim_tolerance, vertex_tol  # noqa: F401  (the per-vertex tolerance model)

# A logical segment is "fragile" when one of its decisions (fit accept, a
# ceil(), a sign test) lies within this relative distance of its boundary:
# FP32 and FP64 may then legitimately take different branches, so only the
# geometric checks apply to it.
FRAGILE = 1e-4


def run_gpu(ex, scene, tol, arcs=False, refine=False):
    import paper_2405_00127_gb300 as P
    enc = P.encode(scene)
    ds = ex.upload(enc)
    out = ex.expand(ds, tol, arcs, refine=refine)
    prims = out.prims.cpu().numpy().astype(np.float64)
    curv = out.curvature.cpu().numpy().astype(np.float64) if arcs else np.zeros(out.n)
    toff = out.tag_offset.cpu().numpy()
    poff = out.path_offset.cpu().numpy()
    pid = out.path_id.cpu().numpy()
    return dict(prims=prims, curv=curv, tag_offset=toff, path_offset=poff, path_id=pid, n=out.n,
                status=out.status, enc=enc)


def compare(ex, scene, tol, arcs=False, ref=None, refine=False, exact=True):
    """Returns a report dict; raises AssertionError with details on any parity failure.

    Robust segments: counts equal and every vertex within prim_tolerance of the
    oracle's.  Fragile segments (several answers correct): with `exact`, every GPU
    vertex within tol + 1e-3 of the exact geometry (exact_gate)."""
    r = ref if ref is not None else oracle.stroke(scene, tol, arcs=arcs, refine=refine)
    g = run_gpu(ex, scene, tol, arcs, refine)
    # every output coordinate is finite, fragile segments included
    assert np.isfinite(g["prims"]).all() and np.isfinite(g["curv"]).all()
    gc = np.diff(g["tag_offset"])
    oc = r["seg_count"]
    assert gc.size == oc.size, (gc.size, oc.size)
    robust = ~oracle.fragility(r)["any"]
    mism = robust & (gc != oc)
    rep = dict(n_seg=int(oc.size), fragile=int((~robust).sum()), count_mismatch=int(mism.sum()),
               gpu_prims=int(g["n"]), oracle_prims=int(oc.sum()), max_dev=0.0, max_dev_rel=0.0)
    # fragile segments by cause, and how often FP32 took the other branch in each
    frag = oracle.fragility(r)
    for k in ("strict", "cond", "sens"):
        rep[f"fragile_{k}"] = int(frag[k].sum())
        rep[f"fragile_{k}_count_differs"] = int((frag[k] & (gc != oc)).sum())
    if exact and gate_applies(scene) and (~robust).any():
        # fragile segments: every GPU vertex on the exact offset, evolute, join or cap
        st = {}
        n_s, n_v, worst, wseg = gate_segments(scene, r, g["prims"], g["tag_offset"], np.nonzero(~robust)[0], tol,
                                              stats=st)
        rep.update(gated_segments=n_s, gated_vertices=n_v, gate_worst=worst, gate_cusp_clause=st.get("cusp_clause", 0))
        assert worst <= tol + 1e-3, f"fragile segment {wseg}: a GPU vertex lies {worst:.4g} from the exact geometry"
    if mism.any():
        bad = np.nonzero(mism)[0][:10]
        raise AssertionError(f"count mismatch on {mism.sum()} robust segments; first {bad.tolist()}: "
                             f"gpu {gc[bad].tolist()} oracle {oc[bad].tolist()} margin {r['seg_margin'][bad].tolist()}")
    # per-primitive comparison on robust segments
    seg_of_oprim = np.repeat(np.arange(oc.size), oc)
    keep_o = robust[seg_of_oprim]
    seg_of_gprim = np.repeat(np.arange(gc.size), gc)
    keep_g = robust[seg_of_gprim]
    O = r["prim"][keep_o]
    G = g["prims"][keep_g]
    assert O.shape[0] == G.shape[0]
    if O.shape[0]:
        tolv = prim_tolerance(r, scene)[keep_o]
        dev = np.abs(G[:, :4] - O[:, :4])
        worst = np.argmax((dev / tolv).max(1))
        rep["max_dev"] = float(dev.max())
        rep["max_dev_rel"] = float((dev / tolv).max())
        if not np.all(dev <= tolv):
            i = worst
            raise AssertionError(f"vertex deviation {dev[i].max():.3g} > tol {tolv[i].min():.3g} at robust prim {i}: "
                                 f"gpu {G[i, :4].tolist()} oracle {O[i, :4].tolist()} kind {r['prim_kind'][keep_o][i]}")
        if arcs:
            # compare arcs by their sagitta c^2 kappa / 8 (the geometry the curvature
            # encodes): the three-point curvature of a tiny arc is itself ill-conditioned
            c2 = (O[:, 2] - O[:, 0]) ** 2 + (O[:, 3] - O[:, 1]) ** 2
            sag = np.abs(g["curv"][keep_g] - O[:, 4]) * c2 / 8
            ok = sag <= tolv.max(1)
            rep["max_sagitta_dev"] = float(sag.max())
            assert np.all(ok), f"arc sagitta deviation {sag.max()}"
    return rep, g, r


def closed_per_path(g):
    """GPU output: every endpoint leaves as often as it enters, per path, bit-exact."""
    from geom import balanced
    P = g["prims"].astype(np.float32)
    po = g["path_offset"]
    bad = []
    for p in range(po.size - 1):
        if not balanced(P[po[p]:po[p + 1], :4]):
            bad.append(p)
    return bad
