"""The exact-geometry gate that judges the GPU's fragile segments, checked on the CPU:
the oracle's own output passes it (every vertex of the hand cases, the fragile
segments of PR1 and of a map-like scene), and vertices moved off the exact
geometry by more than the tolerance fail it."""
import numpy as np
import pytest

import oracle
import workloads as W
from exact_gate import gate_distances, gate_segments, logical_sources, pieces_by_seg


def _oracle_as_gpu(r):
    """The oracle's output in the GPU's layout: rows x0 y0 x1 y1 and per-tag offsets."""
    return r["prim"][:, :4], np.concatenate([[0], np.cumsum(r["seg_count"])])


@pytest.mark.parametrize("which", ["hand", "pr1", "map"])
def test_oracle_output_passes_the_gate(oracle_mod, which):
    if which == "hand":
        sc, tol = W.hand_cases(), 0.25
    elif which == "pr1":
        sc, tol = W.pr1(), 0.25
    else:
        sc, tol = W.map_like(seed=12, n_paths=300), 0.1
    r = oracle.stroke(sc, tol)
    segs = np.arange(r["seg_kind"].size) if which == "hand" else np.nonzero(oracle.fragility(r)["any"])[0]
    assert segs.size > 0
    prims, toff = _oracle_as_gpu(r)
    st = {}
    _, nv, worst, _ = gate_segments(sc, r, prims, toff, segs, tol, stats=st)
    assert st.get("cusp_clause", 0) == 0     # the oracle's own vertices never need the cusp clause
    assert nv > 0 and worst <= tol + 1e-3, worst


def test_displaced_vertices_fail_the_gate(oracle_mod):
    """Every vertex of H6 (circle R 100, h 5), H13 (bevel) and H16 (loop cubic),
    moved by 2 tol across its primitive (along the primitive's normal, either way),
    is caught; a move along the curve stays on the exact geometry and would not be."""
    sc, tol = W.hand_cases(), 0.25
    r = oracle.stroke(sc, tol)
    lsrc, pieces = logical_sources(sc, r), pieces_by_seg(r)
    caught = total = 0
    for path in (5, 12, 15):
        for i in np.nonzero((r["seg_path"] == path) & (r["seg_kind"] == 0))[0]:
            a, n = r["seg_first_prim"][i], r["seg_count"][i]
            P = r["prim"][a:a + n, :4]
            V = np.vstack([P[:, :2], P[:, 2:4]])
            h = float(sc.half_width[path])
            assert gate_distances(sc, r, int(i), V, h, lsrc, pieces.get(int(i))).max() <= tol + 1e-3
            d = P[:, 2:4] - P[:, :2]
            ln = np.hypot(d[:, 0], d[:, 1])
            keep = ln > 0
            nrm = np.stack([-d[keep, 1], d[keep, 0]], 1) / ln[keep, None]
            ends = np.vstack([P[keep, :2], P[keep, 2:4]])
            for sgn in (1.0, -1.0):
                moved = ends + sgn * 2 * tol * np.vstack([nrm, nrm])
                dist = gate_distances(sc, r, int(i), moved, h, lsrc, pieces.get(int(i)))
                caught += int(np.count_nonzero(dist > tol + 1e-3))
                total += moved.shape[0]
    # a moved vertex can still land on another part of the exact geometry (the
    # other side of a join, an evolute, a cap); nearly all cannot
    assert caught >= 0.9 * total, (caught, total)
