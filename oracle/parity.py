"""GPU-against-oracle error statistics (TEST INFRASTRUCTURE ONLY: the benchmark's
CPU-baseline leg reports them; the CUDA library never imports this).

Given the FP64 oracle's result for a scene and the FP32 outline the GPU wrote
for the same scene (per-tag offsets, one tag per logical segment), it reports

- the fragile segments by cause (see oracle.fragility) and, per cause, how
  many of them the GPU counted differently (the reason each widening of the
  plain 1e-4 rule exists);
- count mismatches on robust segments (the parity bar: zero);
- the vertex deviation |v_gpu - v_oracle| on robust segments: max, mean, p99,
  in scene units, relative to the flattening tolerance, and relative to the
  per-vertex FP32 tolerance (prim_tolerance: the parity bar is <= 1).
"""
from __future__ import annotations

import numpy as np

from . import FRAGILE, fragility


def vertex_tol(coord_mag, scale, cond, evo):
    """Per-vertex GPU/oracle tolerance.  The GPU evaluates each vertex in FP32: a
    handful of roundings at the coordinate magnitude (8 ulp); the FP32 error of the
    ES quadrature, density inverse and trigonometry relative to the piece length plus
    half-width (2e-5 (L + h)); and the FP32 resolution of the piece itself, whose
    tangent angles carry an absolute error of about `cond` (16 cond (L + h)).
    Evolute points e = c + N / kappa add `evo` = 16 cond h^2 / L: the normalised
    curvature k0 + k1 (s - 1/2) takes an absolute error of ~8 cond, and near the
    end of an evolute range (|kappa| >= 1/h) dividing by it moves the point by up to
    8 cond h^2 / L."""
    ulp = np.spacing(np.maximum(np.abs(coord_mag), 1.0).astype(np.float32)).astype(np.float64)
    return 8 * ulp + 2e-5 * scale + 16 * cond * scale + evo + 1e-5


def path_polygon_length(scene):
    """Per path, the length of its control polygon (the polyline through all its
    points in order, an upper bound of every subpath's)."""
    pts = np.asarray(scene.pts, np.float64).reshape(-1, 2)
    po = scene.path_pt_off()
    seg = np.hypot(*np.diff(pts, axis=0).T) if pts.shape[0] > 1 else np.zeros(0)
    csum = np.concatenate([[0.0], np.cumsum(seg)])
    lo, hi = po[:-1], np.maximum(po[1:] - 1, po[:-1])
    return csum[np.minimum(hi, csum.size - 1)] - csum[np.minimum(lo, csum.size - 1)]


def prim_tolerance(r, scene):
    """Per-primitive, per-coordinate GPU/oracle tolerance [n_prim, 4] (vertex_tol)
    from the oracle result r of `scene`.  Primitives of dashed paths add the FP32
    error of their cut positions: the device sums arc length along a subpath from
    panels accepted at 1e-6 of each segment's control-polygon length, so a cut,
    and every vertex of the part it bounds, can move along the curve by up to
    1e-6 of the path's control polygon (2e-6 with the Newton inversion of the
    cut)."""
    piece = r["prim_piece"]
    pc = np.maximum(piece, 0)
    has = piece >= 0
    L = np.where(has, r["piece"][pc, 15], 0.0) if r["piece"].shape[0] else np.zeros(piece.size)
    cond = np.minimum(r["prim_cond"], 1.0)
    seg_of = np.repeat(np.arange(r["seg_count"].size), r["seg_count"])
    pth = r["seg_path"][seg_of]
    hw = np.where(scene.fill[pth] != 0, 0.0, scene.half_width[pth].astype(np.float64))   # a fill has no width
    evo = np.where(np.isin(r["prim_kind"], (2, 3)) & has, 16 * cond * hw ** 2 / np.maximum(L, 1e-30), 0.0)
    scale = L + hw
    O = r["prim"]
    # an FP32 rounding of either coordinate can move both (rotations mix them)
    mag = np.repeat(np.maximum(np.abs(O[:, 0:4:2]), np.abs(O[:, 1:4:2])), 2, axis=1)
    tolv = vertex_tol(mag, scale[:, None], cond[:, None], evo[:, None])
    dashed = np.asarray(scene.dash_count)[pth] != 0
    if dashed.any():
        tolv = tolv + np.where(dashed, 2e-6 * path_polygon_length(scene)[pth], 0.0)[:, None]
    return tolv


def outline_error(r, gpu_prims, gpu_tag_offset, tol, scene=None):
    gc = np.diff(np.asarray(gpu_tag_offset, np.int64))
    oc = r["seg_count"]
    if gc.size != oc.size:
        return {"error": f"tag count {gc.size} != oracle segments {oc.size}"}
    frag = fragility(r)
    robust = ~frag["any"]
    n = int(oc.size)
    out = {"segments": n, "fragile": int(frag["any"].sum()), "fragile_fraction": float(frag["any"].mean()) if n else 0.0,
           "robust_count_mismatch": int((robust & (gc != oc)).sum())}
    for k in ("strict", "cond", "sens"):
        out[f"fragile_{k}"] = int(frag[k].sum())
        out[f"fragile_{k}_gpu_count_differs"] = int((frag[k] & (gc != oc)).sum())
    keep_o = np.repeat(robust, oc)
    keep_g = np.repeat(robust & (gc == oc), gc)
    keep_o &= np.repeat(gc == oc, oc)
    O = r["prim"][keep_o, :4]
    G = np.asarray(gpu_prims, np.float64)[keep_g, :4]
    out["gpu_non_finite"] = int((~np.isfinite(np.asarray(gpu_prims, np.float64)[:, :4])).any(1).sum())
    if O.shape[0] and O.shape[0] == G.shape[0]:
        dev = np.abs(G - O)
        d = dev.max(1)
        out.update(vertex_dev_max=float(d.max()), vertex_dev_mean=float(d.mean()),
                   vertex_dev_p99=float(np.percentile(d, 99)), vertex_dev_max_over_tol=float(d.max() / tol),
                   compared_prims=int(O.shape[0]))
        if scene is not None:
            tolv = prim_tolerance(r, scene)[keep_o]
            out["vertex_dev_max_over_vertex_tol"] = float((dev / tolv).max())
    return out


__all__ = ["outline_error", "prim_tolerance", "vertex_tol", "FRAGILE"]
