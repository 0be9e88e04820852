"""GPU-against-oracle error statistics (TEST INFRASTRUCTURE ONLY: the benchmark's
CPU-baseline leg reports them; the CUDA library never imports this).

Given the FP64 oracle's result for a scene and the FP32 outline the GPU wrote
for the same scene (per-tag offsets, one tag per logical segment), it reports

- the fragile segments by cause (see oracle.fragility) and, per cause, how
  many of them the GPU counted differently (the reason each widening of the
  plain 1e-4 rule exists);
- count mismatches on robust segments (the parity bar: zero);
- the vertex deviation |v_gpu - v_oracle| on robust segments: max, mean, p99,
  in scene units and relative to the tolerance.
"""
from __future__ import annotations

import numpy as np

from . import FRAGILE, fragility


def outline_error(r, gpu_prims, gpu_tag_offset, tol):
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
    if O.shape[0] and O.shape[0] == G.shape[0]:
        d = np.abs(G - O).max(1)
        out.update(vertex_dev_max=float(d.max()), vertex_dev_mean=float(d.mean()),
                   vertex_dev_p99=float(np.percentile(d, 99)), vertex_dev_max_over_tol=float(d.max() / tol),
                   compared_prims=int(O.shape[0]))
    return out


__all__ = ["outline_error", "FRAGILE"]
