"""Exact-geometry gate for outline vertices whose count parity is not decidable.

A logical segment whose decisions sit within FP32 resolution of a boundary
("fragile") may legitimately get a different subdivision or primitive count in
FP32 than in the FP64 oracle, so its output is not compared vertex by vertex.
Its vertices must still lie on the exact geometry they stand for:

- the exact parallel curves c(t) +- h n(t) of the source segment (dense FP64
  sampling, refined around derivative minima); at a source cusp or near-cusp
  (Section 7.3) the circle of radius h about the source there, taken as
  | dist(v, source) - h |;
- an evolute: the exact centre-of-curvature locus c + N / kappa of the source,
  where the radius of curvature is at most ~h, or the locus of an Euler-spiral
  fit (Appendix A) of a dyadic parameter range that a near-threshold fit
  decision can give in place of the oracle's pieces (their parents and
  grandparents, and their descendants, down to the depth cap near a cusp);
- a join or cap at the segment's end (Section 8.1): the joint itself (inner
  contour), the circle of radius h about it (round), the miter tips of the
  join for both turn directions, the square-cap corners;
- next to a source cusp only: inside the stroke, within h of the cusp (the
  evolute vertices of pieces below FP32 resolution; counted separately).

gate_distances returns, per vertex, the distance to the nearest of these sets;
the tests require it to be within tol + 1e-3 (the bound on every vertex).
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from geom import bez, bez_d, offset_curve, path_segments, point_polyline_dist


def _rn(T):
    T = np.asarray(T, np.float64)
    return np.array([T[1], -T[0]]) / math.hypot(*T)


def _tangent(c, t):
    d = bez_d(c, t)
    if math.hypot(*d) < 1e-9 * np.abs(np.diff(c, axis=0)).sum():
        # a vanishing derivative: sample toward the inside (Section 7.3)
        d = bez_d(c, t + (1e-3 if t < 0.5 else -1e-3))
    return d


def logical_sources(scene, r):
    """Per logical segment of the oracle result r: (control points or None, index of
    its subpath's first segment among the logical segments, the next logical
    segment index or -1)."""
    src, first, nxt = [], [], []
    segs_by_path, cursor = {}, {}
    sub_first = -1
    n = len(r["seg_kind"])
    for i, (k, p) in enumerate(zip(r["seg_kind"], r["seg_path"])):
        if p not in segs_by_path:
            segs_by_path[p] = path_segments(scene, p)
            cursor[p] = 0
            sub_first = -1
        if k in (0, 1):
            lst = segs_by_path[p]
            while np.allclose(lst[cursor[p]][1], lst[cursor[p]][1][0], atol=0):  # zero-length: skipped
                cursor[p] += 1
            src.append(lst[cursor[p]][1])
            cursor[p] += 1
            if sub_first < 0:
                sub_first = i
        else:
            src.append(None)
        first.append(sub_first)
        if k == 2 or k == 3:
            sub_first = -1
    for i in range(n):
        j = i + 1
        nxt.append(j if j < n and r["seg_path"][j] == r["seg_path"][i] and r["seg_kind"][j] in (0, 1) else -1)
    return src, first, nxt


def _es_evolute_poly(k0, k1, th0, rot, p0, h):
    """Centre-of-curvature locus of an Euler-spiral piece (unit ES mapped by the
    complex factor rot from p0), sampled uniformly in s and in 1/kappa, where the
    radius is at most 4h."""
    Lg = abs(rot)
    if not (Lg > 0):
        return np.zeros((0, 2))
    fine = np.linspace(0, 1, 8001)
    th_f = -th0 + k0 * fine + 0.5 * k1 * (fine * fine - fine)
    zf = np.concatenate([[0], np.cumsum(0.5 * (np.exp(1j * th_f[1:]) + np.exp(1j * th_f[:-1])) * (fine[1] - fine[0]))])
    samp = [np.linspace(0, 1, 4001)]
    if k1 != 0:
        rad = h * np.arange(1, 801) / 400.0
        for sg in (1, -1):
            sj = 0.5 + (sg * Lg / rad - k0) / k1
            samp.append(sj[(sj >= 0) & (sj <= 1)])
    s = np.unique(np.concatenate(samp))
    z = np.interp(s, fine, zf.real) + 1j * np.interp(s, fine, zf.imag)
    z = p0 + z * rot
    th = -th0 + k0 * s + 0.5 * k1 * (s * s - s)
    T = np.exp(1j * th) * rot / Lg
    kap = (k0 + k1 * (s - 0.5)) / Lg
    with np.errstate(divide="ignore", invalid="ignore"):
        ev = z + 1j * T / kap
    ok = np.isfinite(ev) & (np.abs(1 / np.where(kap == 0, np.nan, kap)) <= 4 * h)
    return np.stack([ev.real[ok], ev.imag[ok]], 1)


def _es_fit_poly(c, t0, t1, h):
    """Evolute locus of the Euler-spiral fit (the oracle's Appendix A fit) of the
    source over [t0, t1]."""
    p0, p1 = bez(c, t0), bez(c, t1)
    q0, q1 = _tangent(c, t0), _tangent(c, t1)
    th0, th1, chord, _ = oracle.fit(p0, p1, q0, q1, t1 - t0)
    if not chord > 0:
        return np.zeros((0, 2))
    k0 = th0 + th1
    k1, _ = oracle.gh(k0, th1 - th0)
    # the unit ES end point, by quadrature, maps onto the chord
    fine = np.linspace(0, 1, 8001)
    th_f = -th0 + k0 * fine + 0.5 * k1 * (fine * fine - fine)
    z1 = np.sum(0.5 * (np.exp(1j * th_f[1:]) + np.exp(1j * th_f[:-1])) * (fine[1] - fine[0]))
    ch = complex(*(p1 - p0))
    return _es_evolute_poly(k0, k1, th0, ch / z1, complex(*p0), h)


MAX_DEPTH = 16   # the subdivision depth cap of Algorithm 2 (pieces of 2^-16 at most)


def _fit_ranges(pieces):
    """Dyadic parameter ranges whose Euler-spiral fits a near-threshold decision
    can produce instead of the oracle's pieces: each piece, its parent and
    grandparent (a merge), and its descendants two levels down -- all the way
    to the depth cap for pieces at depth 12 or more, which only occur where the
    fit keeps failing (near a cusp), so that FP32 may subdivide further."""
    out = set()
    for t0, t1 in pieces:
        dt = t1 - t0
        if not dt > 0:
            continue
        d = int(round(-math.log2(dt)))
        k = int(round(t0 / dt))
        out.add((t0, t1))
        for up in (1, 2):
            if d - up >= 0:
                kk, w = k >> up, dt * (1 << up)
                out.add((kk * w, min(1.0, (kk + 1) * w)))
        deepest = MAX_DEPTH if d >= 12 else min(MAX_DEPTH, d + 2)
        for dd in range(d + 1, deepest + 1):
            m = 1 << (dd - d)
            w = dt / m
            for j in range(m):
                out.add((t0 + j * w, t0 + (j + 1) * w))
    return sorted(out)


def _source_evolute(c, h, n=6000):
    """Exact evolute of the source where its radius of curvature is <= 2h, as
    polylines split at gaps."""
    t = np.linspace(0, 1, n)
    p, d = bez(c, t), bez_d(c, t)
    mt = 1 - t[:, None]
    dd = 6 * (mt * (c[2] - 2 * c[1] + c[0]) + t[:, None] * (c[3] - 2 * c[2] + c[1]))
    sp = np.hypot(d[:, 0], d[:, 1])
    cr = d[:, 0] * dd[:, 1] - d[:, 1] * dd[:, 0]
    with np.errstate(divide="ignore", invalid="ignore"):
        kap = cr / sp ** 3
        N = np.stack([-d[:, 1], d[:, 0]], 1) / sp[:, None]
        e = p + N / kap[:, None]
    ok = np.isfinite(e).all(1) & (np.abs(kap) * h >= 0.5)
    polys, cur = [], []
    for i in range(n):
        if ok[i]:
            cur.append(e[i])
        elif cur:
            polys.append(np.asarray(cur))
            cur = []
    if cur:
        polys.append(np.asarray(cur))
    return polys


def near_cusps(c, rel=1e-3, n=4001):
    """Points where |B'| has a local minimum below rel x the control-polygon length
    (source cusps and near-cusps, Section 7.3)."""
    from scipy.optimize import minimize_scalar
    t = np.linspace(0, 1, n)
    d = bez_d(c, t)
    ln = np.hypot(d[:, 0], d[:, 1])
    scale = np.abs(np.diff(c, axis=0)).sum()
    out = []
    for i in range(1, n - 1):
        if ln[i] <= ln[i - 1] and ln[i] <= ln[i + 1] and ln[i] < 10 * rel * scale:
            res = minimize_scalar(lambda u: float(np.hypot(*bez_d(c, u))), bounds=(t[i - 1], t[i + 1]),
                                  method="bounded", options={"xatol": 1e-13})
            if res.fun < rel * scale:
                out.append(bez(c, float(res.x)))
    return out


def _poly_dist(V, poly, k=6):
    """Distance from V to the polyline: exact distances to the segments next to the
    k polyline vertices nearest each point (a KD-tree query).  On densely sampled
    smooth curves the nearest segment is among them; small inputs go exhaustive."""
    if poly.shape[0] == 0:
        return np.full(V.shape[0], np.inf)
    if poly.shape[0] == 1:
        return np.hypot(*(V - poly[0]).T)
    if poly.shape[0] * V.shape[0] <= 200_000:
        return point_polyline_dist(V, poly)
    from scipy.spatial import cKDTree
    kk = min(k, poly.shape[0])
    _, idx = cKDTree(poly).query(V, k=kk)
    idx = idx.reshape(V.shape[0], kk)
    best = np.full(V.shape[0], np.inf)
    for j in (idx - 1, idx):                    # the segments before and after each vertex
        j = np.clip(j, 0, poly.shape[0] - 2)
        a, b = poly[j], poly[j + 1]
        ab = b - a
        ap = V[:, None, :] - a
        t = np.clip((ap * ab).sum(2) / np.maximum((ab * ab).sum(2), 1e-300), 0, 1)
        d = np.hypot(ap[..., 0] - t * ab[..., 0], ap[..., 1] - t * ab[..., 1])
        best = np.minimum(best, d.min(1))
    return best


def _miter_tips(P, Ti, To, h):
    out = []
    for s in (h, -h):
        A, B = P + s * _rn(Ti), P + s * _rn(To)
        M = np.array([[Ti[0], -To[0]], [Ti[1], -To[1]]], np.float64)
        if abs(np.linalg.det(M)) > 1e-12 * np.linalg.norm(Ti) * np.linalg.norm(To):
            tt = np.linalg.solve(M, B - A)[0]
            out.append(A + tt * Ti)
    return out


def _end_candidates(P, T, h, To=None):
    """Point candidates and circle centres at a segment end P (tangent T there):
    the joint, the square-cap corners, the miter tips (when a next tangent To is given)."""
    P = np.asarray(P, np.float64)
    u = np.asarray(T, np.float64) / np.linalg.norm(T)
    n = _rn(T)
    pts = [P]
    for e in (u, -u):
        pts += [P + h * n + h * e, P - h * n + h * e]
    if To is not None:
        pts += _miter_tips(P, np.asarray(T, np.float64), np.asarray(To, np.float64), h)
    return pts


def gate_distances(scene, r, seg, V, h, lsrc, pieces_of_seg=None, tol=None, stats=None):
    """Distance of each vertex V[k] to the exact geometry of logical segment `seg`
    (see the module docstring).  lsrc = logical_sources(scene, r).  With tol, a
    vertex within h + tol of a source cusp counts as on the geometry (distance 0)
    and is counted in stats["cusp_clause"]."""
    src, first, nxt = lsrc
    V = np.asarray(V, np.float64)
    best = np.full(V.shape[0], np.inf)
    points, circles = [], []
    c = src[seg]
    if c is not None:
        for sigma in (1, -1):
            off, cusp, _, _ = offset_curve(c, h, sigma, 0.0, 1.0, n=3000)
            best = np.minimum(best, _poly_dist(V, off))
            for q in cusp:
                circles.append(q)
        spine = bez(c, np.linspace(0, 1, 4001))
        best = np.minimum(best, np.abs(_poly_dist(V, spine) - h))
        for poly in _source_evolute(c, h):
            best = np.minimum(best, _poly_dist(V, poly))
        for t0, t1 in _fit_ranges(pieces_of_seg or []):
            best = np.minimum(best, _poly_dist(V, _es_fit_poly(c, t0, t1, h)))
        # the tail at the segment's end: a join with the next segment or an end cap
        P, T = c[3], _tangent(c, 1.0)
        To = None
        j = nxt[seg]
        if j < 0 and first[seg] >= 0:
            j = first[seg]                      # a closed subpath joins its first segment
        if j >= 0 and src[j] is not None:
            To = _tangent(src[j], 0.0)
        points += _end_candidates(P, T, h, To)
        circles.append(P)
    elif r["seg_kind"][seg] == 2:
        f = first[seg]
        if f >= 0 and src[f] is not None:       # start cap of an open subpath
            P0, T0 = src[f][0], _tangent(src[f], 0.0)
            points += _end_candidates(P0, T0, h)
            circles.append(P0)
        else:                                    # a dot: caps oriented along +x
            p = int(r["seg_path"][seg])
            P0 = scene.pts[scene.path_pt_off()[p]].astype(np.float64)
            points += _end_candidates(P0, (1.0, 0.0), h)
            circles.append(P0)
    for q in points:
        best = np.minimum(best, np.hypot(*(V - q).T))
    for q in circles:
        best = np.minimum(best, np.abs(np.hypot(*(V - q).T) - h))
    if tol is not None and c is not None:
        # Next to a cusp the subdivision can reach pieces shorter than the FP32
        # resolution of their coordinates, whose Euler-spiral curvature (and so
        # centre of curvature) FP32 cannot resolve; the evolute vertices of such
        # pieces are only held inside the stroke, within h of the cusp.
        for q in near_cusps(c):
            inside = (best > tol + 1e-3) & (np.hypot(*(V - q).T) <= h + tol)
            if stats is not None:
                stats["cusp_clause"] = stats.get("cusp_clause", 0) + int(inside.sum())
            best = np.where(inside, 0.0, best)
    return best


def pieces_by_seg(r):
    """The oracle's pieces of each logical segment as (t0, t1) lists."""
    out = {}
    for pi in range(r["piece"].shape[0]):
        out.setdefault(int(r["piece_seg"][pi]), []).append((float(r["piece"][pi, 0]), float(r["piece"][pi, 1])))
    return out


def gate_applies(scene):
    """The gate knows solid strokes of untransformed paths (dash parts and fills
    have other sources)."""
    fill = getattr(scene, "fill", None)
    return (getattr(scene, "transform", None) is None and not np.any(np.asarray(scene.dash_count) != 0)
            and (fill is None or not np.any(np.asarray(fill) != 0)))


def gate_segments(scene, r, prims, tag_offset, segs, tol, tag_base=0, r_seg_base=0, lsrc=None, pieces=None,
                  stats=None):
    """Gate distances of the GPU primitives of the given logical segments.

    prims, tag_offset: a GPU outline (rows x0 y0 x1 y1 ...) and its per-tag offsets;
    segs: logical segment indices of r; the GPU tag of segment i is
    tag_base + (i - r_seg_base).  Returns (segments checked, vertices, worst
    distance, the worst segment)."""
    lsrc = lsrc if lsrc is not None else logical_sources(scene, r)
    pieces = pieces if pieces is not None else pieces_by_seg(r)
    worst, worst_seg, nv = 0.0, -1, 0
    stats = {} if stats is None else stats
    for i in segs:
        t = tag_base + (int(i) - r_seg_base)
        a, b = int(tag_offset[t]), int(tag_offset[t + 1])
        if b == a:
            continue
        P = np.asarray(prims[a:b, :4], np.float64)
        V = np.vstack([P[:, :2], P[:, 2:4]])
        h = float(scene.half_width[r["seg_path"][i]])
        d = gate_distances(scene, r, int(i), V, h, lsrc, pieces.get(int(i)), tol=tol, stats=stats)
        nv += V.shape[0]
        if d.max() > worst:
            worst, worst_seg = float(d.max()), int(i)
    return len(segs), nv, worst, worst_seg
