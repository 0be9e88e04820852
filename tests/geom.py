"""Exact-geometry helpers for the tests (FP64 numpy).  None of this is the
stroke-expansion method: it samples source cubics densely, measures distances,
checks vertex balance and rasterises outlines with the nonzero rule."""
from __future__ import annotations

import numpy as np

from workloads import CUBIC, LINE, MOVE, CLOSE, QUAD, VERB_POINTS


def path_segments(scene, p):
    """List of (is_line, ctrl[4,2]) for path p, in verb order (FP64)."""
    vo = scene.path_verb_off.astype(np.int64)
    po = scene.path_pt_off()
    pts = scene.pts.astype(np.float64)
    k = int(po[p])
    cur = start = None
    segs = []
    for vb in scene.verbs[vo[p]:vo[p + 1]]:
        if vb == MOVE:
            cur = start = pts[k].copy(); k += 1
        elif vb == LINE:
            q = pts[k]; k += 1
            segs.append((True, np.stack([cur, cur + (q - cur) / 3, cur + 2 * (q - cur) / 3, q])))
            cur = q.copy()
        elif vb == CUBIC:
            c = pts[k:k + 3]; k += 3
            segs.append((False, np.vstack([cur[None], c])))
            cur = c[2].copy()
        elif vb == QUAD:        # the cubic through the same curve
            q1, q2 = pts[k], pts[k + 1]; k += 2
            segs.append((False, np.stack([cur, cur + 2 * (q1 - cur) / 3, q2 + 2 * (q1 - q2) / 3, q2])))
            cur = q2.copy()
        elif vb == CLOSE:
            if not np.array_equal(cur, start):
                segs.append((True, np.stack([cur, cur + (start - cur) / 3, cur + 2 * (start - cur) / 3, start])))
            cur = start.copy()
    return segs


def fill_path_segments(scene, p):
    """path_segments for a filled path: every subpath closed with a line back to its
    start (when it does not end there already)."""
    vo = scene.path_verb_off.astype(np.int64)
    po = scene.path_pt_off()
    pts = scene.pts.astype(np.float64)
    k = int(po[p])
    cur = start = None
    segs, drawn = [], False

    def close():
        if drawn and cur is not None and not np.array_equal(cur, start):
            segs.append((True, np.stack([cur, cur + (start - cur) / 3, cur + 2 * (start - cur) / 3, start])))

    for vb in scene.verbs[vo[p]:vo[p + 1]]:
        if vb == MOVE:
            close()
            cur = start = pts[k].copy(); k += 1
            drawn = False
        elif vb == LINE:
            q = pts[k]; k += 1
            segs.append((True, np.stack([cur, cur + (q - cur) / 3, cur + 2 * (q - cur) / 3, q])))
            cur = q.copy(); drawn = True
        elif vb == CUBIC:
            c = pts[k:k + 3]; k += 3
            segs.append((False, np.vstack([cur[None], c])))
            cur = c[2].copy(); drawn = True
        elif vb == QUAD:        # the cubic through the same curve
            q1, q2 = pts[k], pts[k + 1]; k += 2
            segs.append((False, np.stack([cur, cur + 2 * (q1 - cur) / 3, q2 + 2 * (q1 - q2) / 3, q2])))
            cur = q2.copy(); drawn = True
        elif vb == CLOSE:
            close()
            cur = start.copy(); drawn = False
    close()
    return segs


def bez(c, t):
    t = np.asarray(t, np.float64)[..., None]
    mt = 1 - t
    return mt ** 3 * c[0] + 3 * mt ** 2 * t * c[1] + 3 * mt * t ** 2 * c[2] + t ** 3 * c[3]


def bez_d(c, t):
    t = np.asarray(t, np.float64)[..., None]
    mt = 1 - t
    return 3 * (mt ** 2 * (c[1] - c[0]) + 2 * mt * t * (c[2] - c[1]) + t ** 2 * (c[3] - c[2]))


def dense_curve(segs, n=4000):
    return np.concatenate([bez(c, np.linspace(0, 1, n)) for _, c in segs]) if segs else np.zeros((0, 2))


def curve_dist(P, segs, spacing=0.02):
    """Distance from points P[n,2] to the union of the cubics in segs, via a KD-tree on
    samples at most `spacing` apart (error <= spacing / 2)."""
    from scipy.spatial import cKDTree
    samples = []
    for _, c in segs:
        ln = np.sum(np.hypot(*np.diff(bez(c, np.linspace(0, 1, 257)), axis=0).T))
        n = int(min(max(ln / spacing, 2), 2_000_000))
        samples.append(bez(c, np.linspace(0, 1, n + 1)))
    tree = cKDTree(np.concatenate(samples))
    return tree.query(P)[0]


def point_polyline_dist(P, poly):
    """Distance from points P[n,2] to the polyline poly[m,2]."""
    a = poly[:-1]
    b = poly[1:]
    ab = b - a
    L2 = np.maximum((ab ** 2).sum(1), 1e-300)
    best = np.full(P.shape[0], np.inf)
    for j0 in range(0, P.shape[0], 1024):
        Pj = P[j0:j0 + 1024]
        for i0 in range(0, a.shape[0], 1024):
            aa, bb, l2 = a[i0:i0 + 1024], ab[i0:i0 + 1024], L2[i0:i0 + 1024]
            ap = Pj[:, None, :] - aa[None]
            t = np.clip((ap * bb[None]).sum(2) / l2[None], 0, 1)
            d = np.hypot(ap[..., 0] - t * bb[None, :, 0], ap[..., 1] - t * bb[None, :, 1])
            best[j0:j0 + 1024] = np.minimum(best[j0:j0 + 1024], d.min(1))
    return best


def offset_curve(c, h, sigma, t0, t1, n=1500):
    """Exact offset c(t) + sigma*h*right_normal(t) over [t0, t1], sampled densely and
    refined around minima of |c'(t)|, plus the points where the derivative vanishes
    (source cusps), around which the swept normal turns through a half circle."""
    from scipy.optimize import minimize_scalar
    t = np.linspace(t0, t1, n)
    d = bez_d(c, t)
    ln = np.hypot(d[:, 0], d[:, 1])
    scale = np.abs(np.diff(c, axis=0)).sum()
    extra, cusps = [], []
    for i in range(1, n - 1):
        if ln[i] <= ln[i - 1] and ln[i] <= ln[i + 1] and ln[i] < 0.05 * scale:
            res = minimize_scalar(lambda u: float(np.hypot(*bez_d(c, u))), bounds=(t[i - 1], t[i + 1]),
                                  method="bounded", options={"xatol": 1e-13})
            tc = float(res.x)
            extra.append(np.linspace(max(t0, tc - 0.02), min(t1, tc + 0.02), 4001))
            if res.fun < 1e-5 * scale:
                cusps.append(bez(c, tc))
    if extra:
        t = np.unique(np.concatenate([t] + extra))
    p = bez(c, t)
    d = bez_d(c, t)
    ln = np.hypot(d[:, 0], d[:, 1])
    ok = ln > 1e-12 * max(scale, 1e-300)
    rn = np.zeros_like(d)
    rn[ok, 0] = d[ok, 1] / ln[ok]
    rn[ok, 1] = -d[ok, 0] / ln[ok]
    off = p + sigma * h * rn
    cusp = np.asarray(cusps).reshape(-1, 2)
    return off[ok], cusp, ln, p


def balanced(prims, mask=None):
    """Every endpoint occurs as often as a start as it does as an end (bit-exact)."""
    P = prims if mask is None else prims[mask]
    if P.shape[0] == 0:
        return True
    a = np.ascontiguousarray(P[:, 0:2]).view(np.dtype((np.void, 2 * P.itemsize)))[:, 0]
    b = np.ascontiguousarray(P[:, 2:4]).view(np.dtype((np.void, 2 * P.itemsize)))[:, 0]
    ua, ca = np.unique(a, return_counts=True)
    ub, cb = np.unique(b, return_counts=True)
    return ua.shape == ub.shape and np.array_equal(ua, ub) and np.array_equal(ca, cb)


def winding(points, lines):
    """Nonzero-rule winding number of each point w.r.t. a set of directed lines."""
    px, py = points[:, 0][:, None], points[:, 1][:, None]
    w = np.zeros(points.shape[0], np.int64)
    for i0 in range(0, lines.shape[0], 1024):
        L = lines[i0:i0 + 1024]
        x0, y0, x1, y1 = (L[:, k][None, :] for k in range(4))
        side = (x1 - x0) * (py - y0) - (px - x0) * (y1 - y0)
        up = (y0 <= py) & (py < y1) & (side > 0)
        dn = (y1 <= py) & (py < y0) & (side < 0)
        w += up.sum(1) - dn.sum(1)
    return w


def arcs_to_lines(prims, n=16):
    """Flatten arc primitives (x0 y0 x1 y1 curvature) finely so they can be rasterised."""
    out = []
    for x0, y0, x1, y1, k in prims:
        a, b = np.array([x0, y0]), np.array([x1, y1])
        ch = b - a
        c = np.hypot(*ch)
        if k == 0 or c == 0:
            out.append([x0, y0, x1, y1])
            continue
        r = 1.0 / k
        half = np.arcsin(np.clip(c * abs(k) / 2, -1, 1))
        mid = (a + b) / 2
        nrm = np.array([-ch[1], ch[0]]) / c
        cen = mid + nrm * np.sign(r) * np.sqrt(max(r * r - c * c / 4, 0))
        a0 = np.arctan2(*(a - cen)[::-1])
        ang = np.linspace(0, 2 * half * np.sign(k), n + 1)
        q = cen + abs(r) * np.stack([np.cos(a0 + ang), np.sin(a0 + ang)], 1)
        q[0], q[-1] = a, b
        out.extend(np.hstack([q[:-1], q[1:]]).tolist())
    return np.asarray(out)
