"""Pins for the encoding features of Section 8.2 in the oracle: quadratic segments
(degree-elevated, Section 8.1) and per-path affine transforms."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from geom import point_polyline_dist

TOL = 0.25


def _quad_offset(P0, Q1, P2, h, sigma, n=6000):
    """Exact parallel curve of the quadratic (1-t)^2 P0 + 2t(1-t) Q1 + t^2 P2."""
    t = np.linspace(0, 1, n)[:, None]
    P0, Q1, P2 = (np.asarray(v, np.float64) for v in (P0, Q1, P2))
    B = (1 - t) ** 2 * P0 + 2 * t * (1 - t) * Q1 + t ** 2 * P2
    D = 2 * (1 - t) * (Q1 - P0) + 2 * t * (P2 - Q1)
    N = np.stack([D[:, 1], -D[:, 0]], 1) / np.hypot(D[:, 0], D[:, 1])[:, None]
    return B + sigma * h * N


def _seg_set_dist(X, S):
    """Distance of each point of X to the nearest of the segments S [n, 4]."""
    a, d = S[:, :2], S[:, 2:] - S[:, :2]
    l2 = np.maximum((d * d).sum(1), 1e-300)
    ap = X[:, None, :] - a[None]
    t = np.clip((ap * d[None]).sum(2) / l2[None], 0, 1)
    return np.hypot(ap[..., 0] - t * d[None, :, 0], ap[..., 1] - t * d[None, :, 1]).min(1)


QUADS = [((0, 0), (60, 90), (120, 0), 4.0), ((0, 200), (300, 260), (40, 230), 9.0),
         ((500, 0), (510, 400), (700, 10), 2.5), ((0, 500), (5, 501), (400, 700), 12.0)]


def test_quadratic_outline_follows_the_exact_quadratic(oracle_mod):
    """Each side of a stroked quadratic: every vertex within tol of the exact parallel
    curve of the quadratic (evaluated as a quadratic), and every point of that curve
    within tol + the fit error of the side's polyline."""
    b = W._Builder()
    for P0, Q1, P2, h in QUADS:
        b.path([W.M(*P0), W.Q(*Q1, *P2)], h, cap=W.CAP_BUTT)
    sc = b.build()
    r = oracle.stroke(sc, TOL)
    seg_path = r["seg_path"]
    prim_path = np.repeat(seg_path, r["seg_count"])
    fit_err = oracle.FIT_FRAC * TOL / 0.62
    for p, (P0, Q1, P2, h) in enumerate(QUADS):
        for sigma in (1, -1):
            m = (prim_path == p) & (r["prim_side"] == sigma) & np.isin(r["prim_kind"], (0, 1))
            P = r["prim"][m][:, :4]
            assert P.shape[0] >= 2
            exact = _quad_offset(P0, Q1, P2, h, sigma)
            V = np.vstack([P[:, :2], P[:, 2:]])
            assert point_polyline_dist(V, exact).max() <= TOL + 1e-3
            assert _seg_set_dist(exact, P).max() <= TOL + fit_err + 1e-3


def test_quadratic_equals_the_cubic_through_the_same_curve(oracle_mod):
    """A quadratic and the cubic with control points P0 + 2/3 (Q1 - P0), P2 + 2/3 (Q1 - P2)
    (exact here: coordinates are multiples of 3) trace one curve: identical outlines."""
    q = W._Builder()
    c = W._Builder()
    for (x0, y0), (x1, y1), (x2, y2), h in [((0, 0), (60, 90), (120, 0), 4.0), ((0, 210), (300, 261), (42, 231), 9.0)]:
        q.path([W.M(x0, y0), W.Q(x1, y1, x2, y2), W.L(x2 + 30, y2 + 3)], h, join=W.JOIN_ROUND, cap=W.CAP_ROUND)
        c1 = (x0 + 2 * (x1 - x0) / 3, y0 + 2 * (y1 - y0) / 3)
        c2 = (x2 + 2 * (x1 - x2) / 3, y2 + 2 * (y1 - y2) / 3)
        c.path([W.M(x0, y0), W.C(*c1, *c2, x2, y2), W.L(x2 + 30, y2 + 3)], h, join=W.JOIN_ROUND, cap=W.CAP_ROUND)
    a, b = oracle.stroke(q.build(), TOL), oracle.stroke(c.build(), TOL)
    assert np.array_equal(a["seg_count"], b["seg_count"]) and np.array_equal(a["prim"], b["prim"])


def _exact_similarity_scene():
    b = W._Builder()
    b.path([W.M(0, 0), W.C(40, 80, 120, -30, 150, 40), W.L(60, 90), W.Q(20, 140, 0, 60)], 3.0, join=W.JOIN_MITER,
           cap=W.CAP_SQUARE)
    b.path(W.circle_cmds(300, 100, 50), 4.0)
    b.path([W.M(500, 0), W.L(600, 20), W.L(560, 90)], 2.0, dash=[10, 6, 3, 6], dash_offset=2.0)
    b.path([W.M(0, 300), W.C(100, 400, 200, 200, 300, 300), W.Z], 1.0, fill=True)
    return b.build()


def test_transform_equals_transformed_input(oracle_mod):
    """x' = -2y + 16, y' = 2x - 32 is exact in FP32, so the scene under that transform
    and the scene whose points were transformed beforehand, with widths doubled and
    dash lengths doubled, give identical outlines (caps, joins and fills); the dashed
    path's cut parameters come from arc lengths at the two scales, equal to rounding."""
    sc = _exact_similarity_scene()
    m = np.array([0, 2, -2, 0, 16, -32], np.float32)
    a = oracle.stroke(sc.with_transform(m), TOL)
    pre = W.Scene(**{**sc.__dict__})
    pre.pts = np.stack([-2 * sc.pts[:, 1] + 16, 2 * sc.pts[:, 0] - 32], 1).astype(np.float32)
    pre.half_width = sc.half_width * 2
    pre.dash_len = sc.dash_len * 2
    pre.dash_offset = sc.dash_offset * 2
    pre.transform = None
    b = oracle.stroke(pre, TOL)
    assert np.array_equal(a["seg_count"], b["seg_count"])
    dashed = np.repeat(a["seg_path"], a["seg_count"]) == 2
    assert np.array_equal(a["prim"][~dashed], b["prim"][~dashed])
    assert np.abs(a["prim"][dashed] - b["prim"][dashed]).max() < 1e-9


def test_stroke_commutes_with_similarities(oracle_mod):
    """For a similarity T of scale s: stroke(T P, h s, tol s) = T stroke(P, h, tol) —
    same counts on every robust segment, vertices equal to 1e-9 of the scene size."""
    sc = W.pr1(seed=11, n_paths=20)
    s, ang = 1.7, 0.3
    m = np.array([s * math.cos(ang), s * math.sin(ang), -s * math.sin(ang), s * math.cos(ang), 37.5, -12.25])
    a = oracle.stroke(sc, TOL)
    b = oracle.stroke(sc.with_transform(m.astype(np.float32)), TOL * s)
    m = m.astype(np.float32).astype(np.float64)
    robust = (a["seg_margin"] >= 1e-4) & (b["seg_margin"] >= 1e-4)
    assert robust.mean() > 0.95
    assert np.array_equal(a["seg_count"][robust], b["seg_count"][robust])
    keep_a = np.repeat(robust, a["seg_count"])
    keep_b = np.repeat(robust, b["seg_count"])
    A, B = a["prim"][keep_a], b["prim"][keep_b]
    for k in (0, 2):
        x, y = A[:, k], A[:, k + 1]
        tx, ty = m[0] * x + m[2] * y + m[4], m[1] * x + m[3] * y + m[5]
        assert np.abs(tx - B[:, k]).max() < 1e-9 * 2000 and np.abs(ty - B[:, k + 1]).max() < 1e-9 * 2000


@pytest.mark.parametrize("diag", [(3.0, 1 / 3.0), (4.0, 1.0), (0.5, 2.0)])
def test_half_width_scales_by_sqrt_det(oracle_mod, diag):
    """Under a non-uniform scale the pen stays round with half-width h sqrt|det|: the
    outline of a straight line lies at that distance from the transformed line."""
    b = W._Builder()
    b.path([W.M(0, 0), W.L(100, 0)], 2.0, cap=W.CAP_BUTT)
    b.path([W.M(0, 0), W.L(0, 100)], 2.0, cap=W.CAP_BUTT)
    m = np.array([diag[0], 0, 0, diag[1], 5, 7], np.float32)
    r = oracle.stroke(b.build().with_transform(m), TOL)
    h = 2.0 * math.sqrt(abs(diag[0] * diag[1]))
    prim_path = np.repeat(r["seg_path"], r["seg_count"])
    off = np.isin(r["prim_kind"], (0, 1))
    P = r["prim"]
    assert np.allclose(np.abs(P[off & (prim_path == 0)][:, [1, 3]] - 7), h, atol=1e-9)
    assert np.allclose(np.abs(P[off & (prim_path == 1)][:, [0, 2]] - 5), h, atol=1e-9)


def test_dashes_are_measured_before_the_transform(oracle_mod):
    """A dashed line under a uniform scale 2: the pattern [10, 5] becomes dashes 20 long
    with gaps of 10 (butt caps: the cap lines sit at the dash ends)."""
    b = W._Builder()
    b.path([W.M(0, 0), W.L(100, 0)], 1.0, cap=W.CAP_BUTT, dash=[10, 5])
    r = oracle.stroke(b.build().with_transform([2, 0, 0, 2, 0, 0]), TOL)
    caps = r["prim"][r["prim_kind"] == 6]
    xs = np.unique(np.round(np.concatenate([caps[:, 0], caps[:, 2]]), 9))
    want = sorted(set(x for k in range(7) for x in (30.0 * k, 30.0 * k + 20.0) if x <= 200.0))
    assert np.allclose(xs, want)


def test_filled_circle_under_scale(oracle_mod):
    """A filled circle of radius R scaled by s: ceil((pi/2) sqrt(s R / 8 tol)) lines per
    quarter, vertices on the circle of radius s R."""
    R, s = 40.0, 2.5
    b = W._Builder()
    b.path(W.circle_cmds(0, 0, R), 1.0, fill=True)
    r = oracle.stroke(b.build().with_transform([s, 0, 0, s, 0, 0]), 0.1)
    n = int(np.ceil(np.pi / 2 * np.sqrt(s * R / (8 * 0.1))))
    assert r["seg_count"].tolist() == [n, n, n, n, 0]
    rad = np.hypot(r["prim"][:, 0], r["prim"][:, 1])
    assert np.all(np.abs(rad - s * R) <= 2.8e-4 * s * R)
