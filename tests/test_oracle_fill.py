"""Pins of the oracle's fill flattening (Algorithm 1, fill branch: the source
curve itself, offset 0, with the 2/3-power density of Section 2.2)."""
import numpy as np
import pytest

import oracle
import workloads as W
from geom import balanced, bez, curve_dist, winding

TOL = 0.25


def fill_segments(scene, p):
    """FP64 cubics of path p with every subpath closed (a fill closes them all)."""
    vo = scene.path_verb_off.astype(np.int64)
    po = scene.path_pt_off()
    pts = scene.pts.astype(np.float64)
    k = int(po[p])
    subs, cur, start = [], None, None

    def close():
        if subs and subs[-1] and not np.array_equal(cur, start):
            subs[-1].append(np.stack([cur, cur + (start - cur) / 3, cur + 2 * (start - cur) / 3, start]))

    for vb in scene.verbs[vo[p]:vo[p + 1]]:
        if vb == W.MOVE:
            close()
            cur = start = pts[k].copy()
            k += 1
            subs.append([])
        elif vb == W.LINE:
            q = pts[k]
            k += 1
            subs[-1].append(np.stack([cur, cur + (q - cur) / 3, cur + 2 * (q - cur) / 3, q]))
            cur = q.copy()
        elif vb == W.CUBIC:
            c = pts[k:k + 3]
            k += 3
            subs[-1].append(np.vstack([cur[None], c]))
            cur = c[2].copy()
        elif vb == W.CLOSE:
            close()
            cur = start.copy()
            subs.append([])
    close()
    return [c for s in subs for c in s]


def test_fill_count_closed_forms(oracle_mod):
    # constant curvature (k1 = 0): N = sqrt|k0| (b - a) / sqrt(8 tol_n)
    assert oracle.fill_count(0.7, 0.0, 0.0, 1.0, 1e-3) == pytest.approx(np.sqrt(0.7) / np.sqrt(8e-3), rel=1e-12)
    # straight: no curvature, no lines beyond the one every range gets
    assert oracle.fill_count(0.0, 0.0, 0.0, 1.0, 1e-3) == 0.0
    # Euler spiral through an inflection: quadrature of sqrt|k0 + k1 (s - 1/2)|
    from scipy import integrate
    for k0, k1, a, b in [(0.1, 2.0, 0.0, 1.0), (-0.3, 1.5, 0.2, 0.9), (1.0, -4.0, 0.0, 0.6), (0.5, 1e-12, 0.0, 1.0)]:
        ref = integrate.quad(lambda s: np.sqrt(abs(k0 + k1 * (s - 0.5))), a, b, epsabs=1e-14, epsrel=1e-13,
                             points=[0.5 - k0 / k1] if a < 0.5 - k0 / k1 < b else None)[0]
        assert oracle.fill_count(k0, k1, a, b, 2e-3) == pytest.approx(ref / np.sqrt(8 * 2e-3), rel=1e-9)


def test_filled_circle(oracle_mod):
    """A circle of four cubics, filled: each quarter gets ceil((pi/2) sqrt(R / 8 tol))
    lines (the ES of a circle cubic has the circle's curvature to 3e-4), all vertices
    lie on the circle and every chord's sagitta is within the tolerance."""
    R = 100.0
    b = W._Builder()
    b.path(W.circle_cmds(0, 0, R), 3.0, fill=True)
    r = oracle.stroke(b.build(), TOL)
    n = int(np.ceil(np.pi / 2 * np.sqrt(R / (8 * TOL))))
    assert r["seg_count"].tolist() == [n, n, n, n, 0]
    P = r["prim"]
    rad = np.hypot(P[:, 0], P[:, 1])
    assert np.all(np.abs(rad - R) <= 2.8e-4 * R)
    mid = 0.5 * (P[:, :2] + P[:, 2:4])
    assert np.all(R - np.hypot(mid[:, 0], mid[:, 1]) <= TOL + 2.8e-4 * R)
    assert balanced(P[:, :4])


def test_fill_outline_is_the_path(oracle_mod):
    """For filled PR1-like paths: every vertex lies within the fit error of the
    source curve, every point of the source curve within tol plus that of the
    outline, the outline of each path is closed, and a straight segment is one
    line.  The fit is accepted at FIT_FRAC * tol by the paper's error estimate,
    whose true error is at most 1 / 0.62 of the estimate over the paper's
    validation range (the oracle's own brute-force sweep of the metric)."""
    sc = W.pr1(n_paths=6).as_fill()
    r = oracle.stroke(sc, TOL)
    from geom import point_polyline_dist
    prim_path = np.repeat(r["seg_path"], r["seg_count"])
    for p in range(sc.n_paths):
        segs = fill_segments(sc, p)
        P = r["prim"][prim_path == p]
        assert balanced(P[:, :4])
        d = curve_dist(np.vstack([P[:, :2], P[:, 2:4]]), [(False, c) for c in segs], spacing=0.01)
        fit_err = oracle.FIT_FRAC * TOL / 0.62
        assert d.max() <= fit_err + 0.005                  # + half the sample spacing
        dense = np.concatenate([bez(c, np.linspace(0, 1, 400)) for c in segs])
        poly = np.vstack([P[:, :2], P[-1:, 2:4]])           # one subpath per PR1 path, in order
        assert point_polyline_dist(dense, poly).max() <= TOL + fit_err + 1e-6
    lines = W._Builder()
    lines.path([W.M(0, 0), W.L(50, 10), W.L(40, 60)], 1.0, fill=True)
    r2 = oracle.stroke(lines.build(), TOL)
    assert r2["seg_count"].tolist() == [1, 1, 1, 0]   # two lines, the closing line, the marker


def test_fill_winding_matches_the_path(oracle_mod):
    """Nonzero winding of the flattened fill equals that of the exact path away
    from a tol band (a self-crossing loop and an S-curve with a closing line)."""
    b = W._Builder()
    b.path([W.M(0, 0), W.C(300, 200, -100, 200, 200, 0)], 1.0, fill=True)
    b.path([W.M(400, 0), W.C(500, 200, 600, -200, 700, 0), W.L(550, 150)], 1.0, fill=True)
    sc = b.build()
    r = oracle.stroke(sc, TOL)
    prim_path = np.repeat(r["seg_path"], r["seg_count"])
    rng = np.random.default_rng(3)
    for p in range(sc.n_paths):
        segs = fill_segments(sc, p)
        dense = np.concatenate([bez(c, np.linspace(0, 1, 4000)) for c in segs])
        exact = np.concatenate([dense[:-1], dense[1:]], axis=1)
        lo, hi = dense.min(0) - 5, dense.max(0) + 5
        Q = rng.uniform(lo, hi, (6000, 2))
        far = curve_dist(Q, [(False, c) for c in segs], spacing=0.05) > TOL * 1.3 + 0.025
        w_out = winding(Q[far], r["prim"][prim_path == p][:, :4])
        w_ref = winding(Q[far], exact)
        assert np.array_equal(w_out, w_ref)
        assert np.any(w_ref != 0)


def test_fill_ignores_stroke_style_and_keeps_strokes(oracle_mod):
    """A fill's dash, join, cap and width do not change it; stroked paths beside fills
    are expanded exactly as without them."""
    cmds = [W.M(0, 0), W.C(40, 80, 120, -30, 150, 40), W.L(60, 90)]
    a, b_ = W._Builder(), W._Builder()
    a.path(cmds, 2.0, fill=True)
    b_.path(cmds, 9.0, join=W.JOIN_MITER, cap=W.CAP_ROUND, dash=[5, 5], dash_offset=2, fill=True)
    ra, rb = oracle.stroke(a.build(), TOL), oracle.stroke(b_.build(), TOL)
    assert np.array_equal(ra["prim"], rb["prim"])
    mixed = W.concat([W.pr1(n_paths=5), a.build(), W.pr1(seed=2, n_paths=3)])
    rm = oracle.stroke(mixed, TOL)
    rs = oracle.stroke(W.concat([W.pr1(n_paths=5), W.pr1(seed=2, n_paths=3)]), TOL)
    keep = np.repeat(rm["seg_path"] != 5, rm["seg_count"])
    assert np.array_equal(rm["prim"][keep], rs["prim"])


def test_filled_arcs(oracle_mod):
    """Arc output of a filled circle: one arc per quarter-piece range (kappa' ~ 0), each
    through points of the circle, with curvature 1/R."""
    R = 50.0
    b = W._Builder()
    b.path(W.circle_cmds(0, 0, R), 1.0, fill=True)
    r = oracle.stroke(b.build(), TOL, arcs=True)
    P = r["prim"]
    assert np.all(np.abs(np.hypot(P[:, 0], P[:, 1]) - R) <= 2.8e-4 * R)
    assert np.allclose(P[:, 4], 1.0 / R, rtol=2e-3)
    assert balanced(P[:, :4])
