"""Whole-pipeline pins for the oracle: worked cases, exact geometry, invariants and a
nonzero-rule raster against the swept stroke (strong correctness, Section 1)."""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from geom import (arcs_to_lines, balanced, bez, curve_dist, dense_curve, offset_curve, path_segments,
                  point_polyline_dist, winding)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = 0.25


def _load(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]
    return np.array(rows, dtype=np.float64)


@pytest.fixture(scope="module")
def hand(oracle_mod):
    sc = W.hand_cases()
    return sc, oracle.stroke(sc, TOL)


def test_golden_straight_line_outline(hand):
    sc, r = hand
    exp = _load("line_butt_h5.txt")
    got = r["prim"][:4, :4]
    assert r["seg_count"][:2].tolist() == [3, 1]
    assert np.array_equal(got, exp[:, 1:])


def test_golden_round_cap_counts(oracle_mod):
    for h, tol, n in _load("round_cap_counts.txt"):
        sc = W._Builder().path([W.M(0, 0), W.L(50, 0)], h, cap=W.CAP_ROUND).build()
        r = oracle.stroke(sc, tol)
        assert r["seg_count"].tolist() == [2 + n, n]


def test_collinear_cubic_equals_line(hand):
    sc, r = hand
    # H1 line and H2 collinear cubic (translated by y=20): same outline shape
    a = r["prim"][r["seg_path"][np.repeat(np.arange(len(r["seg_count"])), r["seg_count"])] == 0]
    b = r["prim"][r["seg_path"][np.repeat(np.arange(len(r["seg_count"])), r["seg_count"])] == 1]
    assert a.shape == b.shape
    assert np.allclose(a[:, :4] + np.array([0, 20, 0, 20]), b[:, :4], atol=1e-9)


def _prims_by_path(r):
    seg_of_prim = np.repeat(np.arange(len(r["seg_count"])), r["seg_count"])
    return r["seg_path"][seg_of_prim]


@pytest.mark.parametrize("arcs", [False, True])
def test_outlines_are_closed(oracle_mod, arcs):
    """Every vertex is left as often as it is entered (watertight, bit-exact)."""
    for sc in (W.hand_cases(), W.pr1().subset(range(30)), W.map_like(n_paths=300)):
        r = oracle.stroke(sc, TOL, arcs=arcs)
        pp = _prims_by_path(r)
        for p in range(sc.n_paths):
            assert balanced(r["prim"][pp == p][:, :4]), p


def test_circle_offsets(hand):
    """H6: concentric circles R +- h; the cubic circle deviates from a circle by 2.7e-4 R."""
    sc, r = hand
    pp = _prims_by_path(r)
    P = r["prim"][(pp == 5) & (r["prim_kind"] == 0)]
    v = np.vstack([P[:, 0:2], P[:, 2:4]]) - np.array([300.0, 300.0])
    rad = np.hypot(*v.T)
    inner, outer = rad[rad < 100], rad[rad > 100]
    assert np.all(np.abs(inner - 95) < TOL + 0.03) and np.all(np.abs(outer - 105) < TOL + 0.03)
    # chord midpoints stay within the flattening tolerance of the offset circles
    mid = 0.5 * (P[:, 0:2] + P[:, 2:4]) - np.array([300.0, 300.0])
    mr = np.hypot(*mid.T)
    assert np.all(np.minimum(np.abs(mr - 95), np.abs(mr - 105)) < 2 * TOL + 0.03)


def test_evolute_of_overwide_circle_sits_at_centre(hand):
    """H7 (h = 150 > R = 100): the inner side needs evolute patches; the evolute of a
    near-circle collapses towards the centre."""
    sc, r = hand
    pp = _prims_by_path(r)
    ev = r["prim"][(pp == 6) & (r["prim_kind"] == 2)]
    assert ev.shape[0] > 0
    d = np.hypot(*(np.vstack([ev[:, :2], ev[:, 2:4]]) - np.array([300.0, 600.0])).T)
    assert d.max() < 1.0
    # H6 (h < R) needs none
    assert not np.any((pp == 5) & (r["prim_kind"] == 2))


def _piece_table(r):
    return {k: r["piece"][:, i] for i, k in enumerate(oracle.PIECE_FIELDS)}


def test_evolutes_exactly_where_curvature_exceeds_inverse_half_width(oracle_mod):
    sc = W.concat([W.hand_cases(), W.pr1().subset(range(20))])
    r = oracle.stroke(sc, TOL)
    pt = _piece_table(r)
    hw = sc.half_width[r["seg_path"][r["piece_seg"]]]
    k_ends = np.stack([pt["k0"] - 0.5 * pt["k1"], pt["k0"] + 0.5 * pt["k1"]], 1) / pt["L"][:, None]
    need = np.any(np.abs(k_ends) * hw[:, None] > 1.0, axis=1) & (pt["degenerate"] == 0)
    has = np.zeros(len(need), bool)
    sel = r["prim_kind"] == 2
    has[r["prim_piece"][sel]] = True
    assert np.array_equal(need, has)


def _seg_source(sc, r):
    """Map each logical segment to its source control points (None for markers)."""
    out = []
    segs_by_path = {}
    cursor = {}
    for i, (k, p) in enumerate(zip(r["seg_kind"], r["seg_path"])):
        if p not in segs_by_path:
            segs_by_path[p] = path_segments(sc, p)
            cursor[p] = 0
        if k in (0, 1):
            lst = segs_by_path[p]
            # skip zero-length segments, as the oracle does
            while np.allclose(lst[cursor[p]][1], lst[cursor[p]][1][0], atol=0):
                cursor[p] += 1
            out.append(lst[cursor[p]][1])
            cursor[p] += 1
        else:
            out.append(None)
    return out


def offset_gate(sc, r, tol):
    """Distance of every parallel-curve vertex to the exact offset of its source cubic.

    Reading of the gate (Section 7.3, near-cusp == cusp): for an ES piece shorter than
    the half-width, whose offset is a turn about a point of the source, a vertex may
    instead lie on the circle of radius h about that part of the source.  Returns
    (worst distance, number of vertices that needed the near-cusp clause)."""
    src = _seg_source(sc, r)
    pt = _piece_table(r)
    worst, relaxed = 0.0, 0
    for pi in range(r["piece"].shape[0]):
        seg = r["piece_seg"][pi]
        c = src[seg]
        h = float(sc.half_width[r["seg_path"][seg]])
        t0, t1 = pt["t0"][pi], pt["t1"][pi]
        span = t1 - t0
        lo, hi = max(0.0, t0 - 0.5 * span), min(1.0, t1 + 0.5 * span)
        for sigma in (1, -1):
            m = (r["prim_piece"] == pi) & (r["prim_side"] == sigma) & np.isin(r["prim_kind"], (0, 1))
            if not m.any():
                continue
            P = r["prim"][m]
            V = np.vstack([P[:, :2], P[:, 2:4]])
            off, cusp, ln, _ = offset_curve(c, h, sigma, lo, hi, n=3000)
            d = point_polyline_dist(V, off) if off.shape[0] > 1 else np.full(V.shape[0], np.inf)
            if cusp.shape[0]:
                dc = np.min(np.abs(np.hypot(V[:, None, 0] - cusp[None, :, 0], V[:, None, 1] - cusp[None, :, 1]) - h), 1)
                d = np.minimum(d, dc)
            if pt["L"][pi] <= h:
                near = np.abs(point_polyline_dist(V, bez(c, np.linspace(t0, t1, 400))) - h)
                relaxed += int(np.count_nonzero((d > tol + 1e-3) & (near <= tol + 1e-3)))
                d = np.minimum(d, near)
            worst = max(worst, d.max())
    return worst, relaxed


@pytest.mark.parametrize("which", ["hand", "pr1"])
def test_offset_vertices_lie_on_the_exact_offset(oracle_mod, which):
    """Every parallel-curve vertex is within tol + 1e-3 of the exact offset of the source
    cubic (at a source cusp or near-cusp: of the circle of radius h about it)."""
    sc = W.hand_cases() if which == "hand" else W.pr1().subset(range(12))
    r = oracle.stroke(sc, TOL)
    worst, relaxed = offset_gate(sc, r, TOL)
    assert worst <= TOL + 1e-3, worst
    n_vert = 2 * np.count_nonzero(np.isin(r["prim_kind"], (0, 1)))
    assert relaxed <= 0.01 * n_vert


def test_evolute_vertices_lie_on_the_es_evolute(oracle_mod):
    """Evolute vertices lie on the centre-of-curvature locus z + N / kappa of their ES
    piece.  Positions come from a fine trapezoid integration of the mapped piece (not the
    oracle's quadrature), and the locus is sampled both uniformly in s and uniformly in
    1/kappa, so its fast ends near an inflection are resolved."""
    sc = W.hand_cases()
    r = oracle.stroke(sc, TOL)
    pt = _piece_table(r)
    checked = 0
    for pi in np.unique(r["prim_piece"][r["prim_kind"] == 2]):
        k0, k1, th0 = pt["k0"][pi], pt["k1"][pi], pt["th0"][pi]
        rot = pt["rotx"][pi] + 1j * pt["roty"][pi]
        Lg = abs(rot)                            # arc length of the mapped unit ES
        h = float(sc.half_width[r["seg_path"][r["piece_seg"][pi]]])
        fine = np.linspace(0, 1, 400001)
        th_f = -th0 + k0 * fine + 0.5 * k1 * (fine * fine - fine)
        zf = np.concatenate([[0], np.cumsum(0.5 * (np.exp(1j * th_f[1:]) + np.exp(1j * th_f[:-1])) * (fine[1] - fine[0]))])
        samp = [np.linspace(0, 1, 20001)]
        if k1 != 0:
            rad = h * np.arange(1, 4001) / 2000.0
            for sg in (1, -1):
                sj = 0.5 + (sg * Lg / rad - k0) / k1
                samp.append(sj[(sj >= 0) & (sj <= 1)])
        s = np.unique(np.concatenate(samp))
        z = np.interp(s, fine, zf.real) + 1j * np.interp(s, fine, zf.imag)
        z = (pt["p0x"][pi] + 1j * pt["p0y"][pi]) + z * rot
        th = -th0 + k0 * s + 0.5 * k1 * (s * s - s)
        T = np.exp(1j * th) * rot / Lg
        kap = (k0 + k1 * (s - 0.5)) / Lg
        with np.errstate(divide="ignore", invalid="ignore"):
            ev = z + 1j * T / kap
        ok = np.isfinite(ev) & (np.abs(1 / np.where(kap == 0, np.nan, kap)) <= 4 * h)
        poly = np.stack([ev.real[ok], ev.imag[ok]], 1)
        P = r["prim"][(r["prim_piece"] == pi) & (r["prim_kind"] == 2)]
        V = np.vstack([P[:, :2], P[:, 2:4]])
        d = point_polyline_dist(V, poly) if poly.shape[0] > 1 else np.hypot(*(V - poly[0]).T)
        assert d.max() <= TOL + 1e-3, (pi, d.max())
        checked += 1
    assert checked > 0


def _restyle(sc, join, cap):
    s = W.concat([sc])
    s.join[:] = join
    s.cap[:] = cap
    return s


def _raster_check(sc, r, p, n=150, band=TOL + 2e-3):
    pp = _prims_by_path(r)
    prims = r["prim"][pp == p]
    lines = arcs_to_lines(prims) if np.any(prims[:, 4] != 0) else prims[:, :4]
    segs = path_segments(sc, p)
    h = float(sc.half_width[p])
    curve = dense_curve(segs, 6000)
    if curve.shape[0] == 0:
        curve = sc.pts[sc.path_pt_off()[p]][None].astype(np.float64)
    lo, hi = curve.min(0) - h - 2, curve.max(0) + h + 2
    gx = np.linspace(lo[0], hi[0], n) + 0.1234567
    gy = np.linspace(lo[1], hi[1], n) + 0.0765432
    G = np.stack(np.meshgrid(gx, gy), -1).reshape(-1, 2)
    w = winding(G, lines)
    d = curve_dist(G, segs) if segs else np.hypot(*(G - curve[0]).T)
    sure = np.abs(d - h) > band + 0.01
    return w, d, h, sure


@pytest.mark.parametrize("p", [0, 2, 4, 5, 6, 7, 8, 9, 10, 11, 12, 15, 16, 17, 18, 19])
def test_strong_correctness_raster_round_style(oracle_mod, p):
    """With round joins and round caps the stroke is exactly {x : dist(x, path) <= h}.
    The nonzero-rule fill of the outline must agree with it everywhere outside a
    band of tol around the boundary, and every winding number must be >= 0."""
    sc = _restyle(W.hand_cases(), W.JOIN_ROUND, W.CAP_ROUND)
    r = oracle.stroke(sc, TOL)
    w, d, h, sure = _raster_check(sc, r, p)
    assert np.all(w >= 0)
    inside = w != 0
    assert np.array_equal(inside[sure], (d <= h)[sure])


@pytest.mark.parametrize("p", range(4))
def test_strong_correctness_raster_pr1_paths(oracle_mod, p):
    sc = _restyle(W.pr1().subset(range(4)), W.JOIN_ROUND, W.CAP_ROUND)
    for arcs in (False, True):
        r = oracle.stroke(sc, TOL, arcs=arcs)
        w, d, h, sure = _raster_check(sc, r, p, n=120)
        assert np.all(w >= 0)
        assert np.array_equal((w != 0)[sure], (d <= h)[sure])


def test_near_cusp_renders_like_cusp(oracle_mod):
    """Section 7.3: a cusp and a near-cusp give the same stroke (up to tolerance)."""
    b = W._Builder()
    b.path([W.M(-100, 0), W.C(100, 100, -100, 100, 100, 0)], 5, cap=W.CAP_ROUND)
    b.path([W.M(-100, 0), W.C(100.0, 100.001, -99.999, 100.0, 100.0, 0.0)], 5, cap=W.CAP_ROUND)
    sc = b.build()
    r = oracle.stroke(sc, TOL)
    w0, d0, h, sure0 = _raster_check(sc, r, 0, n=200)
    w1, d1, _, sure1 = _raster_check(sc, r, 1, n=200)
    both = sure0 & sure1
    assert np.array_equal((w0 != 0)[both], (w1 != 0)[both])


def test_dashes_are_open_pieces_with_caps(oracle_mod):
    b = W._Builder()
    b.path([W.M(0, 0), W.L(100, 0)], 2, cap=W.CAP_BUTT, dash=[10, 5], dash_offset=0)
    b.path([W.M(0, 10), W.L(100, 10)], 2, cap=W.CAP_BUTT, dash=[10, 5], dash_offset=12)
    sc = b.build()
    r = oracle.stroke(sc, TOL)
    # 0..100 with [10 on, 5 off]: dashes start at 0,15,...,90 -> 7 dashes, each 1 segment + marker
    first = r["seg_path"] == 0
    assert np.count_nonzero(r["seg_kind"][first] == 2) == 7
    P = r["prim"][_prims_by_path(r) == 0]
    xs = np.unique(np.round(np.concatenate([P[:, 0], P[:, 2]]), 9))
    assert xs.tolist() == [0, 10, 15, 25, 30, 40, 45, 55, 60, 70, 75, 85, 90, 100]
    # offset 12: starts 3 into the gap -> first dash at 3..13
    P1 = r["prim"][_prims_by_path(r) == 1]
    xs1 = np.unique(np.round(np.concatenate([P1[:, 0], P1[:, 2]]), 9))
    assert xs1[:4].tolist() == [3, 13, 18, 28]


def test_fragile_fraction_small(oracle_mod):
    r = oracle.stroke(W.pr1(), TOL)
    assert np.mean(r["seg_margin"] < 1e-4) < 0.03
    r = oracle.stroke(W.map_like(n_paths=2000), 0.1)
    assert np.mean(r["seg_margin"] < 1e-4) < 0.02


def test_fragility_causes_partition_the_fragile_segments(oracle_mod):
    """The causes (plain 1e-4 rule, count sensitivity, and the reported but not
    exempt FP32-conditioning class) are disjoint; the fragile segments are exactly
    the first two; the raw margin never falls below the scaled one."""
    for sc, tol in ((W.pr1(), TOL), (W.curvature_stress(seed=13, n_paths=200), TOL)):
        r = oracle.stroke(sc, tol)
        f = oracle.fragility(r)
        assert not (f["strict"] & f["cond"]).any() and not (f["strict"] & f["sens"]).any()
        assert not (f["cond"] & f["sens"]).any()
        assert np.array_equal(f["strict"] | f["sens"], f["any"]) and not (f["cond"] & f["any"]).any()
        assert np.all(r["seg_raw_margin"] >= r["seg_margin"])
        assert f["sens"].any()


def test_arc_output_shares_one_subdivision_between_the_two_sides(oracle_mod):
    """Section 5: the arc count depends on |h| only, so both sides of a piece take the
    same arcs at the same Euler-spiral parameters.  Checked on the output itself: on
    every piece without an evolute patch, the +h and -h sides hold the same number of
    arcs, and the i-th vertices of the two sides are exactly 2h apart, i.e. offsets of
    one spine point."""
    sc = W.pr1(n_paths=40)
    r = oracle.stroke(sc, TOL, arcs=True)
    kind, side, piece, prim = r["prim_kind"], r["prim_side"], r["prim_piece"], r["prim"]
    path_of_seg = r["seg_path"]
    patched = set(piece[(kind == 2) | (kind == 3)].tolist())
    checked = 0
    for p in np.unique(piece[(kind == 0) | (kind == 1)]):
        if p < 0 or int(p) in patched:
            continue
        m = (piece == p) & ((kind == 0) | (kind == 1))
        plus, minus = prim[m & (side == 1)], prim[m & (side == -1)]
        if len(plus) == 0 or len(minus) == 0:
            continue
        assert len(plus) == len(minus), p
        v = np.vstack([plus[:, 0:2], plus[-1:, 2:4]])
        # the -h side lists its arcs in parameter order, each one reversed
        w = np.vstack([minus[:1, 2:4], minus[:, 0:2]])
        h = float(sc.half_width[path_of_seg[r["piece_seg"][p]]])
        gap = np.hypot(*(v - w).T)
        assert np.max(np.abs(gap - 2.0 * h)) <= 1e-9 * (1.0 + h + np.max(np.abs(v))), p
        checked += 1
    assert checked > 500


def test_work_counters(oracle_mod):
    """The arithmetic-roofline units: a line is one fit attempt; its outline is
    four separate primitives (two offsets, two butt caps), eight vertices.  A
    round-joined polyline of k lines takes k fits; its vertex count is the
    primitives plus one per chain."""
    r = oracle.stroke(W._Builder().path([W.M(0, 0), W.L(100, 0)], 5).build(), TOL)
    assert (r["n_fit"], r["n_vert"], r["prim"].shape[0]) == (1, 8, 4)
    pts = [W.M(0, 0), W.L(100, 0), W.L(100, 100), W.L(0, 100)]
    r = oracle.stroke(W._Builder().path(pts, 5, join=W.JOIN_BEVEL).build(), TOL)
    assert r["n_fit"] == 3
    # chains: per line its two offsets, per joint a bevel (1 line) and the inner
    # contour (2 lines through the joint), the two caps
    n_prim = r["prim"].shape[0]
    assert n_prim == 3 * 2 + 2 * 3 + 2
    assert r["n_vert"] == n_prim + (3 * 2 + 2 * 2 + 2)
