"""Closed-form pins for the oracle's joins and caps (Section 8.1 and Algorithm 1:
joins and caps follow SVG semantics).

Every expected vertex here is built from textbook plane geometry, in FP64,
without the oracle's formulas:

- the offset of a point P with tangent T at signed distance s is P + s * n(T),
  n(T) = (T.y, -T.x) / |T| (the right normal; the oracle's +h side);
- the outer side of a join is the side the path turns away from: the +h side
  for a left turn (cross(Ti, To) >= 0), the -h side otherwise;
- a miter tip is the intersection of the two outer offset lines, found by
  solving a 2x2 linear system; SVG draws it when 1 / sin(phi / 2) <= the miter
  limit, phi the angle between the two segments at the joint, and a bevel
  (the chord between the two outer offset points) otherwise;
- the inner side runs from one inner offset point through the joint P to the
  other (the strongly correct inner contour);
- a butt cap is the chord between the two offsets of the end point, a square
  cap the three sides of the h x 2h rectangle beyond it, a round cap the half
  circle of radius h about it, bulging along the outward tangent.

Edges are compared as undirected segments (each side of the outline is
traversed in its own direction) to 1e-9.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

TOL = 0.25
EPS = 1e-9


def _normal(T):
    T = np.asarray(T, np.float64)
    return np.array([T[1], -T[0]]) / math.hypot(*T)


def _edges(poly):
    return [(np.asarray(a, np.float64), np.asarray(b, np.float64)) for a, b in zip(poly[:-1], poly[1:])]


def _same_edge_sets(got, want):
    """Every wanted undirected edge matched by exactly one got edge, and no extra."""
    if len(got) != len(want):
        return False
    used = [False] * len(got)
    for a, b in want:
        hit = False
        for k, (c, d) in enumerate(got):
            if used[k]:
                continue
            if (np.abs(a - c).max() < EPS and np.abs(b - d).max() < EPS) or \
               (np.abs(a - d).max() < EPS and np.abs(b - c).max() < EPS):
                used[k] = hit = True
                break
        if not hit:
            return False
    return True


def _intersect(A, Ta, B, Tb):
    """Intersection of the lines A + t Ta and B + u Tb."""
    M = np.array([[Ta[0], -Tb[0]], [Ta[1], -Tb[1]]], np.float64)
    t, _ = np.linalg.solve(M, np.asarray(B, np.float64) - np.asarray(A, np.float64))
    return np.asarray(A, np.float64) + t * np.asarray(Ta, np.float64)


def expected_join(P, Ti, To, h, style, ml):
    """(outer polyline, inner polyline) of the join at P from tangent Ti to To."""
    P, Ti, To = (np.asarray(v, np.float64) for v in (P, Ti, To))
    left = Ti[0] * To[1] - Ti[1] * To[0] >= 0.0
    s = h if left else -h
    A, B = P + s * _normal(Ti), P + s * _normal(To)
    Ai, Bi = P - s * _normal(Ti), P - s * _normal(To)
    inner = [Ai, P, Bi]
    if style == W.JOIN_BEVEL:
        return [A, B], inner
    if style == W.JOIN_MITER:
        # phi: angle between the two segments at the joint (between -Ti and To)
        cphi = np.dot(-Ti, To) / (np.linalg.norm(Ti) * np.linalg.norm(To))
        phi = math.acos(max(-1.0, min(1.0, cphi)))
        if phi > 0 and 1.0 / math.sin(phi / 2) <= ml:
            return [A, _intersect(A, Ti, B, To), B], inner
        return [A, B], inner
    raise ValueError(style)


def expected_cap(P, T, h, cap, start):
    """Polyline of a butt or square cap at P; T the path's tangent there.  The end
    cap bulges along T, the start cap against it."""
    P, T = np.asarray(P, np.float64), np.asarray(T, np.float64)
    u = T / np.linalg.norm(T)
    out = -u if start else u
    A, B = P + h * _normal(T), P - h * _normal(T)
    if cap == W.CAP_BUTT:
        return [A, B]
    if cap == W.CAP_SQUARE:
        return [A, A + h * out, B + h * out, B]
    raise ValueError(cap)


@pytest.fixture(scope="module")
def hand(oracle_mod):
    sc = W.hand_cases()
    return sc, oracle.stroke(sc, TOL)


def _prims(r, path, kinds):
    seg_of = np.repeat(np.arange(len(r["seg_count"])), r["seg_count"])
    m = (r["seg_path"][seg_of] == path) & np.isin(r["prim_kind"], kinds)
    return r["prim"][m, :4], r["prim_kind"][m], seg_of[m]


def _as_edges(rows):
    return [(row[0:2].copy(), row[2:4].copy()) for row in rows]


KIND = {v: k for k, v in oracle.PRIM_KINDS.items()}
OUTER, INNER, CAP = KIND["join_outer"], KIND["join_inner"], KIND["cap"]


def _check_join(r, path, P, Ti, To, h, style, ml=4.0):
    got, kinds, _ = _prims(r, path, [OUTER, INNER])
    outer, inner = expected_join(P, Ti, To, h, style, ml)
    assert _same_edge_sets(_as_edges(got[kinds == OUTER]), _edges(outer)), (path, got[kinds == OUTER], outer)
    assert _same_edge_sets(_as_edges(got[kinds == INNER]), _edges(inner)), (path, got[kinds == INNER], inner)
    return outer


def test_bevel_join_is_the_outer_chord(hand):
    """H13: bevel at (100, 900) between (100, 0) and (50, 80), h = 8."""
    _, r = hand
    outer = _check_join(r, 12, (100, 900), (100, 0), (50, 80), 8, W.JOIN_BEVEL)
    assert len(outer) == 2


def test_right_angle_miter_tip(hand):
    """H15: a 90-degree left turn at (100, 1100), h = 8: the miter tip is the
    corner pushed out by h along both normals, (100, 1100) + 8 (1, -1)."""
    _, r = hand
    outer = _check_join(r, 14, (100, 1100), (100, 0), (0, 100), 8, W.JOIN_MITER)
    assert np.abs(outer[1] - np.array([108.0, 1092.0])).max() < EPS


def test_miter_limit_exceeded_falls_back_to_bevel(hand):
    """H14: the segments meet at 11.3 degrees; 1 / sin(5.65 deg) = 10.1 > 4 -> bevel."""
    _, r = hand
    phi = math.acos(np.dot((-100, 0), (-100, 20)) / (100 * math.hypot(100, 20)))
    assert 1 / math.sin(phi / 2) > 4.0
    outer = _check_join(r, 13, (100, 1000), (100, 0), (-100, 20), 8, W.JOIN_MITER)
    assert len(outer) == 2


@pytest.mark.parametrize("ratio,miter", [(0.999, True), (1.001, False)])
@pytest.mark.parametrize("turn", [1.0, -1.0])
def test_miter_limit_threshold(oracle_mod, ratio, miter, turn):
    """A joint whose miter ratio 1 / sin(phi / 2) sits 0.1% under (miter) or over
    (bevel) the limit 4, turning left and right."""
    ml, h = 4.0, 3.0
    phi = 2 * math.asin(1.0 / (ml * ratio))          # angle between the segments
    psi = turn * (math.pi - phi)                      # signed turn of the tangent
    P = np.array([100.0, 0.0], np.float32)
    Q = (P + 100 * np.array([math.cos(psi), math.sin(psi)])).astype(np.float32)
    sc = W._Builder().path([W.M(0, 0), W.L(*P), W.L(*Q)], h, join=W.JOIN_MITER, miter_limit=ml).build()
    r = oracle.stroke(sc, TOL)
    To = Q.astype(np.float64) - P
    outer = _check_join(r, 0, P, (100, 0), To, h, W.JOIN_MITER, ml)
    assert len(outer) == (3 if miter else 2)
    if miter:  # the tip lies h / sin(phi / 2) from the joint, on the bisector's far side
        d = np.linalg.norm(outer[1] - P)
        assert abs(d - h / math.sin(phi / 2)) < 1e-6 * d


def test_right_turn_puts_outer_on_minus_h_side(oracle_mod):
    """The mirror of H15 (a right turn): the miter tip is (100, 0) + 8 (1, 1)."""
    sc = W._Builder().path([W.M(0, 0), W.L(100, 0), W.L(100, -100)], 8, join=W.JOIN_MITER).build()
    r = oracle.stroke(sc, TOL)
    outer = _check_join(r, 0, (100, 0), (100, 0), (0, -100), 8, W.JOIN_MITER)
    assert np.abs(outer[1] - np.array([108.0, 8.0])).max() < EPS


def test_closed_square_with_miters(hand):
    """H19: the closed square (700..800)^2 with h = 6 and miter joins: the outer
    contour is the square (694..806)^2 with its four corners as the miter tips,
    every side is offset by h both ways, and every inner join passes through its
    corner."""
    _, r = hand
    corners = [(800, 700), (800, 800), (700, 800), (700, 700)]
    dirs = [(100, 0), (0, 100), (-100, 0), (0, -100)]
    tips = []
    for k, P in enumerate(corners):
        Ti, To = dirs[k], dirs[(k + 1) % 4]
        outer, _ = expected_join(P, Ti, To, 6, W.JOIN_MITER, 4.0)
        tips.append(outer[1])
    assert sorted(map(tuple, np.round(tips, 9))) == sorted([(694, 694), (694, 806), (806, 694), (806, 806)])
    got, kinds, _ = _prims(r, 18, [OUTER, INNER])
    want_o, want_i = [], []
    for k, P in enumerate(corners):
        o, i = expected_join(P, dirs[k], dirs[(k + 1) % 4], 6, W.JOIN_MITER, 4.0)
        want_o += _edges(o)
        want_i += _edges(i)
    assert _same_edge_sets(_as_edges(got[kinds == OUTER]), want_o)
    assert _same_edge_sets(_as_edges(got[kinds == INNER]), want_i)
    # the parallel curves of the four sides: each side translated by +-h along its normal
    off, _, _ = _prims(r, 18, [KIND["offset"], KIND["offset_rev"]])
    want = []
    for k in range(4):
        a, b = np.asarray(corners[k - 1], np.float64), np.asarray(corners[k], np.float64)
        nrm = _normal(b - a)
        want += [(a + 6 * nrm, b + 6 * nrm), (a - 6 * nrm, b - 6 * nrm)]
    assert _same_edge_sets(_as_edges(off), want)


def _cap_edges(r, path, seg_kinds):
    got, _, seg = _prims(r, path, [CAP])
    return _as_edges(got[np.isin(r["seg_kind"][seg], seg_kinds)])


def test_square_caps_extend_by_h(hand):
    """H4: (0, 60) -> (100, 60), h = 5, square caps: rectangles 5 x 10 beyond both ends."""
    _, r = hand
    end = _cap_edges(r, 3, [0])
    start = _cap_edges(r, 3, [2])
    assert _same_edge_sets(end, _edges(expected_cap((100, 60), (100, 0), 5, W.CAP_SQUARE, False)))
    assert _same_edge_sets(start, _edges(expected_cap((0, 60), (100, 0), 5, W.CAP_SQUARE, True)))
    xs = np.array([e[0][0] for e in end + start] + [e[1][0] for e in end + start])
    assert xs.min() == -5.0 and xs.max() == 105.0


def test_butt_caps_are_the_end_chords(hand):
    """H1 (line) and H13's open end on (100, 900) -> (150, 980): butt caps are the
    chords between the two offsets of each end point."""
    _, r = hand
    assert _same_edge_sets(_cap_edges(r, 0, [0]), _edges(expected_cap((100, 0), (100, 0), 5, W.CAP_BUTT, False)))
    assert _same_edge_sets(_cap_edges(r, 0, [2]), _edges(expected_cap((0, 0), (100, 0), 5, W.CAP_BUTT, True)))
    assert _same_edge_sets(_cap_edges(r, 12, [0]), _edges(expected_cap((150, 980), (50, 80), 8, W.CAP_BUTT, False)))


def test_square_cap_on_a_curve_follows_the_sampled_tangent(oracle_mod):
    """A cubic's square caps lie along its end derivatives 3 (P1 - P0) and 3 (P3 - P2)."""
    P = np.array([[0, 0], [30, 0], [60, 30], [60, 60]], np.float64)
    sc = W._Builder().path([W.M(*P[0]), W.C(*P[1], *P[2], *P[3])], 4, cap=W.CAP_SQUARE).build()
    r = oracle.stroke(sc, TOL)
    assert _same_edge_sets(_cap_edges(r, 0, [0]), _edges(expected_cap(P[3], 3 * (P[3] - P[2]), 4, W.CAP_SQUARE, False)))
    assert _same_edge_sets(_cap_edges(r, 0, [2]), _edges(expected_cap(P[0], 3 * (P[1] - P[0]), 4, W.CAP_SQUARE, True)))


def test_round_cap_and_reversal_join_are_half_circles(hand):
    """H3's round caps and H12's round join at a 180-degree reversal: vertices on
    the circle of radius h about the end point, spread evenly over the half turn
    beyond it, with the count of the exact arc rule of Section 2.1,
    ceil(pi / (2 acos(1 - tol / h)))."""
    _, r = hand
    n = math.ceil(math.pi / (2 * math.acos(1 - TOL / 5)))
    for path, P, out_dir, kinds in ((2, (100, 40), (1, 0), [CAP]), (2, (0, 40), (-1, 0), [CAP]),
                                    (11, (100, 800), (1, 0), [OUTER])):
        got, _, _ = _prims(r, path, kinds)
        P = np.asarray(P, np.float64)
        # the primitives of this cap or join: both ends within h of its point
        e = got[(np.linalg.norm(got[:, 0:2] - P, axis=1) < 5 + 1e-9) & (np.linalg.norm(got[:, 2:4] - P, axis=1) < 5 + 1e-9)]
        assert len(e) == n, (path, len(e), n)
        for row in e:
            for v in (row[0:2], row[2:4]):
                assert abs(np.linalg.norm(v - P) - 5) < 1e-9
                assert np.dot(v - P, out_dir) >= -1e-9       # on the far side of the end point
            # equal angular steps: every chord subtends pi / n
            c = np.linalg.norm(row[2:4] - row[0:2])
            assert abs(c - 2 * 5 * math.sin(math.pi / (2 * n))) < 1e-9
