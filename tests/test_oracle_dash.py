"""Pins of the oracle's dashing (SVG dash semantics; the paper dashes on the CPU,
Section 9.3): the arc length it cuts by, where the cuts fall, and the margins it
reports for decisions that FP32 cannot resolve."""
import numpy as np
import pytest

import oracle
import workloads as W

TOL = 0.25


def _folded_length(p):
    """Arc length of a cubic whose control points lie on the x axis: the total
    variation of x(t) on [0, 1], from the roots of x'(t) (a closed form with a
    true cusp wherever x' changes sign)."""
    x0, x1, x2, x3 = p
    a = 3 * (x3 - 3 * x2 + 3 * x1 - x0)
    b = 6 * (x2 - 2 * x1 + x0)
    c = 3 * (x1 - x0)
    roots = [r.real for r in np.roots([a, b, c]) if abs(r.imag) < 1e-14 and 0 < r.real < 1]
    ts = [0.0] + sorted(roots) + [1.0]
    x = lambda t: (1 - t) ** 3 * x0 + 3 * (1 - t) ** 2 * t * x1 + 3 * (1 - t) * t * t * x2 + t ** 3 * x3
    return sum(abs(x(b_) - x(a_)) for a_, b_ in zip(ts[:-1], ts[1:]))


@pytest.mark.parametrize("xs", [(0, 2, -1, 1), (0, 3, -2, 1), (0, 1, 2, 3), (5, -4, 4, 0)])
def test_arc_length_of_folded_cubics(oracle_mod, xs):
    pts = np.array([[x, 0.0] for x in xs])
    assert oracle.seg_length(pts) == pytest.approx(_folded_length(xs), rel=1e-12, abs=1e-12)


def test_arc_length_of_lines_and_partial_lengths(oracle_mod):
    pts = np.array([[1.0, 2.0], [1.0, 2.0], [4.0, 6.0], [4.0, 6.0]])
    assert oracle.seg_length(pts, is_line=True) == pytest.approx(5.0, rel=1e-15)
    assert oracle.seg_length(pts, 0.3, is_line=True) == pytest.approx(1.5, rel=1e-15)
    # a uniformly parametrised straight cubic: length t * |P3 - P0|
    u = np.array([[0.0, 0.0], [1.0, 1.0], [2.0, 2.0], [3.0, 3.0]])
    for t in (0.1, 0.5, 0.9):
        assert oracle.seg_length(u, t) == pytest.approx(t * 3 * np.sqrt(2), rel=1e-13)


def test_arc_length_near_cusp_against_quadpack(oracle_mod):
    """Near-cusp cubics of the curvature-stress workload against QUADPACK's
    adaptive quadrature (scipy), an independent routine."""
    from scipy import integrate
    sc = W.curvature_stress(seed=21, n_paths=40, dashed=False)
    P = sc.pts.astype(np.float64).reshape(-1, 4, 2)
    for p in P:
        sp = lambda t: np.linalg.norm(3 * ((1 - t) ** 2 * (p[1] - p[0]) + 2 * (1 - t) * t * (p[2] - p[1]) + t * t * (p[3] - p[2])))
        ref = integrate.quad(sp, 0, 1, limit=2000, epsabs=1e-13, epsrel=1e-13, points=[0.5])[0]
        assert oracle.seg_length(p) == pytest.approx(ref, rel=1e-10)


def test_param_at_inverts_the_length(oracle_mod):
    p = np.array([[0.0, 0.0], [100.0, 120.0], [-50.0, 80.0], [90.0, 10.0]])
    total = oracle.seg_length(p)
    for f in (0.01, 0.3, 0.77, 0.999):
        t = oracle.seg_param_at(p, f * total)
        assert 0.0 < t < 1.0
        assert oracle.seg_length(p, t) == pytest.approx(f * total, rel=1e-12)


def test_dash_cuts_follow_the_pattern_on_a_curve(oracle_mod):
    """Every dash of a curved path starts and ends where the arc length from the
    subpath start crosses a pattern boundary (pattern [7, 3, 2]: odd, so walked
    twice: on 7, off 3, on 2, off 7, on 3, off 2)."""
    b = W._Builder()
    b.path([W.M(10, 10), W.C(60, 90, 120, -40, 160, 30)], 1.0, cap=W.CAP_BUTT, dash=[7, 3, 2], dash_offset=4)
    sc = b.build()
    r = oracle.stroke(sc, TOL)
    src = sc.pts.astype(np.float64)
    total = oracle.seg_length(src)
    pat = [7, 3, 2, 7, 3, 2]
    bounds, pos, k = [], -4.0, 0
    while pos < total:
        bounds.append((pos, k % 2 == 0))
        pos += pat[k % 6]
        k += 1
    ons = [(max(s, 0.0), min(s + pat[i % 6], total)) for i, (s, on) in enumerate(bounds) if on and s + pat[i % 6] > 0]
    ons = [(a, b_) for a, b_ in ons if b_ > a]
    assert np.count_nonzero(r["seg_kind"] == 2) == len(ons)
    # each dash's butt-cap midpoints sit on the source curve at the dash's arc-length ends
    P = r["prim"][r["prim_kind"] == 6]          # cap primitives: end cap then start cap per dash
    mids = 0.5 * (P[:, :2] + P[:, 2:4])
    def point_at(s):
        t = oracle.seg_param_at(src, s)
        mt = 1 - t
        return mt ** 3 * src[0] + 3 * mt * mt * t * src[1] + 3 * mt * t * t * src[2] + t ** 3 * src[3]
    want = []
    for a, b_ in ons:
        want += [point_at(b_), point_at(a)]
    assert np.allclose(mids, np.array(want), atol=1e-9)


def test_dash_margin_flags_boundary_at_segment_end(oracle_mod):
    b = W._Builder()
    b.path([W.M(0, 0), W.L(100, 0)], 2, dash=[10, 5], dash_offset=0)      # ends exactly on a boundary
    b.path([W.M(0, 5), W.L(97, 5)], 2, dash=[10, 5], dash_offset=0)       # 3 units before 100
    b.path([W.M(0, 9), W.L(100, 9)], 2)                                  # solid
    r = oracle.stroke(b.build(), TOL)
    dm = np.full(3, np.inf)
    np.minimum.at(dm, r["seg_path"], r["seg_dash_margin"])
    assert dm[0] == 0.0
    assert dm[1] == pytest.approx(3.0 / (1e-2 * (97 + 15)), rel=1e-12)
    assert dm[2] == np.inf


def test_short_part_far_from_origin_is_fragile(oracle_mod):
    """The same short, nearly straight dash part is resolved in FP32 near the
    origin but not at coordinates ~1e4 (its control points are rounded there)."""
    def scene(off):
        b = W._Builder()
        b.path([W.M(off, off), W.C(off + 30, off + 0.2, off + 60, off - 0.2, off + 90, off)], 200.0,
               cap=W.CAP_BUTT, dash=[0.5, 9.5], dash_offset=0)
        return b.build()
    near = oracle.stroke(scene(0.0), TOL)
    far = oracle.stroke(scene(1e4), TOL)
    assert np.count_nonzero(far["seg_margin"][far["seg_kind"] == 0] < 1e-4) > \
        np.count_nonzero(near["seg_margin"][near["seg_kind"] == 0] < 1e-4)
