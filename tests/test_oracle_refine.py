"""Pins for the refined flattening mode (Section 4.2): line counts from the exact
density integral of Section 4.1, vertices from two Newton steps started at the
approximation's inverse.  Checked against quadrature and root finding of the
density itself, and against the chord error of the emitted lines."""
import math

import numpy as np
import pytest
import scipy.integrate as si
from scipy.optimize import brentq

import oracle
import workloads as W


def _F(a, b):
    """int_a^b sqrt|u^2 - 1| du by adaptive quadrature (breakpoints at +-1)."""
    pts = [p for p in (-1.0, 1.0) if min(a, b) < p < max(a, b)]
    return si.quad(lambda u: math.sqrt(abs(u * u - 1)), a, b, points=pts or None, epsabs=1e-14, epsrel=1e-13,
                   limit=200)[0]


def test_exact_line_count_matches_density_quadrature(oracle_mod):
    """N = int sqrt|kappa (1 + sigma h kappa)| ds / sqrt(8 tol) with no approximation:
    the refined count equals the quadrature of the density to 1e-9 (the fast count
    is only within 6% of it)."""
    rng = np.random.default_rng(13)
    checked, fast_off = 0, 0.0
    for _ in range(1500):
        k0, k1 = rng.uniform(-4, 4, 2)
        sh = rng.choice([-1, 1]) * rng.uniform(0.01, 2.0)
        a, b = np.sort(rng.uniform(0, 1, 2))
        tol = 1e-3
        dens = lambda s: math.sqrt(abs((k0 + k1 * (s - .5)) * (1 + sh * (k0 + k1 * (s - .5)))))
        pts = [s for s in (0.5 - k0 / k1, 0.5 + (-1 / sh - k0) / k1) if a < s < b] if k1 else []
        q = si.quad(dens, a, b, points=pts or None, epsabs=1e-13, epsrel=1e-12, limit=200)[0] / math.sqrt(8 * tol)
        if q < 0.5:
            continue
        assert oracle.line_count_exact(k0, k1, sh, a, b, tol) == pytest.approx(q, rel=1e-9)
        fast_off = max(fast_off, abs(oracle.line_count(k0, k1, sh, a, b, tol) / q - 1))
        checked += 1
    assert checked > 300
    assert 0.01 < fast_off <= 0.06
    # constant curvature and a straight piece
    assert oracle.line_count_exact(2.0, 0.0, 0.25, 0.0, 1.0, 1e-3) == pytest.approx(
        math.sqrt(abs(2.0 * (1 + 0.25 * 2.0)) / 8e-3), rel=1e-12)
    assert oracle.line_count_exact(0.0, 0.0, 0.3, 0.0, 1.0, 1e-3) == 0.0


def test_refined_vertices_solve_the_density_integral(oracle_mod):
    """Vertex i of n splits the density integral in the ratio i : n - i to FP32
    accuracy of the range's integral after the two Newton steps Section 4.2 calls
    enough; the first step alone is not, and neither is the approximation."""
    rng = np.random.default_rng(5)
    worst, worst_guess = 0.0, 0.0
    for trial in range(300):
        ua, ub = rng.uniform(-6, 6, 2) if trial % 2 else rng.uniform(-1.6, 1.6, 2)
        if abs(ub - ua) < 1e-3:
            continue
        n = int(rng.integers(2, 24))
        T = _F(ua, ub)
        for i in range(1, n):
            u = oracle.refined_u(ua, ub, i, n)
            assert min(ua, ub) <= u <= max(ua, ub)
            worst = max(worst, abs(_F(ua, u) - i / n * T) / abs(T))
            g = oracle.f_approx_inv(oracle.f_exact(ua) + i / n * (oracle.f_exact(ub) - oracle.f_exact(ua)))
            g = min(max(g, min(ua, ub)), max(ua, ub))
            worst_guess = max(worst_guess, abs(_F(ua, g) - i / n * T) / abs(T))
    assert worst <= 2.0 ** -23
    assert worst_guess > 1e-4
    # an exact root found by bracketing agrees
    ua, ub, n = -2.5, 1.3, 7
    T = _F(ua, ub)
    for i in range(1, n):
        r = brentq(lambda u: _F(ua, u) - i / n * T, ua, ub, xtol=1e-15)
        assert oracle.refined_u(ua, ub, i, n) == pytest.approx(r, abs=1e-6)


def test_refined_derivative_is_the_density(oracle_mod):
    for x in (-3.0, -1.2, -0.4, 0.0, 0.7, 1.1, 2.5):
        h = 1e-6
        num = (_F(0.0, x + h) - _F(0.0, x - h)) / (2 * h)
        assert oracle.f_exact_deriv(x) == pytest.approx(num, rel=1e-6)
    assert oracle.f_exact_deriv(1.0) == 0.0 and oracle.f_exact_deriv(-1.0) == 0.0


def _es_offset_curve(rec, sh, n):
    """Dense points of the parallel curve of one ES piece record, from the unit ES
    (pinned against quadrature) placed on the piece's chord."""
    s = np.linspace(0.0, 1.0, n)
    U = np.array([oracle.es_unit_point(rec[10], rec[11], v) for v in s])
    Z = (U[:, 0] + 1j * U[:, 1]) * (rec[16] + 1j * rec[17]) + (rec[2] + 1j * rec[3])
    dZ = np.gradient(Z, s, edge_order=2)
    T = dZ / np.abs(dZ)
    O = Z + sh * (T.imag - 1j * T.real)
    return np.stack([O.real, O.imag], 1)


def _range_sagittas(sc, tol, refine, max_ranges=40):
    """Chord error of every line of the normal parallel-curve ranges, per range."""
    r = oracle.stroke(sc, tol, refine=refine)
    pth = np.repeat(r["seg_path"], r["seg_count"])
    out = []
    for p in np.unique(r["prim_piece"][(r["prim_kind"] == 0) & (r["prim_piece"] >= 0)]):
        rec = r["piece"][p]
        if rec[19]:
            continue
        for side in (1, -1):
            m = (r["prim_piece"] == p) & (r["prim_kind"] == 0) & (r["prim_side"] == side)
            if m.sum() < 4:
                continue
            C = _es_offset_curve(rec, side * float(sc.half_width[pth[m][0]]), 4000)
            sg = []
            for x0, y0, x1, y1 in r["prim"][m][:, :4]:
                i0 = np.argmin(np.hypot(C[:, 0] - x0, C[:, 1] - y0))
                i1 = np.argmin(np.hypot(C[:, 0] - x1, C[:, 1] - y1))
                seg = C[min(i0, i1):max(i0, i1) + 1]
                d = np.array([x1 - x0, y1 - y0])
                sg.append((np.abs((seg[:, 0] - x0) * d[1] - (seg[:, 1] - y0) * d[0]) / np.hypot(*d)).max())
            out.append(np.array(sg))
            if len(out) >= max_ranges:
                return out
    return out


def test_refined_lines_have_equal_chord_error_within_tol(oracle_mod):
    """Equal steps of the exact integral give every line of a range the same chord
    error (the density equalises it), at most tol; the fast mode's lines vary
    several times more and may pass tol by about 1%."""
    sc = W.pr1(seed=3, n_paths=8)
    tol = 0.25
    ref = _range_sagittas(sc, tol, True)
    fast = _range_sagittas(sc, tol, False)
    assert len(ref) >= 20 and len(fast) >= 20
    ref_spread = np.array([s[1:-1].max() / s[1:-1].min() for s in ref])
    fast_spread = np.array([s[1:-1].max() / s[1:-1].min() for s in fast])
    assert ref_spread.max() < 1.005          # higher-order terms of the asymptotic density
    assert np.median(fast_spread - 1) > 4 * np.median(ref_spread - 1)
    assert max(s.max() for s in ref) <= tol


def test_refined_mode_leaves_fills_and_arcs(oracle_mod):
    """Fills already invert their density exactly and arcs place vertices uniformly:
    neither changes in refined mode."""
    fills = W.pr1(seed=4, n_paths=4).as_fill()
    for sc, arcs in ((fills, False), (W.pr1(seed=4, n_paths=4), True)):
        a = oracle.stroke(sc, 0.1, arcs=arcs)
        b = oracle.stroke(sc, 0.1, arcs=arcs, refine=True)
        assert np.array_equal(a["prim"], b["prim"])


def test_refined_circle_offsets_take_the_chord_count(oracle_mod):
    """The parallel curves of a circle of radius R are circles of radius R +- h; with the
    exact integral each quarter takes ceil((pi/2) sqrt((R +- h) / 8 tol)) lines, the
    sagitta rule of Section 2.1 (the fast mode's approximate slope gives other counts)."""
    R, h, tol = 80.0, 6.0, 0.1
    bld = W._Builder()
    bld.path(W.circle_cmds(0, 0, R), h)
    r = oracle.stroke(bld.build(), tol, refine=True)
    off = r["prim_kind"] == 0
    want = sorted(int(np.ceil(np.pi / 2 * np.sqrt((R + sg * h) / (8 * tol)))) for sg in (1, -1))
    seg_of = np.repeat(np.arange(r["seg_count"].size), r["seg_count"])
    for q in range(4):
        got = sorted(int(((seg_of == q) & off & (r["prim_side"] == sd)).sum()) for sd in (1, -1))
        assert got == want
