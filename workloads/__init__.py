"""Seeded synthetic stroke workloads shared by the tests, the smoke check and the bench.

This module only *generates inputs*: SVG-style verb streams (Section 8.2 of
Levien & Uguray, "GPU-friendly Stroke Expansion") plus per-path stroke styles.
It holds none of the stroke-expansion arithmetic, so both the CUDA path and the
FP64 oracle can consume the same scenes without sharing any of the method.

Verb codes (one byte each) and the points they consume:
    MOVE  = 0  (1 point)   starts a subpath
    LINE  = 1  (1 point)
    CUBIC = 2  (3 points)
    CLOSE = 3  (0 points)  closes the current subpath
    QUAD  = 4  (2 points)  quadratic Bezier
Every path starts with MOVE.  Styles are per path, and so is the optional affine
transform (a b c d e f: x' = a x + c y + e, y' = b x + d y + f).

Join codes: 0 bevel, 1 miter, 2 round.  Cap codes: 0 butt, 1 square, 2 round.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MOVE, LINE, CUBIC, CLOSE, QUAD = 0, 1, 2, 3, 4
JOIN_BEVEL, JOIN_MITER, JOIN_ROUND = 0, 1, 2
CAP_BUTT, CAP_SQUARE, CAP_ROUND = 0, 1, 2
VERB_POINTS = np.array([1, 1, 3, 0, 2], dtype=np.int64)
IDENTITY = np.array([1, 0, 0, 1, 0, 0], np.float32)


@dataclasses.dataclass
class Scene:
    verbs: np.ndarray          # uint8 [V]
    pts: np.ndarray            # float32 [M, 2]
    path_verb_off: np.ndarray  # uint32 [P + 1]
    half_width: np.ndarray     # float32 [P]
    join: np.ndarray           # uint8 [P]
    cap: np.ndarray            # uint8 [P]
    miter_limit: np.ndarray    # float32 [P]
    dash_first: np.ndarray     # uint32 [P]
    dash_count: np.ndarray     # uint32 [P]  (0 = solid stroke)
    dash_offset: np.ndarray    # float32 [P]
    dash_len: np.ndarray       # float32 [D]
    fill: np.ndarray = None    # uint8 [P]: 1 = filled path (None = all stroked)
    transform: np.ndarray = None  # float32 [P, 6] per-path affine transform (None = identity)
    coord16: np.ndarray = None    # uint8 [P]: ask for 16-bit coordinates (None = all 32-bit)

    def __post_init__(self):
        if self.fill is None:
            self.fill = np.zeros(self.path_verb_off.shape[0] - 1, np.uint8)

    @property
    def n_paths(self) -> int:
        return int(self.path_verb_off.shape[0] - 1)

    @property
    def n_segments(self) -> int:
        """Input drawing segments (LINE + QUAD + CUBIC verbs)."""
        return int(np.count_nonzero((self.verbs == LINE) | (self.verbs == CUBIC) | (self.verbs == QUAD)))

    def transforms(self) -> np.ndarray:
        """[P, 6] transforms, identity where none is given."""
        if self.transform is None:
            return np.tile(IDENTITY, (self.n_paths, 1))
        return np.asarray(self.transform, np.float32).reshape(-1, 6)

    def with_transform(self, m) -> "Scene":
        """The same paths under one transform (6 numbers) or per-path transforms [P, 6]."""
        m = np.asarray(m, np.float32)
        t = np.tile(m.reshape(1, 6), (self.n_paths, 1)) if m.size == 6 else m.reshape(-1, 6).copy()
        return dataclasses.replace(self, transform=t)

    def path_pt_off(self) -> np.ndarray:
        per_verb = VERB_POINTS[self.verbs]
        csum = np.concatenate([[0], np.cumsum(per_verb)])
        return csum[self.path_verb_off.astype(np.int64)].astype(np.int64)

    def subset(self, paths) -> "Scene":
        """A scene holding only the given paths (in the given order)."""
        paths = np.asarray(paths, dtype=np.int64)
        vo = self.path_verb_off.astype(np.int64)
        po = self.path_pt_off()
        verbs, pts, voff, dfirst, dlen = [], [], [0], [], []
        nd = 0
        for p in paths:
            verbs.append(self.verbs[vo[p]:vo[p + 1]])
            pts.append(self.pts[po[p]:po[p + 1]])
            voff.append(voff[-1] + int(vo[p + 1] - vo[p]))
            f, c = int(self.dash_first[p]), int(self.dash_count[p])
            dfirst.append(nd)
            dlen.append(self.dash_len[f:f + c])
            nd += c
        return Scene(
            verbs=np.concatenate(verbs).astype(np.uint8) if verbs else np.zeros(0, np.uint8),
            pts=np.concatenate(pts).astype(np.float32) if pts else np.zeros((0, 2), np.float32),
            path_verb_off=np.asarray(voff, dtype=np.uint32),
            half_width=self.half_width[paths].copy(),
            join=self.join[paths].copy(),
            cap=self.cap[paths].copy(),
            miter_limit=self.miter_limit[paths].copy(),
            dash_first=np.asarray(dfirst, dtype=np.uint32),
            dash_count=self.dash_count[paths].copy(),
            dash_offset=self.dash_offset[paths].copy(),
            dash_len=np.concatenate(dlen).astype(np.float32) if dlen else np.zeros(0, np.float32),
            fill=self.fill[paths].copy(),
            transform=None if self.transform is None else self.transforms()[paths].copy(),
            coord16=None if self.coord16 is None else np.asarray(self.coord16, np.uint8)[paths].copy(),
        )

    def with_coord16(self, mask=None) -> "Scene":
        """The same scene asking for 16-bit coordinates on the paths in `mask` (default: all)."""
        c = np.ones(self.n_paths, np.uint8) if mask is None else np.asarray(mask, bool).astype(np.uint8)
        return dataclasses.replace(self, coord16=c)

    def as_fill(self, mask=None) -> "Scene":
        """The same geometry with the paths in `mask` (default: all) filled."""
        f = np.ones(self.n_paths, np.uint8) if mask is None else np.asarray(mask, bool).astype(np.uint8)
        return dataclasses.replace(self, fill=f)


def concat(scenes) -> Scene:
    verbs, pts, voff, hw, jn, cp, ml, dfirst, dcount, doff, dlen = [], [], [0], [], [], [], [], [], [], [], []
    nd = 0
    for s in scenes:
        verbs.append(s.verbs)
        pts.append(s.pts)
        voff.extend((s.path_verb_off[1:].astype(np.int64) + voff[-1]).tolist())
        hw.append(s.half_width); jn.append(s.join); cp.append(s.cap); ml.append(s.miter_limit)
        dfirst.append(s.dash_first.astype(np.int64) + nd); dcount.append(s.dash_count)
        doff.append(s.dash_offset); dlen.append(s.dash_len)
        nd += int(s.dash_len.shape[0])
    return Scene(
        verbs=np.concatenate(verbs).astype(np.uint8),
        pts=np.concatenate(pts).astype(np.float32).reshape(-1, 2),
        path_verb_off=np.asarray(voff, dtype=np.uint32),
        half_width=np.concatenate(hw).astype(np.float32),
        join=np.concatenate(jn).astype(np.uint8),
        cap=np.concatenate(cp).astype(np.uint8),
        miter_limit=np.concatenate(ml).astype(np.float32),
        dash_first=np.concatenate(dfirst).astype(np.uint32),
        dash_count=np.concatenate(dcount).astype(np.uint32),
        dash_offset=np.concatenate(doff).astype(np.float32),
        dash_len=np.concatenate(dlen).astype(np.float32),
        fill=np.concatenate([s.fill for s in scenes]).astype(np.uint8),
        transform=(np.concatenate([s.transforms() for s in scenes]).astype(np.float32)
                   if any(s.transform is not None for s in scenes) else None),
        coord16=(np.concatenate([np.zeros(s.n_paths, np.uint8) if s.coord16 is None else np.asarray(s.coord16, np.uint8)
                                 for s in scenes]) if any(s.coord16 is not None for s in scenes) else None),
    )


class _Builder:
    """Incremental builder used by the hand cases."""

    def __init__(self):
        self.verbs, self.pts, self.voff = [], [], [0]
        self.hw, self.join, self.cap, self.ml = [], [], [], []
        self.dfirst, self.dcount, self.doff, self.dlen = [], [], [], []
        self.fill = []
        self.xf = []

    def path(self, cmds, hw, join=JOIN_ROUND, cap=CAP_BUTT, miter_limit=4.0, dash=None, dash_offset=0.0,
             fill=False, transform=None):
        for c in cmds:
            op = c[0]
            self.verbs.append(op)
            for p in c[1:]:
                self.pts.append(p)
        self.voff.append(len(self.verbs))
        self.hw.append(hw); self.join.append(join); self.cap.append(cap); self.ml.append(miter_limit)
        self.dfirst.append(len(self.dlen))
        if dash:
            self.dlen.extend(dash)
            self.dcount.append(len(dash))
        else:
            self.dcount.append(0)
        self.doff.append(dash_offset)
        self.fill.append(1 if fill else 0)
        self.xf.append(None if transform is None else np.asarray(transform, np.float32).reshape(6))
        return self

    def build(self) -> Scene:
        return Scene(
            verbs=np.asarray(self.verbs, np.uint8),
            pts=np.asarray(self.pts, np.float32).reshape(-1, 2),
            path_verb_off=np.asarray(self.voff, np.uint32),
            half_width=np.asarray(self.hw, np.float32),
            join=np.asarray(self.join, np.uint8),
            cap=np.asarray(self.cap, np.uint8),
            miter_limit=np.asarray(self.ml, np.float32),
            dash_first=np.asarray(self.dfirst, np.uint32),
            dash_count=np.asarray(self.dcount, np.uint32),
            dash_offset=np.asarray(self.doff, np.float32),
            dash_len=np.asarray(self.dlen, np.float32),
            fill=np.asarray(self.fill, np.uint8),
            transform=(np.stack([IDENTITY if x is None else x for x in self.xf]).astype(np.float32)
                       if any(x is not None for x in self.xf) else None),
        )


def M(x, y):
    return (MOVE, (x, y))


def L(x, y):
    return (LINE, (x, y))


def C(x1, y1, x2, y2, x3, y3):
    return (CUBIC, (x1, y1), (x2, y2), (x3, y3))


def Q(x1, y1, x2, y2):
    return (QUAD, (x1, y1), (x2, y2))


Z = (CLOSE,)

# Handle length of the standard 4-cubic circle approximation, as a fraction of R.
CIRCLE_K = 0.5522847498


def circle_cmds(cx, cy, r):
    k = CIRCLE_K * r
    return [M(cx + r, cy),
            C(cx + r, cy + k, cx + k, cy + r, cx, cy + r),
            C(cx - k, cy + r, cx - r, cy + k, cx - r, cy),
            C(cx - r, cy - k, cx - k, cy - r, cx, cy - r),
            C(cx + k, cy - r, cx + r, cy - k, cx + r, cy), Z]


def hand_cases() -> Scene:
    """The 20 hand-built cases (tolerance 0.25, line output)."""
    b = _Builder()
    b.path([M(0, 0), L(100, 0)], 5, cap=CAP_BUTT)                                   # H1 line
    b.path([M(0, 20), C(25, 20, 75, 20, 100, 20)], 5, cap=CAP_BUTT)                 # H2 collinear cubic
    b.path([M(0, 40), L(100, 40)], 5, cap=CAP_ROUND)                                # H3 round caps
    b.path([M(0, 60), L(100, 60)], 5, cap=CAP_SQUARE)                               # H4 square caps
    b.path([M(50, 80), L(50, 80)], 5, cap=CAP_ROUND)                                # H5 zero-length dot
    b.path(circle_cmds(300, 300, 100), 5)                                            # H6 circle R100 hw5
    b.path(circle_cmds(300, 600, 100), 150)                                          # H7 hw > R
    b.path(circle_cmds(600, 300, 100), 100)                                          # H8 hw == R
    b.path([M(-100, 0), C(100, 100, -100, 100, 100, 0)], 5, cap=CAP_BUTT)            # H9 symmetric cusp
    b.path([M(-100, 200), C(100, 300, -100, 300, 100, 200)], 50, cap=CAP_BUTT)       # H10 cusp hw50
    b.path([M(-100.001, 400), C(100.0, 500.001, -99.999, 500.0, 100.001, 400.0)], 5)  # H11 jittered cusp
    b.path([M(0, 800), L(100, 800), L(0, 800)], 5, join=JOIN_ROUND, cap=CAP_BUTT)   # H12 180 reversal
    b.path([M(0, 900), L(100, 900), L(150, 980)], 8, join=JOIN_BEVEL)               # H13 bevel
    b.path([M(0, 1000), L(100, 1000), L(0, 1020)], 8, join=JOIN_MITER, miter_limit=4.0)  # H14 miter limit hit
    b.path([M(0, 1100), L(100, 1100), L(100, 1200)], 8, join=JOIN_MITER, miter_limit=4.0)  # H15 90 miter
    b.path([M(0, 1300), C(300, 1500, -100, 1500, 200, 1300)], 6)                     # H16 loop cubic
    b.path([M(0, 1600), C(50, 1700, 50, 1500, 100, 1600)], 6)                        # H17 S-cubic
    zig = [M(400, 1000)]
    for i in range(1, 41):
        zig.append(L(400 + 0.1 * i, 1000 + (0.1 if i % 2 else 0.0)))
    b.path(zig, 5, join=JOIN_MITER)                                                  # H18 tiny segments
    b.path([M(700, 700), L(800, 700), L(800, 800), L(700, 800), Z], 6, join=JOIN_MITER)  # H19 closed square
    k = CIRCLE_K * 1000
    b.path([M(1000, 2000), C(1000, 2000 + k, 1000 - 1000 + k, 3000, 0, 3000)], 4)  # H20 quarter circle R1000
    return b.build()


def _styles(rng, n, hw_lo, hw_hi, joins=(JOIN_MITER, JOIN_ROUND, JOIN_BEVEL), caps=(CAP_BUTT, CAP_SQUARE, CAP_ROUND)):
    hw = rng.uniform(hw_lo, hw_hi, n).astype(np.float32)
    join = rng.choice(np.asarray(joins, np.uint8), n)
    cap = rng.choice(np.asarray(caps, np.uint8), n)
    return hw, join, cap


def _walk_paths(rng, seg_counts, p_line, step_sigma, box, p_quad=0.0):
    """Open single-subpath paths whose successive points form a Gaussian random walk
    (segments are lines with probability p_line, quadratics with p_quad, else cubics)."""
    seg_counts = np.asarray(seg_counts, dtype=np.int64)
    n_paths = seg_counts.shape[0]
    n_seg = int(seg_counts.sum())
    r = rng.random(n_seg)
    is_cubic = r >= p_line + p_quad
    is_quad = (r >= p_line) & ~is_cubic
    seg_verb = np.where(is_cubic, CUBIC, np.where(is_quad, QUAD, LINE)).astype(np.uint8)
    # verbs: MOVE then the path's segments
    path_first_seg = np.concatenate([[0], np.cumsum(seg_counts)])
    verb_off = path_first_seg + np.arange(n_paths + 1)
    verbs = np.empty(n_seg + n_paths, np.uint8)
    move_pos = verb_off[:-1]
    verbs[move_pos] = MOVE
    seg_pos = np.ones(n_seg + n_paths, bool)
    seg_pos[move_pos] = False
    verbs[seg_pos] = seg_verb
    pts_per_seg = np.where(is_cubic, 3, np.where(is_quad, 2, 1))
    pts_per_path = 1 + np.add.reduceat(pts_per_seg, path_first_seg[:-1]) if n_seg else np.ones(n_paths, np.int64)
    pts_per_path = np.where(seg_counts > 0, pts_per_path, 1)
    n_pts = int(pts_per_path.sum())
    steps = rng.normal(0.0, step_sigma, (n_pts, 2))
    pt_off = np.concatenate([[0], np.cumsum(pts_per_path)])
    starts = rng.uniform(0.0, box, (n_paths, 2))
    steps[pt_off[:-1]] = starts
    csum = np.cumsum(steps, axis=0)
    base = np.repeat(csum[pt_off[:-1]] - starts, pts_per_path, axis=0)
    pts = (csum - base).astype(np.float32)
    return verbs, pts, verb_off.astype(np.uint32)


def _scene(verbs, pts, voff, hw, join, cap, ml=None, dash=None):
    n = hw.shape[0]
    if dash is None:
        dfirst = np.zeros(n, np.uint32)
        dcount = np.zeros(n, np.uint32)
        doff = np.zeros(n, np.float32)
        dlen = np.zeros(0, np.float32)
    else:
        dfirst, dcount, doff, dlen = dash
    return Scene(verbs=verbs, pts=pts, path_verb_off=voff, half_width=hw, join=join, cap=cap,
                 miter_limit=np.full(n, 4.0, np.float32) if ml is None else ml,
                 dash_first=dfirst, dash_count=dcount, dash_offset=doff, dash_len=dlen)


def pr1(seed: int = 1, n_paths: int = 200) -> Scene:
    """200 open paths of 8-32 cubics, control points uniform in a 1024x1024 box,
    half-width uniform [0.5, 10], round joins, butt caps (tolerance 0.25, lines)."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(8, 33, n_paths)
    n_seg = int(counts.sum())
    verb_off = np.concatenate([[0], np.cumsum(counts + 1)])
    verbs = np.full(n_seg + n_paths, CUBIC, np.uint8)
    verbs[verb_off[:-1]] = MOVE
    pts = rng.uniform(0.0, 1024.0, (n_paths + 3 * n_seg, 2)).astype(np.float32)
    hw = rng.uniform(0.5, 10.0, n_paths).astype(np.float32)
    return _scene(verbs, pts, verb_off.astype(np.uint32), hw,
                  np.full(n_paths, JOIN_ROUND, np.uint8), np.full(n_paths, CAP_BUTT, np.uint8))


def _dash_styles(seed, n_paths: int, frac: float):
    """A fraction `frac` of the paths dashed, each with a pattern of 2-4 lengths
    uniform in [2, 20] and an offset uniform in [0, period) (its own random
    stream, so the undashed draws of a scene do not change)."""
    rng = np.random.default_rng([*np.atleast_1d(seed).tolist(), 7])
    dashed = rng.random(n_paths) < frac
    k = rng.integers(2, 5, n_paths)
    dcount = np.where(dashed, k, 0).astype(np.uint32)
    dfirst = np.concatenate([[0], np.cumsum(dcount)[:-1]]).astype(np.uint32)
    dlen = rng.uniform(2.0, 20.0, int(dcount.sum())).astype(np.float32)
    doff = np.zeros(n_paths, np.float32)
    for p in np.nonzero(dashed)[0]:
        pat = dlen[dfirst[p]:dfirst[p] + dcount[p]].astype(np.float64)
        period = pat.sum() * (2 if pat.size % 2 else 1)
        doff[p] = rng.uniform(0.0, period)
    return dfirst, dcount, doff, dlen


def map_like(seed: int = 2, n_paths: int = 50_000, dash_frac: float = 0.0) -> Scene:
    """Map-like scene: per-path segment count ceil(lognormal(3, 1)); 60% line segments;
    points form a random walk with N(0, 8^2) steps from a start uniform in 4096^2;
    half-width uniform [0.25, 4]; joins uniform over miter(limit 4)/round/bevel;
    caps uniform over butt/square/round.  (Tolerance 0.1, lines and arcs.)
    With dash_frac > 0 that fraction of the paths is dashed (_dash_styles)."""
    rng = np.random.default_rng(seed)
    counts = np.ceil(rng.lognormal(3.0, 1.0, n_paths)).astype(np.int64)
    verbs, pts, voff = _walk_paths(rng, counts, 0.6, 8.0, 4096.0)
    hw, join, cap = _styles(rng, n_paths, 0.25, 4.0)
    dash = _dash_styles(seed, n_paths, dash_frac) if dash_frac > 0 else None
    return _scene(verbs, pts, voff, hw, join, cap, dash=dash)


def mmark_like(seed: int = 6, n_paths: int = 70_000, scale: float = 2.61, per_path_transforms: bool = False) -> Scene:
    """MotionMark-"Canvas Paths"-like scene: stroked paths of 1..3 segments, each a line,
    quadratic or cubic with equal probability, control points uniform in an 800 x 600
    box; half-width uniform [0.5, 5], joins and caps uniform; the whole scene scaled up
    by one uniform transform (scale, as when fitting it to a 2088 x 1600 target).  With
    per_path_transforms every path gets its own similarity (rotation, scale 0.5..4,
    translation) instead."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(1, 4, n_paths)
    n_seg = int(counts.sum())
    kinds = rng.integers(0, 3, n_seg)
    kind_verb = np.array([LINE, QUAD, CUBIC], np.uint8)[kinds]
    verbs, pts, voff = [], [], [0]
    k = 0
    for p in range(n_paths):
        verbs.append(MOVE)
        n_pt = 1
        for j in range(counts[p]):
            verbs.append(kind_verb[k])
            n_pt += int(VERB_POINTS[kind_verb[k]])
            k += 1
        pts.append(rng.uniform((0.0, 0.0), (800.0, 600.0), (n_pt, 2)))
        voff.append(len(verbs))
    hw, join, cap = _styles(rng, n_paths, 0.5, 5.0)
    sc = _scene(np.asarray(verbs, np.uint8), np.concatenate(pts).astype(np.float32), np.asarray(voff, np.uint32),
                hw, join, cap)
    if not per_path_transforms:
        return sc.with_transform([scale, 0, 0, scale, 0, 0])
    ang = rng.uniform(0, 2 * np.pi, n_paths)
    s_ = np.exp(rng.uniform(np.log(0.5), np.log(4.0), n_paths))
    tx, ty = rng.uniform(-500, 2500, n_paths), rng.uniform(-500, 2000, n_paths)
    m = np.stack([s_ * np.cos(ang), s_ * np.sin(ang), -s_ * np.sin(ang), s_ * np.cos(ang), tx, ty], 1)
    return sc.with_transform(m.astype(np.float32))


def glyph_like(seed: int = 8, n_glyphs: int = 2000, em: int = 2048, px: float = 16.0, stroked_frac: float = 0.25):
    """Text-like scene: glyph outlines with integer coordinates in font units (an em of
    2048) -- closed contours of lines and quadratics, 1-3 contours per glyph -- laid out in
    lines of text by per-glyph transforms scaling the em to `px` pixels; glyphs are
    filled, and `stroked_frac` of them are stroked instead (outlined text, half-width
    40-120 units).  Every path asks for 16-bit coordinates (they fit)."""
    rng = np.random.default_rng(seed)
    verbs, pts, voff = [], [], [0]
    for g in range(n_glyphs):
        for c in range(int(rng.integers(1, 4))):
            n = int(rng.integers(4, 12))
            ang = np.sort(rng.uniform(0, 2 * np.pi, n))
            cx, cy = rng.uniform(0.3 * em, 0.7 * em, 2)
            r = rng.uniform(0.15 * em, 0.35 * em) * rng.uniform(0.6, 1.0, n)
            P = np.stack([cx + r * np.cos(ang), cy + r * np.sin(ang)], 1)
            verbs.append(MOVE)
            pts.append(np.round(P[0]))
            for k in range(1, n + 1):
                q = P[k % n]
                if rng.random() < 0.6:
                    mid = 0.5 * (P[k - 1] + q) + rng.normal(0, 0.05 * em, 2)
                    verbs.append(QUAD)
                    pts.append(np.round(mid))
                    pts.append(np.round(q))
                else:
                    verbs.append(LINE)
                    pts.append(np.round(q))
            verbs.append(CLOSE)
        voff.append(len(verbs))
    # one path per glyph: voff currently per glyph
    s = px / em
    col, row = np.arange(n_glyphs) % 120, np.arange(n_glyphs) // 120
    m = np.stack([np.full(n_glyphs, s), np.zeros(n_glyphs), np.zeros(n_glyphs), np.full(n_glyphs, -s),
                  8 + col * px * 0.62, 8 + (row + 1) * px * 1.25], 1).astype(np.float32)
    stroked = rng.random(n_glyphs) < stroked_frac
    hw = np.where(stroked, rng.uniform(40, 120, n_glyphs), 1.0).astype(np.float32)
    join = rng.choice(np.asarray([JOIN_MITER, JOIN_ROUND, JOIN_BEVEL], np.uint8), n_glyphs)
    cap = np.full(n_glyphs, CAP_BUTT, np.uint8)
    sc = _scene(np.asarray(verbs, np.uint8), np.asarray(pts, np.float32).reshape(-1, 2), np.asarray(voff, np.uint32),
                hw, join, cap)
    sc.fill = (~stroked).astype(np.uint8)
    sc.transform = m
    sc.coord16 = np.ones(n_glyphs, np.uint8)
    return sc


def _min_radius(p):
    """Minimum radius of curvature of cubics p[n, 4, 2] by dense FP64 sampling."""
    t = np.linspace(0.0, 1.0, 257)[None, :, None]
    p = p.astype(np.float64)
    d1 = 3 * ((1 - t) ** 2 * (p[:, 1:2] - p[:, 0:1]) + 2 * (1 - t) * t * (p[:, 2:3] - p[:, 1:2])
              + t ** 2 * (p[:, 3:4] - p[:, 2:3]))
    d2 = 6 * ((1 - t) * (p[:, 2:3] - 2 * p[:, 1:2] + p[:, 0:1]) + t * (p[:, 3:4] - 2 * p[:, 2:3] + p[:, 1:2]))
    cr = np.abs(d1[..., 0] * d2[..., 1] - d1[..., 1] * d2[..., 0])
    sp = np.hypot(d1[..., 0], d1[..., 1])
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(cr > 0, sp ** 3 / cr, np.inf)
    return r.min(axis=1)


def curvature_stress(seed: int = 3, n_paths: int = 100_000, dashed: bool = True) -> Scene:
    """Single-cubic paths with near-cusp or self-crossing control polygons: four points
    uniform in a 256 box, P1 and P2 swapped, N(0,1) jitter on each; half-width
    U[5, 50] times the minimum radius of curvature (clamped to [0.05, 512]);
    dash [10, 5] with offset U[0, 15]; caps uniform.  (Tolerance 0.25, lines.)"""
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.0, 256.0, (n_paths, 4, 2))
    p[:, [1, 2]] = p[:, [2, 1]]
    p += rng.normal(0.0, 1.0, p.shape)
    p = p.astype(np.float32)
    rmin = _min_radius(p)
    hw = np.clip(rng.uniform(5.0, 50.0, n_paths) * rmin, 0.05, 512.0).astype(np.float32)
    verbs = np.tile(np.array([MOVE, CUBIC], np.uint8), n_paths)
    voff = (2 * np.arange(n_paths + 1)).astype(np.uint32)
    cap = rng.choice(np.array([CAP_BUTT, CAP_SQUARE, CAP_ROUND], np.uint8), n_paths)
    join = np.full(n_paths, JOIN_ROUND, np.uint8)
    dash = None
    if dashed:
        dash = (np.zeros(n_paths, np.uint32), np.full(n_paths, 2, np.uint32),
                rng.uniform(0.0, 15.0, n_paths).astype(np.float32), np.array([10.0, 5.0], np.float32))
    return _scene(verbs, p.reshape(-1, 2), voff, hw, join, cap, dash=dash)


def documents(seed: int = 4, n_docs: int = 4096, median: float = 300.0, sigma: float = 1.5,
              max_segs: int = 200_000, dash_frac: float = 0.0):
    """Independent documents whose segment counts are ceil(lognormal(ln median, sigma))
    clipped to [1, max_segs]; map-like geometry and styles inside each (with
    dash_frac > 0, that fraction of each document's paths dashed as in map_like)."""
    rng = np.random.default_rng(seed)
    sizes = np.clip(np.ceil(rng.lognormal(math.log(median), sigma, n_docs)), 1, max_segs).astype(np.int64)
    docs = []
    for target in sizes:
        counts = []
        left = int(target)
        while left > 0:
            c = int(min(left, max(1, math.ceil(rng.lognormal(3.0, 1.0)))))
            counts.append(c)
            left -= c
        verbs, pts, voff = _walk_paths(rng, np.asarray(counts), 0.6, 8.0, 4096.0)
        hw, join, cap = _styles(rng, len(counts), 0.25, 4.0)
        dash = _dash_styles([seed, len(docs)], len(counts), dash_frac) if dash_frac > 0 else None
        docs.append(_scene(verbs, pts, voff, hw, join, cap, dash=dash))
    return docs


def serving_pool(seed: int = 5, n_docs: int = 24, lo: float = 1e3, hi: float = 5e6, dash_frac: float = 0.3):
    """Documents whose segment counts are log-uniform in [lo, hi]: map-like
    geometry and styles, a fraction dash_frac of each document's paths dashed."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), n_docs))
    docs = []
    for k, target in enumerate(sizes):
        n_paths = max(1, int(round(target / 33.1)))   # ceil(lognormal(3, 1)) averages ~33 segments
        docs.append(map_like(seed=int(rng.integers(1 << 31)), n_paths=n_paths, dash_frac=dash_frac))
    return docs
