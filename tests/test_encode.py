"""Host encoder (Section 8.2, Table 1), checked against the verb definition: the
scan of the tag monoid (restated here in numpy) must hand every tag the control
points of the corresponding segment, and the tag sequence must match the
oracle's logical segments one for one."""
import numpy as np
import pytest

import oracle
import workloads as W
from geom import fill_path_segments, path_segments

TAG_END, TAG_F32, TAG_PATH, TAG_XFORM, TAG_STYLE, TAG_CLOSED = 0x04, 0x08, 0x10, 0x20, 0x40, 0x80


@pytest.fixture(scope="module")
def pkg():
    from paper_2405_00127_gb300 import build
    build.build()
    import paper_2405_00127_gb300 as P
    return P


def monoid_scan(tags):
    """Word offset of every tag's first point: a tag adds (count + 1 if it starts a
    subpath) points of 2 words (32-bit) or 1 word (16-bit); its first point is the
    previous tag's last unless it starts a subpath."""
    cc = (tags & 3).astype(np.int64)
    w = np.where(tags & TAG_F32, 2, 1)
    first = np.r_[True, (tags[:-1] & (TAG_END | TAG_PATH)) != 0]
    inc = np.where(cc == 0, 0, (cc + first) * w)
    E = np.concatenate([[0], np.cumsum(inc)[:-1]])
    pt_base = np.where(first | (cc == 0), E, E - w)
    path = np.concatenate([[0], np.cumsum((tags & TAG_PATH) != 0)[:-1]])
    style = np.cumsum((tags & TAG_STYLE) != 0) - 1
    return pt_base, path, style


def decode_points(words, base, n, tag):
    """n points from word `base` at the tag's width."""
    if tag & TAG_F32:
        return words[base:base + 2 * n].view(np.float32).reshape(n, 2).astype(np.float64)
    v = words[base:base + n]
    return np.stack([(v & 0xffff).astype(np.uint16).view(np.int16), (v >> 16).astype(np.uint16).view(np.int16)],
                    1).astype(np.float64)


def xform_index(tags):
    """Transform-stream index of every tag (-1 before the first entry)."""
    return np.cumsum((tags & TAG_XFORM) != 0) - 1


def scenes():
    b = W._Builder()
    b.path([W.M(0, 0), W.L(10, 0), W.L(10, 0), W.C(20, 0, 20, 10, 30, 10)], 2)          # zero-length dropped
    b.path([W.M(0, 0), W.L(10, 0), W.L(10, 10), W.Z], 2)                                  # closing line
    b.path([W.M(0, 0), W.L(10, 0), W.L(0, 0), W.Z], 2)                                    # closed, ends at start
    b.path([W.M(5, 5)], 2)                                                                # empty path
    b.path([W.M(1, 1), W.L(1, 1)], 3, cap=W.CAP_ROUND)                                    # dot
    b.path([W.M(0, 0), W.L(1, 0), W.M(5, 5), W.C(6, 6, 7, 5, 8, 5), W.Z, W.L(9, 9)], 2)  # several subpaths
    b.path([W.M(0, 0), W.L(4, 4)], 2)                                                     # same style as previous? no
    b.path([W.M(0, 0), W.L(4, 4)], 2)                                                     # identical style: shared entry
    f = W._Builder()
    f.path([W.M(0, 0), W.L(10, 0), W.L(10, 10)], 0.0, fill=True)                       # fill closes it
    f.path([W.M(0, 0), W.L(10, 0), W.L(0, 0)], 0.0, fill=True)                          # ends at start
    f.path([W.M(0, 0), W.L(3, 0), W.M(5, 5), W.C(6, 6, 7, 5, 8, 5)], 0.0, fill=True)   # two subpaths
    f.path([W.M(0, 0), W.L(4, 4)], 2)                                                     # a stroke among them
    q = W._Builder()
    q.path([W.M(0, 0), W.Q(5, 9, 10, 0), W.Q(10, 0, 10, 0), W.L(20, 0), W.Q(30, 5, 20, 10), W.Z], 2)   # zero quad dropped
    q.path([W.M(0, 0), W.Q(5, 5, 9, 0)], 2, transform=[2, 0, 0, 2, 1, 1])
    q.path([W.M(0, 0), W.C(1, 2, 3, 2, 4, 0)], 2, transform=[2, 0, 0, 2, 1, 1])                       # shared entry
    q.path([W.M(0, 0), W.L(4, 0)], 2)                                                                   # identity
    q.path([W.M(0, 0), W.Q(1, 1, 2, 0)], 1, fill=True, transform=[0, 1, -1, 0, 5, 5])
    g = W.glyph_like(n_glyphs=12)
    mixed = W.concat([W.pr1(seed=2, n_paths=3), g, W.map_like(seed=3, n_paths=5)]).with_coord16()
    return [b.build(), W.hand_cases(), W.pr1().subset(range(10)), W.map_like(n_paths=200), f.build(),
            W.map_like(seed=8, n_paths=150).as_fill(np.arange(150) % 3 == 0), q.build(),
            W.mmark_like(n_paths=120), W.mmark_like(seed=9, n_paths=80, per_path_transforms=True), g, mixed]


@pytest.mark.parametrize("k", range(11))
def test_tags_match_logical_segments(pkg, oracle_mod, k):
    sc = scenes()[k]
    enc = pkg.encode(sc)
    r = oracle.stroke(sc, 0.25)
    tags = enc.tags
    assert tags.size == r["seg_kind"].size
    kind = np.where(tags & 3 == 0, 3, np.where(tags & TAG_END, 2, -1))
    assert np.array_equal(kind == 2, r["seg_kind"] == 2)
    assert np.array_equal(kind == 3, r["seg_kind"] == 3)
    pt_base, path, style = monoid_scan(tags)
    assert np.array_equal(path, r["seg_path"])
    # path bit on the last tag of each path
    last = np.r_[r["seg_path"][1:] != r["seg_path"][:-1], True]
    assert np.array_equal((tags & TAG_PATH) != 0, last)
    # styles: one entry per run of identical consecutive styles
    st = pkg.styles_of(sc)
    assert np.array_equal(enc.styles[style], st[path])
    # transforms: one entry per run of identical consecutive transforms, the bit on
    # the first tag of each path that starts a run
    xf = sc.transforms()
    if sc.transform is None:
        assert enc.transforms is None and not np.any(tags & TAG_XFORM)
    else:
        xi = xform_index(tags)
        assert np.all(xi >= 0)
        assert np.array_equal(enc.transforms[xi], xf[path])
        first = np.r_[True, path[1:] != path[:-1]]
        assert not np.any((tags & TAG_XFORM != 0) & ~first)
    # control points of every segment tag
    cursor = {}
    for i, t in enumerate(tags):
        if t & 3 in (1, 2, 3) and not t & TAG_END:
            p = int(path[i])
            ps = fill_path_segments(sc, p) if sc.fill[p] else path_segments(sc, p)
            segs = cursor.setdefault(p, [s for s in ps if not np.all(s[1] == s[1][0])])
            is_line, c = segs.pop(0)
            pts = decode_points(enc.points, pt_base[i], (t & 3) + 1, t)
            assert bool(is_line) == ((t & 3) == 1)
            if is_line:
                assert np.array_equal(pts, c[[0, 3]])
            elif (t & 3) == 2:     # the stream holds the quadratic; c is its elevated cubic
                P0, Q1, P2 = pts
                el = np.stack([P0, P0 + 2 * (Q1 - P0) / 3, P2 + 2 * (Q1 - P2) / 3, P2])
                assert np.allclose(el, c, rtol=0, atol=1e-12 * max(1.0, np.abs(c).max()))
            else:
                assert np.array_equal(pts, c)


def test_closed_flag_and_marker_points(pkg):
    sc = scenes()[0]
    enc = pkg.encode(sc)
    tags = enc.tags
    pt_base, path, _ = monoid_scan(tags)
    markers = np.nonzero(tags & TAG_END)[0]
    closed = [(int(path[m]), bool(tags[m] & TAG_CLOSED)) for m in markers]
    assert (1, True) in closed and (2, True) in closed and (0, False) in closed
    for m in markers:     # marker data: the subpath start point
        first = m
        while first > 0 and not tags[first - 1] & TAG_END and (tags[first - 1] & 3) != 0 \
                and path[first - 1] == path[m]:
            first -= 1
        assert np.array_equal(decode_points(enc.points, pt_base[m], 2, tags[m])[1],
                              decode_points(enc.points, pt_base[first], 1, tags[first])[0])


def test_encoder_rejects_bad_input(pkg):
    from paper_2405_00127_gb300 import binding as B
    sc = W.hand_cases()
    bad = W.concat([sc])
    bad.pts[3, 0] = np.nan
    with pytest.raises(B.SeError):
        pkg.encode(bad)
    bad = W.concat([sc])
    bad.half_width[0] = 0.0
    with pytest.raises(B.SeError):
        pkg.encode(bad)
    bad = W.concat([sc])
    bad.verbs[0] = 7
    with pytest.raises(B.SeError):
        pkg.encode(bad)
    bad = sc.with_transform([1, 0, 0, 1, 0, 0])
    bad.transform[2, 4] = np.inf
    with pytest.raises(B.SeError):
        pkg.encode(bad)


def test_sixteen_bit_paths(pkg):
    """Table 1 bit 3: a path asking for 16-bit coordinates gets them exactly when all
    its coordinates are integers in range; its stream takes one word a point, and the
    whole stream is the 32-bit stream's points at their own widths."""
    g = W.glyph_like(n_glyphs=20)
    enc16 = pkg.encode(g)
    enc32 = pkg.encode(W.Scene(**{**g.__dict__, "coord16": None}))
    assert not np.any((enc16.tags & TAG_F32)[(enc16.tags & 3) != 0])
    assert np.all(enc32.tags & TAG_F32)
    n_pts = enc32.points.size // 2
    assert enc16.points.size == n_pts
    b16, _, _ = monoid_scan(enc16.tags)
    b32, _, _ = monoid_scan(enc32.tags)
    for i, t in enumerate(enc16.tags):
        n = (t & 3) + 1 if t & 3 else 0
        if n:
            assert np.array_equal(decode_points(enc16.points, b16[i], n, t),
                                  decode_points(enc32.points, b32[i], n, enc32.tags[i]))
    # a non-integer or out-of-range coordinate keeps its path 32-bit; the others switch
    sc = W.concat([W.glyph_like(seed=3, n_glyphs=3), W.pr1(seed=4, n_paths=2)]).with_coord16()
    big = W.glyph_like(seed=5, n_glyphs=1)
    big.pts = big.pts + 40000.0
    sc = W.concat([sc, big.with_coord16()])
    enc = pkg.encode(sc)
    _, path, _ = monoid_scan(enc.tags)
    f32_paths = sorted(set(path[(enc.tags & TAG_F32) != 0].tolist()))
    assert f32_paths == [3, 4, 5]
