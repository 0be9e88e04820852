"""Nonzero coverage of the expanded outline on the GPU (se_coverage, the downstream
use of the line soup in Section 8.1): the per-pixel path counts and per-path areas
against a CPU raster of the same primitives, and the strong-correctness check of
Section 1 -- with round joins and caps, a path covers exactly the pixel centres
within h of its source curve, outside a band of the tolerance."""
import numpy as np
import pytest

import workloads as W
from geom import curve_dist, dense_curve, path_segments, winding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00127_gb300 import build
    build.build()
    import paper_2405_00127_gb300 as P
    e = P.StrokeExpander(0)
    yield e
    e.close()


def _arc_geometry(P):
    """Centre, radius and signed sweep of arc primitives (x0 y0 x1 y1 k)."""
    a, b, k = P[:, 0:2], P[:, 2:4], P[:, 4]
    ch = b - a
    c = np.hypot(ch[:, 0], ch[:, 1])
    r = 1.0 / np.where(k == 0, np.inf, np.abs(k))
    d = np.sqrt(np.maximum(r * r - c * c / 4, 0))
    nrm = np.stack([-ch[:, 1], ch[:, 0]], 1) / np.maximum(c, 1e-300)[:, None]
    cen = (a + b) / 2 + nrm * (np.sign(k) * d)[:, None]
    return cen, r


def _winding_exact(G, P, arcs):
    """Winding of points G about primitives P: a line's ray crossings, plus for an arc
    the circular segment between arc and chord (+-1 inside it, by turning sense)."""
    w = winding(G, P[:, :4])
    if arcs:
        m = P[:, 4] != 0
        A = P[m]
        cen, r = _arc_geometry(A)
        for i0 in range(0, A.shape[0], 512):
            a, b = A[i0:i0 + 512, 0:2], A[i0:i0 + 512, 2:4]
            cc, rr, kk = cen[i0:i0 + 512], r[i0:i0 + 512], A[i0:i0 + 512, 4]
            inside_circle = np.hypot(G[:, None, 0] - cc[None, :, 0], G[:, None, 1] - cc[None, :, 1]) < rr[None]
            side = (b[None, :, 0] - a[None, :, 0]) * (G[:, None, 1] - a[None, :, 1]) - \
                   (b[None, :, 1] - a[None, :, 1]) * (G[:, None, 0] - a[None, :, 0])
            # the arc bulges to the right of A -> B when it turns left (k > 0); the loop arc
            # A -> B, chord B -> A then runs counterclockwise, adding +1 inside the segment
            seg = inside_circle & (np.sign(side) == -np.sign(kk)[None])
            w = w + (seg * np.sign(kk)[None]).sum(1).astype(np.int64)
    return w


def _dist_to_prims(G, P, arcs):
    a, b = P[:, 0:2], P[:, 2:4]
    best = np.full(G.shape[0], np.inf)
    for i0 in range(0, P.shape[0], 512):
        aa, bb = a[i0:i0 + 512], b[i0:i0 + 512]
        d = bb - aa
        l2 = np.maximum((d * d).sum(1), 1e-300)
        ap = G[:, None, :] - aa[None]
        t = np.clip((ap * d[None]).sum(2) / l2[None], 0, 1)
        dd = np.hypot(ap[..., 0] - t * d[None, :, 0], ap[..., 1] - t * d[None, :, 1])
        best = np.minimum(best, dd.min(1))
    if arcs and np.any(P[:, 4] != 0):
        A = P[P[:, 4] != 0]
        cen, r = _arc_geometry(A)
        for i0 in range(0, A.shape[0], 512):
            dc = np.abs(np.hypot(G[:, None, 0] - cen[None, i0:i0 + 512, 0], G[:, None, 1] - cen[None, i0:i0 + 512, 1])
                        - r[None, i0:i0 + 512])
            best = np.minimum(best, dc.min(1))
    return best


def _gpu_outline(ex, sc, tol, arcs):
    import paper_2405_00127_gb300 as P
    out = ex.expand(ex.upload(P.encode(sc)), tol, arcs)
    prims = out.prims.cpu().numpy().astype(np.float64)
    curv = out.curvature.cpu().numpy().astype(np.float64) if arcs else np.zeros(out.n)
    return out, np.concatenate([prims, curv[:, None]], 1), out.path_offset.cpu().numpy()


@pytest.mark.parametrize("name,arcs", [("hand", False), ("hand", True), ("pr1", False), ("pr1", True),
                                       ("fill", False), ("mmark", False)])
def test_coverage_matches_cpu_raster(ex, name, arcs):
    import paper_2405_00127_gb300 as P
    sc = {"hand": lambda: W.hand_cases().with_transform([0.25, 0, 0, 0.25, 60, 10]),
          "pr1": lambda: W.pr1(seed=5).subset(range(6)).with_transform([0.15, 0, 0, 0.15, 3.3, 7.7]),
          "fill": lambda: W.pr1(seed=6).subset(range(6)).as_fill().with_transform([0.15, 0, 0, 0.15, 0, 0]),
          "mmark": lambda: W.mmark_like(seed=7, n_paths=60).with_transform([0.25, 0, 0, 0.25, 0, 0])}[name]()
    Wd, Ht = (350, 800) if name == "hand" else (200, 200)
    out, prims, poff = _gpu_outline(ex, sc, 0.25, arcs)
    cnt, area = P.coverage(ex, out, sc.n_paths, Wd, Ht, arcs)
    cnt, area = cnt.cpu().numpy(), area.cpu().numpy()
    ref = np.zeros((Ht, Wd), np.int64)
    ambiguous = np.zeros((Ht, Wd), bool)
    ref_area = np.zeros(sc.n_paths, np.int64)
    for p in range(sc.n_paths):
        Pp = prims[poff[p]:poff[p + 1]]
        if Pp.shape[0] == 0:
            continue
        x0, x1 = max(int(np.floor(min(Pp[:, 0].min(), Pp[:, 2].min()))) - 2, 0), min(int(np.ceil(max(Pp[:, 0].max(), Pp[:, 2].max()))) + 3, Wd)
        y0, y1 = max(int(np.floor(min(Pp[:, 1].min(), Pp[:, 3].min()))) - 2, 0), min(int(np.ceil(max(Pp[:, 1].max(), Pp[:, 3].max()))) + 3, Ht)
        if x0 >= x1 or y0 >= y1:
            continue
        gx, gy = np.meshgrid(np.arange(x0, x1) + 0.5, np.arange(y0, y1) + 0.5)
        G = np.stack([gx.ravel(), gy.ravel()], 1)
        w = _winding_exact(G, Pp, arcs)
        cov = (w != 0).reshape(y1 - y0, x1 - x0)
        ref[y0:y1, x0:x1] += cov
        ref_area[p] = cov.sum()
        # pixel centres within FP32 reach of an edge (or its 1e-3 chording) may go either way
        amb = _dist_to_prims(G, Pp, arcs) <= 2e-3 + 4 * np.finfo(np.float32).eps * max(Wd, Ht)
        ambiguous[y0:y1, x0:x1] |= amb.reshape(y1 - y0, x1 - x0)
    ok = ~ambiguous
    assert np.array_equal(cnt[ok], ref[ok])
    # per-path areas: equal up to the ambiguous pixels of that path
    assert np.all(np.abs(area - ref_area) <= ambiguous.sum())
    assert ref.sum() > 1000


@pytest.mark.parametrize("arcs", [False, True])
def test_coverage_is_strongly_correct(ex, arcs):
    """Round joins and caps: each path covers exactly the pixel centres within h of its
    source path, outside a band of tol + the fit error around the boundary (every
    winding >= 0, so the nonzero rule is the stroke)."""
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    sc = W.pr1(seed=8).subset(range(3))
    sc.join[:] = W.JOIN_ROUND
    sc.cap[:] = W.CAP_ROUND
    sc = sc.with_transform([0.2, 0, 0, 0.2, 10, 10])
    out, prims, poff = _gpu_outline(ex, sc, 0.25, arcs)
    Wd = Ht = 240
    band = 0.25 + 0.2 * 0.25 / 0.62 + 0.02
    import torch
    for p in range(sc.n_paths):
        lo, hi = int(poff[p]), int(poff[p + 1])
        one = P.Outline(out.prims[lo:hi], out.curvature[lo:hi] if arcs else None,
                        torch.zeros(hi - lo, dtype=torch.int32, device=ex.device), None, None, hi - lo, 0)
        cnt, _ = P.coverage(ex, one, 1, Wd, Ht, arcs, path_area=False)
        mask = cnt.cpu().numpy() > 0
        segs = [(isl, c * 0.2 + 10) for isl, c in path_segments(sc, p)]
        h = float(sc.half_width[p]) * 0.2
        curve = dense_curve(segs, 4000)
        x0, y0 = np.maximum(np.floor(curve.min(0) - h - 3).astype(int), 0)
        x1, y1 = np.minimum(np.ceil(curve.max(0) + h + 3).astype(int), [Wd, Ht])
        gx, gy = np.meshgrid(np.arange(x0, x1) + 0.5, np.arange(y0, y1) + 0.5)
        G = np.stack([gx.ravel(), gy.ravel()], 1)
        d = curve_dist(G, segs, spacing=0.02)
        sure = np.abs(d - h) > band
        inside = mask[y0:y1, x0:x1].ravel()
        assert np.array_equal(inside[sure], (d <= h)[sure]), p
        assert mask.sum() == mask[y0:y1, x0:x1].sum()    # nothing outside the stroke's box


def _rectilinear_paths(rng, specs):
    """Closed rectilinear polylines with integer vertices: path p passes through
    specs[p][0] random lattice points of the box specs[p][1] = (x0, y0, x1, y1), each
    joined to the next by a horizontal then a vertical move, and closes back to its
    first point.  Every edge lies on an integer line, so no pixel centre is near one
    and the coverage is exact."""
    prims, pid = [], []
    for p, (m, (x0, y0, x1, y1)) in enumerate(specs):
        pts = np.stack([rng.integers(x0, x1 + 1, m), rng.integers(y0, y1 + 1, m)], 1)
        nxt = np.roll(pts, -1, 0)
        corner = np.stack([nxt[:, 0], pts[:, 1]], 1)
        e = np.concatenate([np.stack([pts, corner], 1), np.stack([corner, nxt], 1)], 1).reshape(-1, 4)
        e = e[(e[:, 0] != e[:, 2]) | (e[:, 1] != e[:, 3])]
        prims.append(e)
        pid.append(np.full(e.shape[0], p))
    return np.concatenate(prims).astype(np.float32), np.concatenate(pid).astype(np.int32)


def _rectilinear_reference(prims, pid, n_paths, Wd, Ht):
    """Winding of every pixel centre as the running sum, along its row, of the
    directions of the vertical edges at or left of the column (a histogram per row
    and a cumulative sum), then the nonzero rule."""
    cnt = np.zeros((Ht, Wd), np.int64)
    area = np.zeros(n_paths, np.int64)
    for p in range(n_paths):
        e = prims[(pid == p) & (prims[:, 0] == prims[:, 2]) & (prims[:, 1] != prims[:, 3])].astype(np.int64)
        x, lo, hi = e[:, 0], np.minimum(e[:, 1], e[:, 3]), np.maximum(e[:, 1], e[:, 3])
        d = np.where(e[:, 3] > e[:, 1], 1, -1)
        diff = np.zeros((Ht, Wd + 1), np.int64)
        for r in range(Ht):
            c = (lo <= r) & (r < hi)          # lo <= r + 1/2 < hi for integer lo, hi
            np.add.at(diff[r], np.clip(x[c], 0, Wd), d[c])
        cov = np.cumsum(diff, 1)[:, :Wd] != 0
        cnt += cov
        area[p] = cov.sum()
    return cnt, area


def _row_crossings(prims, pid, p, r):
    e = prims[(pid == p) & (prims[:, 0] == prims[:, 2])]
    lo, hi = np.minimum(e[:, 1], e[:, 3]), np.maximum(e[:, 1], e[:, 3])
    return int(((lo <= r + 0.5) & (r + 0.5 < hi)).sum())


@pytest.mark.parametrize("grid", ["narrow", "wide"])
def test_coverage_long_rows_exact(ex, grid):
    """Rows crossed many times by one path, exact: buckets of a few crossings (one
    thread, a sorting network), of up to 32 (one warp, sorted across its lanes), of
    more within 1,024 columns (one warp, a column histogram), and wider ones (one
    block, sorted in shared memory up to 8,192 crossings and in global memory
    beyond), with paths reaching past the grid."""
    import torch
    import paper_2405_00127_gb300 as P
    rng = np.random.default_rng(11 if grid == "narrow" else 12)
    if grid == "narrow":
        Wd, Ht = 64, 64
        specs = [(200, (2, 2, 30, 30)),            # ~100 crossings per row
                 (40000, (34, 34, 44, 44)),        # ~20k crossings per row, 10 columns
                 (3000, (0, 40, 30, 63)),          # ~1k
                 (60, (-5, 50, 70, 60)),           # beyond the grid on both sides
                 (40, (40, 2, 62, 12))]            # 17 to 32 crossings per row
        specs += [(int(rng.integers(3, 12)), (int(a), int(b), int(a) + 8, int(b) + 8))
                  for a, b in rng.integers(0, 56, (40, 2))]
        big = [(1, 38, 8192)]
        warp = (4, range(2, 12))
    else:
        Wd, Ht = 3000, 12
        specs = [(200, (0, 0, 2990, 10)),          # ~60 crossings per row over ~3,000 columns
                 (40000, (-20, 1, 3020, 11)),      # ~13k crossings per row, past both sides
                 (100, (500, 2, 1900, 9)),         # ~1,400 columns
                 (300, (0, 0, 900, 11))]           # within the histogram
        specs += [(int(rng.integers(3, 12)), (int(a), int(b), int(a) + 8, int(b) + 4))
                  for a in rng.integers(0, 2990, 30) for b in rng.integers(0, 8, 1)]
        big = [(0, 5, 32), (1, 5, 8192), (2, 5, 32)]
        warp = None
    prims, pid = _rectilinear_paths(rng, specs)
    n = prims.shape[0]
    out = P.Outline(torch.from_numpy(prims).to(ex.device), None, torch.from_numpy(pid).to(ex.device),
                    None, None, n, 0)
    cnt, area = P.coverage(ex, out, len(specs), Wd, Ht)
    ref, ref_area = _rectilinear_reference(prims, pid, len(specs), Wd, Ht)
    assert np.array_equal(cnt.cpu().numpy(), ref)
    assert np.array_equal(area.cpu().numpy(), ref_area)
    for p, r, more in big:    # the rows that reach the large-bucket paths really are that large
        assert _row_crossings(prims, pid, p, r) > more
    if warp:                  # and some row of this path has 17 to 32 crossings
        assert any(16 < _row_crossings(prims, pid, warp[0], r) <= 32 for r in warp[1])
