"""GPU parity of fill flattening (Algorithm 1, fill branch: the source curve at
offset 0, 2/3-power density) against the FP64 oracle, segment by segment, alone
and mixed with solid and dashed strokes."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import FRAGILE, closed_per_path, compare

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


def hand_fills():
    b = W._Builder()
    b.path(W.circle_cmds(0, 0, 100), 1.0, fill=True)                                          # circle
    b.path([W.M(200, 0), W.L(260, 10), W.L(240, 70)], 1.0, fill=True)                         # open -> closed
    b.path([W.M(0, 300), W.C(300, 500, -100, 500, 200, 300)], 1.0, fill=True)                 # self-crossing loop
    b.path([W.M(400, 0), W.C(500, 200, 600, -200, 700, 0), W.L(550, 150), W.Z], 1.0, fill=True)  # inflection
    b.path([W.M(0, 600), W.L(30, 600), W.M(50, 650), W.C(60, 660, 70, 650, 80, 650)], 1.0, fill=True)
    b.path([W.M(900, 900), W.L(900, 900)], 1.0, fill=True)                                    # zero-length
    b.path([W.M(5, 5)], 1.0, fill=True)                                                        # empty
    b.path([W.M(0, 800), W.C(40, 880, 120, 770, 150, 840)], 6.0, cap=W.CAP_ROUND,
           dash=[5, 3], dash_offset=1, fill=True)                                              # stroke fields ignored
    b.path([W.M(0, 1000), W.C(40, 1080, 120, 970, 150, 1040)], 6.0, cap=W.CAP_ROUND)            # a stroke beside
    return b.build()


@pytest.mark.parametrize("arcs", [False, True])
def test_hand_fills(ex, oracle_mod, arcs):
    rep, g, _ = compare(ex, hand_fills(), 0.25, arcs)
    assert closed_per_path(g) == []
    print(rep)


@pytest.mark.parametrize("arcs", [False, True])
def test_pr1_filled(ex, oracle_mod, arcs):
    rep, g, _ = compare(ex, W.pr1().as_fill(), 0.25, arcs)
    assert rep["fragile"] <= 0.03 * rep["n_seg"]
    assert closed_per_path(g) == []
    print(rep)


def test_map_like_mixed_fills_strokes_dashes(ex, oracle_mod):
    """30% of the paths dashed strokes, every third path a fill (dash ignored),
    the rest solid strokes: ~10k tags, several scan tiles."""
    sc = W.map_like(seed=14, n_paths=300, dash_frac=0.3)
    sc = sc.as_fill(np.arange(sc.n_paths) % 3 == 0)
    r = oracle.stroke(sc, 0.1)
    dm = np.full(sc.n_paths, np.inf)
    np.minimum.at(dm, r["seg_path"], r["seg_dash_margin"])
    keep = np.nonzero(dm >= FRAGILE)[0]
    sub = sc.subset(keep)
    rep, g, _ = compare(ex, sub, 0.1, False)
    assert closed_per_path(g) == []
    print(rep)
