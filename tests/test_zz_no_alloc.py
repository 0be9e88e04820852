"""The count -> offset scan that allocates nothing, for callers that may not call
cudaMalloc (a device budget reserved up front, a render loop that must not block on
the allocator, a plugin whose host owns all device memory).  Its offsets must equal
the per-tag offsets the regular expansion entry point writes, on two calls in a row
(the shared scratch array keeps the previous call's contents)."""
import numpy as np
import pytest

import workloads as W

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


def _tag_offsets(ex, scene, tol):
    import paper_2405_00127_gb300 as P
    ds = ex.upload(P.encode(scene))
    out = ex.expand(ds, tol)
    return out.tag_offset.clone()


def test_noalloc_offsets_match_expansion_twice(ex):
    import torch
    from paper_2405_00127_gb300 import binding as B
    stream = torch.cuda.current_stream().cuda_stream
    for scene, tol in ((W.pr1(), 0.25), (W.map_like(seed=31, n_paths=5000), 0.1)):
        ref = _tag_offsets(ex, scene, tol)                          # regular entry point
        counts = (ref[1:] - ref[:-1]).to(torch.int32).contiguous()  # per-tag primitive counts
        n = counts.numel()
        got = torch.full((n + 1,), -1, dtype=torch.int64, device=ref.device)
        code = B.se_scan_offsets_noalloc(counts.data_ptr(), n, got.data_ptr(), stream)
        assert code == B.SE_OK
        assert torch.equal(got, ref)
        # independent of the library's scans: the host's prefix sum of the same counts
        host = np.concatenate([[0], np.cumsum(counts.cpu().numpy().astype(np.int64))])
        assert np.array_equal(got.cpu().numpy(), host)
        again = torch.full((n + 1,), -1, dtype=torch.int64, device=ref.device)
        code = B.se_scan_offsets_noalloc(counts.data_ptr(), n, again.data_ptr(), stream)
        assert code == B.SE_OK
        assert torch.equal(again, ref)


def test_noalloc_rejects_oversize(ex):
    import torch
    from paper_2405_00127_gb300 import binding as B
    dummy = torch.zeros(2, dtype=torch.int64, device="cuda")
    code = B.se_scan_offsets_noalloc(dummy.data_ptr(), (1 << 24) + 1, dummy.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    assert code == B.SE_ERR_INVALID_ARG


@pytest.mark.parametrize("n", [0, 1, 4095, 4096, 4097, 3 * 4096 + 17])
def test_noalloc_matches_host_prefix_sum(ex, n):
    """Ragged sizes around the scan tile (4096 counts) and the empty case, whose
    single offset (0) is written without a scan."""
    import torch
    from paper_2405_00127_gb300 import binding as B
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(n + 7)
    h_counts = rng.integers(0, 1000, max(n, 1)).astype(np.uint32)[:n]
    counts = torch.from_numpy(h_counts.view(np.int32).copy()).to("cuda")
    want = np.concatenate([[0], np.cumsum(h_counts.astype(np.int64))])
    for _ in range(2):  # the second call starts from the first call's leftover scratch
        got = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
        code = B.se_scan_offsets_noalloc(counts.data_ptr() if n else 0, n, got.data_ptr(), stream)
        assert code == B.SE_OK
        assert np.array_equal(got.cpu().numpy(), want)
