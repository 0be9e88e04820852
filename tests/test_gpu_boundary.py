"""The boundary's memory and failure contract, through the C ABI on the GPU:

- device memory comes from the caller's allocator (PyTorch's caching allocator
  by default), and the results do not depend on which allocator provides it;
- an allocation the caller's allocator refuses fails the call with SE_ERR_OOM
  and leaves the context usable (the failure is made on the host);
- a bounded device wait that runs out (a look-back flag that nothing sets, a
  bulk-copy barrier phase that nothing completes) returns SE_ERR_TIMEOUT
  instead of hanging, and the context stays usable.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00127_gb300 import build
    build.build()
    import paper_2405_00127_gb300 as P
    from paper_2405_00127_gb300 import binding as B
    return P, B


def _outline(ex, scene, tol=0.25):
    import paper_2405_00127_gb300 as P
    out = ex.expand(ex.upload(P.encode(scene)), tol)
    return out.prims.cpu().numpy(), out.tag_offset.cpu().numpy()


class Counting:
    """Wraps PyTorch's caching allocator, counting calls and live bytes; refuses
    the first `refuse` allocations."""

    def __init__(self, device=0, refuse=0):
        import torch
        self.torch, self.device = torch, device
        self.refuse = refuse
        self.calls = self.frees = 0
        self.live = {}

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.refuse > 0:
            self.refuse -= 1
            return None
        p = self.torch.cuda.caching_allocator_alloc(max(nbytes, 1), self.device, stream)
        self.live[p] = nbytes
        return p

    def free(self, ptr, stream):
        self.frees += 1
        self.live.pop(ptr)
        self.torch.cuda.caching_allocator_delete(ptr)


def test_caller_allocator_provides_the_workspace(lib):
    P, B = lib
    import torch
    sc = W.pr1(n_paths=60)
    cnt = Counting()
    alloc = B.Allocator(cnt.alloc, cnt.free)
    ex = P.StrokeExpander(0, allocator=alloc)
    before = torch.cuda.memory_allocated(0)
    got = _outline(ex, sc)
    assert cnt.calls > 0 and cnt.live, "the library allocated nothing through the caller's allocator"
    # the workspace sits in torch's pool, counted by torch
    assert torch.cuda.memory_allocated(0) - before >= sum(cnt.live.values())
    ex.close()
    assert cnt.live == {} and cnt.frees == cnt.calls   # every block given back on destroy
    ref_ex = P.StrokeExpander(0, allocator="cuda")     # the stream-ordered allocator
    ref = _outline(ref_ex, sc)
    ref_ex.close()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_refused_allocation_is_oom_and_context_stays_usable(lib):
    P, B = lib
    sc = W.pr1(n_paths=30)
    cnt = Counting(refuse=1)
    ex = P.StrokeExpander(0, allocator=B.Allocator(cnt.alloc, cnt.free))
    ds = ex.upload(P.encode(sc))
    with pytest.raises(P.SeError) as e:
        ex.count(ds, 0.25)
    assert e.value.code == B.SE_ERR_OOM
    n = ex.count(ds, 0.25)                               # the next call allocates and succeeds
    assert n > 0
    got = _outline(ex, sc)
    ex.close()
    ref_ex = P.StrokeExpander(0)
    ref = _outline(ref_ex, sc)
    ref_ex.close()
    assert np.array_equal(got[0], ref[0])


def test_allocator_that_always_refuses(lib):
    P, B = lib
    ex = P.StrokeExpander(0, allocator=B.Allocator(lambda n, s: None, lambda p, s: None))
    ds = ex.upload(P.encode(W.hand_cases()))
    for _ in range(2):
        with pytest.raises(P.SeError) as e:
            ex.count(ds, 0.25)
        assert e.value.code == B.SE_ERR_OOM
    ex.close()


def test_mismatched_allocator_pair_is_invalid(lib):
    P, B = lib
    import ctypes
    import torch
    h = ctypes.c_void_p()
    a = B.Allocator(lambda n, s: None, lambda p, s: None)
    code = B.lib().se_ctx_create(0, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), a.alloc_fn,
                                 B.SE_FREE_FN(), None, ctypes.byref(h))
    assert code == B.SE_ERR_INVALID_ARG


@pytest.mark.parametrize("spin_limit", [1, 64, 4096])
def test_bounded_wait_runs_out(lib, spin_limit):
    """The look-back scan's wait on a predecessor that never publishes gives up
    after spin_limit polls with SE_ERR_TIMEOUT; the same context then expands a
    scene exactly as a fresh one does."""
    P, B = lib
    ex = P.StrokeExpander(0)
    code = B.se_debug_scan_timeout(ex.ctx, 5 * 4096 + 17, spin_limit)
    assert code == B.SE_ERR_TIMEOUT, B.STATUS_NAMES.get(code, code)
    sc = W.pr1(n_paths=40)
    got = _outline(ex, sc)
    ex.close()
    fresh = P.StrokeExpander(0)
    ref = _outline(fresh, sc)
    fresh.close()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("spin_limit", [1, 256])
def test_bulk_copy_wait_runs_out(lib, spin_limit):
    """The emit kernels' bulk-copy wait on a barrier phase that nothing completes
    gives up after spin_limit polls with SE_ERR_TIMEOUT; the context then expands
    a scene exactly as a fresh one does."""
    P, B = lib
    ex = P.StrokeExpander(0)
    assert B.se_debug_bulk_timeout(ex.ctx, spin_limit, False) == B.SE_ERR_TIMEOUT
    sc = W.pr1(n_paths=40)
    got = _outline(ex, sc)
    ex.close()
    fresh = P.StrokeExpander(0)
    ref = _outline(fresh, sc)
    fresh.close()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_bulk_copy_lands(lib):
    """With a copy issued and the default bound, the wait succeeds and the bytes arrive intact."""
    P, B = lib
    ex = P.StrokeExpander(0)
    assert B.se_debug_bulk_timeout(ex.ctx, 1 << 22, True) == B.SE_OK
    assert B.se_debug_bulk_timeout(ex.ctx, 0, True) == B.SE_ERR_INVALID_ARG
    ex.close()


def test_timeout_probe_rejects_a_single_tile(lib):
    P, B = lib
    ex = P.StrokeExpander(0)
    assert B.se_debug_scan_timeout(ex.ctx, 4096, 64) == B.SE_ERR_INVALID_ARG
    ex.close()


@pytest.mark.parametrize("arcs", [False, True])
def test_counted_expansion_equals_full_expansion(lib, arcs):
    """se_expand_counted (the count's front half reused: only the primitive scan and
    the emit run) writes exactly what se_expand writes, solid and dashed."""
    P, B = lib
    ex = P.StrokeExpander(0)
    for sc, tol in ((W.pr1(n_paths=80), 0.25), (W.map_like(seed=21, n_paths=400, dash_frac=0.3), 0.1)):
        ds = ex.upload(P.encode(sc))
        a = ex.expand(ds, tol, arcs, reuse_count=True)
        b = ex.expand(ds, tol, arcs, reuse_count=False)
        assert a.n == b.n
        for x, y in ((a.prims, b.prims), (a.tag_offset, b.tag_offset), (a.path_offset, b.path_offset),
                     (a.path_id, b.path_id)):
            assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())
        if arcs:
            assert np.array_equal(a.curvature.cpu().numpy(), b.curvature.cpu().numpy())
    ex.close()


def test_counted_expansion_needs_its_count(lib):
    P, B = lib
    ex = P.StrokeExpander(0)
    s1, s2 = ex.upload(P.encode(W.pr1(n_paths=20))), ex.upload(P.encode(W.hand_cases()))
    params = B.make_params(0.25)
    n1 = ex.count(s1, 0.25)
    bufs = ex.alloc(s1, n1, False, s1.n_tags)
    desc = ex.outline_desc(bufs, n1)
    assert B.se_expand_counted(ex.ctx, s2.desc, params, desc) == B.SE_ERR_INVALID_ARG        # another scene
    assert B.se_expand_counted(ex.ctx, s1.desc, B.make_params(0.5), desc) == B.SE_ERR_INVALID_ARG  # other params
    assert B.se_expand_counted(ex.ctx, s1.desc, params, desc) == B.SE_OK
    assert B.se_expand_counted(ex.ctx, s1.desc, params, desc) == B.SE_ERR_INVALID_ARG        # once per count
    code, n = B.se_sync(ex.ctx)
    assert code == B.SE_OK and n == n1
    ex.count(s2, 0.25)                                     # a count of another scene replaces it
    assert B.se_expand_counted(ex.ctx, s1.desc, params, desc) == B.SE_ERR_INVALID_ARG
    ex.close()
