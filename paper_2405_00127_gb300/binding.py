"""ctypes binding of the C ABI in include/stroke_expand.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device memory
comes from PyTorch tensors; nothing in this module computes any part of the
stroke expansion.  If the compiled library is missing the import fails loudly:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SE_OK, SE_ERR_INVALID_ARG, SE_ERR_INVALID_INPUT, SE_ERR_OOM, SE_ERR_LIMIT, SE_ERR_CAPACITY, SE_ERR_CUDA, \
    SE_ERR_TIMEOUT, SE_ERR_WORKSPACE, SE_ERR_BUDGET = range(10)
STATUS_NAMES = {0: "SE_OK", 1: "SE_ERR_INVALID_ARG", 2: "SE_ERR_INVALID_INPUT", 3: "SE_ERR_OOM",
                4: "SE_ERR_LIMIT", 5: "SE_ERR_CAPACITY", 6: "SE_ERR_CUDA", 7: "SE_ERR_TIMEOUT",
                8: "SE_ERR_WORKSPACE", 9: "SE_ERR_BUDGET"}
SE_OUT_LINES, SE_OUT_ARCS = 0, 1

# Library defaults for the tolerance split (the paper leaves it open).
FIT_FRAC = 0.2
FLAT_FRAC = 1.0

STYLE_DTYPE = np.dtype([("half_width", "<f4"), ("miter_limit", "<f4"), ("join", "u1"), ("cap", "u1"),
                        ("fill", "u1"), ("reserved", "u1"), ("dash_first", "<u4"), ("dash_count", "<u4"),
                        ("dash_offset", "<f4")])
assert STYLE_DTYPE.itemsize == 24

# Every symbol include/stroke_expand.h declares.
EXPORTED = ["se_encode_size", "se_encode", "se_ctx_create", "se_ctx_destroy", "se_ctx_last_error", "se_expand",
            "se_count", "se_sync", "se_total_device", "se_expand_host", "se_profile_enable", "se_profile_read",
            "se_ctx_stats", "se_scan_offsets_noalloc", "se_batch_create", "se_batch_destroy", "se_batch_doc_paths",
            "se_batch_scene", "se_batch_count", "se_batch_expand", "se_batch_capture", "se_batch_launch",
            "se_get_tuning", "se_set_tuning", "se_autotune", "se_server_create", "se_server_destroy",
            "se_server_submit", "se_server_poll", "se_server_release", "se_server_get_stats",
            "se_scene_begin", "se_path_begin", "se_move_to", "se_line_to", "se_cubic_to", "se_close", "se_path_end",
            "se_dash_pattern", "se_scene_from_streams", "se_scene_upload", "se_scene_device", "se_scene_destroy",
            "se_scene_expand", "se_expand_batch", "se_outline_sync", "se_outline_device", "se_outline_copy",
            "se_outline_destroy", "se_server_submit_scene", "se_quad_to", "se_set_transform", "se_coverage",
            "se_set_coord16", "se_server_last_error", "se_debug_scan_timeout", "se_debug_bulk_timeout",
            "se_expand_counted",
            "se_batch_expand_counted"]


class SeError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class se_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_float), ("fit_frac", ctypes.c_float), ("flat_frac", ctypes.c_float),
                ("out_kind", ctypes.c_uint32), ("refine", ctypes.c_uint32)]


class se_scene_dev(ctypes.Structure):
    _fields_ = [("tags", ctypes.c_void_p), ("n_tags", ctypes.c_uint64), ("words", ctypes.c_void_p),
                ("n_words", ctypes.c_uint64), ("styles", ctypes.c_void_p), ("n_styles", ctypes.c_uint32),
                ("n_paths", ctypes.c_uint32), ("dashes", ctypes.c_void_p), ("n_dashes", ctypes.c_uint32),
                ("transforms", ctypes.c_void_p), ("n_transforms", ctypes.c_uint32)]


class se_stats(ctypes.Structure):
    _fields_ = [("n_tags", ctypes.c_uint64), ("n_input_tags", ctypes.c_uint64), ("n_items", ctypes.c_uint64),
                ("n_prims", ctypes.c_uint64),
                ("piece_bytes", ctypes.c_uint32), ("tail_bytes", ctypes.c_uint32),
                ("workspace_bytes", ctypes.c_uint64)]


class se_tuning(ctypes.Structure):
    _fields_ = [("plan_block", ctypes.c_uint32), ("piece_block", ctypes.c_uint32), ("emit_block", ctypes.c_uint32),
                ("emit_blocks_per_sm", ctypes.c_uint32)]


# The caller's device allocator (se_alloc_fn / se_free_fn): bytes, user, stream -> pointer; pointer, user, stream.
SE_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
SE_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class se_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("max_batch_docs", ctypes.c_uint32), ("max_batch_tags", ctypes.c_uint64),
                ("hbm_budget", ctypes.c_uint64), ("alloc_fn", SE_ALLOC_FN), ("free_fn", SE_FREE_FN),
                ("alloc_user", ctypes.c_void_p)]


class se_request_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32), ("batch_docs", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("prims", ctypes.c_void_p), ("curvature", ctypes.c_void_p),
                ("n_prims", ctypes.c_uint64), ("t_submit_ns", ctypes.c_int64), ("t_start_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class se_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("queued", ctypes.c_uint64), ("max_concurrent", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("bytes_in_use", ctypes.c_uint64), ("bytes_peak", ctypes.c_uint64),
                ("hbm_budget", ctypes.c_uint64)]


class se_outline_dev(ctypes.Structure):
    _fields_ = [("prims", ctypes.c_void_p), ("curvature", ctypes.c_void_p), ("path_id", ctypes.c_void_p),
                ("tag_offset", ctypes.c_void_p), ("path_offset", ctypes.c_void_p), ("capacity", ctypes.c_uint64)]


_lib = None


def lib():
    """Load the compiled library (built in-tree by paper_2405_00127_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.SO):
            raise ImportError(f"stroke-expansion library not built: {_build.SO} (run __graft_entry__.build())")
        L = ctypes.CDLL(_build.SO)
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        P = ctypes.POINTER
        L.se_encode_size.argtypes = [vp, u64, vp, u64, vp, u32, vp, vp, P(u64), P(u64)]
        L.se_encode.argtypes = [vp, u64, vp, u64, vp, u32, vp, vp, vp, vp, vp, vp, P(u32), vp, P(u32)]
        L.se_ctx_create.argtypes = [i32, vp, SE_ALLOC_FN, SE_FREE_FN, vp, P(vp)]
        L.se_ctx_destroy.argtypes = [vp]
        L.se_ctx_last_error.argtypes = [vp]
        L.se_ctx_last_error.restype = ctypes.c_char_p
        L.se_expand.argtypes = [vp, P(se_scene_dev), P(se_params), P(se_outline_dev)]
        L.se_expand_counted.argtypes = [vp, P(se_scene_dev), P(se_params), P(se_outline_dev)]
        L.se_count.argtypes = [vp, P(se_scene_dev), P(se_params), P(u64)]
        L.se_sync.argtypes = [vp, P(u64)]
        L.se_total_device.argtypes = [vp, P(vp)]
        L.se_expand_host.argtypes = [vp, vp, u64, vp, u64, vp, u32, u32, vp, u32, vp, u32, P(se_params), vp, vp, u64,
                                     P(u64)]
        L.se_profile_enable.argtypes = [vp, i32]
        L.se_profile_read.argtypes = [vp, P(ctypes.c_float)]
        L.se_ctx_stats.argtypes = [vp, P(se_stats)]
        L.se_scan_offsets_noalloc.argtypes = [vp, u64, vp, vp]
        L.se_debug_scan_timeout.argtypes = [vp, u64, u32]
        L.se_debug_bulk_timeout.argtypes = [vp, u32, ctypes.c_int]
        L.se_batch_create.argtypes = [vp, P(se_scene_dev), u32, P(vp)]
        L.se_batch_destroy.argtypes = [vp]
        L.se_batch_doc_paths.argtypes = [vp, P(u64)]
        L.se_batch_scene.argtypes = [vp, P(se_scene_dev)]
        L.se_batch_count.argtypes = [vp, P(se_params), P(u64)]
        L.se_batch_expand.argtypes = [vp, P(se_params), P(se_outline_dev)]
        L.se_batch_expand_counted.argtypes = [vp, P(se_params), P(se_outline_dev)]
        L.se_batch_capture.argtypes = [vp, P(se_params), P(se_outline_dev)]
        L.se_batch_launch.argtypes = [vp]
        L.se_get_tuning.argtypes = [vp, P(se_tuning)]
        L.se_set_tuning.argtypes = [vp, P(se_tuning)]
        L.se_autotune.argtypes = [vp, P(se_scene_dev), P(se_params), P(se_outline_dev), i32, P(se_tuning)]
        L.se_server_create.argtypes = [i32, P(se_server_config), P(vp)]
        L.se_server_destroy.argtypes = [vp]
        L.se_server_submit.argtypes = [vp, P(se_scene_dev), P(se_params), P(u64)]
        L.se_server_poll.argtypes = [vp, u64, i32, P(se_request_result)]
        L.se_server_release.argtypes = [vp, u64]
        L.se_server_get_stats.argtypes = [vp, P(se_server_stats)]
        L.se_server_last_error.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
        f = ctypes.c_float
        L.se_scene_begin.argtypes = [vp, P(vp)]
        L.se_path_begin.argtypes = [vp, vp]
        L.se_move_to.argtypes = [vp, f, f]
        L.se_line_to.argtypes = [vp, f, f]
        L.se_cubic_to.argtypes = [vp, f, f, f, f, f, f]
        L.se_close.argtypes = [vp]
        L.se_path_end.argtypes = [vp]
        L.se_quad_to.argtypes = [vp, f, f, f, f]
        L.se_set_transform.argtypes = [vp, vp]
        L.se_set_coord16.argtypes = [vp, i32]
        L.se_dash_pattern.argtypes = [vp, vp, u32, P(u32)]
        L.se_scene_from_streams.argtypes = [vp, vp, ctypes.c_size_t, vp, ctypes.c_size_t, vp, ctypes.c_size_t, u32,
                                            vp, ctypes.c_size_t, vp, ctypes.c_size_t, P(vp)]
        L.se_scene_upload.argtypes = [vp]
        L.se_scene_device.argtypes = [vp, P(se_scene_dev)]
        L.se_scene_destroy.argtypes = [vp]
        L.se_scene_expand.argtypes = [vp, f, u32, P(vp)]
        L.se_expand_batch.argtypes = [vp, P(vp), u32, f, u32, P(vp)]
        L.se_outline_sync.argtypes = [vp, P(u64), P(u32)]
        L.se_outline_device.argtypes = [vp, P(vp), P(vp), P(vp)]
        L.se_outline_copy.argtypes = [vp, vp, vp, vp]
        L.se_outline_destroy.argtypes = [vp]
        L.se_server_submit_scene.argtypes = [vp, vp, f, u32, P(u64)]
        L.se_coverage.argtypes = [vp, vp, vp, vp, u64, u32, u32, u32, vp, vp]
        for name in EXPORTED:
            if name != "se_ctx_last_error":
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else ctypes.c_void_p(0)


def _check(code, ctx=None):
    if code not in (SE_OK,):
        msg = se_ctx_last_error(ctx) if ctx else ""
        raise SeError(code, msg)


# --------------------------------------------------------------------------- host encoder

def se_encode_size(verbs, pts, path_verb_off, styles=None, coord16=None):
    """(n_tags, n_words) of the encoding."""
    n_tags, n_words = ctypes.c_uint64(), ctypes.c_uint64()
    c16 = None if coord16 is None else np.ascontiguousarray(coord16, np.uint8)
    code = lib().se_encode_size(_p(verbs), verbs.size, _p(pts), pts.size // 2, _p(path_verb_off),
                                path_verb_off.size - 1, _p(styles), _p(c16), ctypes.byref(n_tags),
                                ctypes.byref(n_words))
    _check(code)
    return n_tags.value, n_words.value


def se_encode(verbs, pts, path_verb_off, styles_in, transforms_in=None, coord16=None):
    """Encode a verb scene; returns (tags u8[n], path data words u32[m], styles STYLE_DTYPE[k],
    transforms f32[j, 6]) -- j = 0 without transforms_in ([n_paths, 6] per-path transforms).
    coord16 (u8 per path, optional) asks for 16-bit coordinates."""
    verbs = np.ascontiguousarray(verbs, np.uint8)
    pts = np.ascontiguousarray(pts, np.float32).reshape(-1)
    voff = np.ascontiguousarray(path_verb_off, np.uint32)
    styles_in = np.ascontiguousarray(styles_in, STYLE_DTYPE)
    n_paths = voff.size - 1
    xf_in = None if transforms_in is None else np.ascontiguousarray(transforms_in, np.float32).reshape(n_paths, 6)
    c16 = None if coord16 is None else np.ascontiguousarray(coord16, np.uint8)
    n_tags, n_words = se_encode_size(verbs, pts, voff, styles_in, c16)
    tags = np.zeros(max(n_tags, 1), np.uint8)
    words = np.zeros(max(n_words, 1), np.uint32)
    styles = np.zeros(max(n_paths, 1), STYLE_DTYPE)
    xf = np.zeros((max(n_paths, 1), 6), np.float32)
    n_styles, n_xf = ctypes.c_uint32(), ctypes.c_uint32()
    code = lib().se_encode(_p(verbs), verbs.size, _p(pts), pts.size // 2, _p(voff), n_paths, _p(styles_in),
                           _p(xf_in), _p(c16), _p(tags), _p(words), _p(styles), ctypes.byref(n_styles), _p(xf),
                           ctypes.byref(n_xf))
    _check(code)
    return tags[:n_tags], words[:n_words], styles[:n_styles.value], xf[:n_xf.value]


# --------------------------------------------------------------------------- device

class Allocator:
    """A device allocator for the library: two Python callables wrapped as the C
    callbacks se_alloc_fn / se_free_fn.  alloc(nbytes, stream) returns a device
    address (int) or None; free(ptr, stream) gives it back.  The object must
    outlive every context (or server) created with it."""

    def __init__(self, alloc, free):
        def _alloc(nbytes, user, stream):
            try:
                p = alloc(int(nbytes), int(stream or 0))
                return int(p) if p else None
            except Exception:
                return None      # the library reports SE_ERR_OOM

        def _free(ptr, user, stream):
            try:
                if ptr:
                    free(int(ptr), int(stream or 0))
            except Exception:
                pass

        self.alloc_fn = SE_ALLOC_FN(_alloc)
        self.free_fn = SE_FREE_FN(_free)


def torch_allocator(device):
    """PyTorch's caching allocator as the library's device allocator: the library's
    workspace and outlines come from the same pool as the tensors around them, in
    stream order on the stream the library names."""
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(max(int(nbytes), 1), device, stream)

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    return Allocator(alloc, free)


def se_ctx_create(device=0, stream=0, allocator=None):
    """allocator: an Allocator, or None for the CUDA stream-ordered allocator."""
    h = ctypes.c_void_p()
    fa = allocator.alloc_fn if allocator is not None else SE_ALLOC_FN()
    ff = allocator.free_fn if allocator is not None else SE_FREE_FN()
    _check(lib().se_ctx_create(int(device), ctypes.c_void_p(stream), fa, ff, None, ctypes.byref(h)))
    return h


def se_ctx_destroy(ctx):
    _check(lib().se_ctx_destroy(ctx))


def se_ctx_last_error(ctx):
    return lib().se_ctx_last_error(ctx).decode()


def se_expand(ctx, scene, params, outline):
    return lib().se_expand(ctx, ctypes.byref(scene), ctypes.byref(params), ctypes.byref(outline))


def se_expand_counted(ctx, scene, params, outline):
    """The expansion after se_count of the same scene and params (status code)."""
    return lib().se_expand_counted(ctx, ctypes.byref(scene), ctypes.byref(params), ctypes.byref(outline))


def se_count(ctx, scene, params):
    n = ctypes.c_uint64()
    code = lib().se_count(ctx, ctypes.byref(scene), ctypes.byref(params), ctypes.byref(n))
    return code, n.value


def se_sync(ctx):
    n = ctypes.c_uint64()
    code = lib().se_sync(ctx, ctypes.byref(n))
    return code, n.value


def se_total_device(ctx):
    p = ctypes.c_void_p()
    _check(lib().se_total_device(ctx, ctypes.byref(p)), ctx)
    return p.value


def se_expand_host(ctx, tags, words, styles, n_paths, dashes, params, host_prims, host_curv, capacity,
                   transforms=None):
    n = ctypes.c_uint64()
    dashes = np.ascontiguousarray(dashes if dashes is not None else np.zeros(0, np.float32), np.float32)
    xf = np.ascontiguousarray(transforms if transforms is not None else np.zeros((0, 6)), np.float32).reshape(-1, 6)
    code = lib().se_expand_host(ctx, _p(tags), tags.size, _p(words), words.size, _p(styles), styles.size,
                                int(n_paths), _p(dashes), dashes.size, _p(xf), xf.shape[0], ctypes.byref(params),
                                _p(host_prims),
                                _p(host_curv) if host_curv is not None else ctypes.c_void_p(0), int(capacity),
                                ctypes.byref(n))
    return code, n.value


def se_profile_enable(ctx, enable=True):
    _check(lib().se_profile_enable(ctx, int(bool(enable))), ctx)


def se_profile_read(ctx):
    ms = (ctypes.c_float * 6)()
    _check(lib().se_profile_read(ctx, ms), ctx)
    return list(ms)


def se_ctx_stats(ctx):
    st = se_stats()
    _check(lib().se_ctx_stats(ctx, ctypes.byref(st)), ctx)
    return {k: getattr(st, k) for k, _ in se_stats._fields_}


def se_scan_offsets_noalloc(d_counts, n, d_offsets, stream=0):
    """Device pointers in, device pointer out; returns the status code."""
    return lib().se_scan_offsets_noalloc(ctypes.c_void_p(d_counts), int(n), ctypes.c_void_p(d_offsets),
                                         ctypes.c_void_p(stream))


def se_debug_scan_timeout(ctx, n, spin_limit):
    """Status of a look-back scan whose first tile never publishes (test hook)."""
    return lib().se_debug_scan_timeout(ctx, int(n), int(spin_limit))


def se_debug_bulk_timeout(ctx, spin_limit, copy):
    """Status of a bulk-copy wait on a barrier phase (copy=False: nothing completes it; test hook)."""
    return lib().se_debug_bulk_timeout(ctx, int(spin_limit), 1 if copy else 0)


def make_params(tol, arcs=False, fit_frac=FIT_FRAC, flat_frac=FLAT_FRAC, refine=False):
    return se_params(float(tol), float(fit_frac), float(flat_frac), SE_OUT_ARCS if arcs else SE_OUT_LINES,
                     int(bool(refine)))


# --------------------------------------------------------------------------- batches and tuning

def se_batch_create(ctx, docs):
    """docs: a sequence of se_scene_dev (device pointers).  Returns the batch handle."""
    arr = (se_scene_dev * max(len(docs), 1))(*docs)
    out = ctypes.c_void_p()
    _check(lib().se_batch_create(ctx, arr, len(docs), ctypes.byref(out)), ctx)
    return out


def se_batch_destroy(batch):
    _check(lib().se_batch_destroy(batch))


def se_batch_doc_paths(batch, n_docs):
    out = np.zeros(n_docs + 1, np.uint64)
    _check(lib().se_batch_doc_paths(batch, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
    return out


def se_batch_scene(batch):
    s = se_scene_dev()
    _check(lib().se_batch_scene(batch, ctypes.byref(s)))
    return s


def se_batch_count(ctx, batch, params):
    n = ctypes.c_uint64()
    code = lib().se_batch_count(batch, ctypes.byref(params), ctypes.byref(n))
    return code, n.value


def se_batch_expand(ctx, batch, params, out):
    _check(lib().se_batch_expand(batch, ctypes.byref(params), ctypes.byref(out)), ctx)


def se_batch_expand_counted(ctx, batch, params, out):
    _check(lib().se_batch_expand_counted(batch, ctypes.byref(params), ctypes.byref(out)), ctx)


def se_batch_capture(ctx, batch, params, out):
    _check(lib().se_batch_capture(batch, ctypes.byref(params), ctypes.byref(out)), ctx)


def se_batch_launch(ctx, batch):
    _check(lib().se_batch_launch(batch), ctx)


def se_get_tuning(ctx):
    t = se_tuning()
    _check(lib().se_get_tuning(ctx, ctypes.byref(t)), ctx)
    return {k: getattr(t, k) for k, _ in se_tuning._fields_}


def se_set_tuning(ctx, **kw):
    t = se_tuning(**{**se_get_tuning(ctx), **kw})
    _check(lib().se_set_tuning(ctx, ctypes.byref(t)), ctx)


def se_autotune(ctx, scene, params, out, reps=3):
    t = se_tuning()
    _check(lib().se_autotune(ctx, ctypes.byref(scene), ctypes.byref(params), ctypes.byref(out), int(reps),
                             ctypes.byref(t)), ctx)
    return {k: getattr(t, k) for k, _ in se_tuning._fields_}


# --------------------------------------------------------------------------- serving

def se_server_create(device, slots, max_batch_docs, max_batch_tags, hbm_budget, allocator=None):
    """allocator: an Allocator for every slot's context and the outlines, or None
    for the CUDA stream-ordered allocator."""
    fa = allocator.alloc_fn if allocator is not None else SE_ALLOC_FN()
    ff = allocator.free_fn if allocator is not None else SE_FREE_FN()
    cfg = se_server_config(slots, max_batch_docs, max_batch_tags, hbm_budget, fa, ff, None)
    out = ctypes.c_void_p()
    _check(lib().se_server_create(int(device), ctypes.byref(cfg), ctypes.byref(out)))
    return out


def se_server_destroy(server):
    _check(lib().se_server_destroy(server))


def se_server_submit(server, scene, params):
    rid = ctypes.c_uint64()
    _check(lib().se_server_submit(server, ctypes.byref(scene), ctypes.byref(params), ctypes.byref(rid)))
    return rid.value


def se_server_poll(server, req_id, wait=False):
    r = se_request_result()
    _check(lib().se_server_poll(server, int(req_id), int(bool(wait)), ctypes.byref(r)))
    return {k: getattr(r, k) for k, _ in se_request_result._fields_}


def se_server_release(server, req_id):
    _check(lib().se_server_release(server, int(req_id)))


def se_server_last_error(server) -> str:
    """The cause of the server's most recent failed batch ("" when none failed)."""
    buf = ctypes.create_string_buffer(1024)
    _check(lib().se_server_last_error(server, buf, len(buf)))
    return buf.value.decode()


def se_server_get_stats(server):
    st = se_server_stats()
    _check(lib().se_server_get_stats(server, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in se_server_stats._fields_}


# --------------------------------------------------------------------------- library-owned scenes and outlines

def scene_from_verbs(ctx, scene):
    """Build a library-owned scene with the path builder (se_set_transform / se_path_begin /
    se_move_to / se_line_to / se_quad_to / se_cubic_to / se_close / se_path_end) from a
    workloads.Scene."""
    L = lib()
    h = ctypes.c_void_p()
    _check(L.se_scene_begin(ctx, ctypes.byref(h)), ctx)
    pts = np.asarray(scene.pts, np.float64)
    k = 0
    firsts = {}
    xf = getattr(scene, "transform", None)
    c16 = getattr(scene, "coord16", None)
    for p in range(scene.n_paths):
        if xf is not None:
            m = np.ascontiguousarray(xf[p], np.float32)
            _check(L.se_set_transform(h, _p(m)), ctx)
        if c16 is not None:
            _check(L.se_set_coord16(h, int(bool(c16[p]))), ctx)
        st = np.zeros(1, STYLE_DTYPE)
        st["half_width"] = scene.half_width[p]
        st["miter_limit"] = scene.miter_limit[p]
        st["join"] = scene.join[p]
        st["cap"] = scene.cap[p]
        st["fill"] = scene.fill[p] if getattr(scene, "fill", None) is not None else 0
        f, c = int(scene.dash_first[p]), int(scene.dash_count[p])
        if c:
            key = (f, c)
            if key not in firsts:
                lens = np.ascontiguousarray(scene.dash_len[f:f + c], np.float32)
                first = ctypes.c_uint32()
                _check(L.se_dash_pattern(h, _p(lens), c, ctypes.byref(first)), ctx)
                firsts[key] = first.value
            st["dash_first"] = firsts[key]
            st["dash_count"] = c
            st["dash_offset"] = scene.dash_offset[p]
        _check(L.se_path_begin(h, _p(st)), ctx)
        for vb in scene.verbs[scene.path_verb_off[p]:scene.path_verb_off[p + 1]]:
            if vb == SE_VERB_MOVE:
                _check(L.se_move_to(h, float(pts[k, 0]), float(pts[k, 1])), ctx); k += 1
            elif vb == SE_VERB_LINE:
                _check(L.se_line_to(h, float(pts[k, 0]), float(pts[k, 1])), ctx); k += 1
            elif vb == SE_VERB_CUBIC:
                q = pts[k:k + 3].reshape(-1)
                _check(L.se_cubic_to(h, *[float(v) for v in q]), ctx); k += 3
            elif vb == SE_VERB_QUAD:
                q = pts[k:k + 2].reshape(-1)
                _check(L.se_quad_to(h, *[float(v) for v in q]), ctx); k += 2
            else:
                _check(L.se_close(h), ctx)
        _check(L.se_path_end(h), ctx)
    return h


SE_VERB_MOVE, SE_VERB_LINE, SE_VERB_CUBIC, SE_VERB_CLOSE, SE_VERB_QUAD = 0, 1, 2, 3, 4


def se_scene_expand(ctx, scene, tol, arcs=False):
    out = ctypes.c_void_p()
    _check(lib().se_scene_expand(scene, float(tol), int(bool(arcs)), ctypes.byref(out)), ctx)
    return out


def se_outline_sync(outline):
    n, npaths = ctypes.c_uint64(), ctypes.c_uint32()
    code = lib().se_outline_sync(outline, ctypes.byref(n), ctypes.byref(npaths))
    return code, n.value, npaths.value


def se_outline_copy(outline, n_prims, n_paths, arcs=False):
    prims = np.zeros((max(n_prims, 1), 4), np.float32)
    curv = np.zeros(max(n_prims, 1), np.float32) if arcs else None
    poff = np.zeros(n_paths + 1, np.uint64)
    _check(lib().se_outline_copy(outline, _p(prims), _p(curv), _p(poff)))
    return prims[:n_prims], (curv[:n_prims] if arcs else None), poff


def se_expand_batch(ctx, scenes, tol, arcs=False):
    arr = (ctypes.c_void_p * max(len(scenes), 1))(*scenes)
    outs = (ctypes.c_void_p * max(len(scenes), 1))()
    _check(lib().se_expand_batch(ctx, arr, len(scenes), float(tol), int(bool(arcs)), outs), ctx)
    return [ctypes.c_void_p(outs[i]) for i in range(len(scenes))]


def se_scene_begin(ctx):
    h = ctypes.c_void_p()
    _check(lib().se_scene_begin(ctx, ctypes.byref(h)), ctx)
    return h


def se_path_begin(scene, style):
    st = np.ascontiguousarray(style, STYLE_DTYPE).reshape(1)
    _check(lib().se_path_begin(scene, _p(st)))


def se_move_to(scene, x, y):
    _check(lib().se_move_to(scene, float(x), float(y)))


def se_line_to(scene, x, y):
    _check(lib().se_line_to(scene, float(x), float(y)))


def se_cubic_to(scene, x1, y1, x2, y2, x3, y3):
    _check(lib().se_cubic_to(scene, float(x1), float(y1), float(x2), float(y2), float(x3), float(y3)))


def se_set_coord16(scene, enable=True):
    _check(lib().se_set_coord16(scene, int(bool(enable))))


def se_quad_to(scene, x1, y1, x2, y2):
    _check(lib().se_quad_to(scene, float(x1), float(y1), float(x2), float(y2)))


def se_set_transform(scene, m=None):
    mm = None if m is None else np.ascontiguousarray(m, np.float32).reshape(6)
    _check(lib().se_set_transform(scene, _p(mm)))


def se_close(scene):
    _check(lib().se_close(scene))


def se_path_end(scene):
    _check(lib().se_path_end(scene))


def se_dash_pattern(scene, lens):
    lens = np.ascontiguousarray(lens, np.float32)
    first = ctypes.c_uint32()
    _check(lib().se_dash_pattern(scene, _p(lens), lens.size, ctypes.byref(first)))
    return first.value


def se_scene_from_streams(ctx, tags, words, styles, n_paths, dashes=None, transforms=None):
    tags = np.ascontiguousarray(tags, np.uint8)
    words = np.ascontiguousarray(words, np.uint32).reshape(-1)
    styles = np.ascontiguousarray(styles, STYLE_DTYPE)
    dashes = np.ascontiguousarray(dashes if dashes is not None else np.zeros(0), np.float32)
    xf = np.ascontiguousarray(transforms if transforms is not None else np.zeros((0, 6)), np.float32).reshape(-1, 6)
    h = ctypes.c_void_p()
    _check(lib().se_scene_from_streams(ctx, _p(tags), tags.size, _p(words), words.size, _p(styles), styles.size,
                                       int(n_paths), _p(dashes), dashes.size, _p(xf), xf.shape[0], ctypes.byref(h)), ctx)
    return h


def se_scene_upload(scene):
    _check(lib().se_scene_upload(scene))


def se_scene_device(scene):
    d = se_scene_dev()
    _check(lib().se_scene_device(scene, ctypes.byref(d)))
    return d


def se_scene_destroy(scene):
    _check(lib().se_scene_destroy(scene))


def se_outline_device(outline):
    p, c, o = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().se_outline_device(outline, ctypes.byref(p), ctypes.byref(c), ctypes.byref(o)))
    return p.value, c.value, o.value


def se_outline_destroy(outline):
    _check(lib().se_outline_destroy(outline))


def se_server_submit_scene(server, scene, tol, arcs=False):
    rid = ctypes.c_uint64()
    _check(lib().se_server_submit_scene(server, scene, float(tol), int(bool(arcs)), ctypes.byref(rid)))
    return rid.value


def se_coverage(ctx, prims_ptr, curv_ptr, path_id_ptr, n_prims, n_paths, width, height, count_ptr, area_ptr=0):
    """Nonzero coverage of an outline on a width x height grid (device pointers)."""
    _check(lib().se_coverage(ctx, ctypes.c_void_p(prims_ptr), ctypes.c_void_p(curv_ptr or 0),
                             ctypes.c_void_p(path_id_ptr), int(n_prims), int(n_paths), int(width), int(height),
                             ctypes.c_void_p(count_ptr), ctypes.c_void_p(area_ptr or 0)), ctx)
