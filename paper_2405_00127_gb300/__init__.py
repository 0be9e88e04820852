"""GB300-native stroke expansion (Levien & Uguray, "GPU-friendly Stroke Expansion").

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/stroke_expand.h``); this package only marshals arguments to it and
uses PyTorch for device memory and streams.

    enc = encode(scene)                       # host encoder (Section 8.2)
    ex = StrokeExpander(device=0)
    ds = ex.upload(enc)                       # device-resident scene
    out = ex.expand(ds, tol=0.25)             # scan -> count -> scan -> write
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import binding as B
from .binding import FIT_FRAC, FLAT_FRAC, STYLE_DTYPE, SeError, make_params

__all__ = ["encode", "Encoded", "StrokeExpander", "DeviceScene", "Outline", "Batch", "Server", "SeError", "make_params",
           "FIT_FRAC", "FLAT_FRAC", "STYLE_DTYPE", "styles_of"]


def styles_of(scene) -> np.ndarray:
    st = np.zeros(scene.n_paths, STYLE_DTYPE)
    st["half_width"] = scene.half_width
    st["miter_limit"] = scene.miter_limit
    st["join"] = scene.join
    st["cap"] = scene.cap
    st["dash_first"] = scene.dash_first
    st["dash_count"] = scene.dash_count
    st["dash_offset"] = scene.dash_offset
    fill = getattr(scene, "fill", None)
    if fill is not None:
        st["fill"] = fill
    return st


@dataclasses.dataclass
class Encoded:
    tags: np.ndarray     # uint8 [n_tags]
    points: np.ndarray   # uint32 [n_words]: the path data stream (32- or 16-bit points per tag)
    styles: np.ndarray   # STYLE_DTYPE [n_styles]
    n_paths: int
    dashes: np.ndarray   # float32 [n_dashes]
    transforms: np.ndarray = None  # float32 [n_transforms, 6] (None or empty: untransformed)


def encode(scene) -> Encoded:
    """Host encoding of a verb scene (a ``workloads.Scene``-like object)."""
    xf = getattr(scene, "transform", None)
    c16 = getattr(scene, "coord16", None)
    tags, points, styles, xforms = B.se_encode(scene.verbs, scene.pts, scene.path_verb_off, styles_of(scene), xf, c16)
    return Encoded(tags, points, styles, int(scene.n_paths), np.asarray(scene.dash_len, np.float32),
                   xforms if xforms.size else None)


def _allocator(kind, device):
    if kind == "torch":
        return B.torch_allocator(device)
    if kind in (None, "cuda"):
        return None
    return kind


@dataclasses.dataclass
class DeviceScene:
    tags: object
    points: object
    styles: object
    dashes: object
    desc: B.se_scene_dev
    n_tags: int
    n_paths: int
    transforms: object = None

    @property
    def dashes_present(self) -> bool:
        return self.dashes is not None


@dataclasses.dataclass
class Outline:
    prims: object        # torch float32 [n, 4]: x0 y0 x1 y1
    curvature: object    # torch float32 [n] (arcs) or None
    path_id: object      # torch int32 [n]
    tag_offset: object   # torch int64 [n_tags + 1] (tags of the dashed rewrite for a dashed scene)
    path_offset: object  # torch int64 [n_paths + 1]
    n: int
    status: int


class StrokeExpander:
    """A library context bound to one CUDA device and stream.

    allocator: "torch" (default) hands the library PyTorch's caching allocator, so
    its workspace comes from the same pool as the tensors; "cuda" keeps the CUDA
    stream-ordered allocator; or a binding.Allocator."""

    def __init__(self, device: int = 0, stream=None, allocator="torch"):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.allocator = _allocator(allocator, device)   # kept alive as long as the context
        self.ctx = B.se_ctx_create(device, self.stream.cuda_stream, self.allocator)

    def close(self):
        if self.ctx:
            B.se_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload(self, enc: Encoded) -> DeviceScene:
        t = self.torch
        dev = self.device
        tags = t.from_numpy(np.ascontiguousarray(enc.tags)).to(dev)
        points = t.from_numpy(np.ascontiguousarray(enc.points, np.uint32).view(np.int32)).to(dev)
        styles = t.from_numpy(np.ascontiguousarray(enc.styles).view(np.uint8)).to(dev)
        dashes = t.from_numpy(np.ascontiguousarray(enc.dashes, np.float32)).to(dev) if enc.dashes.size else None
        has_xf = enc.transforms is not None and enc.transforms.size > 0
        xforms = t.from_numpy(np.ascontiguousarray(enc.transforms, np.float32)).to(dev) if has_xf else None
        desc = B.se_scene_dev(tags.data_ptr(), int(enc.tags.size), points.data_ptr(), int(enc.points.size),
                              styles.data_ptr(), int(enc.styles.size), int(enc.n_paths),
                              dashes.data_ptr() if dashes is not None else 0,
                              int(enc.dashes.size), xforms.data_ptr() if has_xf else 0,
                              int(enc.transforms.shape[0]) if has_xf else 0)
        return DeviceScene(tags, points, styles, dashes, desc, int(enc.tags.size), int(enc.n_paths), xforms)

    def count(self, ds: DeviceScene, tol: float, arcs: bool = False, **kw) -> int:
        code, n = B.se_count(self.ctx, ds.desc, make_params(tol, arcs, **kw))
        if code not in (B.SE_OK, B.SE_ERR_LIMIT):
            raise SeError(code, B.se_ctx_last_error(self.ctx))
        return n

    def expanded_tags(self, ds: DeviceScene) -> int:
        """Tags the last count/expansion ran over: the scene's own, or those of
        its dashed rewrite (call after ``count``)."""
        if not ds.dashes_present:
            return ds.n_tags
        return int(B.se_ctx_stats(self.ctx)["n_tags"])

    def alloc(self, ds: DeviceScene, capacity: int, arcs: bool, n_tags: int | None = None):
        t = self.torch
        dev = self.device
        prims = t.empty((max(capacity, 1), 4), dtype=t.float32, device=dev)
        curv = t.empty(max(capacity, 1), dtype=t.float32, device=dev) if arcs else None
        pid = t.empty(max(capacity, 1), dtype=t.int32, device=dev)
        toff = t.empty((ds.n_tags if n_tags is None else n_tags) + 1, dtype=t.int64, device=dev)
        poff = t.empty(ds.n_paths + 1, dtype=t.int64, device=dev)
        return prims, curv, pid, toff, poff

    def outline_desc(self, bufs, capacity):
        prims, curv, pid, toff, poff = bufs
        return B.se_outline_dev(prims.data_ptr(), curv.data_ptr() if curv is not None else 0, pid.data_ptr(),
                                toff.data_ptr(), poff.data_ptr(), int(capacity))

    def expand_async(self, ds: DeviceScene, params, desc) -> None:
        """Enqueue scan -> count -> scan -> write on the stream (no host sync)."""
        code = B.se_expand(self.ctx, ds.desc, params, desc)
        if code != B.SE_OK:
            raise SeError(code, B.se_ctx_last_error(self.ctx))

    def expand_counted(self, ds: DeviceScene, params, desc) -> None:
        """Enqueue the primitive scan and the emit after ``count`` of the same scene
        and parameters (se_expand_counted: the count's front half is reused)."""
        code = B.se_expand_counted(self.ctx, ds.desc, params, desc)
        if code != B.SE_OK:
            raise SeError(code, B.se_ctx_last_error(self.ctx))

    def expand(self, ds: DeviceScene, tol: float, arcs: bool = False, capacity: int | None = None,
               reuse_count: bool = True, **kw) -> Outline:
        """Count (unless a capacity is given), allocate and expand.  After its own
        count the expansion reuses the count's front half (reuse_count)."""
        params = make_params(tol, arcs, **kw)
        counted = capacity is None
        if counted:
            capacity = self.count(ds, tol, arcs, **kw)
        bufs = self.alloc(ds, capacity, arcs, self.expanded_tags(ds))
        if counted and reuse_count:
            self.expand_counted(ds, params, self.outline_desc(bufs, capacity))
        else:
            self.expand_async(ds, params, self.outline_desc(bufs, capacity))
        code, n = B.se_sync(self.ctx)
        if code not in (B.SE_OK, B.SE_ERR_LIMIT):
            raise SeError(code, B.se_ctx_last_error(self.ctx))
        prims, curv, pid, toff, poff = bufs
        return Outline(prims[:n], curv[:n] if curv is not None else None, pid[:n], toff, poff, n, code)


def coverage(ex: "StrokeExpander", out: Outline, n_paths: int, width: int, height: int, arcs: bool = False,
             path_area: bool = True):
    """Nonzero coverage of an outline on a width x height pixel grid (se_coverage):
    returns (count int32 [height, width] of paths covering each pixel, per-path
    covered pixels int64 [n_paths] or None)."""
    t = ex.torch
    dev = ex.device
    cnt = t.zeros((height, width), dtype=t.int32, device=dev)
    area = t.zeros(max(n_paths, 1), dtype=t.int64, device=dev) if path_area else None
    curv = out.curvature.data_ptr() if (arcs and out.curvature is not None and out.n) else 0
    B.se_coverage(ex.ctx, out.prims.data_ptr() if out.n else 0, curv, out.path_id.data_ptr() if out.n else 0,
                  out.n, n_paths, width, height, cnt.data_ptr(), area.data_ptr() if area is not None else 0)
    return cnt, (area[:n_paths] if area is not None else None)


class Batch:
    """Many device scenes expanded as one (C ABI se_batch_*): one launch
    sequence, optionally replayed from a captured CUDA graph.  Document d's
    primitives are ``out.prims[path_offset[first[d]]:path_offset[first[d+1]]]``."""

    def __init__(self, ex: StrokeExpander, docs):
        self.ex = ex
        self.docs = list(docs)          # keeps the documents' device memory alive
        self.handle = B.se_batch_create(ex.ctx, [d.desc for d in self.docs])
        self.path_first = B.se_batch_doc_paths(self.handle, len(self.docs)).astype(np.int64)
        self.bufs = None
        self.capacity = 0

    @property
    def has_dashes(self) -> bool:
        return any(d.dashes_present for d in self.docs)

    def count(self, tol: float, arcs: bool = False, **kw) -> int:
        code, n = B.se_batch_count(self.ex.ctx, self.handle, make_params(tol, arcs, **kw))
        if code not in (B.SE_OK, B.SE_ERR_LIMIT):
            raise SeError(code, B.se_ctx_last_error(self.ex.ctx))
        return n

    def n_tags(self) -> int:
        if self.has_dashes:
            return int(B.se_ctx_stats(self.ex.ctx)["n_tags"])
        return int(B.se_batch_scene(self.handle).n_tags)

    def prepare(self, tol: float, arcs: bool = False, **kw):
        """Count the batch and allocate its outline; returns the outline descriptor."""
        self.params = make_params(tol, arcs, **kw)
        self.capacity = self.count(tol, arcs, **kw)
        scene = B.se_batch_scene(self.handle)
        n_tags = self.n_tags()
        t = self.ex.torch
        dev = self.ex.device
        cap = max(self.capacity, 1)
        prims = t.empty((cap, 4), dtype=t.float32, device=dev)
        curv = t.empty(cap, dtype=t.float32, device=dev) if arcs else None
        pid = t.empty(cap, dtype=t.int32, device=dev)
        toff = t.empty(n_tags + 1, dtype=t.int64, device=dev)
        poff = t.empty(int(scene.n_paths) + 1, dtype=t.int64, device=dev)
        self.bufs = (prims, curv, pid, toff, poff)
        self.desc = B.se_outline_dev(prims.data_ptr(), curv.data_ptr() if curv is not None else 0, pid.data_ptr(),
                                     toff.data_ptr(), poff.data_ptr(), int(self.capacity))
        return self.desc

    def expand_async(self):
        B.se_batch_expand(self.ex.ctx, self.handle, self.params, self.desc)

    def capture(self):
        B.se_batch_capture(self.ex.ctx, self.handle, self.params, self.desc)

    def launch(self):
        B.se_batch_launch(self.ex.ctx, self.handle)

    def result(self) -> Outline:
        code, n = B.se_sync(self.ex.ctx)
        if code not in (B.SE_OK, B.SE_ERR_LIMIT):
            raise SeError(code, B.se_ctx_last_error(self.ex.ctx))
        prims, curv, pid, toff, poff = self.bufs
        return Outline(prims[:n], curv[:n] if curv is not None else None, pid[:n], toff, poff, n, code)

    def doc_range(self, out: Outline, d: int):
        po = out.path_offset
        return int(po[int(self.path_first[d])]), int(po[int(self.path_first[d + 1])])

    def close(self):
        if self.handle:
            B.se_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """A view of device memory the library owns, for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class Server:
    """The library's serving loop (C ABI se_server_*): requests queue up, slots
    take them in continuous batches under an HBM budget, results stay on the
    device until released."""

    def __init__(self, device: int = 0, slots: int = 4, max_batch_docs: int = 64, max_batch_tags: int = 1 << 22,
                 hbm_budget: int = 100 << 30, allocator="torch"):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.allocator = _allocator(allocator, device)   # kept alive as long as the server
        self.handle = B.se_server_create(device, slots, max_batch_docs, max_batch_tags, hbm_budget, self.allocator)
        self._docs = {}

    def submit(self, ds: DeviceScene, tol: float, arcs: bool = False, **kw) -> int:
        rid = B.se_server_submit(self.handle, ds.desc, make_params(tol, arcs, **kw))
        self._docs[rid] = ds          # the document must outlive its request
        return rid

    def poll(self, rid: int, wait: bool = False) -> dict:
        return B.se_server_poll(self.handle, rid, wait)

    def prims(self, res: dict):
        """The request's primitives as a torch view (valid until released)."""
        n = int(res["n_prims"])
        if n == 0:
            return self.torch.zeros((0, 4), dtype=self.torch.float32, device=self.device)
        return self.torch.as_tensor(_DeviceArray(res["prims"], (n, 4), "<f4"), device=self.device)

    def curvature(self, res: dict):
        n = int(res["n_prims"])
        if not res["curvature"] or n == 0:
            return None
        return self.torch.as_tensor(_DeviceArray(res["curvature"], (n,), "<f4"), device=self.device)

    def release(self, rid: int) -> None:
        B.se_server_release(self.handle, rid)
        self._docs.pop(rid, None)

    def stats(self) -> dict:
        return B.se_server_get_stats(self.handle)

    def last_error(self) -> str:
        """The cause of the most recent failed batch ("" when none failed)."""
        return B.se_server_last_error(self.handle)

    def close(self):
        if self.handle:
            B.se_server_destroy(self.handle)
            self.handle = None
            self._docs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
