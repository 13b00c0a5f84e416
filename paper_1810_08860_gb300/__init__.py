"""Python binding of liblf.so, the GB300 disk-blended light field renderer.

Argument marshalling only: every step of the rendering runs in the library's
CUDA kernels, reached through the C ABI of include/lf.h.  PyTorch provides the
device memory of the outputs and the CUDA streams.  There is no CPU fallback:
if the compiled library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblf.so")

LF_OK = 0
STATUS = {0: "LF_OK", 1: "LF_ERR_INVALID_ARG", 2: "LF_ERR_CUDA", 3: "LF_ERR_OOM", 4: "LF_ERR_STATE",
          5: "LF_ERR_TIMEOUT", 6: "LF_ERR_UNSUPPORTED", 7: "LF_ERR_CAPACITY"}
TEX_FORMATS = {"f32": 0, "u8": 1, "bf16": 2, "fp8": 3}
MESH_FORMATS = {"f32": 0, "f16": 1}


class LFError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), message))
        self.status = status


class Pose(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


class Intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class Config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("max_eyes", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("tri_capacity", ctypes.c_int64), ("z_near", ctypes.c_float),
                ("pad1", ctypes.c_int32), ("wait_limit", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("n_eyes", ctypes.c_int32), ("n_views", ctypes.c_int32), ("active_views", ctypes.c_int32 * 2),
                ("triangles", ctypes.c_int64), ("tiles", ctypes.c_int64), ("error_word", ctypes.c_uint32),
                ("ms_view_setup", ctypes.c_float), ("ms_tri_setup", ctypes.c_float), ("ms_raster", ctypes.c_float)]


class Tuning(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("n_tried", ctypes.c_int32), ("ms", ctypes.c_float), ("tried_tile_w", ctypes.c_int32 * 16),
                ("tried_tile_h", ctypes.c_int32 * 16), ("tried_blocks", ctypes.c_int32 * 16),
                ("tried_ms", ctypes.c_float * 16)]


class FragRecord(ctypes.Structure):
    _fields_ = [("view", ctypes.c_int32), ("n_cover", ctypes.c_int32), ("winner", ctypes.c_int32),
                ("min_id", ctypes.c_int32), ("max_id", ctypes.c_int32), ("id_hash", ctypes.c_uint32)]


FRAG_RECORD_DTYPE = np.dtype([("view", np.int32), ("n_cover", np.int32), ("winner", np.int32),
                              ("min_id", np.int32), ("max_id", np.int32), ("id_hash", np.uint32)])

# Every symbol include/lf.h declares.
EXPORTS = ["lf_config_default", "lf_create", "lf_destroy", "lf_load_views", "lf_build_view_meshes", "lf_render",
           "lf_render_batch", "lf_render_inspect", "lf_render_static", "lf_tune_batch", "lf_get_stats",
           "lf_status_string", "lf_last_error", "lf_load_refiner", "lf_refine_set_kernel", "lf_get_refiner",
           "lf_refine", "lf_refine_gradients", "lf_refine_train_step", "lf_render_refined", "lf_render_host",
           "lf_host_wait", "lf_prefilter", "lf_prefilter_cameras", "lf_set_disk_ovals",
           "lf_cache_create", "lf_cache_destroy", "lf_cache_frame", "lf_cache_pages", "lf_set_wait_limit",
           "lf_set_timing",
           "lf_set_levels", "lf_upload_pages", "lf_levels_wanted"]
HOST_FRAMES_IN_FLIGHT = 3
HOST_FORMS = {"plain": 0, "refined": 1, "batch": 2}

REFINE_N_PARAMS = 11011
REFINE_SHAPES = [("W1", (32, 3, 3, 3)), ("b1", (32,)), ("W2", (32, 32, 3, 3)), ("b2", (32,)),
                 ("W3", (3, 32, 3, 3)), ("b3", (3,))]
REFINE_KERNELS = {"fused": 0, "layers": 1}


def init_refiner_params(seed: int, out_scale: float = 0.1) -> np.ndarray:
    """Initial refinement weights: He-normal hidden layers, a last layer scaled
    by out_scale (so y = x + f(x) starts close to x), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in REFINE_SHAPES:
        if name.startswith("b"):
            parts.append(np.zeros(shape))
        else:
            fan_in = shape[1] * 9
            std = np.sqrt(2.0 / fan_in) * (out_scale if name == "W3" else 1.0)
            parts.append(rng.normal(0.0, std, shape))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)

def prefilter_samples(n: int, seed: int) -> np.ndarray:
    """n stratified prefilter samples (a, b, ds, dt), float32 (lf_prefilter).
    a is stratified over [0, 1) (n strata), b uniform; (ds, dt) lie on a
    jittered k x k grid over [-2, 2)^2 (k = floor(sqrt(n)); the rest uniform),
    so the Lanczos-2 weights of the set sum well above zero."""
    rng = np.random.default_rng(seed)
    s = np.empty((n, 4))
    s[:, 0] = rng.permutation((np.arange(n) + rng.uniform(0.0, 1.0, n)) / n)
    s[:, 1] = rng.uniform(0.0, 1.0, n)
    k = int(np.sqrt(n))
    cells = np.stack(np.meshgrid(np.arange(k), np.arange(k), indexing="ij"), -1).reshape(-1, 2)
    s[:k * k, 2:] = -2.0 + 4.0 * (cells + rng.uniform(0.0, 1.0, (k * k, 2))) / k
    s[k * k:, 2:] = rng.uniform(-2.0, 2.0, (n - k * k, 2))
    s[:, 2:] = np.clip(s[:, 2:], -2.0, 2.0)
    return s.astype(np.float32)


_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblf.so and declare its signatures.  Raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("liblf.so is not built (run __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.lf_config_default.argtypes = [ctypes.POINTER(Config)]
    lib.lf_config_default.restype = None
    lib.lf_create.argtypes = [i32, ctypes.POINTER(Config), ctypes.POINTER(vp)]
    lib.lf_create.restype = ctypes.c_int
    lib.lf_destroy.argtypes = [vp]
    lib.lf_destroy.restype = None
    lib.lf_load_views.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_int]
    lib.lf_load_views.restype = ctypes.c_int
    lib.lf_build_view_meshes.argtypes = [vp, i32, vp, ctypes.c_int]
    lib.lf_build_view_meshes.restype = ctypes.c_int
    for name in ("lf_render", "lf_render_batch"):
        f = getattr(lib, name)
        f.argtypes = [vp, i32, vp, vp, vp, vp]
        f.restype = ctypes.c_int
    lib.lf_tune_batch.argtypes = [vp, i32, vp, vp, vp, i32, vp, ctypes.POINTER(Tuning)]
    lib.lf_tune_batch.restype = ctypes.c_int
    lib.lf_render_static.argtypes = [vp, vp, vp, vp, vp]
    lib.lf_render_static.restype = ctypes.c_int
    lib.lf_render_inspect.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, vp, vp]
    lib.lf_render_inspect.restype = ctypes.c_int
    lib.lf_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.lf_get_stats.restype = ctypes.c_int
    lib.lf_load_refiner.argtypes = [vp, vp]
    lib.lf_load_refiner.restype = ctypes.c_int
    lib.lf_refine_set_kernel.argtypes = [vp, ctypes.c_int]
    lib.lf_refine_set_kernel.restype = ctypes.c_int
    lib.lf_get_refiner.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.lf_get_refiner.restype = ctypes.c_int
    lib.lf_refine.argtypes = [vp, i32, i32, i32, vp, vp, vp]
    lib.lf_refine.restype = ctypes.c_int
    lib.lf_refine_gradients.argtypes = [vp, i32, i32, i32, vp, vp, vp]
    lib.lf_refine_gradients.restype = ctypes.c_int
    lib.lf_refine_train_step.argtypes = [vp, i32, i32, i32, vp, vp, ctypes.c_float, vp]
    lib.lf_refine_train_step.restype = ctypes.c_int
    lib.lf_render_refined.argtypes = [vp, i32, vp, vp, vp, vp]
    lib.lf_render_refined.restype = ctypes.c_int
    lib.lf_render_host.argtypes = [vp, i32, vp, vp, vp, i32, ctypes.POINTER(i64), vp]
    lib.lf_render_host.restype = ctypes.c_int
    lib.lf_host_wait.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_uint32)]
    lib.lf_host_wait.restype = ctypes.c_int
    lib.lf_prefilter.argtypes = [vp, vp, i32, i32, i32, vp, i32, vp, vp]
    lib.lf_prefilter.restype = ctypes.c_int
    lib.lf_cache_create.argtypes = [i32, i32, ctypes.POINTER(vp)]
    lib.lf_cache_create.restype = ctypes.c_int
    lib.lf_cache_destroy.argtypes = [vp]
    lib.lf_cache_destroy.restype = None
    lib.lf_cache_frame.argtypes = [vp, i32, vp, i32, ctypes.POINTER(i32), vp, vp]
    lib.lf_cache_frame.restype = ctypes.c_int
    lib.lf_cache_pages.argtypes = [vp, vp]
    lib.lf_cache_pages.restype = ctypes.c_int
    lib.lf_set_disk_ovals.argtypes = [vp, vp]
    lib.lf_set_disk_ovals.restype = ctypes.c_int
    lib.lf_prefilter_cameras.argtypes = [vp, i32, i32, vp, i32, vp, vp]
    lib.lf_prefilter_cameras.restype = ctypes.c_int
    lib.lf_set_levels.argtypes = [vp, i32, i32]
    lib.lf_set_levels.restype = ctypes.c_int
    lib.lf_upload_pages.argtypes = [vp, i32, vp, vp, vp, vp]
    lib.lf_upload_pages.restype = ctypes.c_int
    lib.lf_levels_wanted.argtypes = [vp, i32, vp, ctypes.POINTER(i32)]
    lib.lf_levels_wanted.restype = ctypes.c_int
    lib.lf_set_wait_limit.argtypes = [vp, i64]
    lib.lf_set_wait_limit.restype = ctypes.c_int
    lib.lf_set_timing.argtypes = [vp, i32]
    lib.lf_set_timing.restype = ctypes.c_int
    lib.lf_status_string.argtypes = [ctypes.c_int]
    lib.lf_status_string.restype = ctypes.c_char_p
    lib.lf_last_error.argtypes = [vp]
    lib.lf_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _poses(poses) -> ctypes.Array:
    P = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(-1, 12))
    arr = (Pose * P.shape[0])()
    ctypes.memmove(arr, P.ctypes.data, P.nbytes)
    return arr


def _intrinsics(intr, sizes) -> ctypes.Array:
    K = np.asarray(intr, dtype=np.float64).reshape(-1, 4)
    arr = (Intrinsics * K.shape[0])()
    for k in range(K.shape[0]):
        arr[k].fx, arr[k].fy, arr[k].cx, arr[k].cy = (float(x) for x in K[k])
        arr[k].width, arr[k].height = int(sizes[k][0]), int(sizes[k][1])
    return arr


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class PageCache:
    """Host-side page cache of streamed images (lf_cache_*): which of n_items
    images occupy which of `capacity` device pages, FIFO eviction of images the
    frame does not want, at most `budget` admissions per frame."""

    def __init__(self, n_items: int, capacity: int):
        self.lib = load_library()
        self.h = ctypes.c_void_p()
        st = self.lib.lf_cache_create(int(n_items), int(capacity), ctypes.byref(self.h))
        if st != LF_OK:
            raise LFError(st, "lf_cache_create failed")
        self.n_items = int(n_items)

    def frame(self, wanted, budget: int):
        """Admit missing wanted images (most important first); returns [(item, page)]."""
        w = np.ascontiguousarray(np.asarray(wanted, dtype=np.int32).ravel())
        items = np.zeros(max(int(budget), 1), np.int32)
        pages = np.zeros(max(int(budget), 1), np.int32)
        n = ctypes.c_int32(0)
        st = self.lib.lf_cache_frame(self.h, w.size, w.ctypes.data_as(ctypes.c_void_p), int(budget), ctypes.byref(n),
                                     items.ctypes.data_as(ctypes.c_void_p), pages.ctypes.data_as(ctypes.c_void_p))
        if st != LF_OK:
            raise LFError(st, "lf_cache_frame failed")
        return list(zip(items[:n.value].tolist(), pages[:n.value].tolist()))

    def pages(self) -> np.ndarray:
        """The page of every image after the last frame (-1: not resident)."""
        out = np.zeros(self.n_items, np.int32)
        st = self.lib.lf_cache_pages(self.h, out.ctypes.data_as(ctypes.c_void_p))
        if st != LF_OK:
            raise LFError(st, "lf_cache_pages failed")
        return out

    def close(self):
        if self.h:
            self.lib.lf_cache_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Renderer:
    """One library context on one GPU."""

    def __init__(self, device: int = 0, tile=(16, 16), max_eyes: int = 2, tri_capacity: int = 0,
                 z_near: float = 0.1, timing: bool = False):
        self.lib = load_library()
        cfg = Config()
        self.lib.lf_config_default(ctypes.byref(cfg))
        cfg.tile_w, cfg.tile_h = int(tile[0]), int(tile[1])
        cfg.max_eyes = int(max_eyes)
        if tri_capacity:
            cfg.tri_capacity = int(tri_capacity)
        cfg.z_near = float(z_near)
        cfg.timing = 1 if timing else 0
        self.device = device
        self.ctx = ctypes.c_void_p()
        self._check(self.lib.lf_create(device, ctypes.byref(cfg), ctypes.byref(self.ctx)), "lf_create")
        self.n_views = 0
        self._src_hw = (0, 0)   # source image size once views are loaded
        self._in_flight = []    # (frame, host tensors) of render_host not yet known to be delivered

    def close(self):
        if self.ctx:
            self.lib.lf_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status: int, what: str):
        if status != LF_OK:
            msg = self.lib.lf_last_error(self.ctx).decode() if self.ctx else ""
            raise LFError(status, "%s failed: %s" % (what, msg))

    # ------------------------------------------------------------ loading

    def load_views(self, lf, tex_format: str = "f32"):
        """Upload source views, disks and the capture sphere (lf_load_views)."""
        n = lf.poses.shape[0]
        poses = _poses(lf.poses)
        intr = _intrinsics(lf.intr, [(lf.width, lf.height)] * n)
        images = np.ascontiguousarray(lf.images, dtype=np.uint8)
        ptrs = (ctypes.c_void_p * n)(*[images.ctypes.data + k * images[0].nbytes for k in range(n)])
        dc = np.ascontiguousarray(lf.disk_c, dtype=np.float32)
        dr = np.ascontiguousarray(lf.disk_r, dtype=np.float32)
        sc = (ctypes.c_double * 3)(*[float(x) for x in lf.sphere_c])
        self._check(self.lib.lf_load_views(self.ctx, n, poses, intr, ptrs, dc.ctypes.data, dr.ctypes.data, sc,
                                           float(lf.sphere_r), TEX_FORMATS[tex_format]), "lf_load_views")
        self.n_views = n
        self.n_fine = 0
        self._src_hw = (lf.height, lf.width)
        if getattr(lf, "disk_ext", None) is not None:
            self.set_disk_ovals(lf.disk_ext)

    def set_disk_ovals(self, extents):
        """Asymmetric oval disks (lf_set_disk_ovals, Sec. 4.4): extents n x 4
        (+u, -u, +v, -v) in metres, e.g. from disks.oval_extents; None: round."""
        if extents is None:
            self._check(self.lib.lf_set_disk_ovals(self.ctx, None), "lf_set_disk_ovals")
            return
        E = np.ascontiguousarray(np.asarray(extents, dtype=np.float32).reshape(-1, 4))
        if E.shape[0] != self.n_views:
            raise ValueError("one row of 4 extents per view")
        self._check(self.lib.lf_set_disk_ovals(self.ctx, E.ctypes.data_as(ctypes.c_void_p)), "lf_set_disk_ovals")

    def build_meshes(self, lf, mesh_format: str = "f32"):
        """Upload the per-view depth grids (lf_build_view_meshes)."""
        depth = np.ascontiguousarray(lf.depth, dtype=np.float32)
        self._check(self.lib.lf_build_view_meshes(self.ctx, int(lf.grid_n), depth.ctypes.data,
                                                  MESH_FORMATS[mesh_format]), "lf_build_view_meshes")

    # ------------------------------------------------------------ rendering

    @staticmethod
    def _eye_arrays(eyes):
        poses = _poses([e.pose for e in eyes])
        intr = _intrinsics([e.intr for e in eyes], [(e.width, e.height) for e in eyes])
        return poses, intr

    def _outputs(self, eyes, out):
        import torch
        if out is None:
            out = [torch.empty((e.height, e.width, 4), dtype=torch.float32, device="cuda:%d" % self.device)
                   for e in eyes]
        for e, o in zip(eyes, out):
            if o.dtype != torch.float32 or not o.is_cuda or not o.is_contiguous() or tuple(o.shape) != (e.height, e.width, 4):
                raise ValueError("each output must be a contiguous float32 CUDA tensor of shape (H, W, 4)")
        ptrs = (ctypes.c_void_p * len(out))(*[o.data_ptr() for o in out])
        return out, ptrs

    def render(self, eyes, out=None, stream=None):
        """Render eye views (lf_render); returns the output tensors (H, W, 4)."""
        poses, intr = self._eye_arrays(eyes)
        out, ptrs = self._outputs(eyes, out)
        self._check(self.lib.lf_render(self.ctx, len(eyes), poses, intr, ptrs, _stream_handle(stream)), "lf_render")
        return out

    def render_host(self, eyes, out=None, form: str = "plain", stream=None):
        """Render eye views and deliver them to host memory (lf_render_host): the
        device->host copy of this frame overlaps the rendering of the next.
        form: "plain" (lf_render), "refined" (lf_render_refined) or "batch" (the
        persistent raster of lf_render_batch).  `out` holds one contiguous
        float32 CPU tensor (H, W, 4) per eye, pinned for an asynchronous copy
        (allocated pinned when None).  Returns (frame, out); the images are
        complete once host_wait(frame) returns."""
        import torch
        if out is None:
            out = [torch.empty((e.height, e.width, 4), dtype=torch.float32, pin_memory=True) for e in eyes]
        for e, o in zip(eyes, out):
            if o.dtype != torch.float32 or o.is_cuda or not o.is_contiguous() or tuple(o.shape) != (e.height, e.width, 4):
                raise ValueError("each host output must be a contiguous float32 CPU tensor of shape (H, W, 4)")
        if len(out) != len(eyes):
            raise ValueError("one host output per eye")
        poses, intr = self._eye_arrays(eyes)
        ptrs = (ctypes.c_void_p * len(out))(*[o.data_ptr() for o in out])
        frame = ctypes.c_int64(-1)
        self._check(self.lib.lf_render_host(self.ctx, len(eyes), poses, intr, ptrs, HOST_FORMS[form],
                                            ctypes.byref(frame), _stream_handle(stream)), "lf_render_host")
        # keep the host buffers alive until their frame is delivered
        self._in_flight = [(f, o) for f, o in self._in_flight if f > frame.value - HOST_FRAMES_IN_FLIGHT]
        self._in_flight.append((frame.value, out))
        return frame.value, out

    def host_wait(self, frame: int = -1) -> int:
        """Wait until `frame` (every frame when negative) of render_host is in host
        memory; returns the OR of the delivered frames' device error bits."""
        err = ctypes.c_uint32(0)
        self._check(self.lib.lf_host_wait(self.ctx, int(frame), ctypes.byref(err)), "lf_host_wait")
        if frame < 0:
            self._in_flight = []
        else:
            self._in_flight = [(f, o) for f, o in self._in_flight if f > frame]
        return err.value

    def render_batch(self, eyes, out=None, stream=None):
        """Render many eyes in one graph-replayed persistent launch (lf_render_batch)."""
        poses, intr = self._eye_arrays(eyes)
        out, ptrs = self._outputs(eyes, out)
        self._check(self.lib.lf_render_batch(self.ctx, len(eyes), poses, intr, ptrs, _stream_handle(stream)),
                    "lf_render_batch")
        return out

    def tune_batch(self, eyes, out=None, replays: int = 3, stream=None) -> dict:
        """Autotune the batched render for this batch layout (lf_tune_batch)."""
        poses, intr = self._eye_arrays(eyes)
        out, ptrs = self._outputs(eyes, out)
        t = Tuning()
        self._check(self.lib.lf_tune_batch(self.ctx, len(eyes), poses, intr, ptrs, int(replays),
                                           _stream_handle(stream), ctypes.byref(t)), "lf_tune_batch")
        tried = [{"tile": (t.tried_tile_w[k], t.tried_tile_h[k]), "blocks_per_sm": t.tried_blocks[k],
                  "ms": t.tried_ms[k]} for k in range(t.n_tried)]
        return {"tile": (t.tile_w, t.tile_h), "blocks_per_sm": t.blocks_per_sm, "ms": t.ms, "tried": tried,
                "out": out}

    def render_static(self, eye, out=None, stream=None):
        """Render one eye without allocating (lf_render_static): per-call scratch
        comes from a static device array; see include/lf.h for its limits."""
        poses, intr = self._eye_arrays([eye])
        out, ptrs = self._outputs([eye], None if out is None else [out])
        self._check(self.lib.lf_render_static(self.ctx, poses, intr, ctypes.c_void_p(ptrs[0]),
                                              _stream_handle(stream)), "lf_render_static")
        return out[0]

    def render_inspect(self, eye, max_records: int = 16, stream=None):
        """Inspection render of one eye: image, per-pixel (pixel, view) coverage
        records, view-selection flags and optionally the touched-texel bitset."""
        import torch
        dev = "cuda:%d" % self.device
        poses, intr = self._eye_arrays([eye])
        out = torch.empty((eye.height, eye.width, 4), dtype=torch.float32, device=dev)
        n_pix = eye.width * eye.height
        rec = torch.zeros((n_pix * max_records * 6,), dtype=torch.int32, device=dev)
        counts = torch.zeros((n_pix,), dtype=torch.int32, device=dev)
        active = torch.zeros((self.n_views,), dtype=torch.uint8, device=dev)
        self._check(self.lib.lf_render_inspect(self.ctx, poses, intr, ctypes.c_void_p(out.data_ptr()),
                                               ctypes.c_void_p(rec.data_ptr()), max_records,
                                               ctypes.c_void_p(counts.data_ptr()), ctypes.c_void_p(active.data_ptr()),
                                               None, _stream_handle(stream)), "lf_render_inspect")
        torch.cuda.synchronize(self.device)
        recs = rec.cpu().numpy().view(FRAG_RECORD_DTYPE).reshape(n_pix, max_records)
        return {"rgba": out, "records": recs, "counts": counts.cpu().numpy(),
                "active": active.cpu().numpy().astype(bool)}

    def unique_texels(self, eyes, src_w: int, src_h: int, stream=None) -> int:
        """Distinct source texels read by the winners' bilinear footprints over
        all the given eyes (one shared bitset: texels both eyes read count once)."""
        import torch
        dev = "cuda:%d" % self.device
        nbits = self.n_views * src_w * src_h
        bits = torch.zeros(((nbits + 31) // 32,), dtype=torch.int32, device=dev)
        for eye in eyes:
            poses, intr = self._eye_arrays([eye])
            out = torch.empty((eye.height, eye.width, 4), dtype=torch.float32, device=dev)
            n_pix = eye.width * eye.height
            rec = torch.zeros((n_pix * 6,), dtype=torch.int32, device=dev)
            counts = torch.zeros((n_pix,), dtype=torch.int32, device=dev)
            active = torch.zeros((self.n_views,), dtype=torch.uint8, device=dev)
            self._check(self.lib.lf_render_inspect(self.ctx, poses, intr, ctypes.c_void_p(out.data_ptr()),
                                                   ctypes.c_void_p(rec.data_ptr()), 1,
                                                   ctypes.c_void_p(counts.data_ptr()),
                                                   ctypes.c_void_p(active.data_ptr()),
                                                   ctypes.c_void_p(bits.data_ptr()), _stream_handle(stream)),
                        "lf_render_inspect")
        torch.cuda.synchronize(self.device)
        total = 0
        for w in torch.split(bits, 1 << 24):
            b = w.cpu().numpy().view(np.uint8)
            total += int(np.unpackbits(b).sum())
        return total

    def stats(self) -> dict:
        s = Stats()
        st = self.lib.lf_get_stats(self.ctx, ctypes.byref(s))
        d = {"n_eyes": s.n_eyes, "n_views": s.n_views, "active_views": [s.active_views[0], s.active_views[1]],
             "triangles": s.triangles, "tiles": s.tiles, "error_word": s.error_word, "status": STATUS.get(st, st),
             "ms_view_setup": s.ms_view_setup, "ms_tri_setup": s.ms_tri_setup, "ms_raster": s.ms_raster}
        if st != LF_OK:
            raise LFError(st, "lf_get_stats: " + self.lib.lf_last_error(self.ctx).decode())
        return d

    # ------------------------------------------------------------ learned refinement

    def load_refiner(self, params):
        """Load refinement weights (flat FP32 vector, REFINE_N_PARAMS) and reset Adam."""
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
        if p.size != REFINE_N_PARAMS:
            raise ValueError("expected %d refiner parameters, got %d" % (REFINE_N_PARAMS, p.size))
        self._check(self.lib.lf_load_refiner(self.ctx, p.ctypes.data_as(ctypes.c_void_p)), "lf_load_refiner")

    def set_refine_kernel(self, kind: str):
        """'fused' (one tcgen05 kernel per tile) or 'layers' (three tcgen05 launches, one per layer)."""
        self._check(self.lib.lf_refine_set_kernel(self.ctx, REFINE_KERNELS[kind]), "lf_refine_set_kernel")

    def set_levels(self, n_fine: int, n_pages: int):
        """Views [0, n_fine) become the streamed fine level with n_pages device pages (Sec. 7.2)."""
        self._check(self.lib.lf_set_levels(self.ctx, int(n_fine), int(n_pages)), "lf_set_levels")
        self.n_fine = int(n_fine)

    def upload_pages(self, views, pages, images, stream=None):
        """Copy fine images (host uint8 H x W x 4 each) into pages; images[k] goes with views[k]."""
        v = np.ascontiguousarray(np.asarray(views, dtype=np.int32).ravel())
        p = np.ascontiguousarray(np.asarray(pages, dtype=np.int32).ravel())
        imgs = [np.ascontiguousarray(im, dtype=np.uint8) for im in images]
        if not (len(imgs) == v.size == p.size):
            raise ValueError("one image per (view, page)")
        ptrs = (ctypes.c_void_p * max(1, len(imgs)))(*[im.ctypes.data for im in imgs])
        self._check(self.lib.lf_upload_pages(self.ctx, int(v.size), v.ctypes.data_as(ctypes.c_void_p),
                                             p.ctypes.data_as(ctypes.c_void_p), ptrs, _stream_handle(stream)),
                    "lf_upload_pages")

    def levels_wanted(self) -> np.ndarray:
        """Fine views the last render call selected (what the next frames want resident)."""
        cap = getattr(self, "n_fine", 0) or self.n_views
        out = np.zeros(max(1, cap), np.int32)
        n = ctypes.c_int32(0)
        self._check(self.lib.lf_levels_wanted(self.ctx, int(cap), out.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.byref(n)), "lf_levels_wanted")
        return out[:n.value].copy()

    def set_timing(self, on: bool):
        """Per-kernel timing events (lf_get_stats' kernel times) on or off for later calls."""
        self._check(self.lib.lf_set_timing(self.ctx, 1 if on else 0), "lf_set_timing")

    def set_wait_limit(self, wait_ns: int):
        """Bound each later device wait to wait_ns nanoseconds (0: the default, 2 s)."""
        self._check(self.lib.lf_set_wait_limit(self.ctx, int(wait_ns)), "lf_set_wait_limit")

    def get_refiner(self) -> dict:
        arrs = {k: np.zeros(REFINE_N_PARAMS, np.float32) for k in ("params", "grad", "m", "v")}
        step, loss = ctypes.c_int32(), ctypes.c_float()
        self._check(self.lib.lf_get_refiner(self.ctx, *(arrs[k].ctypes.data_as(ctypes.c_void_p)
                                                        for k in ("params", "grad", "m", "v")),
                                            ctypes.byref(step), ctypes.byref(loss)), "lf_get_refiner")
        arrs["step"], arrs["loss"] = step.value, loss.value
        return arrs

    @staticmethod
    def _images(t):
        import torch
        if t.dim() == 3:
            t = t.unsqueeze(0)
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.shape[-1] != 4:
            raise ValueError("images must be contiguous CUDA float32 (n, H, W, 4)")
        return t

    def refine(self, images, out=None, stream=None):
        """Refined copies of RGBA images (n, H, W, 4) or (H, W, 4) on this device (lf_refine)."""
        import torch
        x = self._images(images)
        y = torch.empty_like(x) if out is None else self._images(out)
        n, h, w, _ = x.shape
        self._check(self.lib.lf_refine(self.ctx, n, w, h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       _stream_handle(stream)), "lf_refine")
        return y if images.dim() == 4 else y[0]

    def refine_gradients(self, inputs, targets, stream=None):
        x, t = self._images(inputs), self._images(targets)
        if x.shape != t.shape:
            raise ValueError("inputs and targets differ in shape")
        n, h, w, _ = x.shape
        self._check(self.lib.lf_refine_gradients(self.ctx, n, w, h, ctypes.c_void_p(x.data_ptr()),
                                                 ctypes.c_void_p(t.data_ptr()), _stream_handle(stream)),
                    "lf_refine_gradients")

    def refine_train_step(self, inputs, targets, lr: float, stream=None):
        x, t = self._images(inputs), self._images(targets)
        if x.shape != t.shape:
            raise ValueError("inputs and targets differ in shape")
        n, h, w, _ = x.shape
        self._check(self.lib.lf_refine_train_step(self.ctx, n, w, h, ctypes.c_void_p(x.data_ptr()),
                                                  ctypes.c_void_p(t.data_ptr()), float(lr), _stream_handle(stream)),
                    "lf_refine_train_step")

    def prefilter(self, dense, samples, first_view: int = 0, n_views=None, supersample: int = 1, out=None,
                  stream=None):
        """Prefiltered images of views first_view .. (lf_prefilter, Sec. 5 Eq. 5)
        with Lbar from `dense` (a Renderer holding the higher-quality model,
        created with max_eyes >= len(samples)).  samples: J x 4 (a, b, ds, dt).
        Returns a CUDA tensor (n_views, H, W, 4) float32."""
        import torch
        S = np.ascontiguousarray(np.asarray(samples, dtype=np.float32).reshape(-1, 4))
        if n_views is None:
            n_views = max(0, self.n_views - first_view)
        H, W = self._src_hw
        if out is None:
            out = torch.empty((n_views, H, W, 4), dtype=torch.float32, device="cuda:%d" % self.device)
        if out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous() or tuple(out.shape) != (n_views, H, W, 4):
            raise ValueError("out must be a contiguous float32 CUDA tensor of shape (n_views, H, W, 4)")
        self._check(self.lib.lf_prefilter(self.ctx, dense.ctx, int(first_view), int(n_views), S.shape[0],
                                          S.ctypes.data_as(ctypes.c_void_p), int(supersample),
                                          ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), "lf_prefilter")
        return out

    def prefilter_cameras(self, view: int, samples, supersample: int = 1):
        """The render cameras of lf_prefilter for one view: poses (J x 12, R
        row-major then t), intrinsics (J x 4) and the render size (W, H)."""
        S = np.ascontiguousarray(np.asarray(samples, dtype=np.float32).reshape(-1, 4))
        J = S.shape[0]
        poses = (Pose * J)()
        intr = (Intrinsics * J)()
        self._check(self.lib.lf_prefilter_cameras(self.ctx, int(view), J, S.ctypes.data_as(ctypes.c_void_p),
                                                  int(supersample), poses, intr), "lf_prefilter_cameras")
        P = np.array([list(p.R) + list(p.t) for p in poses])
        K = np.array([[k.fx, k.fy, k.cx, k.cy] for k in intr])
        return P, K, (intr[0].width, intr[0].height) if J else (0, 0)

    def render_refined(self, eyes, out=None, stream=None):
        """lf_render followed by the refinement (plain render if no refiner is loaded)."""
        poses, intr = self._eye_arrays(eyes)
        out, ptrs = self._outputs(eyes, out)
        self._check(self.lib.lf_render_refined(self.ctx, len(eyes), poses, intr, ptrs, _stream_handle(stream)),
                    "lf_render_refined")
        return out
