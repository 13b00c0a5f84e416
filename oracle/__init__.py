"""CPU oracle for disk-blended, per-view-geometry light field rendering.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only callers.  The CUDA renderer never
imports this package and shares no code with it.

`lf_oracle.c` restates the method of Overbeck et al. (TOG 2018) Sec. 4.1-4.2
as a plain per-pixel loop: Eq. 1 (one ray query per eye pixel), Eq. 2 (disk
weighted, normalised sum over views), the linear disk kernel of Sec. 4.1, and
the intra-image occlusion test of Sec. 4.2.2, rasterising each view's mesh
with a 1/256-pixel snapped int64 edge-function rasteriser.  Values are FP64.
The integer decisions (near-plane test, snap, depth winner, disk membership)
take one of two modes, `decisions=`:
  "fp64"  the definition: FP64 transform through world coordinates, llrint of
          the FP64 projection, nearest FP64 depth, FP64 disk test;
  "fp32"  the fast renderer's reading of it: the same decisions in FP32 with
          the operation order fixed in the C source (the default, so that the
          CUDA path can be compared with it bit for bit).
`margins` says how close a (pixel, view) lies to each decision boundary, which
explains every place where the two modes differ.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lf_oracle.c")
_LIB = os.path.join(_HERE, "_lf_oracle.so")

STAT_NAMES = ["tri_kept", "tri_clipped", "tri_far", "tri_degenerate", "tri_behind", "frag_cover",
              "frag_win", "src_behind", "frag_overflow"]


def build(force: bool = False) -> str:
    """Compile the oracle (no fused multiply-add contraction) into an in-tree library."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class LightFieldC(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int32), ("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("G", ctypes.c_int32), ("poses", ctypes.c_void_p), ("intr", ctypes.c_void_p),
                ("rgba", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("disk_c", ctypes.c_void_p),
                ("disk_r", ctypes.c_void_p), ("sphere_c", ctypes.c_double * 3),
                ("sphere_r", ctypes.c_double), ("z_near", ctypes.c_float), ("pad", ctypes.c_int32),
                ("disk_ext", ctypes.c_void_p), ("decisions", ctypes.c_int32), ("pad2", ctypes.c_int32)]


DECISIONS = {"fp32": 0, "fp64": 1}


class EyeC(ctypes.Structure):
    _fields_ = [("pose", ctypes.c_double * 12), ("intr", ctypes.c_double * 4),
                ("W", ctypes.c_int32), ("H", ctypes.c_int32)]


FRAG_DTYPE = np.dtype([("pixel", np.int32), ("view", np.int32), ("n_cover", np.int32),
                       ("winner", np.int32), ("min_id", np.int32), ("max_id", np.int32),
                       ("id_hash", np.uint32), ("pad", np.int32), ("w", np.float64),
                       ("s", np.float64), ("t", np.float64)])

_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        lib.orc_render.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int32, vp, vp, vp,
                                   ctypes.c_int]
        lib.orc_render.restype = ctypes.c_int
        lib.orc_select_views.argtypes = [vp, vp, vp, ctypes.c_int64, vp, ctypes.c_int]
        lib.orc_select_views.restype = ctypes.c_int
        lib.orc_pixel_fragments.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            vp, vp, vp, ctypes.c_int32]
        lib.orc_pixel_fragments.restype = ctypes.c_int
        lib.orc_view_triangles.argtypes = [vp, vp, ctypes.c_int32, vp, ctypes.c_int64, vp]
        lib.orc_view_triangles.restype = ctypes.c_int64
        lib.orc_cover_raw.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32]
        lib.orc_cover_raw.restype = ctypes.c_int
        lib.orc_margins.argtypes = [vp, vp, vp, ctypes.c_int64, vp]
        lib.orc_margins.restype = ctypes.c_int
        lib.orc_set_mutation.argtypes = [ctypes.c_int]
        lib.orc_set_mutation.restype = None
        lib.orc_mix32.argtypes = [ctypes.c_uint32]
        lib.orc_mix32.restype = ctypes.c_uint32
        _lib = lib
    return _lib


class _Bound:
    """Keeps the numpy arrays behind a LightFieldC alive."""

    def __init__(self, lf, z_near: float, decisions: str = "fp32"):
        self.poses = np.ascontiguousarray(lf.poses, dtype=np.float64)
        self.intr = np.ascontiguousarray(lf.intr, dtype=np.float64)
        self.rgba = np.ascontiguousarray(lf.images, dtype=np.uint8)
        self.depth = np.ascontiguousarray(lf.depth, dtype=np.float32)
        self.disk_c = np.ascontiguousarray(lf.disk_c, dtype=np.float32)
        self.disk_r = np.ascontiguousarray(lf.disk_r, dtype=np.float32)
        c = LightFieldC()
        c.n_views = self.poses.shape[0]
        c.W, c.H, c.G = lf.width, lf.height, lf.grid_n
        c.poses = self.poses.ctypes.data
        c.intr = self.intr.ctypes.data
        c.rgba = self.rgba.ctypes.data
        c.depth = self.depth.ctypes.data
        c.disk_c = self.disk_c.ctypes.data
        c.disk_r = self.disk_r.ctypes.data
        for k in range(3):
            c.sphere_c[k] = float(lf.sphere_c[k])
        c.sphere_r = float(lf.sphere_r)
        c.z_near = z_near
        ext = getattr(lf, "disk_ext", None)
        self.disk_ext = None if ext is None else np.ascontiguousarray(ext, dtype=np.float32).reshape(-1, 4)
        c.disk_ext = None if self.disk_ext is None else self.disk_ext.ctypes.data
        if decisions not in DECISIONS:
            raise ValueError("decisions must be 'fp32' or 'fp64'")
        c.decisions = DECISIONS[decisions]
        self.c = c


def _eye_c(eye) -> EyeC:
    e = EyeC()
    for k in range(12):
        e.pose[k] = float(eye.pose[k])
    for k in range(4):
        e.intr[k] = float(eye.intr[k])
    e.W, e.H = int(eye.width), int(eye.height)
    return e


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


def render(lf, eye, pixels=None, z_near: float = 0.1, max_slots: int = 32, fragments: bool = False,
           texel_bits: bool = False, threads: int | None = None, decisions: str = "fp32"):
    """Render one eye (all pixels, or an (n, 2) int array of (i, j)).

    Returns a dict: rgba (n x 4 float64, or H x W x 4 when pixels is None),
    stats, and optionally frags (structured records with a `pixel` index into
    the pixel list), n_slots, and unique_texels."""
    lib = _load()
    b = _Bound(lf, z_near, decisions)
    e = _eye_c(eye)
    if pixels is None:
        n = eye.width * eye.height
        pix_ptr = None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        n = pix.shape[0]
        pix_ptr = pix.ctypes.data
    out = np.zeros((n, 4), dtype=np.float64)
    frags = np.zeros(n * max_slots, dtype=FRAG_DTYPE) if fragments else None
    n_slots = np.zeros(n, dtype=np.int32) if fragments else None
    bits = None
    if texel_bits:
        nbits = lf.n_views * lf.width * lf.height
        bits = np.zeros((nbits + 63) // 64, dtype=np.uint64)
    stats = np.zeros(len(STAT_NAMES), dtype=np.int64)
    rc = lib.orc_render(ctypes.byref(b.c), ctypes.byref(e), pix_ptr, n, out.ctypes.data,
                        frags.ctypes.data if frags is not None else None, max_slots,
                        n_slots.ctypes.data if n_slots is not None else None,
                        bits.ctypes.data if bits is not None else None, stats.ctypes.data,
                        _threads(threads))
    if rc != 0:
        raise RuntimeError("orc_render failed with code %d" % rc)
    res = {"stats": dict(zip(STAT_NAMES, stats.tolist()))}
    res["rgba"] = out.reshape(eye.height, eye.width, 4) if pixels is None else out
    if fragments:
        keep = []
        for p in range(n):
            k = min(int(n_slots[p]), max_slots)
            keep.append(frags[p * max_slots:p * max_slots + k])
        res["frags"] = np.concatenate(keep) if keep else np.zeros(0, dtype=FRAG_DTYPE)
        res["n_slots"] = n_slots
    if texel_bits:
        res["unique_texels"] = int(np.unpackbits(bits.view(np.uint8)).sum())
    return res


def select_views(lf, eye, pixels=None, threads: int | None = None, decisions: str = "fp32") -> np.ndarray:
    """Boolean mask of views whose disk contains the sphere crossing of some pixel."""
    lib = _load()
    b = _Bound(lf, 0.1, decisions)
    e = _eye_c(eye)
    active = np.zeros(lf.n_views, dtype=np.uint8)
    if pixels is None:
        rc = lib.orc_select_views(ctypes.byref(b.c), ctypes.byref(e), None, 0, active.ctypes.data,
                                  _threads(threads))
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        rc = lib.orc_select_views(ctypes.byref(b.c), ctypes.byref(e), pix.ctypes.data, pix.shape[0],
                                  active.ctypes.data, _threads(threads))
    if rc != 0:
        raise RuntimeError("orc_select_views failed")
    return active.astype(bool)


def pixel_fragments(lf, eye, i: int, j: int, view: int, z_near: float = 0.1, cap: int = 64,
                    decisions: str = "fp32"):
    """All covering fragments of (pixel, view): ids, FP32 1/z key, FP64 depth."""
    lib = _load()
    b = _Bound(lf, z_near, decisions)
    e = _eye_c(eye)
    ids = np.zeros(cap, dtype=np.int32)
    iz = np.zeros(cap, dtype=np.float32)
    z = np.zeros(cap, dtype=np.float64)
    n = lib.orc_pixel_fragments(ctypes.byref(b.c), ctypes.byref(e), i, j, view, ids.ctypes.data,
                                iz.ctypes.data, z.ctypes.data, cap)
    if n < 0:
        raise RuntimeError("orc_pixel_fragments failed")
    return ids[:n], iz[:n], z[:n]


def view_triangles(lf, eye, view: int, z_near: float = 0.1, decisions: str = "fp32"):
    """Snapped, clipped, positively oriented triangles of one view: (n x 7 int64, stats)."""
    lib = _load()
    b = _Bound(lf, z_near, decisions)
    e = _eye_c(eye)
    cap = 4 * (lf.grid_n - 1) ** 2 + 4
    rows = np.zeros((cap, 7), dtype=np.int64)
    stats = np.zeros(len(STAT_NAMES), dtype=np.int64)
    n = lib.orc_view_triangles(ctypes.byref(b.c), ctypes.byref(e), view, rows.ctypes.data, cap,
                               stats.ctypes.data)
    if n < 0:
        raise RuntimeError("orc_view_triangles failed")
    return rows[:n], dict(zip(STAT_NAMES, stats.tolist()))


def covers(X, Y, i: int, j: int) -> int:
    """Oracle coverage of pixel (i, j) by a snapped triangle in either winding:
    1 covered, 0 not, -1 zero area."""
    lib = _load()
    Xa = np.ascontiguousarray(X, dtype=np.int64)
    Ya = np.ascontiguousarray(Y, dtype=np.int64)
    return int(lib.orc_cover_raw(Xa.ctypes.data, Ya.ctypes.data, i, j))


def mix32(x: int) -> int:
    return int(_load().orc_mix32(x))


def margins(lf, eye, pixel_views, z_near: float = 0.1, decisions: str = "fp64") -> np.ndarray:
    """Distances of (i, j, view) triples to the decision boundaries, (n, 3):
    disk (|p - c|/r - 1, or rho - 1 for ovals; NaN without a crossing),
    coverage (subpixels from the pixel centre to the nearest snapped edge of
    the view's sub-triangles near it), depth ((z2 - z1)/z1 of the two nearest
    covering parents)."""
    lib = _load()
    b = _Bound(lf, z_near, decisions)
    e = _eye_c(eye)
    pv = np.ascontiguousarray(pixel_views, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((pv.shape[0], 3), dtype=np.float64)
    rc = lib.orc_margins(ctypes.byref(b.c), ctypes.byref(e), pv.ctypes.data if pv.size else None, pv.shape[0],
                         out.ctypes.data)
    if rc != 0:
        raise RuntimeError("orc_margins failed with code %d" % rc)
    return out


MUTATIONS = {"fill_rule_flipped": 1, "eye_rotation_transposed": 2, "depth_test_reversed": 3,
             "quadratic_kernel": 4, "smaller_sphere_root": 5, "no_half_texel_shift": 6, "cx_cy_swapped": 7}


def set_mutation(name=None):
    """Plant one of the MUTATIONS in the oracle (None: the correct oracle).
    For the pin tests only: they show that each plausible slip fails a pin."""
    _load().orc_set_mutation(0 if name is None else MUTATIONS[name])
