"""Seeded synthetic inputs for the disk-blended light field renderer.

The paper's captured scenes (Sec. 3, Table 1) are not available, so analytic
scenes stand in for them: textured Lambertian spheres inside a textured
backdrop sphere, photographed by pinhole cameras placed on a capture sphere of
radius 0.35 m (the 70 cm rig diameter of Sec. 3), looking outward.  Each
source view gets RGBA8 pixels ray-cast at pixel centres and a G x G grid of
exact z-depths that stands in for the multiview-stereo depth map and
simplified mesh of Sec. 4.5.

This module only produces inputs.  It holds none of the rendering method's
arithmetic, and both the CPU oracle and the CUDA library read its output.
Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014)
implemented here from its published definition.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfscene.c")
_LIB = os.path.join(_HERE, "_lfscene.so")
PRIM_STRIDE = 20
CAPTURE_RADIUS = 0.35


def build(force: bool = False) -> str:
    """Compile the ray caster into an in-tree shared library."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.lfs_render.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
        lib.lfs_render.restype = ctypes.c_int
        _lib = lib
    return _lib


class SplitMix64:
    """SplitMix64 generator: 64-bit state advanced by the golden-ratio increment."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * 2.0 ** -53)

    def unit_vector(self) -> np.ndarray:
        z = self.uniform(-1.0, 1.0)
        phi = self.uniform(0.0, 2.0 * math.pi)
        s = math.sqrt(max(0.0, 1.0 - z * z))
        return np.array([s * math.cos(phi), s * math.sin(phi), z])

    def in_ball(self, radius: float) -> np.ndarray:
        while True:
            v = np.array([self.uniform(-1, 1), self.uniform(-1, 1), self.uniform(-1, 1)])
            if v @ v <= 1.0:
                return radius * v


# ---------------------------------------------------------------- geometry


def look_rotation(forward, down_hint=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Camera->world rotation whose z axis is `forward` and whose y axis (image
    down) is the projection of `down_hint`; falls back to world z when the two
    are nearly parallel."""
    z = np.asarray(forward, dtype=np.float64)
    z = z / np.linalg.norm(z)
    d = np.asarray(down_hint, dtype=np.float64)
    if abs(d @ z) > 0.999:
        d = np.array([0.0, 0.0, 1.0])
    y = d - (d @ z) * z
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    return np.stack([x, y, z], axis=1)


def yaw_pitch_dir(yaw: float, pitch: float) -> np.ndarray:
    """Direction for yaw about world -y (up) and pitch above the horizon; yaw=pitch=0 is +z."""
    return np.array([math.cos(pitch) * math.sin(yaw), -math.sin(pitch), math.cos(pitch) * math.cos(yaw)])


def pose_array(R: np.ndarray, t) -> np.ndarray:
    out = np.empty(12, dtype=np.float64)
    out[:9] = np.asarray(R, dtype=np.float64).reshape(9)
    out[9:] = np.asarray(t, dtype=np.float64)
    return out


def intrinsics_for_fov(width: int, height: int, hfov_deg: float) -> np.ndarray:
    """Square pixels, principal point at the image centre, horizontal FOV in degrees."""
    f = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return np.array([f, f, width / 2.0, height / 2.0], dtype=np.float64)


def fibonacci_directions(n: int) -> np.ndarray:
    """Quasi-uniform unit vectors: z_k = 1-(2k+1)/n, phi_k = k*pi*(3-sqrt 5)."""
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def mean_nn_distance(points: np.ndarray) -> float:
    p = np.asarray(points, dtype=np.float64)
    best = np.full(len(p), np.inf)
    for s in range(0, len(p), 512):
        d = np.linalg.norm(p[s:s + 512, None, :] - p[None, :, :], axis=2)
        for r in range(d.shape[0]):
            d[r, s + r] = np.inf
        best[s:s + 512] = d.min(axis=1)
    return float(best.mean())


# ---------------------------------------------------------------- scenes


def _prim(kind, centre, radius=0.0, normal=(0, 0, 1), col_a=(1, 1, 1), col_b=(1, 1, 1),
          period=0.0, noise_cell=0.0, noise_amp=0.0, ambient=0.2) -> np.ndarray:
    q = np.zeros(PRIM_STRIDE, dtype=np.float64)
    q[0] = kind
    q[1:4] = centre
    q[4] = radius
    q[5:8] = normal
    q[8:11] = col_a
    q[11:14] = col_b
    q[14] = period
    q[15] = noise_cell
    q[16] = noise_amp
    q[17] = ambient
    return q


LIGHT = np.array([0.35, -0.8, 0.45])


def sphere_scene(seed: int, n_spheres: int, forward_cone_deg: float | None = None,
                 backdrop_radius: float = 6.0) -> np.ndarray:
    """n_spheres textured spheres (radius U[0.2,0.6] m, centre distance U[1.5,4] m)
    inside a textured backdrop sphere.  With forward_cone_deg the sphere
    directions are confined to a cone about +z (so a forward-facing cap rig sees
    them); otherwise they are uniform over the sphere."""
    rng = SplitMix64(seed)
    prims = []
    for _ in range(n_spheres):
        if forward_cone_deg is None:
            d = rng.unit_vector()
        else:
            cz = rng.uniform(math.cos(math.radians(forward_cone_deg)), 1.0)
            phi = rng.uniform(0.0, 2.0 * math.pi)
            s = math.sqrt(1.0 - cz * cz)
            d = np.array([s * math.cos(phi), s * math.sin(phi), cz])
        dist = rng.uniform(1.5, 4.0)
        rad = rng.uniform(0.2, 0.6)
        ca = [rng.uniform(0.15, 0.95) for _ in range(3)]
        cb = [rng.uniform(0.05, 0.6) for _ in range(3)]
        prims.append(_prim(0, d * dist, rad, col_a=ca, col_b=cb, period=rng.uniform(0.08, 0.25),
                           noise_cell=0.05, noise_amp=0.3, ambient=0.2))
    ca = [rng.uniform(0.5, 0.9) for _ in range(3)]
    cb = [rng.uniform(0.1, 0.4) for _ in range(3)]
    prims.append(_prim(1, (0.0, 0.0, 0.0), backdrop_radius, col_a=ca, col_b=cb, period=0.6,
                       noise_cell=0.3, noise_amp=0.25, ambient=0.6))
    return np.stack(prims)


def plane_scene(point, normal, colour, checker_period: float = 0.0, colour_b=None) -> np.ndarray:
    """A single infinite plane; constant colour unless a checker period is given."""
    cb = colour if colour_b is None else colour_b
    return np.stack([_prim(2, point, 0.0, normal, col_a=colour, col_b=cb, period=checker_period,
                           ambient=1.0)])


def ray_cast(prims: np.ndarray, poses: np.ndarray, intr: np.ndarray, width: int, height: int,
             grid_n: int = 0, images: bool = True, pixel_depth: bool = False, light=LIGHT,
             threads: int | None = None):
    """Ray-cast cameras (poses n x 12, intr n x 4) of one size.  Returns
    (rgba8 n x H x W x 4 or None, depth grid n x G x G or None, pixel z-depth or None)."""
    lib = _load()
    prims = np.ascontiguousarray(prims, dtype=np.float64)
    poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(-1, 12))
    intr = np.ascontiguousarray(np.asarray(intr, dtype=np.float64).reshape(-1, 4))
    n = poses.shape[0]
    light = np.ascontiguousarray(light, dtype=np.float64)
    rgba = np.empty((n, height, width, 4), dtype=np.uint8) if images else None
    grid = np.empty((n, grid_n, grid_n), dtype=np.float32) if grid_n else None
    pdep = np.empty((n, height, width), dtype=np.float32) if pixel_depth else None
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.lfs_render(prims.ctypes.data_as(dp), prims.shape[0], light.ctypes.data_as(dp), n,
                        poses.ctypes.data_as(dp), intr.ctypes.data_as(dp), width, height,
                        rgba.ctypes.data if rgba is not None else None,
                        pdep.ctypes.data if pdep is not None else None,
                        grid_n, grid.ctypes.data if grid is not None else None,
                        threads or (os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("lfs_render rejected its arguments")
    return rgba, grid, pdep


# ---------------------------------------------------------------- rigs and inputs


@dataclass
class Eye:
    pose: np.ndarray          # 12 doubles: R (row-major camera->world), centre
    intr: np.ndarray          # fx, fy, cx, cy
    width: int
    height: int


@dataclass
class LightField:
    """Everything the renderer loads: source views, meshes, disks, capture sphere."""
    poses: np.ndarray         # n x 12 float64
    intr: np.ndarray          # n x 4 float64
    width: int
    height: int
    images: np.ndarray        # n x H x W x 4 uint8
    grid_n: int
    depth: np.ndarray         # n x G x G float32 (z-depth in the view's frame)
    disk_c: np.ndarray        # n x 3 float32 (world)
    disk_r: np.ndarray        # n float32
    sphere_c: np.ndarray = field(default_factory=lambda: np.zeros(3))
    sphere_r: float = CAPTURE_RADIUS
    prims: np.ndarray | None = None
    eyes: list = field(default_factory=list)
    name: str = ""
    disk_ext: np.ndarray | None = None  # n x 4 float32 oval extents (+u, -u, +v, -v), or None: round disks

    @property
    def n_views(self) -> int:
        return self.poses.shape[0]


def rig_from_directions(dirs: np.ndarray, radius: float, width: int, height: int, hfov: float):
    poses = np.stack([pose_array(look_rotation(d), radius * d) for d in dirs])
    intr = np.tile(intrinsics_for_fov(width, height, hfov), (len(dirs), 1))
    return poses, intr


def cap_grid_directions(n_side: int = 4, cap_deg: float = 40.0) -> np.ndarray:
    a = np.radians(np.linspace(-cap_deg / 2, cap_deg / 2, n_side))
    return np.stack([yaw_pitch_dir(y, p) for p in a for y in a])


def build_light_field(prims, dirs, width, height, hfov, grid_n, disk_scale=1.2,
                      radius=CAPTURE_RADIUS, name="") -> LightField:
    poses, intr = rig_from_directions(dirs, radius, width, height, hfov)
    rgba, grid, _ = ray_cast(prims, poses, intr, width, height, grid_n=grid_n)
    centres = poses[:, 9:12]
    r = disk_scale * mean_nn_distance(centres)
    return LightField(poses=poses, intr=intr, width=width, height=height, images=rgba, grid_n=grid_n,
                      depth=grid, disk_c=centres.astype(np.float32),
                      disk_r=np.full(len(dirs), r, dtype=np.float32), sphere_c=np.zeros(3),
                      sphere_r=radius, prims=prims, name=name)


def head_pose_eyes(rng: SplitMix64, width: int, height: int, hfov: float, ipd: float = 0.064,
                   ball: float = 0.2, yaw_range=(0.0, 2 * math.pi), pitch_deg=60.0, stereo=True):
    """A random head inside the ball, uniform yaw, pitch within +-pitch_deg, no
    roll; stereo eyes at +-ipd/2 along the head's right axis."""
    centre = rng.in_ball(ball)
    yaw = rng.uniform(*yaw_range)
    pitch = math.radians(rng.uniform(-pitch_deg, pitch_deg))
    R = look_rotation(yaw_pitch_dir(yaw, pitch))
    intr = intrinsics_for_fov(width, height, hfov)
    if not stereo:
        return [Eye(pose_array(R, centre), intr, width, height)]
    right = R[:, 0]
    return [Eye(pose_array(R, centre - 0.5 * ipd * right), intr, width, height),
            Eye(pose_array(R, centre + 0.5 * ipd * right), intr, width, height)]


def tiny_light_field(seed: int = 1) -> LightField:
    """8 spheres in a forward cone, 16 views in a 4x4 grid on a 40 degree cap,
    128x128 at 90 degrees, 32x32 meshes, one 256x256 eye (90 degrees) within
    0.2 m of the centre, facing the cap axis within +-10 degrees."""
    prims = sphere_scene(seed, 8, forward_cone_deg=35.0)
    lf = build_light_field(prims, cap_grid_directions(4, 40.0), 128, 128, 90.0, 32, name="tiny")
    rng = SplitMix64(seed * 7919 + 17)
    lf.eyes = head_pose_eyes(rng, 256, 256, 90.0, yaw_range=(-math.radians(10), math.radians(10)),
                             pitch_deg=10.0, stereo=False)
    return lf


def rig_light_field(seed: int = 1, n_views: int = 1024, width: int = 1024, grid_n: int = 64,
                    n_spheres: int = 24, eye_w: int = 1440, eye_h: int = 1600, n_heads: int = 1) -> LightField:
    """24 spheres, 1,024 Fibonacci views over the full capture sphere, 1024^2 at
    120 degrees, 64x64 meshes, stereo 1440x1600 eyes (100 degrees horizontal,
    IPD 64 mm) at random head poses inside the sphere."""
    prims = sphere_scene(seed, n_spheres)
    lf = build_light_field(prims, fibonacci_directions(n_views), width, width, 120.0, grid_n,
                           name="rig")
    rng = SplitMix64(seed * 7919 + 29)
    for _ in range(n_heads):
        lf.eyes += head_pose_eyes(rng, eye_w, eye_h, 100.0)
    return lf


def truth_image(lf: LightField, eye: Eye) -> np.ndarray:
    """Analytic ray-cast image of the eye view (RGBA8), the view-independent truth."""
    rgba, _, _ = ray_cast(lf.prims, eye.pose[None], eye.intr[None], eye.width, eye.height)
    return rgba[0]
