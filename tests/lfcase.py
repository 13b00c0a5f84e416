"""Hand-built light fields and FP64 geometry written independently of the oracle.

Used by the oracle pins: nothing here calls the oracle or the CUDA library.
The FP64 geometry goes through world coordinates (X_world = R_i X_cam + t_i,
X_eye = R_e^T (X_world - t_e)) rather than a composed camera-to-eye matrix.
"""
from __future__ import annotations

import math

import numpy as np

import scene


def custom_lf(poses, intr, images, depth, disk_c=None, disk_r=None, sphere_c=(0, 0, 0),
              sphere_r=scene.CAPTURE_RADIUS, eyes=()):
    poses = np.asarray(poses, dtype=np.float64).reshape(-1, 12)
    intr = np.asarray(intr, dtype=np.float64).reshape(-1, 4)
    images = np.asarray(images, dtype=np.uint8)
    depth = np.asarray(depth, dtype=np.float32)
    n = poses.shape[0]
    if disk_c is None:
        disk_c = poses[:, 9:12]
    if disk_r is None:
        disk_r = np.full(n, 0.1)
    return scene.LightField(poses=poses, intr=intr, width=images.shape[2], height=images.shape[1],
                            images=images, grid_n=depth.shape[1], depth=depth,
                            disk_c=np.asarray(disk_c, dtype=np.float32).reshape(n, 3),
                            disk_r=np.asarray(disk_r, dtype=np.float32).reshape(n),
                            sphere_c=np.asarray(sphere_c, dtype=np.float64), sphere_r=float(sphere_r),
                            eyes=list(eyes), name="custom")


def grid_cam_points(lf, view):
    """FP64 camera-frame vertices (G, G, 3) of one view: z (s-cx)/fx, z (t-cy)/fy, z."""
    G = lf.grid_n
    fx, fy, cx, cy = lf.intr[view]
    s = np.arange(G) * lf.width / (G - 1)
    t = np.arange(G) * lf.height / (G - 1)
    z = lf.depth[view].astype(np.float64)
    X = z * ((s[None, :] - cx) / fx)
    Y = z * ((t[:, None] - cy) / fy)
    return np.stack([X, Y, z], axis=-1)


def world_to_eye(eye, P):
    R = eye.pose[:9].reshape(3, 3)
    return (np.asarray(P) - eye.pose[9:12]) @ R  # R^T (P - t) for row vectors


def cam_to_world(lf, view, P):
    R = lf.poses[view, :9].reshape(3, 3)
    return np.asarray(P) @ R.T + lf.poses[view, 9:12]


def eye_vertices(lf, eye, view):
    return world_to_eye(eye, cam_to_world(lf, view, grid_cam_points(lf, view)))


def triangle_vertex_index(G, tri_id):
    cell, half = divmod(int(tri_id), 2)
    k, j = divmod(cell, G - 1)
    if half == 0:
        return [(k, j), (k, j + 1), (k + 1, j)]
    return [(k, j + 1), (k + 1, j + 1), (k + 1, j)]


def pixel_rays(eye):
    """Eye-frame ray directions with unit z for every pixel centre: (H, W, 3)."""
    fx, fy, cx, cy = eye.intr
    i = (np.arange(eye.width) + 0.5 - cx) / fx
    j = (np.arange(eye.height) + 0.5 - cy) / fy
    ex, ey = np.meshgrid(i, j)
    return np.stack([ex, ey, np.ones_like(ex)], axis=-1)


def ray_triangle(d, a, b, c):
    """Moller-Trumbore from the origin along d (..., 3) against one triangle.
    Returns (hit mask, t)."""
    e1, e2 = b - a, c - a
    p = np.cross(d, e2)
    det = p @ e1
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / det
        tv = -a
        u = (p @ tv) * inv
        q = np.cross(tv, e1)
        v = (d @ q) * inv
        t = (q @ e2) * inv
    hit = (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
    return hit, t


def project(eye, P):
    fx, fy, cx, cy = eye.intr
    P = np.asarray(P)
    return np.stack([fx * P[..., 0] / P[..., 2] + cx, fy * P[..., 1] / P[..., 2] + cy], axis=-1)


def point_segment_distance(p, a, b):
    ab = b - a
    t = np.clip(((p - a) @ ab) / max(ab @ ab, 1e-300), 0.0, 1.0)
    return np.linalg.norm(p - (a + t[..., None] * ab), axis=-1)


def sphere_crossing(o, d, centre, radius):
    """Larger root of |o + t d - C| = R (FP64)."""
    oc = o - centre
    a = d @ d
    b = oc @ d
    c = oc @ oc - radius * radius
    disc = b * b - a * c
    if disc < 0:
        return None
    t = (-b + math.sqrt(disc)) / a
    return None if t < 0 else o + t * d


def bilinear(image_u8, s, t):
    """Clamp-to-edge bilinear sample at pixel-edge coordinates (s, t), RGB in [0, 1]."""
    H, W = image_u8.shape[:2]
    u, v = s - 0.5, t - 0.5
    i0, j0 = math.floor(u), math.floor(v)
    a, b = u - i0, v - j0
    def tex(i, j):
        i = min(max(i, 0), W - 1)
        j = min(max(j, 0), H - 1)
        return image_u8[j, i, :3].astype(np.float64) / 255.0
    return ((1 - a) * (1 - b) * tex(i0, j0) + a * (1 - b) * tex(i0 + 1, j0)
            + (1 - a) * b * tex(i0, j0 + 1) + a * b * tex(i0 + 1, j0 + 1))
