"""Asymmetric oval disk extents (Sec. 4.4), host-side preprocessing.

Each disk's extents should reach the centres of the disks in its 1-ring of a
Delaunay triangulation of the disk centres: along each of +u, -u, +v and -v
(view i's image x and y axes) the extent is the farthest coordinate on that
axis among the 1-ring neighbours lying in that direction, i.e. in the
90-degree sector around the axis (u >= |v| for +u).  For points on a sphere
the Delaunay triangulation is their convex hull; over a partial capture (a
cap) the hull also closes the cap with faces that span its rim, which are not
Delaunay triangles: faces whose circumscribed circle is wider than 1.5 times
the median nearest-neighbour angle are skipped.  A direction with no
neighbour (at the rim of a partial capture) takes the disk's largest extent.
"""
from __future__ import annotations

import numpy as np


def delaunay_neighbours(disk_c, sphere_c) -> list[set]:
    """1-ring neighbours of each disk centre on the capture sphere."""
    from scipy.spatial import ConvexHull

    d = np.asarray(disk_c, dtype=np.float64) - np.asarray(sphere_c, dtype=np.float64)
    if d.shape[0] < 4:
        raise ValueError("a Delaunay triangulation on the sphere needs at least 4 disk centres")
    u = d / np.linalg.norm(d, axis=1, keepdims=True)
    hull = ConvexHull(u)
    # median nearest-neighbour angle, from the hull's own edges
    ang = np.arccos(np.clip(np.sum(u[hull.simplices] * u[np.roll(hull.simplices, 1, axis=1)], axis=2), -1, 1))
    nn = np.full(len(u), np.inf)
    for k in range(3):
        np.minimum.at(nn, hull.simplices[:, k], ang[:, k])
        np.minimum.at(nn, np.roll(hull.simplices, 1, axis=1)[:, k], ang[:, k])
    limit = np.cos(1.5 * np.median(nn[np.isfinite(nn)]))
    nbrs = [set() for _ in range(len(u))]
    for simplex, eq in zip(hull.simplices, hull.equations):
        # the face's plane lies at cos(circumradius angle) from the centre (unit normal, outward)
        if eq[:3] @ u[simplex].mean(axis=0) <= 0.0 or -eq[3] < limit:
            continue
        for a in simplex:
            nbrs[a].update(int(b) for b in simplex if b != a)
    return nbrs


def oval_extents(lf, scale: float = 1.0) -> np.ndarray:
    """n x 4 float32 extents (+u, -u, +v, -v) in metres for lf_set_disk_ovals."""
    C = np.asarray(lf.disk_c, dtype=np.float64)
    nbrs = delaunay_neighbours(C, lf.sphere_c)
    ext = np.zeros((len(C), 4))
    for i, nb in enumerate(nbrs):
        if not nb:
            raise ValueError("disk %d has no Delaunay neighbour" % i)
        R = np.asarray(lf.poses[i][:9], dtype=np.float64).reshape(3, 3)
        rel = C[sorted(nb)] - C[i]
        u, v = rel @ R[:, 0], rel @ R[:, 1]
        au, av = np.abs(u), np.abs(v)
        sel = [(u > 0) & (u >= av), (u < 0) & (au >= av), (v > 0) & (v >= au), (v < 0) & (av >= au)]
        val = [u, -u, v, -v]
        e = [float(val[k][sel[k]].max()) if sel[k].any() else 0.0 for k in range(4)]
        m = max(e)
        ext[i] = [x if x > 0.0 else m for x in e]
    return (scale * ext).astype(np.float32)
