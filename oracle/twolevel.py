"""FP64 oracle of two-level progressive rendering (Sec. 7.2, "Two-level
progressive rendering"; the tile cache of Sec. 4.2.1).

TEST INFRASTRUCTURE ONLY: the test suite is the only caller.

Two light fields of the same scene, each full and valid on its own: a coarse
level small enough to stay resident and a fine level whose images are
streamed into a bounded cache.  In a frame the renderer draws the visible
fine disks whose images are resident; for fine disks it could not load in
time it also draws the coarse disks in that region, and Eq. 2's normalised
sum blends whatever mix results.

Readings (where the text leaves a choice):
- Residency is per view (a whole fine image is resident or not), the unit
  this renderer streams; the paper streams 64 x 64 tiles.
- A fine disk is visible when the eye's view selection keeps it (its disk
  holds some pixel's sphere crossing, as in `oracle.select_views`).
- "The coarse level disk in that region": every visible coarse disk whose
  disk overlaps a missing visible fine disk on the capture sphere, i.e. whose
  centre lies within r_coarse + r_fine (chord distance) of it.
- The frame is Eq. 2 over the union of the drawn fine and coarse views, each
  with its own disk and mesh; both levels share one image size and sphere.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def drawn_views(fine, coarse, eye, resident):
    """Boolean masks (fine_drawn, coarse_drawn) for one eye; `resident` is a
    boolean mask over the fine views."""
    import oracle

    resident = np.asarray(resident, dtype=bool)
    vis_f = oracle.select_views(fine, eye).astype(bool)
    vis_c = oracle.select_views(coarse, eye).astype(bool)
    fine_drawn = vis_f & resident
    missing = np.nonzero(vis_f & ~resident)[0]
    cf = np.asarray(fine.disk_c, dtype=np.float64)
    cc = np.asarray(coarse.disk_c, dtype=np.float64)
    rf = np.asarray(fine.disk_r, dtype=np.float64)
    rc = np.asarray(coarse.disk_r, dtype=np.float64)
    coarse_drawn = np.zeros(coarse.n_views, dtype=bool)
    for i in missing:
        d = np.linalg.norm(cc - cf[i], axis=1)
        coarse_drawn |= d < rc + rf[i]
    return fine_drawn, coarse_drawn & vis_c


def union_light_field(fine, coarse, fine_mask, coarse_mask):
    """One light field holding the chosen views of both levels (fine first)."""
    fi, ci = np.nonzero(fine_mask)[0], np.nonzero(coarse_mask)[0]

    def cat(a, b):
        return np.concatenate([np.asarray(a)[fi], np.asarray(b)[ci]], axis=0)

    return dataclasses.replace(fine, poses=cat(fine.poses, coarse.poses), intr=cat(fine.intr, coarse.intr),
                               images=cat(fine.images, coarse.images), depth=cat(fine.depth, coarse.depth),
                               disk_c=cat(fine.disk_c, coarse.disk_c), disk_r=cat(fine.disk_r, coarse.disk_r),
                               name="two-level")


def render(fine, coarse, eye, resident, pixels=None, threads=None):
    """The two-level frame for one eye (H x W x 4, or K x 4 at `pixels`)."""
    import oracle

    fmask, cmask = drawn_views(fine, coarse, eye, resident)
    if not fmask.any() and not cmask.any():
        n = eye.width * eye.height if pixels is None else len(pixels)
        out = np.zeros((n, 4))
        return out.reshape(eye.height, eye.width, 4) if pixels is None else out
    lf = union_light_field(fine, coarse, fmask, cmask)
    return oracle.render(lf, eye, pixels=pixels, threads=threads)["rgba"]
