"""Pins of the oracle's asymmetric oval disks (Sec. 4.4) and of the Delaunay
extents helper, on the CPU.

- Closed form: an eye at the sphere centre looking at a view on the sphere
  meets that disk's plane (z = R) at t = R, so (u, v) = R (ex, ey) along the
  view's image axes and the weight is max(0, 1 - rho) with
  rho^2 = (u / e_u)^2 + (v / e_v)^2, the extents chosen by the signs of u and v.
  The oracle's FP64 weights match that to 1e-12; its FP32 membership matches
  the FP64 one away from the rim; each quarter uses its own extents (a swapped
  pair would move the rim by centimetres).
- View selection over a whole frame equals an FP64 brute force away from the rims.
- The helper's 1-ring on a square grid cap is the grid's own adjacency; on the
  Fibonacci sphere every disk has about six neighbours and extents near the spacing.
"""
import math

import numpy as np
import pytest

import oracle
import scene
from paper_1810_08860_gb300 import disks

R_SPHERE = 0.35
EXT = np.array([[0.05, 0.02, 0.03, 0.04]], np.float32)  # +u, -u, +v, -v


def _single_view(ext=EXT, W=64, H=64, G=9, D=2.0):
    Rm = scene.look_rotation([0.0, 0.0, 1.0])
    t = np.array([0.0, 0.0, R_SPHERE])
    img = np.full((1, H, W, 4), 200, np.uint8)
    depth = np.full((1, G, G), D, np.float32)
    return scene.LightField(poses=scene.pose_array(Rm, t)[None], intr=np.array([[32.0, 32.0, 32.0, 32.0]]),
                            width=W, height=H, images=img, grid_n=G, depth=depth,
                            disk_c=t[None].astype(np.float32), disk_r=np.array([0.05], np.float32),
                            sphere_c=np.zeros(3), sphere_r=R_SPHERE, name="oval", disk_ext=ext)


def _centre_eye(f=300.0, W=96, H=80):
    Rm = scene.look_rotation([0.0, 0.0, 1.0])
    return scene.Eye(scene.pose_array(Rm, (0.0, 0.0, 0.0)), np.array([f, f, 47.3, 41.1]), W, H)


def _expected_rho(eye, ext):
    f, _, cx, cy = eye.intr
    zc = float(np.float32(R_SPHERE))  # the disk plane: the disk centre is stored in FP32
    jj, ii = np.mgrid[0:eye.height, 0:eye.width]
    u = zc * (ii + 0.5 - cx) / f
    v = zc * (jj + 0.5 - cy) / eye.intr[1]
    eu = np.where(u >= 0, ext[0], ext[1])
    ev = np.where(v >= 0, ext[2], ext[3])
    return np.sqrt((u / eu) ** 2 + (v / ev) ** 2)


def test_oval_weights_closed_form():
    lf = _single_view()
    eye = _centre_eye()
    ref = oracle.render(lf, eye, fragments=True, max_slots=4)
    rho = _expected_rho(eye, EXT[0].astype(np.float64))
    W = eye.width
    got = {int(f["pixel"]): float(f["w"]) for f in ref["frags"]}
    inside = {k for k in range(eye.width * eye.height) if rho.flat[k] < 1.0}
    rim = np.abs(rho - 1.0) < 1e-5
    assert {k for k in got if not rim.flat[k]} == {k for k in inside if not rim.flat[k]}
    assert len(got) > 500
    for k, w in got.items():
        assert w == pytest.approx(max(0.0, 1.0 - rho.flat[k]), abs=1e-12)
    # every quarter has its own extents: the left/right and up/down rims are where they should be
    row = int(eye.height // 2)
    xs = [k % W for k in got if k // W == row]
    f, _, cx, _ = eye.intr
    assert max(xs) + 0.5 - cx == pytest.approx(f * EXT[0, 0] / R_SPHERE, abs=1.0)
    assert cx - (min(xs) + 0.5) == pytest.approx(f * EXT[0, 1] / R_SPHERE, abs=1.0)
    swapped = _expected_rho(eye, EXT[0, [1, 0, 2, 3]].astype(np.float64)) < 1.0
    assert np.sum(swapped != (rho < 1.0)) > 100


def test_round_mode_is_untouched_without_extents():
    lf = _single_view(ext=None)
    eye = _centre_eye()
    ref = oracle.render(lf, eye, fragments=True, max_slots=4)
    # round disk of radius 0.05 at the sphere crossing: chord distance from c
    for fr in ref["frags"][:200]:
        k = int(fr["pixel"])
        i, j = k % eye.width, k // eye.width
        d = np.array([(i + 0.5 - eye.intr[2]) / eye.intr[0], (j + 0.5 - eye.intr[3]) / eye.intr[1], 1.0])
        p = R_SPHERE * d / np.linalg.norm(d)
        c = np.array([0.0, 0.0, np.float32(R_SPHERE)], np.float64)  # disk centre and radius stored in FP32
        w = max(0.0, 1 - np.linalg.norm(p - c) / float(np.float32(0.05)))
        assert float(fr["w"]) == pytest.approx(w, abs=1e-12)


def test_oval_view_selection_matches_fp64_bruteforce():
    lf = scene.tiny_light_field(1)
    import dataclasses

    lfo = dataclasses.replace(lf, disk_ext=disks.oval_extents(lf))
    eye = lf.eyes[0]
    sel = oracle.select_views(lfo, eye)
    # FP64 plane hits of every pixel ray with every disk plane
    Re = eye.pose[:9].reshape(3, 3)
    o = eye.pose[9:12]
    jj, ii = np.mgrid[0:eye.height, 0:eye.width]
    e = np.stack([(ii + 0.5 - eye.intr[2]) / eye.intr[0], (jj + 0.5 - eye.intr[3]) / eye.intr[1],
                  np.ones_like(ii, float)], -1).reshape(-1, 3) @ Re.T
    want = np.zeros(lf.n_views, np.uint8)
    near_rim = np.zeros(lf.n_views, bool)
    for v in range(lf.n_views):
        Rv = lf.poses[v][:9].reshape(3, 3)
        c = lfo.disk_c[v].astype(np.float64)
        n = Rv[:, 2]
        den = e @ n
        t = ((c - o) @ n) / den
        q = o + t[:, None] * e - c
        u, vv = q @ Rv[:, 0], q @ Rv[:, 1]
        ext = lfo.disk_ext[v].astype(np.float64)
        rho = np.sqrt((u / np.where(u >= 0, ext[0], ext[1])) ** 2 + (vv / np.where(vv >= 0, ext[2], ext[3])) ** 2)
        ok = (den != 0) & (t >= 0)
        want[v] = np.any(ok & (rho < 1.0))
        near_rim[v] = not np.any(ok & (rho < 1.0 - 1e-5)) and np.any(ok & (rho < 1.0 + 1e-5))
    assert want.sum() >= 4
    assert np.array_equal(sel[~near_rim], want[~near_rim])


def test_delaunay_extents_on_a_grid_cap_and_the_sphere():
    lf = scene.tiny_light_field(1)  # 4 x 4 grid of views on a 40 degree cap
    nb = disks.delaunay_neighbours(lf.disk_c, lf.sphere_c)
    # the grid's axial neighbours are always in the 1-ring, nothing beyond one step is
    for k in range(16):
        r, c = divmod(k, 4)
        axial = {(r + dr) * 4 + (c + dc) for dr, dc in ((0, 1), (0, -1), (1, 0), (-1, 0))
                 if 0 <= r + dr < 4 and 0 <= c + dc < 4}
        assert axial <= nb[k]
        assert all(abs(m // 4 - r) <= 1 and abs(m % 4 - c) <= 1 for m in nb[k])
    ext = disks.oval_extents(lf)
    spacing = np.median([np.linalg.norm(lf.disk_c[k] - lf.disk_c[k + 1]) for k in (0, 1, 2, 4, 5, 6)])
    assert np.all(np.abs(ext - spacing) < 0.1 * spacing)
    rig = scene.rig_light_field(1, n_views=1024, width=16, grid_n=2)
    nb = disks.delaunay_neighbours(rig.disk_c, rig.sphere_c)
    assert 5.5 < np.mean([len(x) for x in nb]) < 6.5  # a triangulation of a sphere: 6 on average
    ext = disks.oval_extents(rig)
    s = math.sqrt(4 * math.pi * R_SPHERE ** 2 / 1024)
    assert np.all(ext > 0.4 * s) and np.all(ext < 1.6 * s)
