"""Pins of the two-level progressive rendering oracle (Sec. 7.2), on the CPU.

- Every fine view resident: the frame is the fine level's own render.
- No fine view resident: the frame draws the coarse disks that overlap the
  visible fine ones; when they are all the visible coarse disks, it is the
  coarse level's own render.
- A mixed frame is Eq. 2 over the union: recomputed from the two levels'
  separate per-(pixel, view) records (weights and texel values), it agrees
  with the union render.
- The coarse disks drawn are exactly those within r_c + r_f of a missing
  visible fine disk (checked by brute force).
"""
import numpy as np
import pytest

import oracle
import scene
from oracle import twolevel


@pytest.fixture(scope="module")
def levels():
    prims = scene.sphere_scene(2, 8, forward_cone_deg=35.0)
    fine = scene.build_light_field(prims, scene.cap_grid_directions(6, 40.0), 48, 48, 90.0, 13, name="fine")
    coarse = scene.build_light_field(prims, scene.cap_grid_directions(3, 40.0), 48, 48, 90.0, 13, name="coarse")
    rng = scene.SplitMix64(41)
    eye = scene.head_pose_eyes(rng, 64, 56, 90.0, yaw_range=(-0.15, 0.15), pitch_deg=6.0, stereo=False)[0]
    return fine, coarse, eye


def test_all_fine_resident_is_the_fine_render(levels):
    fine, coarse, eye = levels
    got = twolevel.render(fine, coarse, eye, np.ones(fine.n_views, bool))
    want = oracle.render(fine, eye)["rgba"]
    assert np.array_equal(got, want)
    fmask, cmask = twolevel.drawn_views(fine, coarse, eye, np.ones(fine.n_views, bool))
    assert not cmask.any() and fmask.sum() == oracle.select_views(fine, eye).sum()


def test_no_fine_resident_falls_back_to_coarse(levels):
    fine, coarse, eye = levels
    fmask, cmask = twolevel.drawn_views(fine, coarse, eye, np.zeros(fine.n_views, bool))
    vis_c = oracle.select_views(coarse, eye).astype(bool)
    assert not fmask.any() and cmask.any()
    got = twolevel.render(fine, coarse, eye, np.zeros(fine.n_views, bool))
    if np.array_equal(cmask, vis_c):
        assert np.array_equal(got, oracle.render(coarse, eye)["rgba"])
    assert (got[..., 3] > 0).mean() > 0.5


def test_drawn_coarse_disks_by_brute_force(levels):
    fine, coarse, eye = levels
    rng = np.random.default_rng(3)
    vis_f = oracle.select_views(fine, eye).astype(bool)
    vis_c = oracle.select_views(coarse, eye).astype(bool)
    for _ in range(5):
        resident = rng.uniform(size=fine.n_views) < 0.5
        fmask, cmask = twolevel.drawn_views(fine, coarse, eye, resident)
        assert np.array_equal(fmask, vis_f & resident)
        want = np.zeros(coarse.n_views, bool)
        for k in range(coarse.n_views):
            for i in range(fine.n_views):
                if vis_f[i] and not resident[i]:
                    d = float(np.sqrt(np.sum((coarse.disk_c[k].astype(float) - fine.disk_c[i].astype(float)) ** 2)))
                    want[k] |= d < float(coarse.disk_r[k]) + float(fine.disk_r[i])
        assert np.array_equal(cmask, want & vis_c)


def test_mixed_frame_is_eq2_over_the_union(levels):
    fine, coarse, eye = levels
    resident = np.zeros(fine.n_views, bool)
    resident[::2] = True
    fmask, cmask = twolevel.drawn_views(fine, coarse, eye, resident)
    assert fmask.any() and cmask.any()
    got = twolevel.render(fine, coarse, eye, resident)
    # Eq. 2 by hand: per pixel, sum w I over the drawn views of each level's own records
    num = np.zeros((eye.height * eye.width, 3))
    den = np.zeros(eye.height * eye.width)
    for lf, mask in ((fine, fmask), (coarse, cmask)):
        ids = np.nonzero(mask)[0]
        sub = twolevel.union_light_field(lf, lf, mask, np.zeros(lf.n_views, bool))
        ref = oracle.render(sub, eye, fragments=True, max_slots=32)
        assert ref["stats"]["frag_overflow"] == 0
        for f in ref["frags"]:
            if f["winner"] < 0 or not (f["w"] > 0):
                continue
            v = ids[int(f["view"])]
            img = lf.images[v].astype(np.float64) / 255.0
            s, t = float(f["s"]) - 0.5, float(f["t"]) - 0.5
            i0, j0 = int(np.floor(s)), int(np.floor(t))
            al, be = s - i0, t - j0
            ii = np.clip([i0, i0 + 1], 0, lf.width - 1)
            jj = np.clip([j0, j0 + 1], 0, lf.height - 1)
            c = ((1 - al) * (1 - be) * img[jj[0], ii[0], :3] + al * (1 - be) * img[jj[0], ii[1], :3]
                 + (1 - al) * be * img[jj[1], ii[0], :3] + al * be * img[jj[1], ii[1], :3])
            num[int(f["pixel"])] += float(f["w"]) * c
            den[int(f["pixel"])] += float(f["w"])
    ok = den > 0
    want = np.zeros_like(num)
    want[ok] = num[ok] / den[ok, None]
    g = got.reshape(-1, 4)
    assert np.array_equal(g[:, 3] > 0, ok)
    assert np.max(np.abs(g[ok, :3] - want[ok])) < 1e-9
