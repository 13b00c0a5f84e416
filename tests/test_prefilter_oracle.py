"""Pins of the prefilter oracle (Sec. 5, Eq. 4-5) against what the paper and
the mathematics fix, on the CPU.

- Lanczos-2 closed-form values; the aperture sampler's geometry (on the
  sphere, chord r sqrt(a), angle 2 pi b from the image x axis, uniform area).
- Mesh points: grid vertices exactly, a planar grid's points on its plane, and
  reprojection to the image point they came from.
- A fronto-parallel planar mesh with a linear ramp texture: bilinear
  interpolation reproduces a linear function exactly and a plane occludes
  nothing, so Eq. 5 has the closed form (i + sum_j w_j ds_j / sum_j w_j) / 255
  for any aperture positions.  A ray origin computed with the transposed
  rotation, a dropped half-pixel shift, swapped offsets or a dropped rho each
  break it (planted below).
- A constant-colour light field gives that colour; sample order does not
  matter; a sample on the disk rim (rho = 0) adds nothing.
"""
import math

import numpy as np
import pytest

import scene
from oracle import prefilter as pf

R_SPHERE = 0.35


def _plane_view(W=48, H=40, G=9, D=2.0, disk_r=0.05, fx=24.0, fy=26.0, cx=23.0, cy=21.5):
    """One view at the sphere point (0, 0, R) looking along +z at a plane z = R + D,
    texture R = column index, G = row index (exactly linear), B = 128."""
    Rm = scene.look_rotation([0.5, 0.4, 1.0])  # tilted, so R and R^T differ
    t = Rm[:, 2] * R_SPHERE
    img = np.zeros((1, H, W, 4), np.uint8)
    img[0, :, :, 0] = np.arange(W)[None, :]
    img[0, :, :, 1] = np.arange(H)[:, None]
    img[0, :, :, 2] = 128
    img[0, :, :, 3] = 255
    depth = np.full((1, G, G), D, np.float32)  # z-depth in the view's frame: a plane facing the view
    return scene.LightField(poses=scene.pose_array(Rm, t)[None], intr=np.array([[fx, fy, cx, cy]]), width=W,
                            height=H, images=img, grid_n=G, depth=depth,
                            disk_c=t[None].astype(np.float32), disk_r=np.array([disk_r], np.float32),
                            sphere_c=np.zeros(3), sphere_r=R_SPHERE, name="plane")


def _with_disk(lf, r):
    import dataclasses

    return dataclasses.replace(lf, disk_r=np.full(lf.n_views, r, np.float32))


def _samples(rng, J, ds_range=2.0):
    s = np.empty((J, 4))
    s[:, 0] = rng.uniform(0.0, 1.0, J)
    s[:, 1] = rng.uniform(0.0, 1.0, J)
    s[:, 2:] = rng.uniform(-ds_range, ds_range, (J, 2))
    return s


# ---------------------------------------------------------------- the kernels


def test_lanczos2_closed_form():
    assert pf.lanczos2(0.0) == 1.0
    for x in (1.0, -1.0, 2.0, -2.0, 2.5, -3.0):
        assert abs(float(pf.lanczos2(x))) < 1e-15
    # sinc(1/2) sinc(1/4) = (2/pi) (2 sqrt(2)/pi)
    assert float(pf.lanczos2(0.5)) == pytest.approx(4.0 * math.sqrt(2.0) / math.pi ** 2, abs=1e-15)
    # sinc(3/2) sinc(3/4) = (-2/(3 pi)) (2 sqrt(2)/(3 pi)), the negative lobe
    assert float(pf.lanczos2(1.5)) == pytest.approx(-4.0 * math.sqrt(2.0) / (9.0 * math.pi ** 2), abs=1e-15)
    xs = np.linspace(-1.9, 1.9, 39)
    assert np.allclose(pf.lanczos2(xs), pf.lanczos2(-xs), atol=0.0)


def test_sample_weight_is_rho_times_sigma():
    assert pf.sample_weight((0.25, 0.7, 0.5, 0.0)) == pytest.approx(0.5 * 4.0 * math.sqrt(2.0) / math.pi ** 2)
    assert pf.sample_weight((1.0, 0.1, 0.0, 0.0)) == 0.0  # on the rim
    assert pf.sample_weight((0.0, 0.3, 1.0, 0.2)) == pytest.approx(0.0, abs=1e-16)


def test_aperture_points_on_the_disk():
    lf = scene.tiny_light_field(1)
    rng = np.random.default_rng(4)
    for v in (0, 5, 11):
        c = lf.disk_c[v].astype(np.float64)
        n = c / np.linalg.norm(c)
        c_s = n * lf.sphere_r                      # the disk centre on the sphere
        Rv = lf.poses[v][:9].reshape(3, 3)
        xa = Rv[:, 0] - (Rv[:, 0] @ n) * n
        xa /= np.linalg.norm(xa)
        ya = np.cross(n, xa)
        for a, b in rng.uniform(0, 1, (20, 2)):
            o = pf.aperture_point(lf, v, a, b)
            assert np.linalg.norm(o) == pytest.approx((1 - pf.APERTURE_INSET) * lf.sphere_r, rel=1e-12)
            p = o / np.linalg.norm(o) * lf.sphere_r
            assert np.linalg.norm(p - c_s) == pytest.approx(float(lf.disk_r[v]) * math.sqrt(a), abs=1e-12)
            d = p - c_s
            ang = math.atan2(d @ ya, d @ xa) % (2 * math.pi)
            if a > 1e-6:
                assert min(abs(ang - 2 * math.pi * b), 2 * math.pi - abs(ang - 2 * math.pi * b)) < 1e-9
    # uniform in area: the mean squared chord over a uniform a is r^2 / 2
    a = (np.arange(4000) + 0.5) / 4000
    ch2 = [np.sum((pf.aperture_point(lf, 0, x, 0.3) / (1 - pf.APERTURE_INSET) - lf.disk_c[0]) ** 2) for x in a]
    assert np.mean(ch2) == pytest.approx(0.5 * float(lf.disk_r[0]) ** 2, rel=1e-3)


# ---------------------------------------------------------------- mesh points


def test_mesh_points_at_vertices_and_reprojection():
    lf = scene.tiny_light_field(2)
    W, H, G = lf.width, lf.height, lf.grid_n
    fx, fy, cx, cy = lf.intr[3]
    jj, kk = np.meshgrid(np.arange(G), np.arange(G))
    s, t = jj * W / (G - 1), kk * H / (G - 1)
    X = pf.mesh_points(lf, 3, s.ravel(), t.ravel())
    z = lf.depth[3].astype(np.float64).ravel()
    assert np.allclose(X[:, 2], z, rtol=1e-12)
    assert np.allclose(X[:, 0], z * (s.ravel() - cx) / fx, rtol=1e-12, atol=1e-12)
    rng = np.random.default_rng(5)
    s, t = rng.uniform(0, W, 500), rng.uniform(0, H, 500)
    X = pf.mesh_points(lf, 3, s, t)
    assert np.allclose(fx * X[:, 0] / X[:, 2] + cx, s, atol=1e-9)
    assert np.allclose(fy * X[:, 1] / X[:, 2] + cy, t, atol=1e-9)


def test_mesh_points_of_a_planar_grid_lie_on_the_plane():
    lf = _plane_view()
    # replace the depths by a tilted plane n.X = 1 sampled at the grid vertices
    nrm = np.array([0.1, -0.05, 0.5])
    G, W, H = lf.grid_n, lf.width, lf.height
    fx, fy, cx, cy = lf.intr[0]
    jj, kk = np.meshgrid(np.arange(G), np.arange(G))
    e = np.stack([(jj * W / (G - 1) - cx) / fx, (kk * H / (G - 1) - cy) / fy, np.ones_like(jj, float)], -1)
    lf.depth[0] = (1.0 / (e @ nrm)).astype(np.float32)
    rng = np.random.default_rng(6)
    X = pf.mesh_points(lf, 0, rng.uniform(0, W, 400), rng.uniform(0, H, 400))
    # the grid's depths are FP32-rounded, so the plane holds to FP32 accuracy
    assert np.allclose(X @ nrm, 1.0, atol=2e-6)


# ---------------------------------------------------------------- Eq. 5 closed forms


def _ramp_expectation(samples, pix):
    w = np.array([pf.sample_weight(s) for s in samples])
    return ((pix[:, 0] + np.sum(w * samples[:, 2]) / np.sum(w)) / 255.0,
            (pix[:, 1] + np.sum(w * samples[:, 3]) / np.sum(w)) / 255.0)


def _interior(lf, n, rng, margin=6):
    return np.stack([rng.integers(margin, lf.width - margin, n), rng.integers(margin, lf.height - margin, n)], 1)


def test_planar_ramp_closed_form():
    target = _plane_view()
    dense = _with_disk(target, 0.2)  # its disk holds every aperture point of the target's
    rng = np.random.default_rng(7)
    samples = _samples(rng, 12)
    samples[:, 2:] = rng.uniform(-0.9, 0.9, (12, 2))  # the positive lobe: no near-zero denominator
    pix = _interior(target, 300, rng)
    out = pf.prefilter(target, dense, 0, samples, pixels=pix)
    er, eg = _ramp_expectation(samples, pix)
    assert np.all(out[:, 3] == 1.0)
    # (the 1e-5 R inset moves each aperture along the view's axis: for a plane
    # facing the view that only rescales the ramp about the principal point)
    assert np.max(np.abs(out[:, 0] - er)) < 1e-9
    assert np.max(np.abs(out[:, 1] - eg)) < 1e-9
    assert np.allclose(out[:, 2], 128.0 / 255.0, atol=1e-12)


def test_planar_ramp_with_supersampled_renders():
    target = _plane_view(W=32, H=28, fx=16.0, fy=17.0, cx=15.5, cy=14.0)
    dense = _with_disk(target, 0.2)
    rng = np.random.default_rng(8)
    samples = _samples(rng, 6)
    pix = _interior(target, 100, rng)
    out = pf.prefilter(target, dense, 0, samples, supersample=2, pixels=pix)
    er, eg = _ramp_expectation(samples, pix)
    # a 2x render of the ramp samples it at half-texel steps: still linear, still exact
    assert np.max(np.abs(out[:, 0] - er)) < 1e-9 and np.max(np.abs(out[:, 1] - eg)) < 1e-9


def test_planted_mistakes_break_the_ramp(monkeypatch):
    target = _plane_view()
    dense = _with_disk(target, 0.2)
    rng = np.random.default_rng(9)
    samples = _samples(rng, 10)
    samples[:, 0] = rng.uniform(0.3, 1.0, 10)          # off-centre apertures: parallax matters
    samples[:, 2:] = rng.uniform(-0.9, 0.9, (10, 2))
    pix = _interior(target, 200, rng, margin=8)
    renders = pf.virtual_renders(target, dense, 0, samples)
    er, eg = _ramp_expectation(samples, pix)

    def err(**kw):
        out = pf.prefilter(target, dense, 0, kw.get("samples", samples), pixels=pix, renders=renders)
        return max(np.max(np.abs(out[:, 0] - er)), np.max(np.abs(out[:, 1] - eg)))

    assert err() < 1e-9
    # (1) the sample's origin taken to view i's frame with R instead of R^T
    orig = pf._view_R_t
    monkeypatch.setattr(pf, "_view_R_t", lambda lf, v: (orig(lf, v)[0].T, orig(lf, v)[1]))
    bad = pf.prefilter(target, dense, 0, samples, pixels=pix, renders=renders)
    monkeypatch.setattr(pf, "_view_R_t", orig)
    assert np.max(np.abs(bad[:, 0] - er)) > 1e-5
    # (2) the half-texel shift of the bilinear read dropped
    orig_b = pf._bilinear_premultiplied
    monkeypatch.setattr(pf, "_bilinear_premultiplied", lambda img, u, v: orig_b(img, u + 0.5, v + 0.5))
    assert err() > 1e-5
    monkeypatch.setattr(pf, "_bilinear_premultiplied", orig_b)
    # (3) ds and dt swapped
    assert err(samples=samples[:, [0, 1, 3, 2]]) > 1e-5
    # (4) rho dropped from the weights
    orig_w = pf.sample_weight
    monkeypatch.setattr(pf, "sample_weight", lambda s: float(pf.lanczos2(s[2]) * pf.lanczos2(s[3])))
    assert err() > 1e-5
    monkeypatch.setattr(pf, "sample_weight", orig_w)


def test_constant_colour_field_and_invariances():
    lf = scene.tiny_light_field(1)
    import dataclasses

    const = dataclasses.replace(lf, images=np.broadcast_to(np.array([40, 160, 220, 255], np.uint8),
                                                          lf.images.shape).copy())
    rng = np.random.default_rng(10)
    samples = _samples(rng, 6)
    samples[:, 2:] = rng.uniform(-0.9, 0.9, (6, 2))
    pix = np.stack([rng.integers(0, lf.width, 200), rng.integers(0, lf.height, 200)], 1)
    out = pf.prefilter(const, const, 5, samples, pixels=pix)
    ok = out[:, 3] > 0
    assert ok.mean() > 0.5
    assert np.allclose(out[ok, :3], np.array([40, 160, 220]) / 255.0, atol=1e-12)
    # sample order does not matter; a rim sample (rho = 0) adds nothing
    a = pf.prefilter(lf, lf, 5, samples, pixels=pix)
    b = pf.prefilter(lf, lf, 5, samples[::-1], pixels=pix)
    assert np.allclose(a, b, atol=1e-12)
    rim = np.vstack([samples, [[1.0, 0.4, 0.3, -0.2]]])
    c = pf.prefilter(lf, lf, 5, rim, pixels=pix)
    assert np.allclose(a, c, atol=1e-12)
    # positive weights only: a convex combination of render values in [0, 1]
    assert np.all(a[a[:, 3] > 0, :3] >= -1e-12) and np.all(a[a[:, 3] > 0, :3] <= 1 + 1e-12)


def test_sparse_renders_give_the_same_values():
    lf = scene.tiny_light_field(3)
    rng = np.random.default_rng(12)
    samples = _samples(rng, 4)
    pix = np.stack([rng.integers(0, lf.width, 60), rng.integers(0, lf.height, 60)], 1)
    full = pf.prefilter(lf, lf, 7, samples, pixels=pix)
    sparse = pf.prefilter(lf, lf, 7, samples, pixels=pix, sparse=True)
    assert np.array_equal(full, sparse)


def test_prefilter_sample_sets():
    import paper_1810_08860_gb300 as lfm

    for n in (1, 7, 16, 40):
        S = lfm.prefilter_samples(n, 3)
        assert S.dtype == np.float32 and S.shape == (n, 4)
        assert np.all((S[:, :2] >= 0) & (S[:, :2] < 1)) and np.all(np.abs(S[:, 2:]) <= 2)
        # one a per stratum of [0, 1)
        assert sorted(np.floor(S[:, 0].astype(np.float64) * n).astype(int).tolist()) == list(range(n))
    S = lfm.prefilter_samples(16, 5)
    cells = {(int((x + 2) // 1), int((y + 2) // 1)) for x, y in S[:, 2:].astype(np.float64)}
    assert len(cells) == 16  # a jittered 4 x 4 grid over [-2, 2)^2: one offset per cell
    assert np.array_equal(S, lfm.prefilter_samples(16, 5))  # seeded


# ---------------------------------------------------------------- Lbar per ray (the definition of Eq. 5)


def test_per_ray_lbar_ramp_closed_form():
    """Each ray's own query on the planar ramp gives the closed form exactly."""
    target = _plane_view()
    dense = _with_disk(target, 0.2)
    rng = np.random.default_rng(17)
    samples = _samples(rng, 10)
    samples[:, 2:] = rng.uniform(-0.9, 0.9, (10, 2))
    pix = _interior(target, 80, rng)
    out = pf.prefilter(target, dense, 0, samples, pixels=pix, lbar="ray")
    er, eg = _ramp_expectation(samples, pix)
    assert np.all(out[:, 3] == 1.0)
    assert np.max(np.abs(out[:, 0] - er)) < 1e-12 and np.max(np.abs(out[:, 1] - eg)) < 1e-12


def test_per_ray_lbar_planted_origin_mistake(monkeypatch):
    """The per-ray query from an origin taken to view i's frame with R
    instead of R^T (off-centre apertures) breaks the ramp."""
    target = _plane_view()
    dense = _with_disk(target, 0.2)
    rng = np.random.default_rng(19)
    samples = _samples(rng, 8)
    samples[:, 0] = rng.uniform(0.3, 1.0, 8)
    samples[:, 2:] = rng.uniform(-0.9, 0.9, (8, 2))
    pix = _interior(target, 60, rng, margin=8)
    er, _ = _ramp_expectation(samples, pix)
    orig = pf._view_R_t
    monkeypatch.setattr(pf, "_view_R_t", lambda lf, v: (orig(lf, v)[0].T, orig(lf, v)[1]))
    bad = pf.prefilter(target, dense, 0, samples, pixels=pix, lbar="ray")
    assert np.max(np.abs(bad[:, 0] - er)) > 1e-5


def _sphere_models():
    prims = scene.sphere_scene(1, 8, forward_cone_deg=35.0)
    target = scene.build_light_field(prims, scene.cap_grid_directions(4, 40.0), 64, 64, 90.0, 17, name="target")
    dense = scene.build_light_field(prims, scene.cap_grid_directions(6, 40.0), 64, 64, 90.0, 33, name="dense")
    return target, dense


def test_rendered_lbar_converges_to_the_per_ray_definition():
    """The render-and-resample reading of Lbar against each ray's own query,
    on spheres: the error shrinks as the renders grow (1x, 2x, 4x) - the
    resampling is the reading's one approximation and vanishes in the limit.
    Measured: mean |difference| ~ 9e-3 at 1x (PSNR ~ 36 dB), ~ 3e-3 at 2x,
    ~ 1e-3 at 4x."""
    import paper_1810_08860_gb300 as lfm

    target, dense = _sphere_models()
    samples = lfm.prefilter_samples(16, 12).astype(np.float64)
    rng = np.random.default_rng(1)
    pix = np.stack([rng.integers(0, 64, 100), rng.integers(0, 64, 100)], axis=1)
    ray = pf.prefilter(target, dense, 4, samples, pixels=pix, lbar="ray", details=True)
    mean_err = []
    for S in (1, 2, 4):
        ren = pf.prefilter(target, dense, 4, samples, pixels=pix, supersample=S, details=True)
        ok = (ray["den"] > 0.05 * ray["den_abs"]) & (ren["den"] > 0.05 * ren["den_abs"])
        assert ok.mean() > 0.9
        mean_err.append(float(np.abs(ren["rgba"][ok, :3] - ray["rgba"][ok, :3]).mean()))
    assert mean_err[0] < 0.03
    assert mean_err[1] < 0.6 * mean_err[0] and mean_err[2] < 0.6 * mean_err[1], mean_err
