"""Parity of the CUDA renderer (through the C ABI) with the CPU oracle.

Coverage and view selection must match bit for bit: every (pixel, view) pair
whose disk holds the pixel's sphere crossing, with its covering-triangle
count, id range, id hash and depth-test winner.  Colour must match within
2e-3 max-abs per channel on every pixel both sides call valid, and the valid
masks must be identical.
"""
import math

import numpy as np
import pytest

import oracle
import scene
from tests import lfcase

pytestmark = pytest.mark.gpu

COLOUR_TOL = 2e-3


@pytest.fixture(scope="module")
def lfmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_08860_gb300 as lf

    return lf


@pytest.fixture(scope="module")
def tiny():
    return scene.tiny_light_field(1)


@pytest.fixture(scope="module")
def tiny_renderer(lfmod, tiny):
    r = lfmod.Renderer(0)
    r.load_views(tiny)
    r.build_meshes(tiny)
    yield r
    r.close()


def _ref_records(ref, W, pixels=None):
    """Oracle records grouped by flat pixel index j*W+i, sorted by view.  A
    pixel listed more than once (samples drawn with replacement) keeps the
    records of its first listing."""
    out = {}
    first = {}
    for f in ref["frags"]:
        p = int(f["pixel"])
        k = p
        if pixels is not None:
            i, j = pixels[p]
            k = int(j) * W + int(i)
        if first.setdefault(k, p) != p:
            continue
        out.setdefault(k, []).append((int(f["view"]), int(f["n_cover"]), int(f["winner"]), int(f["min_id"]),
                                      int(f["max_id"]), int(f["id_hash"])))
    return out


def _gpu_records(got, flat_pixels):
    out = {}
    recs, counts = got["records"], got["counts"]
    for k in flat_pixels:
        n = int(counts[k])
        assert n <= recs.shape[1], "record overflow at pixel %d" % k
        if n:
            out[int(k)] = [(int(r["view"]), int(r["n_cover"]), int(r["winner"]), int(r["min_id"]),
                            int(r["max_id"]), int(r["id_hash"])) for r in recs[k][:n]]
    return out


def _check_full_frame(r, lf, eye, max_records=16):
    got = r.render_inspect(eye, max_records=max_records)
    ref = oracle.render(lf, eye, fragments=True, max_slots=max_records)
    assert ref["stats"]["frag_overflow"] == 0
    W, H = eye.width, eye.height
    g = _gpu_records(got, range(W * H))
    o = _ref_records(ref, W)
    assert g.keys() == o.keys()
    bad = [k for k in o if g[k] != o[k]]
    assert not bad, "coverage differs at %d pixels, first %s: gpu %s oracle %s" % (
        len(bad), bad[0], g[bad[0]], o[bad[0]])
    img = got["rgba"].cpu().numpy().astype(np.float64)
    want = ref["rgba"]
    valid = want[..., 3] > 0
    assert np.array_equal(img[..., 3] > 0, valid)
    assert np.all(img[~valid] == 0.0)
    if valid.any():
        err = np.max(np.abs(img[valid][:, :3] - want[valid][:, :3]))
        assert err <= COLOUR_TOL, err
    sel = oracle.select_views(lf, eye)
    assert np.array_equal(got["active"], sel)
    return got, ref


# ---------------------------------------------------------------- tiny configuration (256 x 256 eye, 16 views)


def test_tiny_full_frame(tiny_renderer, tiny):
    got, ref = _check_full_frame(tiny_renderer, tiny, tiny.eyes[0])
    assert ref["stats"]["frag_win"] > 10000
    assert got["active"].sum() >= 4


def test_ragged_offcentre_eye(tiny_renderer, tiny):
    """Eye sizes that are not multiples of the tile, off-centre principal point."""
    for (w, h, fx, fy, cx, cy) in [(75, 53, 50.0, 47.0, 31.3, 29.9), (17, 131, 30.0, 60.0, 9.0, 70.0)]:
        eye = scene.Eye(tiny.eyes[0].pose, np.array([fx, fy, cx, cy]), w, h)
        _check_full_frame(tiny_renderer, tiny, eye)


def test_more_tiny_poses(lfmod):
    for seed in (2, 3):
        lf = scene.tiny_light_field(seed)
        r = lfmod.Renderer(0)
        r.load_views(lf)
        r.build_meshes(lf)
        _check_full_frame(r, lf, lf.eyes[0])
        r.close()


def test_one_pixel_and_empty_eyes(tiny_renderer, tiny):
    one = scene.Eye(tiny.eyes[0].pose, np.array([1.0, 1.0, 0.5, 0.5]), 1, 1)
    _check_full_frame(tiny_renderer, tiny, one)
    # looking away from the cap: no disk holds any crossing, the image is empty
    R = scene.look_rotation([0.0, 0.0, -1.0])
    away = scene.Eye(scene.pose_array(R, (0.0, 0.0, 0.0)), np.array([32.0, 32.0, 32.0, 32.0]), 64, 64)
    got, _ = _check_full_frame(tiny_renderer, tiny, away)
    assert got["active"].sum() == 0
    assert float(got["rgba"].abs().max()) == 0.0


def test_widest_and_tallest_eyes(tiny_renderer, tiny):
    """Eye views at the 32,767-pixel limit of lf_render in one dimension
    (2,048 screen tiles across, ragged in the other dimension)."""
    pose = tiny.eyes[0].pose
    for w, h, K in [(32767, 3, [8000.0, 8000.0, 16383.5, 1.5]), (5, 32767, [8000.0, 8000.0, 2.5, 16383.5])]:
        got, ref = _check_full_frame(tiny_renderer, tiny, scene.Eye(pose, np.array(K), w, h))
        assert (ref["rgba"][..., 3] > 0).sum() > 1000


def test_65536_views_the_maximum(lfmod):
    """The largest view count lf_load_views accepts: 65,536 Fibonacci views of
    8x8 pixels with 2x2 depth grids, about 8,000 of them selected by one eye
    (2,048 view-mask words per screen tile, hundreds of views per tile)."""
    n = 65536
    prims = scene.sphere_scene(4, 8, forward_cone_deg=35.0)
    poses, intr = scene.rig_from_directions(scene.fibonacci_directions(n), scene.CAPTURE_RADIUS, 8, 8, 120.0)
    rgba, grid, _ = scene.ray_cast(prims, poses, intr, 8, 8, grid_n=2)
    r_disk = 1.2 * math.sqrt(4.0 * math.pi * scene.CAPTURE_RADIUS ** 2 / n)  # 1.2 x the mean spacing
    lf = scene.LightField(poses=poses, intr=intr, width=8, height=8, images=rgba, grid_n=2, depth=grid,
                          disk_c=poses[:, 9:12].astype(np.float32), disk_r=np.full(n, r_disk, np.float32),
                          sphere_c=np.zeros(3), sphere_r=scene.CAPTURE_RADIUS, prims=prims, name="many")
    r = lfmod.Renderer(0)
    r.load_views(lf)
    r.build_meshes(lf)
    R = scene.look_rotation([0.0, 0.0, 1.0])
    eye = scene.Eye(scene.pose_array(R, (0.02, -0.01, 0.03)), np.array([40.0, 40.0, 40.0, 30.0]), 80, 60)
    got, ref = _check_full_frame(r, lf, eye)
    assert got["active"].sum() > 4000
    assert (ref["rgba"][..., 3] > 0).all()
    r.close()


def test_eye_outside_the_capture_sphere(tiny_renderer, tiny):
    """Degenerate eye positions for the sphere crossing p of Eq. 2: behind the
    capture sphere looking through it (the outer rays miss the sphere, the
    others take the far crossing, the larger root), on the sphere, and outside
    looking away (both roots negative: no crossing, an empty image)."""
    R = scene.look_rotation([0.0, 0.0, 1.0])
    K = np.array([64.0, 64.0, 64.0, 48.0])  # 128 x 96 at 90 degrees
    behind = scene.Eye(scene.pose_array(R, (0.0, 0.0, -0.6)), K, 128, 96)
    got, ref = _check_full_frame(tiny_renderer, tiny, behind)
    valid = ref["rgba"][..., 3] > 0
    assert 0 < valid.sum() < valid.size
    on = scene.Eye(scene.pose_array(R, (0.0, 0.0, -0.35)), K, 128, 96)
    got, ref = _check_full_frame(tiny_renderer, tiny, on)
    assert (ref["rgba"][..., 3] > 0).sum() > 0
    away = scene.Eye(scene.pose_array(R, (0.0, 0.0, 0.6)), K, 128, 96)
    got, _ = _check_full_frame(tiny_renderer, tiny, away)
    assert got["active"].sum() == 0
    assert float(got["rgba"].abs().max()) == 0.0


def test_tile_shapes_identical(lfmod, tiny, tiny_renderer):
    eye = tiny.eyes[0]
    base = tiny_renderer.render([eye])[0].cpu()
    for tile in [(32, 8), (8, 8)]:
        r = lfmod.Renderer(0, tile=tile)
        r.load_views(tiny)
        r.build_meshes(tiny)
        out = r.render([eye])[0].cpu()
        assert (out == base).all(), tile
        r.close()


def test_render_matches_inspect_and_batch(lfmod, tiny):
    eyes = [tiny.eyes[0], scene.Eye(tiny.eyes[0].pose, np.array([60.0, 60.0, 50.0, 40.0]), 100, 90)]
    r = lfmod.Renderer(0, max_eyes=4)
    r.load_views(tiny)
    r.build_meshes(tiny)
    a = [o.cpu() for o in r.render(eyes)]
    for e, img in zip(eyes, a):
        assert (r.render_inspect(e)["rgba"].cpu() == img).all()
    for _ in range(2):  # capture, then replay
        b = [o.cpu() for o in r.render_batch(eyes)]
        for x, y in zip(a, b):
            assert (x == y).all()
    st = r.stats()
    assert st["error_word"] == 0 and st["n_eyes"] == 2
    r.close()


def test_timed_and_programmatic_launches_agree(lfmod, tiny):
    """Without timing events the triangle set-up and the raster are launched as
    programmatic dependents of the kernel before each; the frames, counters and
    flags must equal those of the timed (fully serialised) launches, also for
    frames enqueued back to back without a synchronisation between them."""
    eyes = [tiny.eyes[0], scene.Eye(tiny.eyes[0].pose, np.array([60.0, 60.0, 50.0, 40.0]), 100, 90)]
    r = lfmod.Renderer(0, max_eyes=2, timing=True)
    r.load_views(tiny)
    r.build_meshes(tiny)
    ref = [o.cpu() for o in r.render(eyes)]
    st_ref = r.stats()
    assert st_ref["ms_raster"] > 0 and st_ref["ms_tri_setup"] > 0
    assert lfmod.STATUS[r.lib.lf_set_timing(r.ctx, 2)] == "LF_ERR_INVALID_ARG"  # 0 or 1 only
    r.set_timing(False)
    got = [o.cpu() for o in r.render(eyes)]
    st = r.stats()
    for x, y in zip(ref, got):
        assert (x == y).all()
    assert st["ms_raster"] == 0
    for k in ("triangles", "tiles", "active_views", "error_word"):
        assert st[k] == st_ref[k], k
    torch = pytest.importorskip("torch")
    outs = [[torch.empty((e.height, e.width, 4), dtype=torch.float32, device="cuda") for e in eyes] for _ in range(6)]
    for o in outs:
        r.render(eyes, out=o)
    torch.cuda.synchronize()
    for o in outs:
        for x, y in zip(ref, o):
            assert (x == y.cpu()).all()
    assert r.stats()["error_word"] == 0
    r.close()


# ---------------------------------------------------------------- against the FP64 definition

# The kernels take the integer decisions in FP32 (the oracle's "fp32" mode, matched
# bit for bit above).  Against the definition - the oracle's "fp64" mode - a record
# may differ only where FP32 rounding can move a decision: within DISK_MARGIN of a
# disk rim (relative), EDGE_MARGIN subpixels of a snapped edge, or DEPTH_MARGIN of a
# depth tie (relative); and no more than MAX_MISMATCH of the records may differ.
DISK_MARGIN, EDGE_MARGIN, DEPTH_MARGIN, MAX_MISMATCH = 1e-5, 2.0, 1e-4, 1e-4


def _against_definition(r, lf, eye, pixels=None, max_records=32):
    """GPU records, selection and colour against the FP64-decision oracle; returns
    (records compared, records that differ)."""
    got = r.render_inspect(eye, max_records=max_records)
    ref = oracle.render(lf, eye, pixels=pixels, fragments=True, max_slots=max_records, decisions="fp64")
    W = eye.width
    if pixels is None:
        flat = list(range(W * eye.height))
        pix = None
    else:
        flat = [int(j) * W + int(i) for i, j in pixels]
        pix = pixels
    g = _gpu_records(got, flat)
    o = _ref_records(ref, W, pixels=pix)
    gk = {(k, rec[0]): rec for k in g for rec in g[k]}
    ok_ = {(k, rec[0]): rec for k in o for rec in o[k]}
    keys = set(gk) | set(ok_)
    diff = sorted(k for k in keys if gk.get(k) != ok_.get(k))
    assert len(diff) <= MAX_MISMATCH * max(1, len(keys)), (len(diff), len(keys))
    if diff:
        pv = np.array([[k % W, k // W, v] for (k, v) in diff], dtype=np.int32)
        m = oracle.margins(lf, eye, pv)
        ok = (np.abs(np.nan_to_num(m[:, 0], nan=1.0)) <= DISK_MARGIN) | (m[:, 1] <= EDGE_MARGIN) | \
            (m[:, 2] <= DEPTH_MARGIN)
        assert ok.all(), [(d, tuple(x)) for d, x, y in zip(diff, m, ok) if not y][:5]
    img = got["rgba"].cpu().numpy().astype(np.float64).reshape(-1, 4)[flat]
    want = ref["rgba"].reshape(-1, 4)
    both = (img[:, 3] > 0) & (want[:, 3] > 0)
    if both.any():
        assert np.max(np.abs(img[both, :3] - want[both, :3])) <= COLOUR_TOL
    odd = {flat[q] for q in np.nonzero((img[:, 3] > 0) != (want[:, 3] > 0))[0]}
    assert odd <= {k for (k, _) in diff}
    sel = oracle.select_views(lf, eye, decisions="fp64")
    for v in np.nonzero(got["active"] != sel)[0]:
        pv = np.array([[i, j, v] for j in range(eye.height) for i in range(eye.width)], dtype=np.int32)
        assert np.nanmin(np.abs(oracle.margins(lf, eye, pv)[:, 0])) <= DISK_MARGIN, v
    return len(keys), len(diff)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiny_frames_against_the_fp64_definition(lfmod, seed):
    lf = scene.tiny_light_field(seed)
    r = lfmod.Renderer(0)
    r.load_views(lf)
    r.build_meshes(lf)
    n, nd = _against_definition(r, lf, lf.eyes[0])
    assert n > 30000
    print("tiny seed %d: %d of %d records differ from the FP64 definition" % (seed, nd, n))
    r.close()


# ---------------------------------------------------------------- hand-built geometry


def _identity_pose(t=(0.0, 0.0, 0.0), R=None):
    return scene.pose_array(np.eye(3) if R is None else R, t)


def test_fold_over_and_clipping(lfmod):
    rng = np.random.default_rng(3)
    G, n = 17, 64
    depth = np.full((1, G, G), 4.0, dtype=np.float32)
    depth[0, 6:11, 6:11] = 1.5
    img = rng.integers(0, 256, size=(1, n, n, 4), dtype=np.uint8)
    intr = scene.intrinsics_for_fov(n, n, 90.0)
    lf = lfcase.custom_lf([_identity_pose()], [intr], img, depth, disk_c=[[0.0, 0.0, 0.0]], disk_r=[10.0],
                          sphere_r=2.0)
    r = lfmod.Renderer(0)
    r.load_views(lf)
    r.build_meshes(lf)
    for off in [(0.5, 0.15, 0.0), (-0.4, 0.45, 0.3)]:
        eye = scene.Eye(_identity_pose(off), np.array([40.0, 40.0, 32.0, 32.0]), 64, 64)
        got, ref = _check_full_frame(r, lf, eye)
        assert (got["records"]["n_cover"] >= 2).sum() > 20
    r.close()
    # a plane that passes beside and behind the eye is clipped at z_near
    depth = np.full((1, 10, 10), 2.0, dtype=np.float32)
    img = rng.integers(0, 256, size=(1, 48, 48, 4), dtype=np.uint8)
    lf = lfcase.custom_lf([_identity_pose((0.0, 0.0, -1.0))], [scene.intrinsics_for_fov(48, 48, 90.0)], img, depth,
                          disk_c=[[0.0, 0.0, 0.0]], disk_r=[10.0], sphere_r=0.5)
    r = lfmod.Renderer(0)
    r.load_views(lf)
    r.build_meshes(lf)
    eye = scene.Eye(_identity_pose((0.0, 0.0, 0.0), scene.look_rotation([1.0, 0.0, 0.2])),
                    np.array([24.0, 24.0, 24.0, 24.0]), 48, 48)
    _check_full_frame(r, lf, eye)
    r.close()


# ---------------------------------------------------------------- storage formats


def test_reduced_precision_textures(lfmod, tiny):
    eye = tiny.eyes[0]
    ref = oracle.render(tiny, eye)["rgba"]
    valid = ref[..., 3] > 0
    errs = {}
    for fmt, tol in [("u8", COLOUR_TOL), ("bf16", 8e-3), ("fp8", 0.08)]:
        r = lfmod.Renderer(0)
        r.load_views(tiny, tex_format=fmt)
        r.build_meshes(tiny)
        img = r.render([eye])[0].cpu().numpy().astype(np.float64)
        assert np.array_equal(img[..., 3] > 0, valid)
        errs[fmt] = float(np.max(np.abs(img[valid][:, :3] - ref[valid][:, :3])))
        assert errs[fmt] <= tol, (fmt, errs[fmt])
        r.close()


def test_f16_offset_meshes_match_oracle_on_the_stored_depths(lfmod, tiny):
    """The FP16-offset mesh is exact against the oracle run on the depths it stores."""
    d = tiny.depth.astype(np.float32)
    z0 = d.reshape(d.shape[0], -1).min(axis=1).astype(np.float32)
    stored = (z0[:, None, None] + (d - z0[:, None, None]).astype(np.float16).astype(np.float32)).astype(np.float32)
    lfq = lfcase.custom_lf(tiny.poses, tiny.intr, tiny.images, stored, disk_c=tiny.disk_c, disk_r=tiny.disk_r)
    r = lfmod.Renderer(0)
    r.load_views(tiny)
    r.build_meshes(tiny, mesh_format="f16")
    _check_full_frame(r, lfq, tiny.eyes[0])
    r.close()


# ---------------------------------------------------------------- rig scale (1,024 views of 1024^2, stereo 1440x1600)


@pytest.fixture(scope="module")
def rig():
    return scene.rig_light_field(1)


@pytest.mark.parametrize("disks", ["round", "oval"])
def test_rig_scale_sampled(lfmod, rig, disks):
    import dataclasses

    import torch

    if disks == "oval":  # asymmetric ovals from the Delaunay 1-ring (Sec. 4.4)
        from paper_1810_08860_gb300 import disks as dk

        rig = dataclasses.replace(rig, disk_ext=dk.oval_extents(rig))
    r = lfmod.Renderer(0)
    r.load_views(rig)
    r.build_meshes(rig)
    out = r.render(rig.eyes)  # the stereo call the benchmark times
    torch.cuda.synchronize()
    st = r.stats()
    assert st["error_word"] == 0
    rng = np.random.default_rng(0)
    for e, eye in enumerate(rig.eyes):
        img = out[e].cpu().numpy().astype(np.float64)
        pix = np.stack([rng.integers(0, eye.width, 3000), rng.integers(0, eye.height, 3000)], axis=1)
        ref = oracle.render(rig, eye, pixels=pix, fragments=True, max_slots=32)
        want = ref["rgba"]
        g = img[pix[:, 1], pix[:, 0]]
        valid = want[:, 3] > 0
        assert valid.mean() > 0.95
        assert np.array_equal(g[:, 3] > 0, valid)
        assert np.max(np.abs(g[valid][:, :3] - want[valid][:, :3])) <= COLOUR_TOL
        # coverage records at the sampled pixels, from the inspection call
        got = r.render_inspect(eye, max_records=32)
        flat = [int(j) * eye.width + int(i) for i, j in pix]
        gr = _gpu_records(got, flat)
        orr = _ref_records(ref, eye.width, pixels=pix)
        for k in set(flat):
            assert gr.get(k, []) == orr.get(k, []), k
        # view selection over every pixel
        sel = oracle.select_views(rig, eye)
        assert np.array_equal(got["active"], sel)
        assert st["active_views"][e] == int(sel.sum())
        assert (got["rgba"].cpu() == out[e].cpu()).all()
        # the same samples against the FP64 definition
        n, nd = _against_definition(r, rig, eye, pixels=pix)
        print("rig %s eye %d: %d of %d sampled records differ from the FP64 definition" % (disks, e, nd, n))
    r.close()


# ---------------------------------------------------------------- asymmetric oval disks (Sec. 4.4)


@pytest.fixture(scope="module")
def tiny_oval(tiny):
    import dataclasses

    from paper_1810_08860_gb300 import disks

    return dataclasses.replace(tiny, disk_ext=disks.oval_extents(tiny))


def test_oval_disks_full_frames(lfmod, tiny_oval, tiny):
    r = lfmod.Renderer(0)
    r.load_views(tiny_oval)
    r.build_meshes(tiny_oval)
    got, ref = _check_full_frame(r, tiny_oval, tiny_oval.eyes[0])
    assert got["active"].sum() >= 4 and ref["stats"]["frag_win"] > 10000
    eye = scene.Eye(tiny.eyes[0].pose, np.array([50.0, 47.0, 31.3, 29.9]), 75, 53)
    _check_full_frame(r, tiny_oval, eye)
    # back to round disks: the plain method again, bit for bit
    oval_img = r.render([tiny.eyes[0]])[0].cpu()
    r.set_disk_ovals(None)
    rr = lfmod.Renderer(0)
    rr.load_views(tiny)
    rr.build_meshes(tiny)
    import torch

    assert torch.equal(r.render([tiny.eyes[0]])[0].cpu(), rr.render([tiny.eyes[0]])[0].cpu())
    assert not torch.equal(oval_img, rr.render([tiny.eyes[0]])[0].cpu())
    r.close()
    rr.close()


def test_oval_disk_errors(lfmod, tiny):
    r = lfmod.Renderer(0)
    r.n_views = tiny.n_views  # the binding's own row check passes; the library must refuse
    with pytest.raises(lfmod.LFError) as info:
        r.set_disk_ovals(np.full((tiny.n_views, 4), 0.05, np.float32))
    assert info.value.status == 4  # no views loaded
    r.load_views(tiny)
    r.build_meshes(tiny)
    bad = np.full((tiny.n_views, 4), 0.05, np.float32)
    bad[3, 2] = 0.0
    with pytest.raises(lfmod.LFError) as info:
        r.set_disk_ovals(bad)
    assert info.value.status == 1
    bad[3, 2] = np.nan
    with pytest.raises(lfmod.LFError):
        r.set_disk_ovals(bad)
    with pytest.raises(ValueError):
        r.set_disk_ovals(np.full((tiny.n_views - 1, 4), 0.05, np.float32))
    # a refused call leaves round disks in place
    base = lfmod.Renderer(0)
    base.load_views(tiny)
    base.build_meshes(tiny)
    import torch

    assert torch.equal(r.render([tiny.eyes[0]])[0].cpu(), base.render([tiny.eyes[0]])[0].cpu())
    r.close()
    base.close()


def test_oval_disks_tiles_and_batch(lfmod, tiny_oval):
    import torch

    eye = tiny_oval.eyes[0]
    base = lfmod.Renderer(0)
    base.load_views(tiny_oval)
    base.build_meshes(tiny_oval)
    want = base.render([eye])[0].cpu()
    for tile in [(32, 8), (8, 8)]:
        r = lfmod.Renderer(0, tile=tile, max_eyes=3)
        r.load_views(tiny_oval)
        r.build_meshes(tiny_oval)
        assert torch.equal(r.render([eye])[0].cpu(), want)
        b = r.render_batch([eye, eye, eye])
        assert all(torch.equal(x.cpu(), want) for x in b)
        r.close()
    base.close()


# ---------------------------------------------------------------- batched render and its autotuner


def test_tuned_batch_matches_per_eye_renders(lfmod, tiny):
    import torch

    rng = scene.SplitMix64(77)
    sizes = [(64, 48), (100, 75), (33, 129), (256, 256), (17, 5), (128, 96)]
    eyes = []
    for (w, h) in sizes:
        e = scene.head_pose_eyes(rng, w, h, 90.0, yaw_range=(-0.2, 0.2), pitch_deg=10.0, stereo=False)[0]
        eyes.append(e)
    r = lfmod.Renderer(0, max_eyes=8)
    r.load_views(tiny)
    r.build_meshes(tiny)
    res = r.tune_batch(eyes, replays=2)
    assert res["tile"] in [(16, 16), (32, 8), (8, 8)]
    assert len(res["tried"]) >= 6 and all(t["ms"] > 0 for t in res["tried"])
    assert res["ms"] == min(t["ms"] for t in res["tried"])
    tuned = [o.clone() for o in res["out"]]
    again = r.render_batch(eyes)
    torch.cuda.synchronize()
    for k, e in enumerate(eyes):
        single = r.render([e])[0]
        torch.cuda.synchronize()
        assert torch.equal(single, tuned[k]) and torch.equal(single, again[k]), k
    r.close()


@pytest.mark.gpu
def test_tuner_never_picks_an_overflowing_configuration(lfmod, tiny):
    # a pool of one triangle record overflows in every configuration: each
    # replay skips its set-up work, so none may be chosen however fast it ran
    rng = scene.SplitMix64(78)
    eyes = [scene.head_pose_eyes(rng, 96, 64, 90.0, yaw_range=(-0.2, 0.2), pitch_deg=10.0, stereo=False)[0]
            for _ in range(3)]
    r = lfmod.Renderer(0, max_eyes=4, tri_capacity=1)
    r.load_views(tiny)
    r.build_meshes(tiny)
    with pytest.raises(lfmod.LFError) as info:
        r.tune_batch(eyes, replays=1)
    assert info.value.status == 7  # LF_ERR_CAPACITY
    r.render(eyes[:1])
    with pytest.raises(lfmod.LFError):
        r.stats()
    r.close()


def test_batch_at_full_batch_sizes_against_the_oracle(lfmod, tiny):
    """The batched form (persistent raster under a captured graph, autotuned)
    on a batch shaped like the 128-eye benchmark batch - 64 stereo head poses
    of sizes 512^2, 1024^2, 1440x1600, 2048^2 and two ragged ones - compared
    directly with the oracle: every eye's sampled pixels in colour and valid
    mask, and every eighth eye's coverage records at those pixels."""
    import torch

    rng = scene.SplitMix64(4243)
    sizes = [(512, 512), (1024, 1024), (1440, 1600), (2048, 2048), (333, 517), (1025, 63)]
    eyes = []
    for k in range(64):
        w, h = sizes[k % len(sizes)]
        eyes += scene.head_pose_eyes(rng, w, h, 90.0, yaw_range=(-math.radians(10), math.radians(10)),
                                     pitch_deg=10.0)
    r = lfmod.Renderer(0, max_eyes=len(eyes))
    r.load_views(tiny)
    r.build_meshes(tiny)
    tuned = [o.clone() for o in r.tune_batch(eyes, replays=1)["out"]]
    replay = r.render_batch(eyes)  # the captured graph again
    torch.cuda.synchronize()
    assert r.stats()["error_word"] == 0
    prng = np.random.default_rng(21)
    for k, e in enumerate(eyes):
        assert torch.equal(tuned[k], replay[k]), k
        pix = np.stack([prng.integers(0, e.width, 200), prng.integers(0, e.height, 200)], axis=1)
        ref = oracle.render(tiny, e, pixels=pix, fragments=(k % 8 == 0), max_slots=16)
        g = replay[k].cpu().numpy().astype(np.float64)[pix[:, 1], pix[:, 0]]
        want = ref["rgba"]
        ok = want[:, 3] > 0
        assert np.array_equal(g[:, 3] > 0, ok), k
        if ok.any():
            assert np.max(np.abs(g[ok, :3] - want[ok, :3])) <= COLOUR_TOL, k
        if k % 8 == 0:
            got = r.render_inspect(e, max_records=16)
            assert torch.equal(got["rgba"], replay[k]), k
            flat = [int(j) * e.width + int(i) for i, j in pix]
            gr = _gpu_records(got, flat)
            orr = _ref_records(ref, e.width, pixels=pix)
            for q in set(flat):
                assert gr.get(q, []) == orr.get(q, []), (k, q)
    r.close()
