"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a
hand-derived fill-rule example, exact FP64 ray/triangle intersection,
closed-form weights, the single-view and constant-colour special cases of
Eq. 2, the intra-image-only depth test of Sec. 4.2.2, order independence of
the sums in Eq. 2, and convergence toward the analytic scene.  The pins run in
both decision modes of the oracle: "fp64" (the definition) and "fp32" (the
fast renderer's reading of it, the mode the CUDA path is compared with bit for
bit); the last group bounds where the two differ and explains every difference.
"""
import math
import os

import numpy as np
import pytest

import oracle
import scene
from tests import lfcase

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODES = pytest.mark.parametrize("decisions", ["fp32", "fp64"])


def _identity_pose(t=(0.0, 0.0, 0.0), R=None):
    R = np.eye(3) if R is None else R
    return scene.pose_array(R, t)


def _noise_image(rng, h, w):
    img = rng.integers(0, 256, size=(h, w, 4), dtype=np.uint8)
    img[..., 3] = 255
    return img


def fold_case(eye_offset=(0.5, 0.15, 0.0), n=64, G=17, seed=3):
    """One view at the origin facing +z with a near 5x5 vertex block in a far depth
    grid (rubber sheets fold over when seen from the side), and an eye off to
    the side.  The disk is huge so every pixel is inside it."""
    rng = np.random.default_rng(seed)
    depth = np.full((1, G, G), 4.0, dtype=np.float32)
    depth[0, 6:11, 6:11] = 1.5
    intr = scene.intrinsics_for_fov(n, n, 90.0)
    lf = lfcase.custom_lf([_identity_pose()], [intr], _noise_image(rng, n, n)[None], depth,
                          disk_c=[[0.0, 0.0, 0.0]], disk_r=[10.0], sphere_r=2.0)
    eye = scene.Eye(_identity_pose(eye_offset), np.array([40.0, 40.0, 32.0, 32.0]), 64, 64)
    return lf, eye


def _fp64_cover_sets(lf, eye, view, z_near=0.1, band=2.0 / 256.0):
    """Exact FP64 coverage of every pixel centre by every parent triangle,
    clipped at z_near, plus a mask of pixels farther than `band` pixels from
    every projected clipped-triangle edge (unambiguous under 1/256 snapping)."""
    G = lf.grid_n
    V = lfcase.eye_vertices(lf, eye, view)
    D = lfcase.pixel_rays(eye)
    H, W = eye.height, eye.width
    centres = np.stack(np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5), axis=-1)
    sets = [[[] for _ in range(W)] for _ in range(H)]
    ambiguous = np.zeros((H, W), dtype=bool)
    for tri in range(2 * (G - 1) ** 2):
        idx = lfcase.triangle_vertex_index(G, tri)
        P = [V[k, j] for (k, j) in idx]
        hit, t = lfcase.ray_triangle(D, P[0], P[1], P[2])
        hit &= t >= z_near
        # FP64 Sutherland-Hodgman clip for the projected outline
        poly = []
        for q in range(3):
            a, b = P[q], P[(q + 1) % 3]
            if a[2] >= z_near:
                poly.append(a)
            if (a[2] >= z_near) != (b[2] >= z_near):
                s = (z_near - a[2]) / (b[2] - a[2])
                poly.append(a + s * (b - a))
        if len(poly) < 3:
            continue
        uv = lfcase.project(eye, np.array(poly))
        dist = np.full((H, W), np.inf)
        for q in range(len(uv)):
            dist = np.minimum(dist, lfcase.point_segment_distance(centres, uv[q], uv[(q + 1) % len(uv)]))
        ambiguous |= dist < band
        for (jj, ii) in zip(*np.nonzero(hit)):
            sets[jj][ii].append(tri)
    return sets, ambiguous


def _record_map(res, W):
    recs = {}
    for f in res["frags"]:
        recs[(int(f["pixel"]) % W, int(f["pixel"]) // W, int(f["view"]))] = f
    return recs


# ---------------------------------------------------------------- fill rule


def test_top_left_golden():
    tris, cover = {}, {}
    with open(os.path.join(GOLDEN, "top_left_square.txt")) as fh:
        for line in fh:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] == "tri":
                v = list(map(int, p[2:]))
                tris[p[1]] = (v[0::2], v[1::2])
                cover.setdefault(p[1], set())
            elif p[0] == "cover":
                cover[p[1]].add((int(p[2]), int(p[3])))
    union = set()
    for name, (X, Y) in tris.items():
        got = {(i, j) for i in range(-1, 7) for j in range(-1, 7) if oracle.covers(X, Y, i, j) == 1}
        assert got == cover[name], name
        # winding must not matter
        got_rev = {(i, j) for i in range(-1, 7) for j in range(-1, 7)
                   if oracle.covers(X[::-1], Y[::-1], i, j) == 1}
        assert got_rev == got
        assert not (union & got)
        union |= got
    assert union == {(i, j) for i in range(4) for j in range(4)}


def test_zero_area_rejected():
    assert oracle.covers([0, 256, 512], [0, 256, 512], 0, 0) == -1


# ---------------------------------------------------------------- snapping and coverage


@MODES
def test_snap_matches_fp64_projection(decisions):
    lf, eye = fold_case()
    rows, stats = oracle.view_triangles(lf, eye, 0, decisions=decisions)
    V = lfcase.eye_vertices(lf, eye, 0)
    worst = 0.0
    for r in rows:
        idx = lfcase.triangle_vertex_index(lf.grid_n, r[0])
        P = np.array([V[k, j] for (k, j) in idx])
        if np.any(P[:, 2] < 0.1):
            continue
        uv = lfcase.project(eye, P) * 256.0
        snapped = np.array([[r[1], r[2]], [r[3], r[4]], [r[5], r[6]]], dtype=np.float64)
        for s in snapped:
            worst = max(worst, np.min(np.max(np.abs(uv - s), axis=1)))
    # round-to-nearest (0.5), plus the FP32 transform error (< 0.5 subpixel here) in the FP32 reading
    assert worst <= (1.0 if decisions == "fp32" else 0.5 + 1e-6), worst


@MODES
@pytest.mark.parametrize("eye_offset", [(0.5, 0.15, 0.0), (-0.4, 0.45, 0.3)])
def test_coverage_matches_fp64_ray_triangle(eye_offset, decisions):
    lf, eye = fold_case(eye_offset)
    res = oracle.render(lf, eye, fragments=True, decisions=decisions)
    recs = _record_map(res, eye.width)
    sets, ambiguous = _fp64_cover_sets(lf, eye, 0)
    checked = multi = 0
    for j in range(eye.height):
        for i in range(eye.width):
            if ambiguous[j, i]:
                continue
            s = sets[j][i]
            f = recs[(i, j, 0)]
            assert f["n_cover"] == len(s), (i, j, s)
            if s:
                assert f["min_id"] == min(s) and f["max_id"] == max(s)
                h = 0
                for t in s:
                    h ^= oracle.mix32(t)
                assert f["id_hash"] == h
            checked += 1
            multi += len(s) >= 2
    # pixel centres lying exactly on projected diagonals are excluded (the fill rule decides them)
    assert checked >= 0.75 * eye.width * eye.height
    assert multi > 20  # the near block folds the mesh over itself


@MODES
def test_clipped_coverage_matches_fp64(decisions):
    """A mesh that passes beside and behind the eye is clipped at z_near."""
    G, n = 10, 48
    rng = np.random.default_rng(5)
    depth = np.full((1, G, G), 2.0, dtype=np.float32)
    intr = scene.intrinsics_for_fov(n, n, 90.0)
    lf = lfcase.custom_lf([_identity_pose((0.0, 0.0, -1.0))], [intr], _noise_image(rng, n, n)[None], depth,
                          disk_c=[[0.0, 0.0, 0.0]], disk_r=[10.0], sphere_r=0.5)
    # eye at the origin looking along world +x: the plane z = 1 spans eye depths -2..2
    R = scene.look_rotation([1.0, 0.0, 0.2])
    eye = scene.Eye(_identity_pose((0.0, 0.0, 0.0), R), np.array([24.0, 24.0, 24.0, 24.0]), 48, 48)
    rows, stats = oracle.view_triangles(lf, eye, 0, decisions=decisions)
    assert stats["tri_clipped"] > 0 and stats["tri_behind"] > 0
    res = oracle.render(lf, eye, fragments=True, decisions=decisions)
    recs = _record_map(res, eye.width)
    sets, ambiguous = _fp64_cover_sets(lf, eye, 0)
    covered = 0
    for j in range(eye.height):
        for i in range(eye.width):
            if ambiguous[j, i]:
                continue
            f = recs[(i, j, 0)]
            assert f["n_cover"] == len(sets[j][i]), (i, j)
            covered += f["n_cover"] > 0
    assert covered > 50


@MODES
def test_watertight_planar_grid(decisions):
    """A fronto-parallel planar grid seen without fold-over covers every pixel
    centre inside its outline exactly once (top-left rule)."""
    G, n = 12, 64
    rng = np.random.default_rng(7)
    depth = np.full((1, G, G), 2.0, dtype=np.float32)
    intr = scene.intrinsics_for_fov(n, n, 90.0)
    lf = lfcase.custom_lf([_identity_pose()], [intr], _noise_image(rng, n, n)[None], depth,
                          disk_c=[[0.0, 0.0, 0.0]], disk_r=[10.0], sphere_r=0.5)
    R = scene.look_rotation([0.15, -0.1, 1.0])
    eye = scene.Eye(_identity_pose((0.05, 0.02, 0.1), R), np.array([50.0, 50.0, 40.0, 40.0]), 80, 80)
    res = oracle.render(lf, eye, fragments=True, decisions=decisions)
    nc = np.zeros((eye.height, eye.width), dtype=int)
    for f in res["frags"]:
        nc[f["pixel"] // eye.width, f["pixel"] % eye.width] = f["n_cover"]
    assert nc.max() == 1
    # the outline: pixels whose FP64 ray hits the plane inside the mesh extent, away from its border
    D = lfcase.pixel_rays(eye)
    Rm, t = eye.pose[:9].reshape(3, 3), eye.pose[9:12]
    dw = D @ Rm.T
    lam = (2.0 - t[2]) / dw[..., 2]
    P = t + lam[..., None] * dw
    half = 2.0 * 1.0  # 90 degree view at depth 2: x, y in [-2, 2]
    inner = (np.abs(P[..., 0]) < half - 0.05) & (np.abs(P[..., 1]) < half - 0.05)
    assert inner.sum() > 1000
    assert np.all(nc[inner] == 1)


@MODES
def test_depth_winner_is_nearest(decisions):
    lf, eye = fold_case()
    res = oracle.render(lf, eye, fragments=True, decisions=decisions)
    multi = [f for f in res["frags"] if f["n_cover"] >= 2]
    assert len(multi) > 20
    for f in multi[::3]:
        i, j = int(f["pixel"]) % eye.width, int(f["pixel"]) // eye.width
        ids, iz, z = oracle.pixel_fragments(lf, eye, i, j, 0, decisions=decisions)
        ok = z > 0
        zmin = z[ok].min()
        zw = z[ids == f["winner"]][0]
        if decisions == "fp64":
            # the nearest FP64 depth, ties to the lowest id
            assert f["winner"] == ids[ok][z[ok] == zmin].min()
            continue
        near_tie = np.sum(np.abs(z[ok] - zmin) <= 1e-5 * zmin) > 1
        if not near_tie:
            assert zw == zmin
        assert f["winner"] == ids[np.argmax(np.where(iz > 0, iz, -np.inf))]


@MODES
def test_intra_view_occlusion_only(decisions):
    """A near mesh in one view must not hide a far mesh of another view
    (Sec. 4.2.2): with equal disks the two colours average exactly."""
    G, n = 4, 32
    intr = scene.intrinsics_for_fov(n, n, 90.0)
    img = np.zeros((2, n, n, 4), dtype=np.uint8)
    img[0, ..., :3] = (200, 40, 10)
    img[1, ..., :3] = (20, 100, 240)
    img[..., 3] = 255
    depth = np.stack([np.full((G, G), 5.0), np.full((G, G), 1.0)]).astype(np.float32)
    lf = lfcase.custom_lf([_identity_pose(), _identity_pose()], [intr, intr], img, depth,
                          disk_c=[[0.0, 0.0, 0.3], [0.0, 0.0, 0.3]], disk_r=[0.5, 0.5], sphere_r=0.35)
    eye = scene.Eye(_identity_pose((0.01, 0.0, 0.0)), np.array([12.0, 12.0, 12.0, 12.0]), 24, 24)
    out = oracle.render(lf, eye, decisions=decisions)["rgba"]
    valid = out[..., 3] > 0
    assert valid.sum() > 300
    want = (np.array([200, 40, 10]) + np.array([20, 100, 240])) / 2.0 / 255.0
    assert np.max(np.abs(out[valid][:, :3] - want)) < 1e-12


# ---------------------------------------------------------------- Eq. 2 special cases


@MODES
def test_single_view_at_eye_reproduces_image(decisions):
    lf0 = scene.tiny_light_field(1)
    v = 5
    c = lf0.poses[v, 9:12]
    lf = lfcase.custom_lf(lf0.poses[v:v + 1], lf0.intr[v:v + 1], lf0.images[v:v + 1], lf0.depth[v:v + 1],
                          disk_c=lf0.disk_c[v:v + 1], disk_r=lf0.disk_r[v:v + 1],
                          sphere_r=float(np.linalg.norm(c)) + 1e-4)
    eye = scene.Eye(lf0.poses[v].copy(), lf0.intr[v].copy(), lf0.width, lf0.height)
    out = oracle.render(lf, eye, decisions=decisions)["rgba"]
    assert np.all(out[..., 3] == 1.0)
    src = lf0.images[v, ..., :3].astype(np.float64) / 255.0
    assert np.max(np.abs(out[..., :3] - src)) < 1e-9


@MODES
def test_single_view_identity_nonsquare_offcentre(decisions):
    """Same identity with W != H, fx != fy and an off-centre principal point,
    so a swapped axis anywhere in the camera model shows up."""
    prims = scene.sphere_scene(6, 8, forward_cone_deg=35.0)
    R = scene.look_rotation([0.1, -0.05, 1.0])
    c = 0.35 * np.array([0.1, -0.05, 1.0]) / np.linalg.norm([0.1, -0.05, 1.0])
    pose = scene.pose_array(R, c)
    intr = np.array([52.0, 44.0, 41.25, 36.5])
    rgba, grid, _ = scene.ray_cast(prims, pose[None], intr[None], 96, 64, grid_n=20)
    lf = lfcase.custom_lf(pose[None], intr[None], rgba, grid, disk_r=[0.1],
                          sphere_r=float(np.linalg.norm(c)) + 1e-4)
    eye = scene.Eye(pose.copy(), intr.copy(), 96, 64)
    out = oracle.render(lf, eye, decisions=decisions)["rgba"]
    assert np.all(out[..., 3] == 1.0)
    assert np.max(np.abs(out[..., :3] - rgba[0, ..., :3] / 255.0)) < 1e-9


@MODES
def test_planar_constant_colour_gives_constant_output(decisions):
    """Eq. 3 with a constant splat colour: a plane of constant radiance is
    reproduced exactly wherever some disk weight is positive."""
    prims = scene.plane_scene((0.0, 0.0, 3.0), (0.0, 0.0, 1.0), (0.4, 0.6, 0.2))
    lf = scene.build_light_field(prims, scene.cap_grid_directions(4, 40.0), 64, 64, 90.0, 16)
    assert np.all(lf.images[..., :3] == np.array([102, 153, 51], dtype=np.uint8))
    eye = scene.Eye(_identity_pose((0.02, -0.03, 0.05)), scene.intrinsics_for_fov(96, 96, 90.0), 96, 96)
    out = oracle.render(lf, eye, decisions=decisions)["rgba"]
    valid = out[..., 3] > 0
    assert valid.mean() > 0.3
    want = np.array([102, 153, 51]) / 255.0
    assert np.max(np.abs(out[valid][:, :3] - want)) < 1e-12


@MODES
def test_view_order_invariance(decisions):
    lf = scene.tiny_light_field(2)
    eye = lf.eyes[0]
    perm = np.random.default_rng(11).permutation(lf.n_views)
    lf2 = lfcase.custom_lf(lf.poses[perm], lf.intr[perm], lf.images[perm], lf.depth[perm],
                           disk_c=lf.disk_c[perm], disk_r=lf.disk_r[perm])
    a = oracle.render(lf, eye, fragments=True, decisions=decisions)
    b = oracle.render(lf2, eye, fragments=True, decisions=decisions)
    assert np.max(np.abs(a["rgba"] - b["rgba"])) < 1e-12
    ka = {(int(f["pixel"]), int(f["view"])): (f["n_cover"], f["winner"], f["id_hash"]) for f in a["frags"]}
    kb = {(int(f["pixel"]), int(perm[f["view"]])): (f["n_cover"], f["winner"], f["id_hash"]) for f in b["frags"]}
    assert ka == kb


# ---------------------------------------------------------------- disk weights


@MODES
def test_weights_closed_form(decisions):
    """Sphere of radius 1, eye at its centre looking down +z: the centre pixel's
    ray crosses at p = (0, 0, 1).  Disks at chord distance 0 and 0.25 with
    r = 0.5 give w = 1 and w = 0.5; a disk at chord 0.6 gives no term."""
    G, n = 2, 16
    intr = scene.intrinsics_for_fov(n, n, 90.0)
    img = np.full((3, n, n, 4), 255, dtype=np.uint8)
    depth = np.full((3, G, G), 3.0, dtype=np.float32)

    def on_sphere(chord):
        th = 2.0 * math.asin(chord / 2.0)
        return [0.0, math.sin(th), math.cos(th)]

    lf = lfcase.custom_lf([_identity_pose()] * 3, [intr] * 3, img, depth,
                          disk_c=[on_sphere(0.0), on_sphere(0.25), on_sphere(0.6)],
                          disk_r=[0.5, 0.5, 0.5], sphere_r=1.0)
    eye = scene.Eye(_identity_pose(), np.array([8.0, 8.0, 8.5, 8.5]), 17, 17)
    res = oracle.render(lf, eye, pixels=np.array([[8, 8]]), fragments=True, decisions=decisions)
    w = {int(f["view"]): float(f["w"]) for f in res["frags"]}
    assert set(w) == {0, 1}
    assert abs(w[0] - 1.0) < 1e-6 and abs(w[1] - 0.5) < 1e-6


@MODES
def test_weights_vanish_outside_disks(decisions):
    lf = scene.tiny_light_field(1)
    eye = lf.eyes[0]
    res = oracle.render(lf, eye, fragments=True, decisions=decisions)
    frags = res["frags"]
    assert len(frags) > 1000
    R = eye.pose[:9].reshape(3, 3)
    o = eye.pose[9:12]
    for f in frags[::97]:
        i, j = int(f["pixel"]) % eye.width, int(f["pixel"]) // eye.width
        e = np.array([(i + 0.5 - eye.intr[2]) / eye.intr[0], (j + 0.5 - eye.intr[3]) / eye.intr[1], 1.0])
        p = lfcase.sphere_crossing(o, R @ e, lf.sphere_c, lf.sphere_r)
        d = np.linalg.norm(p - lf.disk_c[f["view"]].astype(np.float64))
        r = float(lf.disk_r[f["view"]])
        assert d <= r * (1 + (1e-6 if decisions == "fp32" else 1e-12))
        assert abs(f["w"] - max(0.0, 1.0 - d / r)) < 1e-9


@MODES
def test_view_selection_matches_fp64_bruteforce(decisions):
    lf = scene.tiny_light_field(3)
    eye = lf.eyes[0]
    got = oracle.select_views(lf, eye, decisions=decisions)
    D = lfcase.pixel_rays(eye).reshape(-1, 3) @ eye.pose[:9].reshape(3, 3).T
    o = eye.pose[9:12] - lf.sphere_c
    a = np.sum(D * D, axis=1)
    b = D @ o
    c = o @ o - lf.sphere_r ** 2
    t = (-b + np.sqrt(b * b - a * c)) / a
    P = o + t[:, None] * D
    for v in range(lf.n_views):
        margin = np.min(np.linalg.norm(P - (lf.disk_c[v] - lf.sphere_c), axis=1)) - lf.disk_r[v]
        if abs(margin) > (1e-6 if decisions == "fp32" else 1e-12) * lf.disk_r[v]:
            assert got[v] == (margin < 0), v
    assert got.sum() >= 4


# ---------------------------------------------------------------- normalisation


@MODES
def test_normalisation_recomputed_from_records(decisions):
    """Eq. 2 recomputed from the per-view records with an independent bilinear
    sampler; each output channel lies in the convex hull of its samples."""
    lf = scene.tiny_light_field(1)
    eye = lf.eyes[0]
    res = oracle.render(lf, eye, fragments=True, decisions=decisions)
    out = res["rgba"].reshape(-1, 4)
    by_pix = {}
    for f in res["frags"]:
        by_pix.setdefault(int(f["pixel"]), []).append(f)
    rng = np.random.default_rng(0)
    pix = [p for p in by_pix if out[p, 3] > 0]
    for p in rng.choice(pix, size=200, replace=False):
        num, den, samples = np.zeros(3), 0.0, []
        for f in by_pix[p]:
            if f["winner"] < 0:
                continue
            smp = lfcase.bilinear(lf.images[f["view"]], f["s"], f["t"])
            samples.append(smp)
            num += f["w"] * smp
            den += f["w"]
        assert np.max(np.abs(num / den - out[p, :3])) < 1e-12
        S = np.array(samples)
        assert np.all(out[p, :3] >= S.min(axis=0) - 1e-12)
        assert np.all(out[p, :3] <= S.max(axis=0) + 1e-12)


# ---------------------------------------------------------------- convergence to the scene


def _psnr_vs_truth(lf, eye):
    out = oracle.render(lf, eye)["rgba"]
    truth = scene.truth_image(lf, eye)[..., :3] / 255.0
    valid = out[..., 3] > 0
    err = out[..., :3][valid] - truth[valid]
    return -10.0 * math.log10(float(np.mean(err ** 2))), valid.mean()


def test_reconstruction_approaches_analytic_scene():
    """With exact per-view depth, denser meshes and source pixels bring Eq. 2
    closer to the ray-cast scene (a trend, not parity)."""
    prims = scene.sphere_scene(4, 8, forward_cone_deg=35.0)
    dirs = scene.cap_grid_directions(4, 40.0)
    eye = scene.Eye(_identity_pose((0.03, -0.02, 0.05)), scene.intrinsics_for_fov(128, 128, 60.0), 128, 128)
    coarse = scene.build_light_field(prims, dirs, 96, 96, 90.0, 12)
    fine = scene.build_light_field(prims, dirs, 256, 256, 90.0, 64)
    p0, v0 = _psnr_vs_truth(coarse, eye)
    p1, v1 = _psnr_vs_truth(fine, eye)
    assert v0 > 0.5 and v1 > 0.5
    assert p0 > 18.0
    assert p1 > p0 + 1.0, (p0, p1)


# ---------------------------------------------------------------- the FP32 reading against the FP64 definition


def test_fp64_snap_is_the_rounded_fp64_projection():
    """In the FP64 mode every snapped vertex is llrint(256 (f x / z + c)) of
    the vertex taken to the eye through world coordinates, computed here
    independently in numpy (round half to even); only projections within 1e-6
    subpixel of a half are left out."""
    lf, eye = fold_case((-0.4, 0.45, 0.3))
    rows, _ = oracle.view_triangles(lf, eye, 0, decisions="fp64")
    V = lfcase.eye_vertices(lf, eye, 0)
    checked = 0
    for r in rows:
        idx = lfcase.triangle_vertex_index(lf.grid_n, r[0])
        P = np.array([V[k, j] for (k, j) in idx])
        if np.any(P[:, 2] < 0.1):
            continue  # clipped: its snapped points are clip points
        uv = lfcase.project(eye, P) * 256.0
        if np.any(np.abs(np.abs(uv - np.floor(uv)) - 0.5) < 1e-6):
            continue
        want = sorted(map(tuple, np.rint(uv).astype(np.int64).tolist()))
        got = sorted([(int(r[1]), int(r[2])), (int(r[3]), int(r[4])), (int(r[5]), int(r[6]))])
        assert got == want, (r[0], got, want)
        checked += 1
    assert checked > 200


def _records(res):
    return {(int(f["pixel"]), int(f["view"])): (int(f["n_cover"]), int(f["winner"]), int(f["min_id"]),
                                                int(f["max_id"]), int(f["id_hash"])) for f in res["frags"]}


# a (pixel, view) whose two modes differ must lie within FP32 rounding of one decision
# boundary: the disk rim (relative), a snapped edge (subpixels; a vertex moves by at most
# one subpixel between the modes), or a depth near-tie (relative)
DISK_MARGIN, EDGE_MARGIN, DEPTH_MARGIN = 1e-5, 2.0, 1e-4


def explained(m):
    return (np.abs(np.nan_to_num(m[:, 0], nan=1.0)) <= DISK_MARGIN) | (m[:, 1] <= EDGE_MARGIN) | \
        (m[:, 2] <= DEPTH_MARGIN)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fp32_reading_matches_the_definition_up_to_rounding(seed):
    """The FP32 reading (the decisions the CUDA path takes) against the FP64
    definition on full tiny frames: at most 1e-4 of the (pixel, view) records
    differ, every difference lies within FP32 rounding of a decision boundary,
    view selection agrees except for disks whose rim passes within 1e-5 r of
    a pixel's crossing, and colour agrees within 2e-3 where both are valid."""
    lf = scene.tiny_light_field(seed)
    eye = lf.eyes[0]
    a = oracle.render(lf, eye, fragments=True, decisions="fp32")
    b = oracle.render(lf, eye, fragments=True, decisions="fp64")
    ra, rb = _records(a), _records(b)
    keys = set(ra) | set(rb)
    diff = sorted(k for k in keys if ra.get(k) != rb.get(k))
    assert len(keys) > 30000
    assert len(diff) <= 1e-4 * len(keys), len(diff)
    if diff:
        pv = np.array([[p % eye.width, p // eye.width, v] for (p, v) in diff], dtype=np.int32)
        m = oracle.margins(lf, eye, pv)
        assert np.all(explained(m)), [(k, tuple(x)) for k, x, ok in zip(diff, m, explained(m)) if not ok]
    sa = oracle.select_views(lf, eye, decisions="fp32")
    sb = oracle.select_views(lf, eye, decisions="fp64")
    for v in np.nonzero(sa != sb)[0]:
        pv = np.array([[i, j, v] for j in range(eye.height) for i in range(eye.width)], dtype=np.int32)
        assert np.nanmin(np.abs(oracle.margins(lf, eye, pv)[:, 0])) <= DISK_MARGIN
    ca, cb = a["rgba"].reshape(-1, 4), b["rgba"].reshape(-1, 4)
    both = (ca[:, 3] > 0) & (cb[:, 3] > 0)
    assert np.max(np.abs(ca[both, :3] - cb[both, :3])) <= 2e-3
    odd = np.nonzero((ca[:, 3] > 0) != (cb[:, 3] > 0))[0]
    assert set(odd.tolist()) <= {p for (p, _) in diff}


def test_margins_are_zero_on_the_boundaries():
    """orc_margins against hand-placed boundaries: a pixel centre on a snapped
    edge of a fronto-parallel grid, a crossing on a disk rim, and two parents
    at one depth."""
    G, n = 3, 64
    rng = np.random.default_rng(2)
    depth = np.full((1, G, G), 2.0, dtype=np.float32)
    intr = np.array([32.0, 32.0, 32.0, 32.0])
    # sphere of radius 1 about the eye: the centre ray crosses at (0, 0, 1); a disk
    # centred at (0, 0.5, 1) with radius 0.5 (both exact in FP32) has that point on its rim
    lf = lfcase.custom_lf([_identity_pose()], [intr], _noise_image(rng, n, n)[None], depth,
                          disk_c=[[0.0, 0.5, 1.0]], disk_r=[0.5], sphere_r=1.0)
    # eye = the view: grid vertex column j = 1 sits at x = 32 px, so pixel centres
    # (31.5, y) lie half a pixel (128 subpixels) from the vertical edge, and the
    # centre pixel (32, 32) is 128 subpixels from the mesh's cell edges
    eye = scene.Eye(_identity_pose(), intr.copy(), 65, 65)
    m = oracle.margins(lf, eye, np.array([[31, 10, 0], [32, 32, 0]]))
    assert abs(m[0, 1] - 128.0) < 1e-9 and abs(m[1, 1] - 128.0) < 1e-9
    # the crossing of pixel (32, 32): ray (0.5/32, 0.5/32, 1); the rim pin uses the centre ray
    eye_c = scene.Eye(_identity_pose(), np.array([32.0, 32.0, 32.5, 32.5]), 65, 65)
    mc = oracle.margins(lf, eye_c, np.array([[32, 32, 0]]))
    assert abs(mc[0, 0]) < 1e-12
    assert mc[0, 2] == np.inf  # one parent covers the pixel
