"""The allocation-free entry point, lf_render_static, against lf_render.

lf_render_static exists for callers that cannot call cudaMalloc while they
render (a frame loop with a hard deadline, a process whose device memory is
reserved up front by another allocator, a plug-in that may not allocate): it
takes its per-call scratch from a static device array instead of growing
buffers.  This file is collected last so that a run stopping at the first
failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

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


def _call_static(lfmod, r, eye, out):
    """lf_render_static through the C ABI, on the current stream."""
    import torch

    poses = lfmod._poses([eye.pose])
    intr = lfmod._intrinsics([eye.intr], [(eye.width, eye.height)])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return r.lib.lf_render_static(r.ctx, poses, intr, ctypes.c_void_p(out.data_ptr()), stream)


def _check_static(lfmod, r, eye, field=None):
    """Two lf_render_static calls in a row equal lf_render bit for bit (the same
    kernels on the same views); with `field`, colour and valid mask also match
    the CPU oracle."""
    import torch

    import oracle

    ref = r.render([eye])[0].clone()
    torch.cuda.synchronize()
    valid = ref[..., 3] > 0
    assert int(valid.sum()) > 0
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        out = torch.full_like(ref, -1.0)
        assert _call_static(lfmod, r, eye, out) == lfmod.LF_OK, r.lib.lf_last_error(r.ctx)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    if field is not None:
        want = oracle.render(field, eye)["rgba"]
        img = out.cpu().numpy().astype(np.float64)
        ok = want[..., 3] > 0
        assert np.array_equal(img[..., 3] > 0, ok)
        assert float(np.max(np.abs(img[ok][:, :3] - want[ok][:, :3]))) <= COLOUR_TOL


def test_static_scratch_render_matches_lf_render(lfmod):
    field = scene.tiny_light_field(1)
    r = lfmod.Renderer(0)
    r.load_views(field)
    r.build_meshes(field)
    for eye in [field.eyes[0], scene.Eye(field.eyes[0].pose, np.array([60.0, 55.0, 47.5, 40.25]), 97, 83)]:
        _check_static(lfmod, r, eye, field)
    r.close()


def test_static_scratch_big_triangles(lfmod):
    """A zoomed eye (f = 1200 on 256 x 256): a mesh cell spans about 75
    pixels, so many triangles cover more than the 16 screen tiles a
    static-scratch bin takes per triangle and go to their view's list of big
    triangles, which every tile of the view scans, beside binned ones."""
    import oracle

    field = scene.tiny_light_field(1)
    eye = scene.Eye(field.eyes[0].pose, np.array([1200.0, 1200.0, 128.0, 128.0]), 256, 256)
    spans = []
    for v in np.nonzero(oracle.select_views(field, eye))[0]:
        rows, _ = oracle.view_triangles(field, eye, int(v))
        X, Y = rows[:, 1::2], rows[:, 2::2]
        x0, x1 = np.clip(X.min(1) // 4096, 0, 15), np.clip(X.max(1) // 4096, 0, 15)  # 16-pixel tiles
        y0, y1 = np.clip(Y.min(1) // 4096, 0, 15), np.clip(Y.max(1) // 4096, 0, 15)
        on = (X.max(1) >= 0) & (X.min(1) < 256 * 256) & (Y.max(1) >= 0) & (Y.min(1) < 256 * 256)
        spans.append(((x1 - x0 + 1) * (y1 - y0 + 1))[on])
    spans = np.concatenate(spans)
    assert (spans > 16).sum() > 30 and (spans <= 16).sum() > 30  # both paths are taken
    r = lfmod.Renderer(0)
    r.load_views(field)
    r.build_meshes(field)
    _check_static(lfmod, r, eye, field)
    r.close()


def test_static_scratch_at_its_tile_limit(lfmod):
    """An eye of exactly 8,192 screen tiles (1024 x 2048 with 16 x 16 tiles)
    renders; one more row of tiles is refused."""
    import torch

    field = scene.tiny_light_field(1)
    r = lfmod.Renderer(0)
    r.load_views(field)
    r.build_meshes(field)
    eye = scene.Eye(field.eyes[0].pose, np.array([512.0, 512.0, 512.0, 1024.0]), 1024, 2048)
    _check_static(lfmod, r, eye)
    over = scene.Eye(field.eyes[0].pose, np.array([512.0, 512.0, 512.0, 1024.0]), 1024, 2049)
    out = torch.empty((2049, 1024, 4), dtype=torch.float32, device="cuda")
    assert _call_static(lfmod, r, over, out) == 7  # LF_ERR_CAPACITY
    assert b"8192" in r.lib.lf_last_error(r.ctx)
    r.close()


def test_static_scratch_rejects_sizes_beyond_its_limits(lfmod):
    import torch

    field = scene.tiny_light_field(1)
    r = lfmod.Renderer(0)
    r.load_views(field)
    r.build_meshes(field)
    big = scene.Eye(field.eyes[0].pose, np.array([1500.0, 1500.0, 1500.0, 1500.0]), 3000, 3000)
    out = torch.empty((3000, 3000, 4), dtype=torch.float32, device="cuda")
    assert _call_static(lfmod, r, big, out) == 7  # LF_ERR_CAPACITY
    assert b"8192" in r.lib.lf_last_error(r.ctx)
    r.close()
    # more views than the static scratch holds
    n = 33
    rng = np.random.default_rng(1)
    poses = np.stack([scene.pose_array(np.eye(3), (0.0, 0.0, 0.01 * k)) for k in range(n)])
    intr = np.tile(scene.intrinsics_for_fov(8, 8, 90.0), (n, 1))
    imgs = rng.integers(0, 256, size=(n, 8, 8, 4), dtype=np.uint8)
    depth = np.full((n, 4, 4), 2.0, dtype=np.float32)
    many = lfcase.custom_lf(poses, intr, imgs, depth, disk_r=np.full(n, 0.05))
    r = lfmod.Renderer(0)
    r.load_views(many)
    r.build_meshes(many)
    small = scene.Eye(scene.pose_array(np.eye(3), (0.0, 0.0, 0.0)), np.array([8.0, 8.0, 8.0, 8.0]), 16, 16)
    out = torch.empty((16, 16, 4), dtype=torch.float32, device="cuda")
    assert _call_static(lfmod, r, small, out) == 7
    assert b"32 views" in r.lib.lf_last_error(r.ctx)
    r.close()
