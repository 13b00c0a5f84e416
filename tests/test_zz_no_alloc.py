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


def test_static_scratch_render_matches_lf_render(lfmod):
    import torch

    field = scene.tiny_light_field(1)
    r = lfmod.Renderer(0)
    r.load_views(field)
    r.build_meshes(field)
    eyes = [field.eyes[0], scene.Eye(field.eyes[0].pose, np.array([60.0, 55.0, 47.5, 40.25]), 97, 83)]
    for eye in eyes:
        ref = r.render([eye])[0].clone()
        torch.cuda.synchronize()
        valid = ref[..., 3] > 0
        assert int(valid.sum()) > 0
        for _ in range(2):  # two calls in a row share (and reuse) the static scratch
            out = torch.full_like(ref, -1.0)
            assert _call_static(lfmod, r, eye, out) == lfmod.LF_OK, r.lib.lf_last_error(r.ctx)
            torch.cuda.synchronize()
            assert torch.equal(out[..., 3] > 0, valid)
            assert float((out - ref).abs().max()) <= COLOUR_TOL
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
