"""Frames delivered to host memory (lf_render_host, lf_host_wait).

The host path renders with the same kernels as lf_render into device slots of
the context and copies them to the caller's host buffers on a copy stream, so
every delivered image must equal the device render of the same eye bit for
bit, and one of them is also checked against the FP64 oracle here.  Also:
more frames than slots (the call waits for the oldest), pageable buffers,
the refined form, error bits of an overflowing frame, and argument errors.
"""
import ctypes

import numpy as np
import pytest

import oracle
import scene

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


def _eyes(n, seed, w=96, h=64):
    rng = scene.SplitMix64(seed)
    return [scene.head_pose_eyes(rng, w, h, 90.0, yaw_range=(-0.2, 0.2), pitch_deg=8.0, stereo=True)
            for _ in range(n)]


def test_host_frames_equal_device_renders_and_the_oracle(lfmod, tiny):
    import torch

    r = lfmod.Renderer(0)
    r.load_views(tiny)
    r.build_meshes(tiny)
    pairs = [tiny.eyes[0:1]] + _eyes(6, 91)  # 7 frames of 1 and 2 eyes through 3 slots
    delivered = []
    for pair in pairs:
        frame, out = r.render_host(pair)
        delivered.append((frame, pair, out))
    assert [f for f, _, _ in delivered] == list(range(len(pairs)))
    assert r.host_wait() == 0
    for frame, pair, out in delivered:
        ref = [o.cpu() for o in r.render(pair)]
        for a, b in zip(out, ref):
            assert torch.equal(a, b), frame
    # the first frame against the FP64 oracle
    exp = oracle.render(tiny, tiny.eyes[0])["rgba"]
    got = delivered[0][2][0].numpy().astype(np.float64)
    assert np.array_equal(exp[..., 3] > 0, got[..., 3] > 0)
    valid = exp[..., 3] > 0
    assert valid.sum() > 0
    assert np.abs(exp[valid] - got[valid]).max() <= COLOUR_TOL
    r.close()


def test_pageable_buffers_and_waiting_on_one_frame(lfmod, tiny):
    import torch

    r = lfmod.Renderer(0)
    r.load_views(tiny)
    r.build_meshes(tiny)
    pairs = _eyes(4, 92)
    outs = []
    for pair in pairs:
        host = [torch.full((e.height, e.width, 4), -1.0) for e in pair]  # pageable
        frame, out = r.render_host(pair, out=host)
        assert out is host
        outs.append((frame, pair, host))
    assert r.host_wait(1) == 0  # frames 0 and 1
    for frame, pair, host in outs[:2]:
        ref = [o.cpu() for o in r.render(pair)]
        assert all(torch.equal(a, b) for a, b in zip(host, ref))
    r.host_wait()
    for frame, pair, host in outs[2:]:
        ref = [o.cpu() for o in r.render(pair)]
        assert all(torch.equal(a, b) for a, b in zip(host, ref))
    r.close()


def test_refined_host_frames_equal_render_refined(lfmod, tiny):
    import torch

    for kernel in ("fused", "layers"):
        r = lfmod.Renderer(0)
        r.load_views(tiny)
        r.build_meshes(tiny)
        r.load_refiner(lfmod.init_refiner_params(3, out_scale=0.5))
        r.set_refine_kernel(kernel)
        pairs = _eyes(4, 93, w=80, h=72)
        got = [r.render_host(pair, form="refined") for pair in pairs]
        r.host_wait()
        for (frame, out), pair in zip(got, pairs):
            ref = [o.cpu() for o in r.render_refined(pair)]
            plain = [o.cpu() for o in r.render(pair)]
            for a, b, p in zip(out, ref, plain):
                assert torch.equal(a, b), (kernel, frame)
                assert not torch.equal(a, p)  # the refinement changed something
        r.get_refiner()  # raises if a wait of the fused kernel gave up
        r.close()


def test_batch_form_equals_render_batch(lfmod, tiny):
    # the persistent raster launched without a graph, into host memory, against
    # the graph-replayed lf_render_batch of the same eyes (mixed sizes)
    import torch

    rng = scene.SplitMix64(94)
    sizes = [(96, 64), (40, 33), (128, 128), (17, 131), (64, 64)]
    eyes = [scene.head_pose_eyes(rng, w, h, 90.0, yaw_range=(-0.2, 0.2), pitch_deg=8.0, stereo=False)[0]
            for w, h in sizes]
    r = lfmod.Renderer(0, max_eyes=8)
    r.load_views(tiny)
    r.build_meshes(tiny)
    frames = [r.render_host(eyes, form="batch") for _ in range(2)]
    r.host_wait()
    ref = [o.cpu() for o in r.render_batch(eyes)]
    for frame, out in frames:
        for k, (a, b) in enumerate(zip(out, ref)):
            assert torch.equal(a, b), (frame, k)
    # a smaller batch afterwards does not shrink the persistent grid of later ones
    small = [r.render_host(eyes[:1], form="batch")]
    again = r.render_host(eyes, form="batch")
    r.host_wait()
    assert torch.equal(small[0][1][0], ref[0])
    assert all(torch.equal(a, b) for a, b in zip(again[1], ref))
    r.close()


def test_overflowing_frame_reports_capacity(lfmod, tiny):
    # a pool of one triangle record overflows: the set-up skips the excess and
    # the frame's error word reaches the host with the images
    r = lfmod.Renderer(0, tri_capacity=1)
    r.load_views(tiny)
    r.build_meshes(tiny)
    r.render_host(tiny.eyes[0:1])
    with pytest.raises(lfmod.LFError) as info:
        r.host_wait()
    assert info.value.status == 7  # LF_ERR_CAPACITY
    assert r.host_wait() == 0  # the bits were reported once
    r.close()


def test_host_argument_errors(lfmod, tiny):
    import torch

    r = lfmod.Renderer(0)
    with pytest.raises(lfmod.LFError) as info:  # nothing loaded
        r.render_host(tiny.eyes[0:1])
    assert info.value.status == 4  # LF_ERR_STATE
    r.load_views(tiny)
    r.build_meshes(tiny)
    with pytest.raises(lfmod.LFError) as info:
        r.host_wait(0)  # no frame issued yet
    assert info.value.status == 1
    assert r.host_wait() == 0
    eye = tiny.eyes[0]
    poses, intr = r._eye_arrays([eye])
    host = torch.empty((eye.height, eye.width, 4), dtype=torch.float32, pin_memory=True)
    ptrs = (ctypes.c_void_p * 1)(host.data_ptr())
    null = (ctypes.c_void_p * 1)(None)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    frame = ctypes.c_int64(-7)
    assert r.lib.lf_render_host(r.ctx, 1, poses, intr, ptrs, 3, ctypes.byref(frame), stream) == 1
    assert r.lib.lf_render_host(r.ctx, 1, poses, intr, null, 0, ctypes.byref(frame), stream) == 1
    assert r.lib.lf_render_host(r.ctx, 3, poses, intr, ptrs, 0, ctypes.byref(frame), stream) == 1
    assert frame.value == -7  # no frame was issued
    assert r.lib.lf_render_host(r.ctx, 1, poses, intr, ptrs, 0, None, stream) == 0  # frame number optional
    assert r.lib.lf_host_wait(r.ctx, 0, None) == 0
    assert r.lib.lf_host_wait(r.ctx, 1, None) == 1
    r.close()
