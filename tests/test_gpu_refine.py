"""GPU parity of the learned refinement (lf_refine, lf_refine_gradients,
lf_refine_train_step, lf_render_refined) against the FP64 oracle in
oracle/refine.py, through the C ABI.

Tolerances.  The kernels use BF16 copies of the weights (the oracle is given
the same rounded weights) and BF16 layer inputs with FP32 accumulation; the
oracle propagates the variance of those roundings (forward_error_sigma) and
the forward outputs must lie within 8 sigma + 1e-5 of the FP64 result
everywhere.  Gradients pass through three more BF16 roundings per product
(the upstream gradient, the activation, the weight: relative RMS about
3 * 2^-8 / sqrt(3) ~ 0.5 %, plus the forward error carried into dL/dy), so
each parameter tensor's gradient must be within 5 % relative L2 of the
oracle's and point the same way (cosine > 0.998).  Adam is elementwise FP32
arithmetic on identical inputs: within FP32 rounding of the oracle."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import refine
import scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lfmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_08860_gb300 as m

    return m


def _params(lfmod, seed, out_scale=0.3, bias=0.05):
    p = lfmod.init_refiner_params(seed, out_scale=out_scale).astype(np.float64)
    rng = np.random.default_rng(seed + 1000)
    d = refine.unpack(p)
    for k in ("b1", "b2", "b3"):
        d[k] = rng.normal(0.0, bias, d[k].shape)
    return refine.pack(d).astype(np.float32)


def _bf16_weights(params):
    d = refine.unpack(params.astype(np.float64))
    return refine.pack({k: (refine.bf16_round(v) if k.startswith("W") else v) for k, v in d.items()})


def _smooth_image(rng, h, w, invalid=0.1):
    """Smooth colour field plus texture, with holes of alpha 0."""
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    img = np.zeros((h, w, 4))
    for c in range(3):
        fx, fy, ph = rng.uniform(0.02, 0.3), rng.uniform(0.02, 0.3), rng.uniform(0, 6.3)
        img[..., c] = 0.5 + 0.3 * np.sin(fx * xx + fy * yy + ph) + 0.1 * rng.uniform(-1, 1, (h, w))
    img[..., 3] = 1.0
    holes = rng.uniform(size=(h, w)) < invalid
    img[holes] = 0.0
    return img.astype(np.float32)


def _check_forward(got, imgs, params):
    pb = _bf16_weights(params)
    worst = 0.0
    for g, x in zip(got, imgs):
        f = refine.forward(x.astype(np.float64), pb)
        valid = x[..., 3] > 0
        assert np.array_equal(g[..., 3], valid.astype(np.float32))
        assert np.all(g[~valid] == 0.0)
        sigma = refine.forward_error_sigma(x.astype(np.float64), pb)
        err = np.abs(g[..., :3].astype(np.float64) - f["y"])[valid]
        tol = 8.0 * sigma[valid] + 1e-5
        assert np.all(err <= tol), (err.max(), (err / tol).max())
        worst = max(worst, float((err / tol).max()))
    return worst


@pytest.mark.parametrize("kernel", ["layers", "fused"])
def test_refine_matches_oracle_ragged_multi_tile(lfmod, kernel):
    import torch

    rng = np.random.default_rng(3)
    params = _params(lfmod, 3)
    r = lfmod.Renderer(0)
    r.load_refiner(params)
    r.set_refine_kernel(kernel)
    for (n, h, w) in [(2, 70, 100), (1, 9, 61), (1, 1, 1), (3, 31, 27)]:
        imgs = [_smooth_image(rng, h, w) for _ in range(n)]
        x = torch.from_numpy(np.stack(imgs)).cuda()
        y = r.refine(x).cpu().numpy()
        _check_forward(list(y), imgs, params)
    assert r.get_refiner()["step"] == 0  # also checks the fused kernel's error flag
    r.close()


def test_fused_wait_that_runs_out_reports_timeout_and_leaves_the_context_usable(lfmod):
    """Failure detection without hanging the GPU: with a 1 ns wait limit the
    first mbarrier wait of the fused kernel that is not already complete gives
    up (typically the MMA warps' wait for the first layer's input, before any
    MMA is issued).  The kernel must return, lf_get_refiner must report
    LF_ERR_TIMEOUT, and after restoring the default limit the same context must
    refine correctly (the issuers drain their MMAs before the tensor memory is
    freed, also on the abort path)."""
    import torch

    rng = np.random.default_rng(11)
    params = _params(lfmod, 5)
    imgs = [_smooth_image(rng, 90, 120) for _ in range(2)]
    x = torch.from_numpy(np.stack(imgs)).cuda()
    r = lfmod.Renderer(0)
    r.load_refiner(params)
    r.set_refine_kernel("fused")
    r.set_wait_limit(1)
    for _ in range(3):
        r.refine(x)
    torch.cuda.synchronize()
    with pytest.raises(lfmod.LFError) as info:
        r.get_refiner()
    assert info.value.status == 5  # LF_ERR_TIMEOUT
    with pytest.raises(lfmod.LFError):
        r.set_wait_limit(-1)
    r.set_wait_limit(0)  # back to the default bound
    r.load_refiner(params)  # clears the error flag with the Adam state
    y = r.refine(x).cpu().numpy()
    _check_forward(list(y), imgs, params)
    assert r.get_refiner()["step"] == 0
    r.close()


def test_refine_of_an_actual_render(lfmod):
    import torch

    lf = scene.tiny_light_field(1)
    eye = lf.eyes[0]
    r = lfmod.Renderer(0)
    r.load_views(lf)
    r.build_meshes(lf)
    img = r.render([eye])[0]
    params = _params(lfmod, 5)
    r.load_refiner(params)
    torch.cuda.synchronize()
    x = img.cpu().numpy()
    for kernel in ("layers", "fused"):
        r.set_refine_kernel(kernel)
        y = r.refine(img).cpu().numpy()
        _check_forward([y], [x], params)
        # lf_render_refined: the render then the refinement, same numbers
        yr = r.render_refined([eye])[0].cpu().numpy()
        assert np.array_equal(yr, y)
    r.get_refiner()
    r.close()


def test_render_refined_pairs_equal_per_eye_refinement(lfmod):
    # an equal-sized stereo pair is refined by one fused launch into the two
    # caller buffers (launched as a programmatic dependent of the raster); a
    # pair of different sizes by one launch per eye: both equal the refinement
    # of each eye's render on its own
    import torch

    lf = scene.tiny_light_field(1)
    base = lf.eyes[0]
    r = lfmod.Renderer(0, max_eyes=2)
    r.load_views(lf)
    r.build_meshes(lf)
    r.load_refiner(_params(lfmod, 11))
    r.set_refine_kernel("fused")
    other = scene.Eye(base.pose, np.array([70.0, 70.0, 41.0, 37.0]), base.width, base.height)
    small = scene.Eye(base.pose, np.array([60.0, 60.0, 33.0, 30.0]), 70, 61)
    for pair in ([base, other], [base, small]):
        got = [o.cpu() for o in r.render_refined(pair)]
        for eye, g in zip(pair, got):
            want = r.refine(r.render([eye])[0]).cpu()
            assert torch.equal(g, want), (eye.width, eye.height)
    r.get_refiner()  # raises if a wait of the fused kernel gave up
    r.close()


def test_refine_full_size_sampled(lfmod):
    # the stereo eye size of the rig workload, in the fused launch the bench times;
    # each sampled output depends only on the 7x7 window around it
    import torch

    rng = np.random.default_rng(7)
    params = _params(lfmod, 7)
    pb = _bf16_weights(params)
    imgs = [_smooth_image(rng, 1600, 1440, invalid=0.02) for _ in range(2)]
    r = lfmod.Renderer(0)
    r.load_refiner(params)
    r.set_refine_kernel("fused")
    y = r.refine(torch.from_numpy(np.stack(imgs)).cuda()).cpu().numpy()
    r.get_refiner()
    r.close()
    pts = [(0, 0), (0, 1439), (1599, 0), (1599, 1439), (29, 25), (30, 26), (31, 27)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, 1600, 600), rng.integers(0, 1440, 600))]
    for k, x in enumerate(imgs):
        for (py, px) in pts:
            y0, x0 = max(0, py - 3), max(0, px - 3)
            win = x[y0:py + 4, x0:px + 4].astype(np.float64)
            f = refine.forward(win, pb)
            s = refine.forward_error_sigma(win, pb)
            cy, cx = py - y0, px - x0
            if x[py, px, 3] > 0:
                err = np.abs(y[k, py, px, :3] - f["y"][cy, cx])
                assert np.all(err <= 8.0 * s[cy, cx] + 1e-5), (k, py, px, err)
                assert y[k, py, px, 3] == 1.0
            else:
                assert np.all(y[k, py, px] == 0.0)


def test_gradients_match_oracle(lfmod):
    import torch

    rng = np.random.default_rng(11)
    params = _params(lfmod, 11)
    inputs = [_smooth_image(rng, 40, 70, invalid=0.1) for _ in range(2)]
    targets = []
    for x in inputs:
        t = x.copy()
        t[..., :3] += 0.15 * np.sin(np.arange(70)[None, :, None] * 0.3 + np.arange(40)[:, None, None] * 0.2)
        t[rng.uniform(size=(40, 70)) < 0.05] = 0.0
        targets.append(t.astype(np.float32))
    r = lfmod.Renderer(0)
    r.load_refiner(params)
    r.refine_gradients(torch.from_numpy(np.stack(inputs)).cuda(), torch.from_numpy(np.stack(targets)).cuda())
    st = r.get_refiner()
    r.close()
    pb = _bf16_weights(params)
    loss, g = refine.loss_and_grad([x.astype(np.float64) for x in inputs],
                                   [t.astype(np.float64) for t in targets], pb)
    assert abs(st["loss"] - loss) <= 2e-2 * loss
    k = 0
    for name, shape in refine.SHAPES:
        n = int(np.prod(shape))
        a, b = st["grad"][k:k + n].astype(np.float64), g[k:k + n]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert rel < 5e-2 and cos > 0.998, (name, rel, cos)
        k += n


def test_no_valid_pixel_gives_zero_loss_and_gradient(lfmod):
    import torch

    rng = np.random.default_rng(12)
    params = _params(lfmod, 12)
    x = _smooth_image(rng, 16, 20, invalid=0.0)
    t = x.copy()
    t[..., 3] = 0.0
    r = lfmod.Renderer(0)
    r.load_refiner(params)
    r.refine_gradients(torch.from_numpy(x[None]).cuda(), torch.from_numpy(t[None]).cuda())
    st = r.get_refiner()
    assert st["loss"] == 0.0 and np.all(st["grad"] == 0.0)
    r.close()


def test_adam_step_matches_oracle(lfmod):
    import torch

    rng = np.random.default_rng(13)
    params = _params(lfmod, 13)
    x = _smooth_image(rng, 24, 33)
    t = _smooth_image(rng, 24, 33)
    r = lfmod.Renderer(0)
    r.load_refiner(params)
    lr = 1e-3
    xt, tt = torch.from_numpy(x[None]).cuda(), torch.from_numpy(t[None]).cuda()
    r.refine_train_step(xt, tt, lr)
    s1 = r.get_refiner()
    assert s1["step"] == 1
    p1, m1, v1 = refine.adam_step(params.astype(np.float64), s1["grad"], np.zeros(refine.N_PARAMS),
                                  np.zeros(refine.N_PARAMS), 1, lr)
    np.testing.assert_allclose(s1["m"], m1, rtol=1e-6, atol=1e-30)
    np.testing.assert_allclose(s1["v"], v1, rtol=1e-5, atol=1e-30)
    assert np.all(np.abs(s1["params"] - p1) <= 1e-6 * lr + 2e-7 * np.abs(params))
    # a second step continues from the device state
    r.refine_train_step(xt, tt, lr)
    s2 = r.get_refiner()
    p2, m2, v2 = refine.adam_step(s1["params"].astype(np.float64), s2["grad"], s1["m"], s1["v"], 2, lr)
    # m2 = 0.9 m1 + 0.1 g2 can cancel: FP32 rounding is relative to the terms
    terms = 0.9 * np.abs(s1["m"].astype(np.float64)) + 0.1 * np.abs(s2["grad"].astype(np.float64))
    assert np.all(np.abs(s2["m"] - m2) <= 4 * 2.0 ** -24 * terms + 1e-30)
    assert np.all(np.abs(s2["params"] - p2) <= 1e-5 * lr + 2e-7 * np.abs(s1["params"]))
    assert s2["step"] == 2
    r.close()


def test_refiner_state_errors(lfmod):
    import torch

    r = lfmod.Renderer(0)
    x = torch.zeros((1, 8, 8, 4), device="cuda")
    with pytest.raises(lfmod.LFError) as e:
        r.refine(x)
    assert e.value.status == 4  # LF_ERR_STATE: no refiner loaded
    r.load_refiner(_params(lfmod, 1))
    with pytest.raises(lfmod.LFError):
        r.refine(x, out=x)  # not in place
    bad = _params(lfmod, 1)
    bad[5] = np.nan
    with pytest.raises(lfmod.LFError):
        r.load_refiner(bad)
    r.close()


def test_render_refined_without_refiner_is_the_plain_render(lfmod):
    import torch

    lf = scene.tiny_light_field(2)
    r = lfmod.Renderer(0)
    r.load_views(lf)
    r.build_meshes(lf)
    a = r.render([lf.eyes[0]])[0].clone()
    b = r.render_refined([lf.eyes[0]])[0]
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    r.close()


def _supersampled(r, eye, s):
    """Render at s x s samples per pixel and box-filter (weighted by alpha)."""
    import torch

    big = scene.Eye(eye.pose, np.asarray(eye.intr, dtype=np.float64) * s, eye.width * s, eye.height * s)
    img = r.render([big])[0]
    pool = lambda t: torch.nn.functional.avg_pool2d(t.permute(2, 0, 1)[None], s)[0].permute(1, 2, 0)
    rgb, a = pool(img[..., :3] * img[..., 3:4]), pool(img[..., 3:4])
    out = torch.zeros((eye.height, eye.width, 4), device=img.device)
    ok = a[..., 0] > 0
    out[..., :3] = torch.where(ok[..., None], rgb / a.clamp_min(1e-12), torch.zeros_like(rgb))
    out[..., 3] = ok.float()
    return out.contiguous()


def _psnr(a, b):
    v = (a[..., 3] > 0) & (b[..., 3] > 0)
    d = (a[..., :3] - b[..., :3])[v].astype(np.float64)
    return 10.0 * np.log10(1.0 / np.mean(d * d))


def test_training_on_method_generated_pairs_gains_over_the_plain_render(lfmod):
    # fast: 4x4 views on the cap with 12x12 meshes; target: the same scene from
    # 8x8 views with 64x64 meshes, 2x2 supersampled (the method with a denser
    # light field, as the offline model of Sec. 5).  Train on 256 poses, evaluate
    # on 32 held-out poses against the plain fast render.
    import math

    import torch

    prims = scene.sphere_scene(1, 8, forward_cone_deg=35.0)
    fast = scene.build_light_field(prims, scene.cap_grid_directions(4, 40.0), 128, 128, 90.0, 12)
    dense = scene.build_light_field(prims, scene.cap_grid_directions(8, 40.0), 128, 128, 90.0, 64)
    rf = lfmod.Renderer(0)
    rf.load_views(fast)
    rf.build_meshes(fast)
    rd = lfmod.Renderer(0, tri_capacity=64 << 20)
    rd.load_views(dense)
    rd.build_meshes(dense)
    rng = scene.SplitMix64(4242)
    eyes = [scene.head_pose_eyes(rng, 128, 128, 90.0, yaw_range=(-math.radians(10), math.radians(10)),
                                 pitch_deg=10.0, stereo=False)[0] for _ in range(288)]
    X = torch.stack([rf.render([e])[0].clone() for e in eyes])
    T = torch.stack([_supersampled(rd, e, 2) for e in eyes])
    rd.close()
    rf.load_refiner(lfmod.init_refiner_params(1, out_scale=0.1))
    g = torch.Generator().manual_seed(0)
    losses = []
    for it in range(600):
        idx = torch.randint(0, 256, (8,), generator=g)
        rf.refine_train_step(X[idx].contiguous(), T[idx].contiguous(), 2e-3 if it < 420 else 4e-4)
        if it in (0, 599):
            losses.append(rf.get_refiner()["loss"])
    assert losses[1] < 0.8 * losses[0]
    Xt, Tt = X[256:].contiguous(), T[256:].contiguous()
    base = np.mean([_psnr(x, t) for x, t in zip(Xt.cpu().numpy(), Tt.cpu().numpy())])
    for kernel in ("layers", "fused"):
        rf.set_refine_kernel(kernel)
        Y = rf.refine(Xt).cpu().numpy()
        gain = np.mean([_psnr(y, t) for y, t in zip(Y, Tt.cpu().numpy())]) - base
        assert gain > 0.4, (kernel, base, gain)
    rf.get_refiner()
    rf.close()


def test_refinement_rejects_misaligned_images(lfmod):
    """The kernels read and write RGBA as 16-byte texels (the fused kernel's
    input through a TMA tensor map): an image 4 bytes off a 16-byte boundary is
    refused before any launch (LF_ERR_INVALID_ARG), for both kernels and for
    training, and the context keeps working."""
    import torch

    rng = np.random.default_rng(12)
    params = _params(lfmod, 6)
    img = _smooth_image(rng, 40, 52)
    flat = torch.zeros(img.size + 1, dtype=torch.float32, device="cuda")
    flat[1:] = torch.from_numpy(img.reshape(-1)).cuda()
    x = flat[1:].view(1, 40, 52, 4)  # 4 bytes past an aligned base
    assert x.data_ptr() % 16 == 4
    r = lfmod.Renderer(0)
    r.load_refiner(params)
    for kernel in ("fused", "layers"):
        r.set_refine_kernel(kernel)
        with pytest.raises(lfmod.LFError) as info:
            r.refine(x)
        assert info.value.status == 1  # LF_ERR_INVALID_ARG
        y = r.refine(x.clone()).cpu().numpy()
        _check_forward(list(y), [img], params)
    with pytest.raises(lfmod.LFError) as info:
        r.refine_train_step(x, x.clone(), 1e-3)
    assert info.value.status == 1
    assert r.get_refiner()["step"] == 0


def test_training_wait_that_runs_out_reports_timeout_and_leaves_the_context_usable(lfmod):
    """The tcgen05 training kernels bound their waits by the same limit: with
    1 ns a training step's first wait for a tile's MMAs gives up, the kernels
    return (the CTA drains its MMAs before freeing tensor memory), and
    lf_get_refiner reports LF_ERR_TIMEOUT; with the default limit restored
    the same context trains again."""
    import torch

    rng = np.random.default_rng(13)
    params = _params(lfmod, 7)
    x = torch.from_numpy(np.stack([_smooth_image(rng, 64, 80) for _ in range(2)])).cuda()
    t = x.clone()
    t[..., :3] = (t[..., :3] * 0.9 + 0.05).clamp(0, 1)
    r = lfmod.Renderer(0)
    r.load_refiner(params)
    r.set_wait_limit(1)
    r.refine_train_step(x, t, 1e-3)
    torch.cuda.synchronize()
    with pytest.raises(lfmod.LFError) as info:
        r.get_refiner()
    assert info.value.status == 5  # LF_ERR_TIMEOUT
    r.set_wait_limit(0)
    r.load_refiner(params)
    r.refine_train_step(x, t, 1e-3)
    st = r.get_refiner()
    assert st["step"] == 1 and np.isfinite(st["loss"]) and st["loss"] > 0
