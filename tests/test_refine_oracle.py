"""Pins of the refinement oracle (oracle/refine.py) against what mathematics
and independent libraries fix: scipy's 2-D correlation, closed-form shifts,
the adjoint identities of convolution, central finite differences of the
loss, Adam's closed form under a constant gradient, torch's BF16 rounding,
and planted mistakes that each pin must catch."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import refine

scipy_signal = pytest.importorskip("scipy.signal")


def _rand_params(rng, scale=1.0):
    p = {}
    for name, shape in refine.SHAPES:
        fan = 27.0 if name == "W1" else 288.0
        std = np.sqrt(2.0 / fan) if name.startswith("W") else 0.1
        p[name] = rng.normal(0.0, std * scale, shape)
    return refine.pack(p)


def _rand_image(rng, h, w, invalid_frac=0.15):
    img = np.zeros((h, w, 4))
    img[..., :3] = rng.uniform(0.0, 1.0, (h, w, 3))
    img[..., 3] = 1.0
    bad = rng.uniform(size=(h, w)) < invalid_frac
    img[bad] = 0.0
    return img


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(7, 5, 3))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    got = refine.conv3x3(a, W, b)
    want = np.zeros((7, 5, 4))
    for o in range(4):
        want[..., o] = b[o]
        for c in range(3):
            want[..., o] += scipy_signal.correlate2d(a[..., c], W[o, c], mode="same", boundary="fill")
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_conv_single_tap_is_a_shift():
    # W[o, c, 0, 0] = 1 reads a[y-1, x-1]: the image moves one pixel down-right, zeros enter
    rng = np.random.default_rng(2)
    a = rng.normal(size=(6, 9, 2))
    W = np.zeros((2, 2, 3, 3))
    W[0, 0, 0, 0] = 1.0
    W[1, 1, 2, 1] = 1.0  # reads a[y+1, x]: moves up one row
    out = refine.conv3x3(a, W, None)
    assert np.all(out[0, :, 0] == 0) and np.all(out[:, 0, 0] == 0)
    assert np.array_equal(out[1:, 1:, 0], a[:-1, :-1, 0])
    assert np.array_equal(out[:-1, :, 1], a[1:, :, 1]) and np.all(out[-1, :, 1] == 0)


def test_transpose_is_the_adjoint():
    rng = np.random.default_rng(3)
    a = rng.normal(size=(8, 6, 5))
    g = rng.normal(size=(8, 6, 7))
    W = rng.normal(size=(7, 5, 3, 3))
    lhs = np.sum(refine.conv3x3(a, W, None) * g)
    rhs = np.sum(a * refine.conv3x3_transpose(g, W))
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1.0)


def test_weight_grad_is_the_adjoint_in_w():
    rng = np.random.default_rng(4)
    a = rng.normal(size=(5, 9, 3))
    g = rng.normal(size=(5, 9, 4))
    D = rng.normal(size=(4, 3, 3, 3))
    lhs = np.sum(refine.conv3x3(a, D, None) * g)
    rhs = np.sum(refine.conv3x3_weight_grad(g, a) * D)
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1.0)


def test_zero_last_layer_is_the_identity_on_valid_pixels():
    rng = np.random.default_rng(5)
    p = refine.unpack(_rand_params(rng))
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    img = _rand_image(rng, 9, 11)
    out = refine.forward(img, p)["rgba"]
    valid = img[..., 3] > 0
    assert np.array_equal(out[valid, :3], img[valid, :3]) and np.all(out[valid, 3] == 1.0)
    assert np.all(out[~valid] == 0.0)


def test_translation_equivariance_in_the_interior():
    rng = np.random.default_rng(6)
    params = _rand_params(rng)
    img = _rand_image(rng, 20, 20, invalid_frac=0.0)
    out = refine.forward(img, params)["rgba"]
    sh = np.roll(img, (2, 3), axis=(0, 1))
    out_s = refine.forward(sh, params)["rgba"]
    # the receptive field is 7x7: compare away from the border and the wrapped band
    np.testing.assert_allclose(out_s[8:17, 9:17], out[6:15, 6:14], rtol=0, atol=1e-12)


def _fd_check(inputs, targets, params, idx, h=1e-6):
    loss, grad = refine.loss_and_grad(inputs, targets, params)
    fd = []
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd.append((refine.loss_and_grad(inputs, targets, pp)[0] - refine.loss_and_grad(inputs, targets, pm)[0])
                  / (2 * h))
    return loss, grad[idx], np.array(fd)


def _probe_indices(rng):
    sizes = [int(np.prod(s)) for _, s in refine.SHAPES]
    starts = np.cumsum([0] + sizes[:-1])
    idx = []
    for st, n in zip(starts, sizes):
        idx += list(st + rng.choice(n, size=min(n, 6), replace=False))
    return np.array(idx)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    params = _rand_params(rng, scale=1.5)
    inputs = [_rand_image(rng, 7, 6), _rand_image(rng, 7, 6)]
    targets = [_rand_image(rng, 7, 6, invalid_frac=0.1), _rand_image(rng, 7, 6, invalid_frac=0.1)]
    loss, g, fd = _fd_check(inputs, targets, params, _probe_indices(rng))
    assert loss > 0
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-8)


def test_loss_counts_only_pixels_valid_in_both():
    rng = np.random.default_rng(8)
    p = refine.unpack(_rand_params(rng))
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    x = _rand_image(rng, 4, 5, invalid_frac=0.0)
    t = x.copy()
    t[0, 0, :3] += 0.5          # differs at a valid pixel
    t[1, 1, 3] = 0.0            # invalid in the target: excluded
    t[1, 1, :3] += 100.0
    loss, _ = refine.loss_and_grad([x], [t], p)
    assert abs(loss - 3 * 0.25 / (3 * 19)) < 1e-15


def test_adam_closed_form_under_constant_gradient():
    # with a constant gradient the bias-corrected moments are g and g^2 exactly,
    # so each step moves every parameter by lr * g / (|g| + eps)
    rng = np.random.default_rng(9)
    theta0 = rng.normal(size=50)
    g = rng.normal(size=50)
    theta, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    lr = 1e-3
    for t in range(1, 8):
        theta, m, v = refine.adam_step(theta, g, m, v, t, lr)
    np.testing.assert_allclose(theta, theta0 - 7 * lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(10)
    vals = np.concatenate([rng.normal(size=1000).astype(np.float32),
                           np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, 2 ** -130], np.float32)])
    want = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(refine.bf16_round(vals), want)
    assert refine.bf16_round(np.float32(1 + 2 ** -8))[()] == 1.0        # tie to even (down)
    assert refine.bf16_round(np.float32(1 + 3 * 2 ** -8))[()] == 1 + 2 ** -6  # tie to even (up)


def _emulated_kernel_forward(img, params):
    """The arithmetic the bound describes: BF16 weights and layer inputs, FP32 sums."""
    p = refine.unpack(params)
    f32 = np.float32

    def conv(a, W, b):
        a16 = refine.bf16_round(a).astype(f32)
        W16 = refine.bf16_round(W).astype(f32)
        H, Wd, _ = a.shape
        pad = np.zeros((H + 2, Wd + 2, a.shape[2]), f32)
        pad[1:H + 1, 1:Wd + 1] = a16
        out = np.zeros((H, Wd, W.shape[0]), f32)
        for ky in range(3):
            for kx in range(3):
                out = out + (pad[ky:ky + H, kx:kx + Wd] @ W16[:, :, ky, kx].T).astype(f32)
        return out + b.astype(f32)

    x = img[..., :3].astype(f32)
    a1 = np.maximum(conv(x, p["W1"], p["b1"]), 0)
    a2 = np.maximum(conv(a1, p["W2"], p["b2"]), 0)
    return x + conv(a2, p["W3"], p["b3"])


def test_error_sigma_describes_the_emulated_kernel_arithmetic():
    # the emulated kernel (BF16 weights and layer inputs, FP32 sums) against the
    # FP64 forward on the same BF16 weights: within a few sigma everywhere, and
    # sigma is not a gross overestimate (the largest deviation reaches 1 sigma)
    rng = np.random.default_rng(11)
    p = refine.unpack(_rand_params(rng, scale=1.0))
    params = refine.pack({k: (refine.bf16_round(v) if k.startswith("W") else v) for k, v in p.items()})
    img = _rand_image(rng, 40, 36, invalid_frac=0.0)
    y = refine.forward(img, params)["y"]
    sigma = refine.forward_error_sigma(img, params)
    ratio = np.abs(_emulated_kernel_forward(img, params) - y) / (sigma + 1e-12)
    assert ratio.max() < 6.0 and ratio.max() > 1.0
    assert 0.3 < np.sqrt(np.mean(ratio ** 2)) < 1.5


# ---- planted mistakes: each must fail at least one of the pins above --------

def _mut_transpose_unflipped(g, W):
    H, Wd, _ = g.shape
    pad = np.zeros((H + 2, Wd + 2, g.shape[2]))
    pad[1:H + 1, 1:Wd + 1] = g
    out = np.zeros((H, Wd, W.shape[1]))
    for ky in range(3):
        for kx in range(3):
            out += pad[ky:ky + H, kx:kx + Wd] @ W[:, :, ky, kx]
    return out


def _mut_conv_transposed_taps(a, W, b):
    return refine.__dict__["_orig_conv"](a, np.ascontiguousarray(W.transpose(0, 1, 3, 2)), b)


@pytest.mark.parametrize("mutation", ["transpose_unflipped", "conv_taps_transposed", "no_relu_mask",
                                      "adam_no_bias_correction"])
def test_planted_mistakes_are_caught(monkeypatch, mutation):
    rng = np.random.default_rng(12)
    if mutation == "transpose_unflipped":
        monkeypatch.setattr(refine, "conv3x3_transpose", _mut_transpose_unflipped)
        with pytest.raises(AssertionError):
            test_transpose_is_the_adjoint()
        with pytest.raises(AssertionError):
            test_gradient_matches_central_differences()
    elif mutation == "conv_taps_transposed":
        monkeypatch.setitem(refine.__dict__, "_orig_conv", refine.conv3x3)
        monkeypatch.setattr(refine, "conv3x3", _mut_conv_transposed_taps)
        with pytest.raises(AssertionError):
            test_conv_matches_scipy_correlate()
    elif mutation == "no_relu_mask":
        orig = refine.forward

        def fwd(rgba, params):
            f = orig(rgba, params)
            f["z1"] = np.abs(f["z1"]) + 1.0  # every unit looks active to the backward pass
            return f

        monkeypatch.setattr(refine, "forward", fwd)
        with pytest.raises(AssertionError):
            test_gradient_matches_central_differences()
    elif mutation == "adam_no_bias_correction":
        def adam(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
            m = beta1 * m + (1 - beta1) * grad
            v = beta2 * v + (1 - beta2) * grad * grad
            return params - lr * m / (np.sqrt(v) + eps), m, v

        monkeypatch.setattr(refine, "adam_step", adam)
        with pytest.raises(AssertionError):
            test_adam_closed_form_under_constant_gradient()
    del rng
