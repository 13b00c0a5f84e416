"""CPU oracle of the learned refinement: a 3-layer 3x3 convolutional residual
network applied to the normalised render, its MSE loss, its gradients and one
Adam step, all in FP64 with numpy.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): the tests, the smoke
check and the benchmark's CPU legs call it; the CUDA path never imports it.

What it stands in for.  Sec. 5 of Overbeck et al. (TOG 2018) improves the
real-time reconstruction L (Sec. 4, Eq. 2) by projecting a higher-quality
offline reconstruction (denser light field images, depth maps before
simplification) onto it, through the prefilter of Eq. 4-5.  Here a small
network learns that projection in image space instead: trained on pairs of
(fast render, render of a denser light field of the same scene), it maps a
normalised render x to

    y = x + f(x),   f = conv3x3(3->32) . ReLU . conv3x3(32->32) . ReLU . conv3x3(32->3)

with zero padding at the image border.  Pixels with no view weight (alpha 0)
stay (0,0,0,0).

Parameters, in the order of the flat FP32 vector the library takes:
    W1[32][3][3][3], b1[32], W2[32][32][3][3], b2[32], W3[3][32][3][3], b3[3]
where W[o][c][ky][kx] multiplies input channel c at offset (ky-1, kx-1).

Convolutions are written as a sum over the nine taps of a matrix product (the
library matmul is the only primitive); the backward pass is the chain rule
written out layer by layer; Adam is Kingma & Ba (ICLR 2015), Algorithm 1.
"""
from __future__ import annotations

import numpy as np

C_IN, C_HID, C_OUT = 3, 32, 3
SHAPES = [("W1", (C_HID, C_IN, 3, 3)), ("b1", (C_HID,)), ("W2", (C_HID, C_HID, 3, 3)), ("b2", (C_HID,)),
          ("W3", (C_OUT, C_HID, 3, 3)), ("b3", (C_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 11,011


def unpack(flat) -> dict:
    """Flat parameter vector -> dict of FP64 arrays."""
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.shape == (N_PARAMS,), flat.shape
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[k:k + n].reshape(shape)
        k += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def conv3x3(a: np.ndarray, W: np.ndarray, b: np.ndarray | None) -> np.ndarray:
    """out[y, x, o] = b[o] + sum_{c, ky, kx} W[o, c, ky, kx] * a[y+ky-1, x+kx-1, c],
    with a = 0 outside the image.  a: (H, W, C), W: (O, C, 3, 3) -> (H, W, O)."""
    H, Wd, _ = a.shape
    pad = np.zeros((H + 2, Wd + 2, a.shape[2]), dtype=np.float64)
    pad[1:H + 1, 1:Wd + 1] = a
    out = np.zeros((H, Wd, W.shape[0]), dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            out += pad[ky:ky + H, kx:kx + Wd] @ W[:, :, ky, kx].T
    if b is not None:
        out += b
    return out


def conv3x3_transpose(g: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 in its input: ga[y, x, c] = sum_{o, ky, kx}
    W[o, c, ky, kx] * g[y-ky+1, x-kx+1, o], with g = 0 outside the image."""
    H, Wd, _ = g.shape
    pad = np.zeros((H + 2, Wd + 2, g.shape[2]), dtype=np.float64)
    pad[1:H + 1, 1:Wd + 1] = g
    out = np.zeros((H, Wd, W.shape[1]), dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            # output pixel y receives g at y - (ky - 1): rows 2-ky .. 2-ky+H of the padded array
            out += pad[2 - ky:2 - ky + H, 2 - kx:2 - kx + Wd] @ W[:, :, ky, kx]
    return out


def conv3x3_weight_grad(g: np.ndarray, a: np.ndarray) -> np.ndarray:
    """dW[o, c, ky, kx] = sum_{y, x} g[y, x, o] * a[y+ky-1, x+kx-1, c] (a = 0 outside)."""
    H, Wd, _ = a.shape
    pad = np.zeros((H + 2, Wd + 2, a.shape[2]), dtype=np.float64)
    pad[1:H + 1, 1:Wd + 1] = a
    out = np.zeros((g.shape[2], a.shape[2], 3, 3), dtype=np.float64)
    G = g.reshape(-1, g.shape[2])
    for ky in range(3):
        for kx in range(3):
            out[:, :, ky, kx] = G.T @ pad[ky:ky + H, kx:kx + Wd].reshape(-1, a.shape[2])
    return out


def forward(rgba: np.ndarray, params) -> dict:
    """Refine one normalised render (H, W, 4).  Returns the refined RGBA and
    the intermediate values the backward pass needs."""
    p = params if isinstance(params, dict) else unpack(params)
    x = np.asarray(rgba, dtype=np.float64)[..., :3]
    valid = np.asarray(rgba)[..., 3] > 0
    z1 = conv3x3(x, p["W1"], p["b1"])
    a1 = np.maximum(z1, 0.0)
    z2 = conv3x3(a1, p["W2"], p["b2"])
    a2 = np.maximum(z2, 0.0)
    r = conv3x3(a2, p["W3"], p["b3"])
    y = x + r
    out = np.zeros(np.asarray(rgba).shape, dtype=np.float64)
    out[valid, :3] = y[valid]
    out[valid, 3] = 1.0
    return {"rgba": out, "x": x, "valid": valid, "z1": z1, "a1": a1, "z2": z2, "a2": a2, "r": r, "y": y}


def loss_and_grad(inputs, targets, params) -> tuple[float, np.ndarray]:
    """Mean squared error over the RGB channels of the pixels valid in both
    the input and the target, summed over a batch of images of one size, and
    its gradient with respect to the flat parameter vector."""
    p = params if isinstance(params, dict) else unpack(params)
    fw = [forward(x, p) for x in inputs]
    masks = [f["valid"] & (np.asarray(t)[..., 3] > 0) for f, t in zip(fw, targets)]
    n = sum(int(m.sum()) for m in masks)
    if n == 0:
        return 0.0, np.zeros(N_PARAMS)
    scale = 1.0 / (3.0 * n)
    loss = 0.0
    grads = {name: np.zeros(shape) for name, shape in SHAPES}
    for f, t, m in zip(fw, targets, masks):
        d = (f["y"] - np.asarray(t, dtype=np.float64)[..., :3]) * m[..., None]
        loss += float(np.sum(d * d)) * scale
        gr = 2.0 * scale * d                                  # dL/dr = dL/dy (y = x + r)
        grads["W3"] += conv3x3_weight_grad(gr, f["a2"])
        grads["b3"] += gr.sum(axis=(0, 1))
        gz2 = conv3x3_transpose(gr, p["W3"]) * (f["z2"] > 0)  # through ReLU
        grads["W2"] += conv3x3_weight_grad(gz2, f["a1"])
        grads["b2"] += gz2.sum(axis=(0, 1))
        gz1 = conv3x3_transpose(gz2, p["W2"]) * (f["z1"] > 0)
        grads["W1"] += conv3x3_weight_grad(gz1, f["x"])
        grads["b1"] += gz1.sum(axis=(0, 1))
    return loss, pack(grads)


def adam_step(params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at 1-based step `step`.
    Returns (params, m, v)."""
    params, grad = np.asarray(params, np.float64), np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return params - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def bf16_round(a) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_error_sigma(rgba: np.ndarray, params, u: float = 2.0 ** -8) -> np.ndarray:
    """Standard deviation of y_kernel - y (RGB), per element, for a kernel that
    uses the same BF16 weights as `params` (round them with bf16_round first),
    rounds every layer input (x, a1, a2) to BF16 (unit roundoff u) and
    accumulates in FP32.

    Probabilistic rounding-error analysis (Higham & Mary, SIAM J. Sci. Comput.
    41(5), 2019): each rounding is an independent relative error of variance
    u^2/3 (uniform on [-u, u]); for z = sum_i w_i a_i the variance carried to z
    is sum_i w_i^2 (V_i + a_i^2 u^2 / 3), with V_i the variance already on a_i;
    ReLU passes the variance where z > 0.  FP32 accumulation adds terms below
    2^-24 relative, negligible here.  A worst-case bound grows by sum |w|
    (about 20) per layer and says nothing useful at this depth."""
    p = params if isinstance(params, dict) else unpack(params)
    f = forward(rgba, p)
    q = u * u / 3.0

    def layer(a, V, W):
        W2 = W * W
        return conv3x3(V, W2, None) + q * conv3x3(a * a, W2, None)

    V1 = layer(f["x"], np.zeros_like(f["x"]), p["W1"]) * (f["z1"] > 0)
    V2 = layer(f["a1"], V1, p["W2"]) * (f["z2"] > 0)
    V3 = layer(f["a2"], V2, p["W3"])
    return np.sqrt(V3)
