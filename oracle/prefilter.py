"""FP64 oracle of the light field prefilter (Sec. 5, Eq. 4-5).

TEST INFRASTRUCTURE ONLY: the test suite and the benchmark's CPU-baseline leg
are the only callers; the CUDA library never imports this module.

For light field image i of the real-time model and its pixel (s', t'), Eq. 4
integrates rho_i(u, v) sigma(s, t) Lbar(o, e) over the disk D_i (the ray
origin o) and the support of the pixel basis function sigma around (s', t');
the ray leaves o toward the point where the image point (s, t) lands on view
i's own triangle mesh, and Lbar is the light field ray query of a denser,
higher-quality model.  Eq. 5 estimates the integral with J samples:

    I'_i(s', t') = sum_j rho_j sigma_j Lbar_j / sum_j rho_j sigma_j.

Readings where the paper leaves a choice (each stated once here):
- sigma is the separable Lanczos-2 kernel (the kernel Sec. 5.1 settles on),
  sigma(ds, dt) = L2(ds) L2(dt), L2(x) = sinc(x) sinc(x / 2) for |x| < 2; rho is
  the linear disk kernel of Eq. 2, 1 - (chord distance) / r_i.
- The J samples are inputs, shared by every pixel of every view: sample j is
  (a_j, b_j, ds_j, dt_j) with a, b in [0, 1) and ds, dt in [-2, 2).  Its
  aperture point lies on the capture sphere at chord distance r_i sqrt(a_j)
  from view i's disk centre (projected radially onto the sphere), at angle
  2 pi b_j from view i's image x axis in the tangent plane.  A spherical cap's
  area is pi times its chord radius squared, so uniform a gives points uniform
  in area.  rho_j = 1 - sqrt(a_j).  The point is pulled 1e-5 R toward the
  sphere centre so that rays leaving it outward cross the sphere at t > 0 in
  FP32 as well (the renderer keeps crossings with t >= 0 only).
- All rays of one (view, sample) leave the same point o_j, so Lbar for them is
  a pinhole render at o_j with view i's rotation and intrinsics (scaled by the
  integer `supersample`) through the dense model with the method itself (as
  Sec. 5.1 does: denser images, unsimplified depth maps).  The ray toward the
  mesh point X(s, t) reads that render by bilinear interpolation at X's
  projection (texel centres, clamp to edge), on colour premultiplied by the
  render's alpha so that pixels no dense view covers carry no weight: the
  numerator sums rho sigma (alpha rgb)(q), the denominator rho sigma alpha(q).
- (s, t) = (s' + ds, t' + dt), clamped to the image rectangle [0, W] x [0, H]
  that the mesh spans; X is the intersection of view i's camera ray through
  (s, t) with the grid triangle holding (s, t) (the cell's diagonal runs from
  (j+1, k) to (j, k+1), as in the renderer).
- Output: (num / den, 1) where den > 0, else (0, 0, 0, 0); no clamping.
- Two ways to take Lbar (`lbar=`):
    "render"  the reading above: one pinhole render per (view, sample), read
              bilinearly at each mesh point's projection (the fast renderer's
              design; the resampling is its one approximation);
    "ray"     the definition: each ray from o_j through X(s, t) is its own
              query - a 1 x 1 eye at o_j with view i's rotation whose pixel
              centre ray passes exactly through X, at 8 x the view's focal
              length (the method's 1/256-pixel raster grid then lies 1/2048 of
              a source pixel apart) - weighted by that query's alpha.
"""
from __future__ import annotations

import math

import numpy as np

APERTURE_INSET = 1e-5  # fraction of R by which aperture points sit inside the sphere


def lanczos2(x):
    """L2(x) = sinc(x) sinc(x/2) for |x| < 2, else 0; sinc(x) = sin(pi x)/(pi x)."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(np.abs(x) < 2.0, np.sinc(x) * np.sinc(x / 2.0), 0.0)


def sample_weight(sample) -> float:
    """rho_j sigma_j of one sample (a, b, ds, dt)."""
    a, _, ds, dt = (float(v) for v in sample)
    return (1.0 - math.sqrt(a)) * float(lanczos2(ds)) * float(lanczos2(dt))


def _view_R_t(lf, view: int):
    P = np.asarray(lf.poses[view], dtype=np.float64)
    return P[:9].reshape(3, 3), P[9:12]


def aperture_point(lf, view: int, a: float, b: float) -> np.ndarray:
    """World position of the aperture sample (a, b) on view `view`'s disk."""
    C = np.asarray(lf.sphere_c, dtype=np.float64)
    R = float(lf.sphere_r)
    c = np.asarray(lf.disk_c[view], dtype=np.float64)
    n = (c - C) / np.linalg.norm(c - C)                  # radial direction of the disk centre
    Rv, _ = _view_R_t(lf, view)
    x = Rv[:, 0] - (Rv[:, 0] @ n) * n                    # image x axis in the tangent plane
    x /= np.linalg.norm(x)
    y = np.cross(n, x)
    chord = float(lf.disk_r[view]) * math.sqrt(a)
    theta = 2.0 * math.asin(min(1.0, chord / (2.0 * R)))  # chord 2 R sin(theta / 2)
    phi = 2.0 * math.pi * b
    d = math.cos(theta) * n + math.sin(theta) * (math.cos(phi) * x + math.sin(phi) * y)
    return C + (1.0 - APERTURE_INSET) * R * d


def virtual_intrinsics(lf, view: int, supersample: int):
    """(fx, fy, cx, cy), width, height of the render for view `view`."""
    fx, fy, cx, cy = (float(v) for v in lf.intr[view])
    S = int(supersample)
    return np.array([S * fx, S * fy, S * cx, S * cy]), S * lf.width, S * lf.height


def mesh_points(lf, view: int, s, t) -> np.ndarray:
    """Camera-frame points of view `view`'s mesh at image points (s, t) (arrays)."""
    W, H, G = lf.width, lf.height, lf.grid_n
    fx, fy, cx, cy = (float(v) for v in lf.intr[view])
    z = np.asarray(lf.depth[view], dtype=np.float64)     # [k][j]
    s = np.clip(np.asarray(s, dtype=np.float64), 0.0, W)
    t = np.clip(np.asarray(t, dtype=np.float64), 0.0, H)
    gs, gt = s * (G - 1) / W, t * (G - 1) / H
    j = np.clip(np.floor(gs).astype(np.int64), 0, G - 2)
    k = np.clip(np.floor(gt).astype(np.int64), 0, G - 2)
    upper = (gs - j) + (gt - k) > 1.0                    # the half beyond the diagonal

    def vertex(jj, kk):
        sj, tk = jj * W / (G - 1), kk * H / (G - 1)
        zz = z[kk, jj]
        return np.stack([zz * (sj - cx) / fx, zz * (tk - cy) / fy, zz], axis=-1)

    v00, v10, v01, v11 = vertex(j, k), vertex(j + 1, k), vertex(j, k + 1), vertex(j + 1, k + 1)
    a0 = np.where(upper[..., None], v10, v00)
    a1 = np.where(upper[..., None], v11, v10)
    a2 = v01
    n = np.cross(a1 - a0, a2 - a0)
    e = np.stack([(s - cx) / fx, (t - cy) / fy, np.ones_like(s)], axis=-1)
    zz = np.sum(n * a0, axis=-1) / np.sum(n * e, axis=-1)
    return zz[..., None] * e


def _bilinear_premultiplied(img, u, v):
    """Bilinear at (u, v) = (x - 1/2, y - 1/2) on texel centres, clamp to edge,
    of (alpha * rgb, alpha)."""
    Hs, Ws = img.shape[:2]
    pm = np.concatenate([img[..., :3] * img[..., 3:4], img[..., 3:4]], axis=-1)
    i0 = np.floor(u).astype(np.int64)
    j0 = np.floor(v).astype(np.int64)
    al, be = u - i0, v - j0
    ia, ib = np.clip(i0, 0, Ws - 1), np.clip(i0 + 1, 0, Ws - 1)
    ja, jb = np.clip(j0, 0, Hs - 1), np.clip(j0 + 1, 0, Hs - 1)
    return ((1 - al)[..., None] * (1 - be)[..., None] * pm[ja, ia] + al[..., None] * (1 - be)[..., None] * pm[ja, ib]
            + (1 - al)[..., None] * be[..., None] * pm[jb, ia] + al[..., None] * be[..., None] * pm[jb, ib])


def _per_ray(target, dense, view: int, smp, X):
    """(alpha rgb, alpha) of the method's ray query for each ray from the
    sample's aperture point through the camera-frame points X (K x 3)."""
    import oracle
    import scene

    Rv, tv = _view_R_t(target, view)
    ow = aperture_point(target, view, smp[0], smp[1])
    o = Rv.T @ (ow - tv)
    f = 8.0 * float(target.intr[view][0])
    out = np.zeros((X.shape[0], 4))
    for q in range(X.shape[0]):
        x = X[q] - o
        if not x[2] > 0.0:
            continue
        K = np.array([f, f, 0.5 - f * x[0] / x[2], 0.5 - f * x[1] / x[2]])
        v = oracle.render(dense, scene.Eye(scene.pose_array(Rv, ow), K, 1, 1), threads=1)["rgba"].reshape(4)
        out[q, :3] = v[:3] * v[3]
        out[q, 3] = v[3]
    return out


def prefilter(target, dense, view: int, samples, supersample: int = 1, pixels=None, threads=None,
              renders=None, details: bool = False, sparse: bool = False, lbar: str = "render"):
    """Eq. 5 for view `view` of the real-time model `target`, with Lbar from
    the light field `dense`.  samples: J x 4 (a, b, ds, dt).  pixels: K x 2
    integer (i, j), or None for the whole image.  Returns H x W x 4 (or K x 4)
    FP64.  `renders` may pass the J renders (from virtual_renders) in.  With
    details, returns a dict that also holds the denominator and the sum of
    |rho sigma| alpha (the error magnification of the ratio).  With sparse,
    each render is evaluated only at the texels the pixels' bilinear reads
    touch (the same values, for a few pixels of a large view)."""
    samples = np.asarray(samples, dtype=np.float64).reshape(-1, 4)
    W, H = target.width, target.height
    if pixels is None:
        jj, ii = np.mgrid[0:H, 0:W]
        pix = np.stack([ii.ravel(), jj.ravel()], axis=1)
    else:
        pix = np.asarray(pixels, dtype=np.int64).reshape(-1, 2)
    Rv, tv = _view_R_t(target, view)
    if lbar not in ("render", "ray"):
        raise ValueError("lbar must be 'render' or 'ray'")
    if renders is None and not sparse and lbar == "render":
        renders = virtual_renders(target, dense, view, samples, supersample, threads)
    Ks, Ws, Hs = virtual_intrinsics(target, view, supersample)
    num = np.zeros((pix.shape[0], 3))
    den = np.zeros(pix.shape[0])
    den_abs = np.zeros(pix.shape[0])
    for jdx, smp in enumerate(samples):
        a, b, ds, dt = smp
        w = sample_weight(smp)
        X = mesh_points(target, view, pix[:, 0] + 0.5 + ds, pix[:, 1] + 0.5 + dt)
        if lbar == "ray":
            val = _per_ray(target, dense, view, smp, X)
            num += w * val[:, :3]
            den += w * val[:, 3]
            den_abs += abs(w) * val[:, 3]
            continue
        o = Rv.T @ (aperture_point(target, view, a, b) - tv)   # the sample's origin in view i's frame
        x = X - o
        qx = Ks[0] * x[:, 0] / x[:, 2] + Ks[2]
        qy = Ks[1] * x[:, 1] / x[:, 2] + Ks[3]
        if renders is None:  # sparse: render only the texels the bilinear reads touch
            img = _sparse_render(target, dense, view, smp, supersample, qx - 0.5, qy - 0.5, threads)
        else:
            img = renders[jdx]
        val = _bilinear_premultiplied(img, qx - 0.5, qy - 0.5)
        num += w * val[:, :3]
        den += w * val[:, 3]
        den_abs += abs(w) * val[:, 3]
    out = np.zeros((pix.shape[0], 4))
    ok = den > 0.0
    out[ok, :3] = num[ok] / den[ok, None]
    out[ok, 3] = 1.0
    if pixels is None:
        out, den, den_abs = out.reshape(H, W, 4), den.reshape(H, W), den_abs.reshape(H, W)
    return {"rgba": out, "den": den, "den_abs": den_abs} if details else out


def _sparse_render(target, dense, view: int, smp, supersample, u, v, threads):
    """A render image holding only the texels around (u, v) (zero elsewhere)."""
    import oracle
    import scene

    Rv, _ = _view_R_t(target, view)
    Ks, Ws, Hs = virtual_intrinsics(target, view, supersample)
    i0 = np.floor(u).astype(np.int64)
    j0 = np.floor(v).astype(np.int64)
    ii = np.clip(np.concatenate([i0, i0 + 1, i0, i0 + 1]), 0, Ws - 1)
    jj = np.clip(np.concatenate([j0, j0, j0 + 1, j0 + 1]), 0, Hs - 1)
    need = np.unique(np.stack([ii, jj], axis=1), axis=0)
    eye = scene.Eye(scene.pose_array(Rv, aperture_point(target, view, smp[0], smp[1])), Ks, Ws, Hs)
    img = np.zeros((Hs, Ws, 4))
    img[need[:, 1], need[:, 0]] = oracle.render(dense, eye, pixels=need, threads=threads)["rgba"]
    return img


def virtual_renders(target, dense, view: int, samples, supersample: int = 1, threads=None):
    """Lbar renders (FP64 oracle of the method on `dense`), one per sample."""
    import oracle
    import scene

    samples = np.asarray(samples, dtype=np.float64).reshape(-1, 4)
    Rv, _ = _view_R_t(target, view)
    Ks, Ws, Hs = virtual_intrinsics(target, view, supersample)
    out = []
    for a, b, _, _ in samples:
        o = aperture_point(target, view, a, b)
        eye = scene.Eye(scene.pose_array(Rv, o), Ks, Ws, Hs)
        out.append(oracle.render(dense, eye, threads=threads)["rgba"])
    return out
