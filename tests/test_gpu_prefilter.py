"""lf_prefilter (Sec. 5, Eq. 5) through the C ABI against the FP64 oracle.

Both sides take the same samples.  The GPU renders Lbar with the method's own
kernels (coverage and view selection bit-exact, colour within 2e-3 of the
oracle's renders) and forms Eq. 5 in FP32, so a pixel may differ from the
oracle by 2e-3 times the ratio's error magnification sum |w| alpha / sum w alpha,
plus FP32 rounding of the mesh point and its projection (the 2e-4 term).
Where the oracle's denominator is well away from 0 the valid masks agree.
"""
import numpy as np
import pytest

import scene
from oracle import prefilter as opf

pytestmark = pytest.mark.gpu


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
def models():
    """A 16-view real-time model (64^2, 17^2 meshes) and a 36-view dense one
    (64^2, 33^2 meshes) of the same 8-sphere scene on a 40-degree cap."""
    prims = scene.sphere_scene(1, 8, forward_cone_deg=35.0)
    target = scene.build_light_field(prims, scene.cap_grid_directions(4, 40.0), 64, 64, 90.0, 17, name="target")
    dense = scene.build_light_field(prims, scene.cap_grid_directions(6, 40.0), 64, 64, 90.0, 33, name="dense")
    return target, dense


def _samples(seed, J):
    """Stratified samples (the library's helper): with the pixel offsets on a
    jittered grid over the Lanczos-2 support the weights sum well above 0,
    where a handful of uniform offsets can land mostly in the negative lobes."""
    import paper_1810_08860_gb300 as lfm

    return lfm.prefilter_samples(J, seed).astype(np.float64)  # the values the library receives


def _renderers(lfmod, target, dense, J, tri_capacity=0):
    rt = lfmod.Renderer(0)
    rt.load_views(target)
    rt.build_meshes(target)
    rd = lfmod.Renderer(0, max_eyes=J, tri_capacity=tri_capacity)
    rd.load_views(dense)
    rd.build_meshes(dense)
    return rt, rd


def _check(got, ref):
    den, den_abs, want = ref["den"], ref["den_abs"], ref["rgba"]
    sure = den > 0.05 * np.maximum(den_abs, 1e-30)
    assert sure.mean() > 0.5
    assert np.array_equal(got[..., 3][sure] > 0, want[..., 3][sure] > 0)
    ok = sure & (want[..., 3] > 0)
    tol = 2e-3 * den_abs[ok] / den[ok] + 2e-4
    err = np.abs(got[ok][:, :3] - want[ok][:, :3]).max(axis=1)
    assert np.all(err <= tol), (err.max(), np.argmax(err - tol))


@pytest.mark.parametrize("supersample", [1, 2])
def test_prefilter_matches_oracle(lfmod, models, supersample):
    target, dense = models
    J = 16
    samples = _samples(11 + supersample, J)  # seeds 12 and 13
    w = np.array([opf.sample_weight(x) for x in samples])
    assert w.sum() > 0.5 * np.abs(w).sum()  # a set whose weights do not nearly cancel
    rt, rd = _renderers(lfmod, target, dense, J)
    first, n = 4, 3
    out = rt.prefilter(rd, samples, first_view=first, n_views=n, supersample=supersample).cpu().numpy()
    for k in range(n):
        ref = opf.prefilter(target, dense, first + k, samples, supersample=supersample, details=True)
        _check(out[k].astype(np.float64), ref)
    rt.close()
    rd.close()


def test_prefilter_errors(lfmod, models):
    import torch

    target, dense = models
    samples = _samples(3, 4)
    rt, rd = _renderers(lfmod, target, dense, 2)  # max_eyes 2 < 4 samples
    with pytest.raises(lfmod.LFError) as info:
        rt.prefilter(rd, samples, first_view=0, n_views=1)
    assert info.value.status == 1
    with pytest.raises(lfmod.LFError):
        rt.prefilter(rt, samples[:2], first_view=0, n_views=1)       # the same context twice
    with pytest.raises(lfmod.LFError):
        rt.prefilter(rd, samples[:2], first_view=15, n_views=2,
                     out=torch.empty((2, 64, 64, 4), device="cuda"))  # beyond the last view
    bad = samples[:2].copy()
    bad[0, 2] = 2.5
    with pytest.raises(lfmod.LFError):
        rt.prefilter(rd, bad, first_view=0, n_views=1)
    with pytest.raises(lfmod.LFError):
        rt.prefilter(rd, samples[:2], first_view=0, n_views=1, supersample=5)
    rt.close()
    rd.close()
    # a dense scratch of one triangle record overflows: reported, not hidden
    rt, rd = _renderers(lfmod, target, dense, 4, tri_capacity=1)
    with pytest.raises(lfmod.LFError) as info:
        rt.prefilter(rd, samples, first_view=0, n_views=1)
    assert info.value.status == 7
    rt.close()
    rd.close()


@pytest.mark.parametrize("supersample", [1, 2])
def test_prefilter_against_the_per_ray_definition(lfmod, models, supersample):
    """The GPU prefilter against Eq. 5 with each ray's own Lbar query (the
    oracle's per-ray mode) on sampled pixels.  The GPU implements the
    render-and-resample reading, so a pixel may differ from the definition by
    the render parity bound above plus that reading's own distance from the
    definition at the same pixel, which the oracle measures."""
    target, dense = models
    J = 16
    samples = _samples(12, J)
    rt, rd = _renderers(lfmod, target, dense, J)
    view = 4
    out = rt.prefilter(rd, samples, first_view=view, n_views=1, supersample=supersample).cpu().numpy()
    g_img = out[0].astype(np.float64)
    rng = np.random.default_rng(2)
    pix = np.stack([rng.integers(0, 64, 120), rng.integers(0, 64, 120)], axis=1)
    ray = opf.prefilter(target, dense, view, samples, pixels=pix, lbar="ray", details=True)
    ren = opf.prefilter(target, dense, view, samples, pixels=pix, supersample=supersample, details=True)
    sure = (ray["den"] > 0.05 * ray["den_abs"]) & (ren["den"] > 0.05 * ren["den_abs"])
    assert sure.mean() > 0.8
    g = g_img[pix[:, 1], pix[:, 0]]
    assert np.array_equal(g[sure, 3] > 0, ray["rgba"][sure, 3] > 0)
    reading = np.abs(ren["rgba"][sure, :3] - ray["rgba"][sure, :3]).max(axis=1)
    tol = 2e-3 * ren["den_abs"][sure] / ren["den"][sure] + 2e-4 + reading
    err = np.abs(g[sure, :3] - ray["rgba"][sure, :3]).max(axis=1)
    assert np.all(err <= tol), (err.max(), np.argmax(err - tol))
    print("prefilter %dx: GPU vs per-ray definition mean %.2e max %.2e (reading: mean %.2e)" % (
        supersample, err.mean(), err.max(), reading.mean()))
    rt.close()
    rd.close()
