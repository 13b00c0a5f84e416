"""Two-level progressive rendering (Sec. 7.2) on the GPU, through the C ABI,
against the oracle in oracle/twolevel.py.

The context holds both light fields of one scene: the fine level's views
first, then the coarse level's.  lf_set_levels makes the fine images
streamed (device pages), lf_upload_pages makes chosen fine views resident,
and every render draws the resident visible fine views plus the visible
coarse views that overlap a missing visible fine one.  The oracle renders
Eq. 2 over the union of the views it draws (fine first, then coarse, in
view order), so the GPU frame must equal it: coverage records bit-exact
(view ids mapped from the union's order to the context's), valid masks
identical, colour within 2e-3.
"""
import numpy as np
import pytest

import oracle
import scene
from oracle import twolevel

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
def levels():
    """A 36-view fine level and a 9-view coarse level (larger disks) of one
    8-sphere scene on a 40-degree cap, 48^2 images, 13^2 meshes."""
    prims = scene.sphere_scene(2, 8, forward_cone_deg=35.0)
    fine = scene.build_light_field(prims, scene.cap_grid_directions(6, 40.0), 48, 48, 90.0, 13, name="fine")
    coarse = scene.build_light_field(prims, scene.cap_grid_directions(3, 40.0), 48, 48, 90.0, 13, name="coarse")
    rng = scene.SplitMix64(41)
    eyes = [scene.head_pose_eyes(rng, 64, 56, 90.0, yaw_range=(-0.15, 0.15), pitch_deg=6.0, stereo=False)[0]
            for _ in range(4)]
    both = twolevel.union_light_field(fine, coarse, np.ones(fine.n_views, bool), np.ones(coarse.n_views, bool))
    return fine, coarse, both, eyes


def _renderer(lfmod, both, n_fine, n_pages, **kw):
    r = lfmod.Renderer(0, **kw)
    r.load_views(both)
    r.build_meshes(both)
    r.set_levels(n_fine, n_pages)
    return r


def _upload(r, fine, views, pages):
    if len(views):
        r.upload_pages(views, pages, [fine.images[v] for v in views])


def _check_frame(r, fine, coarse, eye, resident, max_records=16):
    """The GPU frame against the oracle's two-level frame for this residency."""
    fmask, cmask = twolevel.drawn_views(fine, coarse, eye, resident)
    got = r.render_inspect(eye, max_records=max_records)
    W, H = eye.width, eye.height
    img = got["rgba"].cpu().numpy().astype(np.float64)
    if not fmask.any() and not cmask.any():
        assert float(np.abs(img).max()) == 0.0
        return got, fmask, cmask
    lf_u = twolevel.union_light_field(fine, coarse, fmask, cmask)
    ref = oracle.render(lf_u, eye, fragments=True, max_slots=max_records)
    assert ref["stats"]["frag_overflow"] == 0
    to_ctx = np.concatenate([np.nonzero(fmask)[0], fine.n_views + np.nonzero(cmask)[0]])
    want = {}
    for f in ref["frags"]:
        want.setdefault(int(f["pixel"]), []).append((int(to_ctx[f["view"]]), int(f["n_cover"]), int(f["winner"]),
                                                     int(f["min_id"]), int(f["max_id"]), int(f["id_hash"])))
    have = {}
    for p in range(W * H):
        n = int(got["counts"][p])
        assert n <= max_records
        if n:
            have[p] = [(int(x["view"]), int(x["n_cover"]), int(x["winner"]), int(x["min_id"]), int(x["max_id"]),
                        int(x["id_hash"])) for x in got["records"][p][:n]]
    assert have.keys() == want.keys()
    bad = [p for p in want if have[p] != want[p]]
    assert not bad, (len(bad), bad[0], have[bad[0]], want[bad[0]])
    valid = ref["rgba"][..., 3] > 0
    assert np.array_equal(img[..., 3] > 0, valid)
    if valid.any():
        assert np.max(np.abs(img[valid][:, :3] - ref["rgba"][valid][:, :3])) <= COLOUR_TOL
    # the views drawn are the union's, the wanted ones the eye's fine selection
    drawn = np.zeros(fine.n_views + coarse.n_views, bool)
    drawn[to_ctx] = True
    assert np.array_equal(got["active"], drawn)
    return got, fmask, cmask


def test_all_fine_resident_is_the_fine_render(lfmod, levels):
    fine, coarse, both, eyes = levels
    nf = fine.n_views
    r = _renderer(lfmod, both, nf, nf)
    _upload(r, fine, np.arange(nf), np.arange(nf)[::-1])  # pages in another order than views
    for eye in eyes[:2]:
        _, fmask, cmask = _check_frame(r, fine, coarse, eye, np.ones(nf, bool))
        assert not cmask.any() and fmask.any()
        assert np.array_equal(r.levels_wanted(), np.nonzero(oracle.select_views(fine, eye))[0])
    r.close()


def test_no_fine_resident_falls_back_to_coarse(lfmod, levels):
    fine, coarse, both, eyes = levels
    r = _renderer(lfmod, both, fine.n_views, 4)
    for eye in eyes:
        _, fmask, cmask = _check_frame(r, fine, coarse, eye, np.zeros(fine.n_views, bool))
        assert not fmask.any() and cmask.any()
    r.close()


def test_mixed_residency_and_eviction(lfmod, levels):
    """Random residencies, then pages overwritten by other views: the evicted
    views are missing again and their region falls back to the coarse level."""
    fine, coarse, both, eyes = levels
    nf, pages = fine.n_views, 12
    rng = np.random.default_rng(5)
    r = _renderer(lfmod, both, nf, pages)
    resident = np.zeros(nf, bool)
    page_view = -np.ones(pages, int)
    for step in range(4):
        views = rng.choice(nf, size=pages if step == 0 else 5, replace=False)
        views = np.array([v for v in views if not resident[v]][:pages])
        slots = rng.choice(pages, size=len(views), replace=False)
        _upload(r, fine, views, slots)
        for v, p in zip(views, slots):
            if page_view[p] >= 0:
                resident[page_view[p]] = False
            page_view[p] = v
            resident[v] = True
        assert resident.sum() == (page_view >= 0).sum()
        _, fmask, cmask = _check_frame(r, fine, coarse, eyes[step % len(eyes)], resident)
        if step:
            assert fmask.any() or cmask.any()
    r.close()


def test_progressive_frames_with_the_page_cache(lfmod, levels):
    """The progressive loop of Sec. 7.2: each frame draws what is resident and
    reports the fine views it selected; the host cache (FIFO, a per-frame
    budget) admits missing ones into pages for the next frames.  Every frame
    equals the oracle's two-level frame for the residency it was drawn with,
    and with pages for all the wanted views the frames converge to the fine
    render."""
    fine, coarse, both, eyes = levels
    nf, pages, budget = fine.n_views, 16, 4
    r = _renderer(lfmod, both, nf, pages)
    cache = lfmod.PageCache(nf, pages)
    resident = np.zeros(nf, bool)
    eye = eyes[0]
    for frame in range(6):
        _check_frame(r, fine, coarse, eye, resident)
        wanted = r.levels_wanted()
        adm = cache.frame(wanted, budget)
        _upload(r, fine, [v for v, _ in adm], [p for _, p in adm])
        resident = cache.pages() >= 0
    if len(r.levels_wanted()) <= pages:
        assert resident[r.levels_wanted()].all()
        got = r.render([eye])[0].cpu().numpy().astype(np.float64)
        want = oracle.render(fine, eye)["rgba"]
        v = want[..., 3] > 0
        assert np.array_equal(got[..., 3] > 0, v)
        assert np.max(np.abs(got[v][:, :3] - want[v][:, :3])) <= COLOUR_TOL
    cache.close()
    r.close()


def test_batch_and_tile_shapes_agree(lfmod, levels):
    import torch

    fine, coarse, both, eyes = levels
    nf = fine.n_views
    views = np.arange(0, nf, 3)
    base = _renderer(lfmod, both, nf, len(views))
    _upload(base, fine, views, np.arange(len(views)))
    want = [base.render([e])[0].cpu() for e in eyes]
    for tile in [(8, 8), (32, 8)]:
        r = _renderer(lfmod, both, nf, len(views), tile=tile, max_eyes=len(eyes))
        _upload(r, fine, views, np.arange(len(views)))
        for _ in range(2):  # capture, then replay
            out = r.render_batch(eyes)
            assert all(torch.equal(o.cpu(), w) for o, w in zip(out, want))
        r.close()
    base.close()


def test_level_errors(lfmod, levels):
    fine, coarse, both, _ = levels
    r = lfmod.Renderer(0)
    with pytest.raises(lfmod.LFError) as info:
        r.set_levels(4, 2)
    assert info.value.status == 4  # no views
    r.load_views(both)
    r.build_meshes(both)
    with pytest.raises(lfmod.LFError) as info:
        r.upload_pages([0], [0], [fine.images[0]])
    assert info.value.status == 4  # no levels
    for nf, npg in [(0, 1), (both.n_views, 1), (10, 0), (10, 11)]:
        with pytest.raises(lfmod.LFError) as info:
            r.set_levels(nf, npg)
        assert info.value.status == 1
    r.set_levels(fine.n_views, 4)
    with pytest.raises(lfmod.LFError):
        r.set_levels(fine.n_views, 4)  # already split
    for views, pages in [([fine.n_views], [0]), ([0], [4]), ([0, 0], [0, 1]), ([0, 1], [2, 2])]:
        with pytest.raises(lfmod.LFError) as info:
            r.upload_pages(views, pages, [fine.images[0]] * len(views))
        assert info.value.status == 1
    import torch

    out = torch.empty((8, 8, 4), device="cuda")
    import ctypes

    poses = lfmod._poses([both.poses[0]])
    intr = lfmod._intrinsics([[8.0, 8.0, 4.0, 4.0]], [(8, 8)])
    st = r.lib.lf_render_static(r.ctx, poses, intr, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 6  # LF_ERR_UNSUPPORTED
    # loading the views again returns to one level
    r.load_views(both)
    r.build_meshes(both)
    r.set_levels(fine.n_views, 2)
    r.close()
