"""GPU backward pass vs the FP64 oracle (supplementary "Backward Derivative").

Upstream gradients dl/dC are seeded normals, set to zero at pixels the oracle
flags as within rounding distance of a discrete decision (cutoffs, stop,
depth order, gamma saturation, a near-tie of the most influential boundary
point), so both sides differentiate the same piecewise-smooth function.
Pixels whose most influential boundary point lies within D_TOL = 5e-3 px are
excluded too: dl/db of Eq. 6 points along (q - b)/|q - b|, and the FP32
I_uv of the GPU places b ~1e-6 px away from the oracle's, which turns that
direction by ~1e-6 / |q - b|. Gradients are
compared to the oracle's analytic gradient (relative 1e-3 in norm, plus an
elementwise bound) and to central finite differences of the oracle.
"""
import numpy as np
import pytest

from tests.gpu_util import GRAD_TOL, gpu_forward, grad_rel, make_renderer

pytestmark = pytest.mark.gpu

D_TOL = 5e-3


def _run(oracle, sc, cams, seed=0, tile=16, use_boundary=True, renderer=None):
    import torch
    g = gpu_forward(sc, cams, tile=tile, use_boundary=use_boundary, stages=(), renderer=renderer)
    rd, dev = g["renderer"], g["dev"]
    rng = np.random.default_rng(seed)
    opts = {"use_boundary": 1 if use_boundary else 0, "tol_d": D_TOL}
    dls, refs = [], []
    for c in cams:
        ref = oracle.render(sc, c, opts=opts)
        dl = rng.normal(size=(c["height"], c["width"], 3))
        dl[ref["flags"] != 0] = 0.0
        dls.append(dl)
        refs.append(ref)
    dl_flat = np.concatenate([d.reshape(-1, 3) for d in dls])
    grads = rd.backward(dev, cams, torch.as_tensor(dl_flat, dtype=torch.float32, device="cuda"))
    rd.sync_status()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    ref_g = None
    inter = []
    for c, dl in zip(cams, dls):
        r = oracle.backward(sc, c, dl, opts=opts, intermediates=True)
        inter.append(r)
        if ref_g is None:
            ref_g = {k: r[k].copy() for k in ("ctrl", "color", "opacity", "r_b", "log_scale", "quat", "sh")
                     if k in r}
        else:
            for k in ref_g:
                ref_g[k] += r[k]
    return g, out, ref_g, inter, dls


def _assert_close(got, ref, name, elem_tol=GRAD_TOL):
    rel = grad_rel(got, ref)
    assert rel < GRAD_TOL, f"{name}: relative error {rel}"
    scale = np.abs(ref).max()
    bound = elem_tol * np.abs(ref) + 0.1 * elem_tol * scale
    bad = np.abs(got - ref) > bound
    if bad.any():
        idx = np.argsort(-(np.abs(got - ref) / bound).ravel())[:6]
        worst = [(np.unravel_index(i, ref.shape), float(got.ravel()[i]), float(ref.ravel()[i])) for i in idx]
        raise AssertionError(f"{name}: {int(bad.sum())} of {bad.size} elements off (scale {scale:.3g}); "
                             f"worst (index, gpu, oracle): {worst}")


CASES = [
    ("config1", lambda S: S.config_scene(1)[:2]),
    ("two_wide_boundary", lambda S: S.tiny_scene("two", size=(72, 64), r_b=0.08)),
    ("ico1_ragged", lambda S: S.tiny_scene("ico1", noise=0.04, size=(90, 70), r_b=0.04)),
    ("degree3", lambda S: S.tiny_scene("ico1", n=3, noise=0.03, size=(70, 66), r_b=0.04)),
    ("degree1", lambda S: S.tiny_scene("octa", n=1, size=(48, 40), r_b=0.04)),
    ("degree4", lambda S: S.tiny_scene("octa", n=4, noise=0.02, size=(56, 48), r_b=0.04)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_gradients_match_oracle_analytic(oracle, scenes, name, make):
    sc, cams = make(scenes)
    g, got, ref, inter, _ = _run(oracle, sc, cams)
    for k in ("ctrl", "color", "opacity", "r_b"):
        if np.abs(ref[k]).max() == 0:
            assert np.abs(got[k]).max() < 1e-6, k
            continue
        _assert_close(got[k], ref[k], k)
    # intermediate per-Gaussian and per-boundary-point gradients
    rd = g["renderer"]
    gg = rd.stage("ggrad").astype(np.float64)
    og = inter[0]["ggrad"]
    # GPU layout: dmu x,y, dK a,b,c, do, dcol r,g,b ; oracle: dmu, dK, dcol, do
    assert grad_rel(gg[:, 0:5], og[:, 0:5]) < GRAD_TOL
    assert grad_rel(gg[:, 5], og[:, 8]) < GRAD_TOL
    assert grad_rel(gg[:, 6:9], og[:, 5:8]) < GRAD_TOL
    bg = rd.stage("bgrad").astype(np.float64)
    ob = inter[0]["bgrad"][: len(bg)]
    if np.abs(ob).max() > 0:
        assert grad_rel(bg[:, :3], ob) < GRAD_TOL


def test_gradients_multiview_batch(oracle, scenes):
    sc, cams = scenes.config_scene(4)
    crops = [scenes.crop_camera(cams[0], 60, 70, 90, 70), scenes.crop_camera(cams[5], 200, 180, 80, 97)]
    _, got, ref, _, _ = _run(oracle, sc, crops, seed=3)
    for k in ("ctrl", "color", "opacity", "r_b"):
        _assert_close(got[k], ref[k], k)


def test_gradients_multiview_batch_small_boundary_scale(oracle, scenes):
    """Config 4 at the paper's other boundary scale, r_b = 1e-3 (Table 4):
    sigma = k_b fx r_b / z is about 0.2-0.7 px, so Eq. 7's gamma leaves
    saturation only inside the boundary pixel itself. Crops of a 1024^2, an
    800^2 and a 256^2 view in one batched call."""
    sc, cams = scenes.config_scene(4, r_b=1e-3)
    pick = {}
    for c in cams:
        pick.setdefault(c["width"], c)
    crops = [scenes.crop_camera(pick[1024], 440, 430, 90, 70), scenes.crop_camera(pick[800], 330, 350, 80, 97),
             scenes.crop_camera(pick[256], 90, 96, 72, 60)]
    _, got, ref, _, _ = _run(oracle, sc, crops, seed=4)
    for k in ("ctrl", "color", "opacity", "r_b"):
        _assert_close(got[k], ref[k], k)
    assert np.abs(ref["r_b"]).max() > 0


@pytest.mark.parametrize("blend_cap", [0, 1])
def test_dense_tiles_room_crop(oracle, scenes, blend_cap):
    """Config 5 (100,000 degree-3 triangles, opacity Beta(5,1)): a 96^2 crop of
    a view whose near surfaces give Gaussians of ~16 px support. Its tiles hold
    up to ~8,800 (Gaussian, tile) pairs (the long-segment sort in global
    memory), pixels walk ~450 list entries and reach the transmittance stop,
    and the blend records run to many headers per pixel. Image (stable pixels)
    and gradients against the oracle, with the default record capacity and
    with none at all (every warp block re-walks its tile list)."""
    from tests.gpu_util import FWD_TOL, compare_images
    sc, cams = scenes.config_scene(5)
    crop = scenes.crop_camera(cams[5], 640, 192, 96, 96)
    rd = make_renderer(sc, [crop], pairs_per_px=64, max_blend_pairs=blend_cap)
    g, got, ref, inter, _ = _run(oracle, sc, [crop], seed=6, renderer=rd)
    counts = rd.counts()
    ranges = rd.stage("g_ranges")
    assert int(np.diff(ranges).max()) > 4096  # the global-memory radix sort of long tile lists ran
    if blend_cap:
        assert counts["walked_blocks"] >= 6 * 6 * 8 - 1, counts  # (at most one chunk fits)
    else:
        assert counts["rec_headers"] > 96 * 96, counts  # more than one record per pixel
        assert counts["walked_blocks"] == 0, counts
    ref_img = oracle.render(sc, crop)
    err, unstable = compare_images(g["images"][0], ref_img, ref_img["flags"], oracle)
    assert err < FWD_TOL, err
    assert unstable < 0.1
    # norm within 1e-3 as everywhere; elementwise 2e-3: a pixel here blends ~100-450 pairs
    # whose FP32 chain-rule terms reach one control point through up to 9,216 pixels
    for k in ("ctrl", "color", "opacity", "r_b"):
        if np.abs(ref[k]).max() == 0:
            continue
        _assert_close(got[k], ref[k], k, elem_tol=2e-3)


@pytest.mark.parametrize("cap", [1, 3000])
def test_blend_record_overflow_falls_back_to_tile_walk(oracle, scenes, cap):
    """max_blend_pairs below what the forward composites: the warp blocks
    whose records do not fit are listed by the forward and the backward
    re-walks their tile lists (retaking the forward's decisions) instead of
    replaying records; no error is raised and the gradients still match the
    oracle. cap = 1: every block walks; cap = 3000: some blocks replay, the
    rest walk."""
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(90, 70), r_b=0.04)
    rd = make_renderer(sc, cams, max_blend_pairs=cap)
    _, got, ref, _, _ = _run(oracle, sc, cams, seed=7, renderer=rd)
    # warp blocks (8 x 4 pixels at tile 16) holding a composited pixel (T < 1)
    T = rd.stage("T").reshape(70, 90)
    cells = np.zeros(((70 + 3) // 4, (90 + 7) // 8), bool)
    ys, xs = np.nonzero(T < 1.0)
    cells[ys // 4, xs // 8] = True
    blocks = int(cells.sum())
    walked = rd.counts()["walked_blocks"]
    assert (walked >= blocks - 1) if cap == 1 else (0 < walked < blocks), (walked, blocks)
    for k in ("ctrl", "color", "opacity", "r_b"):
        _assert_close(got[k], ref[k], k)


@pytest.mark.parametrize("tile", [8, 32])
def test_tile_walk_at_other_tile_sizes(oracle, scenes, tile):
    """Every warp block re-walks its tile list (max_blend_pairs = 1) at tile 8
    (one pixel per lane, two warps per tile) and tile 32 (four pixels per
    lane, the walk's two-slot primitive cache): gradients against the
    oracle."""
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(90, 70), r_b=0.04)
    rd = make_renderer(sc, cams, tile=tile, max_blend_pairs=1)
    _, got, ref, _, _ = _run(oracle, sc, cams, seed=8, renderer=rd)
    assert rd.counts()["walked_blocks"] > 0
    for k in ("ctrl", "color", "opacity", "r_b"):
        _assert_close(got[k], ref[k], k)


def test_gradients_without_boundary_term(oracle, scenes):
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(64, 60), r_b=0.04)
    _, got, ref, _, _ = _run(oracle, sc, cams, use_boundary=False)
    for k in ("ctrl", "color", "opacity"):
        _assert_close(got[k], ref[k], k)
    assert np.abs(got["r_b"]).max() == 0.0


@pytest.mark.parametrize("tile", [8, 32])
def test_gradients_other_tile_sizes(oracle, scenes, tile):
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(90, 70), r_b=0.04)
    _, got, ref, _, _ = _run(oracle, sc, cams, tile=tile)
    for k in ("ctrl", "color", "opacity", "r_b"):
        _assert_close(got[k], ref[k], k)


def test_gradients_vs_finite_differences_config3_crop(oracle, scenes):
    """Config 3: 20k triangles, 1024^2 view; 256^2 centre crop; 50 random
    parameters (control points, colours, opacities, boundary scales); FP64
    central differences of the oracle with h = 1e-6, relative error <= 1e-3."""
    import torch
    sc, cams = scenes.config_scene(3)
    cam = scenes.crop_camera(cams[0], 384, 384, 256, 256)
    opts = {"tol_d": 1e-2}
    idm, uv, _ = oracle.raster(sc, cam)
    base = oracle.render(sc, cam, idm, uv, opts=opts, records=True)
    rng = np.random.default_rng(11)
    dl = rng.normal(size=(256, 256, 3))
    dl[base["flags"] != 0] = 0.0
    g = gpu_forward(sc, [cam], stages=())
    grads = g["renderer"].backward(g["dev"], [cam], torch.as_tensor(dl.reshape(-1, 3), dtype=torch.float32,
                                                                    device="cuda"))
    g["renderer"].sync_status()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    s64 = oracle.scene_to64(sc)
    visible = np.unique(idm[idm >= 0])
    rmax = int(np.ceil(max(base["gauss"][:, 12].max(), base["gauss"][:, 13].max()))) + 2
    kinds = ["ctrl", "color", "opacity", "r_b"]
    m = s64["ctrl"].shape[1]
    results = []
    tries = 0
    while len(results) < 50 and tries < 600:
        kind = kinds[tries % 4]
        tries += 1
        prim = int(rng.choice(visible))
        idx = (prim, int(rng.integers(m)), int(rng.integers(3))) if kind in ("ctrl", "color") else (prim,)
        # only pixels within the support of this primitive's Gaussians can change
        near = np.zeros_like(idm, bool)
        ys, xs = np.nonzero(idm == prim)
        for y, x in zip(ys, xs):
            near[max(0, y - rmax):y + rmax + 1, max(0, x - rmax):x + rmax + 1] = True
        ref_hash = oracle.render(sc, cam, idm, uv, opts=opts, pixels=near)["hash"]
        vals = []
        for sgn in (1.0, -1.0):
            s2 = {k: v.copy() for k, v in s64.items()}
            s2[kind][idx] += sgn * 1e-6
            r = oracle.render(sc, cam, idm, uv, opts=opts, scene64=s2, pixels=near)
            if r["hash"] != ref_hash:
                break  # the step crosses a discrete decision: draw another parameter
            vals.append(float((r["image"][near] * dl[near]).sum()))
        if len(vals) < 2:
            continue
        fd = (vals[0] - vals[1]) / 2e-6
        results.append((kind, idx, got[kind][idx], fd))
    fds = np.array([r[3] for r in results])
    scale = np.abs(fds).max()
    assert scale > 0
    bad = [(k, i, a, f) for k, i, a, f in results if abs(a - f) > GRAD_TOL * max(abs(f), 1e-2 * scale)]
    assert len(results) == 50
    assert not bad, bad[:5]


def test_autograd_function_matches_backward(scenes):
    import torch
    from paper_2503_13961_gb300 import render as R
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(64, 48), r_b=0.04)
    rd = make_renderer(sc, cams)
    dev = R.scene_to_device(sc)
    leaf = {k: dev[k].clone().requires_grad_(k in ("ctrl", "color", "opacity", "r_b")) for k in R.SCENE_KEYS}
    leaf.update(degree=dev["degree"], bg=dev["bg"])
    img = R.render(rd, leaf, cams)
    target = torch.rand_like(img)
    loss = (img - target).abs().mean()
    loss.backward()
    dimg = torch.sign(img.detach() - target) / img.numel()
    rd.forward(dev, cams)
    ref = rd.backward(dev, cams, dimg)
    rd.sync_status()
    for k in ("ctrl", "color", "opacity", "r_b"):
        a, b = leaf[k].grad.cpu().numpy(), ref[k].cpu().numpy()
        assert np.allclose(a, b, rtol=1e-4, atol=1e-7 * np.abs(b).max()), k


def test_l1_loss_helper(scenes):
    import torch
    from paper_2503_13961_gb300 import render as R
    sc, cams = scenes.tiny_scene("ico1", size=(16, 16))
    rd = make_renderer(sc, cams)
    a = torch.rand(256, 3, device="cuda")
    b = torch.rand(256, 3, device="cuda")
    loss = torch.zeros(1, device="cuda")
    d = rd.l1_loss_grad(a, b, 0.5, loss=loss)
    torch.cuda.synchronize()
    assert torch.allclose(d, 0.5 * torch.sign(a - b))
    assert torch.allclose(loss, 0.5 * (a - b).abs().sum(), rtol=1e-5)
    # a ragged length (the four-value loop's tail) and arrays one float off a
    # 16-byte boundary (the one-value loop only)
    for off in (0, 1):
        buf_a = torch.rand(3 * 1001 + off, device="cuda")
        buf_b = torch.rand(3 * 1001 + off, device="cuda")
        a, b = buf_a[off:], buf_b[off:]
        dbuf = torch.empty(3 * 1001 + off, device="cuda")
        loss = torch.zeros(1, device="cuda")
        d = rd.l1_loss_grad(a, b, 0.25, d_images=dbuf[off:], loss=loss)
        torch.cuda.synchronize()
        assert torch.equal(d, 0.25 * torch.sign(a - b)), off
        assert torch.allclose(loss, 0.25 * (a - b).abs().sum(), rtol=1e-5), off
    del R


@pytest.mark.parametrize("R", [1, 3])
def test_attribute_map_gradients_match_oracle(oracle, scenes, R):
    """Rotation / scaling attribute maps of leg resolution R (Eq. 5): gradients
    of their texels (and of the other parameters) against the oracle."""
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(90, 70), r_b=0.04)
    sc = scenes.with_attribute_maps(sc, R, seed=R)
    _, got, ref, _, _ = _run(oracle, sc, cams, seed=5)
    for k in ("ctrl", "color", "opacity", "r_b", "log_scale", "quat"):
        assert got[k].shape == ref[k].shape, k
        _assert_close(got[k], ref[k], k)
    assert np.abs(ref["log_scale"]).max() > 0 and np.abs(ref["quat"]).max() > 0


@pytest.mark.parametrize("D", [1, 3])
def test_sh_colour_gradients_match_oracle(oracle, scenes, D):
    """View-dependent colour of SH degree D: gradients of the coefficients and
    of the control points (which move the view direction) against the oracle."""
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(90, 70), r_b=0.04)
    sc = scenes.with_sh(sc, D, seed=D)
    _, got, ref, _, _ = _run(oracle, sc, cams, seed=9)
    for k in ("ctrl", "color", "opacity", "r_b", "sh"):
        assert got[k].shape == ref[k].shape, k
        _assert_close(got[k], ref[k], k)


def test_full_size_batched_backward_equals_the_plain_path(scenes):
    # the benchmark's launch configuration (64 views of mixed size in one
    # graph-captured call, tile 16): its gradients are the sum over the views
    # of the plain single-view path, which the crops above check against the
    # oracle; views are independent given the parameters, so only the FP32
    # summation order differs
    import torch
    from paper_2503_13961_gb300 import render as R
    sc, cams = scenes.config_scene(4)
    P = sum(c["width"] * c["height"] for c in cams)
    rd = make_renderer(sc, cams, graph=True, tile=16)
    dev = R.scene_to_device(sc)
    gen = torch.Generator(device="cuda").manual_seed(11)
    dl = torch.randn((P, 3), device="cuda", generator=gen) / P
    rd.forward(dev, cams)
    g_all = rd.backward(dev, cams, dl)
    rd.sync_status()
    Pmax = max(c["width"] * c["height"] for c in cams)
    one = R.Renderer(degree=2, max_prims=sc["ctrl"].shape[0], max_views=1, max_pixels=Pmax,
                     max_pairs=8 * Pmax, max_boundary_pairs=8 * Pmax, tile_size=16)
    acc = {k: torch.zeros_like(v) for k, v in g_all.items()}
    off = 0
    for c in cams:
        n = c["width"] * c["height"]
        one.forward(dev, [c])
        g = one.backward(dev, [c], dl[off:off + n].contiguous())
        for k in acc:
            acc[k] += g[k]
        off += n
    one.sync_status()
    torch.cuda.synchronize()
    for k in ("ctrl", "color", "opacity", "r_b"):
        a, b = g_all[k].double().cpu().numpy(), acc[k].double().cpu().numpy()
        assert np.abs(b).max() > 0, k
        rel = grad_rel(a, b)
        assert rel < 1e-4, (k, rel)
    rd.close()
    one.close()
