"""Split and prune geometry on the GPU (Sec. 3.3 "Splitting and Pruning")
against the FP64 oracle, through the C ABI: per-primitive area, aspect
ratio, mean control-point gradient and the prune / split flags; the exact
1 -> 4 midpoint subdivision of control points, colours, attribute maps and
per-primitive attributes.

Tolerances: the pieces' control points to 2e-6 of the parent's extent
(every de Casteljau weight is 0, 1/2 or 1: a few FP32 roundings). FP32
positions put ~1e-7 |p| of absolute error into every edge vector, so the
area is compared to 1e-5 relative + 2e-6 |p|max L (L the longest corner
edge) and the aspect ratio s to 1e-4 + 1e-6 |p|max s / L relative, where
the two longest corner edges differ by more than 1e-4 (the box's axis
follows the longest edge, so a near tie may pick either axis); the mean
gradient to 1e-5. The flags are compared where every measure is farther
from its threshold than its tolerance; elsewhere either decision is valid.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 1e-5


def _dev(scene):
    from paper_2503_13961_gb300 import render as R
    return R.scene_to_device(scene)


def _corner_edges(ctrl, n):
    from oracle import split as S
    P = [ctrl[S.index(n, n, 0)], ctrl[S.index(n, 0, n)], ctrl[S.index(n, 0, 0)]]
    return sorted(float(np.linalg.norm(P[(e + 1) % 3] - P[e])) for e in range(3))


def _tolerances(ctrl, n, s_ref):
    # FP32 positions carry ~1e-7 |p| of absolute error into every edge vector
    L = _corner_edges(ctrl, n)[2]
    mag = float(np.abs(ctrl).max())
    tol_area = 2e-6 * mag * L
    tol_aspect = 1e-4 + 1e-6 * mag * s_ref / max(L, 1e-30)
    return tol_area, tol_aspect


def _near_tie(ctrl, n):
    L = _corner_edges(ctrl, n)
    return L[2] - L[1] <= 1e-4 * L[2]


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_metrics_and_flags_match_the_oracle(n):
    import torch
    from oracle import split as S
    from paper_2503_13961_gb300 import render as R
    from paper_2503_13961_gb300 import scenes
    sc = scenes.mixed_shapes_scene(400, n, seed=n)
    dev = _dev(sc)
    rng = np.random.default_rng(7)
    g = (rng.normal(size=sc["ctrl"].shape) * 10.0 ** rng.uniform(-4, -2, size=(len(sc["ctrl"]), 1, 1)))
    g = g.astype(np.float32)
    out = R.prim_metrics(dev, torch.as_tensor(g, device="cuda"))
    torch.cuda.synchronize()
    area, asp = out["area"].cpu().numpy(), out["aspect"].cpu().numpy()
    grad, flags = out["grad"].cpu().numpy(), out["flags"].cpu().numpy()
    compared = [0, 0]
    for m in range(len(sc["ctrl"])):
        c = sc["ctrl"][m].astype(np.float64)
        a_ref, s_ref, g_ref = S.area(c, n), S.aspect(c, n), S.avg_grad(g[m])
        t_area, t_asp = _tolerances(c, n, s_ref)
        t_area += REL * a_ref
        assert abs(area[m] - a_ref) <= t_area, (m, area[m], a_ref)
        assert abs(grad[m] - g_ref) <= REL * g_ref, (m, grad[m], g_ref)
        tie = _near_tie(c, n)
        if not tie and math.isfinite(s_ref) and t_asp < 1e-2:
            assert abs(asp[m] - s_ref) <= t_asp * s_ref, (m, asp[m], s_ref)
        near = (abs(a_ref - S.TAU_A) <= t_area or not t_asp < 1e-2 or abs(s_ref - S.TAU_S) <= t_asp * S.TAU_S
                or abs(g_ref - S.TAU_G) <= 1e-4 * S.TAU_G)
        if not near and not tie:
            prune, split = S.decisions(c, n, g[m])
            assert flags[m] == (1 if prune else 0) | (2 if split else 0), (m, flags[m], prune, split)
            compared[0] += 1
        compared[1] += int(flags[m] & 1)
    # not vacuous: most flags compared, both outcomes present
    assert compared[0] > 300 and 20 < compared[1] < 380
    assert 0 < int((flags & 2).astype(bool).sum()) < len(flags)


def test_metrics_without_gradients_leave_the_split_bit_clear():
    import torch
    from paper_2503_13961_gb300 import render as R
    from paper_2503_13961_gb300 import scenes
    dev = _dev(scenes.mixed_shapes_scene(64, 2, seed=3))
    out = R.prim_metrics(dev)
    torch.cuda.synchronize()
    assert not (out["flags"].cpu().numpy() & 2).any()


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_subdivision_matches_the_oracle(n):
    import torch
    from oracle import split as S
    from paper_2503_13961_gb300 import render as R
    from paper_2503_13961_gb300 import scenes
    sc = scenes.mixed_shapes_scene(200, n, seed=10 + n)
    sc = scenes.with_sh(sc, 2, seed=n)
    dev = _dev(sc)
    sel = np.array([5, 0, 199, 17, 17, 63], np.int32)  # repeats allowed
    out = R.subdivide(dev, torch.as_tensor(sel, device="cuda"))
    torch.cuda.synchronize()
    got = {k: out[k].cpu().numpy() for k in R.SCENE_KEYS + ("sh",)}
    assert got["ctrl"].shape == (4 * len(sel),) + sc["ctrl"].shape[1:]
    for s, m in enumerate(sel):
        c = sc["ctrl"][m].astype(np.float64)
        ext = np.ptp(c, axis=0).max()
        want = S.subdivide(c, n)
        want_col = S.subdivide(sc["color"][m], n)
        for p in range(4):
            q = 4 * s + p
            assert np.abs(got["ctrl"][q] - want[p]).max() <= 2e-6 * max(ext, 1e-3) + 2e-6 * np.abs(c).max()
            assert np.abs(got["color"][q] - want_col[p]).max() <= 2e-6
            assert got["opacity"][q] == sc["opacity"][m] and got["r_b"][q] == sc["r_b"][m]
            assert np.array_equal(got["log_scale"][q], sc["log_scale"][m])
            assert np.array_equal(got["quat"][q], sc["quat"][m])
            assert np.array_equal(got["sh"][q], sc["sh"][m])


def test_subdivision_resamples_attribute_maps(oracle):
    import torch
    from oracle import split as S
    from paper_2503_13961_gb300 import render as R
    from paper_2503_13961_gb300 import scenes
    sc = scenes.with_attribute_maps(scenes.mixed_shapes_scene(50, 2, seed=21), 3, seed=4)
    dev = _dev(sc)
    sel = np.arange(0, 50, 7, dtype=np.int32)
    out = R.subdivide(dev, torch.as_tensor(sel, device="cuda"))
    torch.cuda.synchronize()
    ls, qt = out["log_scale"].cpu().numpy(), out["quat"].cpu().numpy()
    assert ls.shape == (4 * len(sel), 6, 3) and qt.shape == (4 * len(sel), 6, 4)
    for s, m in enumerate(sel):
        wl = S.subdivide_map(sc["log_scale"][m], 3, oracle.attr_weights)
        wq = S.subdivide_map(sc["quat"][m], 3, oracle.attr_weights)
        for p in range(4):
            assert np.abs(ls[4 * s + p] - wl[p]).max() < 2e-6
            assert np.abs(qt[4 * s + p] - wq[p]).max() < 2e-6


def test_invalid_indices_and_empty_selection():
    import torch
    from paper_2503_13961_gb300 import render as R
    from paper_2503_13961_gb300 import scenes
    dev = _dev(scenes.mixed_shapes_scene(8, 2, seed=1))
    out = R.subdivide(dev, torch.as_tensor([3, -1, 8], dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    c = out["ctrl"].cpu().numpy()
    assert np.isfinite(c[0:4]).all()
    assert np.isnan(c[4:12]).all() and np.isnan(out["opacity"].cpu().numpy()[4:12]).all()
    empty = R.subdivide(dev, torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert empty["ctrl"].shape[0] == 0


def test_full_size_room_split_sampled_and_rendered(scenes):
    # the config-5 room: 100,000 degree-3 primitives; every one split (400,000
    # pieces), measures of all, sampled against the oracle; the split scene
    # renders through the same library
    import torch
    from oracle import split as S
    from paper_2503_13961_gb300 import render as R
    sc, cams = scenes.config_scene(5)[:2]
    n = sc["degree"]
    dev = _dev(sc)
    M = sc["ctrl"].shape[0]
    met = R.prim_metrics(dev)
    out = R.subdivide(dev, torch.arange(M, dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    area = met["area"].cpu().numpy()
    rng = np.random.default_rng(8)
    for m in rng.choice(M, 300, replace=False):
        c = sc["ctrl"][m].astype(np.float64)
        ref = S.area(c, n)
        assert abs(area[m] - ref) <= REL * ref + _tolerances(c, n, 1.0)[0]
        want = S.subdivide(c, n)
        got = out["ctrl"][4 * m:4 * m + 4].cpu().numpy()
        assert np.abs(got - want).max() <= 4e-6 * np.abs(c).max()
    # renders: a 400 x 300 window of the first view of the split scene
    small = scenes.crop_camera(cams[0], 600, 450, 400, 300)
    rd = R.Renderer(degree=n, max_prims=4 * M, max_views=1, max_pixels=400 * 300,
                    max_pairs=64 * 400 * 300, max_boundary_pairs=64 * 400 * 300)
    img = rd.forward(out, [small])
    rd.sync_status()
    assert torch.isfinite(img).all() and float(img.abs().sum()) > 0
    rd.close()


def test_pieces_of_flat_patches_share_the_area():
    import torch
    from paper_2503_13961_gb300 import render as R
    from paper_2503_13961_gb300 import scenes
    sc = scenes.mixed_shapes_scene(300, 3, seed=30, curve=0.0)
    dev = _dev(sc)
    out = R.subdivide(dev, torch.arange(300, dtype=torch.int32, device="cuda"))
    a1 = R.prim_metrics(dev)["area"].double().cpu().numpy()
    a2 = R.prim_metrics(out)["area"].double().view(300, 4).cpu().numpy()
    # each piece of a flat patch is a quarter of it, within the FP32 position error
    for m in range(300):
        c = sc["ctrl"][m].astype(np.float64)
        tol = 1e-5 * a1[m] + 2 * _tolerances(c, 3, 1.0)[0]
        assert np.abs(a2[m] - a1[m] / 4).max() <= tol, (m, a2[m], a1[m])


def _expected_masks(cells, M, words):
    want = np.zeros((M, words), np.uint64)
    for m, cs in enumerate(cells):
        for c in cs:
            want[m, c >> 6] |= np.uint64(1) << np.uint64(c & 63)
    return want


def test_visibility_measures_match_the_oracle(oracle, scenes):
    # 8 views of mixed size of the benchmark scene in one forward: the views
    # each primitive is seen in and its visibility texture, bit-exact (the
    # raster is); a second forward of 8 other views accumulates; the
    # occlusion flags follow the oracle's ratios
    import torch
    from oracle import split as S
    from paper_2503_13961_gb300 import render as R
    from tests.gpu_util import make_renderer
    sc, cams = scenes.config_scene(4)
    M = sc["ctrl"].shape[0]
    dev = _dev(sc)
    rd = make_renderer(sc, cams[:16])  # capacities of both forwards
    vc = cm = None
    rasters = []
    for part in (cams[:8], cams[8:16]):
        rd.forward(dev, part)
        rd.sync_status()
        vc, cm = rd.visibility(M, vc, cm)
        rasters += [oracle.raster(sc, c)[0::2] for c in part]
        count, cells = S.visibility(rasters, M)
        torch.cuda.synchronize()
        assert np.array_equal(vc.cpu().numpy(), count)
        assert np.array_equal(cm.cpu().numpy().view(np.uint64), _expected_masks(cells, M, 2))
    assert 0 < int((count > 0).sum()) < M  # some primitives seen, some hidden
    out = R.prim_metrics(dev, view_count=vc, n_views=16, cell_mask=cm, tess_level=8)
    torch.cuda.synchronize()
    flags = out["flags"].cpu().numpy()
    by_v, by_a = S.occluded(count, 16, cells)
    assert np.array_equal((flags & 4) != 0, np.array(by_v))
    assert np.array_equal((flags & 8) != 0, np.array(by_a))
    assert 0 < int(np.sum(by_a)) < M
    rd.close()


def test_visibility_over_more_than_64_views(oracle, scenes):
    # 140 small views in one forward: the view bits go in groups of 64, and
    # primitives are seen in more than 64 of them
    import torch
    from oracle import split as S
    from tests.gpu_util import make_renderer
    sc, _ = scenes.config_scene(1)
    rng = np.random.default_rng(12)
    cams = scenes.make_views(rng, [(32, 24)] * 140, 3.0, 4.5)
    M = sc["ctrl"].shape[0]
    dev = _dev(sc)
    rd = make_renderer(sc, cams)
    rd.forward(dev, cams)
    rd.sync_status()
    vc, cm = rd.visibility(M)
    torch.cuda.synchronize()
    count, cells = S.visibility([oracle.raster(sc, c)[0::2] for c in cams], M)
    assert np.array_equal(vc.cpu().numpy(), count) and int(count.max()) > 64
    assert np.array_equal(cm.cpu().numpy().view(np.uint64), _expected_masks(cells, M, 2))
    rd.close()


def test_edge_prior_matches_the_oracle(oracle, scenes):
    # training images of 6 views of the benchmark scene: edge magnitudes per
    # pixel, their back-projection onto the primitives through I_id, and the
    # split flag of the edge prior
    import torch
    from oracle import split as S
    from paper_2503_13961_gb300 import render as R
    from tests.gpu_util import make_renderer
    sc, cams = scenes.config_scene(4)
    cams = cams[:6]
    M = sc["ctrl"].shape[0]
    rng = np.random.default_rng(31)
    imgs = [scenes.photo_pair(rng, c["width"], c["height"])[0] for c in cams]
    train = torch.as_tensor(np.concatenate([i.reshape(-1, 3) for i in imgs]), device="cuda")
    edges = R.edge_magnitude(train, cams)
    torch.cuda.synchronize()
    got = edges.cpu().numpy().astype(np.float64)
    off = 0
    per_view = []
    for c, img in zip(cams, imgs):
        n = c["width"] * c["height"]
        want = S.edge_magnitude(img)
        g = got[off:off + n].reshape(want.shape)
        assert np.all(np.abs(g - want) <= 1e-5 * want + 2e-3), c["width"]
        per_view.append(g)
        off += n
    dev = _dev(sc)
    rd = make_renderer(sc, cams)
    rd.forward(dev, cams)
    rd.sync_status()
    es, ec = rd.edge_prior(edges, M)
    torch.cuda.synchronize()
    ids = [oracle.raster(sc, c)[0] for c in cams]
    s_ref, n_ref = S.edge_prior(ids, per_view, M)
    assert np.array_equal(ec.cpu().numpy(), n_ref)
    es = es.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(es - s_ref) <= 1e-5 * s_ref + 1e-3)
    out = R.prim_metrics(dev, edge_sum=torch.as_tensor(es, dtype=torch.float32, device="cuda"),
                         edge_count=ec)
    torch.cuda.synchronize()
    split = (out["flags"].cpu().numpy() & 2) != 0
    want = np.array(S.split_by_edges(s_ref, n_ref))
    avg = s_ref / np.maximum(n_ref, 1)
    far = np.abs(avg - S.TAU_B) > 1e-4 * S.TAU_B
    assert np.array_equal(split[far], want[far])
    assert 100 < int(want.sum()) < int((n_ref > 0).sum()) - 100
    rd.close()
