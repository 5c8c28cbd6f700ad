"""The seeded generator produces the five workloads with the stated sizes."""
import numpy as np
import pytest


@pytest.mark.parametrize("cfg,M,n,views,size", [
    (1, 16, 2, 1, (64, 64)), (2, 2000, 2, 1, (800, 800)), (3, 20000, 2, 1, (1024, 1024)),
])
def test_config_sizes(scenes, cfg, M, n, views, size):
    out = scenes.config_scene(cfg)
    sc, cams = out[0], out[1]
    assert sc["ctrl"].shape == (M, scenes.ncp(n), 3) and sc["degree"] == n
    assert sc["ctrl"].dtype == np.float32
    assert len(cams) == views and (cams[0]["width"], cams[0]["height"]) == size
    assert np.all((sc["opacity"] >= 0.5) & (sc["opacity"] <= 1.0))


def test_config4_views(scenes):
    sc, cams = scenes.config_scene(4)
    assert len(cams) == 64 and sc["ctrl"].shape[0] == 20000
    assert {c["width"] for c in cams} <= {256, 512, 800, 1024}
    for c in cams:
        eye = -np.asarray(c["R"], np.float64).T @ np.asarray(c["t"], np.float64)
        assert 3.5 - 1e-4 <= np.linalg.norm(eye) <= 5.0 + 1e-4


def test_seeded_and_deterministic(scenes):
    a = scenes.config_scene(2)[0]
    b = scenes.config_scene(2)[0]
    assert all(np.array_equal(a[k], b[k]) for k in ("ctrl", "color", "opacity"))
    c = scenes.config_scene(2, seed=1)[0]
    assert not np.array_equal(a["ctrl"], c["ctrl"])


def test_shared_edges_share_control_points(scenes):
    # edge control points are drawn once per edge, so neighbouring patches meet
    sc, _ = scenes.config_scene(1)
    pts = sc["ctrl"].reshape(-1, 3)
    uniq = np.unique(np.round(pts, 6), axis=0)
    assert len(uniq) < len(pts)


def test_random_gaussians_have_ties(scenes):
    g = scenes.random_gaussians(0, 40, 30, 400)
    assert len(np.unique(g["depth"])) < 400


def test_photo_pairs_are_seeded_and_in_range(scenes):
    import numpy as np
    a = scenes.photo_pair(np.random.default_rng(3), 37, 21)
    b = scenes.photo_pair(np.random.default_rng(3), 37, 21)
    for x, y in zip(a, b):
        assert x.shape == (21, 37, 3) and x.dtype == np.float32 and np.array_equal(x, y)
        assert x.min() >= 0.0 and x.max() <= 1.0
    img, gt = a
    assert np.abs(img - gt).max() > 0  # the target differs from the image
    assert np.array_equal(gt[7], np.broadcast_to(gt[7, 0], gt[7].shape))  # a flat stripe every seventh row


def test_mixed_shapes_cover_the_prune_thresholds(scenes):
    import numpy as np
    sc = scenes.mixed_shapes_scene(300, 2, seed=4)
    assert sc["ctrl"].shape == (300, 6, 3) and sc["color"].shape == (300, 6, 3)
    assert np.array_equal(sc["ctrl"], scenes.mixed_shapes_scene(300, 2, seed=4)["ctrl"])
    corners = sc["ctrl"][:, [0, 3, 5]].astype(np.float64)
    edge = np.linalg.norm(corners[:, 1] - corners[:, 0], axis=1)
    # edges spread over three decades: tiny and large primitives both present
    assert edge.min() < 1e-2 and edge.max() > 0.3
    assert (sc["r_b"] >= 5e-3).all() and (sc["r_b"] <= 2e-2).all()
