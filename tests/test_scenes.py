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
