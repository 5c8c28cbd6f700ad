"""The oracle's box mode (candidate Gaussians limited to their support box,
where o G >= alpha_min can hold) must give exactly the all-pairs result, and
compositing a subset of pixels must give the same values as the full image."""
import numpy as np


def test_box_mode_equals_all_pairs(oracle, scenes):
    for sc, cams in (scenes.config_scene(1), scenes.tiny_scene("two", size=(40, 36), r_b=3e-2),
                     scenes.tiny_scene("ico1", noise=0.04, size=(50, 50))):
        a = oracle.render(sc, cams[0])
        b = oracle.render(sc, cams[0], opts={"all_pairs": 1})
        assert np.array_equal(a["image"], b["image"])
        assert a["hash"] == b["hash"]
        assert np.array_equal(a["n"], b["n"])


def test_pixel_subset_matches_full_image(oracle, scenes):
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(50, 50))
    full = oracle.render(sc, cams[0])
    mask = np.random.default_rng(0).random((50, 50)) < 0.2
    part = oracle.render(sc, cams[0], pixels=mask)
    assert np.array_equal(part["image"][mask], full["image"][mask])


def test_crop_gives_the_same_interior(oracle, scenes):
    # compositing a pixel depends only on nearby pixels: rendering a window of
    # a view as its own camera gives the same colours away from the window's
    # border (the boundary set differs only on that border)
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(64, 64), r_b=1e-2)
    cam = cams[0]
    full = oracle.render(sc, cam)
    crop = scenes.crop_camera(cam, 16, 8, 32, 40)
    part = oracle.render(sc, crop)
    assert np.array_equal(full["id"][8:48, 16:48], part["id"])
    m = 8
    a = full["image"][8:48, 16:48][m:-m, m:-m]
    b = part["image"][m:-m, m:-m]
    assert np.abs(a - b).max() < 1e-12
