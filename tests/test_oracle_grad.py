"""Pin of the oracle's analytic backward (supplementary "Backward Derivative"
plus the projection / EWA chain rule) against FP64 central finite differences
of the oracle's own forward pass with the raster frozen (I_id, I_uv, B fixed,
as the paper treats them).

A finite-difference step is discarded (and another parameter drawn) when
either side flips any per-pixel discrete decision (survivor set, order,
alpha_max clamp, stop point, most influential boundary point, gamma
saturation); the oracle reports these as a decision hash. Pixels whose
boundary distance |q - b*| is below 1e-2 px are given zero upstream gradient:
at d -> 0 the term |q - b| of Eq. 6 has a cusp and central differences with
h = 1e-6 lose accuracy there.
"""
import numpy as np
import pytest

H_STEP = 1e-6


def fd_check(oracle, scene, cam, opts, nparams, seed, kinds=("ctrl", "color", "opacity", "r_b")):
    opts = dict(opts, tol_d=1e-2)
    idm, uv, _ = oracle.raster(scene, cam)
    rng = np.random.default_rng(seed)
    W, H = cam["width"], cam["height"]
    dl = rng.normal(size=(H, W, 3))
    base = oracle.render(scene, cam, idm, uv, opts=opts)
    dl[base["flags"] != 0] = 0.0
    g = oracle.backward(scene, cam, dl, idm, uv, opts=opts)
    s64 = oracle.scene_to64(scene)
    M, m = s64["ctrl"].shape[:2]
    out = []
    tries = 0
    while len(out) < nparams and tries < 20 * nparams:
        kind = kinds[tries % len(kinds)]
        tries += 1
        if kind in ("ctrl", "color"):
            idx = (int(rng.integers(M)), int(rng.integers(m)), int(rng.integers(3)))
        elif kind in ("log_scale", "quat", "sh"):
            shp = s64[kind].shape
            idx = tuple(int(rng.integers(d)) for d in shp)
        else:
            idx = (int(rng.integers(M)),)
        vals = []
        for sgn in (1.0, -1.0):
            s2 = {k: v.copy() for k, v in s64.items()}
            s2[kind][idx] += sgn * H_STEP
            r = oracle.render(scene, cam, idm, uv, opts=opts, scene64=s2)
            if r["hash"] != base["hash"]:
                break
            vals.append(float((r["image"] * dl).sum()))
        if len(vals) < 2:
            continue
        out.append((kind, idx, float(g[kind][idx]), (vals[0] - vals[1]) / (2 * H_STEP)))
    return out, g


CASES = [
    ("octa", {}, 0.05, (48, 40), 3e-2),
    ("octa", {"use_boundary": 0}, 0.05, (48, 40), 1e-2),
    ("two", {}, 0.0, (40, 40), 1e-1),
    ("ico1", {}, 0.04, (44, 44), 2e-2),
]


@pytest.mark.parametrize("kind,opts,noise,size,r_b", CASES)
def test_analytic_gradient_matches_central_differences(oracle, scenes, kind, opts, noise, size, r_b):
    sc, cams = scenes.tiny_scene(kind, noise=noise, size=size, r_b=r_b)
    res, g = fd_check(oracle, sc, cams[0], opts, 48, seed=hash(kind) % 1000)
    assert len(res) >= 40
    gmax = max(abs(r[3]) for r in res)
    for kind_, idx, an, num in res:
        err = abs(an - num) / max(abs(num), 1e-3 * gmax)
        assert err < 1e-5, (kind_, idx, an, num)
    # not vacuous: every parameter kind received a non-zero gradient
    assert all(np.abs(g[k]).max() > 0 for k in ("ctrl", "color", "opacity"))
    if opts.get("use_boundary", 1):
        assert np.abs(g["r_b"]).max() > 0
    else:
        assert np.abs(g["r_b"]).max() == 0


def test_config1_gradient(oracle, scenes):
    sc, cams = scenes.config_scene(1)
    res, _ = fd_check(oracle, sc, cams[0], {}, 40, seed=7)
    gmax = max(abs(r[3]) for r in res)
    assert gmax > 0
    for kind_, idx, an, num in res:
        assert abs(an - num) <= 1e-5 * max(abs(num), 1e-3 * gmax), (kind_, idx, an, num)


@pytest.mark.parametrize("R", [1, 3])
def test_attribute_map_gradients_match_central_differences(oracle, scenes, R):
    """Rotation and scaling attribute maps (Eq. 5, leg resolution R): the
    analytic gradient of the maps' texels through Sigma3D, EWA and the blending
    equals central differences of the oracle's forward pass."""
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(44, 44), r_b=2e-2)
    sc = scenes.with_attribute_maps(sc, R, seed=R)
    res, g = fd_check(oracle, sc, cams[0], {}, 40, seed=7 + R,
                      kinds=("log_scale", "quat", "log_scale", "quat", "ctrl", "color"))
    assert len(res) >= 32
    gmax = max(abs(r[3]) for r in res)
    for kind_, idx, an, num in res:
        err = abs(an - num) / max(abs(num), 1e-3 * gmax)
        assert err < 1e-5, (kind_, idx, an, num)
    assert np.abs(g["log_scale"]).max() > 0 and np.abs(g["quat"]).max() > 0
