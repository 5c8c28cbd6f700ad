"""Pins of the oracle's attribute maps (Sec. 3.2, Eq. 5): the texture
interpolation Theta on a triangular texel grid of leg resolution R, and the
sub-primitive attributes it feeds.

Theta interpolates linearly on the triangle of the level-(R - 1) barycentric
lattice that holds (u, v); texel (i, j) sits at (i, j) / (R - 1) in the
control-point order. It must return a texel's value at its node, reproduce
every affine function of (u, v) exactly, and use non-negative weights that
sum to one.
"""
import numpy as np
import pytest


def _nodes(R):
    n = R - 1
    out = []
    for i in range(n, -1, -1):
        for j in range(n - i, -1, -1):
            out.append((i, j))
    return out


@pytest.mark.parametrize("R", [2, 3, 4, 6])
def test_texels_sit_at_lattice_nodes_in_control_point_order(oracle, R):
    n = R - 1
    for t, (i, j) in enumerate(_nodes(R)):
        idx, w = oracle.attr_weights(R, i / n, j / n)
        got = np.zeros(R * (R + 1) // 2)
        np.add.at(got, idx, w)
        want = np.zeros_like(got)
        want[t] = 1.0
        assert np.allclose(got, want, atol=1e-12), (R, i, j)
    # the corner u = 1 is texel 0, like control point p_n00
    idx, w = oracle.attr_weights(R, 1.0, 0.0)
    assert idx[np.argmax(w)] == 0


@pytest.mark.parametrize("R", [1, 2, 3, 5])
def test_affine_fields_are_reproduced_exactly(oracle, R):
    rng = np.random.default_rng(R)
    a, b, c = rng.normal(size=3)
    n = max(R - 1, 1)
    nodes = _nodes(R)
    tex = np.array([a + b * i / n + c * j / n for i, j in nodes]) if R > 1 else np.array([a])
    for _ in range(200):
        u, v = rng.uniform(size=2)
        if u + v > 1.0:
            u, v = 1.0 - u, 1.0 - v
        idx, w = oracle.attr_weights(R, u, v)
        assert np.all(w >= -1e-15) and abs(w.sum() - 1.0) < 1e-12
        val = float((w * tex[idx]).sum())
        want = a + b * u + c * v if R > 1 else a
        assert abs(val - want) < 1e-12
    # edges of the simplex (u + v = 1, u = 0, v = 0)
    for t in np.linspace(0.0, 1.0, 11):
        for u, v in ((t, 1.0 - t), (0.0, t), (t, 0.0)):
            idx, w = oracle.attr_weights(R, u, v)
            val = float((w * tex[idx]).sum())
            want = a + b * u + c * v if R > 1 else a
            assert abs(val - want) < 1e-12


def test_replicated_texels_render_like_one_texel(oracle, scenes):
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(48, 44), r_b=2e-2)
    ref = oracle.render(sc, cams[0])
    s3 = dict(sc, attr_res=3)
    s3["log_scale"] = np.repeat(np.asarray(sc["log_scale"])[:, None, :], 6, axis=1)
    s3["quat"] = np.repeat(np.asarray(sc["quat"])[:, None, :], 6, axis=1)
    got = oracle.render(s3, cams[0])
    assert np.abs(got["image"] - ref["image"]).max() < 1e-12


def test_maps_vary_the_sub_primitives(oracle, scenes):
    # not vacuous: noisy maps change the rendered image
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(48, 44), r_b=2e-2)
    ref = oracle.render(sc, cams[0])
    got = oracle.render(scenes.with_attribute_maps(sc, 3), cams[0])
    assert np.abs(got["image"] - ref["image"]).max() > 1e-3
