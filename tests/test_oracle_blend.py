"""Pins of the oracle's sub-primitives and discontinuity-aware blending
(Sec. 3.2, Eq. 3-8; supplementary blending equations).

Expected values come from the paper's stated values of gamma (golden file),
textbook special cases of the EWA projection, explicit products
prod_j (1 - alpha_j) written out per pixel, and the qualitative statements of
Fig. 4.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def test_gamma_matches_paper_values(oracle):
    for d, sigma, g in _load_golden("gamma_eq7.txt"):
        assert abs(oracle.gamma(d, sigma) - g) < 1e-15


def test_gamma_monotone_and_continuous_at_sigma(oracle):
    ds = np.linspace(0, 3, 301)
    g = np.array([oracle.gamma(d, 1.3) for d in ds])
    assert np.all(np.diff(g) >= 0)
    assert g.min() == 0.5 and g.max() == 1.0
    assert abs(oracle.gamma(1.3 * (1 - 1e-9), 1.3) - 1.0) < 1e-8


def _pix_xy(rec, W):
    p = rec[:, 0].astype(int)
    return p % W, p // W


@pytest.mark.parametrize("kind", ["octa", "ico1"])
def test_ewa_isotropic_closed_form(oracle, scenes, kind):
    # Isotropic 3D Gaussian (identity rotation, scale s): Sigma2D = s^2 J J^T + dil I
    # with J the pinhole Jacobian at the Gaussian's camera-space point. The
    # camera rotation is FP32-rounded, so W W^T = I holds to ~1e-7 only.
    sc, cams = scenes.tiny_scene(kind, noise=0.03, size=(40, 36))
    cam = cams[0]
    out = oracle.render(sc, cam, records=True)
    g = out["gauss"]
    assert len(g) > 50
    s = math.exp(float(sc["log_scale"][0, 0]))
    fx, fy, cx, cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    z = g[:, 7]
    tx = (g[:, 2] - cx) * z / fx
    ty = (g[:, 3] - cy) * z / fy
    J00, J02 = fx / z, -fx * tx / z ** 2
    J11, J12 = fy / z, -fy * ty / z ** 2
    dil = oracle.DEFAULTS["dilation"]
    A = s * s * (J00 ** 2 + J02 ** 2) + dil
    B = s * s * (J02 * J12)
    C = s * s * (J11 ** 2 + J12 ** 2) + dil
    det = A * C - B * B
    assert np.allclose(g[:, 4], C / det, rtol=1e-6)
    assert np.allclose(g[:, 5], -B / det, rtol=1e-6, atol=1e-7)
    assert np.allclose(g[:, 6], A / det, rtol=1e-6)


def test_ewa_quaternion_rotation_swaps_axes(oracle, scenes):
    # A 90 degree rotation about world z maps the scale axes x <-> y, so an
    # anisotropic Gaussian (sx, sy, sz) rotated that way equals the
    # unrotated Gaussian with scales (sy, sx, sz).
    sc, cams = scenes.tiny_scene("ico1", noise=0.02, size=(40, 36))
    cam = cams[0]
    a = dict(sc)
    a["log_scale"] = np.tile(np.log(np.array([0.02, 0.05, 0.08], np.float32)), (len(sc["opacity"]), 1))
    b = dict(a)
    b["log_scale"] = np.tile(np.log(np.array([0.05, 0.02, 0.08], np.float32)), (len(sc["opacity"]), 1))
    a["quat"] = np.tile(np.array([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)], np.float32),
                        (len(sc["opacity"]), 1))
    ga = oracle.render(a, cam, records=True)["gauss"]
    gb = oracle.render(b, cam, records=True)["gauss"]
    assert np.allclose(ga[:, 4:7], gb[:, 4:7], rtol=1e-6)


def _tiny_tri_scene(scenes, centres, W=16, H=16, depths=None, opacity=0.9, colors=None, size=0.45):
    """Flat triangles facing a camera at (4,0,0), each around a pixel centre."""
    cam = scenes.look_at_camera((4.0, 0.0, 0.0), (0, 0, 0), W, H)
    fx, cx, cy = float(cam["fx"]), float(cam["cx"]), float(cam["cy"])
    tris = []
    for i, (px, py) in enumerate(centres):
        X = 0.0 if depths is None else depths[i]
        dist = 4.0 - X
        pts = []
        for ox, oy in ((-size, -size * 0.8), (size * 1.1, -size * 0.6), (-size * 0.2, size * 1.2)):
            Y = (px + ox - cx) * dist / fx
            Z = -(py + oy - cy) * dist / fx
            pts.append((X, Y, Z))
        tris.append(pts)
    sc = scenes.triangles_scene(tris, n=2, opacity=opacity, gauss_scale=0.7 * 4.0 / fx)
    if colors is not None:
        sc["color"][:] = np.asarray(colors, np.float32)[:, None, :]
    return sc, cam


def test_opacity_zero_renders_background(oracle, scenes):
    sc, cams = scenes.tiny_scene("octa", noise=0.05, size=(32, 32))
    sc = dict(sc)
    sc["opacity"] = np.zeros_like(sc["opacity"])
    sc["bg"] = np.array([0.2, 0.5, 0.9], np.float32)
    img = oracle.render(sc, cams[0])["image"]
    assert np.array_equal(img, np.broadcast_to(sc["bg"].astype(np.float64), img.shape))


def test_single_gaussian_closed_form(oracle, scenes):
    # one flat triangle covering exactly one pixel centre -> one Gaussian;
    # without boundary term (w = 1): C = alpha c + (1 - alpha) bg,
    # alpha = o exp(-1/2 d^T K d) where >= alpha_min, else C = bg.
    sc, cam = _tiny_tri_scene(scenes, [(7.0, 8.0)], opacity=0.8, colors=[(0.9, 0.3, 0.1)])
    sc["bg"] = np.array([0.1, 0.2, 0.3], np.float32)
    out = oracle.render(sc, cam, opts={"use_boundary": 0}, records=True)
    assert out["F"] == 1
    g = out["gauss"][0]
    ys, xs = np.mgrid[0:16, 0:16]
    dx, dy = xs - g[2], ys - g[3]
    o = float(sc["opacity"][0])
    a = o * np.exp(-0.5 * (g[4] * dx * dx + g[6] * dy * dy) - g[5] * dx * dy)
    a = np.where(a >= oracle.DEFAULTS["alpha_min"], np.minimum(a, oracle.DEFAULTS["alpha_max"]), 0.0)
    c = sc["color"][0, 0].astype(np.float64)
    bg = sc["bg"].astype(np.float64)
    expect = a[..., None] * c + (1 - a[..., None]) * bg
    assert np.abs(out["image"] - expect).max() < 1e-12
    assert (a > 0).sum() > 9


def _brute_force(oracle, sc, cam, out, use_boundary):
    """Explicit products over the depth-sorted survivors of every pixel."""
    W, H = cam["width"], cam["height"]
    g = out["gauss"]
    F = len(g)
    am, aM, ts = (oracle.DEFAULTS[k] for k in ("alpha_min", "alpha_max", "t_stop"))
    bg = sc["bg"].astype(np.float64)
    img = np.zeros((H, W, 3))
    for y in range(H):
        for x in range(W):
            p = y * W + x
            if use_boundary:
                w, _ = oracle.wvalues(sc, cam, [p] * F, g[:, 1].astype(int), out["id"], out["uv"])
            else:
                w = np.ones(F)
            dx, dy = x - g[:, 2], y - g[:, 3]
            G = np.exp(-0.5 * (g[:, 4] * dx * dx + g[:, 6] * dy * dy) - g[:, 5] * dx * dy)
            a = np.minimum(g[:, 11] * w * G, aM)
            keep = [i for i in range(F) if a[i] >= am]
            keep.sort(key=lambda i: (g[i, 7], i))
            used = []
            for i in keep:
                prod = np.prod([1 - a[j] for j in used + [i]])
                if prod < ts:
                    break
                used.append(i)
            C = np.zeros(3)
            for k, i in enumerate(used):
                C += np.prod([1 - a[j] for j in used[:k]]) * a[i] * g[i, 8:11]
            C += np.prod([1 - a[j] for j in used]) * bg
            img[y, x] = C
    return img


@pytest.mark.parametrize("use_boundary", [0, 1])
def test_brute_force_products_few_gaussians(oracle, scenes, use_boundary):
    # Two overlapping triangles at different depths (3 + 1 covered pixels),
    # opacity 1 so that alpha_max clamps at the centres.
    sc, cam = _tiny_tri_scene(scenes, [(3.0, 4.0), (4.0, 4.0)], W=8, H=8, depths=[0.0, 0.7],
                              opacity=1.0, colors=[(1, 0, 0), (0, 0, 1)], size=0.9)
    sc["r_b"][:] = 0.05
    out = oracle.render(sc, cam, opts={"use_boundary": use_boundary}, records=True)
    assert 2 <= out["F"] <= 6
    expect = _brute_force(oracle, sc, cam, out, use_boundary)
    assert np.abs(out["image"] - expect).max() < 1e-13


def test_fig4_scenario(oracle, scenes):
    # Fig. 4: R_a, R_b share an edge; G_c belongs to a primitive far away.
    # p1 inside R_a near the shared edge: w from R_a's Gaussian > w from R_b's.
    # p2 deep inside R_b: Gaussians of R_a and of the far primitive get w = 0,
    # R_b's own get w = 1.
    sc, cams = scenes.tiny_scene("two", n=2, size=(64, 64), r_b=0.05)
    cam = cams[0]
    idm, uv, _ = oracle.raster(sc, cam)
    W = cam["width"]
    ya, xa = np.nonzero(idm == 0)
    yb, xb = np.nonzero(idm == 1)
    # p1: pixel of R_a adjacent (4-neighbour) to R_b
    p1 = None
    for x, y in zip(xa, ya):
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            if 0 <= x + dx < W and 0 <= y + dy < cam["height"] and idm[y + dy, x + dx] == 1:
                p1 = y * W + x
        if p1 is not None:
            break
    assert p1 is not None
    # p2: pixel of R_b farthest from any other id
    far = [(min(np.hypot(xb - x, yb - y).max(), 99), 0) for x, y in [(0, 0)]]
    dist = np.full(idm.shape, np.inf)
    oy, ox = np.nonzero(idm != 1)
    for x, y in zip(xb, yb):
        dist[y, x] = np.min(np.hypot(ox - x, oy - y))
    y2, x2 = np.unravel_index(np.argmax(np.where(np.isfinite(dist), dist, -1)), dist.shape)
    p2 = y2 * W + x2
    assert dist[y2, x2] > 4
    w, _ = oracle.wvalues(sc, cam, [p1, p1, p2, p2, p2], [0, 1, 0, 2, 1], idm, uv)
    assert w[0] > w[1]
    assert 0.5 <= w[0] <= 1.0 and 0.0 <= w[1] <= 0.5
    assert w[2] == 0.0 and w[3] == 0.0 and w[4] == 1.0
    del far


def test_w_transitions_from_one_to_zero_across_edge(oracle, scenes):
    # Sec. 3.2 after Eq. 7: w goes from 1 to 0 across the boundary region.
    sc, cams = scenes.tiny_scene("two", n=2, size=(64, 64), r_b=0.08)
    cam = cams[0]
    idm, uv, _ = oracle.raster(sc, cam)
    W = cam["width"]
    row = 32
    xs = np.arange(W)
    ids = idm[row]
    sel = (ids == 0) | (ids == 1)
    pix = (row * W + xs[sel]).tolist()
    w, _ = oracle.wvalues(sc, cam, pix, [0] * len(pix), idm, uv)
    idr = ids[sel]
    assert np.all(w[idr == 0] >= 0.5) and np.all(w[idr == 1] <= 0.5)
    assert w.max() == 1.0 and w.min() == 0.0
    # values step through (0, 1) near the edge
    assert np.any((w > 0.05) & (w < 0.95))
