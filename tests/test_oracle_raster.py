"""Pins of the oracle's tessellation + rasterization (Sec. 3.2, "Tessellation
and Rasterization") and boundary set B.

The expected values come from closed-form geometry computed here in FP64:
point-in-triangle tests against exactly projected vertices, ray-plane
intersections for the depth test and for barycentric interpolation.
Only pixels closer to an edge than the 1/256-pixel snapping can move are
exempt.
"""
import numpy as np
import pytest

SNAP = 2.0 / 256.0  # a snapped vertex moves by at most 0.5/256 px per axis


def _project(cam, P):
    R = np.asarray(cam["R"], np.float64)
    t = np.asarray(cam["t"], np.float64)
    X = P @ R.T + t
    x = float(cam["fx"]) * X[:, 0] / X[:, 2] + float(cam["cx"])
    y = float(cam["fy"]) * X[:, 1] / X[:, 2] + float(cam["cy"])
    return np.stack([x, y], 1), X[:, 2]


def _pix_grid(cam):
    W, H = cam["width"], cam["height"]
    ys, xs = np.mgrid[0:H, 0:W]
    return xs.astype(np.float64), ys.astype(np.float64)


def _edge_dist(xs, ys, a, b):
    """Signed distance of pixel centres to the line a->b."""
    d = b - a
    return (d[0] * (ys - a[1]) - d[1] * (xs - a[0])) / np.hypot(*d)


def _inside_tri(xs, ys, v):
    d = [_edge_dist(xs, ys, v[i], v[(i + 1) % 3]) for i in range(3)]
    area = (v[1][0] - v[0][0]) * (v[2][1] - v[0][1]) - (v[1][1] - v[0][1]) * (v[2][0] - v[0][0])
    s = 1.0 if area > 0 else -1.0
    dd = np.stack([s * x for x in d])
    return dd.min(0), np.abs(dd).min(0)


@pytest.mark.parametrize("level", [1, 3, 8])
def test_flat_triangle_coverage_matches_point_in_triangle(oracle, scenes, level):
    sc, cams = scenes.tiny_scene("one", n=1, size=(61, 47))
    cam = cams[0]
    idm, uv, _ = oracle.raster(sc, cam, tess_level=level)
    v, _ = _project(cam, sc["ctrl"][0].astype(np.float64))
    xs, ys = _pix_grid(cam)
    mind, absd = _inside_tri(xs, ys, v)
    expect = mind > 0
    ok = (idm >= 0) == expect
    assert np.all(ok | (absd < SNAP)), "coverage differs away from the edges"
    assert expect.sum() > 150


def test_shared_edges_are_watertight(oracle, scenes):
    # a square split into two triangles, each tessellated at level 8: every
    # pixel inside the square is covered by exactly one flat triangle.
    sc, cams = scenes.tiny_scene("two", n=1, size=(53, 53))
    cam = cams[0]
    sc = dict(sc)
    for k in ("ctrl", "color", "opacity", "r_b", "log_scale", "quat"):
        sc[k] = sc[k][:2]
    _, _, _, cover = oracle.raster(sc, cam, ztest=False, cover=True)
    v, _ = _project(cam, np.array([[0, -0.8, -0.8], [0, 0.8, -0.8], [0, 0.8, 0.8], [0, -0.8, 0.8]], float))
    xs, ys = _pix_grid(cam)
    dists = [_edge_dist(xs, ys, v[i], v[(i + 1) % 4]) for i in range(4)]
    sgn = np.sign(np.mean([d[26, 26] for d in dists]))
    inner = np.min(np.stack([sgn * d for d in dists]), 0)
    assert np.all(cover[inner > SNAP] == 1)
    assert np.all(cover[inner < -SNAP] == 0)
    assert (inner > SNAP).sum() > 250


def test_pixel_count_matches_projected_area(oracle, scenes):
    sc, cams = scenes.tiny_scene("two", n=2, size=(80, 80))
    cam = cams[0]
    sc = dict(sc)
    for k in ("ctrl", "color", "opacity", "r_b", "log_scale", "quat"):
        sc[k] = sc[k][:2]
    idm, _, _ = oracle.raster(sc, cam)
    v, _ = _project(cam, np.array([[0, -0.8, -0.8], [0, 0.8, -0.8], [0, 0.8, 0.8], [0, -0.8, 0.8]], float))
    x, y = v[:, 0], v[:, 1]
    area = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    perim = np.sum(np.hypot(np.diff(np.r_[x, x[0]]), np.diff(np.r_[y, y[0]])))
    assert abs((idm >= 0).sum() - area) < 0.5 * perim


def test_depth_test_on_crossing_planes(oracle, scenes):
    # triangle A in the plane x = 0, triangle B in the plane x = 0.6 y; they
    # cross along the z axis. The nearer plane along each pixel ray must win.
    A = [(0.0, -1.0, -1.0), (0.0, 1.0, -1.0), (0.0, 0.0, 1.2)]
    B = [(-0.6, -1.0, -0.9), (0.6, 1.0, -0.9), (0.0, 0.0, 1.3)]
    sc = scenes.triangles_scene([A, B], n=2)
    cam = scenes.look_at_camera((4.0, 0.3, 0.2), (0, 0, 0), 70, 64)
    idm, _, _ = oracle.raster(sc, cam)
    R = np.asarray(cam["R"], np.float64)
    t = np.asarray(cam["t"], np.float64)
    eye = -R.T @ t
    xs, ys = _pix_grid(cam)
    dcam = np.stack([(xs - float(cam["cx"])) / float(cam["fx"]), (ys - float(cam["cy"])) / float(cam["fy"]),
                     np.ones_like(xs)], -1)
    dw = dcam @ R  # world ray directions (camera z = 1)
    nA = np.array([1.0, 0.0, 0.0])
    nB = np.array([1.0, -0.6, 0.0])
    sA = -(eye @ nA) / (dw @ nA)  # camera-z of the hit (ray parametrised by camera z)
    sB = -(eye @ nB) / (dw @ nB)
    both = (idm >= 0)
    vA, _ = _project(cam, np.array(A))
    vB, _ = _project(cam, np.array(B))
    mA, aA = _inside_tri(xs, ys, vA)
    mB, aB = _inside_tri(xs, ys, vB)
    inA, inB = mA > SNAP, mB > SNAP
    sel = inA & inB & (np.abs(sA - sB) > 1e-4 * np.abs(sA))
    want = np.where(sA < sB, 0, 1)
    assert sel.sum() > 200
    assert np.all(idm[sel] == want[sel])
    assert np.all(idm[inA & ~inB & (aB > SNAP)] == 0)


def test_perspective_correct_uv_on_flat_triangle(oracle, scenes):
    # On a flat triangle S(I_uv(q)) must be the point the ray of q hits, so it
    # projects back onto the pixel centre, up to the 1/256-px vertex snapping
    # (barycentrics are taken relative to the snapped flat triangle).
    sc, cams = scenes.tiny_scene("one", n=2, size=(64, 48))
    cam = cams[0]
    idm, uv, _ = oracle.raster(sc, cam)
    ys, xs = np.nonzero(idm >= 0)
    ctrl = sc["ctrl"][0].astype(np.float64)
    pts = []
    for x, y in zip(xs, ys):
        u, v = uv[y, x]
        pts.append(oracle.bernstein(2, u, v, 1 - u - v) @ ctrl)
    proj, _ = _project(cam, np.array(pts))
    err = np.abs(proj - np.stack([xs, ys], 1)).max()
    assert err < 1.0 / 256.0, err


def test_boundary_set_follows_the_edges(oracle, scenes):
    # B (4-neighbourhood id change) of two triangles sharing a diagonal and a
    # third one apart: every B pixel lies within one pixel of an edge, and every
    # foreground pixel within 0.7 px of the shared diagonal is in B.
    sc, cams = scenes.tiny_scene("two", n=1, size=(64, 64))
    cam = cams[0]
    idm, uv, _ = oracle.raster(sc, cam)
    out = oracle.render(sc, cam, idm, uv, records=True)
    bpix = out["bnd"][:, 0].astype(int)
    W = cam["width"]
    bx, by = bpix % W, bpix // W
    edges = []
    for t in range(3):
        v, _ = _project(cam, sc["ctrl"][t][[0, 1, 2]].astype(np.float64))
        edges += [(v[i], v[(i + 1) % 3]) for i in range(3)]
    d = np.min(np.stack([np.abs(_edge_dist(bx.astype(float), by.astype(float), a, b)) for a, b in edges]), 0)
    assert np.all(d <= 1.0 + SNAP)
    # shared diagonal of the square: vertices b=(0,.8,-.8) and c=(0,-.8,.8)
    dv, _ = _project(cam, np.array([[0, 0.8, -0.8], [0, -0.8, 0.8]], float))
    xs, ys = _pix_grid(cam)
    near = (np.abs(_edge_dist(xs, ys, dv[0], dv[1])) < 0.7) & (idm >= 0) & (idm <= 1)
    inB = np.zeros_like(idm, bool)
    inB[by, bx] = True
    assert near.sum() > 15
    assert np.all(inB[near])
    # boundary records: bidx order is pixel order, ids match the index map
    assert np.all(np.diff(bpix) > 0)
    assert np.all(out["bnd"][:, 1].astype(int) == idm.ravel()[bpix])


def test_boundary_points_on_flat_surface_project_onto_their_pixels(oracle, scenes):
    # Sec. 3.2: 3D boundary points come from Eq. 3 at I_uv; on a flat
    # primitive they lie on the pixel ray, so b == q (up to the 1/256-px
    # vertex snapping) and sigma = k fx r_b / z.
    sc, cams = scenes.tiny_scene("two", n=2, size=(48, 48), r_b=2e-2)
    cam = cams[0]
    out = oracle.render(sc, cam, records=True)
    b = out["bnd"]
    W = cam["width"]
    q = np.stack([b[:, 0] % W, b[:, 0] // W], 1)
    assert np.abs(b[:, 2:4] - q).max() < 1.0 / 256.0
    sig = 3.0 * float(cam["fx"]) * 2e-2 / b[:, 5]
    assert np.allclose(b[:, 4], sig, rtol=1e-6)
