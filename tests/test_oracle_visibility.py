"""Pins of the oracle's visibility measures for pruning (Sec. 3.3, the
visibility count over training views and the visibility texture).

A flat triangle facing the camera and covering many pixels is visible in
every view and through all L^2 cells of its lattice; a triangle hidden
behind a larger one is visible nowhere; the cell decoded from the depth key
is the lattice triangle that holds the pixel's I_uv (checked away from cell
borders, an independent computation from the barycentric coordinates).
"""
import numpy as np

from oracle import split as S


def _facing_triangle(scenes, z=0.0, s=1.0):
    # corners in the plane x = z facing a camera on the +x axis
    return [((z, -s, -s), (z, s, -s), (z, 0.0, s))]


def test_facing_triangle_is_fully_visible(oracle, scenes):
    sc = scenes.triangles_scene(_facing_triangle(scenes), n=2)
    cams = [scenes.look_at_camera((4.0, 0.0, 0.0), (0, 0, 0), 256, 256),
            scenes.look_at_camera((4.0, 0.3, 0.2), (0, 0, 0), 200, 180)]
    rasters = [oracle.raster(sc, c)[0::2] for c in cams]
    count, cells = S.visibility(rasters, 1)
    assert count.tolist() == [2]
    up = {2 * (a * 8 + b) for a in range(8) for b in range(8) if a + b <= 7}
    down = {2 * (a * 8 + b) + 1 for a in range(8) for b in range(8) if a + b <= 6}
    assert cells[0] == up | down
    assert len(cells[0]) == 64
    by_v, by_a = S.occluded(count, 2, cells)
    assert by_v == [False] and by_a == [False]


def test_hidden_triangle_is_invisible(oracle, scenes):
    tris = _facing_triangle(scenes, z=0.5, s=2.0) + _facing_triangle(scenes, z=-0.5, s=0.5)
    sc = scenes.triangles_scene(tris, n=1)
    cams = [scenes.look_at_camera((4.0, 0.0, 0.0), (0, 0, 0), 128, 128)]
    count, cells = S.visibility([oracle.raster(sc, c)[0::2] for c in cams], 2)
    assert count.tolist() == [1, 0] and cells[1] == set()
    assert S.occluded(count, 1, cells) == ([False, True], [False, True])
    # seen in 1 of 20 tracked views: below tau_v = 0.08
    assert S.occluded(count, 20, cells)[0] == [True, True]


def test_cell_of_a_pixel_holds_its_uv(oracle, scenes):
    sc = scenes.triangles_scene(_facing_triangle(scenes), n=2)
    cam = scenes.look_at_camera((4.0, 0.2, -0.1), (0, 0, 0), 160, 150)
    idm, uv, key = oracle.raster(sc, cam)
    L = 8
    fg = idm >= 0
    sub = (key[fg] & np.uint64(0xFFFFFFFF)).astype(np.int64) - idm[fg].astype(np.int64) * 2 * L * L
    u, v = uv[fg][:, 0] * L, uv[fg][:, 1] * L
    a, b = np.floor(u), np.floor(v)
    fu, fv = u - a, v - b
    down = (fu + fv > 1).astype(np.int64)
    want = 2 * (a.astype(np.int64) * L + b.astype(np.int64)) + down
    # away from the cell borders the two computations must agree
    far = (np.minimum(np.minimum(fu, fv), np.abs(fu + fv - 1)) > 1e-3) & (fu < 1 - 1e-3) & (fv < 1 - 1e-3)
    assert far.sum() > 1000
    assert np.array_equal(sub[far], want[far])


def test_sobel_edge_magnitude_closed_forms():
    H, W = 12, 10
    # constant image: no edges
    assert np.abs(S.edge_magnitude(np.full((H, W, 3), 0.3))).max() == 0.0
    # a luma ramp of slope s per pixel along x: 8 s inside, 4 s at the replicated border
    s = 0.01
    ramp = np.repeat((s * np.arange(W))[None, :, None], H, axis=0).repeat(3, axis=2)
    e = S.edge_magnitude(ramp)
    assert np.allclose(e[:, 1:-1], 8 * s * 255) and np.allclose(e[:, [0, -1]], 4 * s * 255)
    # a vertical step of luma h: 4 h on the two columns beside it, 0 elsewhere
    step = np.zeros((H, W, 3))
    step[:, 5:] = 0.5
    e = S.edge_magnitude(step)
    assert np.allclose(e[:, 4], 4 * 0.5 * 255) and np.allclose(e[:, 5], 4 * 0.5 * 255)
    assert np.abs(np.delete(e, [4, 5], axis=1)).max() == 0.0
    # transposing the image transposes the magnitude; colour weights are the luma's
    rng = np.random.default_rng(0)
    img = rng.uniform(size=(9, 11, 3))
    assert np.allclose(S.edge_magnitude(img.transpose(1, 0, 2)), S.edge_magnitude(img).T)
    red = np.zeros((H, W, 3))
    red[:, 5:, 0] = 1.0
    assert np.allclose(S.edge_magnitude(red)[:, 4], 4 * 0.299 * 255)


def test_edge_prior_back_projects_through_the_index_map():
    ids = [np.array([[0, 0, 1], [-1, 1, 1]]), np.array([[1, -1, 0], [0, 0, 0]])]
    edges = [np.array([[1.0, 3.0, 5.0], [7.0, 9.0, 11.0]]), np.array([[2.0, 4.0, 6.0], [8.0, 10.0, 12.0]])]
    s, n = S.edge_prior(ids, edges, 3)
    assert s.tolist() == [1 + 3 + 6 + 8 + 10 + 12, 5 + 9 + 11 + 2, 0.0] and n.tolist() == [6, 4, 0]
    assert S.split_by_edges(s, n, tau_b=6.0) == [True, True, False]
