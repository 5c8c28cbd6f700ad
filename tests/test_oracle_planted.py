"""The pins of the newer oracle parts catch plausible mistakes: each test
plants one in a copy of the oracle's arithmetic (on the CPU, in the test
only) and checks that the pin that guards it fails, while the oracle as
committed passes it.
"""
import numpy as np

from oracle import loss as L
from oracle import split as S


def _fd_error(grad_fn, loss_fn, seed=5, H=13, W=11, lam=0.2):
    rng = np.random.default_rng(seed)
    x, y = rng.uniform(size=(H, W, 3)), rng.uniform(size=(H, W, 3))
    y = 0.5 * y + 0.5 * x
    g = grad_fn(x, y, lam)
    h = 1e-6
    worst = 0.0
    for i, j, c in [(0, 0, 0), (H - 1, W - 1, 2), (6, 5, 1), (3, 8, 0), (9, 2, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[i, j, c] += h
        xm[i, j, c] -= h
        num = (loss_fn(xp, y, lam) - loss_fn(xm, y, lam)) / (2 * h)
        worst = max(worst, abs(g[i, j, c] - num) / max(abs(num), 1e-3 * np.abs(g).max()))
    return worst


def test_loss_gradient_pin_catches_a_wrong_adjoint(monkeypatch):
    assert _fd_error(L.loss_grad, L.loss) < 1e-6
    # plant: the adjoint taken as the window shifted by one pixel (a transposed
    # operand that is not the transpose)
    shifted = lambda m: np.roll(L.window_filter(m), 1, axis=1)  # noqa: E731
    monkeypatch.setattr(L, "window_filter_adjoint", shifted)
    assert _fd_error(L.loss_grad, L.loss) > 1e-3


def test_loss_gradient_pin_catches_a_dropped_term(monkeypatch):
    # plant: the covariance partial c dropped (y F^T c missing)
    real_adj = L.window_filter_adjoint
    calls = {"n": 0}

    def adj(m):
        calls["n"] += 1
        return real_adj(m) if calls["n"] % 3 else np.zeros_like(m)  # every third call is F^T c
    monkeypatch.setattr(L, "window_filter_adjoint", adj)
    assert _fd_error(L.loss_grad, L.loss) > 1e-3


def test_subdivision_pin_catches_a_wrong_de_casteljau_step(oracle, monkeypatch):
    n = 3
    rng = np.random.default_rng(1)
    ctrl = rng.normal(size=(S.ncp(n), 3))

    def worst_error():
        pieces = S.subdivide(ctrl, n)
        err = 0.0
        for p in range(4):
            for _ in range(10):
                a, b = rng.uniform(size=2)
                if a + b > 1:
                    a, b = 1 - a, 1 - b
                uvw = (a, b, 1 - a - b)
                want = oracle.bernstein(n, *S.piece_point(p, uvw)) @ ctrl
                got = oracle.bernstein(n, *uvw) @ pieces[p]
                err = max(err, float(np.abs(got - want).max()))
        return err

    assert worst_error() < 1e-13

    # plant: the v-term of a de Casteljau level reads the u-neighbour
    def bad_blossom(c, n_, params):
        c = np.asarray(c, np.float64)
        net = {(i, j, k): c[S.index(n_, i, j)] for (i, j, k) in S.triples(n_)}
        for r in range(n_):
            u, v, w = params[r]
            m = n_ - r - 1
            net = {(i, j, k): u * net[(i + 1, j, k)] + v * net[(i + 1, j, k)] + w * net[(i, j, k + 1)]
                   for (i, j, k) in S.triples(m)}
        return net[(0, 0, 0)]
    monkeypatch.setattr(S, "blossom", bad_blossom)
    assert worst_error() > 1e-3


def test_visibility_pin_catches_an_off_by_one_cell(oracle, scenes, monkeypatch):
    # the facing-triangle pin (every one of the L^2 lattice triangles seen,
    # by id) guards the decoding of the depth key
    sc = scenes.triangles_scene([((0.0, -1.0, -1.0), (0.0, 1.0, -1.0), (0.0, 0.0, 1.0))], n=2)
    cam = scenes.look_at_camera((4.0, 0.0, 0.0), (0, 0, 0), 256, 256)
    idm, _, key = oracle.raster(sc, cam)
    up = {2 * (a * 8 + b) for a in range(8) for b in range(8) if a + b <= 7}
    down = {2 * (a * 8 + b) + 1 for a in range(8) for b in range(8) if a + b <= 6}
    assert S.visibility([(idm, key)], 1)[1][0] == up | down
    # plant: the sub-triangle decoded one off (as if the key's low bits were misread)
    plain = S.visibility

    def bad_visibility(rasters, M, tess_level=8):
        return plain([(i, k + (i >= 0).astype(np.uint64)) for i, k in rasters], M, tess_level)
    monkeypatch.setattr(S, "visibility", bad_visibility)
    assert S.visibility([(idm, key)], 1)[1][0] != up | down
