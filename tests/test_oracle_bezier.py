"""Pins of the oracle's Bezier-triangle evaluation (Sec. 3.1, Eq. 1-2).

Each check is fixed by mathematics, not by the oracle itself: partition of
unity and non-negativity of the Bernstein basis on the simplex, corner
interpolation, agreement with the de Casteljau recursion, linear precision
(a flat triangle lifted to degree n evaluates to the affine map) and the
degree-1 case being plain barycentric interpolation.
"""
import numpy as np
import pytest


def _simplex(rng, k):
    x = rng.dirichlet([1.0, 1.0, 1.0], size=k)
    return x[:, 0], x[:, 1], x[:, 2]


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_partition_of_unity_and_nonnegative(oracle, n):
    rng = np.random.default_rng(n)
    u, v, w = _simplex(rng, 200)
    for a, b, c in zip(u, v, w):
        B = oracle.bernstein(n, a, b, c)
        assert B.shape == ((n + 1) * (n + 2) // 2,)
        assert abs(B.sum() - 1.0) < 1e-14
        assert (B >= 0).all()


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_corners_interpolate(oracle, scenes, n):
    # S(1,0,0) = p_n00, S(0,1,0) = p_0n0, S(0,0,1) = p_00n (Eq. 1 at the corners)
    rng = np.random.default_rng(10 + n)
    ctrl = rng.normal(size=((n + 1) * (n + 2) // 2, 3))
    corners = {(1, 0, 0): scenes.cp_index(n, n, 0), (0, 1, 0): scenes.cp_index(n, 0, n),
               (0, 0, 1): scenes.cp_index(n, 0, 0)}
    for (u, v, w), idx in corners.items():
        B = oracle.bernstein(n, u, v, w)
        assert np.allclose(B @ ctrl, ctrl[idx], atol=1e-15)
        assert np.allclose(oracle.decasteljau(n, ctrl, u, v, w), ctrl[idx], atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_decasteljau_equals_bernstein(oracle, n):
    rng = np.random.default_rng(20 + n)
    ctrl = rng.normal(size=((n + 1) * (n + 2) // 2, 3))
    u, v, w = _simplex(rng, 100)
    for a, b, c in zip(u, v, w):
        s1 = oracle.bernstein(n, a, b, c) @ ctrl
        s2 = oracle.decasteljau(n, ctrl, a, b, c)
        assert np.max(np.abs(s1 - s2)) < 1e-14


def test_degree1_is_barycentric_interpolation(oracle):
    rng = np.random.default_rng(3)
    p = rng.normal(size=(3, 3))  # p_100, p_010, p_001 in index order
    u, v, w = _simplex(rng, 50)
    for a, b, c in zip(u, v, w):
        got = oracle.bernstein(1, a, b, c) @ p
        assert np.allclose(got, a * p[0] + b * p[1] + c * p[2], atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_linear_precision_of_lifted_flat_triangle(oracle, scenes, n):
    # Control points placed on the lattice (i P0 + j P1 + k P2)/n reproduce the
    # flat triangle exactly: sum_ijk B_ijk (i, j, k)/n = (u, v, w).
    rng = np.random.default_rng(30 + n)
    P0, P1, P2 = rng.normal(size=(3, 3))
    m = (n + 1) * (n + 2) // 2
    ctrl = np.zeros((m, 3))
    for i in range(n, -1, -1):
        for j in range(n - i, -1, -1):
            k = n - i - j
            ctrl[scenes.cp_index(n, i, j)] = (i * P0 + j * P1 + k * P2) / n
    u, v, w = _simplex(rng, 50)
    for a, b, c in zip(u, v, w):
        got = oracle.bernstein(n, a, b, c) @ ctrl
        assert np.allclose(got, a * P0 + b * P1 + c * P2, atol=1e-14)


def test_generator_lifting_keeps_flat_triangles_flat(oracle, scenes):
    # a flat scene lifted with zero noise stays on its plane x = 0
    sc, _ = scenes.tiny_scene("two", n=3, noise=0.0)
    assert np.allclose(sc["ctrl"][:2, :, 0], 0.0, atol=1e-7)
