"""Pins of the oracle's split and prune geometry (Sec. 3.3 "Splitting and
Pruning"): exact 1 -> 4 midpoint subdivision of degree-n BG-triangles, the
four-triangle area estimate and the bounding-rectangle aspect ratio.

The pieces come from the blossom (de Casteljau with a different parameter
per level); they are checked against the Bernstein form of Eq. 1 (the C
oracle's basis, a different algorithm): every piece must reproduce the
parent surface on its part of the domain. Area and aspect are checked on
shapes with closed forms.
"""
import math

import numpy as np
import pytest

from oracle import split as S


def _bez(oracle, ctrl, n, uvw):
    return oracle.bernstein(n, *uvw) @ np.asarray(ctrl, np.float64)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_pieces_reproduce_the_parent_surface(oracle, n):
    rng = np.random.default_rng(n)
    ctrl = rng.normal(size=(S.ncp(n), 3))
    pieces = S.subdivide(ctrl, n)
    for p in range(4):
        for _ in range(20):
            a, b = rng.uniform(size=2)
            if a + b > 1:
                a, b = 1 - a, 1 - b
            uvw = (a, b, 1 - a - b)
            want = _bez(oracle, ctrl, n, S.piece_point(p, uvw))
            got = _bez(oracle, pieces[p], n, uvw)
            assert np.abs(got - want).max() < 1e-13, (n, p)
        # corners of the piece sit on the parent's surface points
        for corner, uvw in zip((S.index(n, n, 0), S.index(n, 0, n), S.index(n, 0, 0)), S.PIECES[p]):
            assert np.abs(pieces[p, corner] - _bez(oracle, ctrl, n, uvw)).max() < 1e-13


def test_degree_one_pieces_are_the_midpoint_triangles():
    P = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 4.0, 1.0]])  # p100, p010, p001
    pieces = S.subdivide(P, 1)
    pu, pv, pw = P
    want = [[pu, (pu + pv) / 2, (pu + pw) / 2], [(pu + pv) / 2, pv, (pv + pw) / 2],
            [(pu + pw) / 2, (pv + pw) / 2, pw], [(pv + pw) / 2, (pu + pw) / 2, (pu + pv) / 2]]
    assert np.abs(pieces - np.array(want)).max() == 0.0


@pytest.mark.parametrize("n", [2, 3])
def test_linear_precision_and_orientation(n):
    rng = np.random.default_rng(10 + n)
    Amat, t = rng.normal(size=(3, 2)), rng.normal(size=3)
    ctrl = np.array([Amat @ (i / n, j / n) + t for (i, j, _) in S.triples(n)])
    pieces = S.subdivide(ctrl, n)
    for p in range(4):
        for (i, j, k) in S.triples(n):
            u, v, _ = S.piece_point(p, (i / n, j / n, k / n))
            assert np.abs(pieces[p, S.index(n, i, j)] - (Amat @ (u, v) + t)).max() < 1e-13
        # every piece keeps the parent's orientation: its corner normal points the same way
        q = pieces[p]
        c = [q[S.index(n, n, 0)], q[S.index(n, 0, n)], q[S.index(n, 0, 0)]]
        nrm = np.cross(c[1] - c[0], c[2] - c[0])
        par = np.cross(ctrl[S.index(n, 0, n)] - ctrl[0], ctrl[S.index(n, 0, 0)] - ctrl[0])
        assert nrm @ par > 0


def _heron(a, b, c):
    la, lb, lc = np.linalg.norm(b - c), np.linalg.norm(a - c), np.linalg.norm(a - b)
    s = (la + lb + lc) / 2
    return math.sqrt(max(s * (s - la) * (s - lb) * (s - lc), 0.0))


def test_area_of_flat_and_quadratic_patches():
    P = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    assert abs(S.area(P, 1) - 3.0) < 1e-14
    # a planar degree-3 patch (affine control net) has the corner triangle's area
    n = 3
    ctrl = np.array([P[0] * i / n + P[1] * j / n + P[2] * k / n for (i, j, k) in S.triples(n)])
    assert abs(S.area(ctrl, n) - 3.0) < 1e-13
    # quadratic patch: the edge-midpoint surface points are (p_a + 2 p_ab + p_b) / 4
    rng = np.random.default_rng(3)
    q = rng.normal(size=(6, 3))
    p200, p020, p002 = q[S.index(2, 2, 0)], q[S.index(2, 0, 2)], q[S.index(2, 0, 0)]
    p110, p101, p011 = q[S.index(2, 1, 1)], q[S.index(2, 1, 0)], q[S.index(2, 0, 1)]
    muv, muw, mvw = (p200 + 2 * p110 + p020) / 4, (p200 + 2 * p101 + p002) / 4, (p020 + 2 * p011 + p002) / 4
    want = (_heron(p200, muv, muw) + _heron(muv, p020, mvw) + _heron(muw, mvw, p002)
            + _heron(mvw, muw, muv))
    assert abs(S.area(q, 2) - want) < 1e-12


def test_aspect_ratio_closed_forms_and_invariance():
    eq = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, math.sqrt(3) / 2, 0.0]])
    assert abs(S.aspect(eq, 1) - 2 / math.sqrt(3)) < 1e-14
    ri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    assert abs(S.aspect(ri, 1) - 2.0) < 1e-14  # hypotenuse sqrt(2), height sqrt(2) / 2
    sliver = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, 0.01, 0.0]])
    assert abs(S.aspect(sliver, 1) - 100.0) < 1e-10
    assert S.aspect(np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]]), 1) == math.inf
    # rigid motions and uniform scaling leave it unchanged, off-plane bulges do not count
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    n = 2
    ctrl = np.array([eq[0] * i / n + eq[1] * j / n + eq[2] * k / n for (i, j, k) in S.triples(n)])
    ctrl[S.index(n, 1, 1)] += (0.0, 0.0, 0.7)
    moved = 2.5 * ctrl @ Q.T + rng.normal(size=3)
    assert abs(S.aspect(moved, n) - 2 / math.sqrt(3)) < 1e-12
    # control points bulging in-plane stretch the box: 1 x (sqrt(3) / 2 + 1/2)
    wide = ctrl.copy()
    wide[S.index(n, 1, 1)] = (0.5, -0.5, 0.0)
    assert abs(S.aspect(wide, n) - (math.sqrt(3) / 2 + 0.5)) < 1e-14


def test_area_is_additive_over_the_pieces_of_a_flat_patch():
    rng = np.random.default_rng(5)
    P = rng.normal(size=(3, 3))
    n = 3
    ctrl = np.array([P[0] * i / n + P[1] * j / n + P[2] * k / n for (i, j, k) in S.triples(n)])
    pieces = S.subdivide(ctrl, n)
    assert abs(sum(S.area(pieces[p], n) for p in range(4)) - S.area(ctrl, n)) < 1e-13
    # each piece of a flat patch is a quarter of it
    for p in range(4):
        assert abs(S.area(pieces[p], n) - S.area(ctrl, n) / 4) < 1e-13


@pytest.mark.parametrize("R", [1, 3])
def test_attribute_maps_of_the_pieces(oracle, R):
    rng = np.random.default_rng(6)
    a, b, c = rng.normal(size=(3, 4))
    nodes = S.texel_nodes(R)
    tex = np.array([a + b * u + c * v for (u, v) in nodes]) if R > 1 else rng.normal(size=(1, 4))
    out = S.subdivide_map(tex, R, oracle.attr_weights)
    for p in range(4):
        if R == 1:
            assert np.array_equal(out[p], tex)
            continue
        # an affine field is reproduced on every piece
        for t, (u, v) in enumerate(nodes):
            pu, pv, _ = S.piece_point(p, (u, v, 1 - u - v))
            assert np.abs(out[p, t] - (a + b * pu + c * pv)).max() < 1e-13


def test_split_and_prune_decisions():
    big = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    assert S.decisions(big, 1) == (False, False)
    tiny = big * 0.01  # area 5e-5 < 3e-4
    assert S.decisions(tiny, 1)[0]
    thin = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, 0.04, 0.0]])  # aspect 25, area 0.02
    assert S.decisions(thin, 1)[0]
    g = np.full((3, 3), 0.0011)  # |g| = 0.0019 per control point
    assert S.decisions(big, 1, g)[1] and not S.decisions(big, 1, g * 0.9)[1]
