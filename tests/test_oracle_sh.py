"""Pins of the oracle's view-dependent colour: real spherical harmonics of
bands 1..3 (their coefficients per primitive, Sec. 3.2 "SH coefficients",
one set per primitive), added to the diffuse colour of Eq. 4.

The basis comes from the associated Legendre definition; these tests tie it
to what mathematics fixes: orthonormality on the sphere, the addition theorem
(sum over m of Y_lm^2 = (2l + 1) / (4 pi) everywhere), the band-1 closed form,
and, for the colour term, the central differences of the whole forward pass.
"""
import math

import numpy as np
import pytest


def _sphere_quadrature(n_theta=48, n_phi=96):
    # Gauss-Legendre in cos(theta) x uniform phi: exact for polynomials of the
    # degrees involved (products of two band-3 harmonics)
    x, wx = np.polynomial.legendre.leggauss(n_theta)
    phi = np.arange(n_phi) * 2 * math.pi / n_phi
    dirs, w = [], []
    for xi, wi in zip(x, wx):
        s = math.sqrt(1 - xi * xi)
        for p in phi:
            dirs.append((s * math.cos(p), s * math.sin(p), xi))
            w.append(wi * 2 * math.pi / n_phi)
    return np.array(dirs), np.array(w)


def test_basis_is_orthonormal_on_the_sphere(oracle):
    dirs, w = _sphere_quadrature()
    Y = np.array([oracle.sh_basis(3, d) for d in dirs])  # [N, 15]
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(15)).max() < 1e-10


def test_addition_theorem_and_band1_closed_form(oracle):
    rng = np.random.default_rng(0)
    for _ in range(50):
        d = rng.normal(size=3)
        Y = oracle.sh_basis(3, d)
        for l in (1, 2, 3):
            band = Y[l * l - 1: (l + 1) ** 2 - 1]
            assert abs((band ** 2).sum() - (2 * l + 1) / (4 * math.pi)) < 1e-12
        x, y, z = d / np.linalg.norm(d)
        c1 = math.sqrt(3 / (4 * math.pi))
        assert np.allclose(Y[:3], c1 * np.array([-y, z, -x]), atol=1e-14)
        # m = 0 of band 2 is the zonal Legendre polynomial
        assert abs(Y[5] - math.sqrt(5 / (4 * math.pi)) * (3 * z * z - 1) / 2) < 1e-13


def test_zero_coefficients_leave_the_diffuse_colour(oracle, scenes):
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(48, 44), r_b=2e-2)
    ref = oracle.render(sc, cams[0])
    s3 = scenes.with_sh(sc, 3, scale=0.0)
    got = oracle.render(s3, cams[0])
    assert np.abs(got["image"] - ref["image"]).max() < 1e-14
    # not vacuous: non-zero coefficients change the image
    got = oracle.render(scenes.with_sh(sc, 3), cams[0])
    assert np.abs(got["image"] - ref["image"]).max() > 1e-2


@pytest.mark.parametrize("D", [1, 3])
def test_sh_gradients_match_central_differences(oracle, scenes, D):
    from tests.test_oracle_grad import fd_check
    sc, cams = scenes.tiny_scene("ico1", noise=0.04, size=(44, 44), r_b=2e-2)
    sc = scenes.with_sh(sc, D, seed=D)
    res, g = fd_check(oracle, sc, cams[0], {}, 40, seed=11 + D, kinds=("sh", "sh", "ctrl", "color"))
    assert len(res) >= 32
    gmax = max(abs(r[3]) for r in res)
    for kind_, idx, an, num in res:
        err = abs(an - num) / max(abs(num), 1e-3 * gmax)
        assert err < 1e-5, (kind_, idx, an, num)
    assert np.abs(g["sh"]).max() > 0
