"""Pins of the oracle's real spherical-harmonic basis (the colour model of the
Gaussian primitive, Sec. 7: SH coefficients per primitive, degree 3).

Pins, none of which reuses the oracle's own construction:
  * orthonormality on the sphere by an exact product quadrature;
  * the special case reducing to a library routine: scipy's complex SH
    (Condon-Shortley phase included) converted to the real, phase-free basis;
  * textbook closed forms at the axes.
"""
import numpy as np
import pytest
from scipy import special

import oracle


def _quadrature(nz=8, nphi=16):
    z, wz = np.polynomial.legendre.leggauss(nz)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    Z, P = np.meshgrid(z, phi, indexing="ij")
    s = np.sqrt(1 - Z ** 2)
    dirs = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    return dirs, w


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_orthonormal_by_quadrature(deg):
    # Gauss-Legendre in z (exact to degree 15) x uniform azimuth (exact for
    # trigonometric degree < 16): exact for products of two l <= 3 harmonics.
    dirs, w = _quadrature()
    Y = oracle.sh_basis(deg, dirs)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye((deg + 1) ** 2)).max() < 1e-12


def _real_from_scipy(l, m, theta, phi):
    # scipy: Y_l^m = K P_l^m(cos theta) e^{i m phi}, P_l^m with the
    # Condon-Shortley factor (-1)^m.  Real phase-free basis:
    #   m > 0: sqrt2 (-1)^m Re Y_l^m ; m < 0: sqrt2 (-1)^|m| Im Y_l^|m| ; m = 0: Y_l^0
    am = abs(m)
    Yc = special.sph_harm_y(l, am, theta, phi)
    if m == 0:
        return Yc.real
    sgn = (-1.0) ** am
    return np.sqrt(2.0) * sgn * (Yc.real if m > 0 else Yc.imag)


def test_matches_scipy_complex_harmonics():
    g = np.random.default_rng(3)
    d = g.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = oracle.sh_basis(3, d)
    for l in range(4):
        for m in range(-l, l + 1):
            ref = _real_from_scipy(l, m, theta, phi)
            assert np.abs(Y[:, l * l + l + m] - ref).max() < 1e-12, (l, m)


def test_axis_values_closed_form():
    # Y_00 = 1/(2 sqrt(pi)); Y_1,{-1,0,1} = sqrt(3/(4 pi)) (y, z, x) with no phase sign
    c1 = np.sqrt(3 / (4 * np.pi))
    Y = oracle.sh_basis(1, np.eye(3))
    assert abs(Y[0, 0] - 0.5 / np.sqrt(np.pi)) < 1e-15
    assert np.allclose(Y[0, 1:], [0, 0, c1], atol=1e-15)   # +x
    assert np.allclose(Y[1, 1:], [c1, 0, 0], atol=1e-15)   # +y
    assert np.allclose(Y[2, 1:], [0, c1, 0], atol=1e-15)   # +z
    # l = 2, m = 0 at +z: (1/4) sqrt(5/pi) (3 z^2 - 1) = (1/2) sqrt(5/pi)
    Y2 = oracle.sh_basis(2, [[0, 0, 1]])
    assert abs(Y2[0, 6] - 0.5 * np.sqrt(5 / np.pi)) < 1e-14
    # l = 3, m = 3 at +x: (1/4) sqrt(35/(2 pi)) x (x^2 - 3 y^2)
    Y3 = oracle.sh_basis(3, [[1, 0, 0]])
    assert abs(Y3[0, 15] - 0.25 * np.sqrt(35 / (2 * np.pi))) < 1e-14


def test_degree0_is_constant():
    g = np.random.default_rng(5)
    d = g.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(0, d)
    assert np.all(np.abs(Y[:, 0] - 0.5 / np.sqrt(np.pi)) < 1e-15)
