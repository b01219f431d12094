"""Pins of the surface maps and metric terms (Sec. 3.2) against closed forms."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle.assembly import quadrature


def test_sphere_points_on_unit_sphere_and_gnomonic_area_element():
    rng = np.random.default_rng(0)
    u, v = rng.random(50), rng.random(50)
    for m in range(6):
        F, Fu, Fv = geo.sphere_map(m, u, v)
        np.testing.assert_allclose(np.linalg.norm(F, axis=-1), 1.0, atol=1e-15)
        # tangent vectors are orthogonal to the position on the unit sphere
        np.testing.assert_allclose(np.sum(F * Fu, -1), 0.0, atol=1e-14)
        a, G11, G12, G22 = geo.metric(Fu, Fv)
        # closed form of the gnomonic area element with the factor 4 of d(2u-1)/du d(2v-1)/dv
        x, y = 2 * u - 1, 2 * v - 1
        np.testing.assert_allclose(a, 4.0 / (1 + x * x + y * y) ** 1.5, rtol=1e-13)
        # a = |Fu x Fv|
        np.testing.assert_allclose(a, np.linalg.norm(np.cross(Fu, Fv), axis=-1), rtol=1e-13)
        # G = a K^{-1}: G K = a I
        K11 = np.sum(Fu * Fu, -1); K12 = np.sum(Fu * Fv, -1); K22 = np.sum(Fv * Fv, -1)
        np.testing.assert_allclose(G11 * K11 + G12 * K12, a, rtol=1e-12)
        np.testing.assert_allclose(G11 * K12 + G12 * K22, 0.0, atol=1e-12)


def test_sphere_patches_cover_sphere_once():
    # the six face normals are the +-axes; every direction falls in one face
    rng = np.random.default_rng(1)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    hits = np.zeros(len(d), int)
    for m, (ax, bx, nx, sg) in enumerate(geo.CUBE_FACES):
        c = d / (d[:, nx:nx + 1] * sg)
        inside = (d[:, nx] * sg > 0) & (np.abs(c[:, ax]) < 1) & (np.abs(c[:, bx]) < 1)
        hits += inside
    assert (hits == 1).all()


def test_torus_metric_closed_form():
    R, r = 1.0, 0.4
    rng = np.random.default_rng(2)
    u, v = rng.random(40), rng.random(40)
    _, Fu, Fv = geo.torus_map(u, v, R, r)
    a, G11, G12, G22 = geo.metric(Fu, Fv)
    np.testing.assert_allclose(a, 4 * np.pi ** 2 * r * (R + r * np.cos(2 * np.pi * v)), rtol=1e-13)
    np.testing.assert_allclose(G12, 0.0, atol=1e-12)
    np.testing.assert_allclose(G11, r / (R + r * np.cos(2 * np.pi * v)), rtol=1e-12)


@pytest.mark.parametrize("kind,n,tol", [("sphere", 4, 2e-4), ("sphere", 8, 4e-6), ("torus", 8, 1e-12)])
def test_quadrature_area(kind, n, tol):
    s = geo.Surface(kind, 2, n, n if kind == "sphere" else n // 2)
    q = quadrature(s)
    area = sum(float(np.sum(q["W"] * a)) for a in q["a"])
    assert area == pytest.approx(s.area_exact(), rel=tol)
