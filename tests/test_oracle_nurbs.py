"""Pins of the NURBS geometry maps (Sec. 2.2) and of the oracle on NURBS surfaces."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import wm_workloads as wl
from oracle.assembly import assemble, evaluate, load_vector, quadrature
from oracle.geometry import metric
from oracle.nurbs import NurbsSurface, patch_map
from oracle.space import GluedSpace

R, r = 1.0, 0.4


def test_nurbs_torus_lies_on_the_torus():
    # (sqrt(x^2 + y^2) - R)^2 + z^2 = r^2 at every parameter, including knots and ends
    (patch,) = wl.nurbs_torus(R, r)
    rng = np.random.default_rng(0)
    u = np.concatenate([rng.random(200), [0.0, 0.25, 0.5, 0.75, 1.0]])
    v = np.concatenate([rng.random(200), [0.0, 0.25, 0.5, 1.0, 0.75]])
    F, _, _ = patch_map(patch, u, v)
    rho = np.hypot(F[:, 0], F[:, 1])
    np.testing.assert_allclose((rho - R) ** 2 + F[:, 2] ** 2, r * r, rtol=0, atol=1e-15)
    # closed in both directions
    t = rng.random(20)
    np.testing.assert_allclose(patch_map(patch, 0 * t, t)[0], patch_map(patch, 0 * t + 1, t)[0], atol=1e-15)
    np.testing.assert_allclose(patch_map(patch, t, 0 * t)[0], patch_map(patch, t, 0 * t + 1)[0], atol=1e-15)


@pytest.mark.parametrize("which", ["torus", "bulged", "weighted"])
def test_nurbs_derivatives_match_central_differences(which):
    patch = {"torus": wl.nurbs_torus(R, r)[0], "bulged": wl.nurbs_bulged_cube(0.3)[2],
             "weighted": wl.nurbs_bulged_cube(0.4, weight=2.5)[5]}[which]
    rng = np.random.default_rng(1)
    u, v = 0.05 + 0.9 * rng.random(50), 0.05 + 0.9 * rng.random(50)
    _, Fu, Fv = patch_map(patch, u, v)
    h = 1e-6
    du = (patch_map(patch, u + h, v)[0] - patch_map(patch, u - h, v)[0]) / (2 * h)
    dv = (patch_map(patch, u, v + h)[0] - patch_map(patch, u, v - h)[0]) / (2 * h)
    # avoid the knots of the circle, where the map is only C1
    np.testing.assert_allclose(Fu, du, rtol=0, atol=2e-8 * np.abs(Fu).max())
    np.testing.assert_allclose(Fv, dv, rtol=0, atol=2e-8 * np.abs(Fv).max())


def test_flat_cube_is_the_cube_map():
    # bulge 0, unit weights: F_m(u, v) is the cube point itself, K = 4 I, a = 4, G = I
    patches = wl.nurbs_bulged_cube(0.0)
    rng = np.random.default_rng(2)
    u, v = rng.random(30), rng.random(30)
    for m, (ax, bx, nx, sg) in enumerate(wl.CUBE_FACES):
        F, Fu, Fv = patch_map(patches[m], u, v)
        c = np.zeros((30, 3))
        c[:, ax], c[:, bx], c[:, nx] = 2 * u - 1, 2 * v - 1, sg
        np.testing.assert_allclose(F, c, atol=1e-15)
        a, G11, G12, G22 = metric(Fu, Fv)
        np.testing.assert_allclose(a, 4.0, rtol=1e-15)
        np.testing.assert_allclose(G11, 1.0, rtol=1e-15)
        np.testing.assert_allclose(G12, 0.0, atol=1e-15)
        np.testing.assert_allclose(G22, 1.0, rtol=1e-15)


@pytest.mark.parametrize("p,n", [(2, 4), (3, 2), (1, 4)])
def test_cube_surfaces_glue_and_assemble(p, n):
    # the anchor matching finds the cube topology on any conforming six-patch
    # surface; the flat cube has area 24 exactly, the bulged one is closed (S 1 = 0)
    for bulge, weight in ((0.0, 1.0), (0.3, 1.0), (0.4, 2.5)):
        s = NurbsSurface("cube", wl.nurbs_bulged_cube(bulge, weight), p, n)
        sp_ = GluedSpace(s)
        m = n + p
        assert sp_.N == 6 * m * m - 12 * m + 8
        S, M = assemble(sp_)
        one = np.ones(sp_.N)
        assert abs(S - S.T).max() < 1e-13 * abs(S).max()
        assert np.abs(S @ one).max() < 1e-12 * abs(S).max()
        area = one @ (M @ one)
        if bulge == 0.0:
            assert area == pytest.approx(24.0, rel=1e-14)
        else:
            assert area > 24.0
        # glued functions are continuous across every patch edge
        coef = np.random.default_rng(3).standard_normal(sp_.N)
        t = np.linspace(0.05, 0.95, 5)
        pts, vals = [], []
        for mm in range(6):
            for (uu, vv) in [(t, 0 * t), (t, 0 * t + 1), (0 * t, t), (0 * t + 1, t)]:
                pts.append(s.map(mm, uu, vv)[0])
                vals.append(evaluate(sp_, coef, mm, uu, vv))
        pts, vals = np.concatenate(pts), np.concatenate(vals)
        from scipy.spatial import cKDTree
        pairs = cKDTree(pts).query_pairs(1e-10)
        assert len(pairs) >= 6 * 4 * 5 // 2
        for i, j in pairs:
            assert vals[i] == pytest.approx(vals[j], abs=1e-12)


def test_nurbs_torus_area_and_energies_of_physical_functions():
    # The same surface as the analytic torus with another parametrisation: the
    # area 4 pi^2 R r and the energies of f = cos(theta) = x / sqrt(x^2 + y^2)
    # ((2 pi)^2 r / (2 sqrt(R^2 - r^2))) and g = cos(t) = (sqrt(x^2 + y^2) - R) / r
    # ((2 pi)^2 R / (2 r)) depend on the surface only.
    f = lambda X: X[..., 0] / np.hypot(X[..., 0], X[..., 1])  # noqa: E731
    g = lambda X: (np.hypot(X[..., 0], X[..., 1]) - R) / r    # noqa: E731
    exact = {"f": (2 * np.pi) ** 2 * r / (2 * np.sqrt(R * R - r * r)), "g": (2 * np.pi) ** 2 * R / (2 * r)}
    errs = []
    for n in (16, 32):
        s = NurbsSurface("periodic", wl.nurbs_torus(R, r), 2, n, n // 2)
        sp_ = GluedSpace(s)
        S, M = assemble(sp_)
        q = quadrature(s)
        area = float(np.sum(q["W"] * q["a"][0]))
        assert area == pytest.approx(4 * np.pi ** 2 * R * r, rel=1e-6)
        lu = spla.splu(M.tocsc())
        row = []
        for name, fn in (("f", f), ("g", g)):
            c = lu.solve(load_vector(sp_, fn))
            row.append(abs(c @ (S @ c) - exact[name]) / exact[name])
        errs.append(row)
    assert max(errs[1]) < 2e-4, errs
    assert all(e0 / e1 > 8 for e0, e1 in zip(*errs)), errs


def test_cube_face_arrangement_is_one_table():
    # the NURBS cube inputs, the oracle's gnomonic sphere and the library's six-patch
    # gluing use one face arrangement (the library checks shared edges at set-up)
    from oracle.geometry import CUBE_FACES
    assert tuple(tuple(f) for f in wl.CUBE_FACES) == tuple(tuple(f) for f in CUBE_FACES)
