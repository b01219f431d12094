"""Pins of the glued space and the assembled M, S (Secs. 2.3, 3.1, 3.2)."""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse.linalg as spla

from oracle import geometry as geo
from oracle.assembly import assemble, evaluate, load_vector, quadrature
from oracle.space import GluedSpace


@pytest.mark.parametrize("n,p", [(1, 2), (2, 2), (8, 2), (4, 3), (2, 1)])
def test_glued_dof_count(n, p):
    sp_ = GluedSpace(geo.Surface("sphere", p, n))
    m = n + p
    # a closed cube-like grid: 6 faces, 12 shared edges, 8 shared corners
    assert sp_.N == 6 * m * m - 12 * m + 8
    # every global DOF is used; interior DOFs are used once
    counts = np.bincount(sp_.l2g.ravel())
    assert counts.min() >= 1 and counts.max() == 3
    assert (counts == 3).sum() == 8


def test_numbering_rule_scan_order():
    sp_ = GluedSpace(geo.Surface("sphere", 2, 2))
    flat = sp_.l2g.ravel()
    # new indices appear in increasing order along the scan
    seen = -1
    for g in flat:
        if g > seen:
            assert g == seen + 1
            seen = g
    assert (sp_.l2g[0].ravel() == np.arange(16)).all()


@pytest.mark.parametrize("p", [2, 3])
def test_glued_functions_are_continuous(p):
    s = geo.Surface("sphere", p, 4)
    sp_ = GluedSpace(s)
    coef = np.random.default_rng(3).standard_normal(sp_.N)
    # sample points along every patch edge and compare with the patch on the other side
    t = np.linspace(0.05, 0.95, 7)
    edges = [(t, 0 * t), (t, 0 * t + 1), (0 * t, t), (0 * t + 1, t)]
    pts, vals = [], []
    for m in range(6):
        for (u, v) in edges:
            F, _, _ = s.map(m, u, v)
            pts.append(F)
            vals.append(evaluate(sp_, coef, m, u, v))
    pts = np.concatenate(pts)
    vals = np.concatenate(vals)
    from scipy.spatial import cKDTree
    pairs = cKDTree(pts).query_pairs(1e-10)
    assert len(pairs) >= 6 * 4 * 7 // 2
    for i, j in pairs:
        assert vals[i] == pytest.approx(vals[j], abs=1e-12)


@pytest.mark.parametrize("kind,p,n", [("sphere", 2, 4), ("sphere", 3, 2), ("torus", 3, 8)])
def test_matrix_invariants(kind, p, n):
    s = geo.Surface(kind, p, n, n if kind == "sphere" else n // 2 if n > 8 else 8)
    sp_ = GluedSpace(s)
    S, M = assemble(sp_)
    assert abs(S - S.T).max() < 1e-13 * abs(S).max()
    assert abs(M - M.T).max() < 1e-15 * abs(M).max() + 1e-18
    one = np.ones(sp_.N)
    # S 1 = 0 (the gradient of a constant vanishes for any quadrature)
    assert np.abs(S @ one).max() < 1e-12 * abs(S).max()
    # 1^T M 1 is the quadrature area; it tends to the exact area
    q = quadrature(s)
    area_q = sum(float(np.sum(q["W"] * a)) for a in q["a"])
    assert one @ (M @ one) == pytest.approx(area_q, rel=1e-13)
    assert one @ (M @ one) == pytest.approx(s.area_exact(), rel=5e-3)
    # M SPD, S SPSD with a one-dimensional kernel
    ev = np.linalg.eigvalsh(M.toarray())
    assert ev.min() > 0
    es = np.linalg.eigvalsh(S.toarray())
    assert es[0] > -1e-10 and es[1] > 1e-6


def test_sphere_first_harmonics_eigenvalue():
    # Y_{1,m} are the coordinate functions; their eigenvalue of -Delta is
    # l(l+1) = 2, and l = 2 gives 6; the discrete eigenvalues converge to them
    errs = []
    for n in (4, 8):
        s = geo.Surface("sphere", 3, n)
        sp_ = GluedSpace(s)
        S, M = assemble(sp_)
        vals = scipy.linalg.eigh(S.toarray(), M.toarray(), eigvals_only=True)[:10]
        assert vals[0] == pytest.approx(0.0, abs=1e-9)
        # a triple eigenvalue near 2 (the three l = 1 harmonics), then five near 6
        assert np.ptp(vals[1:4]) < 1e-9
        np.testing.assert_allclose(vals[1:4], 2.0, rtol=2e-4)
        np.testing.assert_allclose(vals[4:9], 6.0, rtol=2e-3)
        assert vals[9] > 11.0
        errs.append(abs(vals[1] - 2.0))
    assert errs[1] < errs[0] / 16


@pytest.mark.parametrize("p", [2])
def test_spherical_harmonic_convergence_rate(p):
    # (kappa^2 - Delta) u = Y on S^2 with Y = x (an l = 1 harmonic): u = Y / (kappa^2 + 2)
    # (Sec. 4.1.1); L2 errors fall at the rate 2^{-j(p+1)} (Eq. eq:approximation)
    kappa = 1.0
    errs = []
    for n in (2, 4, 8):
        s = geo.Surface("sphere", p, n)
        sp_ = GluedSpace(s)
        S, M = assemble(sp_)
        f = load_vector(sp_, lambda X: X[..., 0])
        uh = spla.spsolve((S + kappa ** 2 * M).tocsc(), f)
        # L2 error by a finer Gauss rule on every element
        q = quadrature(geo.Surface("sphere", p + 2, n))
        e2 = 0.0
        g = np.polynomial.legendre.leggauss(p + 3)
        for m in range(6):
            uu, vv = q["u"].ravel(), q["v"].ravel()
            X, _, _ = s.map(m, uu, vv)
            val = evaluate(sp_, uh, m, uu, vv)
            e2 += float(np.sum(q["W"].ravel() * q["a"][m].ravel() * (val - X[:, 0] / (kappa ** 2 + 2)) ** 2))
        errs.append(np.sqrt(e2))
    rates = [errs[i] / errs[i + 1] for i in range(2)]
    assert rates[-1] > 0.75 * 2 ** (p + 1), (errs, rates)


def _params_of(s, X):
    """Patch index and parameters (m, u, v) of points X [n, 3] on surface s: the
    inverse of the gnomonic cube-sphere patches and of the torus map (Sec. 2.2)."""
    if s.kind == "torus":
        u = np.mod(np.arctan2(X[:, 1], X[:, 0]) / (2 * np.pi), 1.0)
        rho = np.hypot(X[:, 0], X[:, 1])
        v = np.mod(np.arctan2(X[:, 2], rho - s.R) / (2 * np.pi), 1.0)
        return np.zeros(len(X), dtype=int), u, v
    ax = np.argmax(np.abs(X), axis=-1)
    sg = np.sign(X[np.arange(len(X)), ax])
    m = np.full(len(X), -1)
    u = np.zeros(len(X))
    v = np.zeros(len(X))
    for k, (a, b, n, sgn) in enumerate(geo.CUBE_FACES):
        sel = (ax == n) & (sg == sgn)
        m[sel] = k
        c = X[sel] / np.abs(X[sel][:, n])[:, None]
        u[sel] = (c[:, a] + 1) / 2
        v[sel] = (c[:, b] + 1) / 2
    assert (m >= 0).all()
    return m, u, v


@pytest.mark.parametrize("kind,p,nu,nv", [("torus", 3, 8, 6), ("torus", 2, 5, 7), ("sphere", 2, 3, None),
                                           ("sphere", 3, 2, None)])
def test_spline_reproduction(kind, p, nu, nv):
    # The Galerkin projection of a function of the space is that function: with
    # f = sum_j c_j phi_j evaluated pointwise, the load vector by the mass matrix's
    # own Gauss rule is exactly M c, so M^{-1} F = c up to rounding.  This ties the
    # element connectivity and the load assembly to the global basis evaluation.
    s = geo.Surface(kind, p, nu, nv)
    sp_ = GluedSpace(s)
    _, M = assemble(sp_)
    c0 = np.random.default_rng(5).standard_normal(sp_.N)

    def f(X):
        Xf = X.reshape(-1, 3)
        m, u, v = _params_of(s, Xf)
        out = np.zeros(len(Xf))
        for k in np.unique(m):
            sel = m == k
            out[sel] = evaluate(sp_, c0, k, u[sel], v[sel])
        return out.reshape(X.shape[:-1])

    c = spla.spsolve(M.tocsc(), load_vector(sp_, f))
    assert np.abs(c - c0).max() < 1e-11 * np.abs(c0).max()


@pytest.mark.parametrize("p", [2, 3])
def test_torus_energies_closed_form(p):
    # Torus metric (Sec. 2.2): K = diag((2 pi rho)^2, (2 pi r)^2), a = 4 pi^2 rho r,
    # rho = R + r cos 2 pi v, so the stiffness weight is G = diag(r / rho, rho / r).
    # For f = cos(2 pi k u): int f^2 = 2 pi^2 R r and int |grad f|^2 =
    # (2 pi k)^2 r / (2 sqrt(R^2 - r^2)); for g = cos(2 pi v): int g^2 = 2 pi^2 R r
    # and int |grad g|^2 = (2 pi)^2 R / (2 r).  The L2 projections' energies
    # converge to these at the rate h^{2p}.
    R, r = 1.0, 0.4

    def uv(X):
        u = np.arctan2(X[..., 1], X[..., 0]) / (2 * np.pi)
        v = np.arctan2(X[..., 2], np.hypot(X[..., 0], X[..., 1]) - R) / (2 * np.pi)
        return u, v

    cases = [(lambda X: np.cos(2 * np.pi * uv(X)[0]), (2 * np.pi) ** 2 * r / (2 * np.sqrt(R * R - r * r))),
             (lambda X: np.cos(4 * np.pi * uv(X)[0]), (4 * np.pi) ** 2 * r / (2 * np.sqrt(R * R - r * r))),
             (lambda X: np.cos(2 * np.pi * uv(X)[1]), (2 * np.pi) ** 2 * R / (2 * r))]
    mass = 2 * np.pi ** 2 * R * r
    errs = []
    for n in (16, 32):
        sp_ = GluedSpace(geo.Surface("torus", p, n, n // 2, R, r))
        S, M = assemble(sp_)
        lu = spla.splu(M.tocsc())
        row = []
        for fn, energy in cases:
            c = lu.solve(load_vector(sp_, fn))
            assert c @ (M @ c) == pytest.approx(mass, rel=1e-4)
            row.append(abs(c @ (S @ c) - energy) / energy)
        errs.append(row)
    assert max(errs[1]) < (5e-5 if p == 2 else 5e-7), errs
    for e0, e1 in zip(*errs):
        assert e0 / e1 > 0.75 * 2 ** (2 * p), errs
