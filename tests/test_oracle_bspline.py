"""Pins of the oracle's B-spline bases (Definition 2.1, Fig. 1)."""
import numpy as np
import pytest

from oracle import bspline as bs

# Fig. 1(b),(c): the plotted pieces of the p = 1 and p = 2 bases on the open
# knot vectors [0,0,1/3,2/3,1,1] and [0,0,0,1/3,2/3,1,1,1] (printed formulas).
T = 1.0 / 3.0
FIG1_P1 = [
    (0, 0, T, lambda x: 3 * -(x - T)),
    (1, 0, T, lambda x: 3 * x),
    (1, T, 2 * T, lambda x: (1 - 3 * x) + 1),
    (2, T, 2 * T, lambda x: 3 * (x - T)),
    (2, 2 * T, 1, lambda x: 3 * (1 - x - T) + 1),
    (3, 2 * T, 1, lambda x: 3 * (x - 2 * T)),
]
FIG1_P2 = [
    (0, 0, T, lambda x: (3 * x - 1) ** 2),
    (1, 0, T, lambda x: 2 * (3 * x) * (1 - 3 * x) + .5 * (3 * x) ** 2),
    (2, 0, T, lambda x: .5 * (x * 3) ** 2),
    (3, 2 * T, 1, lambda x: 2 * (3 * (x - 2 * T)) * (1 - 3 * (x - 2 * T)) + .5 * (1 - 3 * (x - 2 * T)) ** 2),
    (4, 2 * T, 1, lambda x: (3 * (x - 2 * T)) ** 2),
    (1, T, 2 * T, lambda x: .5 * (1 - 3 * (x - T)) ** 2),
    (2, T, 2 * T, lambda x: -(((x * 3) - 1) - 1) * ((x * 3) - 1) + .5),
    (2, 2 * T, 1, lambda x: .5 * (3 - (x * 3)) ** 2),
    (3, T, 2 * T, lambda x: .5 * (3 * (x - T)) ** 2),
]


@pytest.mark.parametrize("p,pieces", [(1, FIG1_P1), (2, FIG1_P2)])
def test_fig1_pieces(p, pieces):
    kn = bs.open_knot_vector(3, p)
    for idx, a, b, f in pieces:
        x = np.linspace(a, b, 17)[1:-1]
        np.testing.assert_allclose(bs.basis(kn, p, x)[:, idx], f(x), atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 4, 8])
def test_partition_of_unity_and_derivative(p, n):
    kn = bs.open_knot_vector(n, p)
    x = np.linspace(0, 1, 101)
    B = bs.basis(kn, p, x)
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-14)
    assert (B >= -1e-15).all()
    D = bs.basis_deriv(kn, p, x)
    np.testing.assert_allclose(D.sum(1), 0.0, atol=1e-11)
    # derivative against a central difference away from knots
    h = 1e-6
    xm = (np.arange(n) + 0.37) / n
    Dfd = (bs.basis(kn, p, xm + h) - bs.basis(kn, p, xm - h)) / (2 * h)
    np.testing.assert_allclose(bs.basis_deriv(kn, p, xm), Dfd, atol=1e-6 * n)


@pytest.mark.parametrize("p", [2, 3])
def test_periodic_basis(p):
    n = 8
    x = np.linspace(0, 1, 97)[:-1]
    B = bs.periodic_basis(n, p, x)
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-14)
    # DOF i is the cardinal spline shifted by i/n: phi_i(x) = phi_0(x - i/n)
    np.testing.assert_allclose(B[:, 3], bs.periodic_basis(n, p, (x - 3 / n) % 1.0)[:, 0], atol=1e-14)
    # cardinal B-spline closed form for p = 2 on [0, 1): t^2 / 2
    t = np.linspace(0, 0.99, 7)
    np.testing.assert_allclose(bs.cardinal(2, t), t ** 2 / 2, atol=1e-15)
    np.testing.assert_allclose(bs.cardinal(3, t + 1), (-3 * (t + 1) ** 3 + 12 * (t + 1) ** 2 - 12 * (t + 1) + 4) / 6, atol=1e-14)


def test_element_tables_match_global_basis():
    n, p, nq = 4, 2, 3
    val, der, dofs = bs.element_tables(n, p, nq, periodic=False)
    g, _ = bs.gauss_legendre01(nq)
    kn = bs.open_knot_vector(n, p)
    for e in range(n):
        B = bs.basis(kn, p, (e + g) / n)
        np.testing.assert_allclose(B[:, dofs[e]].T, val[e], atol=1e-15)
        # nothing else is alive on the element
        mask = np.ones(n + p, bool)
        mask[dofs[e]] = False
        assert np.abs(B[:, mask]).max() == 0
