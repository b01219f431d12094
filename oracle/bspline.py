"""B-spline bases by the Cox–de Boor recursion (Definition 2.1, Sec. 2.1).

Test infrastructure (see ``oracle/__init__``).  Plain loops over the recursion,
float64.  The recursion's first quotient is read with denominator
xi_{l+p} - xi_l (the printed xi_{l+p} - xi_j is an index typo); 0/0 := 0.
"""
import numpy as np


def open_knot_vector(n_el, p):
    """p-open uniform knot vector Xi_{j,p} with n_el = 2^j elements (Sec. 2.3).

    p+1 zeros, the interior knots i/n_el, p+1 ones.  It carries n_el + p basis
    functions.
    """
    inner = [i / n_el for i in range(1, n_el)]
    return np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1))


def basis(knots, p, x):
    """All degree-p basis functions b_l^p of ``knots`` at the points ``x``.

    Returns an array [len(x), len(knots)-p-1].  Degree 0 uses half-open
    intervals [xi_l, xi_{l+1}); the right end point of the knot vector is
    assigned to the last non-empty interval so that the basis sums to one on
    the closed parameter interval.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    kn = np.asarray(knots, dtype=np.float64)
    nk = len(kn)
    B = np.zeros((len(x), nk - 1))
    last = max(l for l in range(nk - 1) if kn[l] < kn[l + 1])
    for l in range(nk - 1):
        if kn[l] < kn[l + 1]:
            inside = (x >= kn[l]) & (x < kn[l + 1])
            if l == last:
                inside |= x == kn[l + 1]
            B[:, l] = inside
    for d in range(1, p + 1):
        Bn = np.zeros((len(x), nk - 1 - d))
        for l in range(nk - 1 - d):
            den1 = kn[l + d] - kn[l]
            den2 = kn[l + d + 1] - kn[l + 1]
            t = np.zeros(len(x))
            if den1 > 0:
                t += (x - kn[l]) / den1 * B[:, l]
            if den2 > 0:
                t += (kn[l + d + 1] - x) / den2 * B[:, l + 1]
            Bn[:, l] = t
        B = Bn
    return B


def basis_deriv(knots, p, x):
    """First derivatives of the degree-p basis functions at ``x``.

    Uses the textbook identity
    d/dx b_l^p = p b_l^{p-1}/(xi_{l+p}-xi_l) - p b_{l+1}^{p-1}/(xi_{l+p+1}-xi_{l+1}).
    """
    kn = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    if p == 0:
        return np.zeros((len(x), len(kn) - 1))
    Bm = basis(kn, p - 1, x)  # [len(x), len(kn)-p]
    nb = len(kn) - p - 1
    D = np.zeros((len(x), nb))
    for l in range(nb):
        den1 = kn[l + p] - kn[l]
        den2 = kn[l + p + 1] - kn[l + 1]
        if den1 > 0:
            D[:, l] += p / den1 * Bm[:, l]
        if den2 > 0:
            D[:, l] -= p / den2 * Bm[:, l + 1]
    return D


def cardinal(p, t):
    """Cardinal B-spline N_p on the integer knots 0, 1, ..., p+1 (zero elsewhere)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    kn = np.arange(p + 2, dtype=np.float64)
    inside = (t >= 0) & (t < p + 1)
    out = np.zeros(len(t))
    if inside.any():
        out[inside] = basis(kn, p, t[inside])[:, 0]
    return out


def cardinal_deriv(p, t):
    """Derivative of the cardinal B-spline N_p."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    kn = np.arange(p + 2, dtype=np.float64)
    inside = (t >= 0) & (t < p + 1)
    out = np.zeros(len(t))
    if inside.any():
        out[inside] = basis_deriv(kn, p, t[inside])[:, 0]
    return out


def periodic_basis(n_el, p, x):
    """Periodic uniform degree-p splines on [0,1) with n_el elements.

    DOF i carries phi_i(x) = N_p((n_el x - i) mod n_el), so it is supported on
    elements i, ..., i+p (mod n_el).  Returns [len(x), n_el].
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.zeros((len(x), n_el))
    for i in range(n_el):
        out[:, i] = cardinal(p, np.mod(n_el * x - i, n_el))
    return out


def periodic_basis_deriv(n_el, p, x):
    """x-derivatives of ``periodic_basis``."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.zeros((len(x), n_el))
    for i in range(n_el):
        out[:, i] = n_el * cardinal_deriv(p, np.mod(n_el * x - i, n_el))
    return out


def gauss_legendre01(nq):
    """Gauss–Legendre nodes and weights on [0, 1]."""
    g, w = np.polynomial.legendre.leggauss(nq)
    return (g + 1.0) / 2.0, w / 2.0


def element_tables(n_el, p, nq, periodic):
    """1D basis values and derivatives at the Gauss points of every element.

    Returns (val, der, dofs): val/der are [n_el, p+1, nq]; dofs [n_el, p+1] are
    the 1D DOF indices of the p+1 functions alive on each element (open knots:
    e..e+p; periodic: e-p..e mod n_el).
    """
    g, _ = gauss_legendre01(nq)
    val = np.zeros((n_el, p + 1, nq))
    der = np.zeros((n_el, p + 1, nq))
    dofs = np.zeros((n_el, p + 1), dtype=np.int64)
    if periodic:
        for e in range(n_el):
            x = (e + g) / n_el
            B = periodic_basis(n_el, p, x)
            D = periodic_basis_deriv(n_el, p, x)
            for a in range(p + 1):
                i = (e - p + a) % n_el
                dofs[e, a] = i
                val[e, a] = B[:, i]
                der[e, a] = D[:, i]
    else:
        kn = open_knot_vector(n_el, p)
        for e in range(n_el):
            x = (e + g) / n_el
            B = basis(kn, p, x)
            D = basis_deriv(kn, p, x)
            for a in range(p + 1):
                dofs[e, a] = e + a
                val[e, a] = B[:, e + a]
                der[e, a] = D[:, e + a]
    return val, der, dofs
