"""Pins of the sqrt(M) noise by the Hale–Higham–Trefethen sum (Sec. 3.3, Eq. eq:sqrt).

The exact square root of a small symmetric positive definite matrix comes from
its eigendecomposition, V diag(sqrt(mu)) V^T; a diagonal matrix reduces the
rule to the scalar sum, whose limit is sqrt(lambda).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import geometry as geo
from oracle import sqrt_mass as sq
from oracle.assembly import assemble
from oracle.space import GluedSpace


def _scalar(lo, hi, n, lam):
    w2, c = sq.hht_rule(lo, hi, n)
    return lam * (c[None, :] / (lam[:, None] + w2[None, :])).sum(axis=1)


@pytest.mark.parametrize("kappa", [10.0, 1e2, 1e4, 1e7])
def test_scalar_rule_converges_exponentially(kappa):
    # lambda A sum_k c_k / (lambda + w_k^2) -> sqrt(lambda) for every lambda in
    # [lo, hi]; the error falls geometrically in the number of nodes and stays
    # inside exp(-pi^2 K / (ln kappa + 3))
    lo, hi = 0.37, 0.37 * kappa
    lam = np.geomspace(lo, hi, 301)
    errs = []
    for n in (4, 8, 16, 32):
        err = float(np.abs(_scalar(lo, hi, n, lam) / np.sqrt(lam) - 1.0).max())
        assert err <= max(math.exp(-math.pi ** 2 * n / (math.log(kappa) + 3.0)), 4e-15), (n, err)
        errs.append(err)
    assert errs[1] < errs[0] / 50 and errs[2] < max(errs[1] / 50, 4e-15)


def test_rule_is_exact_in_the_limit_for_diagonal_matrices():
    # a diagonal A: every entry follows the scalar rule, including the interval ends
    lam = np.array([1.0, 1.5, 7.0, 60.0, 99.9])
    y = np.arange(1.0, 6.0)
    out = sq.sqrt_apply(sp.diags(lam), y, 1.0, 100.0, 24)
    np.testing.assert_allclose(out, np.sqrt(lam) * y, rtol=1e-13)


def test_rule_needs_valid_bounds():
    for args in [(0.0, 1.0, 8), (2.0, 1.0, 8), (1.0, 2.0, 0)]:
        with pytest.raises(ValueError):
            sq.hht_rule(*args)


@pytest.mark.parametrize("kind,p,n", [("sphere", 1, 4), ("sphere", 2, 2), ("sphere", 3, 2), ("torus", 3, 8),
                                      ("sphere", 2, 8)])
def test_mass_bounds_bracket_the_spectrum(kind, p, n):
    space = GluedSpace(geo.Surface(kind, p, n, n if kind == "sphere" else 8))
    _, M = assemble(space)
    ev = np.linalg.eigvalsh(M.toarray())
    lo, hi = sq.mass_spectrum_bounds(space)
    assert 0.0 < lo <= ev[0] and ev[-1] <= hi
    assert hi <= 1.5 * ev[-1]


@pytest.mark.parametrize("kind,p,n", [("sphere", 2, 2), ("torus", 3, 8)])
def test_sqrt_of_mass_matches_eigendecomposition(kind, p, n):
    space = GluedSpace(geo.Surface(kind, p, n, n if kind == "sphere" else 8))
    _, M = assemble(space)
    mu, V = np.linalg.eigh(M.toarray())
    root = (V * np.sqrt(mu)) @ V.T
    lo, hi = sq.mass_spectrum_bounds(space)
    y = np.random.default_rng(4).standard_normal((space.N, 3))
    # exponential convergence, and no loss of accuracy from the nodes near the
    # quarter period where cn is small
    for n_nodes, tol in ((8, 1e-2), (24, 1e-8), (48, 1e-13), (96, 1e-13)):
        f = sq.sqrt_apply(M, y, lo, hi, n_nodes)
        err = np.linalg.norm(f - root @ y) / np.linalg.norm(root @ y)
        assert err < tol, (n_nodes, err)


def test_noise_covariance_is_mass():
    # f = R y with R the rule's matrix: Cov(f) = R R^T must reproduce M
    space = GluedSpace(geo.Surface("sphere", 2, 2))
    _, M = assemble(space)
    lo, hi = sq.mass_spectrum_bounds(space)
    R = sq.sqrt_apply(M, np.eye(space.N), lo, hi, 48)
    np.testing.assert_allclose(R, R.T, atol=1e-14 * np.abs(R).max())
    np.testing.assert_allclose(R @ R.T, M.toarray(), atol=1e-12 * abs(M).max())
    f = sq.noise_loads_sqrt(M, lo, hi, 48, np.eye(space.N)[:2])
    np.testing.assert_allclose(f, R[:, :2].T, atol=1e-15)
