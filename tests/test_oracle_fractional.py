"""Pins of the fractional solve (Sec. 3.4) against brute force.

A dense generalised eigen-decomposition S V = M V diag(mu), V^T M V = I gives
every operator of the method in closed form on a tiny mesh:
  A_sigma^{-1} = V diag(1/(mu + sigma)) V^T,  L^{-beta} M^{-1} = V diag((kappa^2+mu)^{-beta}) V^T.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import fractional as fr
from oracle import geometry as geo
from oracle.assembly import assemble, load_vector
from oracle.space import GluedSpace


@pytest.fixture(scope="module")
def tiny():
    s = geo.Surface("sphere", 2, 2)
    sp_ = GluedSpace(s)
    S, M = assemble(sp_)
    mu, V = scipy.linalg.eigh(S.toarray(), M.toarray())
    b = np.random.default_rng(0).standard_normal((3, sp_.N))
    return sp_, S, M, mu, V, b


def _sinc_symbol(bp, kappa, k, lo, hi, mu):
    y, c = fr.sinc_rule(bp, k, lo, hi)
    return np.array([np.sum(c / (m + np.exp(y) + kappa ** 2)) for m in mu])


@pytest.mark.parametrize("beta,mode", [(0.75, "standard"), (1.3, "standard"), (2.6, "standard"),
                                       (1.2, "improved"), (1.8, "improved"), (0.9, "improved"),
                                       (2.0, "standard")])
def test_fields_match_eigen_brute_force(tiny, beta, mode):
    sp_, S, M, mu, V, b = tiny
    kappa, k, lo, hi = 2.0, 0.4, -25, 25
    u = fr.sample_fields(S, M, b, kappa, beta, k, lo, hi, mode)
    n, bp, passes = fr.split_beta(beta, mode)
    sym = (kappa ** 2 + mu) ** -float(n)
    if passes:
        sym = sym * _sinc_symbol(bp, kappa, k, lo, hi, mu) ** passes
    ref = (V @ (sym[:, None] * (V.T @ b.T))).T
    np.testing.assert_allclose(u, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_fine_sinc_tends_to_fractional_power(tiny):
    # with many nodes the sinc map tends to L^{-beta'} itself
    sp_, S, M, mu, V, b = tiny
    kappa, beta = 1.5, 0.6
    u = fr.sample_fields(S, M, b[:1], kappa, beta, 2 / math.sqrt(400), -400, 400)
    ref = (V @ (((kappa ** 2 + mu) ** -beta)[:, None] * (V.T @ b[:1].T))).T
    np.testing.assert_allclose(u, ref, rtol=1e-6, atol=1e-8 * np.abs(ref).max())


def test_harmonic_rhs_scalar_sinc():
    # rhs = <Y, phi_i> with Y = z an l = 1 harmonic: the field is close to
    # (scalar sinc value at lambda = kappa^2 + 2) * Y
    s = geo.Surface("sphere", 3, 4)
    sp_ = GluedSpace(s)
    S, M = assemble(sp_)
    f = load_vector(sp_, lambda X: X[..., 2])
    kappa, beta, K = 1.0, 0.5, 50
    u = fr.sample_fields(S, M, f[None], kappa, beta, 2 / math.sqrt(K), -K, K)[0]
    y_coef = np.linalg.solve(M.toarray(), f)  # L2 projection of Y
    lam = kappa ** 2 + 2.0
    np.testing.assert_allclose(u, fr.scalar_sinc(beta, K, lam) * y_coef, rtol=0, atol=3e-3 * np.abs(y_coef).max())


@pytest.mark.parametrize("beta,mode", [(0.8, fr.STANDARD), (1.3, fr.STANDARD), (2.0, fr.STANDARD),
                                       (0.9, fr.IMPROVED), (1.5, fr.IMPROVED), (1.9, fr.IMPROVED)])
def test_gradient_matches_finite_differences(tiny, beta, mode):
    # every split: one pass (0.8, 1.3), integer beta (2.0: no pass), two passes
    # with n = 0, 0 and 1 integer solves (improved split: 0.9, 1.5, 1.9)
    sp_, S, M, mu, V, b = tiny
    kappa, k, lo, hi = 1.7, 0.5, -12, 12
    g = np.random.default_rng(1).standard_normal(b.shape)
    L, dLdb, dLdk = fr.field_loss_grad(S, M, b, g, kappa, beta, k, lo, hi, mode)
    h = 1e-6
    Lp = fr.field_loss_grad(S, M, b, g, kappa + h, beta, k, lo, hi, mode)[0]
    Lm = fr.field_loss_grad(S, M, b, g, kappa - h, beta, k, lo, hi, mode)[0]
    assert dLdk == pytest.approx((Lp - Lm) / (2 * h), rel=1e-6)
    d = np.random.default_rng(2).standard_normal(b.shape)
    Lp = fr.field_loss_grad(S, M, b + h * d, g, kappa, beta, k, lo, hi, mode)[0]
    Lm = fr.field_loss_grad(S, M, b - h * d, g, kappa, beta, k, lo, hi, mode)[0]
    assert float(np.sum(dLdb * d)) == pytest.approx((Lp - Lm) / (2 * h), rel=1e-6)
    # closed form of the loss through the eigen-decomposition: each pass
    # multiplies mode mu by the sinc symbol, each integer solve by 1/(kappa^2 + mu)
    n, bp, passes = fr.split_beta(beta, mode)
    sym = (kappa ** 2 + mu) ** -float(n) * _sinc_symbol(bp, kappa, k, lo, hi, mu) ** passes
    u = (V @ (sym[:, None] * (V.T @ b.T))).T
    dd = u - g
    assert L == pytest.approx(float(np.sum(dd * (M @ dd.T).T)), rel=1e-10)
