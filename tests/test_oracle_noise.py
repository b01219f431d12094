"""Pins of Philox4x32-10 and the white-noise loads (Sec. 3.3)."""
import os

import numpy as np
import pytest

from oracle import geometry as geo
from oracle.assembly import assemble, quadrature
from oracle.noise import n_quad, noise_adjoint, noise_from_xi, noise_loads
from oracle.philox import normals, philox4x32_10, uniform53
from oracle.space import GluedSpace

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        out = philox4x32_10(np.array(v[:4], dtype=np.uint64).reshape(4, 1),
                            np.array(v[4:6], dtype=np.uint64))
        assert [int(o[0]) for o in out] == v[6:]
        n += 1
    assert n == 3


def test_uniform53_range_and_normals_moments():
    assert uniform53(0, 0) == 2.0 ** -53
    assert uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0
    z = normals(123, 0, np.arange(200000))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    # the two halves of one Philox pair are independent draws
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 0.01
    # different samples and seeds give different streams
    assert not np.allclose(normals(123, 1, np.arange(10)), z[:10])
    assert not np.allclose(normals(124, 0, np.arange(10)), z[:10])


@pytest.mark.parametrize("kind,p,nu,nv", [("sphere", 2, 2, 2), ("torus", 3, 8, 8)])
def test_noise_covariance_is_quadrature_mass(kind, p, nu, nv):
    s = geo.Surface(kind, p, nu, nv)
    sp_ = GluedSpace(s)
    _, M = assemble(sp_)
    q = quadrature(s)
    nQ = n_quad(s)
    # columns of B: the loads of unit noise at each quadrature point
    B = np.stack([noise_from_xi(sp_, np.eye(1, nQ, j).ravel(), q) for j in range(nQ)], axis=1)
    np.testing.assert_allclose(B @ B.T, M.toarray(), atol=1e-15 * nQ, rtol=1e-12)
    # 1^T b = sum_q sqrt(w_q a_q) xi_q (partition of unity)
    xi = np.random.default_rng(5).standard_normal(nQ)
    wa = np.concatenate([np.sqrt(q["W"] * a).ravel() for a in q["a"]])
    assert noise_from_xi(sp_, xi, q).sum() == pytest.approx(wa @ xi, rel=1e-12)


def test_noise_loads_statistics():
    # sample covariance of the loads tends to M
    s = geo.Surface("sphere", 2, 1)
    sp_ = GluedSpace(s)
    _, M = assemble(sp_)
    b = noise_loads(sp_, seed=9, n_samples=4000)
    C = b.T @ b / len(b)
    Md = M.toarray()
    err = np.abs(C - Md).max() / np.abs(Md).max()
    assert err < 0.1


@pytest.mark.parametrize("kind,p,nu,nv", [("sphere", 2, 2, 2), ("torus", 3, 8, 4)])
def test_noise_adjoint_is_the_transpose(kind, p, nu, nv):
    # <B xi, g> = <xi, B^T g> for random xi and g, and B^T 1 = sqrt(w a) at
    # every Gauss point (the glued basis is a partition of unity)
    s = geo.Surface(kind, p, nu, nv)
    sp_ = GluedSpace(s)
    q = quadrature(s)
    nQ = n_quad(s)
    rng = np.random.default_rng(17)
    xi = rng.standard_normal(nQ)
    g = rng.standard_normal(sp_.N)
    bt = noise_adjoint(sp_, g, q)
    assert bt.shape == (nQ,)
    assert noise_from_xi(sp_, xi, q) @ g == pytest.approx(xi @ bt, rel=1e-12)
    wa = np.concatenate([np.sqrt(q["W"] * a).ravel() for a in q["a"]])
    np.testing.assert_allclose(noise_adjoint(sp_, np.ones(sp_.N), q), wa, rtol=1e-12)
    # column j of B^T is the load of unit noise at point j, read at DOF i
    B = np.stack([noise_from_xi(sp_, np.eye(1, nQ, j).ravel(), q) for j in range(0, nQ, 7)], axis=1)
    i = rng.integers(0, sp_.N, 5)
    for ii in i:
        e = np.zeros(sp_.N)
        e[ii] = 1.0
        np.testing.assert_allclose(noise_adjoint(sp_, e, q)[0::7], B[ii], rtol=1e-12, atol=1e-16)

