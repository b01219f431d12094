"""White-noise load vectors (Sec. 3.3).

Test infrastructure (see ``oracle/__init__``).

The discrete white noise must satisfy f ~ N(0, M).  It is drawn at the Gauss
points: b_i = sum_q sqrt(w_q a_q) xi_q phi_i(x_q) with i.i.d. xi_q ~ N(0, 1).
Written as b = B xi with B_iq = sqrt(w_q a_q) phi_i(x_q), Cov(b) = B B^T is the
mass matrix assembled with the same Gauss rule -- exactly, with no matrix square
root.

Global quadrature index (a format shared with the CUDA library):
q = ((m n_v + e_v) n_u + e_u) nq^2 + g_v nq + g_u.
"""
import numpy as np

from .assembly import local_bases, quadrature
from .philox import STREAM_NOISE, STREAM_TARGET, normals


def n_quad(surf):
    return surf.n_patches * surf.n_v * surf.n_u * surf.nq * surf.nq


def noise_from_xi(space, xi, quad=None):
    """b = B xi for xi given at all global quadrature points (length n_quad)."""
    surf = space.surf
    if quad is None:
        quad = quadrature(surf)
    phi, _, _ = local_bases(surf)
    conn = space.connectivity()
    nq = surf.nq
    xi = np.asarray(xi, dtype=np.float64).reshape(surf.n_patches, surf.n_v, surf.n_u, nq, nq)
    b = np.zeros(space.N)
    for m in range(surf.n_patches):
        wq = np.sqrt(quad["W"] * quad["a"][m]) * xi[m]
        loc = np.einsum("yxkgh,yxgh->yxk", phi, wq)
        np.add.at(b, conn[m].ravel(), loc.ravel())
    return b


def noise_adjoint(space, g, quad=None):
    """B^T g at all global quadrature points (length n_quad): the gradient of a
    loss with respect to the Gauss-point noise xi, given g = dL/db (b = B xi),
    (B^T g)_q = sqrt(w_q a_q) sum_i phi_i(x_q) g_i over the glued functions i
    whose support holds x_q."""
    surf = space.surf
    if quad is None:
        quad = quadrature(surf)
    phi, _, _ = local_bases(surf)
    conn = space.connectivity()
    g = np.asarray(g, dtype=np.float64)
    out = []
    for m in range(surf.n_patches):
        gl = g[conn[m]]  # [n_v, n_u, (p+1)^2]: the element's glued coefficients
        val = np.einsum("yxkgh,yxk->yxgh", phi, gl)
        out.append((np.sqrt(quad["W"] * quad["a"][m]) * val).ravel())
    return np.concatenate(out)


def noise_loads(space, seed, n_samples, quad=None):
    """[n_samples, N] load vectors of samples 0..n_samples-1 drawn with ``seed``."""
    q = np.arange(n_quad(space.surf))
    if quad is None:
        quad = quadrature(space.surf)
    return np.stack([noise_from_xi(space, normals(seed, s, q, STREAM_NOISE), quad)
                     for s in range(n_samples)])


def target_fields(space, seed, n_samples):
    """[n_samples, N] i.i.d. N(0,1) DOF coefficients (the loss target fields g_s)."""
    i = np.arange(space.N)
    return np.stack([normals(seed, s, i, STREAM_TARGET) for s in range(n_samples)])
