"""Mass and stiffness matrices of S^0_{j,p} (Eqs. eq:FEM, eq:mass, eq:stiffness).

Test infrastructure (see ``oracle/__init__``).

M_ij = sum_m int_{[0,1]^2} phi_j phi_i a_m,
S_ij = sum_m int_{[0,1]^2} [d_u phi_j, d_v phi_j] K_m^{-1} [d_u phi_i, d_v phi_i]^T a_m,
evaluated with the tensor Gauss–Legendre rule of nq = p+1 points per element
direction (the same rule as the white-noise loads), element by element, and
summed into a global CSR matrix.  The element matrices are written out with
einsum over all quadrature points -- no sum factorisation or other reordering.
"""
import numpy as np
import scipy.sparse as sp

from .bspline import element_tables, gauss_legendre01
from .geometry import metric


def quadrature(surf):
    """Gauss points of every element of every patch with the metric there.

    Returns dict with u, v [n_v, n_u, nq, nq] (parameter coordinates, indexed
    [e_v, e_u, g_v, g_u]), weights W (same shape, including the element size
    1/(n_u n_v)), and a, G11, G12, G22 per patch as lists.
    """
    nq = surf.nq
    g, w = gauss_legendre01(nq)
    eu = np.arange(surf.n_u)
    ev = np.arange(surf.n_v)
    U = ((eu[None, :, None, None] + g[None, None, None, :]) / surf.n_u
         + 0 * ev[:, None, None, None] + 0 * g[None, None, :, None])
    V = ((ev[:, None, None, None] + g[None, None, :, None]) / surf.n_v
         + 0 * eu[None, :, None, None] + 0 * g[None, None, None, :])
    W = (w[:, None] * w[None, :])[None, None] / (surf.n_u * surf.n_v) + 0 * U
    out = {"u": U, "v": V, "W": W, "a": [], "G11": [], "G12": [], "G22": []}
    for m in range(surf.n_patches):
        _, Fu, Fv = surf.map(m, U, V)
        a, G11, G12, G22 = metric(Fu, Fv)
        out["a"].append(a)
        out["G11"].append(G11)
        out["G12"].append(G12)
        out["G22"].append(G22)
    return out


def local_bases(surf):
    """2D basis values and parameter derivatives on every element.

    Returns phi, du, dv with shape [n_v, n_u, (p+1)^2, nq, nq] (local index
    k = k_v (p+1) + k_u; quadrature index [g_v, g_u]).
    """
    p, nq = surf.p, surf.nq
    vu, du_, _ = element_tables(surf.n_u, p, nq, surf.periodic)
    vv, dv_, _ = element_tables(surf.n_v, p, nq, surf.periodic)
    # [e_v, e_u, k_v, k_u, g_v, g_u]
    phi = np.einsum("yag,xbh->yxabgh", vv, vu)
    du = np.einsum("yag,xbh->yxabgh", vv, du_)
    dv = np.einsum("yag,xbh->yxabgh", dv_, vu)
    sh = (surf.n_v, surf.n_u, (p + 1) ** 2, nq, nq)
    return phi.reshape(sh), du.reshape(sh), dv.reshape(sh)


def element_matrices(surf, quad=None):
    """Element mass and stiffness matrices per patch: lists of [n_v, n_u, k, l]."""
    if quad is None:
        quad = quadrature(surf)
    phi, du, dv = local_bases(surf)
    W = quad["W"]
    Me, Se = [], []
    for m in range(surf.n_patches):
        a = quad["a"][m]
        G11, G12, G22 = quad["G11"][m], quad["G12"][m], quad["G22"][m]
        Me.append(np.einsum("yxkgh,yxgh,yxlgh->yxkl", phi, W * a, phi))
        gu = G11[:, :, None] * du + G12[:, :, None] * dv   # (G grad phi_l)_u
        gv = G12[:, :, None] * du + G22[:, :, None] * dv
        Se.append(np.einsum("yxkgh,yxgh,yxlgh->yxkl", du, W, gu)
                  + np.einsum("yxkgh,yxgh,yxlgh->yxkl", dv, W, gv))
    return Me, Se


def assemble(space, quad=None):
    """Global (S, M) as scipy CSR matrices in float64."""
    surf = space.surf
    conn = space.connectivity()
    Me, Se = element_matrices(surf, quad)
    N = space.N
    S = sp.csr_matrix((N, N))
    M = sp.csr_matrix((N, N))
    nk = conn.shape[-1]
    for m in range(surf.n_patches):
        c = conn[m].reshape(-1, nk)
        rows = np.repeat(c, nk, axis=1).ravel()
        cols = np.tile(c, (1, nk)).ravel()
        M = M + sp.coo_matrix((Me[m].ravel(), (rows, cols)), shape=(N, N)).tocsr()
        S = S + sp.coo_matrix((Se[m].ravel(), (rows, cols)), shape=(N, N)).tocsr()
    S.sum_duplicates()
    M.sum_duplicates()
    return S.tocsr(), M.tocsr()


def load_vector(space, f, quad=None):
    """Load vector F_i = <f, phi_i> by the same Gauss rule; f(x) takes [...,3] points."""
    surf = space.surf
    if quad is None:
        quad = quadrature(surf)
    phi, _, _ = local_bases(surf)
    conn = space.connectivity()
    F = np.zeros(space.N)
    for m in range(surf.n_patches):
        X, _, _ = surf.map(m, quad["u"], quad["v"])
        fq = f(X) * quad["W"] * quad["a"][m]
        loc = np.einsum("yxkgh,yxgh->yxk", phi, fq)
        np.add.at(F, conn[m].ravel(), loc.ravel())
    return F


def evaluate(space, coef, m, u, v):
    """Value of the glued spline with coefficients ``coef`` at parameters (u, v) of patch m."""
    from .bspline import basis, open_knot_vector, periodic_basis
    surf = space.surf
    u = np.atleast_1d(u)
    v = np.atleast_1d(v)
    if surf.periodic:
        Bu = periodic_basis(surf.n_u, surf.p, u)
        Bv = periodic_basis(surf.n_v, surf.p, v)
    else:
        Bu = basis(open_knot_vector(surf.n_u, surf.p), surf.p, u)
        Bv = basis(open_knot_vector(surf.n_v, surf.p), surf.p, v)
    C = coef[space.l2g[m]]  # [i_v, i_u]
    return np.einsum("ni,ji,nj->n", Bu, C, Bv)
