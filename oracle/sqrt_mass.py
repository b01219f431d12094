"""Noise loads f = sqrt(M) y by the Hale–Higham–Trefethen sum (Sec. 3.3, Eq. eq:sqrt).

Test infrastructure (see ``oracle/__init__``).

For a symmetric positive definite A with spectrum inside [lo, hi]:
    A^{-1/2} = (2/pi) int_0^inf (A + w^2 I)^{-1} dw.
The substitution w = sqrt(lo) sn(t|q) / cn(t|q) with the elliptic parameter
q = 1 - lo/hi maps t in [0, K(q)) onto w in [0, inf), with
dw/dt = sqrt(lo) dn(t|q) / cn(t|q)^2 and K(q) the complete elliptic integral of
the first kind.  The integrand is even and 2K-periodic in t, so the midpoint
rule with K^ nodes t_k = (k - 1/2) K / K^ converges exponentially:
    A^{1/2} y ~= A sum_k c_k (A + w_k^2 I)^{-1} y,
    c_k = 2 K sqrt(lo) dn(t_k|q) / (pi K^ cn(t_k|q)^2),  w_k = sqrt(lo) sn(t_k|q) / cn(t_k|q).
Reading: the paper's prefactor and node spacing name the complete elliptic
integral of the second kind; the substitution above makes both K(q), the
integral of the first kind, with parameter 1 - 1/kappa_M.

The spectrum bounds of the assembled mass matrix come from its definition:
M = sum_e M_e with every element matrix M_e positive definite on its (p+1)^2
local functions (distinct DOFs).  With D_e = diag(M_e) and
B_e = D_e^{-1/2} M_e D_e^{-1/2}, x_e^T M_e x_e >= lambda_min(B_e) x_e^T D_e x_e,
and the D_e sum to diag(M), so lambda_min(M) >= min_e lambda_min(B_e) min_i M_ii.
M has non-negative entries, so its largest eigenvalue is at most its largest
row sum.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.special as sps

from .assembly import assemble, element_matrices


def hht_rule(lo, hi, n_nodes):
    """Shifts w_k^2 and weights c_k of the K^ = n_nodes point rule for A^{1/2} = A sum_k c_k (A + w_k^2)^{-1}."""
    if not 0.0 < lo < hi or n_nodes < 1:
        raise ValueError("need 0 < lo < hi and n_nodes >= 1")
    q = 1.0 - lo / hi
    K = sps.ellipk(q)
    t = (np.arange(1, n_nodes + 1) - 0.5) * K / n_nodes
    sn, cn, dn, _ = sps.ellipj(t, q)
    w2 = lo * (sn / cn) ** 2
    c = 2.0 * K * math.sqrt(lo) / (math.pi * n_nodes) * dn / cn ** 2
    # Past K/2, cn(t) is small and known only to absolute accuracy; there the
    # quarter-period reflection u = K - t (sn(t) = cn(u)/dn(u),
    # cn(t) = k' sn(u)/dn(u), dn(t) = k'/dn(u)) gives the same values from
    # functions of the small argument u.  k'^2 is taken as 1 - q, the
    # complementary parameter of the q the elliptic functions were given.
    far = t > 0.5 * K
    kp2 = 1.0 - q
    snu, cnu, dnu, _ = sps.ellipj(K - t[far], q)
    w2[far] = lo / kp2 * (cnu / snu) ** 2
    c[far] = 2.0 * K * math.sqrt(lo / kp2) / (math.pi * n_nodes) * dnu / snu ** 2
    return w2, c


def sqrt_apply(A, y, lo, hi, n_nodes):
    """A^{1/2} y ([N] or [N, ns]) by the rule, with one sparse LU per shift."""
    A = sp.csc_matrix(A)
    w2, c = hht_rule(lo, hi, n_nodes)
    eye = sp.identity(A.shape[0], format="csc")
    acc = np.zeros_like(np.asarray(y, dtype=np.float64))
    for wk, ck in zip(w2, c):
        acc += ck * spla.splu((A + wk * eye).tocsc()).solve(y)
    return A @ acc


def mass_spectrum_bounds(space, quad=None):
    """(lo, hi) with lo <= lambda_min(M) and lambda_max(M) <= hi for the assembled M."""
    Me, _ = element_matrices(space.surf, quad)
    lam = np.inf
    for Mm in Me:
        A = Mm.reshape(-1, Mm.shape[-2], Mm.shape[-1])
        d = np.sqrt(np.einsum("eii->ei", A))
        lam = min(lam, float(np.linalg.eigvalsh(A / d[:, :, None] / d[:, None, :]).min()))
    _, M = assemble(space, quad)
    hi = float(np.abs(M).sum(axis=1).max())
    return lam * float(M.diagonal().min()), hi


def noise_loads_sqrt(M, lo, hi, n_nodes, y):
    """Loads f_s = sqrt(M) y_s for i.i.d. N(0,1) DOF vectors y ([ns, N]); Cov(f) = M."""
    return sqrt_apply(M, np.asarray(y, dtype=np.float64).T, lo, hi, n_nodes).T
