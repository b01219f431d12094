"""Fractional powers: integer split, improved split and the sinc sum (Sec. 3.4).

Test infrastructure (see ``oracle/__init__``).

With A = kappa^2 M + S and L = M^{-1} A, the field is u = L^{-beta} M^{-1} f.

* Integer part (Sec. 3.4): A w_1 = f, A w_k = M w_{k-1}; then w_n = L^{-n} M^{-1} f.
* Fractional part beta' in (0,1), Eq. eq:beta-approx rewritten with y = -2t,
  node step k (the printed step 1/sqrt(K) in t is k = 2/sqrt(K) in y) and the
  printed "I" read as M (the discrete operator is M^{-1}A):
      L^{-beta'} v = sum_l c_l (S + sigma_l M)^{-1} M v,
      y_l = l k,  c_l = (sin(pi beta')/pi) k e^{(1-beta') y_l},  sigma_l = e^{y_l} + kappa^2,
  for l = l_lo .. l_hi.  The Balakrishnan exponent is read as -beta.
* Improved split (Sec. 3.4): for beta' in (0, 1/3) and n >= 1 use
  beta = (n-1) + 2 beta'', beta'' = (beta'+1)/2; for beta' in (2/3, 1) use
  beta = n + 2 beta'', beta'' = beta'/2; the sinc map for beta'' is applied twice
  with the same node range, the second time to M times the first result.  At
  the open interval ends, and for n = 0 with beta' < 1/3, the standard split is used.

Solves are direct sparse LU factorisations (scipy ``splu``), one per shift,
reused for all samples.
"""
import math

import numpy as np
import scipy.sparse.linalg as spla

STANDARD = "standard"
IMPROVED = "improved"


def split_beta(beta, mode=STANDARD):
    """Return (n_int, beta_frac, n_passes) of the integer/fractional split."""
    if beta <= 0:
        raise ValueError("beta must be positive")
    n = int(math.floor(beta))
    bp = beta - n
    if bp == 0.0:
        return n, 0.0, 0
    if mode == IMPROVED:
        if bp < 1.0 / 3.0 and n >= 1:
            return n - 1, (bp + 1.0) / 2.0, 2
        if bp > 2.0 / 3.0:
            return n, bp / 2.0, 2
    return n, bp, 1


def sinc_rule(beta_frac, k, l_lo, l_hi):
    """Nodes y_l, weights c_l for l = l_lo..l_hi (Eq. eq:beta-approx in y = -2t)."""
    l = np.arange(l_lo, l_hi + 1, dtype=np.float64)
    y = l * k
    c = math.sin(math.pi * beta_frac) / math.pi * k * np.exp((1.0 - beta_frac) * y)
    return y, c


def auto_nodes(beta_frac, kappa, tol):
    """Sinc step k and node range [l_lo, l_hi] for an absolute error <= tol per
    unit load (Eq. eq:K-convergence measures the error against ||f||).

    In y = -2t the rule of Eq. eq:beta-approx is a trapezoidal sum of
    f(y) = s e^{(1-g) y} / (e^y + mu), s = sin(pi g) / pi, whose integral is
    mu^{-g} for every eigenvalue mu >= kappa^2 of M^{-1}(S + kappa^2 M).
    Three parts of the error are set to tol / 3 each:
      * the step, from the trapezoidal bound for functions analytic in the
        strip |Im y| < pi/2 (the poles sit at Im y = +-pi): 2 M' e^{-pi^2/k},
        with M' = 2 s (1/g + 1/((1-g) kappa^2)) bounding the strip integral;
      * the upper tail, sum over y > y_hi ~ s e^{-g y_hi} / g;
      * the lower tail, sum over y < y_lo ~ s e^{(1-g) y_lo} / ((1-g) kappa^2).
    """
    g = float(beta_frac)
    if not 0.0 < g < 1.0 or not kappa > 0.0 or not 0.0 < tol < 1.0:
        raise ValueError("need 0 < beta_frac < 1, kappa > 0, 0 < tol < 1")
    s = math.sin(math.pi * g) / math.pi
    mu = kappa * kappa
    m = 2.0 * s * (1.0 / g + 1.0 / ((1.0 - g) * mu))
    k = math.pi ** 2 / math.log(3.0 * m / tol)
    y_hi = math.log(3.0 * s / (g * tol)) / g
    y_lo = math.log(tol * (1.0 - g) * mu / (3.0 * s)) / (1.0 - g)
    return k, int(math.floor(y_lo / k)), int(math.ceil(y_hi / k))


def scalar_sinc(beta_frac, K, lam):
    """The paper's scalar u_K(lambda) with K (2K+1 nodes, t_k = k/sqrt(K))."""
    y, c = sinc_rule(beta_frac, 2.0 / math.sqrt(K), -K, K)
    return float(np.sum(c / (np.exp(y) + lam)))


class Shifted:
    """Factorisations of S + sigma M, cached per shift.

    S + sigma M is symmetric (both bilinear forms of Sec. 3.2 are), so the LU
    factorisation takes the symmetric minimum-degree ordering of its pattern;
    the solve is the same direct solve, with far less fill on large meshes.
    """

    def __init__(self, S, M):
        self.S = S.tocsc()
        self.M = M.tocsc()
        self.cache = {}

    def solve(self, sigma, rhs):
        key = float(sigma)
        if key not in self.cache:
            self.cache[key] = spla.splu((self.S + sigma * self.M).tocsc(), permc_spec="MMD_AT_PLUS_A")
        return self.cache[key].solve(rhs)


def fractional_apply(sh, M, beta_frac, kappa, k, l_lo, l_hi, v, return_terms=False):
    """L^{-beta'} applied to columns of v ([N, ns]) by the sinc sum."""
    y, c = sinc_rule(beta_frac, k, l_lo, l_hi)
    rhs = M @ v
    u = np.zeros_like(v)
    terms = []
    for yl, cl in zip(y, c):
        x = sh.solve(math.exp(yl) + kappa**2, rhs)
        u += cl * x
        if return_terms:
            terms.append(x)
    return (u, terms) if return_terms else u


def sample_fields(S, M, b, kappa, beta, k, l_lo, l_hi, mode=STANDARD, sh=None):
    """Fields u_s ([ns, N]) for loads b ([ns, N]) by the split and the sinc sum."""
    if sh is None:
        sh = Shifted(S, M)
    n, bp, passes = split_beta(beta, mode)
    w = np.asarray(b, dtype=np.float64).T.copy()  # [N, ns]
    # w_0 := M^{-1} b so that every pass starts from L^{-1} style updates
    if n >= 1:
        w = sh.solve(kappa**2, w)
        for _ in range(n - 1):
            w = sh.solve(kappa**2, M @ w)
        v = w
    else:
        v = None
    if passes == 0:
        return v.T
    for p_ in range(passes):
        if v is None:
            # n = 0: the first pass takes the load itself (M M^{-1} b = b)
            y, c = sinc_rule(bp, k, l_lo, l_hi)
            u = np.zeros_like(w)
            for yl, cl in zip(y, c):
                u += cl * sh.solve(math.exp(yl) + kappa**2, w)
            v = u
        else:
            v = fractional_apply(sh, M, bp, kappa, k, l_lo, l_hi, v)
    return v.T


def field_loss_grad(S, M, b, g, kappa, beta, k, l_lo, l_hi, mode=STANDARD):
    """Loss L = sum_s ||u_s - g_s||_M^2 and its gradients by the adjoint identity.

    Returns (L, dL/db [ns, N], dL/dkappa) for every split: n >= 0 integer
    solves and 0, 1 or 2 fractional passes (the improved split of Sec. 3.4
    applies the sinc map twice, the second time to M times the first result).
    Derivation: a pass maps its right-hand side r to v = sum_l c_l x_l,
    x_l = A_l^{-1} r, A_l = S + sigma_l M, sigma_l = e^{y_l} + kappa^2.  With
    the symmetric A_l its adjoint maps dL/dv to dL/dr = sum_l c_l z_l,
    z_l = A_l^{-1} dL/dv, and dx_l/dkappa = -A_l^{-1} (2 kappa M) x_l adds
    -2 kappa c_l z_l^T M x_l to dL/dkappa; dL/du = gt = 2 M (u - g).  A pass
    after the first (or after integer solves) takes r = M v_prev, so
    dL/dv_prev = M dL/dr.  The integer chain w_i = A0^{-1} M w_{i-1}
    (A0 = S + kappa^2 M, w_1 = A0^{-1} b) is differentiated the same way.
    """
    sh = Shifted(S, M)
    n, bp, passes = split_beta(beta, mode)
    y, c = sinc_rule(bp, k, l_lo, l_hi)
    sig = np.exp(y) + kappa**2
    B = np.asarray(b, dtype=np.float64).T
    ws = []
    v = None
    if n >= 1:
        w = sh.solve(kappa**2, B)
        ws.append(w)
        for _ in range(n - 1):
            w = sh.solve(kappa**2, M @ w)
            ws.append(w)
        v = w
    # fractional passes: the right-hand side is b (first pass with n = 0) or M v
    xss = []
    for _ in range(passes):
        r = B if v is None else M @ v
        xs = [sh.solve(s, r) for s in sig]
        v = sum(cl * x for cl, x in zip(c, xs))
        xss.append(xs)
    u = v
    G = np.asarray(g, dtype=np.float64).T
    d = u - G
    L = float(np.sum(d * (M @ d)))
    gt = 2.0 * (M @ d)
    dk = 0.0
    dout = gt  # dL/d(output of the step being differentiated)
    dLdr = None
    for p_ in range(passes - 1, -1, -1):
        zs = [sh.solve(s, dout) for s in sig]
        dLdr = sum(cl * z for cl, z in zip(c, zs))
        for cl, x, z in zip(c, xss[p_], zs):
            dk += -2.0 * kappa * cl * float(np.sum(z * (M @ x)))
        if p_ > 0 or n >= 1:
            dout = M @ dLdr  # r = M v_prev
    if n >= 1:
        # dL/dw_n = dout; w_i = A0^{-1} (M w_{i-1}) (w_1 = A0^{-1} b): lambda_i = A0^{-1} dL/dw_i
        lam = sh.solve(kappa**2, dout)
        for i in range(n - 1, -1, -1):
            # w_{i+1} depends on kappa through A0: dw/dkappa = -A0^{-1} 2 kappa M w
            dk += -2.0 * kappa * float(np.sum(lam * (M @ ws[i])))
            if i > 0:
                lam = sh.solve(kappa**2, M @ lam)
        dLdb = lam
    else:
        dLdb = dLdr
    return L, dLdb.T, dk
