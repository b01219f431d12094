"""NURBS surface patches as the geometry map (Sec. 2.2, NURBS parametrisations).

Test infrastructure (see ``oracle/__init__``).

A patch of degrees (p_u, p_v) with knot vectors Xi_u, Xi_v on [0, 1] and
control points P_ij with weights w_ij maps
    F(u, v) = A(u, v) / W(u, v),  A = sum_ij N_i(u) M_j(v) w_ij P_ij,  W = sum_ij N_i(u) M_j(v) w_ij,
with N_i, M_j the B-splines of Definition 2.1 on Xi_u, Xi_v.  Its derivatives
follow from the quotient rule: d_u F = (d_u A - F d_u W) / W, and likewise in v.

``NurbsSurface`` has the interface of ``geometry.Surface`` (map, periodic,
n_patches, n_u, n_v, p, nq, coarsen), so the glued space, the quadrature and
the assembly of the oracle apply to it unchanged: topology "periodic" (one
patch, periodic in u and v, the torus's spline space) or "cube" (six patches
in the cube-face arrangement of the sphere, glued by matching anchors).
"""
import numpy as np

from .bspline import basis, basis_deriv


def patch_map(patch, u, v):
    """Point and first derivatives (F, F_u, F_v), each [..., 3], of one NURBS patch."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    shape = np.broadcast(u, v).shape
    uf = np.broadcast_to(u, shape).ravel()
    vf = np.broadcast_to(v, shape).ravel()
    pu, pv = patch["degree_u"], patch["degree_v"]
    Nu = basis(patch["knots_u"], pu, uf)            # [n, n_u]
    dNu = basis_deriv(patch["knots_u"], pu, uf)
    Nv = basis(patch["knots_v"], pv, vf)            # [n, n_v]
    dNv = basis_deriv(patch["knots_v"], pv, vf)
    cpw = np.asarray(patch["cpw"], dtype=np.float64)   # [n_v, n_u, 4]
    w = cpw[..., 3]
    wP = cpw[..., :3] * w[..., None]
    A = np.einsum("ni,nj,jic->nc", Nu, Nv, wP)
    Au = np.einsum("ni,nj,jic->nc", dNu, Nv, wP)
    Av = np.einsum("ni,nj,jic->nc", Nu, dNv, wP)
    W = np.einsum("ni,nj,ji->n", Nu, Nv, w)[:, None]
    Wu = np.einsum("ni,nj,ji->n", dNu, Nv, w)[:, None]
    Wv = np.einsum("ni,nj,ji->n", Nu, dNv, w)[:, None]
    F = A / W
    Fu = (Au - F * Wu) / W
    Fv = (Av - F * Wv) / W
    return F.reshape(shape + (3,)), Fu.reshape(shape + (3,)), Fv.reshape(shape + (3,))


class NurbsSurface:
    """A surface given by NURBS patches; `topology` is "periodic" or "cube"."""

    def __init__(self, topology, patches, p, n_u, n_v=None):
        if topology not in ("periodic", "cube"):
            raise ValueError("topology is 'periodic' or 'cube'")
        if len(patches) != (1 if topology == "periodic" else 6):
            raise ValueError("periodic takes one patch, cube six")
        self.kind = "nurbs"
        self.topology = topology
        self.patches = patches
        self.p = p
        self.n_u = n_u
        self.n_v = n_u if n_v is None else n_v
        self.periodic = topology == "periodic"
        self.n_patches = len(patches)
        self.nq = p + 1
        if not self.periodic and self.n_u != self.n_v:
            raise ValueError("cube-arranged patches are square")

    def map(self, m, u, v):
        return patch_map(self.patches[m], u, v)

    def coarsen(self):
        return NurbsSurface(self.topology, self.patches, self.p, self.n_u // 2, self.n_v // 2)

    def area_exact(self):
        return None
