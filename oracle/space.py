"""The C0-glued spline space S^0_{j,p} on a multi-patch surface (Eq. def::space2).

Test infrastructure (see ``oracle/__init__``).

Global numbering rule (a format shared with the CUDA library, which derives it
by a different method -- combinatorial edge matching):
scan patches m = 0, 1, ...; within a patch scan local DOFs row by row
(i_v outer, i_u inner); a local DOF receives the index of an earlier local DOF
that is the same global function, else the next unused index.

Here two local DOFs are identified when their anchors F_m(greville) coincide:
on an open knot vector only the first/last function of a row is non-zero on a
patch edge, its Greville abscissa is exactly 0 or 1, and conforming patches
(Sec. 2.2) map these to the same physical points.

Periodic torus: local DOF (i_u, i_v) is global index i_v * n_u + i_u.
"""
import numpy as np
from scipy.spatial import cKDTree

from .bspline import open_knot_vector


def greville(n_el, p):
    """Greville abscissae of the p-open knot vector with n_el elements."""
    kn = open_knot_vector(n_el, p)
    return np.array([kn[i + 1:i + p + 1].mean() for i in range(n_el + p)])


class GluedSpace:
    """Local-to-global map and element connectivity of S^0_{j,p}."""

    def __init__(self, surf):
        self.surf = surf
        p = surf.p
        if surf.periodic:
            self.nloc_u, self.nloc_v = surf.n_u, surf.n_v
            l2g = np.arange(surf.n_u * surf.n_v, dtype=np.int64).reshape(1, surf.n_v, surf.n_u)
            self.l2g = l2g
            self.N = surf.n_u * surf.n_v
        else:
            n = surf.n_u
            self.nloc_u = self.nloc_v = n + p
            gv = greville(n, p)
            U, V = np.meshgrid(gv, gv)  # U[i_v, i_u]
            pts = np.concatenate([surf.map(m, U, V)[0].reshape(-1, 3)
                                  for m in range(surf.n_patches)])
            # identify coincident anchors (pairs closer than 1e-9), then number
            # in scan order: each point takes the index of its first twin
            first = np.arange(len(pts))
            for i, j in sorted(cKDTree(pts).query_pairs(1e-9)):
                first[j] = min(first[j], first[i])
            l2g_flat = np.full(len(pts), -1, dtype=np.int64)
            nxt = 0
            for i in range(len(pts)):
                if first[i] == i:
                    l2g_flat[i] = nxt
                    nxt += 1
                else:
                    l2g_flat[i] = l2g_flat[first[i]]
            l2g = l2g_flat.reshape(surf.n_patches, n + p, n + p)
            self.l2g = l2g
            self.N = nxt

    def connectivity(self):
        """[n_patches, n_v, n_u, (p+1)^2] global DOFs of every element."""
        s = self.surf
        p = s.p
        conn = np.zeros((s.n_patches, s.n_v, s.n_u, (p + 1) ** 2), dtype=np.int64)
        ku = np.arange(p + 1)
        for m in range(s.n_patches):
            for ev in range(s.n_v):
                for kv in range(p + 1):
                    if s.periodic:
                        iv = (ev - p + kv) % s.n_v
                        iu = (np.arange(s.n_u)[:, None] - p + ku[None, :]) % s.n_u
                    else:
                        iv = ev + kv
                        iu = np.arange(s.n_u)[:, None] + ku[None, :]
                    conn[m, ev, :, kv * (p + 1):(kv + 1) * (p + 1)] = self.l2g[m, iv][iu]
        return conn
