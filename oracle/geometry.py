"""Surface parametrisations and pulled-back metric terms (Secs. 2.2 and 3.2).

Test infrastructure (see ``oracle/__init__``).

Cube-sphere: six patches F_m(u, v) = c_m(u, v) / |c_m(u, v)| (gnomonic reading
of the paper's six-patch unit sphere), with c_m the point of cube face m:
the coordinate ``a_axis`` carries 2u-1, ``b_axis`` carries 2v-1 and
``n_axis`` is fixed to ``n_sign``.  The face table is a format shared with the
CUDA library (both sides must parametrise the same patches); the interface
identification is derived independently on each side.

Torus: one doubly periodic patch
F(u, v) = ((R + r cos 2 pi v) cos 2 pi u, (R + r cos 2 pi v) sin 2 pi u, r sin 2 pi v).

Metric (Sec. 3.2): K = [dF_u.dF_u, dF_u.dF_v; dF_v.dF_u, dF_v.dF_v],
a = sqrt(det K), and the stiffness weight G = a K^{-1}.
"""
import numpy as np

# (a_axis, b_axis, n_axis, n_sign) for patches 0..5: +x, -x, +y, -y, +z, -z
CUBE_FACES = (
    (1, 2, 0, +1.0),
    (2, 1, 0, -1.0),
    (2, 0, 1, +1.0),
    (0, 2, 1, -1.0),
    (0, 1, 2, +1.0),
    (1, 0, 2, -1.0),
)


def sphere_map(m, u, v):
    """Point and first derivatives of patch m of the cube-sphere.

    Returns (F, Fu, Fv), each [..., 3].
    """
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    ax, bx, nx, sg = CUBE_FACES[m]
    c = np.zeros(u.shape + (3,))
    c[..., ax] = 2.0 * u - 1.0
    c[..., bx] = 2.0 * v - 1.0
    c[..., nx] = sg
    cu = np.zeros(3)
    cu[ax] = 2.0
    cv = np.zeros(3)
    cv[bx] = 2.0
    nrm = np.sqrt(np.sum(c * c, axis=-1))[..., None]
    F = c / nrm
    Fu = cu / nrm - c * (c @ cu)[..., None] / nrm**3
    Fv = cv / nrm - c * (c @ cv)[..., None] / nrm**3
    return F, Fu, Fv


def torus_map(u, v, R, r):
    """Point and first derivatives of the periodic torus patch."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    tu = 2.0 * np.pi * u
    tv = 2.0 * np.pi * v
    rho = R + r * np.cos(tv)
    F = np.stack([rho * np.cos(tu), rho * np.sin(tu), r * np.sin(tv)], axis=-1)
    Fu = np.stack([-2 * np.pi * rho * np.sin(tu), 2 * np.pi * rho * np.cos(tu),
                   np.zeros_like(tu)], axis=-1)
    Fv = np.stack([-2 * np.pi * r * np.sin(tv) * np.cos(tu),
                   -2 * np.pi * r * np.sin(tv) * np.sin(tu),
                   2 * np.pi * r * np.cos(tv)], axis=-1)
    return F, Fu, Fv


def metric(Fu, Fv):
    """First fundamental form K, surface measure a and G = a K^{-1} (Sec. 3.2).

    Returns (a, G11, G12, G22), each of the leading shape of Fu.
    """
    K11 = np.sum(Fu * Fu, axis=-1)
    K12 = np.sum(Fu * Fv, axis=-1)
    K22 = np.sum(Fv * Fv, axis=-1)
    det = K11 * K22 - K12 * K12
    a = np.sqrt(det)
    return a, K22 / a, -K12 / a, K11 / a


class Surface:
    """A surface description: kind 'sphere' (6 patches) or 'torus' (1 patch)."""

    def __init__(self, kind, p, n_u, n_v=None, R=1.0, r=0.4):
        self.kind = kind
        self.p = p
        self.n_u = n_u
        self.n_v = n_u if n_v is None else n_v
        self.R = R
        self.r = r
        self.periodic = kind == "torus"
        self.n_patches = 6 if kind == "sphere" else 1
        if kind == "sphere" and self.n_u != self.n_v:
            raise ValueError("cube-sphere patches are square")
        self.nq = p + 1

    def map(self, m, u, v):
        if self.kind == "sphere":
            return sphere_map(m, u, v)
        return torus_map(u, v, self.R, self.r)

    def coarsen(self):
        """The surface at the next coarser dyadic level."""
        if self.kind == "sphere":
            return Surface("sphere", self.p, self.n_u // 2)
        return Surface("torus", self.p, self.n_u // 2, self.n_v // 2, self.R, self.r)

    def area_exact(self):
        if self.kind == "sphere":
            return 4.0 * np.pi
        return 4.0 * np.pi**2 * self.R * self.r
