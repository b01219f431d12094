"""Workload descriptions and seeded synthetic inputs.

Shared by the tests, ``bench.py`` and ``__graft_entry__`` on both sides of the
parity check (the CUDA library and the CPU oracle).  It holds no arithmetic of
the method: only surface sizes, parameters, seeds and plain numpy draws of test
vectors.  The white noise itself is drawn inside each implementation from
Philox4x32-10 with the seeds given here.

Surfaces are the paper's analytic test geometries: the six-patch unit sphere
(Sec. 4.1) at dyadic refinement levels, and a doubly periodic torus.  There is
no public dataset; every input is synthetic.
"""
import numpy as np

# Each workload: surface (kind, p, elements per patch side), Matérn parameters,
# sinc node set y_l = l k for l in [l_lo, l_hi], sample count and seeds, solver
# (smoother degree and interval ratio where paper_2605_24882_gb300.autotune
# found a better pair than the library default 4 / 12).
WORKLOADS = {
    # plain method, FP64, one sample; sphere 6 x (8 x 8), p = 2, 488 glued DOFs
    "sphere_p2_j3_fp64": dict(
        kind="sphere", p=2, n_u=8, n_v=8, kappa=2.0, beta=0.75, split="standard",
        k=0.4, l_lo=-25, l_hi=25, n_samples=1, seed=0, precision="fp64",
        levels=3, rtol=1e-11),
    # batching + mixed precision; sphere 6 x (64 x 64), p = 2, 25,352 DOFs;
    # beta = 1.3: one integer solve, then beta' = 0.3 by 71 sinc nodes
    "sphere_p2_j6_mixed_s256": dict(
        kind="sphere", p=2, n_u=64, n_v=64, kappa=5.0, beta=1.3, split="standard",
        k=0.3, l_lo=-35, l_hi=35, n_samples=256, seed=0, precision="mixed",
        levels=7, rtol=1e-8, smoother_degree=5, cheb_ratio=8.0),
    # second geometry: periodic bicubic torus R = 1, r = 0.4, 512 x 256 elements
    "torus_p3_512x256_s1024": dict(
        kind="torus", p=3, n_u=512, n_v=256, R=1.0, r=0.4, kappa=10.0, beta=0.6,
        split="standard", k=0.3, l_lo=-35, l_hi=35, n_samples=1024, seed=0,
        precision="mixed", levels=6, rtol=1e-8, smoother_degree=6, cheb_ratio=24.0),
    # differentiation: sphere 6 x (128 x 128), p = 3, 101,402 DOFs; loss target seed 7
    "sphere_p3_j7_adjoint_s64": dict(
        kind="sphere", p=3, n_u=128, n_v=128, kappa=4.0, beta=0.8, split="standard",
        k=0.3, l_lo=-35, l_hi=35, n_samples=64, seed=0, target_seed=7,
        precision="fp64", levels=8, rtol=1e-12),
}


def uneven_instances(seed=11, n_inst=96, j_lo=3, j_hi=9):
    """The uneven multi-instance batch: spheres (p = 2) and tori (p = 3) at levels j.

    Sphere level j has 6 x 2^j x 2^j elements; torus level j has 2^{j+1} x 2^j.
    kappa ~ U[1, 20], beta ~ U[0.55, 1.95] with the improved split, 1..64 samples.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        j = int(rng.integers(j_lo, j_hi + 1))
        torus = bool(rng.integers(0, 2))
        d = dict(kappa=float(rng.uniform(1.0, 20.0)), beta=float(rng.uniform(0.55, 1.95)),
                 n_samples=int(rng.integers(1, 65)), seed=int(rng.integers(0, 2**31)),
                 split="improved", k=0.3, l_lo=-35, l_hi=35, precision="mixed", rtol=1e-8)
        if torus:
            d.update(kind="torus", p=3, n_u=2 ** (j + 1), n_v=2 ** j, R=1.0, r=0.4)
        else:
            d.update(kind="sphere", p=2, n_u=2 ** j, n_v=2 ** j)
        d["levels"] = j - 2 if torus else j + 1
        out.append(d)
    return out


def scaled(name, **over):
    """A copy of workload ``name`` with fields overridden (smaller test cases)."""
    d = dict(WORKLOADS[name])
    d.update(over)
    return d


def random_vectors(seed, n_vec, n):
    """[n_vec, n] float64 standard normal test vectors."""
    return np.random.default_rng(seed).standard_normal((n_vec, n))


def random_shifts(seed, n, lo=1e-2, hi=1e4):
    """n log-uniform shifts in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


# ---------------------------------------------------------------- NURBS inputs
# Geometry input for the NURBS surface kinds: control nets only (no method
# arithmetic).  A patch is a dict with degree_u, degree_v, knots_u, knots_v and
# cpw [n_v, n_u, 4] = (x, y, z, weight).

# Cube-face arrangement of six-patch surfaces: patch m maps (u, v) to the cube
# point whose coordinate a_axis is 2u-1, b_axis is 2v-1 and n_axis is n_sign
# (the arrangement the library's six-patch gluing expects).
CUBE_FACES = ((1, 2, 0, +1.0), (2, 1, 0, -1.0), (2, 0, 1, +1.0),
              (0, 2, 1, -1.0), (0, 1, 2, +1.0), (1, 0, 2, -1.0))

_H = np.sqrt(0.5)
# full circle as a rational quadratic curve: 9 control points (x, y, w), knots at quarters
_CIRCLE = np.array([[1, 0, 1], [1, 1, _H], [0, 1, 1], [-1, 1, _H], [-1, 0, 1],
                    [-1, -1, _H], [0, -1, 1], [1, -1, _H], [1, 0, 1]], dtype=np.float64)
_CIRCLE_KNOTS = np.array([0, 0, 0, .25, .25, .5, .5, .75, .75, 1, 1, 1], dtype=np.float64)


def nurbs_torus(R=1.0, r=0.4):
    """The torus ((R + r cos t) cos s, (R + r cos t) sin s, r sin t) exactly, as
    the tensor product of two rational quadratic circles (one periodic patch)."""
    cpw = np.zeros((9, 9, 4))
    for j in range(9):          # tube circle (v)
        cx, cz, wv = _CIRCLE[j]
        for i in range(9):      # main circle (u)
            ax, ay, wu = _CIRCLE[i]
            rho = R + r * cx
            cpw[j, i] = (ax * rho, ay * rho, r * cz, wu * wv)
    return [dict(degree_u=2, degree_v=2, knots_u=_CIRCLE_KNOTS.copy(), knots_v=_CIRCLE_KNOTS.copy(), cpw=cpw)]


def nurbs_bulged_cube(bulge=0.3, weight=1.0):
    """Six biquadratic patches on the cube [-1, 1]^3 in the cube-face arrangement:
    corner and edge-midpoint control points on the cube edges (shared exactly by
    neighbouring patches), the face centre pushed outward by `bulge` with
    weight `weight`.  bulge = 0 and weight = 1 give the flat cube surface."""
    knots = np.array([0, 0, 0, 1, 1, 1], dtype=np.float64)
    patches = []
    for ax, bx, nx, sg in CUBE_FACES:
        cpw = np.zeros((3, 3, 4))
        for j in range(3):
            for i in range(3):
                c = np.zeros(3)
                c[ax] = i - 1.0
                c[bx] = j - 1.0
                c[nx] = sg * (1.0 + (bulge if (i == 1 and j == 1) else 0.0))
                cpw[j, i, :3] = c
                cpw[j, i, 3] = weight if (i == 1 and j == 1) else 1.0
        patches.append(dict(degree_u=2, degree_v=2, knots_u=knots.copy(), knots_v=knots.copy(), cpw=cpw))
    return patches
