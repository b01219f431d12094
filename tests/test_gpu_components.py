"""GPU parity of each step of the path against the CPU oracle, through the C ABI."""
import os

import numpy as np
import pytest
import torch

from oracle import geometry as geo
from oracle.assembly import assemble, evaluate, quadrature
from oracle.noise import n_quad, noise_loads
from oracle.philox import normals as or_normals
from oracle.philox import philox4x32_10 as or_philox
from oracle.space import GluedSpace
from wm_workloads import random_shifts, random_vectors

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")

SURFS = [("sphere", 2, 8, 8, 3), ("sphere", 3, 4, 4, 2), ("torus", 3, 32, 16, 2), ("sphere", 1, 4, 4, 3)]


@pytest.fixture(scope="module")
def wm():
    from paper_2605_24882_gb300 import build as b
    b.build()
    import paper_2605_24882_gb300 as wm
    return wm


_cache = {}


def setup(wm, kind, p, nu, nv, levels):
    key = (kind, p, nu, nv, levels)
    if key not in _cache:
        hier = wm.Hierarchy(wm.Geometry(kind, p, nu, nv), levels)
        s = geo.Surface(kind, p, nu, nv)
        sp_ = GluedSpace(s)
        S, M = assemble(sp_)
        _cache[key] = (hier, s, sp_, S, M)
    return _cache[key]


@pytest.mark.parametrize("surf", SURFS)
def test_dof_map_bit_exact(wm, surf):
    hier, s, sp_, S, M = setup(wm, *surf)
    assert hier.num_dofs(0) == sp_.N
    assert np.array_equal(hier.dof_map(0), sp_.l2g.astype(np.int32))
    # coarser levels too
    for l in range(1, surf[4]):
        sc = geo.Surface(surf[0], surf[1], surf[2] >> l, surf[3] >> l)
        assert np.array_equal(hier.dof_map(l), GluedSpace(sc).l2g.astype(np.int32))


@pytest.mark.parametrize("surf", SURFS)
def test_metric(wm, surf):
    hier, s, sp_, S, M = setup(wm, *surf)
    q = quadrature(s)
    mt = hier.metric(0).cpu().numpy()
    ref = np.stack([np.stack([q[k][m] for k in ("a", "G11", "G12", "G22")], -1).reshape(-1, 4)
                    for m in range(s.n_patches)])
    np.testing.assert_allclose(mt, ref.reshape(-1, 4), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("surf", SURFS)
def test_apply_shifted_fp64_and_fp32(wm, surf):
    hier, s, sp_, S, M = setup(wm, *surf)
    nv = 37  # two tiles, ragged tail
    x = random_vectors(1, nv, sp_.N)
    sg = random_shifts(2, nv)
    ref = (S @ x.T).T + sg[:, None] * (M @ x.T).T
    xt = torch.tensor(x, device="cuda")
    y = hier.apply_shifted(xt, sg, precision="fp64").cpu().numpy()
    scale = np.abs(S).sum(1).max() + sg.max() * np.abs(M).sum(1).max()
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-13 * scale * np.abs(x).max())
    y32 = hier.apply_shifted(xt, sg, precision="mixed").cpu().numpy()
    np.testing.assert_allclose(y32, ref, rtol=0, atol=2e-6 * scale * np.abs(x).max())
    ym = hier.apply_mass(xt).cpu().numpy()
    np.testing.assert_allclose(ym, (M @ x.T).T, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("surf", SURFS[:3])
def test_apply_coarse_levels(wm, surf):
    hier, *_ = setup(wm, *surf)
    for l in range(1, surf[4]):
        sc = geo.Surface(surf[0], surf[1], surf[2] >> l, surf[3] >> l)
        S, M = assemble(GluedSpace(sc))
        x = random_vectors(3, 5, S.shape[0])
        sg = random_shifts(4, 5)
        y = hier.apply_shifted(torch.tensor(x, device="cuda"), sg, level=l).cpu().numpy()
        np.testing.assert_allclose(y, (S @ x.T).T + sg[:, None] * (M @ x.T).T, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("surf", SURFS[:3])
def test_prolongation_reproduces_coarse_spline(wm, surf):
    hier, s, sp_, S, M = setup(wm, *surf)
    sc = geo.Surface(surf[0], surf[1], surf[2] >> 1, surf[3] >> 1)
    spc = GluedSpace(sc)
    xc = random_vectors(5, 3, spc.N)
    xf = hier.prolongate(torch.tensor(xc, device="cuda"), level=0).cpu().numpy()
    rng = np.random.default_rng(6)
    for m in range(s.n_patches):
        u, v = rng.random(25), rng.random(25)
        for k in range(3):
            np.testing.assert_allclose(evaluate(sp_, xf[k], m, u, v), evaluate(spc, xc[k], m, u, v),
                                       rtol=1e-12, atol=1e-12)
    # restriction is the transpose: <R r, xc> = <r, P xc>
    r = random_vectors(7, 3, sp_.N)
    rc = hier.restrict(torch.tensor(r, device="cuda"), level=0).cpu().numpy()
    np.testing.assert_allclose(np.sum(rc * xc, 1), np.sum(r * xf, 1), rtol=1e-12)


def test_philox_known_answers_and_streams(wm):
    rows = [[int(t, 16) for t in l.split()] for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if not l.startswith("#")]
    for v in rows:
        ctr = torch.tensor(np.array(v[:4], dtype=np.uint32).view(np.int32)[None], device="cuda")
        out = wm.philox4x32_10(ctr, v[4] | (v[5] << 32)).cpu().numpy().view(np.uint32)[0]
        assert [int(o) for o in out] == v[6:]
    rng = np.random.default_rng(8)
    ctr = rng.integers(0, 2**32, size=(1000, 4), dtype=np.uint64).astype(np.uint32)
    key = 0x1234567890ABCDEF
    out = wm.philox4x32_10(torch.tensor(ctr.view(np.int32), device="cuda"), key).cpu().numpy().view(np.uint32)
    ref = or_philox(ctr.T.astype(np.uint64), np.array([key & 0xFFFFFFFF, key >> 32], dtype=np.uint64)).T
    assert np.array_equal(out, ref)


def test_normals(wm):
    for seed, sample, stream, q0, n in [(0, 0, 0, 0, 1001), (7, 3, 1, 12345, 999), (2**40 + 3, 255, 0, 2**33, 64)]:
        z = wm.normals(seed, sample, stream, q0, n).cpu().numpy()
        ref = or_normals(seed, sample, np.arange(q0, q0 + n), stream)
        np.testing.assert_allclose(z, ref, rtol=4e-15, atol=4e-15)


@pytest.mark.parametrize("surf", SURFS[:3])
def test_noise_loads(wm, surf):
    hier, s, sp_, S, M = setup(wm, *surf)
    b = hier.noise_loads(seed=11, n_samples=35).cpu().numpy()
    ref = noise_loads(sp_, 11, 35)
    np.testing.assert_allclose(b, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vcycle_is_a_good_symmetric_preconditioner(wm, precision):
    hier, s, sp_, S, M = setup(wm, "sphere", 2, 8, 8, 3)
    nv = 6
    sg = np.array([0.05, 1.0, 25.0, 400.0, 1e4, 3e4])
    r = random_vectors(9, nv, sp_.N)
    z = hier.vcycle(torch.tensor(r, device="cuda"), sg, precision=precision, smoother_degree=2).cpu().numpy()
    import scipy.sparse.linalg as spla
    for k in range(nv):
        A = (S + sg[k] * M).tocsc()
        x = spla.spsolve(A, r[k])
        e = z[k] - x
        rel = np.sqrt(e @ (A @ e) / (x @ (A @ x)))
        assert rel < 0.6, (k, sg[k], rel)
    if precision == "fp64":
        r2 = random_vectors(10, nv, sp_.N)
        z2 = hier.vcycle(torch.tensor(r2, device="cuda"), sg, precision=precision).cpu().numpy()
        np.testing.assert_allclose(np.sum(z * r2, 1), np.sum(r * z2, 1), rtol=1e-9)


def test_schedule_changes_only_rounding(wm):
    # the kernel schedule maps the same solves onto the SMs differently: fields
    # agree to the solver tolerance, values out of range are refused
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 16), 4)
    kw = dict(kappa=3.0, beta=1.3, sinc_k=0.4, l_lo=-15, l_hi=15, n_samples=40, seed=2, precision="mixed",
              rtol=1e-10)
    assert hier.schedule() == {"uni_run": 8, "uni_waves": 4, "vec_rows": 128, "vcycle_rows": 16, "tail_fused": 1}
    u0, _ = hier.sample_fields(**kw)
    hier.set_schedule(uni_run=2, uni_waves=16, vec_rows=64, vcycle_rows=32, tail_fused=0)
    u1, st = hier.sample_fields(**kw)
    assert st["n_not_converged"] == 0
    d = u1 - u0
    assert float(torch.sqrt((d * hier.apply_mass(d)).sum() / (u0 * hier.apply_mass(u0)).sum())) < 1e-8
    with pytest.raises(wm.WMError):
        hier.set_schedule(uni_run=9)
    with pytest.raises(wm.WMError):
        hier.set_schedule(tail_fused=2)
    assert hier.set_schedule() == {"uni_run": 8, "uni_waves": 4, "vec_rows": 128, "vcycle_rows": 16, "tail_fused": 1}


@pytest.mark.parametrize("case", [("sphere", 2, 16, 4), ("sphere", 1, 8, 3), ("sphere", 3, 4, 3), ("sphere", 2, 4, 3)])
def test_fused_coarse_tail_matches_per_level_launches(wm, case):
    # the coarse end of the V-cycle in one kernel per tile (levels without a
    # stencil form and the coarse solve; on the 4 x 4 meshes the whole cycle)
    # does the per-level kernels' arithmetic in their order: the same z up to
    # float rounding, on a full and a ragged tile with a shift per system
    kind, p, n, levels = case
    hier = wm.Hierarchy(wm.Geometry(kind, p, n), levels)
    nv = 45
    sg = np.geomspace(0.05, 1e5, nv)
    r = torch.tensor(random_vectors(21, nv, hier.num_dofs(0)), device="cuda")
    for deg in (1, 3):
        hier.set_schedule(tail_fused=1)
        z1 = hier.vcycle(r, sg, precision="mixed", smoother_degree=deg).cpu().numpy()
        hier.set_schedule(tail_fused=0)
        z0 = hier.vcycle(r, sg, precision="mixed", smoother_degree=deg).cpu().numpy()
        hier.set_schedule()
        assert np.isfinite(z1).all() and np.abs(z0).max() > 0
        np.testing.assert_allclose(z1, z0, rtol=0, atol=2e-6 * np.abs(z0).max())


def test_coarse_smoother_degree(wm):
    # another Chebyshev degree on the coarser levels changes the preconditioner,
    # not the fields beyond the solver tolerance
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 16), 4)
    kw = dict(kappa=3.0, beta=1.3, sinc_k=0.4, l_lo=-15, l_hi=15, n_samples=33, seed=4, precision="mixed",
              rtol=1e-10, smoother_degree=4)
    u0, _ = hier.sample_fields(**kw)
    for dc in (2, 6):
        u1, st = hier.sample_fields(smoother_degree_coarse=dc, **kw)
        assert st["n_not_converged"] == 0
        d = u1 - u0
        assert float(torch.sqrt((d * hier.apply_mass(d)).sum() / (u0 * hier.apply_mass(u0)).sum())) < 1e-8
