"""GPU checks of the multi-instance entry point and of the torus at full size.

* wm_sample_fields_batched on a seeded uneven batch (spheres p = 2 and tori
  p = 3 at refinement levels 3-4, kappa ~ U[1, 20], beta ~ U[0.55, 1.95], the
  improved split, 1..64 samples): every instance against the CPU oracle.
* The periodic bicubic torus 512 x 256 (131,072 DOFs) at full size: the
  problem is invariant under a rotation about the torus axis by one element,
  so shifting the loads by one DOF column along u must shift the fields the
  same way (to the solver tolerance); the mixed fields must agree with the
  float64 path; and on a two-node set (two sparse LU factorisations of the
  oracle) both precisions must match the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import geometry as geo
from oracle.assembly import assemble
from oracle.fractional import sample_fields as oracle_fields
from oracle.noise import noise_loads
from oracle.space import GluedSpace
from wm_workloads import WORKLOADS, uneven_instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wm():
    from paper_2605_24882_gb300 import build as b
    b.build()
    import paper_2605_24882_gb300 as wm
    return wm


def mnorm_rel(u, ref, M):
    d = u - ref
    num = np.einsum("si,si->s", d, (M @ d.T).T)
    den = np.einsum("si,si->s", ref, (M @ ref.T).T)
    return np.sqrt(num / den)


def test_uneven_instances_batched_against_oracle(wm):
    insts = uneven_instances(seed=11, n_inst=6, j_lo=3, j_hi=4)
    hiers, descs = [], []
    for c in insts:
        g = wm.Geometry(c["kind"], c["p"], c["n_u"], c["n_v"], c.get("R", 1.0), c.get("r", 0.4))
        hiers.append(wm.Hierarchy(g, c["levels"]))
        descs.append(wm.Hierarchy.make_desc(c["kappa"], c["beta"], c["k"], c["l_lo"], c["l_hi"], c["n_samples"],
                                            c["seed"], c["split"], c["precision"], c["rtol"]))
    outs, stats = wm.sample_fields_batched(hiers, descs)
    assert len(outs) == len(insts)
    for c, u, st in zip(insts, outs, stats):
        s = geo.Surface(c["kind"], c["p"], c["n_u"], c["n_v"], c.get("R", 1.0), c.get("r", 0.4))
        sp_ = GluedSpace(s)
        S, M = assemble(sp_)
        b = noise_loads(sp_, c["seed"], c["n_samples"])
        ref = oracle_fields(S, M, b, c["kappa"], c["beta"], c["k"], c["l_lo"], c["l_hi"], c["split"])
        err = mnorm_rel(u.cpu().numpy(), ref, M)
        assert st["n_not_converged"] == 0, (c, st)
        assert err.max() < 1e-6, (c["kind"], c["n_u"], c["beta"], err.max())
    # the same instance alone gives the same fields as inside the batch
    u1, _ = hiers[0].sample_fields(kappa=insts[0]["kappa"], beta=insts[0]["beta"], sinc_k=insts[0]["k"],
                                   l_lo=insts[0]["l_lo"], l_hi=insts[0]["l_hi"], n_samples=insts[0]["n_samples"],
                                   seed=insts[0]["seed"], split=insts[0]["split"], precision="mixed", rtol=1e-8)
    np.testing.assert_allclose(u1.cpu().numpy(), outs[0].cpu().numpy(), rtol=0, atol=1e-12 * float(u1.abs().max()))


def test_torus_full_size_rotation_and_fp64(wm):
    n_u, n_v, ns = 512, 256, 4
    hier = wm.Hierarchy(wm.Geometry("torus", 3, n_u, n_v, 1.0, 0.4), 6)
    N = hier.num_dofs(0)
    assert N == n_u * n_v
    kw = dict(kappa=10.0, beta=0.6, sinc_k=0.3, l_lo=-35, l_hi=35, n_samples=ns, seed=0, precision="mixed", rtol=1e-8)
    u, b, st = hier.sample_fields(return_loads=True, **kw)
    assert st["n_not_converged"] == 0 and st["n_systems"] == 71 * ns
    # DOFs are numbered row by row (v outer, u inner): roll every row by one along u
    b_rot = torch.roll(b.view(ns, n_v, n_u), shifts=1, dims=2).reshape(ns, N).contiguous()
    u_rot, _ = hier.sample_fields(b=b_rot, **kw)
    u_exp = torch.roll(u.view(ns, n_v, n_u), shifts=1, dims=2).reshape(ns, N)

    def rel(a, ref):
        d = a - ref
        return torch.sqrt((d * hier.apply_mass(d)).sum(1) / (ref * hier.apply_mass(ref)).sum(1))

    assert float(rel(u_rot, u_exp).max()) < 1e-6
    u64, st64 = hier.sample_fields(b=b, **dict(kw, precision="fp64"))
    assert st64["n_not_converged"] == 0
    assert float(rel(u, u64).max()) < 1e-6


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-6), ("fp64", 1e-9)])
def test_torus_full_size_against_the_oracle(wm, precision, tol):
    # the 512 x 256 bicubic torus of the torus workload, through its whole
    # hierarchy and kernel configuration, against the oracle's direct solves on
    # a two-node set (one sparse LU per shift) and two samples
    c = WORKLOADS["torus_p3_512x256_s1024"]
    kw = dict(kappa=c["kappa"], beta=c["beta"], sinc_k=c["k"], l_lo=-1, l_hi=0, n_samples=2, seed=c["seed"],
              precision=precision, rtol=1e-10 if precision == "mixed" else 1e-12,
              smoother_degree=c["smoother_degree"], cheb_ratio=c["cheb_ratio"])
    hier = wm.Hierarchy(wm.Geometry("torus", 3, c["n_u"], c["n_v"], c["R"], c["r"]), c["levels"])
    u, b, st = hier.sample_fields(return_loads=True, **kw)
    assert st["n_not_converged"] == 0 and st["n_systems"] == 2 * 2
    sp_ = GluedSpace(geo.Surface("torus", 3, c["n_u"], c["n_v"], c["R"], c["r"]))
    S, M = assemble(sp_)
    b_or = noise_loads(sp_, c["seed"], 2)
    np.testing.assert_allclose(b.cpu().numpy(), b_or, rtol=1e-11, atol=1e-13 * np.abs(b_or).max())
    u_or = oracle_fields(S, M, b_or, c["kappa"], c["beta"], c["k"], -1, 0)
    d = u.cpu().numpy() - u_or
    err = np.sqrt(np.einsum("si,si->s", d, (M @ d.T).T) / np.einsum("si,si->s", u_or, (M @ u_or.T).T))
    assert err.max() < tol, (err, st)


def test_instances_sharing_a_hierarchy_share_the_solves(wm):
    # five instances on one hierarchy (kappa, beta under both splits, 1..40
    # samples, seeds, first samples all different) are solved stage by stage in
    # the same batched solves; each must match the oracle and its own run
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 3)
    sp_ = GluedSpace(geo.Surface("sphere", 2, 8))
    S, M = assemble(sp_)
    cases = [(2.0, 0.75, "standard", 3, 1, 0), (5.0, 1.3, "standard", 40, 2, 7), (1.5, 1.5, "improved", 17, 3, 0),
             (8.0, 0.9, "improved", 1, 4, 5), (3.0, 2.0, "standard", 33, 5, 0)]
    descs = [wm.Hierarchy.make_desc(kap, beta, 0.4, -20, 20, ns, seed, split, "mixed", 1e-9, sample0=s0)
             for kap, beta, split, ns, seed, s0 in cases]
    outs, stats = wm.sample_fields_batched([hier] * len(cases), descs)
    for (kap, beta, split, ns, seed, s0), u, st in zip(cases, outs, stats):
        n_int, _, passes = wm.beta_plan(beta, split)
        assert st["n_not_converged"] == 0 and st["n_systems"] == ns * (n_int + passes * 41), st
        b = noise_loads(sp_, seed, s0 + ns)[s0:]
        ref = oracle_fields(S, M, b, kap, beta, 0.4, -20, 20, split)
        assert mnorm_rel(u.cpu().numpy(), ref, M).max() < 1e-6, (kap, beta, split)
        alone, _ = hier.sample_fields(kappa=kap, beta=beta, sinc_k=0.4, l_lo=-20, l_hi=20, n_samples=ns, seed=seed,
                                      split=split, precision="mixed", rtol=1e-9, sample0=s0)
        assert mnorm_rel(u.cpu().numpy(), alone.cpu().numpy(), M).max() < 1e-7


def test_uneven_batch_96_instances(wm):
    # the uneven configuration: 96 spheres (p = 2) and tori (p = 3) at levels
    # 3..9 (488 .. 1,579,016 DOFs), kappa ~ U[1, 20], beta ~ U[0.55, 1.95] with
    # the improved split, 1..64 samples, seed 11; one hierarchy per distinct
    # surface, so the instances of a surface share their batched solves.
    # Checks: instances up to 6,536 DOFs against the oracle; for every larger
    # one, its first and last samples against the float64 path run alone.
    import collections
    insts = uneven_instances()
    hiers = {}
    H, D = [], []
    for c in insts:
        key = (c["kind"], c["n_u"], c["n_v"])
        if key not in hiers:
            g = wm.Geometry(c["kind"], c["p"], c["n_u"], c["n_v"], c.get("R", 1.0), c.get("r", 0.4))
            hiers[key] = wm.Hierarchy(g, c["levels"])
        H.append(hiers[key])
        D.append(wm.Hierarchy.make_desc(c["kappa"], c["beta"], c["k"], c["l_lo"], c["l_hi"], c["n_samples"],
                                        c["seed"], c["split"], c["precision"], c["rtol"]))
    assert len(hiers) == 14
    outs, stats = wm.sample_fields_batched(H, D)
    assert all(st["n_not_converged"] == 0 for st in stats)
    oracle_cache = collections.OrderedDict()
    for c, h, u, st in zip(insts, H, outs, stats):
        N = h.num_dofs(0)
        assert u.shape == (c["n_samples"], N)
        if N <= 6536:
            key = (c["kind"], c["n_u"])
            if key not in oracle_cache:
                sp_ = GluedSpace(geo.Surface(c["kind"], c["p"], c["n_u"], c["n_v"], c.get("R", 1.0), c.get("r", 0.4)))
                oracle_cache[key] = (sp_,) + tuple(assemble(sp_))
            sp_, S, M = oracle_cache[key]
            b = noise_loads(sp_, c["seed"], c["n_samples"])
            ref = oracle_fields(S, M, b, c["kappa"], c["beta"], c["k"], c["l_lo"], c["l_hi"], c["split"])
            assert mnorm_rel(u.cpu().numpy(), ref, M).max() < 1e-6, (c["kind"], c["n_u"], c["beta"])
        else:
            for s0 in sorted({0, c["n_samples"] - 1}):
                u64, st64 = h.sample_fields(kappa=c["kappa"], beta=c["beta"], sinc_k=c["k"], l_lo=c["l_lo"],
                                            l_hi=c["l_hi"], n_samples=1, seed=c["seed"], split=c["split"],
                                            precision="fp64", rtol=1e-10, sample0=s0)
                d = u[s0:s0 + 1] - u64
                rel = torch.sqrt((d * h.apply_mass(d)).sum() / (u64 * h.apply_mass(u64)).sum())
                assert float(rel) < 1e-6, (c["kind"], c["n_u"], c["beta"], s0, float(rel))
