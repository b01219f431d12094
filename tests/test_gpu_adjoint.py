"""GPU adjoint (wm_sample_fields_backward) against the oracle's adjoint
gradient and central finite differences (float64)."""
import numpy as np
import pytest
import torch

from oracle import geometry as geo
from oracle.assembly import assemble
from oracle.fractional import field_loss_grad
from oracle.noise import noise_loads, target_fields
from oracle.space import GluedSpace
from wm_workloads import WORKLOADS, random_vectors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wm():
    from paper_2605_24882_gb300 import build as b
    b.build()
    import paper_2605_24882_gb300 as wm
    return wm


def gpu_loss(hier, b, g, **kw):
    u, _ = hier.sample_fields(b=b, **kw)
    d = u - g
    return float((d * hier.apply_mass(d)).sum()), u


@pytest.mark.parametrize("beta,split", [(0.8, "standard"), (1.3, "standard"), (2.0, "standard"),
                                        (0.9, "improved"), (1.5, "improved"), (1.9, "improved")])
def test_adjoint_matches_oracle_and_fd(wm, beta, split):
    # one fractional pass (0.8, 1.3), integer beta (2.0), and the improved
    # split's two passes with 0, 0 and 1 integer solves (0.9, 1.5, 1.9)
    kind, p, n = "sphere", 3, 4
    hier = wm.Hierarchy(wm.Geometry(kind, p, n), 2)
    sp_ = GluedSpace(geo.Surface(kind, p, n))
    S, M = assemble(sp_)
    ns, kappa, k, lo, hi = 3, 1.7, 0.5, -12, 12
    b_or = noise_loads(sp_, 4, ns)
    g_or = target_fields(sp_, 7, ns)
    L_or, dLdb_or, dLdk_or = field_loss_grad(S, M, b_or, g_or, kappa, beta, k, lo, hi, split)
    kw = dict(beta=beta, split=split, sinc_k=k, l_lo=lo, l_hi=hi, n_samples=ns, precision="fp64", rtol=1e-13,
              max_iter=400)
    b = torch.tensor(b_or, device="cuda")
    g = torch.tensor(g_or, device="cuda")
    L, u = gpu_loss(hier, b, g, kappa=kappa, **kw)
    assert L == pytest.approx(L_or, rel=1e-10)
    grad_u = 2.0 * hier.apply_mass(u - g)
    gb, gk = hier.sample_fields_backward(b, grad_u, kappa=kappa, **kw)
    np.testing.assert_allclose(gb.cpu().numpy(), dLdb_or, rtol=1e-8, atol=1e-10 * np.abs(dLdb_or).max())
    assert gk == pytest.approx(dLdk_or, rel=1e-8)
    # central finite differences on the GPU forward (float64)
    h = 1e-6
    Lp, _ = gpu_loss(hier, b, g, kappa=kappa + h, **kw)
    Lm, _ = gpu_loss(hier, b, g, kappa=kappa - h, **kw)
    assert gk == pytest.approx((Lp - Lm) / (2 * h), rel=1e-5)


@pytest.mark.parametrize("beta,split", [(1.3, "standard"), (1.9, "improved")])
def test_checkpointed_backward(wm, beta, split):
    # a forward call with ckpt="keep" leaves every per-node solution in the
    # workspace; the backward with the same descriptor and loads then solves the
    # adjoint systems only and gives the gradients of the recomputing backward
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 3)
    ns, kappa = 5, 2.0
    kw = dict(beta=beta, split=split, sinc_k=0.4, l_lo=-12, l_hi=12, n_samples=ns, precision="fp64", rtol=1e-12)
    b = hier.noise_loads(3, ns)
    g = torch.tensor(random_vectors(8, ns, hier.num_dofs(0)), device="cuda")
    u, st = hier.sample_fields(b=b, kappa=kappa, ckpt="keep", **kw)
    assert st["ckpt_kept"] == 1
    grad_u = 2.0 * hier.apply_mass(u - g)
    gb1, gk1, s1 = hier.sample_fields_backward(b, grad_u, kappa=kappa, ckpt="keep", return_stats=True, **kw)
    gb0, gk0, s0 = hier.sample_fields_backward(b, grad_u, kappa=kappa, return_stats=True, **kw)
    assert s1["ckpt_used"] == 1 and s0["ckpt_used"] == 0
    assert s1["n_systems"] < s0["n_systems"]  # no forward solves
    torch.testing.assert_close(gb1, gb0, rtol=1e-12, atol=1e-14 * float(gb0.abs().max()))
    assert gk1 == pytest.approx(gk0, rel=1e-12)
    # other loads or another kappa: the checkpoint does not match and is not used
    b2 = b.clone()
    b2[0, 0] += 1e-3
    _, _, s2 = hier.sample_fields_backward(b2, grad_u, kappa=kappa, ckpt="keep", return_stats=True, **kw)
    _, _, s3 = hier.sample_fields_backward(b, grad_u, kappa=kappa + 0.1, ckpt="keep", return_stats=True, **kw)
    assert s2["ckpt_used"] == 0 and s3["ckpt_used"] == 0


def test_autograd_function(wm):
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 3)
    kw = dict(beta=0.75, sinc_k=0.4, l_lo=-10, l_hi=10, n_samples=4, precision="fp64", rtol=1e-12)
    b = hier.noise_loads(2, 4).requires_grad_(True)
    kappa = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    w = torch.tensor(random_vectors(3, 4, hier.num_dofs(0)), device="cuda")
    u = wm.WMField.apply(b, kappa, hier, kw)
    (u * w).sum().backward()
    gb, gk = hier.sample_fields_backward(b.detach(), w, kappa=2.0, **kw)
    torch.testing.assert_close(b.grad, gb, rtol=1e-12, atol=1e-14)
    assert kappa.grad.item() == pytest.approx(gk, rel=1e-12)


def test_adjoint_workload_full_size_fd(wm):
    """Sphere 6 x 128 x 128, p = 3 (101,402 DOFs), kappa = 4, beta = 0.8, 64
    samples, target fields from seed 7: dL/dkappa against central finite
    differences (delta = 1e-6) and dL/db against a directional difference."""
    c = WORKLOADS["sphere_p3_j7_adjoint_s64"]
    hier = wm.Hierarchy(wm.Geometry(c["kind"], c["p"], c["n_u"]), c["levels"])
    ns = c["n_samples"]
    N = hier.num_dofs(0)
    assert N == 101402
    kw = dict(beta=c["beta"], sinc_k=c["k"], l_lo=c["l_lo"], l_hi=c["l_hi"], n_samples=ns, precision="fp64",
              rtol=1e-13, max_iter=400)
    b = hier.noise_loads(c["seed"], ns)
    g = torch.stack([wm.normals(c["target_seed"], s, 1, 0, N) for s in range(ns)])
    kappa = c["kappa"]
    L, u = gpu_loss(hier, b, g, kappa=kappa, **kw)
    grad_u = 2.0 * hier.apply_mass(u - g)
    gb, gk = hier.sample_fields_backward(b, grad_u, kappa=kappa, **kw)
    h = 1e-6
    Lp, _ = gpu_loss(hier, b, g, kappa=kappa + h, **kw)
    Lm, _ = gpu_loss(hier, b, g, kappa=kappa - h, **kw)
    assert gk == pytest.approx((Lp - Lm) / (2 * h), rel=1e-5)
    d = torch.tensor(random_vectors(5, ns, N), device="cuda")
    eps = 1e-3 * float(b.abs().max())
    Lp, _ = gpu_loss(hier, b + eps * d, g, kappa=kappa, **kw)
    Lm, _ = gpu_loss(hier, b - eps * d, g, kappa=kappa, **kw)
    assert float((gb * d).sum()) == pytest.approx((Lp - Lm) / (2 * eps), rel=1e-5)
