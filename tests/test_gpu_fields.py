"""GPU parity of the fields u_s (the whole path) against the CPU oracle."""
import numpy as np
import pytest
import torch

from oracle import geometry as geo
from oracle.assembly import assemble
from oracle.fractional import sample_fields as oracle_fields
from oracle.noise import noise_loads
from oracle.space import GluedSpace
from wm_workloads import WORKLOADS

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


def run_case(wm, kind, p, nu, nv, levels, kappa, beta, k, lo, hi, ns, seed, precision, rtol, split="standard",
             samples=None, **extra):
    hier = wm.Hierarchy(wm.Geometry(kind, p, nu, nv), levels)
    u, b, st = hier.sample_fields(return_loads=True, kappa=kappa, beta=beta, sinc_k=k, l_lo=lo, l_hi=hi,
                                  n_samples=ns, seed=seed, split=split, precision=precision, rtol=rtol, **extra)
    s = geo.Surface(kind, p, nu, nv)
    sp_ = GluedSpace(s)
    S, M = assemble(sp_)
    idx = np.arange(ns) if samples is None else np.asarray(samples)
    b_or = noise_loads(sp_, seed, ns)[idx] if samples is None else None
    if b_or is None:
        from oracle.noise import noise_from_xi, n_quad
        from oracle.philox import normals
        q = np.arange(n_quad(s))
        b_or = np.stack([noise_from_xi(sp_, normals(seed, int(si), q)) for si in idx])
    np.testing.assert_allclose(b.cpu().numpy()[idx], b_or, rtol=1e-11, atol=1e-13 * np.abs(b_or).max())
    u_or = oracle_fields(S, M, b_or, kappa, beta, k, lo, hi, split)
    return mnorm_rel(u.cpu().numpy()[idx], u_or, M), st, hier, u


def test_plain_fp64_sphere_p2_j3(wm):
    c = WORKLOADS["sphere_p2_j3_fp64"]
    err, st, *_ = run_case(wm, "sphere", 2, 8, 8, c["levels"], c["kappa"], c["beta"], c["k"], c["l_lo"], c["l_hi"],
                           c["n_samples"], c["seed"], "fp64", c["rtol"])
    assert err.max() < 1e-9, (err, st)
    assert st["n_not_converged"] == 0 and st["n_nodes"] == 51


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_sphere_batched_integer_plus_fraction(wm, precision, tol):
    # beta = 1.3: one integer solve then 71 nodes; 40 samples = ragged second tile
    err, st, *_ = run_case(wm, "sphere", 2, 16, 16, 4, 5.0, 1.3, 0.3, -35, 35, 40, 3, precision,
                           1e-11 if precision == "fp64" else 1e-8)
    assert err.max() < tol, (err, st)
    assert st["n_int_solves"] == 1 and st["n_systems"] == 40 + 71 * 40


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_torus_p3(wm, precision, tol):
    err, st, *_ = run_case(wm, "torus", 3, 32, 16, 2, 10.0, 0.6, 0.3, -35, 35, 33, 0, precision,
                           1e-11 if precision == "fp64" else 1e-8)
    assert err.max() < tol, (err, st)


def test_double_float_residual_and_its_fallback(wm):
    """Mixed precision evaluates the replacement residuals b - A x in
    double-float arithmetic; at rtol 1e-8 its error bound passes, at 1e-12
    it cannot, and the solve switches to float64 residuals and still
    converges to the float64 answer."""
    kw = dict(kappa=5.0, beta=0.7, sinc_k=0.3, l_lo=-35, l_hi=35, n_samples=40, seed=5)
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 16), 4)
    u8, st8 = hier.sample_fields(precision="mixed", rtol=1e-8, **kw)
    assert st8["n_replacements"] > 0 and st8["n_df_fallbacks"] == 0, st8
    u12, st12 = hier.sample_fields(precision="mixed", rtol=1e-12, **kw)
    assert st12["n_df_fallbacks"] >= 1 and st12["n_not_converged"] == 0, st12
    assert st12["max_rel_residual"] <= 1e-12
    ref, _ = hier.sample_fields(precision="fp64", rtol=1e-12, **kw)
    ref = ref.cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(u12.cpu().numpy() - ref).max() < 1e-9 * scale
    assert np.abs(u8.cpu().numpy() - ref).max() < 1e-5 * scale


@pytest.mark.parametrize("beta,split", [(0.7, "standard"), (1.8, "improved")])
def test_tolerance_driven_nodes_reach_the_fractional_power(wm, beta, split):
    """Node sets from wm_sinc_nodes: the float64 fields on a small sphere against
    the exact discrete fractional power from a dense generalised eigendecomposition
    (S v = lambda M v, u = V diag((lambda + kappa^2)^-beta) V^T b): the error in
    the M-norm stays below tol ||b||_{M^-1} (per pass), and the mixed path agrees
    with the oracle on the same nodes."""
    import scipy.linalg as sla
    kappa, tol, ns = 3.0, 1e-8, 3
    k, lo, hi = wm.sinc_nodes(beta, kappa, tol, split)
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 3)
    u, b, st = hier.sample_fields(return_loads=True, kappa=kappa, beta=beta, sinc_k=k, l_lo=lo, l_hi=hi,
                                  n_samples=ns, seed=9, split=split, precision="fp64", rtol=1e-12)
    assert st["n_nodes"] == hi - lo + 1
    sp_ = GluedSpace(geo.Surface("sphere", 2, 8))
    S, M = assemble(sp_)
    lam, V = sla.eigh(S.toarray(), M.toarray())  # V^T M V = I
    bn = b.cpu().numpy()
    u_ex = (V @ (((lam + kappa ** 2) ** -beta)[:, None] * (V.T @ bn.T))).T
    d = u.cpu().numpy() - u_ex
    err = np.sqrt(np.einsum("si,si->s", d, (M @ d.T).T))
    bnorm = np.sqrt(np.einsum("si,si->s", bn, sla.solve(M.toarray(), bn.T).T))
    passes = st["n_frac_passes"]
    assert (err <= passes * tol * bnorm).all(), (err / bnorm)
    um, stm = hier.sample_fields(kappa=kappa, beta=beta, sinc_k=k, l_lo=lo, l_hi=hi, n_samples=ns, seed=9,
                                 split=split, precision="mixed", rtol=1e-8)
    u_or = oracle_fields(S, M, bn, kappa, beta, k, lo, hi, split)
    assert mnorm_rel(um.cpu().numpy(), u_or, M).max() < 1e-6


@pytest.mark.parametrize("kind,p,nu,nv,levels,precision,tol", [
    ("sphere", 2, 16, 16, 4, "mixed", 1e-6), ("torus", 3, 32, 16, 2, "fp64", 1e-9)])
def test_bpx_preconditioner(wm, kind, p, nu, nv, levels, precision, tol):
    """The additive BPX preconditioner (multilevel diagonal scaling, Sec. 3.5) in
    place of the V-cycle: same fields as the oracle, more (cheaper) iterations."""
    rtol = 1e-8 if precision == "mixed" else 1e-11
    err, st, hier, u = run_case(wm, kind, p, nu, nv, levels, 5.0, 1.3, 0.3, -35, 35, 40, 3, precision, rtol,
                                preconditioner="bpx", max_iter=2000)
    assert st["n_not_converged"] == 0
    assert err.max() < tol, (err, st)
    _, st_v = hier.sample_fields(kappa=5.0, beta=1.3, sinc_k=0.3, l_lo=-35, l_hi=35, n_samples=40, seed=3,
                                 precision=precision, rtol=rtol)
    assert st["max_iterations"] > st_v["max_iterations"]


def test_improved_split_two_passes(wm):
    err, st, *_ = run_case(wm, "sphere", 2, 8, 8, 3, 3.0, 1.8, 0.4, -20, 20, 5, 4, "mixed", 1e-9, split="improved")
    assert st["n_frac_passes"] == 2 and st["n_int_solves"] == 1
    assert err.max() < 1e-6, err


def test_integer_beta_only(wm):
    err, st, *_ = run_case(wm, "sphere", 3, 4, 4, 2, 1.5, 2.0, 0.4, -5, 5, 3, 1, "fp64", 1e-12)
    assert st["n_frac_passes"] == 0 and st["n_int_solves"] == 2
    assert err.max() < 1e-9, err


def test_system_batching_and_host_output(wm):
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 3)
    kw = dict(kappa=2.0, beta=0.75, sinc_k=0.4, l_lo=-25, l_hi=25, n_samples=7, seed=2, precision="mixed",
              rtol=1e-9)
    u1, _ = hier.sample_fields(**kw)
    u2, st = hier.sample_fields(max_systems=64, **kw)
    assert st["n_batches"] == (51 * 7 + 63) // 64
    np.testing.assert_allclose(u2.cpu().numpy(), u1.cpu().numpy(), rtol=1e-8, atol=1e-12)
    host = torch.empty(u1.shape, dtype=torch.float64).pin_memory()
    u3, _ = hier.sample_fields(out=host, **kw)
    assert np.array_equal(u3.numpy(), u1.cpu().numpy())
    # no samples: nothing to do
    u0, st0 = hier.sample_fields(**dict(kw, n_samples=0))
    assert u0.shape[0] == 0


def test_invalid_arguments(wm):
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 3)
    with pytest.raises(wm.WMError):
        hier.sample_fields(kappa=-1.0, beta=0.7, n_samples=1)
    with pytest.raises(wm.WMError):
        hier.sample_fields(kappa=1.0, beta=0.7, n_samples=1, l_lo=3, l_hi=2)
    with pytest.raises(wm.WMError):
        wm.Hierarchy(wm.Geometry("sphere", 2, 8), 9)


def test_full_size_bench_workload_sampled(wm):
    """The bench workload (sphere 6x64x64, p=2, beta=1.3, 256 samples, mixed) at
    full size in the bench's launch configuration; the oracle checks samples 0 and 255."""
    c = WORKLOADS["sphere_p2_j6_mixed_s256"]
    err, st, *_ = run_case(wm, "sphere", 2, 64, 64, c["levels"], c["kappa"], c["beta"], c["k"], c["l_lo"],
                           c["l_hi"], c["n_samples"], c["seed"], "mixed", c["rtol"], samples=[0, 255])
    assert err.max() < 1e-6, (err, st)
    assert st["n_systems"] == 256 * 72 and st["n_not_converged"] == 0


def test_failure_reporting_not_converged_and_nonfinite(wm):
    """Host-side fault injection: an iteration cap of 1 must report
    NOT_CONVERGED (fields still written), NaN-poisoned loads NONFINITE."""
    from paper_2605_24882_gb300 import _capi
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 3)
    kw = dict(kappa=2.0, beta=0.75, sinc_k=0.4, l_lo=-5, l_hi=5, n_samples=3, seed=1, precision="mixed")
    with pytest.raises(wm.WMError) as e:
        hier.sample_fields(max_iter=1, **kw)
    assert e.value.code == _capi.WM_ERR_NOT_CONVERGED
    u, st = hier.sample_fields(max_iter=1, check_convergence=False, **kw)
    assert st["n_not_converged"] > 0 and torch.isfinite(u).all()
    b = hier.noise_loads(1, 3)
    b[1, 7] = float("nan")
    with pytest.raises(wm.WMError) as e:
        hier.sample_fields(b=b, **kw)
    assert e.value.code == _capi.WM_ERR_NONFINITE


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sample_range_split_reproduces_the_whole_run(wm, precision):
    # A replica job splits one sample range: the rank holding samples n .. 2n - 1
    # calls with sample0 = n.  Its loads must be rows n .. 2n - 1 of a 2n-sample
    # run bit for bit (and the oracle's loads of those samples), its fields the same.
    from oracle.noise import noise_loads
    n = 32
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 16), 4)
    kw = dict(kappa=3.0, beta=1.3, sinc_k=0.4, l_lo=-20, l_hi=20, seed=9, precision=precision, rtol=1e-10)
    u2, b2, st2 = hier.sample_fields(return_loads=True, n_samples=2 * n, **kw)
    u1, b1, st1 = hier.sample_fields(return_loads=True, n_samples=n, sample0=n, **kw)
    assert torch.equal(b1, b2[n:])
    sp_ = GluedSpace(geo.Surface("sphere", 2, 16))
    b_or = noise_loads(sp_, 9, 2 * n)[n:]
    np.testing.assert_allclose(b1.cpu().numpy(), b_or, rtol=1e-11, atol=1e-13 * np.abs(b_or).max())
    torch.testing.assert_close(u1, u2[n:], rtol=1e-12, atol=1e-14 * float(u2.abs().max()))
