"""sqrt(M) white-noise loads on the GPU against the oracle (Sec. 3.3, Eq. eq:sqrt).

Both sides draw y_s from Philox stream 2 (DOF index, sample s) by their own
implementations and apply the same n-node rule on the oracle's spectrum bounds.
"""
import json

import numpy as np
import pytest
import torch

import paper_2605_24882_gb300 as wm
from oracle import geometry as geo
from oracle import sqrt_mass as sq
from oracle.assembly import assemble
from oracle.philox import normals
from oracle.space import GluedSpace

pytestmark = pytest.mark.gpu


def _oracle(kind, p, nu, nv, seed, samples, n_nodes):
    sp_ = GluedSpace(geo.Surface(kind, p, nu, None if kind == "sphere" else nv))
    _, M = assemble(sp_)
    lo, hi = sq.mass_spectrum_bounds(sp_)
    Y = np.stack([normals(seed, s, np.arange(sp_.N), 2) for s in samples])
    return lo, hi, sq.noise_loads_sqrt(M, lo, hi, n_nodes, Y)


def _rel(f, f_or):
    return np.linalg.norm(f - f_or, axis=1) / np.linalg.norm(f_or, axis=1)


@pytest.mark.parametrize("kind,p,nu,nv,ns", [("sphere", 2, 4, 4, 37), ("torus", 3, 16, 8, 5),
                                              ("sphere", 3, 2, 2, 64), ("sphere", 1, 8, 8, 1)])
def test_sqrt_noise_matches_oracle(kind, p, nu, nv, ns):
    n_nodes = 40
    lo, hi, f_or = _oracle(kind, p, nu, nv, 11, range(ns), n_nodes)
    hier = wm.Hierarchy(wm.Geometry(kind, p, nu, nv), 1)
    f, it = hier.noise_loads_sqrt(11, ns, lo, hi, n_nodes, rtol=1e-13)
    torch.cuda.synchronize()
    err = _rel(f.cpu().numpy(), f_or)
    assert err.max() < 1e-11, (err.max(), it)
    assert 0 < it < 1000


def test_sqrt_noise_full_size_sampled():
    # sphere 6 x 64 x 64, p = 2 (25,352 DOFs), 40 samples in two tiles; the
    # oracle computes samples 0 and 39 by direct solves
    n_nodes = 32
    lo, hi, f_or = _oracle("sphere", 2, 64, 64, 3, [0, 39], n_nodes)
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 64), 1)
    f, it = hier.noise_loads_sqrt(3, 40, lo, hi, n_nodes, rtol=1e-12)
    torch.cuda.synchronize()
    err = _rel(f[[0, 39]].cpu().numpy(), f_or)
    assert err.max() < 1e-10, (err.max(), it)


def test_sqrt_noise_throughput():
    # 256 samples on the 25,352-DOF sphere with the library's own spectrum
    # bounds; the time is reported (CUDA events around one call)
    g = wm.Geometry("sphere", 2, 64)
    hier = wm.Hierarchy(g, 1)
    lo, hi = g.mass_bounds(0)
    n_nodes = 20
    hier.noise_loads_sqrt(5, 32, lo, hi, n_nodes, rtol=1e-10)   # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    f, it = hier.noise_loads_sqrt(5, 256, lo, hi, n_nodes, rtol=1e-10)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"sqrt_noise": {"samples": 256, "dofs": hier.num_dofs(0), "nodes": n_nodes,
                                     "iterations": it, "ms": ms, "samples_per_s": 256e3 / ms,
                                     "bounds": [lo, hi]}}))
    assert bool(torch.isfinite(f).all()) and 0 < it < 1000


def test_sqrt_noise_errors():
    g = wm.Geometry("sphere", 2, 2)
    hier = wm.Hierarchy(g, 1)
    lo, hi = g.mass_bounds(0)
    f, it = hier.noise_loads_sqrt(1, 0, lo, hi, 8)
    assert f.shape[0] == 0 and it == 0
    for args in [(1, 3, lo, hi, 0), (1, 3, hi, lo, 8), (1, 3, 0.0, hi, 8)]:
        with pytest.raises(wm.WMError) as e:
            hier.noise_loads_sqrt(*args)
        assert e.value.code == wm._capi.WM_ERR_INVALID_ARG
    with pytest.raises(wm.WMError) as e:
        hier.noise_loads_sqrt(1, 3, lo, hi, 8, rtol=1e-14, max_iter=1)
    assert e.value.code == wm._capi.WM_ERR_NOT_CONVERGED


def test_fields_from_sqrt_noise_match_oracle():
    # the paper's sampling chain with the square-root noise: f = sqrt(M) y
    # (Eq. eq:sqrt), then u = L^{-beta} M^{-1} f; the library's loads enter its
    # sampler as given loads, the oracle's loads enter the oracle's sampler
    from oracle.fractional import sample_fields as oracle_fields
    ns, n_nodes = 6, 32
    sp_ = GluedSpace(geo.Surface("sphere", 2, 8))
    S, M = assemble(sp_)
    lo, hi = sq.mass_spectrum_bounds(sp_)
    Y = np.stack([normals(13, s, np.arange(sp_.N), 2) for s in range(ns)])
    f_or = sq.noise_loads_sqrt(M, lo, hi, n_nodes, Y)
    u_or = oracle_fields(S, M, f_or, 2.0, 1.3, 0.4, -25, 25)
    hier = wm.Hierarchy(wm.Geometry("sphere", 2, 8), 3)
    f, _ = hier.noise_loads_sqrt(13, ns, lo, hi, n_nodes, rtol=1e-12)
    u, st = hier.sample_fields(b=f, kappa=2.0, beta=1.3, sinc_k=0.4, l_lo=-25, l_hi=25, n_samples=ns,
                               precision="mixed", rtol=1e-10)
    torch.cuda.synchronize()
    d = u.cpu().numpy() - u_or
    err = np.sqrt(np.einsum("si,si->s", d, (M @ d.T).T) / np.einsum("si,si->s", u_or, (M @ u_or.T).T))
    assert err.max() < 1e-6, (err, st)
