"""Fields on NURBS surfaces (Sec. 2.2 geometries) on the GPU against the oracle.

The library evaluates the NURBS maps on the host and uploads the metric; the
oracle evaluates them with its own bases.  Everything after the metric (element
matrices, noise loads, the batched solves) is the sampler's usual path.
"""
import numpy as np
import pytest
import torch

import paper_2605_24882_gb300 as wm
import wm_workloads as wl
from oracle.assembly import assemble
from oracle.fractional import sample_fields as oracle_fields
from oracle.noise import noise_loads
from oracle.nurbs import NurbsSurface
from oracle.space import GluedSpace

pytestmark = pytest.mark.gpu

CASES = [("periodic", 2, 32, 16, 2), ("cube", 2, 8, 8, 3)]


def _patches(topo):
    return wl.nurbs_torus(1.0, 0.4) if topo == "periodic" else wl.nurbs_bulged_cube(0.3, 2.0)


@pytest.mark.parametrize("topo,p,nu,nv,levels", CASES)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_nurbs_fields_match_oracle(topo, p, nu, nv, levels, precision, tol):
    patches = _patches(topo)
    sp_ = GluedSpace(NurbsSurface(topo, patches, p, nu, nv))
    S, M = assemble(sp_)
    b_or = noise_loads(sp_, 9, 4)
    u_or = oracle_fields(S, M, b_or, 3.0, 1.3, 0.4, -25, 25)
    g = wm.Geometry.nurbs(topo, patches, p, nu, nv)
    hier = wm.Hierarchy(g, levels)
    np.testing.assert_array_equal(hier.metric(0).cpu().numpy(), g.metric_host(0))
    u, b, st = hier.sample_fields(return_loads=True, kappa=3.0, beta=1.3, sinc_k=0.4, l_lo=-25, l_hi=25,
                                  n_samples=4, seed=9, precision=precision,
                                  rtol=1e-11 if precision == "fp64" else 1e-9)
    torch.cuda.synchronize()
    np.testing.assert_allclose(b.cpu().numpy(), b_or, rtol=1e-11, atol=1e-14)
    d = u.cpu().numpy() - u_or
    err = np.sqrt(np.einsum("si,si->s", d, (M @ d.T).T) / np.einsum("si,si->s", u_or, (M @ u_or.T).T))
    assert err.max() < tol, (err, st)
