"""CPU checks of the C ABI library: it loads, exports every declared symbol,
and its host-only entry points behave (no GPU call is made here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_24882_gb300 import build as b
    b.build()
    from paper_2605_24882_gb300 import _capi
    return _capi.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "wmfield.h")).read()
    return sorted(set(re.findall(r"^(?:int|void|const char\*)\s+(wm_[a-z0-9_]+)\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["wm_setup_geometry", "wm_assemble_hierarchy", "wm_sample_fields",
                     "wm_sample_fields_backward", "wm_sample_fields_batched", "wm_apply_mass",
                     "wm_num_dofs", "wm_error_string", "wm_destroy_hier", "wm_destroy_geom"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_beta_plan_matches_oracle(lib):
    from oracle.fractional import split_beta
    import paper_2605_24882_gb300 as wm
    for beta in [0.3, 0.75, 1.0, 1.3, 1.8, 2.0, 2.25, 0.9, 1.2, 3.7]:
        for split in ["standard", "improved"]:
            n, bf, ps = wm.beta_plan(beta, split)
            n2, bf2, ps2 = split_beta(beta, split)
            assert (n, ps) == (n2, ps2) and bf == pytest.approx(bf2, abs=1e-15)
    with pytest.raises(wm.WMError):
        wm.beta_plan(-1.0)


def test_sinc_nodes_match_oracle(lib):
    """The library's tolerance-driven node sets (host-only call) equal the oracle's."""
    from oracle.fractional import auto_nodes, split_beta
    import paper_2605_24882_gb300 as wm
    from paper_2605_24882_gb300 import _capi
    for beta in [0.3, 0.6, 0.75, 1.3, 1.1, 1.9]:
        for split in ["standard", "improved"]:
            for kappa in [0.5, 5.0, 20.0]:
                for tol in [1e-4, 1e-8]:
                    k, lo, hi = wm.sinc_nodes(beta, kappa, tol, split)
                    _, g, _ = split_beta(beta, split)
                    k2, lo2, hi2 = auto_nodes(g, kappa, tol)
                    assert (lo, hi) == (lo2, hi2) and k == pytest.approx(k2, rel=1e-14)
    with pytest.raises(wm.WMError) as e:
        wm.sinc_nodes(2.0, 5.0, 1e-8)
    assert e.value.code == _capi.WM_ERR_UNSUPPORTED
    for args in [(0.5, 0.0, 1e-8), (0.5, 5.0, 0.0), (0.5, 5.0, 2.0), (-1.0, 5.0, 1e-8)]:
        with pytest.raises(wm.WMError):
            wm.sinc_nodes(*args)


def test_geometry_validation(lib):
    import paper_2605_24882_gb300 as wm
    from paper_2605_24882_gb300 import _capi
    wm.Geometry("sphere", 2, 8)
    wm.Geometry("torus", 3, 32, 16)
    for args in [("sphere", 0, 8), ("sphere", 5, 8), ("sphere", 2, 6), ("torus", 3, 8, 4)]:
        with pytest.raises(wm.WMError) as e:
            wm.Geometry(*args)
        assert e.value.code == _capi.WM_ERR_INVALID_ARG
    assert lib.wm_error_string(-4).decode() == "not converged"
    assert lib.wm_num_dofs(None, 0) == _capi.WM_ERR_INVALID_ARG


def _oracle_space(kind, p, nu, nv, level):
    from oracle import geometry as geo
    from oracle.space import GluedSpace
    return GluedSpace(geo.Surface(kind, p, nu >> level, None if kind == "sphere" else nv >> level))


@pytest.mark.parametrize("kind,p,nu,nv", [("sphere", 1, 8, 8), ("sphere", 2, 8, 8), ("sphere", 3, 4, 4),
                                           ("sphere", 4, 2, 2), ("torus", 3, 32, 16), ("torus", 2, 16, 32)])
def test_host_dof_maps_match_oracle(lib, kind, p, nu, nv):
    # The library glues by matching integer lattice points of patch edges; the
    # oracle by matching the physical anchors of Greville points.  Both number
    # by the same scan rule, so the maps and connectivities agree bit for bit
    # at every level of the hierarchy.
    import numpy as np
    import paper_2605_24882_gb300 as wm
    g = wm.Geometry(kind, p, nu, nv)
    lowest = 1 if kind == "sphere" else 2 * p + 2
    level = 0
    while (min(nu, nv) >> level) >= lowest:
        sp_ = _oracle_space(kind, p, nu, nv, level)
        n, lu, lv, ne, _ = g.level_sizes(level, prolongation=False)
        l2g, conn = g.dof_map(level)
        assert (n, lu, lv) == (sp_.N, sp_.l2g.shape[2], sp_.l2g.shape[1])
        assert ne == sp_.surf.n_patches * sp_.surf.n_u * sp_.surf.n_v
        assert np.array_equal(l2g, sp_.l2g)
        assert np.array_equal(conn, sp_.connectivity().reshape(ne, -1))
        level += 1
    assert level >= 2
    with pytest.raises(wm.WMError):
        g.dof_map(level)


def test_host_dof_map_at_the_largest_sphere(lib):
    # sphere p = 2 with 512 x 512 elements per patch: 1,579,016 glued DOFs, the
    # largest surface of the uneven multi-instance workload
    import numpy as np
    import paper_2605_24882_gb300 as wm
    sp_ = _oracle_space("sphere", 2, 512, 512, 0)
    l2g, _ = wm.Geometry("sphere", 2, 512).dof_map(0)
    assert sp_.N == 1579016 and l2g.max() + 1 == sp_.N
    assert np.array_equal(l2g, sp_.l2g)


@pytest.mark.parametrize("kind,p,nu,nv", [("sphere", 2, 8, 8), ("sphere", 3, 4, 4), ("sphere", 1, 4, 4),
                                           ("torus", 3, 32, 16), ("torus", 2, 32, 16)])
def test_host_prolongation_refines_splines_exactly(lib, kind, p, nu, nv):
    # Knot insertion (Sec. 2.3): the spaces are nested, so the fine coefficients
    # P c describe the same function as the coarse coefficients c.  Checked by
    # the oracle's own basis evaluation at random parameters of every patch.
    import numpy as np
    import scipy.sparse as sp
    import paper_2605_24882_gb300 as wm
    from oracle.assembly import evaluate
    g = wm.Geometry(kind, p, nu, nv)
    fine, coarse = _oracle_space(kind, p, nu, nv, 0), _oracle_space(kind, p, nu, nv, 1)
    row_ptr, col, val = g.prolongation(0)
    P = sp.csr_matrix((val, col, row_ptr), shape=(fine.N, coarse.N))
    assert (val > 0).all()
    same_row = np.diff(np.repeat(np.arange(fine.N), np.diff(row_ptr))) == 0
    assert (np.diff(col.astype(np.int64))[same_row] > 0).all()            # columns ascend within a row
    np.testing.assert_allclose(P @ np.ones(coarse.N), 1.0, rtol=0, atol=1e-14)   # partition of unity
    rng = np.random.default_rng(2)
    c = rng.standard_normal(coarse.N)
    f = P @ c
    for m in range(fine.surf.n_patches):
        u, v = rng.random(40), rng.random(40)
        np.testing.assert_allclose(evaluate(fine, f, m, u, v), evaluate(coarse, c, m, u, v), rtol=0, atol=1e-12)


def test_host_queries_reject_bad_arguments(lib):
    import numpy as np
    import paper_2605_24882_gb300 as wm
    from paper_2605_24882_gb300 import _capi
    g = wm.Geometry("sphere", 2, 4)
    n, lu, lv, ne, nnz = g.level_sizes(0)
    assert nnz > 0 and g.level_sizes(2)[4] == 0          # 4 -> 2 -> 1 elements: level 2 is the coarsest
    for bad in (-1, 3):
        assert lib.wm_geom_level_sizes(g._h, bad, None, None, None, None, None) == _capi.WM_ERR_INVALID_ARG
    assert lib.wm_geom_prolongation(g._h, 2, None, None, None, 0) == _capi.WM_ERR_INVALID_ARG
    small = np.zeros(6 * lu * lv - 1, dtype=np.int32)
    assert lib.wm_geom_dof_map(g._h, 0, small.ctypes.data, small.size, None, 0) == _capi.WM_ERR_INVALID_ARG
    assert (small == 0).all()
    rp, col, val = (np.zeros(n + 1, np.int32), np.zeros(nnz, np.int32), np.zeros(nnz))
    assert lib.wm_geom_prolongation(g._h, 0, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                    nnz - 1) == _capi.WM_ERR_INVALID_ARG
    assert lib.wm_geom_level_sizes(None, 0, None, None, None, None, None) == _capi.WM_ERR_INVALID_ARG


@pytest.mark.parametrize("lo,hi,n", [(1.0, 10.0, 4), (0.37, 37.0, 16), (2e-6, 0.3, 24), (1e-9, 0.33, 48),
                                     (1.0, 1.0 + 1e-9, 3), (0.5, 2.0, 1)])
def test_hht_rule_matches_oracle(lib, lo, hi, n):
    # the library's elliptic functions (arithmetic-geometric mean scale) against
    # scipy's through the oracle's rule; both reflect the nodes past K/2
    import numpy as np
    import paper_2605_24882_gb300 as wm
    from oracle.sqrt_mass import hht_rule
    w2, c = wm.hht_rule(lo, hi, n)
    w2o, co = hht_rule(lo, hi, n)
    np.testing.assert_allclose(w2, w2o, rtol=1e-12, atol=0)
    np.testing.assert_allclose(c, co, rtol=1e-12, atol=0)
    lam = np.geomspace(lo, hi, 64)
    s = lam * (c[None, :] / (lam[:, None] + w2[None, :])).sum(axis=1)
    so = lam * (co[None, :] / (lam[:, None] + w2o[None, :])).sum(axis=1)
    np.testing.assert_allclose(s, so, rtol=1e-13)


def test_hht_rule_rejects_bad_arguments(lib):
    import paper_2605_24882_gb300 as wm
    from paper_2605_24882_gb300 import _capi
    for args in [(0.0, 1.0, 4), (2.0, 1.0, 4), (1.0, 2.0, 0), (-1.0, 2.0, 4)]:
        with pytest.raises(wm.WMError) as e:
            wm.hht_rule(*args)
        assert e.value.code == _capi.WM_ERR_INVALID_ARG


@pytest.mark.parametrize("kind,p,nu,nv", [("sphere", 1, 4, 4), ("sphere", 2, 8, 8), ("sphere", 3, 4, 4),
                                           ("sphere", 2, 2, 2), ("torus", 3, 16, 8), ("torus", 2, 16, 16)])
def test_mass_bounds_bracket_the_oracle_spectrum(lib, kind, p, nu, nv):
    import numpy as np
    import paper_2605_24882_gb300 as wm
    from oracle import geometry as geo
    from oracle.assembly import assemble
    from oracle.space import GluedSpace
    g = wm.Geometry(kind, p, nu, nv)
    for level in range(2):
        if kind == "torus" and (min(nu, nv) >> level) < 2 * p + 2:
            break
        sp_ = GluedSpace(geo.Surface(kind, p, nu >> level, None if kind == "sphere" else nv >> level))
        _, M = assemble(sp_)
        ev = np.linalg.eigvalsh(M.toarray())
        lo, hi = g.mass_bounds(level)
        assert 0.0 < lo <= ev[0] and ev[-1] <= hi, (level, lo, ev[0], ev[-1], hi)
        # the bounds stay within small factors of the spectrum: the area element
        # varies by 5.2 on the gnomonic sphere, 2.3 on this torus
        assert ev[0] / lo < 40 and hi / ev[-1] < 20, (ev[0] / lo, hi / ev[-1])
    with pytest.raises(wm.WMError):
        g.mass_bounds(-1)


def _nurbs_cases():
    import wm_workloads as wl
    return [("periodic", wl.nurbs_torus(1.0, 0.4), 2, 32, 16), ("periodic", wl.nurbs_torus(1.2, 0.3), 3, 16, 16),
            ("cube", wl.nurbs_bulged_cube(0.3, 2.0), 2, 4, 4), ("cube", wl.nurbs_bulged_cube(0.0), 3, 2, 2),
            ("cube", wl.nurbs_bulged_cube(0.5), 1, 8, 8)]


@pytest.mark.parametrize("case", range(5))
def test_nurbs_host_metric_and_maps_match_oracle(lib, case):
    # the library evaluates the rational map on the host (span search, Cox–de Boor
    # on the span, quotient rule); the oracle through its full-knot-vector bases
    import numpy as np
    import paper_2605_24882_gb300 as wm
    from oracle.assembly import quadrature
    from oracle.nurbs import NurbsSurface
    from oracle.space import GluedSpace
    topo, patches, p, nu, nv = _nurbs_cases()[case]
    g = wm.Geometry.nurbs(topo, patches, p, nu, nv)
    for level in range(2):
        s = NurbsSurface(topo, patches, p, nu >> level, nv >> level)
        q = quadrature(s)
        ref = np.concatenate([np.stack([q[k][m] for k in ("a", "G11", "G12", "G22")], -1).reshape(-1, 4)
                              for m in range(s.n_patches)])
        met = g.metric_host(level)
        np.testing.assert_allclose(met, ref, rtol=0, atol=1e-14 * np.abs(ref).max())
        l2g, conn = g.dof_map(level)
        sp_ = GluedSpace(s)
        assert np.array_equal(l2g, sp_.l2g)
        assert np.array_equal(conn, sp_.connectivity().reshape(conn.shape[0], -1))


@pytest.mark.parametrize("case", range(5))
def test_nurbs_mass_bounds_bracket_the_oracle_spectrum(lib, case):
    import numpy as np
    import paper_2605_24882_gb300 as wm
    from oracle.assembly import assemble
    from oracle.nurbs import NurbsSurface
    from oracle.space import GluedSpace
    topo, patches, p, nu, nv = _nurbs_cases()[case]
    g = wm.Geometry.nurbs(topo, patches, p, nu, nv)
    _, M = assemble(GluedSpace(NurbsSurface(topo, patches, p, nu, nv)))
    ev = np.linalg.eigvalsh(M.toarray())
    lo, hi = g.mass_bounds(0)
    assert 0.0 < lo <= ev[0] and ev[-1] <= hi


def test_nurbs_setup_rejects_bad_input(lib):
    import numpy as np
    import paper_2605_24882_gb300 as wm
    import wm_workloads as wl
    from paper_2605_24882_gb300 import _capi

    def rejected(topo, patches, p=2, nu=16, nv=8):
        with pytest.raises(wm.WMError) as e:
            wm.Geometry.nurbs(topo, patches, p, nu, nv)
        return e.value.code == _capi.WM_ERR_INVALID_ARG

    torus = wl.nurbs_torus()
    t = [dict(q) for q in torus]
    t[0]["cpw"] = torus[0]["cpw"].copy()
    t[0]["cpw"][0, 0, 0] += 1e-3                       # no longer closed
    assert rejected("periodic", t)
    t = [dict(q) for q in torus]
    t[0]["knots_u"] = torus[0]["knots_u"][::-1].copy()  # decreasing
    assert rejected("periodic", t)
    t = [dict(q) for q in torus]
    t[0]["knots_u"] = torus[0]["knots_u"] * 0.5         # not clamped to [0, 1]
    assert rejected("periodic", t)
    t = [dict(q) for q in torus]
    t[0]["cpw"] = torus[0]["cpw"].copy()
    t[0]["cpw"][4, 4, 3] = 0.0                          # non-positive weight
    assert rejected("periodic", t)
    assert rejected("periodic", torus, p=2, nu=4, nv=8)  # fewer than 2p+2 elements
    assert rejected("periodic", torus + torus)           # two patches
    cube = wl.nurbs_bulged_cube(0.2)
    c = [dict(q) for q in cube]
    c[3]["cpw"] = cube[3]["cpw"].copy()
    c[3]["cpw"][0, 1, :3] += 1e-3                        # an edge control point off the shared edge
    assert rejected("cube", c, nu=4, nv=4)
    assert rejected("cube", cube[:5], nu=4, nv=4)
    assert rejected("cube", cube, nu=4, nv=8)
    # analytic kinds have no host metric; NURBS kinds need their own entry point
    g = wm.Geometry("sphere", 2, 4)
    with pytest.raises(wm.WMError) as e:
        g.metric_host(0)
    assert e.value.code == _capi.WM_ERR_UNSUPPORTED
    d = _capi.GeomDesc(kind=_capi.WM_NURBS_CUBE, degree=2, elems_u=4, elems_v=4, R=0.0, r=0.0)
    h = C.c_void_p()
    assert lib.wm_setup_geometry(C.byref(d), C.byref(h)) == _capi.WM_ERR_INVALID_ARG
    np.testing.assert_equal(h.value, None)


def _stencil_cases():
    import wm_workloads as wl
    return [("sphere", 2, 8, 8, None), ("sphere", 3, 4, 4, None), ("sphere", 1, 8, 8, None),
            ("torus", 3, 32, 16, None), ("torus", 2, 16, 16, None), ("cube", 2, 8, 8, wl.nurbs_bulged_cube(0.3))]


@pytest.mark.parametrize("case", range(6))
def test_stencil_form_reproduces_the_operators(lib, case):
    # The shared-memory kernels compute row i in the frame of its owner patch:
    # y_i = sum over the (2p+1)^2 window cells s of coef_i[s] x[ext(cell s)], the
    # coefficients placed by slot.  With the oracle's S and M in those slots this
    # must give S x and M x exactly: every DOF owned once, every non-zero column
    # of a row in exactly one window cell, padding and empty corner cells unused.
    import numpy as np
    import paper_2605_24882_gb300 as wm
    from oracle import geometry as geo
    from oracle.assembly import assemble
    from oracle.nurbs import NurbsSurface
    from oracle.space import GluedSpace
    kind, p, nu, nv, patches = _stencil_cases()[case]
    if patches is None:
        g = wm.Geometry(kind, p, nu, nv)
        surf = geo.Surface(kind, p, nu, None if kind == "sphere" else nv)
    else:
        g = wm.Geometry.nurbs(kind, patches, p, nu, nv)
        surf = NurbsSurface(kind, patches, p, nu, nv)
    S, M = assemble(GluedSpace(surf))
    S, M = S.toarray(), M.toarray()
    ext, own, col, slot = g.stencil(0)
    N, SW = S.shape[0], 2 * p + 1
    owned = own[own >= 0]
    assert np.array_equal(np.sort(owned), np.arange(N))
    x = np.random.default_rng(4).standard_normal(N)
    yS, yM = np.zeros(N), np.zeros(N)
    for m, iv, iu in zip(*np.nonzero(own >= 0)):
        i = own[m, iv, iu]
        s = slot[i]
        assert len(set(s[s >= 0].tolist())) == (s >= 0).sum()         # one stored entry per cell
        assert set(col[i][s >= 0].tolist()) == set(np.nonzero(M[i])[0].tolist())
        for w in np.nonzero(s >= 0)[0]:
            cell = ext[m, iv + s[w] // SW, iu + s[w] % SW]
            assert cell == col[i, w]                                   # the slot's window cell holds the column
            yS[i] += S[i, cell] * x[cell]
            yM[i] += M[i, cell] * x[cell]
        assert (col[i][s < 0] == i).all()                               # padding repeats the row index
    np.testing.assert_allclose(yS, S @ x, rtol=0, atol=1e-13 * np.abs(S).max() * np.abs(x).sum())
    np.testing.assert_allclose(yM, M @ x, rtol=0, atol=1e-13 * np.abs(M).max() * np.abs(x).sum())
