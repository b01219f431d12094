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
