"""ctypes declarations of the C ABI in include/wmfield.h (marshalling only)."""
import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libwmfield.so")

WM_OK = 0
WM_ERR_INVALID_ARG = -1
WM_ERR_OOM = -2
WM_ERR_CUDA = -3
WM_ERR_NOT_CONVERGED = -4
WM_ERR_NONFINITE = -5
WM_ERR_UNSUPPORTED = -7

WM_SPHERE6 = 0
WM_TORUS = 1
WM_NURBS_PERIODIC = 2
WM_NURBS_CUBE = 3
WM_FP64 = 0
WM_MIXED = 1
WM_SPLIT_STANDARD = 0
WM_SPLIT_IMPROVED = 1
WM_NOISE_DRAW = 0
WM_NOISE_GIVEN = 1
WM_CKPT_RECOMPUTE = 0
WM_CKPT_KEEP = 1


class GeomDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("degree", C.c_int), ("elems_u", C.c_int), ("elems_v", C.c_int),
                ("R", C.c_double), ("r", C.c_double)]


class NurbsPatch(C.Structure):
    _fields_ = [("degree_u", C.c_int), ("degree_v", C.c_int), ("n_u", C.c_int), ("n_v", C.c_int),
                ("knots_u", C.c_void_p), ("knots_v", C.c_void_p), ("cpw", C.c_void_p)]


class SampleDesc(C.Structure):
    _fields_ = [("kappa", C.c_double), ("beta", C.c_double), ("split", C.c_int), ("sinc_k", C.c_double),
                ("l_lo", C.c_int), ("l_hi", C.c_int), ("seed", C.c_uint64), ("n_samples", C.c_int),
                ("noise_mode", C.c_int), ("precision", C.c_int), ("rtol", C.c_double), ("max_iter", C.c_int),
                ("smoother_degree", C.c_int), ("cheb_ratio", C.c_double), ("max_systems", C.c_int),
                ("preconditioner", C.c_int), ("sample0", C.c_int), ("ckpt", C.c_int),
                ("smoother_degree_coarse", C.c_int)]


class Schedule(C.Structure):
    _fields_ = [("uni_run", C.c_int), ("uni_waves", C.c_int), ("vec_rows", C.c_int), ("vcycle_rows", C.c_int),
                ("tail_fused", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("n_systems", C.c_int), ("n_batches", C.c_int), ("max_iterations", C.c_int),
                ("total_iterations", C.c_int), ("n_not_converged", C.c_int), ("max_rel_residual", C.c_double),
                ("n_int_solves", C.c_int), ("n_frac_passes", C.c_int), ("n_nodes", C.c_int),
                ("n_replacements", C.c_int), ("n_df_fallbacks", C.c_int), ("ckpt_kept", C.c_int),
                ("ckpt_used", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = C.c_void_p
_i = C.c_int
_d = C.c_double
_i64 = C.c_int64
_u64 = C.c_uint64

_PROTOS = {
    "wm_setup_geometry": (_i, [C.POINTER(GeomDesc), C.POINTER(_vp)]),
    "wm_setup_geometry_nurbs": (_i, [C.POINTER(GeomDesc), C.POINTER(NurbsPatch), _i, C.POINTER(_vp)]),
    "wm_geom_metric": (_i, [_vp, _i, _vp, _i64]),
    "wm_assemble_hierarchy": (_i, [_vp, _i, _vp, C.POINTER(_vp)]),
    "wm_num_levels": (_i, [_vp]),
    "wm_num_dofs": (_i, [_vp, _i]),
    "wm_num_quad_points": (_i, [_vp, _i]),
    "wm_dof_map": (_i, [_vp, _i, _vp, _i64]),
    "wm_geom_level_sizes": (_i, [_vp, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), C.POINTER(_i),
                                 C.POINTER(_i64)]),
    "wm_geom_dof_map": (_i, [_vp, _i, _vp, _i64, _vp, _i64]),
    "wm_geom_prolongation": (_i, [_vp, _i, _vp, _vp, _vp, _i64]),
    "wm_geom_mass_bounds": (_i, [_vp, _i, C.POINTER(_d), C.POINTER(_d)]),
    "wm_geom_stencil": (_i, [_vp, _i, _vp, _i64, _vp, _i64, _vp, _vp, _i64, C.POINTER(_i)]),
    "wm_hht_rule": (_i, [_d, _d, _i, _vp, _vp]),
    "wm_metric": (_i, [_vp, _i, _vp, _vp]),
    "wm_apply_shifted": (_i, [_vp, _i, _i, C.POINTER(_d), _vp, _vp, _i, _vp]),
    "wm_apply_mass": (_i, [_vp, _i, _vp, _vp, _i, _vp]),
    "wm_prolongate": (_i, [_vp, _i, _vp, _vp, _i, _vp]),
    "wm_restrict": (_i, [_vp, _i, _vp, _vp, _i, _vp]),
    "wm_vcycle": (_i, [_vp, _i, C.POINTER(_d), _vp, _vp, _i, _i, _d, _vp]),
    "wm_philox4x32_10": (_i, [_vp, _u64, _vp, _i64, _vp]),
    "wm_normals": (_i, [_u64, _i, _i, _i64, _i64, _vp, _vp]),
    "wm_noise_loads": (_i, [_vp, _u64, _i, _vp, _vp]),
    "wm_noise_loads_noalloc": (_i, [_vp, _u64, _i, _vp, _vp]),
    "wm_noise_loads_sqrt": (_i, [_vp, _u64, _i, _d, _d, _i, _d, _i, _vp, C.POINTER(_i), _vp]),
    "wm_sample_fields": (_i, [_vp, C.POINTER(SampleDesc), _vp, _vp, C.POINTER(Stats), _vp]),
    "wm_sample_fields_batched": (_i, [_i, C.POINTER(_vp), C.POINTER(SampleDesc), C.POINTER(_vp),
                                      C.POINTER(Stats), _vp]),
    "wm_sample_fields_backward": (_i, [_vp, C.POINTER(SampleDesc), _vp, _vp, _vp, C.POINTER(_d), C.POINTER(Stats),
                                       _vp]),
    "wm_beta_plan": (_i, [_d, _i, C.POINTER(_i), C.POINTER(_d), C.POINTER(_i)]),
    "wm_sinc_nodes": (_i, [_d, _i, _d, _d, C.POINTER(_d), C.POINTER(_i), C.POINTER(_i)]),
    "wm_set_schedule": (_i, [_vp, C.POINTER(Schedule)]),
    "wm_get_schedule": (_i, [_vp, C.POINTER(Schedule)]),
    "wm_profile_enable": (_i, [_i]),
    "wm_profile_read": (_i, [_i, C.POINTER(_d), C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_d), C.POINTER(_d),
                             C.POINTER(C.c_char_p)]),
    "wm_profile_categories": (_i, []),
    "wm_error_string": (C.c_char_p, [_i]),
    "wm_last_error": (C.c_char_p, []),
    "wm_destroy_hier": (None, [_vp]),
    "wm_destroy_geom": (None, [_vp]),
}

_lib = None


def lib():
    """The loaded library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libwmfield.so is missing: run paper_2605_24882_gb300.build.build() "
                              "(nvcc, sm_103a) before using the sampler")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class WMError(RuntimeError):
    def __init__(self, code, where):
        L = lib()
        msg = "%s: %s (%d)" % (where, L.wm_error_string(code).decode(), code)
        detail = L.wm_last_error().decode()
        if detail:
            msg += ": " + detail
        super().__init__(msg)
        self.code = code


def check(code, where):
    if code < 0:
        raise WMError(code, where)
    return code
