"""GB300 sampler of Whittle–Matérn Gaussian random fields on surfaces.

Python binding of the C ABI (include/wmfield.h): argument marshalling only.
Every numerical step runs in the CUDA library libwmfield.so; PyTorch provides
device memory and streams.  There is no CPU fallback: without the built
library every call raises.

    import paper_2605_24882_gb300 as wm
    geo = wm.Geometry("sphere", degree=2, elems=64)
    hier = wm.Hierarchy(geo, n_levels=7)
    u = hier.sample_fields(kappa=5.0, beta=1.3, sinc_k=0.3, l_lo=-35, l_hi=35,
                           n_samples=256, precision="mixed")
"""
import ctypes as C

import numpy as np
import torch

from . import _capi
from ._capi import WMError, check, lib

__all__ = ["Geometry", "Hierarchy", "philox4x32_10", "normals", "beta_plan", "sinc_nodes", "hht_rule", "WMError",
           "WMField"]

_PREC = {"fp64": _capi.WM_FP64, "mixed": _capi.WM_MIXED}
_SPLIT = {"standard": _capi.WM_SPLIT_STANDARD, "improved": _capi.WM_SPLIT_IMPROVED}


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev_f64(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
    return C.c_void_p(t.data_ptr())


class Geometry:
    """Surface description: 'sphere' (six cube-face patches) or 'torus' (periodic);
    `Geometry.nurbs` builds one from NURBS patches."""

    def __init__(self, kind, degree, elems, elems_v=None, R=1.0, r=0.4):
        d = _capi.GeomDesc(kind=_capi.WM_SPHERE6 if kind == "sphere" else _capi.WM_TORUS, degree=degree,
                           elems_u=elems, elems_v=elems if elems_v is None else elems_v, R=R, r=r)
        h = C.c_void_p()
        check(lib().wm_setup_geometry(C.byref(d), C.byref(h)), "wm_setup_geometry")
        self._h = h
        self.desc = d

    @classmethod
    def nurbs(cls, topology, patches, degree, elems, elems_v=None):
        """Surface from NURBS patches: topology 'periodic' (one patch) or 'cube' (six,
        in the cube-face arrangement); each patch a dict with degree_u, degree_v,
        knots_u, knots_v and cpw [n_v, n_u, 4] (x, y, z, weight)."""
        kind = _capi.WM_NURBS_PERIODIC if topology == "periodic" else _capi.WM_NURBS_CUBE
        d = _capi.GeomDesc(kind=kind, degree=degree, elems_u=elems, elems_v=elems if elems_v is None else elems_v,
                           R=0.0, r=0.0)
        keep = []
        arr = (_capi.NurbsPatch * len(patches))()
        for i, q in enumerate(patches):
            ku = np.ascontiguousarray(q["knots_u"], dtype=np.float64)
            kv = np.ascontiguousarray(q["knots_v"], dtype=np.float64)
            cpw = np.ascontiguousarray(q["cpw"], dtype=np.float64)
            if cpw.ndim != 3 or cpw.shape[2] != 4:
                raise ValueError("cpw must be [n_v, n_u, 4]")
            keep += [ku, kv, cpw]
            arr[i] = _capi.NurbsPatch(degree_u=q["degree_u"], degree_v=q["degree_v"], n_u=cpw.shape[1],
                                      n_v=cpw.shape[0], knots_u=ku.ctypes.data, knots_v=kv.ctypes.data,
                                      cpw=cpw.ctypes.data)
        self = cls.__new__(cls)
        h = C.c_void_p()
        check(lib().wm_setup_geometry_nurbs(C.byref(d), arr, len(patches), C.byref(h)), "wm_setup_geometry_nurbs")
        self._h = h
        self.desc = d
        return self

    def metric_host(self, level=0):
        """Host-only (NURBS kinds): metric terms [n_quad, 4] = (a, G11, G12, G22) at the level's Gauss points."""
        n_p = 6 if self.desc.kind in (_capi.WM_SPHERE6, _capi.WM_NURBS_CUBE) else 1
        nq = self.desc.degree + 1
        n_quad = n_p * (self.desc.elems_u >> level) * (self.desc.elems_v >> level) * nq * nq
        out = np.empty((n_quad, 4), dtype=np.float64)
        check(lib().wm_geom_metric(self._h, level, out.ctypes.data, out.size), "wm_geom_metric")
        return out

    def level_sizes(self, level=0, prolongation=True):
        """Host-only: (N, n_loc_u, n_loc_v, elements, prolongation entries) of a level;
        the last is 0 when `prolongation` is False or at the coarsest level."""
        n, lu, lv, ne, nnz = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int64(0)
        check(lib().wm_geom_level_sizes(self._h, level, C.byref(n), C.byref(lu), C.byref(lv), C.byref(ne),
                                        C.byref(nnz) if prolongation else None), "wm_geom_level_sizes")
        return n.value, lu.value, lv.value, ne.value, nnz.value

    def dof_map(self, level=0):
        """Host-only: local-to-global map [patches, n_loc_v, n_loc_u] and element
        connectivity [elements, (p+1)^2] of a level (int32 numpy arrays)."""
        _, lu, lv, ne, _ = self.level_sizes(level, prolongation=False)
        n_p = 6 if self.desc.kind in (_capi.WM_SPHERE6, _capi.WM_NURBS_CUBE) else 1
        l2g = np.empty((n_p, lv, lu), dtype=np.int32)
        conn = np.empty((ne, (self.desc.degree + 1) ** 2), dtype=np.int32)
        check(lib().wm_geom_dof_map(self._h, level, l2g.ctypes.data, l2g.size, conn.ctypes.data, conn.size),
              "wm_geom_dof_map")
        return l2g, conn

    def prolongation(self, level=0):
        """Host-only: knot-insertion prolongation from level+1 to level as CSR
        arrays (row_ptr int32 [N_fine+1], col int32, val float64)."""
        n, _, _, _, nnz = self.level_sizes(level)
        row_ptr = np.empty(n + 1, dtype=np.int32)
        col = np.empty(nnz, dtype=np.int32)
        val = np.empty(nnz, dtype=np.float64)
        check(lib().wm_geom_prolongation(self._h, level, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data,
                                         nnz), "wm_geom_prolongation")
        return row_ptr, col, val

    def stencil(self, level=0):
        """Host-only: the stencil form (ext, own, col, slot) of a level's rows as int
        numpy arrays (see wm_geom_stencil); raises WMError (unsupported) for levels
        that the row kernels serve."""
        n, lu, lv, _, _ = self.level_sizes(level, prolongation=False)
        n_p = 6 if self.desc.kind in (_capi.WM_SPHERE6, _capi.WM_NURBS_CUBE) else 1
        p = self.desc.degree
        W = C.c_int()
        check(lib().wm_geom_stencil(self._h, level, None, 0, None, 0, None, None, 0, C.byref(W)), "wm_geom_stencil")
        ext = np.empty((n_p, lv + 2 * p, lu + 2 * p), dtype=np.int32)
        own = np.empty((n_p, lv, lu), dtype=np.int32)
        col = np.empty((n, W.value), dtype=np.int32)
        slot = np.empty((n, W.value), dtype=np.int16)
        check(lib().wm_geom_stencil(self._h, level, ext.ctypes.data, ext.size, own.ctypes.data, own.size,
                                    col.ctypes.data, slot.ctypes.data, col.size, C.byref(W)), "wm_geom_stencil")
        return ext, own, col, slot

    def mass_bounds(self, level=0):
        """Host-only: (lo, hi) bracketing the spectrum of the level's mass matrix."""
        lo, hi = C.c_double(), C.c_double()
        check(lib().wm_geom_mass_bounds(self._h, level, C.byref(lo), C.byref(hi)), "wm_geom_mass_bounds")
        return lo.value, hi.value

    def __del__(self):
        if getattr(self, "_h", None) and _capi._lib is not None:
            _capi._lib.wm_destroy_geom(self._h)
            self._h = None


def sinc_nodes(beta, kappa, tol, split="standard"):
    """Sinc step and node range (k, l_lo, l_hi) for an error <= tol per unit load
    in the fractional pass of beta (pass them as sinc_k, l_lo, l_hi)."""
    k, lo, hi = C.c_double(), C.c_int(), C.c_int()
    check(lib().wm_sinc_nodes(beta, _SPLIT[split], kappa, tol, C.byref(k), C.byref(lo), C.byref(hi)),
          "wm_sinc_nodes")
    return k.value, lo.value, hi.value


def hht_rule(lo, hi, n_nodes):
    """Shifts w_k^2 and weights c_k (float64 numpy arrays) of the n_nodes-point
    rule sqrt(A) y ~= A sum_k c_k (A + w_k^2 I)^{-1} y for spectra in [lo, hi]."""
    w2 = np.empty(n_nodes, dtype=np.float64)
    c = np.empty(n_nodes, dtype=np.float64)
    check(lib().wm_hht_rule(lo, hi, n_nodes, w2.ctypes.data if n_nodes > 0 else None,
                            c.ctypes.data if n_nodes > 0 else None), "wm_hht_rule")
    return w2, c


def beta_plan(beta, split="standard"):
    n, bf, ps = C.c_int(), C.c_double(), C.c_int()
    check(lib().wm_beta_plan(beta, _SPLIT[split], C.byref(n), C.byref(bf), C.byref(ps)), "wm_beta_plan")
    return n.value, bf.value, ps.value


def philox4x32_10(ctr, key, stream=None):
    """Philox4x32-10 of counters ctr (int32 CUDA tensor [n, 4], bit patterns) with a 64-bit key."""
    if not (ctr.is_cuda and ctr.dtype == torch.int32 and ctr.dim() == 2 and ctr.shape[1] == 4):
        raise TypeError("ctr must be an int32 CUDA tensor [n, 4]")
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    check(lib().wm_philox4x32_10(C.c_void_p(ctr.data_ptr()), key, C.c_void_p(out.data_ptr()), ctr.shape[0],
                                 _stream(stream)), "wm_philox4x32_10")
    return out


def normals(seed, sample, stream_id, q0, n, device="cuda", stream=None):
    out = torch.empty(n, dtype=torch.float64, device=device)
    check(lib().wm_normals(seed, sample, stream_id, q0, n, C.c_void_p(out.data_ptr()), _stream(stream)),
          "wm_normals")
    return out


class Hierarchy:
    """Dyadic spline hierarchy with the assembled operators on the GPU."""

    def __init__(self, geometry, n_levels, stream=None):
        h = C.c_void_p()
        check(lib().wm_assemble_hierarchy(geometry._h, n_levels, _stream(stream), C.byref(h)),
              "wm_assemble_hierarchy")
        self._h = h
        self.geometry = geometry
        self.n_levels = n_levels

    def __del__(self):
        if getattr(self, "_h", None) and _capi._lib is not None:
            _capi._lib.wm_destroy_hier(self._h)
            self._h = None

    def num_dofs(self, level=0):
        return check(lib().wm_num_dofs(self._h, level), "wm_num_dofs")

    def num_quad_points(self, level=0):
        return check(lib().wm_num_quad_points(self._h, level), "wm_num_quad_points")

    def dof_map(self, level=0):
        g = self.geometry.desc
        p = g.degree
        n = (g.elems_u >> level), (g.elems_v >> level)
        if g.kind in (_capi.WM_TORUS, _capi.WM_NURBS_PERIODIC):
            shape = (1, n[1], n[0])
        else:
            shape = (6, n[1] + p, n[0] + p)
        out = np.zeros(shape, dtype=np.int32)
        check(lib().wm_dof_map(self._h, level, out.ctypes.data_as(C.c_void_p), out.size), "wm_dof_map")
        return out

    def metric(self, level=0, stream=None):
        out = torch.empty((self.num_quad_points(level), 4), dtype=torch.float64, device="cuda")
        check(lib().wm_metric(self._h, level, C.c_void_p(out.data_ptr()), _stream(stream)), "wm_metric")
        return out

    def apply_shifted(self, x, sigma, level=0, precision="fp64", stream=None):
        x = x.contiguous()
        y = torch.empty_like(x)
        sg = (C.c_double * x.shape[0])(*[float(s) for s in sigma])
        check(lib().wm_apply_shifted(self._h, level, x.shape[0], sg, _dev_f64(x, "x"), _dev_f64(y, "y"),
                                     _PREC[precision], _stream(stream)), "wm_apply_shifted")
        return y

    def apply_mass(self, x, level=0, stream=None):
        x = x.contiguous()
        y = torch.empty_like(x)
        check(lib().wm_apply_mass(self._h, level, _dev_f64(x, "x"), _dev_f64(y, "y"), x.shape[0],
                                  _stream(stream)), "wm_apply_mass")
        return y

    def prolongate(self, xc, level=0, stream=None):
        xc = xc.contiguous()
        xf = torch.empty((xc.shape[0], self.num_dofs(level)), dtype=torch.float64, device=xc.device)
        check(lib().wm_prolongate(self._h, level, _dev_f64(xc, "xc"), _dev_f64(xf, "xf"), xc.shape[0],
                                  _stream(stream)), "wm_prolongate")
        return xf

    def restrict(self, rf, level=0, stream=None):
        rf = rf.contiguous()
        rc = torch.empty((rf.shape[0], self.num_dofs(level + 1)), dtype=torch.float64, device=rf.device)
        check(lib().wm_restrict(self._h, level, _dev_f64(rf, "rf"), _dev_f64(rc, "rc"), rf.shape[0],
                                _stream(stream)), "wm_restrict")
        return rc

    def vcycle(self, r, sigma, precision="fp64", smoother_degree=2, cheb_ratio=8.0, stream=None):
        r = r.contiguous()
        z = torch.empty_like(r)
        sg = (C.c_double * r.shape[0])(*[float(s) for s in sigma])
        check(lib().wm_vcycle(self._h, r.shape[0], sg, _dev_f64(r, "r"), _dev_f64(z, "z"), _PREC[precision],
                              smoother_degree, cheb_ratio, _stream(stream)), "wm_vcycle")
        return z

    def set_schedule(self, **kw):
        """Kernel schedule of this hierarchy's batched solves (uni_run, uni_waves,
        vec_rows, vcycle_rows, tail_fused; unnamed fields keep their values; no
        arguments: the defaults)."""
        if not kw:
            check(lib().wm_set_schedule(self._h, None), "wm_set_schedule")
            return self.schedule()
        sc = _capi.Schedule()
        check(lib().wm_get_schedule(self._h, C.byref(sc)), "wm_get_schedule")
        for k, v in kw.items():
            setattr(sc, k, int(v))
        check(lib().wm_set_schedule(self._h, C.byref(sc)), "wm_set_schedule")
        return self.schedule()

    def schedule(self):
        sc = _capi.Schedule()
        check(lib().wm_get_schedule(self._h, C.byref(sc)), "wm_get_schedule")
        return sc.as_dict()

    def noise_loads(self, seed, n_samples, stream=None):
        b = torch.empty((n_samples, self.num_dofs(0)), dtype=torch.float64, device="cuda")
        check(lib().wm_noise_loads(self._h, seed, n_samples, C.c_void_p(b.data_ptr()), _stream(stream)),
              "wm_noise_loads")
        return b

    def noise_loads_sqrt(self, seed, n_samples, lo, hi, n_nodes, rtol=1e-12, max_iter=1000, stream=None):
        """Loads f = sqrt(M) y [n_samples, N] (float64 CUDA tensor) by the n_nodes-point
        Hale–Higham–Trefethen rule on [lo, hi]; returns (f, CG iterations)."""
        f = torch.empty((n_samples, self.num_dofs(0)), dtype=torch.float64, device="cuda")
        it = C.c_int()
        check(lib().wm_noise_loads_sqrt(self._h, seed, n_samples, lo, hi, n_nodes, rtol, max_iter,
                                        C.c_void_p(f.data_ptr()), C.byref(it), _stream(stream)),
              "wm_noise_loads_sqrt")
        return f, it.value

    @staticmethod
    def make_desc(kappa, beta, sinc_k=0.3, l_lo=-35, l_hi=35, n_samples=1, seed=0, split="standard",
                  precision="mixed", rtol=1e-8, max_iter=200, smoother_degree=4, cheb_ratio=12.0,
                  max_systems=0, noise_given=False, preconditioner="vcycle", sample0=0, ckpt="recompute",
                  smoother_degree_coarse=0):
        return _capi.SampleDesc(kappa=kappa, beta=beta, split=_SPLIT[split], sinc_k=sinc_k, l_lo=l_lo, l_hi=l_hi,
                                seed=seed, n_samples=n_samples, sample0=sample0,
                                ckpt={"recompute": _capi.WM_CKPT_RECOMPUTE, "keep": _capi.WM_CKPT_KEEP}[ckpt],
                                smoother_degree_coarse=smoother_degree_coarse,
                                noise_mode=_capi.WM_NOISE_GIVEN if noise_given else _capi.WM_NOISE_DRAW,
                                precision=_PREC[precision], rtol=rtol, max_iter=max_iter,
                                smoother_degree=smoother_degree, cheb_ratio=cheb_ratio, max_systems=max_systems,
                                preconditioner={"vcycle": 0, "bpx": 1}[preconditioner])

    def sample_fields(self, b=None, return_loads=False, out=None, stream=None, check_convergence=True, **kw):
        """Fields u [n_samples, N] (float64 CUDA tensor, or ``out`` which may be a host tensor).

        With ``b`` given the loads are taken from it, else drawn from Philox
        with ``seed``.  Returns u (and the loads, and the stats dict).
        """
        d = self.make_desc(noise_given=b is not None, **kw)
        N = self.num_dofs(0)
        u = out if out is not None else torch.empty((d.n_samples, N), dtype=torch.float64, device="cuda")
        if b is None and return_loads:
            b = torch.empty((d.n_samples, N), dtype=torch.float64, device="cuda")
        st = _capi.Stats()
        bptr = C.c_void_p(b.data_ptr()) if b is not None else None
        rc = lib().wm_sample_fields(self._h, C.byref(d), C.c_void_p(u.data_ptr()), bptr, C.byref(st),
                                    _stream(stream))
        if rc == _capi.WM_ERR_NOT_CONVERGED and not check_convergence:
            rc = 0
        check(rc, "wm_sample_fields")
        if return_loads:
            return u, b, st.as_dict()
        return u, st.as_dict()

    def sample_fields_backward(self, b, grad_u, stream=None, return_stats=False, **kw):
        """(dL/db, dL/dkappa) for loads b and dL/du = grad_u (and the stats dict)."""
        d = self.make_desc(noise_given=True, **kw)
        gb = torch.empty_like(b)
        gk = C.c_double(0.0)
        st = _capi.Stats()
        check(lib().wm_sample_fields_backward(self._h, C.byref(d), _dev_f64(b, "b"), _dev_f64(grad_u, "grad_u"),
                                              _dev_f64(gb, "grad_b"), C.byref(gk), C.byref(st), _stream(stream)),
              "wm_sample_fields_backward")
        if return_stats:
            return gb, gk.value, st.as_dict()
        return gb, gk.value


def sample_fields_batched(hiers, descs, stream=None, outs=None):
    """Fields of several independent problems in one call (list of tensors, stats list).

    Instances that share a Hierarchy object (and solver settings) share the
    batched solves.  ``outs``: optional list of [n_samples, N] float64 CUDA
    tensors to write into."""
    n = len(hiers)
    H = (C.c_void_p * n)(*[h._h for h in hiers])
    D = (_capi.SampleDesc * n)(*descs)
    if outs is None:
        outs = [torch.empty((d.n_samples, h.num_dofs(0)), dtype=torch.float64, device="cuda")
                for h, d in zip(hiers, descs)]
    U = (C.c_void_p * n)(*[C.c_void_p(u.data_ptr()) for u in outs])
    st = (_capi.Stats * n)()
    check(lib().wm_sample_fields_batched(n, H, D, U, st, _stream(stream)), "wm_sample_fields_batched")
    return outs, [s.as_dict() for s in st]


def profile_enable(on=True):
    """Start (reset) or stop live per-kernel event timing inside the library."""
    check(lib().wm_profile_enable(1 if on else 0), "wm_profile_enable")


def profile_read():
    """{category: dict(ms, timed, launches, bytes, flops)} since profile_enable(True)."""
    out = {}
    for c in range(lib().wm_profile_categories()):
        ms, nt, na, by, fl, name = C.c_double(), C.c_int64(), C.c_int64(), C.c_double(), C.c_double(), C.c_char_p()
        check(lib().wm_profile_read(c, C.byref(ms), C.byref(nt), C.byref(na), C.byref(by), C.byref(fl),
                                    C.byref(name)), "wm_profile_read")
        out[name.value.decode()] = dict(ms=ms.value, timed=nt.value, launches=na.value, bytes=by.value,
                                        flops=fl.value)
    return out


class WMField(torch.autograd.Function):
    """u = F(b, kappa): the fields of loads b [n_samples, N]; the backward pass
    runs the adjoint solves (wm_sample_fields_backward) for dL/db and dL/dkappa.

    ``kw`` holds the remaining sampler parameters (beta, sinc_k, l_lo, l_hi,
    n_samples, precision, rtol, ...), without kappa and b.  The forward keeps
    its per-node solutions in the hierarchy's workspace when they fit
    (``ckpt="keep"``, the default here), so that the backward solves only the
    adjoint systems; ``ckpt="recompute"`` re-solves them in the backward.
    """

    @staticmethod
    def forward(ctx, b, kappa, hier, kw):
        kappa_f = float(kappa)
        kw = dict(kw)
        kw.setdefault("ckpt", "keep")
        u, _ = hier.sample_fields(b=b.detach().contiguous(), kappa=kappa_f, **kw)
        ctx.save_for_backward(b)
        ctx.hier, ctx.kw, ctx.kappa = hier, kw, kappa_f
        ctx.kappa_is_tensor = isinstance(kappa, torch.Tensor)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (b,) = ctx.saved_tensors
        gb, gk = ctx.hier.sample_fields_backward(b.detach().contiguous(), grad_u.contiguous(), kappa=ctx.kappa,
                                                 **ctx.kw)
        gk_t = torch.tensor(gk, dtype=torch.float64) if ctx.kappa_is_tensor else None
        return gb, gk_t, None, None
