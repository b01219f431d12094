// C ABI of the sampler: handles, hierarchy assembly and the sampling driver.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>

#include "wm_solver.h"
#include "wm_stencil.h"

namespace {

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_level(wm_hier_t h, int level) {
  if (!h) return WM_ERR_INVALID_ARG;
  if (level < 0 || level >= (int)h->lv.size()) {
    wm_set_error("level %d out of range [0, %d)", level, (int)h->lv.size());
    return WM_ERR_INVALID_ARG;
  }
  return WM_OK;
}

WorkSpace& workspace(wm_hier_t h) {
  if (!h->ws) h->ws = new WorkSpace();
  return *h->ws;
}

// per-system bytes of a batched solve (float64 solution, recursion vectors and
// V-cycle levels in the solve's precision)
size_t bytes_per_system(const wm_hier* h, bool dbl) {
  size_t e = dbl ? sizeof(double) : sizeof(float);
  size_t b = (size_t)h->lv[0].N * (sizeof(double) + 3 * e);
  for (size_t l = 0; l < h->lv.size(); ++l) b += (size_t)h->lv[l].N * e * (l + 1 < h->lv.size() ? 5 : 3);
  return b;
}

// temporary tiled copies of caller vectors for the component entry points
struct Tmp {
  DevBuf<double> a, b, sg;
  DevBuf<float> fa, fb;
  ~Tmp() {
    a.release();
    b.release();
    sg.release();
    fa.release();
    fb.release();
  }
};

}  // namespace

extern "C" const char* wm_error_string(int code) {
  switch (code) {
    case WM_OK: return "ok";
    case WM_ERR_INVALID_ARG: return "invalid argument";
    case WM_ERR_OOM: return "out of memory";
    case WM_ERR_CUDA: return "CUDA error";
    case WM_ERR_NOT_CONVERGED: return "not converged";
    case WM_ERR_NONFINITE: return "non-finite value";
    case WM_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown error";
  }
}

// ------------------------------------------------------------------ geometry
extern "C" int wm_setup_geometry(const wm_geom_desc* d, wm_geom_t* out) {
  if (!d || !out) return WM_ERR_INVALID_ARG;
  *out = nullptr;
  if (d->kind != WM_SPHERE6 && d->kind != WM_TORUS) {
    wm_set_error("unknown surface kind %d", d->kind);
    return WM_ERR_INVALID_ARG;
  }
  if (d->degree < 1 || d->degree > 4) {
    wm_set_error("degree %d outside 1..4", d->degree);
    return WM_ERR_INVALID_ARG;
  }
  if (d->elems_u < 1 || d->elems_v < 1 || (d->elems_u & (d->elems_u - 1)) || (d->elems_v & (d->elems_v - 1))) {
    wm_set_error("element counts must be powers of two");
    return WM_ERR_INVALID_ARG;
  }
  if (d->kind == WM_SPHERE6 && d->elems_u != d->elems_v) {
    wm_set_error("cube-sphere patches are square");
    return WM_ERR_INVALID_ARG;
  }
  if (d->kind == WM_TORUS) {
    if (!(d->R > d->r && d->r > 0)) {
      wm_set_error("torus needs R > r > 0");
      return WM_ERR_INVALID_ARG;
    }
    if (d->elems_u < 2 * d->degree + 2 || d->elems_v < 2 * d->degree + 2) {
      wm_set_error("periodic patch needs at least 2p+2 elements per direction");
      return WM_ERR_INVALID_ARG;
    }
  }
  wm_geom* g = new (std::nothrow) wm_geom;
  if (!g) return WM_ERR_OOM;
  g->d = *d;
  g->np = d->kind == WM_SPHERE6 ? 6 : 1;
  *out = g;
  return WM_OK;
}

extern "C" int wm_setup_geometry_nurbs(const wm_geom_desc* d, const wm_nurbs_patch* patches, int n_patches,
                                       wm_geom_t* out) {
  if (!d || !out || !patches) return WM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!wm_is_nurbs(d->kind)) {
    wm_set_error("kind %d is not a NURBS kind", d->kind);
    return WM_ERR_INVALID_ARG;
  }
  const bool periodic = wm_periodic(d->kind);
  if (n_patches != (periodic ? 1 : 6)) {
    wm_set_error("%s takes %d patches", periodic ? "WM_NURBS_PERIODIC" : "WM_NURBS_CUBE", periodic ? 1 : 6);
    return WM_ERR_INVALID_ARG;
  }
  if (d->degree < 1 || d->degree > 4) {
    wm_set_error("degree %d outside 1..4", d->degree);
    return WM_ERR_INVALID_ARG;
  }
  if (d->elems_u < 1 || d->elems_v < 1 || (d->elems_u & (d->elems_u - 1)) || (d->elems_v & (d->elems_v - 1))) {
    wm_set_error("element counts must be powers of two");
    return WM_ERR_INVALID_ARG;
  }
  if (!periodic && d->elems_u != d->elems_v) {
    wm_set_error("cube-arranged patches are square");
    return WM_ERR_INVALID_ARG;
  }
  if (periodic && (d->elems_u < 2 * d->degree + 2 || d->elems_v < 2 * d->degree + 2)) {
    wm_set_error("periodic patch needs at least 2p+2 elements per direction");
    return WM_ERR_INVALID_ARG;
  }
  std::vector<WmNurbs> copy(n_patches);
  for (int m = 0; m < n_patches; ++m) {
    const wm_nurbs_patch& q = patches[m];
    if (q.degree_u < 1 || q.degree_u > 8 || q.degree_v < 1 || q.degree_v > 8 || q.n_u < q.degree_u + 1 ||
        q.n_v < q.degree_v + 1 || !q.knots_u || !q.knots_v || !q.cpw) {
      wm_set_error("patch %d: degrees 1..8, n >= degree + 1 and all arrays given", m);
      return WM_ERR_INVALID_ARG;
    }
    WmNurbs& c = copy[m];
    c.pu = q.degree_u;
    c.pv = q.degree_v;
    c.nu = q.n_u;
    c.nv = q.n_v;
    c.ku.assign(q.knots_u, q.knots_u + q.n_u + q.degree_u + 1);
    c.kv.assign(q.knots_v, q.knots_v + q.n_v + q.degree_v + 1);
    c.cpw.assign(q.cpw, q.cpw + (size_t)q.n_u * q.n_v * 4);
  }
  WM_TRY(wm_host_nurbs_check(d->kind, copy));
  wm_geom* g = new (std::nothrow) wm_geom;
  if (!g) return WM_ERR_OOM;
  g->d = *d;
  g->np = n_patches;
  g->nurbs.swap(copy);
  *out = g;
  return WM_OK;
}

extern "C" void wm_destroy_geom(wm_geom_t g) { delete g; }

static void release_level(wm_level& L) {
  L.d_conn.release(); L.d_col.release(); L.d_diag_slot.release(); L.d_metric.release();
  L.d_Se.release(); L.d_Me.release(); L.d_asm_ptr.release(); L.d_asm_idx.release();
  L.d_S64.release(); L.d_M64.release(); L.d_S32.release(); L.d_M32.release();
  L.d_dS64.release(); L.d_dM64.release(); L.d_dS32.release(); L.d_dM32.release();
  L.d_bu.release(); L.d_du.release(); L.d_bv.release(); L.d_dv.release();
  L.d_Pptr.release(); L.d_Pcol.release(); L.d_Rptr.release(); L.d_Rcol.release();
  L.d_Pval64.release(); L.d_Rval64.release(); L.d_Pval32.release(); L.d_Rval32.release();
  L.d_ng_ptr.release(); L.d_ng_idx.release(); L.d_Sdense.release(); L.d_Mdense.release(); L.d_noise_w.release();
  L.d_pk32.release(); L.d_pk64.release(); L.d_P32.release(); L.d_R32.release(); L.d_P64.release();
  L.d_R64.release();
  L.d_ext.release(); L.d_own.release(); L.d_csm32.release(); L.d_csm64.release(); L.d_csmdf.release();
}

extern "C" void wm_destroy_hier(wm_hier_t h) {
  if (!h) return;
  if (h->ws) {
    h->ws->release();
    delete h->ws;
  }
  for (auto& L : h->lv) release_level(L);
  h->d_gw.release();
  h->d_gx.release();
  delete h;
}

static int assemble(wm_hier* h, int n_levels, cudaStream_t s) {
  const wm_geom_desc& g = h->g;
  h->lv.resize(n_levels);
  for (int l = 0; l < n_levels; ++l) {
    wm_level& L = h->lv[l];
    int nu = g.elems_u >> l, nv = g.elems_v >> l;
    WM_TRY(wm_host_build_level(g, h->np, nu, nv, L));
    wm_host_tables(g, h->gx, L);
    std::vector<int32_t> ngp, ngi;
    wm_host_noise_map(L, ngp, ngi);
    WM_TRY(L.d_conn.upload(L.conn, s));
    WM_TRY(L.d_col.upload(L.col, s));
    WM_TRY(L.d_diag_slot.upload(L.diag_slot, s));
    WM_TRY(L.d_ng_ptr.upload(ngp, s));
    WM_TRY(L.d_ng_idx.upload(ngi, s));
    WM_TRY(L.d_bu.upload(L.bu, s));
    WM_TRY(L.d_du.upload(L.du, s));
    WM_TRY(L.d_bv.upload(L.bv, s));
    WM_TRY(L.d_dv.upload(L.dv, s));
    WM_TRY(L.d_metric.alloc((size_t)L.E * h->nq * h->nq * 4));
    WM_TRY(L.d_Se.alloc((size_t)L.E * L.nk * L.nk));
    WM_TRY(L.d_Me.alloc((size_t)L.E * L.nk * L.nk));
    size_t nw = (size_t)L.N * L.W;
    WM_TRY(L.d_S64.alloc(nw));
    WM_TRY(L.d_M64.alloc(nw));
    WM_TRY(L.d_S32.alloc(nw));
    WM_TRY(L.d_M32.alloc(nw));
    WM_TRY(L.d_dS64.alloc(L.N));
    WM_TRY(L.d_dM64.alloc(L.N));
    WM_TRY(L.d_dS32.alloc(L.N));
    WM_TRY(L.d_dM32.alloc(L.N));
    if (wm_is_nurbs(g.kind)) {
      // NURBS maps are evaluated on the host (wm_host_nurbs_metric) and uploaded
      std::vector<double> met;
      WM_TRY(wm_host_nurbs_metric(h->nurbs, nu, nv, h->gx, met));
      WM_CUDA(cudaMemcpyAsync(L.d_metric.p, met.data(), met.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      WM_CUDA(cudaStreamSynchronize(s));
    } else {
      WM_TRY(wm_k_metric(h, L, s));
    }
    if (l == 0) WM_TRY(wm_k_noise_weights(h, L, s));
    WM_TRY(wm_k_element_matrices(h, L, s));
    WM_TRY(wm_k_assemble_rows(h, L, s));
    WM_TRY(wm_k_pack_rows(L, s));
    WM_TRY(wm_sten_build(g, h->np, L, s));
    // element matrices are not needed after assembly
    WM_CUDA(cudaStreamSynchronize(s));
    L.d_Se.release();
    L.d_Me.release();
    // host integer tables kept only where needed later
    L.conn.clear();
    L.conn.shrink_to_fit();
  }
  for (int l = 0; l + 1 < n_levels; ++l) {
    std::vector<int32_t> Pp, Pc, Rp, Rc;
    std::vector<double> Pv, Rv;
    // connectivity is rebuilt implicitly from l2g inside the prolongation
    WM_TRY(wm_host_prolongation(g, h->np, h->lv[l], h->lv[l + 1], Pp, Pc, Pv, Rp, Rc, Rv));
    wm_level& F = h->lv[l];
    F.nP = F.N;
    F.nR = h->lv[l + 1].N;
    F.nnzP = (int64_t)Pc.size();
    WM_TRY(F.d_Pptr.upload(Pp, s));
    WM_TRY(F.d_Pcol.upload(Pc, s));
    WM_TRY(F.d_Pval64.upload(Pv, s));
    WM_TRY(F.d_Rptr.upload(Rp, s));
    WM_TRY(F.d_Rcol.upload(Rc, s));
    WM_TRY(F.d_Rval64.upload(Rv, s));
    std::vector<float> Pf(Pv.begin(), Pv.end()), Rf(Rv.begin(), Rv.end());
    WM_TRY(F.d_Pval32.upload(Pf, s));
    WM_TRY(F.d_Rval32.upload(Rf, s));
    {
      std::vector<PkTr32> p32(Pc.size()), r32(Rc.size());
      std::vector<PkTr64> p64(Pc.size()), r64(Rc.size());
      for (size_t t = 0; t < Pc.size(); ++t) {
        p32[t] = {Pc[t], (float)Pv[t]};
        p64[t] = {Pv[t], Pc[t], 0};
      }
      for (size_t t = 0; t < Rc.size(); ++t) {
        r32[t] = {Rc[t], (float)Rv[t]};
        r64[t] = {Rv[t], Rc[t], 0};
      }
      WM_TRY(F.d_P32.upload(p32, s));
      WM_TRY(F.d_R32.upload(r32, s));
      WM_TRY(F.d_P64.upload(p64, s));
      WM_TRY(F.d_R64.upload(r64, s));
      WM_CUDA(cudaStreamSynchronize(s));
    }
    WM_CUDA(cudaStreamSynchronize(s));
  }
  wm_level& C = h->lv[n_levels - 1];
  if (C.N <= 160) {
    WM_TRY(C.d_Sdense.alloc((size_t)C.N * C.N));
    WM_TRY(C.d_Mdense.alloc((size_t)C.N * C.N));
    WM_TRY(wm_k_dense_coarse(C, s));
  }
  WM_CUDA(cudaStreamSynchronize(s));
  return WM_OK;
}

// Levels a hierarchy of this surface may have: halving down to one element per
// patch side (cube sphere) or to 2p+2 elements per side (periodic torus).
static int max_levels(const wm_geom_desc& g) {
  int minside = std::min(g.elems_u, g.elems_v);
  int lowest = wm_periodic(g.kind) ? 2 * g.degree + 2 : 1;
  int maxlev = 0;
  while ((minside >> maxlev) >= lowest) ++maxlev;
  return maxlev;
}

extern "C" int wm_assemble_hierarchy(wm_geom_t geom, int n_levels, void* stream, wm_hier_t* out) {
  if (!geom || !out) return WM_ERR_INVALID_ARG;
  *out = nullptr;
  const wm_geom_desc& g = geom->d;
  int maxlev = max_levels(g);
  if (n_levels < 1 || n_levels > maxlev) {
    wm_set_error("n_levels %d outside 1..%d for this surface", n_levels, maxlev);
    return WM_ERR_INVALID_ARG;
  }
  wm_hier* h = new (std::nothrow) wm_hier;
  if (!h) return WM_ERR_OOM;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    wm_set_error("no current CUDA device");
    return WM_ERR_CUDA;
  }
  h->g = g;
  h->nurbs = geom->nurbs;
  h->np = geom->np;
  h->p = g.degree;
  h->nq = g.degree + 1;
  wm_gauss_legendre01(h->nq, h->gx, h->gw);
  cudaStream_t s = as_stream(stream);
  int rc = h->d_gw.upload(h->gw, s);
  if (rc == WM_OK) rc = h->d_gx.upload(h->gx, s);
  if (rc == WM_OK) rc = assemble(h, n_levels, s);
  if (rc != WM_OK) {
    wm_destroy_hier(h);
    return rc;
  }
  *out = h;
  return WM_OK;
}

extern "C" int wm_set_schedule(wm_hier_t h, const wm_schedule* sc) {
  if (!h) return WM_ERR_INVALID_ARG;
  const wm_schedule def{8, 4, 128, 16, 1};
  const wm_schedule v = sc ? *sc : def;
  if (v.uni_run < 1 || v.uni_run > kUniGroup || v.uni_waves < 1 || v.uni_waves > 64 || v.vec_rows < 32 ||
      v.vec_rows > 4096 || v.vcycle_rows < 8 || v.vcycle_rows > 1024 || v.tail_fused < 0 || v.tail_fused > 1) {
    wm_set_error("schedule out of range: uni_run 1..%d, uni_waves 1..64, vec_rows 32..4096, vcycle_rows 8..1024, "
                 "tail_fused 0..1",
                 kUniGroup);
    return WM_ERR_INVALID_ARG;
  }
  h->sched = v;
  return WM_OK;
}

extern "C" int wm_get_schedule(wm_hier_t h, wm_schedule* out) {
  if (!h || !out) return WM_ERR_INVALID_ARG;
  *out = h->sched;
  return WM_OK;
}

extern "C" int wm_num_levels(wm_hier_t h) { return h ? (int)h->lv.size() : WM_ERR_INVALID_ARG; }

extern "C" int wm_num_dofs(wm_hier_t h, int level) {
  WM_TRY(check_level(h, level));
  return h->lv[level].N;
}

extern "C" int wm_num_quad_points(wm_hier_t h, int level) {
  WM_TRY(check_level(h, level));
  return h->lv[level].E * h->nq * h->nq;
}

extern "C" int wm_dof_map(wm_hier_t h, int level, int32_t* out, int64_t cap) {
  WM_TRY(check_level(h, level));
  const wm_level& L = h->lv[level];
  if (!out || cap < (int64_t)L.l2g.size()) return WM_ERR_INVALID_ARG;
  std::memcpy(out, L.l2g.data(), L.l2g.size() * sizeof(int32_t));
  return (int)L.l2g.size();
}

// ------------------------------------------------------- host-only space queries
static int check_geom_level(wm_geom_t g, int level, int need) {
  if (!g) return WM_ERR_INVALID_ARG;
  if (level < 0 || level + need >= max_levels(g->d)) {
    wm_set_error("level %d outside 0..%d for this surface", level, max_levels(g->d) - 1 - need);
    return WM_ERR_INVALID_ARG;
  }
  return WM_OK;
}

static int geom_level(wm_geom_t g, int level, int need, wm_level& L) {
  WM_TRY(check_geom_level(g, level, need));
  return wm_host_build_level(g->d, g->np, g->d.elems_u >> level, g->d.elems_v >> level, L);
}

static int geom_prolongation(wm_geom_t g, int level, std::vector<int32_t>& Pp, std::vector<int32_t>& Pc,
                             std::vector<double>& Pv) {
  wm_level F, C;
  WM_TRY(geom_level(g, level, 1, F));
  WM_TRY(geom_level(g, level + 1, 0, C));
  std::vector<int32_t> Rp, Rc;
  std::vector<double> Rv;
  return wm_host_prolongation(g->d, g->np, F, C, Pp, Pc, Pv, Rp, Rc, Rv);
}

extern "C" int wm_geom_level_sizes(wm_geom_t g, int level, int* n_dofs, int* n_loc_u, int* n_loc_v,
                                   int* n_elems, int64_t* prolong_nnz) {
  wm_level L;
  WM_TRY(geom_level(g, level, 0, L));
  if (n_dofs) *n_dofs = L.N;
  if (n_loc_u) *n_loc_u = L.nlu;
  if (n_loc_v) *n_loc_v = L.nlv;
  if (n_elems) *n_elems = L.E;
  if (prolong_nnz) {
    *prolong_nnz = 0;
    if (level + 1 < max_levels(g->d)) {
      std::vector<int32_t> Pp, Pc;
      std::vector<double> Pv;
      WM_TRY(geom_prolongation(g, level, Pp, Pc, Pv));
      *prolong_nnz = (int64_t)Pc.size();
    }
  }
  return WM_OK;
}

extern "C" int wm_geom_dof_map(wm_geom_t g, int level, int32_t* l2g, int64_t l2g_cap, int32_t* conn,
                               int64_t conn_cap) {
  wm_level L;
  WM_TRY(geom_level(g, level, 0, L));
  if (!l2g || l2g_cap < (int64_t)L.l2g.size() || (conn && conn_cap < (int64_t)L.conn.size())) {
    wm_set_error("output buffers too small");
    return WM_ERR_INVALID_ARG;
  }
  std::memcpy(l2g, L.l2g.data(), L.l2g.size() * sizeof(int32_t));
  if (conn) std::memcpy(conn, L.conn.data(), L.conn.size() * sizeof(int32_t));
  return WM_OK;
}

extern "C" int wm_geom_stencil(wm_geom_t g, int level, int32_t* ext, int64_t ext_cap, int32_t* own,
                               int64_t own_cap, int32_t* col, int16_t* slot, int64_t row_cap, int* W) {
  wm_level L;
  WM_TRY(geom_level(g, level, 0, L));
  if (W) *W = L.W;
  if (!ext && !own && !col && !slot) return WM_OK;
  std::vector<int32_t> e, o;
  std::vector<int16_t> sl;
  WM_TRY(wm_host_stencil(g->d, g->np, L, e, o, sl));
  if (!ext || !own || !col || !slot || ext_cap < (int64_t)e.size() || own_cap < (int64_t)o.size() ||
      row_cap < (int64_t)L.col.size()) {
    wm_set_error("output buffers too small");
    return WM_ERR_INVALID_ARG;
  }
  std::memcpy(ext, e.data(), e.size() * sizeof(int32_t));
  std::memcpy(own, o.data(), o.size() * sizeof(int32_t));
  std::memcpy(col, L.col.data(), L.col.size() * sizeof(int32_t));
  std::memcpy(slot, sl.data(), sl.size() * sizeof(int16_t));
  return WM_OK;
}

static int geom_nurbs_metric(wm_geom_t g, int level, std::vector<double>& met) {
  std::vector<double> gx, gw;
  wm_gauss_legendre01(g->d.degree + 1, gx, gw);
  return wm_host_nurbs_metric(g->nurbs, g->d.elems_u >> level, g->d.elems_v >> level, gx, met);
}

extern "C" int wm_geom_mass_bounds(wm_geom_t g, int level, double* lo, double* hi) {
  WM_TRY(check_geom_level(g, level, 0));
  if (!lo || !hi) return WM_ERR_INVALID_ARG;
  const int nu = g->d.elems_u >> level, nv = g->d.elems_v >> level;
  if (!wm_is_nurbs(g->d.kind)) return wm_host_mass_bounds(g->d, nu, nv, lo, hi);
  std::vector<double> met;
  WM_TRY(geom_nurbs_metric(g, level, met));
  double amin = met[0], amax = met[0];
  for (size_t q = 0; q < met.size(); q += 4) {
    amin = std::min(amin, met[q]);
    amax = std::max(amax, met[q]);
  }
  return wm_host_mass_bounds_metric(g->d, nu, nv, amin, amax, lo, hi);
}

extern "C" int wm_geom_metric(wm_geom_t g, int level, double* out, int64_t cap) {
  WM_TRY(check_geom_level(g, level, 0));
  if (!wm_is_nurbs(g->d.kind)) {
    wm_set_error("the metric of the analytic kinds is computed on the GPU (wm_metric)");
    return WM_ERR_UNSUPPORTED;
  }
  std::vector<double> met;
  WM_TRY(geom_nurbs_metric(g, level, met));
  if (!out || cap < (int64_t)met.size()) {
    wm_set_error("output buffer too small");
    return WM_ERR_INVALID_ARG;
  }
  std::memcpy(out, met.data(), met.size() * sizeof(double));
  return WM_OK;
}

extern "C" int wm_geom_prolongation(wm_geom_t g, int level, int32_t* row_ptr, int32_t* col, double* val,
                                    int64_t nnz_cap) {
  std::vector<int32_t> Pp, Pc;
  std::vector<double> Pv;
  WM_TRY(geom_prolongation(g, level, Pp, Pc, Pv));
  if (!row_ptr || !col || !val || nnz_cap < (int64_t)Pc.size()) {
    wm_set_error("output buffers too small");
    return WM_ERR_INVALID_ARG;
  }
  std::memcpy(row_ptr, Pp.data(), Pp.size() * sizeof(int32_t));
  std::memcpy(col, Pc.data(), Pc.size() * sizeof(int32_t));
  std::memcpy(val, Pv.data(), Pv.size() * sizeof(double));
  return WM_OK;
}

extern "C" int wm_metric(wm_hier_t h, int level, double* out, void* stream) {
  WM_TRY(check_level(h, level));
  if (!out) return WM_ERR_INVALID_ARG;
  const wm_level& L = h->lv[level];
  WM_CUDA(cudaMemcpyAsync(out, L.d_metric.p, sizeof(double) * L.d_metric.n, cudaMemcpyDeviceToDevice,
                          as_stream(stream)));
  return WM_OK;
}

// ------------------------------------------------------------------ operators
extern "C" int wm_apply_shifted(wm_hier_t h, int level, int n_vec, const double* sigma, const double* x, double* y,
                                int precision, void* stream) {
  WM_TRY(check_level(h, level));
  if (n_vec < 0 || (n_vec > 0 && (!sigma || !x || !y))) return WM_ERR_INVALID_ARG;
  if (precision != WM_FP64 && precision != WM_MIXED) return WM_ERR_INVALID_ARG;
  if (n_vec == 0) return WM_OK;
  cudaStream_t s = as_stream(stream);
  const wm_level& L = h->lv[level];
  int tiles = (n_vec + WM_LANES - 1) / WM_LANES;
  size_t n = (size_t)tiles * L.N * WM_LANES;
  Tmp t;
  WM_TRY(t.a.alloc(n));
  WM_TRY(t.b.alloc(n));
  std::vector<double> sg((size_t)tiles * WM_LANES, 0.0);
  std::copy(sigma, sigma + n_vec, sg.begin());
  WM_TRY(t.sg.upload(sg, s));
  WM_TRY(wm_k_to_tiled(x, n_vec, L.N, t.a.p, tiles, s));
  if (precision == WM_FP64) {
    WM_TRY(wm_k_apply<double>(L, tiles, t.sg.p, t.a.p, t.b.p, nullptr, s));
  } else {
    WM_TRY(t.fa.alloc(n));
    WM_TRY(t.fb.alloc(n));
    WM_TRY(wm_convert_f32(t.a.p, t.fa.p, n, s));
    WM_TRY(wm_k_apply<float>(L, tiles, t.sg.p, t.fa.p, t.fb.p, nullptr, s));
    WM_TRY(wm_widen_f32(t.fb.p, t.b.p, n, s));
  }
  WM_TRY(wm_k_from_tiled(t.b.p, tiles, L.N, y, n_vec, s));
  WM_CUDA(cudaStreamSynchronize(s));
  return WM_OK;
}

extern "C" int wm_apply_mass(wm_hier_t h, int level, const double* x, double* y, int n_vec, void* stream) {
  WM_TRY(check_level(h, level));
  if (n_vec < 0 || (n_vec > 0 && (!x || !y))) return WM_ERR_INVALID_ARG;
  if (n_vec == 0) return WM_OK;
  cudaStream_t s = as_stream(stream);
  const wm_level& L = h->lv[level];
  int tiles = (n_vec + WM_LANES - 1) / WM_LANES;
  size_t n = (size_t)tiles * L.N * WM_LANES;
  Tmp t;
  WM_TRY(t.a.alloc(n));
  WM_TRY(t.b.alloc(n));
  WM_TRY(wm_k_to_tiled(x, n_vec, L.N, t.a.p, tiles, s));
  WM_TRY(wm_k_apply_mass64(L, tiles, t.a.p, t.b.p, nullptr, s));
  WM_TRY(wm_k_from_tiled(t.b.p, tiles, L.N, y, n_vec, s));
  WM_CUDA(cudaStreamSynchronize(s));
  return WM_OK;
}

static int transfer(wm_hier_t h, int level, const double* in, double* out, int n_vec, bool prolong, void* stream) {
  WM_TRY(check_level(h, level));
  if (level + 1 >= (int)h->lv.size()) return WM_ERR_INVALID_ARG;
  if (n_vec < 0 || (n_vec > 0 && (!in || !out))) return WM_ERR_INVALID_ARG;
  if (n_vec == 0) return WM_OK;
  cudaStream_t s = as_stream(stream);
  const wm_level& F = h->lv[level];
  const wm_level& C = h->lv[level + 1];
  int tiles = (n_vec + WM_LANES - 1) / WM_LANES;
  Tmp t;
  WM_TRY(t.a.alloc((size_t)tiles * std::max(F.N, C.N) * WM_LANES));
  WM_TRY(t.b.alloc((size_t)tiles * std::max(F.N, C.N) * WM_LANES));
  if (prolong) {
    WM_TRY(wm_k_to_tiled(in, n_vec, C.N, t.a.p, tiles, s));
    WM_CUDA(cudaMemsetAsync(t.b.p, 0, sizeof(double) * (size_t)tiles * F.N * WM_LANES, s));
    WM_TRY(wm_k_prolong_add<double>(F, tiles, t.a.p, t.b.p, nullptr, s));
    WM_TRY(wm_k_from_tiled(t.b.p, tiles, F.N, out, n_vec, s));
  } else {
    WM_TRY(wm_k_to_tiled(in, n_vec, F.N, t.a.p, tiles, s));
    WM_TRY(wm_k_restrict<double>(F, tiles, t.a.p, t.b.p, nullptr, s));
    WM_TRY(wm_k_from_tiled(t.b.p, tiles, C.N, out, n_vec, s));
  }
  WM_CUDA(cudaStreamSynchronize(s));
  return WM_OK;
}

extern "C" int wm_prolongate(wm_hier_t h, int level, const double* xc, double* xf, int n_vec, void* stream) {
  return transfer(h, level, xc, xf, n_vec, true, stream);
}

extern "C" int wm_restrict(wm_hier_t h, int level, const double* rf, double* rc, int n_vec, void* stream) {
  return transfer(h, level, rf, rc, n_vec, false, stream);
}

static int set_batch_meta(WorkSpace& ws, const wm_schedule& sc, int tiles, const std::vector<double>& sigma,
                          const std::vector<int>& sid, const std::vector<int>& src, cudaStream_t s) {
  size_t n = (size_t)tiles * WM_LANES;
  std::vector<double> sg(n, sigma.empty() ? 1.0 : sigma[0]);
  std::vector<int> si(n, 0), sr(n, -1);
  for (size_t g = 0; g < n; ++g) {
    if (g < sigma.size()) {
      sg[g] = sigma[g];
      si[g] = sid[g];
      sr[g] = src[g];
    } else if (g > 0) {  // padding systems (zero right-hand side) copy the last real shift
      sg[g] = sg[g - 1];
      si[g] = si[g - 1];
    }
  }
  // tiles whose 32 shifts are equal (bit for bit) take the combined-coefficient kernels
  std::vector<int> uni(tiles, 1);
  int n_uni = 0;
  for (int t = 0; t < tiles; ++t) {
    for (int l = 1; l < WM_LANES; ++l)
      if (std::memcmp(&sg[(size_t)t * WM_LANES + l], &sg[(size_t)t * WM_LANES], sizeof(double)) != 0) {
        uni[t] = 0;
        break;
      }
    n_uni += uni[t];
  }
  ws.n_uni_tiles = n_uni;
  // groups of at most kUniGroup consecutive one-shift tiles with the same shift
  // index (one block of the one-shift kernel per group and spatial block)
  std::vector<int2> grp;
  for (int t = 0; t < tiles; ++t) {
    if (!uni[t]) continue;
    const int st = si[(size_t)t * WM_LANES];
    if (!grp.empty()) {
      int2& last = grp.back();
      const int lt = last.x + last.y;  // tile after the last group
      if (lt == t && last.y < std::min(kUniGroup, sc.uni_run) && si[(size_t)last.x * WM_LANES] == st) {
        last.y += 1;
        continue;
      }
    }
    grp.push_back(make_int2(t, 1));
  }
  ws.n_uni_groups = (int)grp.size();
  ws.uni_waves = sc.uni_waves;
  if (!grp.empty()) {
    WM_TRY(ws.uni_groups.alloc(grp.size()));
    WM_CUDA(cudaMemcpyAsync(ws.uni_groups.p, grp.data(), grp.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
  }
  WM_CUDA(cudaMemcpyAsync(ws.sigma.p, sg.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  WM_CUDA(cudaMemcpyAsync(ws.sid.p, si.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  WM_CUDA(cudaMemcpyAsync(ws.src_of.p, sr.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  WM_CUDA(cudaMemcpyAsync(ws.tile_uni.p, uni.data(), tiles * sizeof(int), cudaMemcpyHostToDevice, s));
  WM_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
  return WM_OK;
}

extern "C" int wm_vcycle(wm_hier_t h, int n_vec, const double* sigma, const double* r, double* z, int precision,
                         int smoother_degree, double cheb_ratio, void* stream) {
  if (!h || n_vec < 0 || (n_vec > 0 && (!sigma || !r || !z))) return WM_ERR_INVALID_ARG;
  if (precision != WM_FP64 && precision != WM_MIXED) return WM_ERR_INVALID_ARG;
  if (smoother_degree < 1 || smoother_degree > 8 || !(cheb_ratio > 1.0)) return WM_ERR_INVALID_ARG;
  if (h->lv.back().N > 160) {
    wm_set_error("coarsest level too large for the dense coarse solve");
    return WM_ERR_UNSUPPORTED;
  }
  if (n_vec == 0) return WM_OK;
  cudaStream_t s = as_stream(stream);
  WorkSpace& ws = workspace(h);
  int tiles = (n_vec + WM_LANES - 1) / WM_LANES;
  WM_TRY(ws.reserve(h, tiles, n_vec, precision == WM_FP64));
  std::vector<double> sg(sigma, sigma + n_vec);
  // systems with the same shift (bit for bit) share its index: one coarse
  // inverse and one smoother bound per distinct shift
  std::vector<double> shl;
  std::vector<int> sid(n_vec), src(n_vec);
  {
    std::map<uint64_t, int> index;
    for (int g = 0; g < n_vec; ++g) {
      uint64_t key;
      std::memcpy(&key, &sg[g], sizeof(key));
      auto it = index.find(key);
      if (it == index.end()) {
        it = index.emplace(key, (int)shl.size()).first;
        shl.push_back(sg[g]);
      }
      sid[g] = it->second;
      src[g] = g;
    }
  }
  WM_TRY(set_batch_meta(ws, h->sched, tiles, sg, sid, src, s));
  WM_TRY(wm_prepare_shifts(h, ws, shl, s));
  Batch bt;
  bt.schedule(h->sched);
  bt.tiles = tiles;
  bt.nsys = n_vec;
  bt.nshift = (int)shl.size();
  bt.precision = precision;
  bt.degree = smoother_degree;
  bt.cheb_ratio = cheb_ratio;
  WM_TRY(wm_k_to_tiled(r, n_vec, h->lv[0].N, ws.x.p, tiles, s));
  WM_TRY(wm_vcycle_apply(h, ws, bt, ws.x.p, ws.x.p, s));
  WM_TRY(wm_k_from_tiled(ws.x.p, tiles, h->lv[0].N, z, n_vec, s));
  WM_CUDA(cudaStreamSynchronize(s));
  return WM_OK;
}

// ------------------------------------------------------------------ noise
extern "C" int wm_philox4x32_10(const uint32_t* ctr, uint64_t key, uint32_t* out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return WM_ERR_INVALID_ARG;
  WM_TRY(wm_k_philox(ctr, key, out, n, as_stream(stream)));
  WM_CUDA(cudaStreamSynchronize(as_stream(stream)));
  return WM_OK;
}

extern "C" int wm_normals(uint64_t seed, int sample, int stream_id, int64_t q0, int64_t n, double* out,
                          void* stream) {
  if (n < 0 || q0 < 0 || sample < 0 || (n > 0 && !out)) return WM_ERR_INVALID_ARG;
  WM_TRY(wm_k_normals(seed, sample, stream_id, q0, n, out, as_stream(stream)));
  WM_CUDA(cudaStreamSynchronize(as_stream(stream)));
  return WM_OK;
}

// loads of samples sample0 + [0, ns) into rows row0 + [0, ns) of the sample-tiled buffer b_t
static int draw_loads(wm_hier_t h, WorkSpace& ws, uint64_t seed, int sample0, int ns, double* b_t, cudaStream_t s,
                      int row0 = 0) {
  const wm_level& L = h->lv[0];
  // sample chunks bounded so that the element scratch stays below ~1 GiB
  size_t per_sample = (size_t)L.E * L.nk;
  int chunk = (int)std::max<size_t>(1, std::min<size_t>(ns, (size_t)(1u << 27) / per_sample));
  WM_TRY(ws.noise_scratch.alloc(per_sample * chunk));
  for (int s0 = 0; s0 < ns; s0 += chunk) {
    int c = std::min(chunk, ns - s0);
    WM_TRY(wm_k_noise_tiled(h, seed, sample0 + s0, row0 + s0, c, b_t, ws.noise_scratch.p, s));
  }
  return WM_OK;
}

extern "C" int wm_noise_loads(wm_hier_t h, uint64_t seed, int n_samples, double* b, void* stream) {
  if (!h || n_samples < 0 || (n_samples > 0 && !b)) return WM_ERR_INVALID_ARG;
  if (n_samples == 0) return WM_OK;
  cudaStream_t s = as_stream(stream);
  WorkSpace& ws = workspace(h);
  int stiles = (n_samples + WM_LANES - 1) / WM_LANES;
  WM_TRY(ws.samp[0].alloc((size_t)stiles * h->lv[0].N * WM_LANES));
  WM_TRY(draw_loads(h, ws, seed, 0, n_samples, ws.samp[0].p, s));
  WM_TRY(wm_k_from_tiled(ws.samp[0].p, stiles, h->lv[0].N, b, n_samples, s));
  WM_CUDA(cudaStreamSynchronize(s));
  return WM_OK;
}

// ------------------------------------------------------------------ sampler
namespace {

struct Plan {
  int n_int = 0, passes = 0;
  double bp = 0.0;
  std::vector<double> c, sigma;  // per node
};

int make_plan(const wm_sample_desc* d, Plan& P) {
  if (!(d->kappa > 0) || !std::isfinite(d->kappa)) return WM_ERR_INVALID_ARG;
  WM_TRY(wm_split_beta(d->beta, d->split, &P.n_int, &P.bp, &P.passes));
  if (P.passes > 0) {
    if (!(d->sinc_k > 0) || d->l_lo > d->l_hi) return WM_ERR_INVALID_ARG;
    double pre = std::sin(M_PI * P.bp) / M_PI * d->sinc_k;
    for (int l = d->l_lo; l <= d->l_hi; ++l) {
      double y = l * d->sinc_k;
      P.c.push_back(pre * std::exp((1.0 - P.bp) * y));
      P.sigma.push_back(std::exp(y) + d->kappa * d->kappa);
    }
  }
  return WM_OK;
}

int validate_desc(wm_hier_t h, const wm_sample_desc* d) {
  if (!h || !d) return WM_ERR_INVALID_ARG;
  if (d->n_samples < 0 || d->max_iter < 1 || !(d->rtol > 0) || d->smoother_degree < 1 ||
      d->smoother_degree > 8 || d->smoother_degree_coarse < 0 || d->smoother_degree_coarse > 8 || !(d->cheb_ratio > 1.0) || d->max_systems < 0 || d->sample0 < 0 ||
      (int64_t)d->sample0 + d->n_samples > (int64_t)INT32_MAX) {
    wm_set_error("invalid sample descriptor");
    return WM_ERR_INVALID_ARG;
  }
  if (d->precision != WM_FP64 && d->precision != WM_MIXED) return WM_ERR_INVALID_ARG;
  if (d->noise_mode != WM_NOISE_DRAW && d->noise_mode != WM_NOISE_GIVEN) return WM_ERR_INVALID_ARG;
  if (d->ckpt != WM_CKPT_RECOMPUTE && d->ckpt != WM_CKPT_KEEP) {
    wm_set_error("unknown checkpoint policy %d", d->ckpt);
    return WM_ERR_INVALID_ARG;
  }
  if (d->preconditioner != WM_PRECOND_VCYCLE && d->preconditioner != WM_PRECOND_BPX) {
    wm_set_error("unknown preconditioner %d", d->preconditioner);
    return WM_ERR_INVALID_ARG;
  }
  if (h->lv.back().N > 160) {
    wm_set_error("coarsest level has %d DOFs (> 160): use more levels", h->lv.back().N);
    return WM_ERR_UNSUPPORTED;
  }
  return WM_OK;
}

// All systems of one pass: g = j * ns + s with shift sigma[j], right-hand side
// rhs_t (sample-tiled).  x of every batch goes to `sink`.
struct Pass {
  std::vector<double> sigma;  // per node j
  int ns = 0;
  int sid_base = 0;           // index of node 0's shift in the call's shift list
  int nshift_total = 0;       // length of the call's shift list
};

// The call's shift list: the fractional shifts sigma_l (index j), then
// kappa^2 of the integer part (index n_nodes) when there is one.  Smoother
// bounds and coarse inverses are prepared once for the whole list.
std::vector<double> call_shifts(const Plan& P, double kappa) {
  std::vector<double> all = P.sigma;
  if (P.n_int > 0) all.push_back(kappa * kappa);
  return all;
}

// systems per batched solve: the caller's cap, else what fits 80% of free
// memory (plus what the workspace already holds); extra_bytes per DOF-system
// for callers that keep more per-system vectors (the adjoint)
int64_t batch_size(wm_hier_t h, WorkSpace& ws, const wm_sample_desc* d, int64_t nsys, size_t extra_bytes) {
  bool dbl = d->precision == WM_FP64;
  size_t per = bytes_per_system(h, dbl) + extra_bytes * (size_t)h->lv[0].N;
  int64_t maxsys = d->max_systems > 0 ? d->max_systems : 0;
  if (maxsys == 0) {
    size_t freeb = 0, totb = 0;
    if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) {
      cudaGetLastError();
      freeb = 0;
    }
    size_t have = ws.x.n / std::max(1, h->lv[0].N);  // systems the workspace already holds
    // 80% of what this workspace could reach (free memory plus what it holds),
    // so that repeated calls do not ratchet the workspace up to all of the memory
    size_t budget = (size_t)((double)(freeb + have * per) * 0.8);
    maxsys = std::max<int64_t>(WM_LANES, (int64_t)(budget / per) / WM_LANES * WM_LANES);
  }
  int64_t per_batch = std::min<int64_t>(nsys, maxsys);
  if (per_batch > WM_LANES) per_batch = per_batch / WM_LANES * WM_LANES;
  return std::max<int64_t>(1, per_batch);
}

// one batched solve of the systems [g0, g1) of a pass (g = j * ns + s); the
// solutions are left in ws.x
int solve_range(wm_hier_t h, WorkSpace& ws, const wm_sample_desc* d, const Pass& ps, int64_t g0, int64_t g1,
                const double* rhs_t, wm_stats* st, int* worst, cudaStream_t s) {
  bool dbl = d->precision == WM_FP64;
  int nj = (int)ps.sigma.size();
  int nb = (int)(g1 - g0);
  int tiles = (nb + WM_LANES - 1) / WM_LANES;
  std::vector<double> sg(nb);
  std::vector<int> sid(nb), src(nb);
  for (int k = 0; k < nb; ++k) {
    int64_t g = g0 + k;
    int j = (int)(g / ps.ns);
    sg[k] = ps.sigma[j];
    sid[k] = ps.sid_base + j;
    src[k] = (int)(g % ps.ns);
  }
  WM_TRY(set_batch_meta(ws, h->sched, tiles, sg, sid, src, s));
  Batch bt;
  bt.schedule(h->sched);
  bt.tiles = tiles;
  bt.nsys = nb;
  bt.nshift = ps.nshift_total;
  bt.precision = d->precision;
  bt.rtol = d->rtol;
  bt.max_iter = d->max_iter;
  bt.degree = d->smoother_degree;
  bt.degree_coarse = d->smoother_degree_coarse;
  bt.cheb_ratio = d->cheb_ratio;
  bt.replace_drop = dbl ? 0.0 : 1e-4;
  bt.df_residual = !dbl;
  bt.precond = d->preconditioner;
  BatchResult br;
  WM_TRY(wm_solve_batch(h, ws, bt, rhs_t, &br, s));
  if (br.flags & 1) *worst = std::min(*worst, WM_ERR_NONFINITE);
  if ((br.n_not_converged > 0 || (br.flags & 2)) && *worst == WM_OK) *worst = WM_ERR_NOT_CONVERGED;
  if (st) {
    st->n_systems += nb;
    st->n_batches += 1;
    st->max_iterations = std::max(st->max_iterations, br.iterations);
    st->total_iterations += br.iterations;
    st->n_not_converged += br.n_not_converged;
    st->max_rel_residual = std::max(st->max_rel_residual, br.max_rel_residual);
    st->n_replacements += br.replacements;
    st->n_df_fallbacks += br.df_fallbacks;
  }
  return WM_OK;
}

template <typename Sink>
int run_pass(wm_hier_t h, WorkSpace& ws, const wm_sample_desc* d, const Pass& ps, const double* rhs_t,
             wm_stats* st, int* worst, Sink sink, cudaStream_t s) {
  int nj = (int)ps.sigma.size();
  int64_t nsys = (int64_t)nj * ps.ns;
  (void)nj;
  int64_t per_batch = batch_size(h, ws, d, nsys, 0);
  WM_TRY(ws.reserve(h, (int)((per_batch + WM_LANES - 1) / WM_LANES), ps.nshift_total, d->precision == WM_FP64));
  for (int64_t g0 = 0; g0 < nsys; g0 += per_batch) {
    int64_t g1 = std::min(nsys, g0 + per_batch);
    WM_TRY(solve_range(h, ws, d, ps, g0, g1, rhs_t, st, worst, s));
    WM_TRY(sink((int)g0, (int)g1, s));
  }
  return WM_OK;
}

}  // namespace

// Sample-tiled buffers: samp[0] loads, samp[1] current iterate, samp[2]
// accumulator, samp[3] pass right-hand side, samp[4] staging of host outputs.

namespace {

// descriptor fields that decide the forward solutions (the loads are compared
// separately, bit for bit)
bool same_solutions(const wm_sample_desc& a, const wm_sample_desc& b) {
  return a.kappa == b.kappa && a.beta == b.beta && a.split == b.split && a.sinc_k == b.sinc_k && a.l_lo == b.l_lo &&
         a.l_hi == b.l_hi && a.n_samples == b.n_samples && a.sample0 == b.sample0 && a.precision == b.precision &&
         a.rtol == b.rtol && a.max_iter == b.max_iter && a.smoother_degree == b.smoother_degree &&
         a.smoother_degree_coarse == b.smoother_degree_coarse && a.cheb_ratio == b.cheb_ratio &&
         a.max_systems == b.max_systems && a.preconditioner == b.preconditioner;
}

__global__ void k_count_diff(size_t n, const double* __restrict__ a, const double* __restrict__ b, int* cnt) {
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k < n && __double_as_longlong(a[k]) != __double_as_longlong(b[k])) atomicAdd(cnt, 1);
}

// true when the n doubles of a and b are identical bit for bit
int equal_bits(WorkSpace& ws, const double* a, const double* b, size_t n, bool* eq, cudaStream_t s) {
  int* cnt = ws.counters.p + 7;
  WM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
  WM_LAUNCH(WM_PC_SINC, s, k_count_diff<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, b, cnt));
  WM_CUDA(cudaGetLastError());
  WM_CUDA(cudaMemcpyAsync(ws.host_small + 12, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
  WM_CUDA(cudaStreamSynchronize(s));
  *eq = ws.host_small[12] == 0;
  return WM_OK;
}

// whether `bytes` more may be kept: at most half of the free device memory
bool may_keep(size_t bytes) {
  size_t freeb = 0, totb = 0;
  if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return bytes <= freeb / 2;
}

// the fractional pass of a plan: all nodes x samples
Pass frac_pass(const Plan& P, int ns, int nshift_total) {
  Pass fp;
  fp.sigma = P.sigma;
  fp.ns = ns;
  fp.sid_base = 0;
  fp.nshift_total = nshift_total;
  return fp;
}

size_t pass_tiles(const Plan& P, int ns) { return ((size_t)P.sigma.size() * ns + WM_LANES - 1) / WM_LANES; }

}  // namespace

static int sample_fields_impl(wm_hier_t h, const wm_sample_desc* d, double* u, double* b, wm_stats* st,
                              cudaStream_t s) {
  WM_TRY(validate_desc(h, d));
  Plan P;
  WM_TRY(make_plan(d, P));
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->n_int_solves = P.n_int;
    st->n_frac_passes = P.passes;
    st->n_nodes = (int)P.c.size();
  }
  int ns = d->n_samples;
  if (ns == 0) return WM_OK;
  if (!u) return WM_ERR_INVALID_ARG;
  if (d->noise_mode == WM_NOISE_GIVEN && !b) return WM_ERR_INVALID_ARG;
  const wm_level& L0 = h->lv[0];
  int N = L0.N;
  int stiles = (ns + WM_LANES - 1) / WM_LANES;
  size_t sn = (size_t)stiles * N * WM_LANES;
  WorkSpace& ws = workspace(h);
  for (int k = 0; k < 4; ++k) WM_TRY(ws.samp[k].alloc(sn));
  double* b_t = ws.samp[0].p;
  double* cur = ws.samp[1].p;
  double* acc = ws.samp[2].p;
  double* rhs = ws.samp[3].p;
  bool u_dev = is_device_ptr(u);
  bool b_dev = b ? is_device_ptr(b) : true;
  if ((!u_dev || !b_dev)) WM_TRY(ws.samp[4].alloc((size_t)ns * N));
  // loads
  if (d->noise_mode == WM_NOISE_DRAW) {
    WM_TRY(draw_loads(h, ws, d->seed, d->sample0, ns, b_t, s));
    if (b) {
      if (b_dev) {
        WM_TRY(wm_k_from_tiled(b_t, stiles, N, b, ns, s));
      } else {
        WM_TRY(wm_k_from_tiled(b_t, stiles, N, ws.samp[4].p, ns, s));
        WM_CUDA(cudaMemcpyAsync(b, ws.samp[4].p, sizeof(double) * ns * N, cudaMemcpyDeviceToHost, s));
      }
    }
  } else {
    const double* src = b;
    if (!b_dev) {
      WM_CUDA(cudaMemcpyAsync(ws.samp[4].p, b, sizeof(double) * ns * N, cudaMemcpyHostToDevice, s));
      src = ws.samp[4].p;
    }
    WM_TRY(wm_k_to_tiled(src, ns, N, b_t, stiles, s));
  }
  int worst = WM_OK;
  const std::vector<double> shifts = call_shifts(P, d->kappa);
  {
    int64_t most = (int64_t)std::max<size_t>(1, P.sigma.size()) * ns;
    int64_t per_batch = batch_size(h, ws, d, most, 0);
    WM_TRY(ws.reserve(h, (int)((per_batch + WM_LANES - 1) / WM_LANES), (int)shifts.size(),
                      d->precision == WM_FP64));
    WM_TRY(wm_prepare_shifts(h, ws, shifts, s));
  }
  // checkpoint for the backward: loads, integer iterates, pass right-hand sides
  // and every pass's solutions, when asked for and when they fit
  WorkSpace::Ckpt& ck = ws.ck;
  bool keep = false;
  if (d->ckpt == WM_CKPT_KEEP) {
    ck.release();
    const size_t xt = pass_tiles(P, ns) * N * WM_LANES;
    const size_t bytes = sizeof(double) * (sn * (1 + P.n_int + P.passes) + xt * P.passes);
    keep = may_keep(bytes);
    if (keep) {
      WM_TRY(ck.b.alloc(sn));
      WM_TRY(wm_copy(b_t, ck.b.p, sn, s));
      ck.w.resize(P.n_int);
      for (int i = 0; i < P.n_int; ++i) WM_TRY(ck.w[i].alloc(sn));
      for (int p = 0; p < P.passes; ++p) {
        WM_TRY(ck.r[p].alloc(sn));
        WM_TRY(ck.x[p].alloc(xt));
      }
    }
  }
  // integer part: (S + kappa^2 M) w_1 = b, (S + kappa^2 M) w_i = M w_{i-1}
  Pass ip;
  ip.sigma = {d->kappa * d->kappa};
  ip.ns = ns;
  ip.sid_base = (int)P.sigma.size();
  ip.nshift_total = (int)shifts.size();
  for (int i = 0; i < P.n_int; ++i) {
    const double* r = b_t;
    if (i > 0) {
      WM_TRY(wm_k_apply_mass64(L0, stiles, cur, rhs, nullptr, s));
      r = rhs;
    }
    auto sink = [&](int g0, int g1, cudaStream_t ss) -> int {
      // systems g = s: the batch [g0, g1) is tile-aligned with the sample tiles
      size_t off = (size_t)(g0 / WM_LANES) * N * WM_LANES;
      size_t n = (size_t)((g1 - g0 + WM_LANES - 1) / WM_LANES) * N * WM_LANES;
      return wm_copy(ws.x.p, cur + off, n, ss);
    };
    WM_TRY(run_pass(h, ws, d, ip, r, st, &worst, sink, s));
    if (keep) WM_TRY(wm_copy(cur, ck.w[i].p, sn, s));
  }
  // fractional passes
  if (P.passes > 0) {
    WM_TRY(ws.coef.upload(P.c, s));
    const Pass fp = frac_pass(P, ns, (int)shifts.size());
    for (int pass = 0; pass < P.passes; ++pass) {
      const double* r = b_t;
      if (P.n_int > 0 || pass > 0) {
        WM_TRY(wm_k_apply_mass64(L0, stiles, cur, rhs, nullptr, s));
        r = rhs;
      }
      if (keep) WM_TRY(wm_copy(r, ck.r[pass].p, sn, s));
      WM_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * sn, s));
      double* xk = keep ? ck.x[pass].p : nullptr;
      auto sink = [&](int g0, int g1, cudaStream_t ss) -> int {
        if (xk) {
          size_t off = (size_t)(g0 / WM_LANES) * N * WM_LANES;
          size_t n = (size_t)((g1 - g0 + WM_LANES - 1) / WM_LANES) * N * WM_LANES;
          WM_TRY(wm_copy(ws.x.p, xk + off, n, ss));
        }
        return wm_sinc_accumulate(h, ns, g0, g1, ws.coef.p, ws.x.p, acc, ss);
      };
      WM_TRY(run_pass(h, ws, d, fp, r, st, &worst, sink, s));
      std::swap(cur, acc);
    }
  }
  if (keep) {
    ck.desc = *d;
    ck.valid = true;
    if (st) st->ckpt_kept = 1;
  }
  // fields
  if (u_dev) {
    WM_TRY(wm_k_from_tiled(cur, stiles, N, u, ns, s));
  } else {
    WM_TRY(wm_k_from_tiled(cur, stiles, N, ws.samp[4].p, ns, s));
    WM_CUDA(cudaMemcpyAsync(u, ws.samp[4].p, sizeof(double) * ns * N, cudaMemcpyDeviceToHost, s));
  }
  WM_CUDA(cudaStreamSynchronize(s));
  // keep the buffer roles stable for the next call
  if (cur != ws.samp[1].p) std::swap(ws.samp[1].p, ws.samp[2].p);
  return worst;
}

extern "C" int wm_sample_fields(wm_hier_t h, const wm_sample_desc* d, double* u, double* b, wm_stats* st,
                                void* stream) {
  return sample_fields_impl(h, d, u, b, st, as_stream(stream));
}

namespace {

// rows [row0, row0 + n) of a sample-tiled buffer to [n][N] (caller layout)
__global__ void k_rows_from_tiled(const double* __restrict__ src, int N, int row0, int n, double* __restrict__ dst) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)n * N) return;
  int v = (int)(k / N), i = (int)(k - (int64_t)v * N);
  int r = row0 + v;
  dst[k] = src[((size_t)(r / WM_LANES) * N + i) * WM_LANES + (r % WM_LANES)];
}

// rows of a sample-tiled buffer whose flag is set become zero
__global__ void k_zero_rows(int N, const int* __restrict__ flag, double* __restrict__ v) {
  int st = blockIdx.y;
  int r = st * WM_LANES + threadIdx.x;
  if (!flag[r]) return;
  for (int i = blockIdx.x * blockDim.y + threadIdx.y; i < N; i += gridDim.x * blockDim.y)
    v[((size_t)st * N + i) * WM_LANES + threadIdx.x] = 0.0;
}

// acc[row r] += sum over the entries e of row r (CSR ptr over rows) of
// coef[e] x[system sys[e]], systems of the batch stored [tiles][N][32]; the
// entries of a row are summed in order (deterministic)
__global__ void k_rows_accumulate(int N, const int* __restrict__ ptr, const int* __restrict__ sys,
                                  const double* __restrict__ coef, const double* __restrict__ x,
                                  double* __restrict__ acc) {
  int st = blockIdx.y;
  int r = st * WM_LANES + threadIdx.x;
  int e0 = ptr[r], e1 = ptr[r + 1];
  if (e0 == e1) return;
  for (int i = blockIdx.x * blockDim.y + threadIdx.y; i < N; i += gridDim.x * blockDim.y) {
    double a = 0.0;
    for (int e = e0; e < e1; ++e) {
      int g = sys[e];
      a += coef[e] * x[((size_t)(g / WM_LANES) * N + i) * WM_LANES + (g % WM_LANES)];
    }
    acc[((size_t)st * N + i) * WM_LANES + threadIdx.x] += a;
  }
}

// solver settings that instances must share to be packed into one batch
bool same_solver(const wm_sample_desc& a, const wm_sample_desc& b) {
  return a.precision == b.precision && a.rtol == b.rtol && a.max_iter == b.max_iter &&
         a.smoother_degree == b.smoother_degree && a.smoother_degree_coarse == b.smoother_degree_coarse &&
         a.cheb_ratio == b.cheb_ratio &&
         a.preconditioner == b.preconditioner && a.max_systems == b.max_systems;
}

// Instances of one hierarchy with the same solver settings, solved together.
// Their samples are rows off_i .. off_i + n_i - 1 of shared sample-tiled
// buffers.  Stage k of an instance is its k-th integer solve or, after those,
// its fractional passes; every stage but the first takes M times the previous
// stage's result, the first takes the loads.  Stage k of all instances that
// have one is a single list of systems (the instances' shifts and weights side
// by side), solved in batches by the batched PCG; each batch's solutions are
// summed into the rows of their samples with their weights (1 for an integer
// solve).
int sample_fields_group(wm_hier_t h, const std::vector<const wm_sample_desc*>& D, const std::vector<double*>& U,
                        const std::vector<wm_stats*>& ST, cudaStream_t s) {
  const int m = (int)D.size();
  std::vector<Plan> P(m);
  std::vector<int> off(m + 1, 0);
  for (int i = 0; i < m; ++i) {
    WM_TRY(validate_desc(h, D[i]));
    if (D[i]->noise_mode != WM_NOISE_DRAW) {
      wm_set_error("wm_sample_fields_batched draws the loads (WM_NOISE_DRAW)");
      return WM_ERR_INVALID_ARG;
    }
    WM_TRY(make_plan(D[i], P[i]));
    if (ST[i]) {
      std::memset(ST[i], 0, sizeof(*ST[i]));
      ST[i]->n_int_solves = P[i].n_int;
      ST[i]->n_frac_passes = P[i].passes;
      ST[i]->n_nodes = (int)P[i].c.size();
    }
    if (D[i]->n_samples > 0 && (!U[i] || !is_device_ptr(U[i]))) {
      wm_set_error("wm_sample_fields_batched: u[%d] must be device memory", i);
      return WM_ERR_INVALID_ARG;
    }
    off[i + 1] = off[i] + D[i]->n_samples;
  }
  const int S = off[m];
  if (S == 0) return WM_OK;
  const wm_level& L0 = h->lv[0];
  const int N = L0.N;
  const int stiles = (S + WM_LANES - 1) / WM_LANES;
  const size_t sn = (size_t)stiles * N * WM_LANES;
  WorkSpace& ws = workspace(h);
  for (int k = 0; k < 3; ++k) WM_TRY(ws.samp[k].alloc(sn));
  double* b_t = ws.samp[0].p;
  double* cur = ws.samp[1].p;
  double* rhs = ws.samp[2].p;
  for (int i = 0; i < m; ++i)
    if (D[i]->n_samples > 0) WM_TRY(draw_loads(h, ws, D[i]->seed, D[i]->sample0, D[i]->n_samples, b_t, s, off[i]));
  // the call's shift list: every distinct shift of every instance
  std::vector<double> shl;
  std::map<uint64_t, int> index;
  auto shift_id = [&](double v) {
    uint64_t key;
    std::memcpy(&key, &v, sizeof(key));
    auto it = index.find(key);
    if (it == index.end()) {
      it = index.emplace(key, (int)shl.size()).first;
      shl.push_back(v);
    }
    return it->second;
  };
  std::vector<std::vector<int>> node_sid(m);
  std::vector<int> kappa_sid(m);
  int K = 0;
  for (int i = 0; i < m; ++i) {
    for (double v : P[i].sigma) node_sid[i].push_back(shift_id(v));
    kappa_sid[i] = shift_id(D[i]->kappa * D[i]->kappa);
    if (D[i]->n_samples > 0) K = std::max(K, P[i].n_int + P[i].passes);
  }
  const wm_sample_desc& d0 = *D[0];
  int64_t most = 0;
  for (int i = 0; i < m; ++i) most += (int64_t)std::max<size_t>(1, P[i].sigma.size()) * D[i]->n_samples;
  const int64_t per_batch = batch_size(h, ws, &d0, most, 0);
  WM_TRY(ws.reserve(h, (int)((per_batch + WM_LANES - 1) / WM_LANES), (int)shl.size(), d0.precision == WM_FP64));
  WM_TRY(wm_prepare_shifts(h, ws, shl, s));
  // per-call row flags and accumulation lists, released on every return
  struct GroupBufs {
    DevBuf<int> flag, ptr, sys;
    DevBuf<double> coef;
    ~GroupBufs() {
      flag.release();
      ptr.release();
      sys.release();
      coef.release();
    }
  } gb;
  DevBuf<int>& d_flag = gb.flag;
  DevBuf<int>& d_ptr = gb.ptr;
  DevBuf<int>& d_sys = gb.sys;
  DevBuf<double>& d_coef = gb.coef;
  WM_TRY(d_flag.alloc((size_t)stiles * WM_LANES));
  WM_TRY(d_ptr.alloc((size_t)stiles * WM_LANES + 1));
  int worst = WM_OK;
  const unsigned gx = (unsigned)std::max(1, std::min(256, (N + 7) / 8));
  for (int k = 0; k < K; ++k) {
    // right-hand sides: the loads, or M times the previous stage's result
    const double* r = b_t;
    if (k > 0) {
      WM_TRY(wm_k_apply_mass64(L0, stiles, cur, rhs, nullptr, s));
      r = rhs;
    }
    // systems of stage k: (shift, shift index, sample row, weight, instance)
    std::vector<double> sg, cf;
    std::vector<int> sid, src, inst;
    std::vector<int> flag((size_t)stiles * WM_LANES, 0);
    for (int i = 0; i < m; ++i) {
      const int ns = D[i]->n_samples;
      if (ns == 0 || k >= P[i].n_int + P[i].passes) continue;
      for (int v = 0; v < ns; ++v) flag[off[i] + v] = 1;
      if (k < P[i].n_int) {
        for (int v = 0; v < ns; ++v) {
          sg.push_back(D[i]->kappa * D[i]->kappa);
          sid.push_back(kappa_sid[i]);
          src.push_back(off[i] + v);
          cf.push_back(1.0);
          inst.push_back(i);
        }
      } else {
        for (size_t j = 0; j < P[i].sigma.size(); ++j)
          for (int v = 0; v < ns; ++v) {
            sg.push_back(P[i].sigma[j]);
            sid.push_back(node_sid[i][j]);
            src.push_back(off[i] + v);
            cf.push_back(P[i].c[j]);
            inst.push_back(i);
          }
      }
    }
    WM_CUDA(cudaMemcpyAsync(d_flag.p, flag.data(), flag.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    // the rows of this stage start from zero; the others keep their result
    WM_LAUNCH(WM_PC_SINC, s, k_zero_rows<<<dim3(gx, stiles), dim3(WM_LANES, 8), 0, s>>>(N, d_flag.p, cur));
    WM_CUDA(cudaGetLastError());
    const int64_t nsys = (int64_t)sg.size();
    for (int64_t g0 = 0; g0 < nsys; g0 += per_batch) {
      const int64_t g1 = std::min(nsys, g0 + per_batch);
      const int nb = (int)(g1 - g0);
      const int tiles = (nb + WM_LANES - 1) / WM_LANES;
      std::vector<double> bsg(sg.begin() + g0, sg.begin() + g1);
      std::vector<int> bsid(sid.begin() + g0, sid.begin() + g1), bsrc(src.begin() + g0, src.begin() + g1);
      WM_TRY(set_batch_meta(ws, h->sched, tiles, bsg, bsid, bsrc, s));
      Batch bt;
      bt.schedule(h->sched);
      bt.tiles = tiles;
      bt.nsys = nb;
      bt.nshift = (int)shl.size();
      bt.precision = d0.precision;
      bt.rtol = d0.rtol;
      bt.max_iter = d0.max_iter;
      bt.degree = d0.smoother_degree;
      bt.degree_coarse = d0.smoother_degree_coarse;
      bt.cheb_ratio = d0.cheb_ratio;
      bt.replace_drop = d0.precision == WM_FP64 ? 0.0 : 1e-4;
      bt.df_residual = d0.precision != WM_FP64;
      bt.precond = d0.preconditioner;
      BatchResult br;
      WM_TRY(wm_solve_batch(h, ws, bt, r, &br, s));
      if (br.flags & 1) worst = std::min(worst, WM_ERR_NONFINITE);
      if ((br.n_not_converged > 0 || (br.flags & 2)) && worst == WM_OK) worst = WM_ERR_NOT_CONVERGED;
      // per-instance statistics from the per-system state of the batch
      std::vector<int> act(nb);
      std::vector<double> rr(nb), bb(nb);
      WM_CUDA(cudaMemcpyAsync(act.data(), ws.active.p, nb * sizeof(int), cudaMemcpyDeviceToHost, s));
      WM_CUDA(cudaMemcpyAsync(rr.data(), ws.rr.p, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
      WM_CUDA(cudaMemcpyAsync(bb.data(), ws.bb.p, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
      // weighted sums of this batch's solutions into their sample rows (CSR over rows)
      std::vector<int> ptr((size_t)stiles * WM_LANES + 1, 0), esys(nb);
      std::vector<double> ecf(nb);
      for (int q = 0; q < nb; ++q) ptr[bsrc[q] + 1]++;
      for (size_t v = 0; v + 1 < ptr.size(); ++v) ptr[v + 1] += ptr[v];
      {
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        for (int q = 0; q < nb; ++q) {
          esys[fill[bsrc[q]]] = q;
          ecf[fill[bsrc[q]]++] = cf[g0 + q];
        }
      }
      WM_TRY(d_sys.alloc(nb));
      WM_TRY(d_coef.alloc(nb));
      WM_CUDA(cudaMemcpyAsync(d_ptr.p, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      WM_CUDA(cudaMemcpyAsync(d_sys.p, esys.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
      WM_CUDA(cudaMemcpyAsync(d_coef.p, ecf.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s));
      WM_LAUNCH(WM_PC_SINC, s, k_rows_accumulate<<<dim3(gx, stiles), dim3(WM_LANES, 8), 0, s>>>(
                                   N, d_ptr.p, d_sys.p, d_coef.p, ws.x.p, cur));
      WM_CUDA(cudaGetLastError());
      WM_CUDA(cudaStreamSynchronize(s));  // the host vectors above go out of scope
      std::vector<char> seen(m, 0);
      for (int q = 0; q < nb; ++q) {
        const int i = inst[g0 + q];
        wm_stats* st = ST[i];
        if (!st) continue;
        st->n_systems += 1;
        st->n_not_converged += act[q] ? 1 : 0;
        if (bb[q] > 0) st->max_rel_residual = std::max(st->max_rel_residual, std::sqrt(rr[q] / bb[q]));
        if (!seen[i]) {
          seen[i] = 1;
          st->n_batches += 1;
          st->max_iterations = std::max(st->max_iterations, br.iterations);
          st->total_iterations += br.iterations;
          st->n_replacements += br.replacements;
          st->n_df_fallbacks += br.df_fallbacks;
        }
      }
    }
  }
  // fields: each instance's rows to its [n_i][N] output
  for (int i = 0; i < m; ++i) {
    const int ns = D[i]->n_samples;
    if (ns == 0) continue;
    const int64_t n = (int64_t)ns * N;
    WM_LAUNCH(WM_PC_LAYOUT, s, k_rows_from_tiled<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cur, N, off[i], ns,
                                                                                            U[i]));
    WM_CUDA(cudaGetLastError());
  }
  WM_CUDA(cudaStreamSynchronize(s));
  return worst;
}

}  // namespace

extern "C" int wm_sample_fields_batched(int n_inst, const wm_hier_t* h, const wm_sample_desc* d, double* const* u,
                                        wm_stats* st, void* stream) {
  if (n_inst < 0 || (n_inst > 0 && (!h || !d || !u))) return WM_ERR_INVALID_ARG;
  for (int i = 0; i < n_inst; ++i)
    if (!h[i]) return WM_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  // groups: instances with the same hierarchy and solver settings, in order of first appearance
  std::vector<char> done(n_inst, 0);
  std::vector<std::vector<int>> groups;
  for (int i = 0; i < n_inst; ++i) {
    if (done[i]) continue;
    groups.emplace_back();
    for (int j = i; j < n_inst; ++j) {
      if (done[j] || h[j] != h[i] || !same_solver(d[j], d[i])) continue;
      done[j] = 1;
      groups.back().push_back(j);
    }
  }
  int worst = WM_OK;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const std::vector<int>& G = groups[gi];
    std::vector<const wm_sample_desc*> D;
    std::vector<double*> U;
    std::vector<wm_stats*> ST;
    for (int j : G) {
      D.push_back(&d[j]);
      U.push_back(u[j]);
      ST.push_back(st ? &st[j] : nullptr);
    }
    int rc = sample_fields_group(h[G[0]], D, U, ST, s);
    // with several groups each one sizes its batches to the free memory: hand the
    // workspace of a hierarchy back once its last group is done
    if (groups.size() > 1 && h[G[0]]->ws) {
      bool later = false;
      for (size_t gj = gi + 1; gj < groups.size(); ++gj) later |= h[groups[gj][0]] == h[G[0]];
      if (!later) {
        cudaStreamSynchronize(s);
        h[G[0]]->ws->release();
      }
    }
    if (rc == WM_ERR_NOT_CONVERGED || rc == WM_ERR_NONFINITE) {
      worst = std::min(worst, rc);
      continue;
    }
    if (rc != WM_OK) return rc;
  }
  return worst;
}

// Adjoint of the sampler for a scalar loss L(u) (see the header).  Buffers:
// samp[0] loads, samp[1] dL/du, samp[2] dL/dr of the current pass (then the
// integer-chain adjoints lambda_i), samp[3] M-products; per batch ws.x holds
// the forward solutions (when recomputed) and then the adjoint solutions, and
// ws.mx the M-products of the forward ones.
extern "C" int wm_sample_fields_backward(wm_hier_t h, const wm_sample_desc* d, const double* b, const double* grad_u,
                                         double* grad_b, double* grad_kappa, wm_stats* st, void* stream) {
  WM_TRY(validate_desc(h, d));
  if (!b || !grad_u) return WM_ERR_INVALID_ARG;
  Plan P;
  WM_TRY(make_plan(d, P));
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->n_int_solves = P.n_int;
    st->n_frac_passes = P.passes;
    st->n_nodes = (int)P.c.size();
  }
  int ns = d->n_samples;
  if (ns == 0) {
    if (grad_kappa) *grad_kappa = 0.0;
    return WM_OK;
  }
  if (!is_device_ptr(b) || !is_device_ptr(grad_u) || (grad_b && !is_device_ptr(grad_b))) {
    wm_set_error("backward takes device buffers");
    return WM_ERR_INVALID_ARG;
  }
  cudaStream_t s = as_stream(stream);
  const wm_level& L0 = h->lv[0];
  const int N = L0.N;
  const int stiles = (ns + WM_LANES - 1) / WM_LANES;
  const size_t sn = (size_t)stiles * N * WM_LANES;
  const double kappa = d->kappa;
  WorkSpace& ws = workspace(h);
  for (int k = 0; k < 4; ++k) WM_TRY(ws.samp[k].alloc(sn));
  double* b_t = ws.samp[0].p;
  double* g_t = ws.samp[1].p;
  double* dr = ws.samp[2].p;
  double* tmp = ws.samp[3].p;
  WM_TRY(wm_k_to_tiled(b, ns, N, b_t, stiles, s));
  WM_TRY(wm_k_to_tiled(grad_u, ns, N, g_t, stiles, s));
  int worst = WM_OK;
  double dk = 0.0;
  std::vector<double> dots;
  const std::vector<double> shifts = call_shifts(P, kappa);
  int64_t per_batch_f = batch_size(h, ws, d, (int64_t)std::max<size_t>(1, P.sigma.size()) * ns, 2 * sizeof(double));
  int tiles_max_f = (int)((per_batch_f + WM_LANES - 1) / WM_LANES);
  WM_TRY(ws.reserve(h, tiles_max_f, (int)shifts.size(), d->precision == WM_FP64));
  WM_TRY(wm_prepare_shifts(h, ws, shifts, s));
  WM_TRY(ws.mx.alloc((size_t)tiles_max_f * N * WM_LANES));
  Pass ip;
  ip.sigma = {kappa * kappa};
  ip.ns = ns;
  ip.sid_base = (int)P.sigma.size();
  ip.nshift_total = (int)shifts.size();
  const Pass fp = frac_pass(P, ns, (int)shifts.size());
  if (P.passes > 0) WM_TRY(ws.coef.upload(P.c, s));
  // forward quantities: integer iterates w_i, pass right-hand sides r_p and
  // (where kept) every system's pass solution x_p
  std::vector<const double*> wv(P.n_int, nullptr);
  const double* rp[2] = {nullptr, nullptr};
  const double* xp[2] = {nullptr, nullptr};
  bool use_ck = false;
  if (d->ckpt == WM_CKPT_KEEP && ws.ck.valid && same_solutions(ws.ck.desc, *d) && ws.ck.b.n == sn)
    WM_TRY(equal_bits(ws, b_t, ws.ck.b.p, sn, &use_ck, s));
  if (use_ck) {
    for (int i = 0; i < P.n_int; ++i) wv[i] = ws.ck.w[i].p;
    for (int p = 0; p < P.passes; ++p) {
      rp[p] = ws.ck.r[p].p;
      xp[p] = ws.ck.x[p].p;
    }
    if (st) st->ckpt_used = 1;
  } else {
    // integer chain, keeping every iterate
    ws.chain.resize(P.n_int);
    for (int i = 0; i < P.n_int; ++i) {
      WM_TRY(ws.chain[i].alloc(sn));
      const double* r = b_t;
      if (i > 0) {
        WM_TRY(wm_k_apply_mass64(L0, stiles, ws.chain[i - 1].p, tmp, nullptr, s));
        r = tmp;
      }
      double* wi = ws.chain[i].p;
      auto sink = [&](int g0, int g1, cudaStream_t ss) -> int {
        size_t off = (size_t)(g0 / WM_LANES) * N * WM_LANES;
        size_t n = (size_t)((g1 - g0 + WM_LANES - 1) / WM_LANES) * N * WM_LANES;
        return wm_copy(ws.x.p, wi + off, n, ss);
      };
      WM_TRY(run_pass(h, ws, d, ip, r, st, &worst, sink, s));
      wv[i] = wi;
    }
    // pass right-hand sides; every pass but the last is solved forward for the
    // next one's right-hand side (its solutions kept when asked for and they fit)
    const double* v = P.n_int > 0 ? wv[P.n_int - 1] : nullptr;
    for (int p = 0; p < P.passes; ++p) {
      if (v == nullptr) {
        rp[p] = b_t;
      } else {
        WM_TRY(ws.rpass[p].alloc(sn));
        WM_TRY(wm_k_apply_mass64(L0, stiles, v, ws.rpass[p].p, nullptr, s));
        rp[p] = ws.rpass[p].p;
      }
      if (p + 1 == P.passes) break;
      const size_t xt = pass_tiles(P, ns) * N * WM_LANES;
      double* xk = nullptr;
      if (d->ckpt == WM_CKPT_KEEP && (ws.xpass[p].n >= xt || may_keep(sizeof(double) * xt))) {
        WM_TRY(ws.xpass[p].alloc(xt));
        xk = ws.xpass[p].p;
      }
      WM_TRY(ws.vpass.alloc(sn));
      WM_CUDA(cudaMemsetAsync(ws.vpass.p, 0, sizeof(double) * sn, s));
      auto sink = [&](int g0, int g1, cudaStream_t ss) -> int {
        if (xk) {
          size_t off = (size_t)(g0 / WM_LANES) * N * WM_LANES;
          size_t n = (size_t)((g1 - g0 + WM_LANES - 1) / WM_LANES) * N * WM_LANES;
          WM_TRY(wm_copy(ws.x.p, xk + off, n, ss));
        }
        return wm_sinc_accumulate(h, ns, g0, g1, ws.coef.p, ws.x.p, ws.vpass.p, ss);
      };
      WM_TRY(run_pass(h, ws, d, fp, rp[p], st, &worst, sink, s));
      xp[p] = xk;
      v = ws.vpass.p;
    }
  }
  // adjoint of the passes, last first: dL/d(out) -> dL/dr = sum_l c_l z_l, with
  // z_l = A_l^{-1} dL/d(out); dL/dkappa += -2 kappa sum_l c_l z_l^T M x_l
  const double* dout = g_t;
  for (int p = P.passes - 1; p >= 0; --p) {
    const int64_t nsys = (int64_t)P.sigma.size() * ns;
    WM_CUDA(cudaMemsetAsync(dr, 0, sizeof(double) * sn, s));
    for (int64_t g0 = 0; g0 < nsys; g0 += per_batch_f) {
      const int64_t g1 = std::min(nsys, g0 + per_batch_f);
      const int tiles = (int)((g1 - g0 + WM_LANES - 1) / WM_LANES);
      if (grad_kappa) {
        const double* xb = nullptr;
        if (xp[p]) {
          xb = xp[p] + (size_t)(g0 / WM_LANES) * N * WM_LANES;
        } else {
          WM_TRY(solve_range(h, ws, d, fp, g0, g1, rp[p], st, &worst, s));
          xb = ws.x.p;
        }
        WM_TRY(wm_k_apply_mass64(L0, tiles, xb, ws.mx.p, nullptr, s));
      }
      WM_TRY(solve_range(h, ws, d, fp, g0, g1, dout, st, &worst, s));
      WM_TRY(wm_sinc_accumulate(h, ns, (int)g0, (int)g1, ws.coef.p, ws.x.p, dr, s));
      if (grad_kappa) {
        WM_TRY(wm_system_dots(ws, tiles, N, ws.x.p, ws.mx.p, dots, s));
        for (int64_t g = g0; g < g1; ++g) dk += -2.0 * kappa * P.c[(size_t)(g / ns)] * dots[(size_t)(g - g0)];
      }
    }
    if (p > 0 || P.n_int > 0) {  // this pass's right-hand side was M v: dL/dv = M dL/dr
      WM_TRY(wm_k_apply_mass64(L0, stiles, dr, tmp, nullptr, s));
      dout = tmp;
    } else {
      dout = dr;  // n = 0: the first pass took the loads themselves
    }
  }
  // integer chain: dL/dw_n = dout; lambda_i = A0^{-1} dL/dw_i, dL/dw_{i-1} = M lambda_i,
  // dL/dkappa += -2 kappa lambda_i^T M w_i, dL/db = lambda_1
  for (int i = P.n_int - 1; i >= 0; --i) {
    // dout is M dL/dr of the first pass (or dL/du for integer beta), never dr
    const double* incoming = dout;
    if (i < P.n_int - 1) {
      WM_TRY(wm_k_apply_mass64(L0, stiles, dr, tmp, nullptr, s));
      incoming = tmp;
    }
    auto sink = [&](int g0, int g1, cudaStream_t ss) -> int {
      size_t off = (size_t)(g0 / WM_LANES) * N * WM_LANES;
      size_t nn = (size_t)((g1 - g0 + WM_LANES - 1) / WM_LANES) * N * WM_LANES;
      return wm_copy(ws.x.p, dr + off, nn, ss);
    };
    WM_TRY(run_pass(h, ws, d, ip, incoming, st, &worst, sink, s));
    if (grad_kappa) {
      WM_TRY(wm_k_apply_mass64(L0, stiles, wv[i], tmp, nullptr, s));
      WM_TRY(wm_system_dots(ws, stiles, N, dr, tmp, dots, s));
      for (int g = 0; g < ns; ++g) dk += -2.0 * kappa * dots[g];
    }
  }
  // dL/db: lambda_1 with integer solves, else dL/dr of the first pass
  const double* gb = P.n_int > 0 ? dr : (P.passes > 0 ? dout : g_t);
  if (grad_b) WM_TRY(wm_k_from_tiled(gb, stiles, N, grad_b, ns, s));
  WM_CUDA(cudaStreamSynchronize(s));
  if (grad_kappa) *grad_kappa = dk;
  return worst;
}
