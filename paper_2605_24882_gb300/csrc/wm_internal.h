// Internal declarations of the GB300 Whittle–Matérn sampler library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "wmfield.h"

// Systems are packed 32 to a tile: a batched vector is stored [tiles][N][32],
// so the 32 systems of a tile sit in one 128-byte (float) or 256-byte (double)
// row per DOF and a warp reads one DOF of 32 systems in one coalesced access.
#define WM_LANES 32

void wm_set_error(const char* fmt, ...);

#define WM_CUDA(call)                                                             \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      wm_set_error("%s failed at %s:%d: %s", #call, __FILE__, __LINE__,           \
                   cudaGetErrorString(e_));                                       \
      return e_ == cudaErrorMemoryAllocation ? WM_ERR_OOM : WM_ERR_CUDA;          \
    }                                                                             \
  } while (0)

#define WM_TRY(expr)                          \
  do {                                        \
    int wm_try_rc_ = (expr);                  \
    if (wm_try_rc_ != WM_OK) return wm_try_rc_; \
  } while (0)

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  int alloc(size_t count) {
    if (count <= n && p) return WM_OK;
    release();
    if (count == 0) return WM_OK;
    cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      n = 0;
      wm_set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
      return WM_ERR_OOM;
    }
    n = count;
    return WM_OK;
  }
  int upload(const std::vector<T>& v, cudaStream_t s) {
    WM_TRY(alloc(v.size()));
    if (!v.empty()) WM_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return WM_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

// Packed operator rows and transfer entries: one aligned load per stored
// nonzero (column index with both matrix values), so a warp reads a row entry
// with one broadcast load instead of three.
struct __align__(16) PkRow32 {
  int col;
  float s, m;
  int pad;
};
struct __align__(8) PkRow64 {
  double s, m;
  int col, pad;
};
struct __align__(8) PkTr32 {
  int col;
  float v;
};
struct __align__(16) PkTr64 {
  double v;
  int col, pad;
};

// ---------------------------------------------------------------- host setup
// Topology of a surface kind: periodic single patch, or six cube-face patches.
inline bool wm_periodic(int kind) { return kind == WM_TORUS || kind == WM_NURBS_PERIODIC; }
inline bool wm_is_nurbs(int kind) { return kind == WM_NURBS_PERIODIC || kind == WM_NURBS_CUBE; }

// Host copy of a NURBS patch of the geometry map.
struct WmNurbs {
  int pu = 0, pv = 0, nu = 0, nv = 0;
  std::vector<double> ku, kv, cpw;  // knots, [nv][nu][4] control points and weights
};

struct wm_geom {
  wm_geom_desc d;
  int np;  // patches
  std::vector<WmNurbs> nurbs;  // NURBS kinds only
};

// One level of the dyadic hierarchy.
struct wm_level {
  int nu = 0, nv = 0;    // elements per patch side
  int nlu = 0, nlv = 0;  // local DOFs per patch side
  int N = 0;             // glued DOFs
  int E = 0;             // elements (all patches)
  int nk = 0;            // local functions per element, (p+1)^2
  int W = 0;             // stored entries per operator row (max row length)
  int64_t nnz = 0;       // non-padding entries of all rows
  int64_t nnzP = 0;      // entries of the prolongation to this level
  std::vector<int32_t> l2g;   // [np][nlv][nlu]
  std::vector<int32_t> conn;  // [E][nk]
  std::vector<int32_t> col;   // [N][W], padded with the row index
  std::vector<int32_t> diag_slot;  // [N]
  // 1D tables at the Gauss points of each element: [n][p+1][nq]
  std::vector<double> bu, du, bv, dv;
  // device copies
  DevBuf<int32_t> d_conn, d_col, d_diag_slot;
  DevBuf<double> d_metric;  // [E][nq*nq][4]
  DevBuf<double> d_Se, d_Me;  // element matrices [E][nk][nk]
  DevBuf<int32_t> d_asm_ptr, d_asm_idx;  // (row, slot) -> element-matrix entries
  DevBuf<double> d_S64, d_M64;  // [N][W]
  DevBuf<float> d_S32, d_M32;
  DevBuf<double> d_dS64, d_dM64;  // diagonals [N]
  DevBuf<float> d_dS32, d_dM32;
  DevBuf<double> d_bu, d_du, d_bv, d_dv;
  // prolongation from the next coarser level to this one (CSR over fine rows)
  // and restriction to it (CSR over coarse rows); empty on the coarsest level
  DevBuf<int32_t> d_Pptr, d_Pcol, d_Rptr, d_Rcol;
  DevBuf<double> d_Pval64, d_Rval64;
  DevBuf<float> d_Pval32, d_Rval32;
  int nP = 0, nR = 0;  // rows of P (fine N) and R (coarse N)
  // packed copies of the rows, the prolongation (fine rows) and restriction
  // (coarse rows)
  DevBuf<PkRow32> d_pk32;
  DevBuf<PkRow64> d_pk64;
  DevBuf<PkTr32> d_P32, d_R32;
  DevBuf<PkTr64> d_P64, d_R64;
  // stencil form (shared-memory kernels): extended patch grids with halo p,
  // owner map, per-row (2p+1)^2 coefficient pairs (S, M); sten = false when the
  // level uses the row (ELL) kernels only
  bool sten = false;
  int ELU = 0, ELV = 0, nbu = 0, nbv = 0;
  DevBuf<int32_t> d_ext, d_own;
  DevBuf<float2> d_csm32;
  DevBuf<double2> d_csm64;
  // the same coefficients as float pairs (S_hi, S_lo, M_hi, M_lo) for the
  // double-float residual
  DevBuf<float4> d_csmdf;
  // noise gather on this level: DOF i <- sum over (e, k) entries
  DevBuf<int32_t> d_ng_ptr, d_ng_idx;
  // finest level: sqrt(w_q a_q) of every Gauss point [E][nq*nq], the
  // sample-independent factor of the noise loads
  DevBuf<double> d_noise_w;
  // coarse dense operators (coarsest level only): [N][N] row-major
  DevBuf<double> d_Sdense, d_Mdense;
};

struct WorkSpace;

struct wm_hier {
  wm_geom_desc g;
  std::vector<WmNurbs> nurbs;  // NURBS kinds only
  int np = 0, p = 0, nq = 0;
  std::vector<wm_level> lv;
  std::vector<double> gw, gx;  // Gauss weights and nodes on [0,1]
  DevBuf<double> d_gw, d_gx;
  WorkSpace* ws = nullptr;
  int device = 0;  // the CUDA device holding the hierarchy's buffers
  wm_schedule sched{8, 4, 128, 16, 1};  // kernel schedule of the batched solves
};

// host helpers (wm_host_setup.cpp)
int wm_host_build_level(const wm_geom_desc& g, int np, int nu, int nv, wm_level& L);
void wm_gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);
int wm_host_prolongation(const wm_geom_desc& g, int np, const wm_level& fine, const wm_level& coarse,
                         std::vector<int32_t>& Pptr, std::vector<int32_t>& Pcol, std::vector<double>& Pval,
                         std::vector<int32_t>& Rptr, std::vector<int32_t>& Rcol, std::vector<double>& Rval);
void wm_host_tables(const wm_geom_desc& g, const std::vector<double>& gx, wm_level& L);
void wm_host_assembly_map(const wm_level& L, std::vector<int32_t>& ptr, std::vector<int32_t>& idx);
void wm_host_noise_map(const wm_level& L, std::vector<int32_t>& ptr, std::vector<int32_t>& idx);
int wm_host_stencil(const wm_geom_desc& g, int np, const wm_level& L, std::vector<int32_t>& ext,
                    std::vector<int32_t>& own, std::vector<int16_t>& slot);
int wm_split_beta(double beta, int split, int* n, double* bp, int* passes);
int wm_host_mass_bounds(const wm_geom_desc& g, int nu, int nv, double* lo, double* hi);
// NURBS geometry: metric (a, G11, G12, G22) at the Gauss points gx of every
// element of a level ([E][nq^2][4], element order (m nv + ev) nu + eu); checks
// of a patch set (knots, weights, closure or edge agreement)
int wm_host_nurbs_metric(const std::vector<WmNurbs>& patches, int nu, int nv, const std::vector<double>& gx,
                         std::vector<double>& out);
int wm_host_nurbs_check(int kind, const std::vector<WmNurbs>& patches);
// bounds of the mass spectrum from the area element extremes at the Gauss points
int wm_host_mass_bounds_metric(const wm_geom_desc& g, int nu, int nv, double amin, double amax, double* lo,
                               double* hi);

// ---------------------------------------------------------------- kernels
// geometry and assembly (wm_assembly.cu)
int wm_k_metric(const wm_hier* h, const wm_level& L, cudaStream_t s);
int wm_k_element_matrices(const wm_hier* h, wm_level& L, cudaStream_t s);
int wm_k_assemble_rows(const wm_hier* h, wm_level& L, cudaStream_t s);
int wm_k_dense_coarse(const wm_level& L, cudaStream_t s);
int wm_k_pack_rows(wm_level& L, cudaStream_t s);

// noise (wm_noise.cu)
int wm_k_philox(const uint32_t* ctr, uint64_t key, uint32_t* out, int64_t n, cudaStream_t s);
int wm_k_normals(uint64_t seed, int sample, int stream_id, int64_t q0, int64_t n, double* out,
                 cudaStream_t s);
// loads of rows [row0, row0+ns) of a tiled [tiles][N][32] buffer (row v at tile
// v/32, lane v%32), row row0 + k holding the loads of sample sample_first + k
// (its Philox counters); `bl` is scratch of E*nk*ns doubles
// sqrt(w_q a_q) of the level's Gauss points into L.d_noise_w (after its metric)
int wm_k_noise_weights(const wm_hier* h, wm_level& L, cudaStream_t s);
int wm_k_noise_tiled(const wm_hier* h, uint64_t seed, int sample_first, int row0, int ns, double* b_tiled,
                     double* bl, cudaStream_t s);

// batched operators (wm_operator.cu); vectors are [tiles][N][32]
template <typename T>
int wm_k_apply(const wm_level& L, int tiles, const double* sigma, const T* x, T* y,
               const int* tile_active, cudaStream_t s);
int wm_k_apply_mass64(const wm_level& L, int tiles, const double* x, double* y,
                      const int* tile_active, cudaStream_t s);
template <typename T>
int wm_k_prolong_add(const wm_level& fine, int tiles, const T* xc, T* xf, const int* tile_active,
                     cudaStream_t s);
template <typename T>
int wm_k_restrict(const wm_level& fine, int tiles, const T* rf, T* rc, const int* tile_active,
                  cudaStream_t s);

// layout conversion between [n][N] and [tiles][N][32]
int wm_k_to_tiled(const double* src, int n, int N, double* dst, int tiles, cudaStream_t s);
int wm_k_from_tiled(const double* src, int tiles, int N, double* dst, int n, cudaStream_t s);

// ---------------------------------------------------------------- profiling
// Launch categories for live per-kernel timing (CUDA events around each launch
// when enabled through wm_profile_enable) and launch counting (always on).
enum {
  WM_PC_APPLY64 = 0,   // operator apply of the outer CG (q = A p)
  WM_PC_SMOOTH0,       // Chebyshev smoothing steps on the finest level
  WM_PC_SMOOTHC,       // Chebyshev smoothing steps on coarser levels
  WM_PC_RESID0,        // residual before restriction, finest level
  WM_PC_RESIDC,        // residual before restriction, coarser levels
  WM_PC_RESTRICT,      // restriction P^T
  WM_PC_PROLONG,       // prolongation P (add)
  WM_PC_COARSE,        // dense coarse solve
  WM_PC_CGVEC,         // outer CG vector updates and dot products
  WM_PC_SCALAR,        // per-system scalar kernels
  WM_PC_NOISE,         // Philox white-noise loads
  WM_PC_SINC,          // sinc accumulation, mass apply of pass rhs, copies
  WM_PC_SETUP,         // smoother bounds (power iteration), coarse inverses
  WM_PC_LAYOUT,        // [n][N] <-> tiled layout conversions
  WM_PC_ASSEMBLY,      // metric, element matrices, rows
  WM_PC_APPLY,         // component operator applies
  WM_PC_TRUERES,       // float64 true residual b - A x (residual replacement)
  WM_PC_VTAIL,         // fused coarse end of the V-cycle (levels without a stencil form, coarse solve)
  WM_PC_COUNT
};
void wm_prof_begin(int cat, cudaStream_t s);
void wm_prof_end(int cat, cudaStream_t s);
// algorithmic bytes and flops of the launch just made (counted while timing is on)
void wm_prof_units(int cat, double bytes, double flops);
#define WM_LAUNCH(cat, s, ...)  \
  do {                          \
    wm_prof_begin((cat), (s));  \
    __VA_ARGS__;                \
    wm_prof_end((cat), (s));    \
  } while (0)
