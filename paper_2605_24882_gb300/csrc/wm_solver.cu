// Batched shifted solves (S + sigma_g M) x_g = r_g for all systems g of a pass
// (Eq. eq:beta-approx nodes x samples, or the integer-part solves of Sec. 3.4)
// by flexible preconditioned conjugate gradients whose preconditioner is one
// geometric multigrid V-cycle over the dyadic spline hierarchy (Sec. 3.5):
// three-term Chebyshev–Jacobi smoothing, restriction P^T and knot-insertion
// prolongation P, and a dense float64 solve on the coarsest level -- or, as an
// option, the additive BPX preconditioner (multilevel diagonal scaling).
//
// Precision (WM_MIXED): the recursion (r, p, q, z) and the V-cycle are float32;
// the solution x and the right-hand sides are float64, and the true residuals
// b - A x are formed in double-float arithmetic (float64 when their error
// bound is too large for the tolerance).  A system's recursive residual is
// replaced by its true residual whenever it has fallen by `replace_drop` since
// the last replacement, and a system is declared converged only on its true
// residual, so float32 rounding in the recursion cannot stall or fake
// convergence.  WM_FP64 runs the same algorithm with every vector in float64.
//
// Layout: systems are packed 32 per tile, vectors are [tiles][N][32]; lane =
// system.  Levels with a stencil form run their operator steps in the
// shared-memory kernels of wm_stencil.cu; the row kernels here give each warp
// one row of kTPW tiles, a row's packed entries (column, S, M) loaded once per
// warp and reused for 4 x 32 systems.  Per-system dot products are per-lane
// sums over rows followed by a fixed-order reduction over warps and chunks
// (deterministic, no atomics).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "wm_solver.h"
#include "wm_stencil.h"

namespace {

constexpr int kWarps = 8;
constexpr int kTPW = 4;  // tiles per warp in operator kernels
const dim3 kBlk(WM_LANES, kWarps);

template <typename T>
struct RowT;
template <>
struct RowT<float> {
  using type = PkRow32;
};
template <>
struct RowT<double> {
  using type = PkRow64;
};
template <typename T>
struct TrT;
template <>
struct TrT<float> {
  using type = PkTr32;
};
template <>
struct TrT<double> {
  using type = PkTr64;
};

__device__ __forceinline__ PkRow32 ld_row(const PkRow32* p) {
  int4 v = __ldg(reinterpret_cast<const int4*>(p));
  PkRow32 r;
  r.col = v.x;
  r.s = __int_as_float(v.y);
  r.m = __int_as_float(v.z);
  r.pad = 0;
  return r;
}
__device__ __forceinline__ PkRow64 ld_row(const PkRow64* p) {
  PkRow64 r;
  r.s = __ldg(&p->s);
  r.m = __ldg(&p->m);
  r.col = __ldg(&p->col);
  r.pad = 0;
  return r;
}
__device__ __forceinline__ PkTr32 ld_tr(const PkTr32* p) {
  int2 v = __ldg(reinterpret_cast<const int2*>(p));
  PkTr32 r;
  r.col = v.x;
  r.v = __int_as_float(v.y);
  return r;
}
__device__ __forceinline__ PkTr64 ld_tr(const PkTr64* p) {
  PkTr64 r;
  r.v = __ldg(&p->v);
  r.col = __ldg(&p->col);
  r.pad = 0;
  return r;
}

struct RowRange {
  int i0, i1;
};
__device__ __forceinline__ RowRange chunk_rows(int N, int chunks) {
  int per = (N + chunks - 1) / chunks;
  int i0 = blockIdx.x * per;
  int i1 = min(N, i0 + per);
  return {i0, i1};
}

__device__ __forceinline__ size_t vidx(int t, int N, int i) { return ((size_t)t * N + i) * WM_LANES + threadIdx.x; }

// Reduce acc[d][k] over the warps of the block and store the partial of tile
// t = tile0 + k, chunk blockIdx.x, at part[d][(t * chunks + chunk) * 32 + lane].
template <int ND, int NT>
__device__ __forceinline__ void block_reduce_store(double (&acc)[ND][NT], double* const* part, int chunks, int tile0,
                                                   int tiles) {
  __shared__ double sm[ND][NT][kWarps][WM_LANES];
#pragma unroll
  for (int d = 0; d < ND; ++d)
#pragma unroll
    for (int k = 0; k < NT; ++k) sm[d][k][threadIdx.y][threadIdx.x] = acc[d][k];
  __syncthreads();
  if (threadIdx.y == 0) {
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int k = 0; k < NT; ++k) {
        int t = tile0 + k;
        if (t >= tiles) continue;
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += sm[d][k][w][threadIdx.x];
        part[d][((size_t)t * chunks + blockIdx.x) * WM_LANES + threadIdx.x] = s;
      }
  }
}

// per-thread dot accumulator: products summed in T, flushed into double
// every 16 rows (bounded float rounding, little float64 work)
template <typename T>
struct Acc {
  double d = 0.0;
  T f = 0;
  int n = 0;
  __device__ __forceinline__ void add(T v) {
    f += v;
    if (++n == 16) {
      d += (double)f;
      f = 0;
      n = 0;
    }
  }
  __device__ __forceinline__ double get() const { return d + (double)f; }
};

// ------------------------------------------------------------ outer CG kernels
// r = rhs (of the system's sample), x = 0; partial ||rhs||^2 in float64
template <typename T>
__global__ void k_gather_rhs(int N, int chunks, int tiles, const double* __restrict__ src,
                             const int* __restrict__ src_of, T* __restrict__ r, double* __restrict__ x,
                             double* part_rr) {
  int t = blockIdx.y;
  int g = t * WM_LANES + threadIdx.x;
  int s = src_of[g];
  RowRange rr = chunk_rows(N, chunks);
  double acc[1][1] = {{0.0}};
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    double v = s >= 0 ? src[((size_t)(s / WM_LANES) * N + i) * WM_LANES + (s % WM_LANES)] : 0.0;
    r[vidx(t, N, i)] = (T)v;
    x[vidx(t, N, i)] = 0.0;
    acc[0][0] += v * v;
  }
  double* parts[1] = {part_rr};
  block_reduce_store<1, 1>(acc, parts, chunks, t, tiles);
}

// q = A p with partial (p, q), tiles kTPW per warp
template <typename T>
__global__ void __launch_bounds__(256) k_apply_pq(int N, int W, int chunks, int tiles,
                                                  const typename RowT<T>::type* __restrict__ pk,
                                                  const double* __restrict__ sigma, const T* __restrict__ p,
                                                  T* __restrict__ q, const int* __restrict__ tile_active,
                                                  double* part_pq) {
  const int t0 = blockIdx.y * kTPW;
  const int lane = threadIdx.x;
  bool act[kTPW];
  T sg[kTPW];
  bool any = false;
#pragma unroll
  for (int k = 0; k < kTPW; ++k) {
    int t = t0 + k;
    act[k] = t < tiles && tile_active[t];
    any |= act[k];
    sg[k] = act[k] ? (T)sigma[t * WM_LANES + lane] : (T)0;
  }
  if (!any) return;
  RowRange rr = chunk_rows(N, chunks);
  Acc<T> acc[kTPW];
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    T aS[kTPW], aM[kTPW];
#pragma unroll
    for (int k = 0; k < kTPW; ++k) aS[k] = aM[k] = 0;
    const auto* e = pk + (size_t)i * W;
    for (int w = 0; w < W; ++w) {
      auto en = ld_row(e + w);
#pragma unroll
      for (int k = 0; k < kTPW; ++k)
        if (act[k]) {
          T v = p[((size_t)(t0 + k) * N + en.col) * WM_LANES + lane];
          aS[k] += en.s * v;
          aM[k] += en.m * v;
        }
    }
#pragma unroll
    for (int k = 0; k < kTPW; ++k)
      if (act[k]) {
        size_t o = vidx(t0 + k, N, i);
        T qv = aS[k] + sg[k] * aM[k];
        q[o] = qv;
        acc[k].add(p[o] * qv);
      }
  }
  double a[1][kTPW];
#pragma unroll
  for (int k = 0; k < kTPW; ++k) a[0][k] = acc[k].get();
  double* parts[1] = {part_pq};
  block_reduce_store<1, kTPW>(a, parts, chunks, t0, tiles);
}

// float64 true residual b - A x of the systems flagged for replacement; their
// recursive residual is overwritten, partial ||b - A x||^2 in float64
template <typename T>
__global__ void __launch_bounds__(256) k_true_residual(int N, int W, int chunks, int tiles,
                                                       const PkRow64* __restrict__ pk, const double* __restrict__ sigma,
                                                       const double* __restrict__ x, const double* __restrict__ rhs,
                                                       const int* __restrict__ src_of, const int* __restrict__ rep,
                                                       const int* __restrict__ tile_rep, T* __restrict__ r,
                                                       double* part_rr) {
  const int t0 = blockIdx.y * kTPW;
  const int lane = threadIdx.x;
  bool act[kTPW];
  double sg[kTPW];
  int src[kTPW];
  bool mine[kTPW];
  bool any = false;
#pragma unroll
  for (int k = 0; k < kTPW; ++k) {
    int t = t0 + k;
    act[k] = t < tiles && tile_rep[t];
    any |= act[k];
    int g = t * WM_LANES + lane;
    sg[k] = act[k] ? sigma[g] : 0.0;
    src[k] = act[k] ? src_of[g] : -1;
    mine[k] = act[k] && rep[g];
  }
  if (!any) return;
  RowRange rr = chunk_rows(N, chunks);
  double acc[1][kTPW];
#pragma unroll
  for (int k = 0; k < kTPW; ++k) acc[0][k] = 0.0;
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    double aS[kTPW], aM[kTPW];
#pragma unroll
    for (int k = 0; k < kTPW; ++k) aS[k] = aM[k] = 0.0;
    const PkRow64* e = pk + (size_t)i * W;
    for (int w = 0; w < W; ++w) {
      PkRow64 en = ld_row(e + w);
#pragma unroll
      for (int k = 0; k < kTPW; ++k)
        if (act[k]) {
          double v = x[((size_t)(t0 + k) * N + en.col) * WM_LANES + lane];
          aS[k] += en.s * v;
          aM[k] += en.m * v;
        }
    }
#pragma unroll
    for (int k = 0; k < kTPW; ++k)
      if (mine[k]) {
        int s = src[k];
        double b = s >= 0 ? rhs[((size_t)(s / WM_LANES) * N + i) * WM_LANES + (s % WM_LANES)] : 0.0;
        double rt = b - (aS[k] + sg[k] * aM[k]);
        r[vidx(t0 + k, N, i)] = (T)rt;
        acc[0][k] += rt * rt;
      }
  }
  double* parts[1] = {part_rr};
  block_reduce_store<1, kTPW>(acc, parts, chunks, t0, tiles);
}

// exact widening of a float to float64 by its bits (normal floats and zeros;
// the others through the conversion instruction), keeping the float64 pipe,
// which also executes conversions on this part, for the FMA
__device__ __forceinline__ double to_f64(float f) {
#ifdef WM_XR_CVT
  return (double)f;
#else
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 255u) return (u & 0x7FFFFFFFu) == 0u ? __hiloint2double((int)(u & 0x80000000u), 0) : (double)f;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
#endif
}
__device__ __forceinline__ double to_f64(double f) { return f; }

// x += alpha p (float64), r -= alpha q; partial (r, r)
template <typename T>
__global__ void k_update_xr(int N, int chunks, int tiles, const double* __restrict__ alpha, const T* __restrict__ p,
                            const T* __restrict__ q, double* __restrict__ x, T* __restrict__ r,
                            const int* __restrict__ tile_active, double* part_rr) {
  int t = blockIdx.y;
  if (!tile_active[t]) return;
  double a = alpha[t * WM_LANES + threadIdx.x];
  T af = (T)a;
  RowRange rr = chunk_rows(N, chunks);
  Acc<T> acc;
  int i = rr.i0 + threadIdx.y;
#ifndef WM_XR_ROWS
#define WM_XR_ROWS 4
#endif
  constexpr int UR = WM_XR_ROWS;  // rows of a warp in flight together (the sum keeps row order)
  for (; i + (UR - 1) * kWarps < rr.i1; i += UR * kWarps) {
    double xv[UR];
    T pv[UR], qv[UR], rv[UR];
#pragma unroll
    for (int u = 0; u < UR; ++u) {
      const size_t k = vidx(t, N, i + u * kWarps);
      xv[u] = x[k];
      pv[u] = p[k];
      qv[u] = q[k];
      rv[u] = r[k];
    }
#pragma unroll
    for (int u = 0; u < UR; ++u) {
      const size_t k = vidx(t, N, i + u * kWarps);
      x[k] = xv[u] + a * to_f64(pv[u]);
      const T rn = rv[u] - af * qv[u];
      r[k] = rn;
      acc.add(rn * rn);
    }
  }
  for (; i < rr.i1; i += kWarps) {
    size_t k = vidx(t, N, i);
    x[k] += a * to_f64(p[k]);
    T rv = r[k] - af * q[k];
    r[k] = rv;
    acc.add(rv * rv);
  }
  double v[1][1] = {{acc.get()}};
  double* parts[1] = {part_rr};
  block_reduce_store<1, 1>(v, parts, chunks, t, tiles);
}

// partials (r, z) and (z, q)
template <typename T>
__global__ void k_dots_rz_zq(int N, int chunks, int tiles, const T* __restrict__ r, const T* __restrict__ z,
                             const T* __restrict__ q, const int* __restrict__ tile_active, double* part_rz,
                             double* part_zq, const int* __restrict__ skip) {
  int t = blockIdx.y;
  if (!tile_active[t] || (skip && skip[t])) return;  // skip: tiles whose partials another kernel formed
  RowRange rr = chunk_rows(N, chunks);
  Acc<T> a0, a1;
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    size_t k = vidx(t, N, i);
    T zv = z[k];
    a0.add(r[k] * zv);
    if (q) a1.add(zv * q[k]);
  }
  double v[2][1] = {{a0.get()}, {a1.get()}};
  double* parts[2] = {part_rz, part_zq};
  block_reduce_store<2, 1>(v, parts, chunks, t, tiles);
}

// p = z + beta p; with beta = 0 (the first direction, a restart) p = z without
// reading p, which may hold anything before the first direction is formed
template <typename T>
__global__ void k_update_p(int N, int chunks, const double* __restrict__ beta, const T* __restrict__ z,
                           T* __restrict__ p, const int* __restrict__ tile_active) {
  int t = blockIdx.y;
  if (!tile_active[t]) return;
  T b = (T)beta[t * WM_LANES + threadIdx.x];
  RowRange rr = chunk_rows(N, chunks);
  constexpr int UR = 4;  // rows of a warp in flight together
  int i = rr.i0 + threadIdx.y;
  for (; i + (UR - 1) * kWarps < rr.i1; i += UR * kWarps) {
    T zv[UR], pv[UR];
#pragma unroll
    for (int u = 0; u < UR; ++u) {
      const size_t k = vidx(t, N, i + u * kWarps);
      zv[u] = z[k];
      pv[u] = b == (T)0 ? (T)0 : p[k];
    }
#pragma unroll
    for (int u = 0; u < UR; ++u) p[vidx(t, N, i + u * kWarps)] = b == (T)0 ? zv[u] : zv[u] + b * pv[u];
  }
  for (; i < rr.i1; i += kWarps) {
    size_t k = vidx(t, N, i);
    p[k] = b == (T)0 ? z[k] : z[k] + b * p[k];
  }
}

// ------------------------------------------------------------ per-system scalars
__device__ __forceinline__ double sum_parts(const double* part, int chunks, int g) {
  int t = g / WM_LANES, l = g % WM_LANES;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part[((size_t)t * chunks + c) * WM_LANES + l];
  return s;
}

// The CG's per-system scalars: one block per tile, lane = system.  The
// chunk partials of a tile's 32 systems (several hundred per system for the
// stencil kernels' spatial blocks) are summed by the block's warps, warp y
// taking chunks y, y + kSumWarps, ..., and the warps' sums are added in warp
// order by warp 0, which then does the system's update: the loads of a long
// sum are spread over eight warps instead of one chain per system.
constexpr int kSumWarps = 8;
const dim3 kSumBlk(WM_LANES, kSumWarps);
struct SumSm {
  double v[kSumWarps][WM_LANES];
};
// sum of the chunk partials of system (tile blockIdx.x, lane); valid in warp 0.
// Every thread of the block calls it; `want` false skips the lane's loads (0).
__device__ __forceinline__ double tile_parts(const double* part, int chunks, bool want, SumSm& sm) {
  const int t = blockIdx.x, lane = threadIdx.x, y = threadIdx.y;
  double s = 0.0;
  if (want)
    for (int c = y; c < chunks; c += kSumWarps) s += part[((size_t)t * chunks + c) * WM_LANES + lane];
  sm.v[y][lane] = s;
  __syncthreads();
  double r = 0.0;
  if (y == 0)
#pragma unroll
    for (int w = 0; w < kSumWarps; ++w) r += sm.v[w][lane];
  __syncthreads();  // sm may be reused
  return r;
}

__global__ void __launch_bounds__(WM_LANES * kSumWarps)
    k_scal_init(int chunks, const double* part_rr, const double* part_rz, const int* src_of, double* bb,
                double* rho, double* rr, double* rr_ref, int* active, int* restart, int* flags) {
  __shared__ SumSm sm;
  const double b2 = tile_parts(part_rr, chunks, true, sm);
  const double rz = tile_parts(part_rz, chunks, true, sm);
  if (threadIdx.y != 0) return;
  const int g = blockIdx.x * WM_LANES + threadIdx.x;
  bb[g] = b2;
  rr[g] = b2;
  rr_ref[g] = b2;
  rho[g] = rz;
  restart[g] = 0;
  int a = 0;
  if (src_of[g] >= 0) {
    if (!(isfinite(b2) && isfinite(rz))) {
      atomicOr(&flags[0], 1);  // a non-finite right-hand side or preconditioned residual
    } else if (b2 > 0.0) {
      a = 1;
    }
  }
  active[g] = a;
}

__global__ void __launch_bounds__(WM_LANES * kSumWarps)
    k_scal_alpha(int chunks, const double* part_pq, const double* rho, int* active, double* alpha, int* flags) {
  __shared__ SumSm sm;
  const int g = blockIdx.x * WM_LANES + threadIdx.x;
  const bool act = active[g] != 0;
  const double pq = tile_parts(part_pq, chunks, act, sm);
  if (threadIdx.y != 0) return;
  double a = 0.0;
  if (act) {
    if (pq > 0.0 && isfinite(pq)) {
      a = rho[g] / pq;
    } else {
      atomicOr(&flags[0], 2);
      active[g] = 0;
    }
  }
  alpha[g] = a;
}

// recursive-residual test: flags systems for a float64 residual replacement;
// counters: [0] active systems, [1] flagged systems, [2] active tiles, [3] flagged tiles
__global__ void __launch_bounds__(WM_LANES * kSumWarps)
    k_scal_conv(int chunks, const double* part_rr, const double* bb, const double* rr_ref, double rtol2,
                double drop2, double* rr, int* active, int* rep, int* tile_active, int* tile_rep, int* counters,
                int* flags) {
  __shared__ SumSm sm;
  const int g = blockIdx.x * WM_LANES + threadIdx.x;
  const bool act = active[g] != 0;
  const double r2 = tile_parts(part_rr, chunks, act, sm);
  if (threadIdx.y != 0) return;
  int need = 0;
  if (act) {
    rr[g] = r2;
    if (!isfinite(r2)) {
      atomicOr(&flags[0], 1);
      active[g] = 0;
    } else {
      need = (r2 <= drop2 * rr_ref[g] || r2 <= rtol2 * bb[g]) ? 1 : 0;
    }
  }
  rep[g] = need;
  const int t = blockIdx.x;
  if (active[g]) {
    atomicAdd(&counters[0], 1);
    if (atomicExch(&tile_active[t], 1) == 0) atomicAdd(&counters[2], 1);
  }
  if (need) {
    atomicAdd(&counters[1], 1);
    if (atomicExch(&tile_rep[t], 1) == 0) atomicAdd(&counters[3], 1);
  }
}

// after a replacement: new reference norm, restart flag, convergence on the
// true residual; recounts active systems and tiles
__global__ void __launch_bounds__(WM_LANES * kSumWarps)
    k_scal_replace(int chunks, const double* part_rr, const double* bb, double rtol2, const int* rep, double* rr,
                   double* rr_ref, int* active, int* restart, int* tile_active, int* counters, int* flags) {
  __shared__ SumSm sm;
  const int g = blockIdx.x * WM_LANES + threadIdx.x;
  const bool mine = rep[g] && active[g];
  const double r2 = tile_parts(part_rr, chunks, mine, sm);
  if (threadIdx.y != 0) return;
  if (mine) {
    rr[g] = r2;
    rr_ref[g] = r2;
    restart[g] = 1;
    if (!isfinite(r2)) {
      atomicOr(&flags[0], 1);
      active[g] = 0;
    } else if (r2 <= rtol2 * bb[g]) {
      active[g] = 0;
    }
  }
  if (active[g]) {
    atomicAdd(&counters[0], 1);
    if (atomicExch(&tile_active[blockIdx.x], 1) == 0) atomicAdd(&counters[2], 1);
  }
}

// double-float residual check: counts flagged systems whose rounding-error
// bound 2^-42 ||B|| exceeds a tenth of the tolerance rtol ||b|| (those
// residuals are recomputed in float64)
__global__ void __launch_bounds__(WM_LANES * kSumWarps)
    k_df_check(int chunks, const double* part_b, const double* bb, double lim2, const int* rep, int* counter) {
  __shared__ SumSm sm;
  const int g = blockIdx.x * WM_LANES + threadIdx.x;
  const bool mine = rep[g] != 0;
  const double b2 = tile_parts(part_b, chunks, mine, sm);
  if (threadIdx.y != 0 || !mine) return;
  if (!(ldexp(b2, -84) <= lim2 * bb[g])) atomicAdd(counter, 1);
}

__global__ void __launch_bounds__(WM_LANES * kSumWarps)
    k_scal_beta(int chunks, const double* part_rz, const double* part_zq, const double* alpha, const int* active,
                int* restart, double* rho, double* beta) {
  __shared__ SumSm sm;
  const int g = blockIdx.x * WM_LANES + threadIdx.x;
  const bool upd = active[g] && !restart[g];
  const double rz = tile_parts(part_rz, chunks, true, sm);
  const double zq = tile_parts(part_zq, chunks, upd, sm);
  if (threadIdx.y != 0) return;
  double b = 0.0;
  if (upd) {
    const double r0 = rho[g];
    // Polak–Ribiere: (z_new, r_new - r_old) / (z_old, r_old) with r_new - r_old = -alpha q
    if (r0 != 0.0) b = -alpha[g] * zq / r0;
  }
  restart[g] = 0;
  beta[g] = b;
  rho[g] = rz;
}

__global__ void k_sum_parts(int nsys_pad, int chunks, const double* part, double* out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsys_pad) return;
  out[g] = sum_parts(part, chunks, g);
}

__global__ void k_fill_tile_active(int tiles, int* tile_active, const int* active) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tiles) return;
  int a = 0;
  for (int l = 0; l < WM_LANES; ++l) a |= active[t * WM_LANES + l];
  tile_active[t] = a;
}

// ------------------------------------------------------------ V-cycle kernels
// Chebyshev coefficients for step k on [lmax/ratio, 1.1 lmax]:
// k = 0: d = D^{-1} res / theta; k >= 1: d = rho_k rho_{k-1} d + (2 rho_k/delta) D^{-1} res.
struct ChebCoef {
  double c1, c2;
};
__device__ __forceinline__ ChebCoef cheb_coef(double lmax, double ratio, int k) {
  const double hi = 1.1;
  double b = hi * lmax, a = b / ratio;
  double theta = 0.5 * (b + a), delta = 0.5 * (b - a);
  double s1 = theta / delta;
  if (k == 0) return {0.0, 1.0 / theta};
  double rp = 1.0 / s1, rk = rp;
  for (int j = 1; j <= k; ++j) {
    rk = 1.0 / (2.0 * s1 - rp);
    if (j < k) rp = rk;
  }
  return {rk * rp, 2.0 * rk / delta};
}

// (c1, c2) of every smoothing step for every level and shift, computed once
// per batch in float64 (the smoothing kernels only load them)
__global__ void k_cheb_table(int nlev, int nshift, int degree, int degree_coarse, double ratio,
                             const double* __restrict__ lmax, float2* __restrict__ t32, double2* __restrict__ t64) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlev * nshift * WM_MAX_CHEB) return;
  int k = t % WM_MAX_CHEB;
  int ls = t / WM_MAX_CHEB;
  const int deg = ls < nshift ? degree : degree_coarse;  // level 0, or a coarser one
  ChebCoef c = k < deg ? cheb_coef(lmax[ls], ratio, k) : ChebCoef{0.0, 0.0};
  t32[t] = make_float2((float)c.c1, (float)c.c2);
  t64[t] = make_double2(c.c1, c.c2);
}

template <typename T>
struct C2T;
template <>
struct C2T<float> {
  using type = float2;
};
template <>
struct C2T<double> {
  using type = double2;
};

struct TileSet {
  bool act[kTPW];
  bool any;
};
__device__ __forceinline__ TileSet tile_set(int t0, int tiles, const int* tile_active) {
  TileSet ts;
  ts.any = false;
#pragma unroll
  for (int k = 0; k < kTPW; ++k) {
    int t = t0 + k;
    ts.act[k] = t < tiles && tile_active[t];
    ts.any |= ts.act[k];
  }
  return ts;
}

// first pre-smoothing step from z = 0: z = c2 D^{-1} r
template <typename T>
__global__ void k_cheb_first(int N, int chunks, int tiles, const T* __restrict__ r, const T* __restrict__ dS,
                             const T* __restrict__ dM, const double* __restrict__ sigma,
                             const typename C2T<T>::type* __restrict__ ctab, const int* __restrict__ sid,
                             T* __restrict__ z, const int* __restrict__ tile_active, const int* __restrict__ skip) {
  const int t0 = blockIdx.y * kTPW;
  TileSet ts = tile_set(t0, tiles, tile_active);
  if (skip) {  // tiles done by another kernel
    ts.any = false;
#pragma unroll
    for (int k = 0; k < kTPW; ++k) {
      ts.act[k] = ts.act[k] && !skip[t0 + k];
      ts.any |= ts.act[k];
    }
  }
  if (!ts.any) return;
  T sg[kTPW], c2[kTPW];
#pragma unroll
  for (int k = 0; k < kTPW; ++k) {
    int g = (t0 + k) * WM_LANES + threadIdx.x;
    sg[k] = ts.act[k] ? (T)sigma[g] : (T)0;
    c2[k] = ts.act[k] ? ctab[sid[g] * WM_MAX_CHEB].y : (T)0;
  }
  RowRange rr = chunk_rows(N, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    T ds = dS[i], dm = dM[i];
#pragma unroll
    for (int k = 0; k < kTPW; ++k)
      if (ts.act[k]) {
        size_t o = vidx(t0 + k, N, i);
        z[o] = c2[k] * r[o] / (ds + sg[k] * dm);
      }
  }
}

// z = D^{-1} r with D = diag(S + sigma M) (the BPX level scaling)
template <typename T>
__global__ void k_diag_scale(int N, int chunks, int tiles, const T* __restrict__ r, const T* __restrict__ dS,
                             const T* __restrict__ dM, const double* __restrict__ sigma, T* __restrict__ z,
                             const int* __restrict__ tile_active) {
  const int t0 = blockIdx.y * kTPW;
  TileSet ts = tile_set(t0, tiles, tile_active);
  if (!ts.any) return;
  T sg[kTPW];
#pragma unroll
  for (int k = 0; k < kTPW; ++k) sg[k] = ts.act[k] ? (T)sigma[(t0 + k) * WM_LANES + threadIdx.x] : (T)0;
  RowRange rr = chunk_rows(N, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    T ds = dS[i], dm = dM[i];
#pragma unroll
    for (int k = 0; k < kTPW; ++k)
      if (ts.act[k]) {
        size_t o = vidx(t0 + k, N, i);
        z[o] = r[o] / (ds + sg[k] * dm);
      }
  }
}

// Chebyshev step k in three-term form: out = z + c1 (z - prev) + c2 D^{-1} (r - A z)
// (c1 = 0 at step 0; prev = nullptr for z_prev = 0; out may alias prev)
template <typename T>
__global__ void __launch_bounds__(256) k_cheb_step(int N, int W, int chunks, int tiles, int kstep,
                                                   const typename RowT<T>::type* __restrict__ pk,
                                                   const T* __restrict__ dS, const T* __restrict__ dM,
                                                   const double* __restrict__ sigma,
                                                   const typename C2T<T>::type* __restrict__ ctab,
                                                   const int* __restrict__ sid, const T* __restrict__ r,
                                                   const T* __restrict__ zin, const T* prev, T* out,
                                                   const int* __restrict__ tile_active) {
  const int t0 = blockIdx.y * kTPW;
  const int lane = threadIdx.x;
  TileSet ts = tile_set(t0, tiles, tile_active);
  if (!ts.any) return;
  T sg[kTPW], c1[kTPW], c2[kTPW];
#pragma unroll
  for (int k = 0; k < kTPW; ++k) {
    sg[k] = c1[k] = c2[k] = 0;
    if (!ts.act[k]) continue;  // (t0 + k may lie past the last tile)
    int g = (t0 + k) * WM_LANES + lane;
    typename C2T<T>::type cf = ctab[sid[g] * WM_MAX_CHEB + kstep];
    sg[k] = (T)sigma[g];
    c1[k] = kstep > 0 ? cf.x : (T)0;
    c2[k] = cf.y;
  }
  RowRange rr = chunk_rows(N, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    T aS[kTPW], aM[kTPW];
#pragma unroll
    for (int k = 0; k < kTPW; ++k) aS[k] = aM[k] = 0;
    const auto* e = pk + (size_t)i * W;
    for (int w = 0; w < W; ++w) {
      auto en = ld_row(e + w);
#pragma unroll
      for (int k = 0; k < kTPW; ++k)
        if (ts.act[k]) {
          T v = zin[((size_t)(t0 + k) * N + en.col) * WM_LANES + lane];
          aS[k] += en.s * v;
          aM[k] += en.m * v;
        }
    }
    T ds = dS[i], dm = dM[i];
#pragma unroll
    for (int k = 0; k < kTPW; ++k)
      if (ts.act[k]) {
        size_t o = vidx(t0 + k, N, i);
        T res = r[o] - (aS[k] + sg[k] * aM[k]);
        T zc = zin[o];
        T zp = prev ? prev[o] : (T)0;
        out[o] = zc + c1[k] * (zc - zp) + c2[k] * res / (ds + sg[k] * dm);
      }
  }
}

// res = r - A z
template <typename T>
__global__ void __launch_bounds__(256) k_residual(int N, int W, int chunks, int tiles,
                                                  const typename RowT<T>::type* __restrict__ pk,
                                                  const double* __restrict__ sigma, const T* __restrict__ r,
                                                  const T* __restrict__ z, T* __restrict__ res,
                                                  const int* __restrict__ tile_active) {
  const int t0 = blockIdx.y * kTPW;
  const int lane = threadIdx.x;
  TileSet ts = tile_set(t0, tiles, tile_active);
  if (!ts.any) return;
  T sg[kTPW];
#pragma unroll
  for (int k = 0; k < kTPW; ++k) sg[k] = ts.act[k] ? (T)sigma[(t0 + k) * WM_LANES + lane] : (T)0;
  RowRange rr = chunk_rows(N, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    T aS[kTPW], aM[kTPW];
#pragma unroll
    for (int k = 0; k < kTPW; ++k) aS[k] = aM[k] = 0;
    const auto* e = pk + (size_t)i * W;
    for (int w = 0; w < W; ++w) {
      auto en = ld_row(e + w);
#pragma unroll
      for (int k = 0; k < kTPW; ++k)
        if (ts.act[k]) {
          T v = z[((size_t)(t0 + k) * N + en.col) * WM_LANES + lane];
          aS[k] += en.s * v;
          aM[k] += en.m * v;
        }
    }
#pragma unroll
    for (int k = 0; k < kTPW; ++k)
      if (ts.act[k]) {
        size_t o = vidx(t0 + k, N, i);
        res[o] = r[o] - (aS[k] + sg[k] * aM[k]);
      }
  }
}

// out (+)= T in over CSR rows with packed entries (restriction: =, prolongation: +=)
template <typename T, bool ADD>
__global__ void __launch_bounds__(256) k_transfer(int Nout, int Nin, int chunks, int tiles,
                                                  const int32_t* __restrict__ ptr,
                                                  const typename TrT<T>::type* __restrict__ ent,
                                                  const T* __restrict__ in, T* __restrict__ out,
                                                  const int* __restrict__ tile_active) {
  const int t0 = blockIdx.y * kTPW;
  const int lane = threadIdx.x;
  TileSet ts = tile_set(t0, tiles, tile_active);
  if (!ts.any) return;
  RowRange rr = chunk_rows(Nout, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    T acc[kTPW], old[kTPW];
#pragma unroll
    for (int k = 0; k < kTPW; ++k) {
      acc[k] = 0;
      old[k] = ADD && ts.act[k] ? out[((size_t)(t0 + k) * Nout + i) * WM_LANES + lane] : (T)0;
    }
    // entries UR at a time: their loads and gathers in flight together, the
    // products summed in entry order (restriction rows are the longer ones:
    // (p + 2)^2 entries against at most (p + 1)^2)
    constexpr int UR = ADD ? 4 : 8;
    const int j1 = ptr[i + 1];
    int j = ptr[i];
    for (; j + UR <= j1; j += UR) {
      typename TrT<T>::type en[UR];
      T v[UR][kTPW];
#pragma unroll
      for (int u = 0; u < UR; ++u) en[u] = ld_tr(ent + j + u);
#pragma unroll
      for (int u = 0; u < UR; ++u)
#pragma unroll
        for (int k = 0; k < kTPW; ++k)
          v[u][k] = ts.act[k] ? in[((size_t)(t0 + k) * Nin + en[u].col) * WM_LANES + lane] : (T)0;
#pragma unroll
      for (int u = 0; u < UR; ++u)
#pragma unroll
        for (int k = 0; k < kTPW; ++k)
          if (ts.act[k]) acc[k] += en[u].v * v[u][k];
    }
    for (; j < j1; ++j) {
      auto en = ld_tr(ent + j);
#pragma unroll
      for (int k = 0; k < kTPW; ++k)
        if (ts.act[k]) acc[k] += en.v * in[((size_t)(t0 + k) * Nin + en.col) * WM_LANES + lane];
    }
#pragma unroll
    for (int k = 0; k < kTPW; ++k)
      if (ts.act[k]) {
        size_t o = ((size_t)(t0 + k) * Nout + i) * WM_LANES + lane;
        if (ADD)
          out[o] = old[k] + acc[k];
        else
          out[o] = acc[k];
      }
  }
}

// z = A_c^{-1} r on the coarsest level, in float64, with the inverse of the
// system's shift
template <typename T>
__global__ void k_coarse_solve(int N, const double* __restrict__ Ainv, const int* __restrict__ sid,
                               const T* __restrict__ r, T* __restrict__ z, const int* __restrict__ tile_active) {
  int t = blockIdx.y;
  if (!tile_active[t]) return;
  int g = t * WM_LANES + threadIdx.x;
  const double* A = Ainv + (size_t)sid[g] * N * N;
  for (int i = blockIdx.x * kWarps + threadIdx.y; i < N; i += gridDim.x * kWarps) {
    double acc = 0.0;
    for (int j = 0; j < N; ++j) acc += A[(size_t)i * N + j] * (double)r[vidx(t, N, j)];
    z[vidx(t, N, i)] = (T)acc;
  }
}

// ------------------------------------------------ fused coarse end of a V-cycle
// From the first level without a stencil form down to the dense coarse solve
// and back up in one kernel (float): one block per tile of 32 systems, every
// vector of those levels in shared memory (lane = system, warps over rows),
// each step the arithmetic of the per-level kernels above in their order
// (k_cheb_first, k_cheb_step, k_residual, k_transfer, k_coarse_solve) with a
// block barrier in place of a launch boundary.  Vectors are rows of 32 floats
// at row offsets of the dynamic shared area.  Where they fit (STAGED), the
// levels' tables (operator rows, diagonals, transfers) are copied behind the
// vectors at the start, so that no step waits on L1 or L2.
constexpr int kTailMax = 6;    // smoothing levels of a fused tail
// One block of 32 warps per SM: each warp walks its rows one at a time, so the
// rows per warp set the latency of a step; without staging the shared-memory
// carve-out is kept to what the block needs so that the tables stay in L1.
#ifndef WM_TAIL_WARPS
#define WM_TAIL_WARPS 32
#endif
constexpr int kTailWarps = WM_TAIL_WARPS;
struct TailLv {
  int N = 0, W = 0, nu = 0;
  int oz0 = 0, oz1 = 0, orr = -1;   // rows of the two iterates and of r (orr < 0: r in global memory)
  const PkRow32* pk = nullptr;
  const float* dS = nullptr;
  const float* dM = nullptr;
  const float2* ctab = nullptr;     // this level's Chebyshev table [nshift][WM_MAX_CHEB]
  const int32_t* Pptr = nullptr;    // z_l += P z_{l+1}, rows of this level
  const PkTr32* P = nullptr;
  const int32_t* Rptr = nullptr;    // r_{l+1} = R res_l, rows of the next level
  const PkTr32* R = nullptr;
  // staged copies: byte offsets in the table area and element counts
  int opk = 0, odS = 0, odM = 0, oPp = 0, oP = 0, oRp = 0, oR = 0;
  int npk = 0, nPp = 0, nP = 0, nRp = 0, nR = 0;
};
struct TailDesc {
  int nl = 0, Nc = 0;
  int orc = 0, ozc = 0, ores = 0;   // rows of the coarse r and z, and of the residual scratch
  int tab0 = 0;                     // byte offset of the table area (STAGED)
  const double* ainv = nullptr;     // [nshift][Nc][Nc]
  TailLv lv[kTailMax];
};
template <typename E>
__device__ __forceinline__ void tail_copy(char* dst, const E* src, int n, int tid, int nt) {
  static_assert(sizeof(E) % 4 == 0, "word copies");
  constexpr int NW = (int)(sizeof(E) / 4);
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int w = tid; w < n * NW; w += nt) d[w] = __ldg(s + w);
}

template <bool STAGED>
__global__ void __launch_bounds__(WM_LANES * kTailWarps, 1)
    k_vcycle_tail(const TailDesc D, const double* __restrict__ sigma, const int* __restrict__ sid,
                  const float* __restrict__ rin, float* __restrict__ zout, const int* __restrict__ tile_active) {
  extern __shared__ __align__(16) float sh[];
  const int t = blockIdx.x;
  if (!tile_active[t]) return;  // the whole block
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int g = t * WM_LANES + lane;
  const float sg = (float)sigma[g];
  const int sd = sid[g];
  char* const tb = reinterpret_cast<char*>(sh) + D.tab0;
  if constexpr (STAGED) {
    const int tid = wy * WM_LANES + lane, nt = WM_LANES * kTailWarps;
    for (int l = 0; l < D.nl; ++l) {
      const TailLv& L = D.lv[l];
      tail_copy(tb + L.opk, L.pk, L.npk, tid, nt);
      tail_copy(tb + L.odS, L.dS, L.N, tid, nt);
      tail_copy(tb + L.odM, L.dM, L.N, tid, nt);
      tail_copy(tb + L.oPp, L.Pptr, L.nPp, tid, nt);
      tail_copy(tb + L.oP, L.P, L.nP, tid, nt);
      tail_copy(tb + L.oRp, L.Rptr, L.nRp, tid, nt);
      tail_copy(tb + L.oR, L.R, L.nR, tid, nt);
    }
    __syncthreads();
  }
  // the level's tables: staged copies or global memory (read-only path)
  auto row_at = [&](const TailLv& L, int i, int w) -> PkRow32 {
    if constexpr (STAGED) {
      const int4 v = *reinterpret_cast<const int4*>(tb + L.opk + ((size_t)i * L.W + w) * sizeof(PkRow32));
      PkRow32 r;
      r.col = v.x;
      r.s = __int_as_float(v.y);
      r.m = __int_as_float(v.z);
      r.pad = 0;
      return r;
    } else {
      return ld_row(L.pk + (size_t)i * L.W + w);
    }
  };
  auto dS_at = [&](const TailLv& L, int i) -> float {
    if constexpr (STAGED)
      return reinterpret_cast<const float*>(tb + L.odS)[i];
    else
      return __ldg(L.dS + i);
  };
  auto dM_at = [&](const TailLv& L, int i) -> float {
    if constexpr (STAGED)
      return reinterpret_cast<const float*>(tb + L.odM)[i];
    else
      return __ldg(L.dM + i);
  };
  auto ptr_at = [&](const int32_t* gp, int off, int i) -> int {
    if constexpr (STAGED)
      return reinterpret_cast<const int32_t*>(tb + off)[i];
    else
      return __ldg(gp + i);
  };
  auto tr_at = [&](const PkTr32* gp, int off, int j) -> PkTr32 {
    if constexpr (STAGED) {
      const int2 v = reinterpret_cast<const int2*>(tb + off)[j];
      PkTr32 r;
      r.col = v.x;
      r.v = __int_as_float(v.y);
      return r;
    } else {
      return ld_tr(gp + j);
    }
  };
  const float* rg = rin + (size_t)t * D.lv[0].N * WM_LANES + lane;
  auto V = [&](int row0, int i) -> float& { return sh[(row0 + i) * WM_LANES + lane]; };
  auto rval = [&](const TailLv& L, int i) { return L.orr < 0 ? rg[(size_t)i * WM_LANES] : V(L.orr, i); };
  // (the entries of a row are loaded UR at a time, then summed in order: one
  // block works a row at a time per warp, so the loads must overlap)
  constexpr int UR = STAGED ? 4 : 8;
  auto apply_row = [&](const TailLv& L, int zin, int i, float& aS, float& aM) {
    aS = 0.f;
    aM = 0.f;
    int w = 0;
    for (; w + UR <= L.W; w += UR) {
      PkRow32 en[UR];
      float v[UR];
#pragma unroll
      for (int u = 0; u < UR; ++u) en[u] = row_at(L, i, w + u);
#pragma unroll
      for (int u = 0; u < UR; ++u) v[u] = V(zin, en[u].col);
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        aS += en[u].s * v[u];
        aM += en[u].m * v[u];
      }
    }
    for (; w < L.W; ++w) {
      const PkRow32 en = row_at(L, i, w);
      const float v = V(zin, en.col);
      aS += en.s * v;
      aM += en.m * v;
    }
  };
  // three-term step k from z = zin; out may be prev (each row reads prev before it writes out)
  auto cheb = [&](const TailLv& L, int k, int zin, int prev, int out) {
    const float2 cf = L.ctab[sd * WM_MAX_CHEB + k];
    const float c1 = k > 0 ? cf.x : 0.f, c2 = cf.y;
    for (int i = wy; i < L.N; i += kTailWarps) {
      float aS, aM;
      apply_row(L, zin, i, aS, aM);
      const float ds = dS_at(L, i), dm = dM_at(L, i);
      const float res = rval(L, i) - (aS + sg * aM);
      const float zc = V(zin, i);
      const float zp = prev >= 0 ? V(prev, i) : 0.f;
      V(out, i) = zc + c1 * (zc - zp) + c2 * res / (ds + sg * dm);
    }
    __syncthreads();
  };
  auto transfer = [&](const int32_t* ptr, int optr, const PkTr32* ent, int oent, int nout, int in, int out,
                      bool add) {
    for (int i = wy; i < nout; i += kTailWarps) {
      float acc = 0.f;
      const int j1 = ptr_at(ptr, optr, i + 1);
      int j = ptr_at(ptr, optr, i);
      for (; j + 4 <= j1; j += 4) {
        PkTr32 en[4];
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) en[u] = tr_at(ent, oent, j + u);
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = V(in, en[u].col);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc += en[u].v * v[u];
      }
      for (; j < j1; ++j) {
        const PkTr32 en = tr_at(ent, oent, j);
        acc += en.v * V(in, en.col);
      }
      if (add)
        V(out, i) += acc;
      else
        V(out, i) = acc;
    }
    __syncthreads();
  };
  int cur[kTailMax], oth[kTailMax];
  // down: pre-smoothing from z = 0, residual, restriction
  for (int l = 0; l < D.nl; ++l) {
    const TailLv& L = D.lv[l];
    {
      const float c2 = L.ctab[sd * WM_MAX_CHEB].y;
      for (int i = wy; i < L.N; i += kTailWarps) {
        const float ds = dS_at(L, i), dm = dM_at(L, i);
        V(L.oz0, i) = c2 * rval(L, i) / (ds + sg * dm);
      }
      __syncthreads();
    }
    int c = L.oz0, o = L.oz1;
    for (int k = 1; k < L.nu; ++k) {
      cheb(L, k, c, k >= 2 ? o : -1, o);
      const int x = c;
      c = o;
      o = x;
    }
    for (int i = wy; i < L.N; i += kTailWarps) {
      float aS, aM;
      apply_row(L, c, i, aS, aM);
      V(D.ores, i) = rval(L, i) - (aS + sg * aM);
    }
    __syncthreads();
    const bool last = l + 1 == D.nl;
    transfer(L.Rptr, L.oRp, L.R, L.oR, last ? D.Nc : D.lv[l + 1].N, D.ores, last ? D.orc : D.lv[l + 1].orr, false);
    cur[l] = c;
    oth[l] = o;
  }
  // dense coarse solve in float64 with the inverse of the system's shift
  {
    const double* A = D.ainv + (size_t)sd * D.Nc * D.Nc;
    for (int i = wy; i < D.Nc; i += kTailWarps) {
      const double* Ai = A + (size_t)i * D.Nc;
      double acc = 0.0;
      int j = 0;
      for (; j + 4 <= D.Nc; j += 4) {
        double a[4];
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = Ai[j + u];
          v[u] = V(D.orc, j + u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc += a[u] * (double)v[u];
      }
      for (; j < D.Nc; ++j) acc += Ai[j] * (double)V(D.orc, j);
      V(D.ozc, i) = (float)acc;
    }
    __syncthreads();
  }
  // up: prolongation of the coarser correction, post-smoothing
  for (int l = D.nl - 1; l >= 0; --l) {
    const TailLv& L = D.lv[l];
    int c = cur[l], o = oth[l];
    transfer(L.Pptr, L.oPp, L.P, L.oP, L.N, l + 1 < D.nl ? cur[l + 1] : D.ozc, c, true);
    for (int k = 0; k < L.nu; ++k) {
      cheb(L, k, c, k >= 1 ? o : -1, o);
      const int x = c;
      c = o;
      o = x;
    }
    cur[l] = c;
  }
  float* zg = zout + (size_t)t * D.lv[0].N * WM_LANES + lane;
  for (int i = wy; i < D.lv[0].N; i += kTailWarps) zg[(size_t)i * WM_LANES] = V(cur[0], i);
}

// inverse of S_c + sigma M_c for each shift by in-place Gauss–Jordan
// elimination (SPD: no pivoting) in shared memory; one block per shift
__global__ void k_coarse_inverse(int N, const double* __restrict__ Sd, const double* __restrict__ Md,
                                 const double* __restrict__ shifts, double* __restrict__ Ainv) {
  extern __shared__ double A[];
  double* colk = A + (size_t)N * N;
  int sidx = blockIdx.x;
  double sg = shifts[sidx];
  int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < N * N; e += nt) A[e] = Sd[e] + sg * Md[e];
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    double piv = A[(size_t)k * N + k];
    __syncthreads();
    for (int i = tid; i < N; i += nt) colk[i] = A[(size_t)i * N + k];
    __syncthreads();
    double ip = 1.0 / piv;
    for (int j = tid; j < N; j += nt) A[(size_t)k * N + j] = (j == k ? 1.0 : A[(size_t)k * N + j]) * ip;
    __syncthreads();
    for (int e = tid; e < N * N; e += nt) {
      int i = e / N, j = e % N;
      if (i == k) continue;
      double f = colk[i];
      double akj = A[(size_t)k * N + j];
      A[e] = (j == k ? 0.0 : A[e]) - f * akj;
    }
    __syncthreads();
  }
  for (int e = tid; e < N * N; e += nt) Ainv[(size_t)sidx * N * N + e] = A[e];
}

// power iteration helpers for lambda_max(D^{-1}(S + sigma M)), float64
__global__ void k_power_init(int N, double* v) {
  int t = blockIdx.y;
  for (int i = blockIdx.x * kWarps + threadIdx.y; i < N; i += gridDim.x * kWarps) {
    uint32_t h = (uint32_t)(i * 2654435761u) ^ (uint32_t)((t * WM_LANES + threadIdx.x) * 2246822519u);
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    v[vidx(t, N, i)] = 0.5 + (double)(h & 0xFFFF) / 65536.0;
  }
}

// w = D^{-1} A v; partials (w, w), (v, v)
__global__ void __launch_bounds__(256) k_power_step(int N, int W, int chunks, int tiles,
                                                    const PkRow64* __restrict__ pk, const double* __restrict__ dS,
                                                    const double* __restrict__ dM, const double* __restrict__ sigma,
                                                    const double* __restrict__ v, double* __restrict__ w,
                                                    double* part_ww, double* part_vv) {
  int t = blockIdx.y;
  double sg = sigma[t * WM_LANES + threadIdx.x];
  const double* vt = v + (size_t)t * N * WM_LANES;
  RowRange rr = chunk_rows(N, chunks);
  double acc[2][1] = {{0.0}, {0.0}};
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    double aS = 0.0, aM = 0.0;
    for (int k = 0; k < W; ++k) {
      PkRow64 en = ld_row(pk + (size_t)i * W + k);
      double x = vt[(size_t)en.col * WM_LANES + threadIdx.x];
      aS += en.s * x;
      aM += en.m * x;
    }
    double wv = (aS + sg * aM) / (dS[i] + sg * dM[i]);
    w[vidx(t, N, i)] = wv;
    double vv = vt[(size_t)i * WM_LANES + threadIdx.x];
    acc[0][0] += wv * wv;
    acc[1][0] += vv * vv;
  }
  double* parts[2] = {part_ww, part_vv};
  block_reduce_store<2, 1>(acc, parts, chunks, t, tiles);
}

__global__ void k_power_scale(int N, int chunks, const double* part_ww, double* w) {
  int t = blockIdx.y;
  int g = t * WM_LANES + threadIdx.x;
  double nw = sqrt(sum_parts(part_ww, chunks, g));
  double inv = nw > 0 ? 1.0 / nw : 0.0;
  RowRange rr = chunk_rows(N, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) w[vidx(t, N, i)] *= inv;
}

__global__ void k_power_final(int nshift, int chunks, const double* part_ww, const double* part_vv, double* lmax) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nshift) return;
  double ww = sum_parts(part_ww, chunks, g), vv = sum_parts(part_vv, chunks, g);
  lmax[g] = vv > 0 ? sqrt(ww / vv) : 1.0;
}

// ------------------------------------------------------------ sinc accumulation
// v[s] += sum over the nodes j of this batch of c_j x_{(j,s)}; systems are
// g = j * ns + s, batch [g0, g1) stored from tile 0.
__global__ void k_sinc_accumulate(int N, int ns, int g0, int g1, const double* __restrict__ c,
                                  const double* __restrict__ x, double* __restrict__ v) {
  int st = blockIdx.y;
  int s = st * WM_LANES + threadIdx.x;
  if (s >= ns) return;
  if (g1 - 1 - s < 0) return;
  int jlo = g0 - s <= 0 ? 0 : (g0 - s + ns - 1) / ns;
  int jhi = (g1 - 1 - s) / ns;
  for (int i = blockIdx.x * kWarps + threadIdx.y; i < N; i += gridDim.x * kWarps) {
    double acc = 0.0;
    for (int j = jlo; j <= jhi; ++j) {
      int gg = j * ns + s - g0;
      acc += c[j] * x[((size_t)(gg / WM_LANES) * N + i) * WM_LANES + (gg % WM_LANES)];
    }
    v[((size_t)st * N + i) * WM_LANES + threadIdx.x] += acc;
  }
}

__global__ void k_copy_tiles(size_t n, const double* __restrict__ a, double* __restrict__ b) {
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k < n) b[k] = a[k];
}

template <typename T>
__global__ void k_convert(size_t n, const double* __restrict__ a, T* __restrict__ b) {
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k < n) b[k] = (T)a[k];
}
template <typename T>
__global__ void k_widen(size_t n, const T* __restrict__ a, double* __restrict__ b) {
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k < n) b[k] = (double)a[k];
}

__global__ void k_reduce_stats(int nsys, const double* rr, const double* bb, const int* active, double* out_maxrel,
                               int* out_nc) {
  __shared__ double smax[256];
  __shared__ int scnt[256];
  double m = 0.0;
  int c = 0;
  for (int g = threadIdx.x; g < nsys; g += blockDim.x) {
    if (bb[g] > 0) m = fmax(m, sqrt(rr[g] / bb[g]));
    c += active[g];
  }
  smax[threadIdx.x] = m;
  scnt[threadIdx.x] = c;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
      scnt[threadIdx.x] += scnt[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out_maxrel = smax[0];
    *out_nc = scnt[0];
  }
}

inline unsigned nblk(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }
inline int groups(int tiles) { return (tiles + kTPW - 1) / kTPW; }

}  // namespace

// ====================================================================== host
// algorithmic bytes/flops of a launch over the active tiles: `b` bytes and `f`
// flops per system of one tile
static inline void units(int cat, const Batch& bt, double b, double f) {
  double sys = (double)bt.active_tiles * WM_LANES;
  wm_prof_units(cat, b * sys, f * sys);
}

int Batch::chunks_for(int N) const {
  // row chunks per tile: at least vec_rows (128) rows each, at most 64 (the
  // partial-sum buffers); with tile groups this keeps thousands of blocks in flight
  return std::max(1, std::min(64, (N + vec_rows - 1) / vec_rows));
}

// row chunks per tile inside the V-cycle (no partial sums there): at least
// vcycle_rows (16) rows each (two per warp), so that the small coarse levels
// still spread over the SMs instead of running a few long, latency-bound warps
int Batch::vcycle_chunks(int N) const { return std::max(1, std::min(64, (N + vcycle_rows - 1) / vcycle_rows)); }

// the one-shift tiles of the current batch
static UniTiles uni_of(const WorkSpace& ws) {
  UniTiles u;
  u.flag = ws.tile_uni.p;
  u.n = ws.n_uni_tiles;
  u.groups = ws.uni_groups.p;
  u.n_groups = ws.n_uni_groups;
  u.waves = ws.uni_waves;
  return u;
}

template <typename T>
static T* vb(VBuf& b);
template <>
double* vb<double>(VBuf& b) { return b.d.p; }
template <>
float* vb<float>(VBuf& b) { return b.f.p; }

int VBuf::alloc(size_t n, bool dbl) {
  if (dbl) return d.alloc(n);
  return f.alloc(n);
}

int WorkSpace::reserve(const wm_hier* h, int tiles, int nshift, bool dbl) {
  const int L = (int)h->lv.size();
  size_t n0 = (size_t)tiles * h->lv[0].N * WM_LANES;
  WM_TRY(x.alloc(n0));
  WM_TRY(r.alloc(n0, dbl));
  WM_TRY(p.alloc(n0, dbl));
  WM_TRY(q.alloc(n0, dbl));
  lvl.resize(L);
  for (int l = 0; l < L; ++l) {
    size_t n = (size_t)tiles * h->lv[l].N * WM_LANES;
    WM_TRY(lvl[l].za.alloc(n, dbl));
    WM_TRY(lvl[l].zb.alloc(n, dbl));
    if (l < L - 1) WM_TRY(lvl[l].res.alloc(n, dbl));
    if (l > 0) WM_TRY(lvl[l].r.alloc(n, dbl));
  }
  size_t ns = (size_t)tiles * WM_LANES;
  WM_TRY(sigma.alloc(ns));
  WM_TRY(sid.alloc(ns));
  WM_TRY(src_of.alloc(ns));
  WM_TRY(active.alloc(ns));
  WM_TRY(rep.alloc(ns));
  WM_TRY(restart.alloc(ns));
  WM_TRY(tile_active.alloc(tiles));
  WM_TRY(tile_rep.alloc(tiles));
  WM_TRY(tile_uni.alloc(tiles));
  WM_TRY(rho.alloc(ns));
  WM_TRY(alpha.alloc(ns));
  WM_TRY(beta.alloc(ns));
  WM_TRY(bb.alloc(ns));
  WM_TRY(rr.alloc(ns));
  WM_TRY(rr_ref.alloc(ns));
  size_t nch = (size_t)std::max(64, wm_sten_chunks(h->lv[0], h->np));
  size_t np = (size_t)std::max(tiles, (nshift + WM_LANES - 1) / WM_LANES) * nch * WM_LANES;
  for (int k = 0; k < 3; ++k) WM_TRY(part[k].alloc(np));
  WM_TRY(flags.alloc(4));
  WM_TRY(counters.alloc(8));
  WM_TRY(lmax.alloc((size_t)L * std::max(1, nshift)));
  const wm_level& C = h->lv[L - 1];
  WM_TRY(ainv.alloc((size_t)std::max(1, nshift) * C.N * C.N));
  WM_TRY(shifts.alloc(std::max(1, nshift)));
  WM_TRY(statd.alloc(2));
  if (!host_small) WM_CUDA(cudaMallocHost((void**)&host_small, 64));
  return WM_OK;
}

void WorkSpace::release() {
  x.release();
  r.release();
  p.release();
  q.release();
  for (auto& l : lvl) {
    l.za.release();
    l.zb.release();
    l.res.release();
    l.r.release();
  }
  lvl.clear();
  sigma.release(); sid.release(); src_of.release(); active.release(); rep.release(); restart.release();
  tile_active.release(); tile_rep.release(); tile_uni.release(); uni_groups.release();
  rho.release(); alpha.release(); beta.release(); bb.release(); rr.release(); rr_ref.release();
  for (auto& pp : part) pp.release();
  flags.release(); counters.release(); lmax.release(); ainv.release(); shifts.release(); statd.release();
  for (auto& b : samp) b.release();
  noise_scratch.release();
  pw_v.release(); pw_w.release(); pw_sigma.release(); coef.release();
  cheb32.release(); cheb64.release();
  ckpt.release(); mx.release(); dots.release();
  for (auto& c : chain) c.release();
  chain.clear();
  for (int k = 0; k < 2; ++k) {
    rpass[k].release();
    xpass[k].release();
  }
  vpass.release();
  ck.release();
  if (host_small) cudaFreeHost(host_small);
  host_small = nullptr;
  // the prepared bounds and inverses went with their buffers
  prep_shifts.clear();
  prep_lmax = prep_ainv = nullptr;
  n_uni_tiles = n_uni_groups = 0;
}

// lambda_max(D^{-1}(S + sigma M)) on every non-coarsest level for each shift,
// by 15 power iterations in float64 on a batch of one system per shift.
static int estimate_lmax(const wm_hier* h, WorkSpace& ws, const std::vector<double>& shifts, cudaStream_t s) {
  int nsh = (int)shifts.size();
  int tiles = (nsh + WM_LANES - 1) / WM_LANES;
  const int L = (int)h->lv.size();
  std::vector<double> sg((size_t)tiles * WM_LANES, shifts.empty() ? 1.0 : shifts.back());
  for (int k = 0; k < nsh; ++k) sg[k] = shifts[k];
  WM_TRY(ws.pw_sigma.upload(sg, s));
  size_t n0 = (size_t)tiles * h->lv[0].N * WM_LANES;
  WM_TRY(ws.pw_v.alloc(n0));
  WM_TRY(ws.pw_w.alloc(n0));
  Batch bt;
  bt.tiles = tiles;
  for (int l = 0; l < L - 1; ++l) {
    const wm_level& Lv = h->lv[l];
    int ch = bt.chunks_for(Lv.N);
    WM_LAUNCH(WM_PC_SETUP, s, k_power_init<<<dim3(64, tiles), kBlk, 0, s>>>(Lv.N, ws.pw_v.p));
    double* v = ws.pw_v.p;
    double* w = ws.pw_w.p;
    for (int it = 0; it < 15; ++it) {
      WM_LAUNCH(WM_PC_SETUP, s, k_power_step<<<dim3(ch, tiles), kBlk, 0, s>>>(
                                    Lv.N, Lv.W, ch, tiles, Lv.d_pk64.p, Lv.d_dS64.p, Lv.d_dM64.p, ws.pw_sigma.p, v, w,
                                    ws.part[0].p, ws.part[1].p));
      if (it < 14) WM_LAUNCH(WM_PC_SETUP, s, k_power_scale<<<dim3(ch, tiles), kBlk, 0, s>>>(Lv.N, ch, ws.part[0].p, w));
      std::swap(v, w);
    }
    WM_LAUNCH(WM_PC_SETUP, s, k_power_final<<<nblk(nsh, 128), 128, 0, s>>>(nsh, ch, ws.part[0].p, ws.part[1].p,
                                                                           ws.lmax.p + (size_t)l * nsh));
    WM_CUDA(cudaGetLastError());
  }
  return WM_OK;
}

int wm_prepare_shifts(const wm_hier* h, WorkSpace& ws, const std::vector<double>& shifts, cudaStream_t s) {
  int nsh = (int)shifts.size();
  // bounds and inverses depend only on the hierarchy and the shifts: reuse them
  // when a call repeats the previous shifts and the buffers were not reallocated
  if (shifts == ws.prep_shifts && ws.lmax.p == ws.prep_lmax && ws.ainv.p == ws.prep_ainv && nsh > 0) return WM_OK;
  ws.prep_shifts.clear();
  WM_TRY(ws.shifts.upload(shifts, s));
  WM_TRY(estimate_lmax(h, ws, shifts, s));
  const wm_level& C = h->lv.back();
  size_t smem = ((size_t)C.N * C.N + C.N) * sizeof(double);
  if (smem > 220 * 1024) {
    wm_set_error("coarsest level has %d DOFs; at most 160 supported (use more levels)", C.N);
    return WM_ERR_UNSUPPORTED;
  }
  WM_CUDA(cudaFuncSetAttribute(k_coarse_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  WM_LAUNCH(WM_PC_SETUP, s, k_coarse_inverse<<<nsh, 256, smem, s>>>(C.N, C.d_Sdense.p, C.d_Mdense.p, ws.shifts.p,
                                                                    ws.ainv.p));
  WM_CUDA(cudaGetLastError());
  ws.prep_shifts = shifts;
  ws.prep_lmax = ws.lmax.p;
  ws.prep_ainv = ws.ainv.p;
  return WM_OK;
}

template <typename T>
static const typename RowT<T>::type* rows_of(const wm_level& L);
template <>
const PkRow32* rows_of<float>(const wm_level& L) { return L.d_pk32.p; }
template <>
const PkRow64* rows_of<double>(const wm_level& L) { return L.d_pk64.p; }
template <typename T>
static const typename TrT<T>::type* P_of(const wm_level& L);
template <>
const PkTr32* P_of<float>(const wm_level& L) { return L.d_P32.p; }
template <>
const PkTr64* P_of<double>(const wm_level& L) { return L.d_P64.p; }
template <typename T>
static const typename TrT<T>::type* R_of(const wm_level& L);
template <>
const PkTr32* R_of<float>(const wm_level& L) { return L.d_R32.p; }
template <>
const PkTr64* R_of<double>(const wm_level& L) { return L.d_R64.p; }
template <typename T>
static const T* dS_of(const wm_level& L) {
  return std::is_same<T, double>::value ? (const T*)L.d_dS64.p : (const T*)L.d_dS32.p;
}
template <typename T>
static const T* dM_of(const wm_level& L) {
  return std::is_same<T, double>::value ? (const T*)L.d_dM64.p : (const T*)L.d_dM32.p;
}

template <typename T>
static const typename C2T<T>::type* cheb_tab(WorkSpace& ws);
template <>
const float2* cheb_tab<float>(WorkSpace& ws) { return ws.cheb32.p; }
template <>
const double2* cheb_tab<double>(WorkSpace& ws) { return ws.cheb64.p; }

// Chebyshev coefficients of the batch's smoother for every level and shift
static int build_cheb_table(const wm_hier* h, WorkSpace& ws, const Batch& bt, cudaStream_t s) {
  int n = (int)h->lv.size() * bt.nshift * WM_MAX_CHEB;
  WM_TRY(ws.cheb32.alloc(n));
  WM_TRY(ws.cheb64.alloc(n));
  WM_LAUNCH(WM_PC_SETUP, s, k_cheb_table<<<nblk(n, 128), 128, 0, s>>>((int)h->lv.size(), bt.nshift, bt.degree,
                                                                      bt.degree_of(1),
                                                                      bt.cheb_ratio, ws.lmax.p, ws.cheb32.p,
                                                                      ws.cheb64.p));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// The V-cycle from level l down to the coarse solve and back in one launch of
// k_vcycle_tail (float), z into level l's za.  *done stays false when the
// levels do not fit it: a coarser level with a stencil form, more than
// kTailMax smoothing levels, or vectors beyond a block's shared memory.
static int vcycle_tail(const wm_hier* h, WorkSpace& ws, const Batch& bt, int l, const float* rin, cudaStream_t s,
                       bool* done) {
  *done = false;
  const int L = (int)h->lv.size();
  const int nl = L - 1 - l;
  if (nl < 1 || nl > kTailMax) return WM_OK;
  TailDesc D;
  D.nl = nl;
  int row = 0, maxn = 0;
  for (int k = 0; k < nl; ++k) {
    const wm_level& Lv = h->lv[l + k];
    if (Lv.sten) return WM_OK;
    TailLv& tl = D.lv[k];
    tl.N = Lv.N;
    tl.W = Lv.W;
    tl.nu = bt.degree_of(l + k);
    if (k > 0) {
      tl.orr = row;
      row += Lv.N;
    }
    tl.oz0 = row;
    tl.oz1 = row + Lv.N;
    row += 2 * Lv.N;
    tl.pk = Lv.d_pk32.p;
    tl.dS = Lv.d_dS32.p;
    tl.dM = Lv.d_dM32.p;
    tl.ctab = ws.cheb32.p + (size_t)(l + k) * bt.nshift * WM_MAX_CHEB;
    tl.Pptr = Lv.d_Pptr.p;
    tl.P = Lv.d_P32.p;
    tl.Rptr = Lv.d_Rptr.p;
    tl.R = Lv.d_R32.p;
    maxn = std::max(maxn, Lv.N);
  }
  const wm_level& Cv = h->lv[L - 1];
  D.Nc = Cv.N;
  D.ores = row;
  row += maxn;
  D.orc = row;
  D.ozc = row + Cv.N;
  row += 2 * Cv.N;
  D.ainv = ws.ainv.p;
  const size_t vec = (size_t)row * WM_LANES * sizeof(float);
  // the table area: every array at a 16-byte boundary
  size_t tab = 0;
  auto put = [&](int& off, size_t bytes) {
    off = (int)tab;
    tab += (bytes + 15) / 16 * 16;
  };
  for (int k = 0; k < nl; ++k) {
    const wm_level& Lv = h->lv[l + k];
    TailLv& tl = D.lv[k];
    tl.npk = (int)Lv.d_pk32.n;
    tl.nPp = (int)Lv.d_Pptr.n;
    tl.nP = (int)Lv.d_P32.n;
    tl.nRp = (int)Lv.d_Rptr.n;
    tl.nR = (int)Lv.d_R32.n;
    if ((size_t)Lv.N > Lv.d_dS32.n || (size_t)Lv.N > Lv.d_dM32.n || (size_t)Lv.N * Lv.W > Lv.d_pk32.n)
      return WM_OK;  // (tables smaller than the level: not this path)
    put(tl.opk, sizeof(PkRow32) * tl.npk);
    put(tl.odS, sizeof(float) * Lv.N);
    put(tl.odM, sizeof(float) * Lv.N);
    put(tl.oPp, sizeof(int32_t) * tl.nPp);
    put(tl.oP, sizeof(PkTr32) * tl.nP);
    put(tl.oRp, sizeof(int32_t) * tl.nRp);
    put(tl.oR, sizeof(PkTr32) * tl.nR);
  }
  D.tab0 = (int)vec;
  int dev = 0, cap = 0, per_sm = 0;
  WM_CUDA(cudaGetDevice(&dev));
  WM_CUDA(cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  WM_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  const bool staged = vec + tab <= (size_t)cap;
  if (!staged && vec > (size_t)cap) return WM_OK;
  const size_t smem = staged ? vec + tab : vec;
  const int pct = (int)std::min<size_t>(100, (smem + 1024 + per_sm - 1) * 100 / std::max(per_sm, 1));
  const dim3 blk(WM_LANES, kTailWarps);
  float* zo = vb<float>(ws.lvl[l].za);
  if (staged) {
    WM_CUDA(cudaFuncSetAttribute(k_vcycle_tail<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    WM_CUDA(cudaFuncSetAttribute(k_vcycle_tail<true>, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    WM_LAUNCH(WM_PC_VTAIL, s, k_vcycle_tail<true><<<bt.tiles, blk, smem, s>>>(D, ws.sigma.p, ws.sid.p, rin, zo,
                                                                                ws.tile_active.p));
  } else {
    WM_CUDA(cudaFuncSetAttribute(k_vcycle_tail<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    WM_CUDA(cudaFuncSetAttribute(k_vcycle_tail<false>, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    WM_LAUNCH(WM_PC_VTAIL, s, k_vcycle_tail<false><<<bt.tiles, blk, smem, s>>>(D, ws.sigma.p, ws.sid.p, rin, zo,
                                                                                 ws.tile_active.p));
  }
  WM_CUDA(cudaGetLastError());
  double fl = 2.0 * Cv.N * Cv.N;
  for (int k = 0; k < nl; ++k) {
    const wm_level& Lv = h->lv[l + k];
    fl += (2.0 * bt.degree_of(l + k) + 1.0) * (4.0 * Lv.nnz + 8.0 * Lv.N) + 4.0 * Lv.nnzP;
  }
  units(WM_PC_VTAIL, bt, 2.0 * sizeof(float) * h->lv[l].N, fl);
  *done = true;
  return WM_OK;
}

// partial sums the outer CG wants from the V-cycle's last step
template <typename T>
struct VDots {
  const T* q = nullptr;
  double* prz = nullptr;
  double* pzq = nullptr;
  bool fused = false;
};

// one V-cycle from level l on residual rin, returns the buffer holding z.
// With dots given (level 0 of the outer solve), the last post-smoothing step of
// the one-shift tiles also forms the partials (r, z) and (z, q) of the outer CG
// in dots->prz / dots->pzq; dots->fused reports whether it did.
template <typename T>
static int vcycle(const wm_hier* h, WorkSpace& ws, const Batch& bt, int l, const T* rin, T** zout, cudaStream_t s,
                  VDots<T>* dots = nullptr) {
  const int L = (int)h->lv.size();
  const wm_level& Lv = h->lv[l];
  LevelBufs& B = ws.lvl[l];
  const int* ta = ws.tile_active.p;
  const int tiles = bt.tiles;
  const int ch = bt.vcycle_chunks(Lv.N);
  const dim3 ggrid(ch, groups(tiles));
  const typename C2T<T>::type* ctab = cheb_tab<T>(ws) + (size_t)l * bt.nshift * WM_MAX_CHEB;
  const auto* pk = rows_of<T>(Lv);
  const T* dS = dS_of<T>(Lv);
  const T* dM = dM_of<T>(Lv);
  T* za = vb<T>(B.za);
  T* zb = vb<T>(B.zb);
  const double Tb = (double)sizeof(T);
  const int csm = l == 0 ? WM_PC_SMOOTH0 : WM_PC_SMOOTHC;
  const int cre = l == 0 ? WM_PC_RESID0 : WM_PC_RESIDC;
  if (l == L - 1) {
    int gx = std::max(1, std::min(64, (Lv.N + kWarps - 1) / kWarps));
    WM_LAUNCH(WM_PC_COARSE, s, k_coarse_solve<T><<<dim3(gx, tiles), kBlk, 0, s>>>(Lv.N, ws.ainv.p, ws.sid.p, rin, za,
                                                                                   ta));
    units(WM_PC_COARSE, bt, 2.0 * Tb * Lv.N, 2.0 * Lv.N * Lv.N);
    WM_CUDA(cudaGetLastError());
    *zout = za;
    return WM_OK;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (bt.tail_fused && !Lv.sten) {
      bool done = false;
      WM_TRY(vcycle_tail(h, ws, bt, l, rin, s, &done));
      if (done) {
        *zout = za;
        return WM_OK;
      }
    }
  }
  T* res = vb<T>(B.res);
  const int nu = bt.degree_of(l);
  int step_rc = WM_OK;
  // three-term step k from z = cur: the result overwrites z_prev in `oth`
  // (has_prev false: z_prev = 0, or unused at k = 0)
  auto cheb_step = [&](int k, const T* zin, T* zo, bool has_prev, VDots<T>* dd) {
    const T* prev = has_prev ? zo : nullptr;
    if (Lv.sten) {
      const bool fuse = dd && ws.n_uni_tiles > 0;
      int e = wm_sten_cheb_step<T>(Lv, h->np, h->p, tiles, k, ws.sigma.p, ctab, ws.sid.p, rin, zin, prev, zo, ta,
                                   uni_of(ws), csm, s, fuse ? dd->q : nullptr,
                                   fuse ? dd->prz : nullptr, fuse ? dd->pzq : nullptr);
      if (fuse) dd->fused = true;
      if (e != WM_OK) step_rc = e;
    } else {
      WM_LAUNCH(csm, s, k_cheb_step<T><<<ggrid, kBlk, 0, s>>>(Lv.N, Lv.W, ch, tiles, k, pk, dS, dM, ws.sigma.p,
                                                              ctab, ws.sid.p, rin, zin, prev, zo, ta));
    }
    units(csm, bt, (has_prev ? 4.0 : 3.0) * Tb * Lv.N, 2.0 * Lv.nnz + 8.0 * Lv.N);
  };
  // pre-smoothing from z = 0; with a stencil form the one-shift tiles do the
  // first two steps in one pass over r (z1 in za, z2 in zb)
  T* cur = za;
  T* oth = zb;
  int k1 = 1;
  if (Lv.sten && ws.n_uni_tiles > 0 && nu >= 2) {
    WM_TRY(wm_sten_cheb_first2<T>(Lv, h->np, h->p, tiles, ws.sigma.p, ctab, ws.sid.p, rin, za, zb, ta, uni_of(ws),
                                  csm, s));
    units(csm, bt, 3.0 * Tb * Lv.N, 2.0 * Lv.nnz + 8.0 * Lv.N);
    if (ws.n_uni_tiles < tiles) {
      WM_LAUNCH(csm, s, k_cheb_first<T><<<ggrid, kBlk, 0, s>>>(Lv.N, ch, tiles, rin, dS, dM, ws.sigma.p, ctab,
                                                               ws.sid.p, za, ta, ws.tile_uni.p));
      int e = wm_sten_cheb_step<T>(Lv, h->np, h->p, tiles, 1, ws.sigma.p, ctab, ws.sid.p, rin, za, nullptr, zb, ta,
                                   uni_of(ws), csm, s, nullptr, nullptr, nullptr, true);
      if (e != WM_OK) return e;
    }
    std::swap(cur, oth);  // cur = z2, oth = z1
    k1 = 2;
  } else {
    WM_LAUNCH(csm, s, k_cheb_first<T><<<ggrid, kBlk, 0, s>>>(Lv.N, ch, tiles, rin, dS, dM, ws.sigma.p, ctab,
                                                             ws.sid.p, za, ta, (const int*)nullptr));
    units(csm, bt, 2.0 * Tb * Lv.N, 3.0 * Lv.N);
  }
  for (int k = k1; k < nu; ++k) {
    cheb_step(k, cur, oth, k >= 2, nullptr);  // z_0 = 0
    std::swap(cur, oth);
  }
  // residual, restriction, coarse correction
  if (Lv.sten) {
    WM_TRY(wm_sten_residual<T>(Lv, h->np, h->p, tiles, ws.sigma.p, rin, cur, res, ta, uni_of(ws), cre, s));
  } else {
    WM_LAUNCH(cre, s, k_residual<T><<<ggrid, kBlk, 0, s>>>(Lv.N, Lv.W, ch, tiles, pk, ws.sigma.p, rin, cur, res,
                                                           ta));
  }
  units(cre, bt, 3.0 * Tb * Lv.N, 4.0 * Lv.nnz + 3.0 * Lv.N);
  WM_TRY(step_rc);
  const wm_level& Cv = h->lv[l + 1];
  T* rc = vb<T>(ws.lvl[l + 1].r);
  const int chc = bt.vcycle_chunks(Cv.N);
  WM_LAUNCH(WM_PC_RESTRICT, s, k_transfer<T, false><<<dim3(chc, groups(tiles)), kBlk, 0, s>>>(
                                   Cv.N, Lv.N, chc, tiles, Lv.d_Rptr.p, R_of<T>(Lv), res, rc, ta));
  units(WM_PC_RESTRICT, bt, Tb * (Lv.N + Cv.N), 2.0 * Lv.nnzP);
  T* zc = nullptr;
  WM_TRY(vcycle<T>(h, ws, bt, l + 1, rc, &zc, s));
  WM_LAUNCH(WM_PC_PROLONG, s, k_transfer<T, true><<<ggrid, kBlk, 0, s>>>(Lv.N, Cv.N, ch, tiles, Lv.d_Pptr.p,
                                                                         P_of<T>(Lv), zc, cur, ta));
  units(WM_PC_PROLONG, bt, Tb * (2.0 * Lv.N + Cv.N), 2.0 * Lv.nnzP);
  // post-smoothing from the corrected z (no z_prev at step 0)
  for (int k = 0; k < nu; ++k) {
    cheb_step(k, cur, oth, k >= 1, k == nu - 1 ? dots : nullptr);
    std::swap(cur, oth);
  }
  WM_TRY(step_rc);
  WM_CUDA(cudaGetLastError());
  *zout = cur;
  return WM_OK;
}

// BPX (additive multilevel diagonal scaling, Sec. 3.5):
// z = sum_l P_{0<-l} D_l^{-1} R_{l<-0} r, with the dense coarse solve in place of
// D^{-1} on the coarsest level; restrictions down, then scaled levels added up
// the prolongation chain.  Returns the buffer holding z (level 0's za).
template <typename T>
static int bpx(const wm_hier* h, WorkSpace& ws, const Batch& bt, const T* rin, T** zout, cudaStream_t s) {
  const int L = (int)h->lv.size();
  const int* ta = ws.tile_active.p;
  const int tiles = bt.tiles;
  const double Tb = (double)sizeof(T);
  for (int l = 0; l + 1 < L; ++l) {
    const wm_level& Lv = h->lv[l];
    const wm_level& Cv = h->lv[l + 1];
    const T* rl = l == 0 ? rin : vb<T>(ws.lvl[l].r);
    const int chc = bt.vcycle_chunks(Cv.N);
    WM_LAUNCH(WM_PC_RESTRICT, s, k_transfer<T, false><<<dim3(chc, groups(tiles)), kBlk, 0, s>>>(
                                     Cv.N, Lv.N, chc, tiles, Lv.d_Rptr.p, R_of<T>(Lv), rl, vb<T>(ws.lvl[l + 1].r),
                                     ta));
    units(WM_PC_RESTRICT, bt, Tb * (Lv.N + Cv.N), 2.0 * Lv.nnzP);
  }
  {
    const wm_level& Cv = h->lv[L - 1];
    const T* rc = L == 1 ? rin : vb<T>(ws.lvl[L - 1].r);
    int gx = std::max(1, std::min(64, (Cv.N + kWarps - 1) / kWarps));
    WM_LAUNCH(WM_PC_COARSE, s, k_coarse_solve<T><<<dim3(gx, tiles), kBlk, 0, s>>>(Cv.N, ws.ainv.p, ws.sid.p, rc,
                                                                                   vb<T>(ws.lvl[L - 1].za), ta));
    units(WM_PC_COARSE, bt, 2.0 * Tb * Cv.N, 2.0 * Cv.N * Cv.N);
  }
  for (int l = L - 2; l >= 0; --l) {
    const wm_level& Lv = h->lv[l];
    const wm_level& Cv = h->lv[l + 1];
    const T* rl = l == 0 ? rin : vb<T>(ws.lvl[l].r);
    T* zl = vb<T>(ws.lvl[l].za);
    const int ch = bt.vcycle_chunks(Lv.N);
    const dim3 ggrid(ch, groups(tiles));
    const int cat = l == 0 ? WM_PC_SMOOTH0 : WM_PC_SMOOTHC;
    WM_LAUNCH(cat, s, k_diag_scale<T><<<ggrid, kBlk, 0, s>>>(Lv.N, ch, tiles, rl, dS_of<T>(Lv), dM_of<T>(Lv),
                                                             ws.sigma.p, zl, ta));
    units(cat, bt, 2.0 * Tb * Lv.N, 3.0 * Lv.N);
    WM_LAUNCH(WM_PC_PROLONG, s, k_transfer<T, true><<<ggrid, kBlk, 0, s>>>(Lv.N, Cv.N, ch, tiles, Lv.d_Pptr.p,
                                                                           P_of<T>(Lv), vb<T>(ws.lvl[l + 1].za), zl,
                                                                           ta));
    units(WM_PC_PROLONG, bt, Tb * (2.0 * Lv.N + Cv.N), 2.0 * Lv.nnzP);
  }
  WM_CUDA(cudaGetLastError());
  *zout = vb<T>(ws.lvl[0].za);
  return WM_OK;
}

static int set_all_tiles_active(WorkSpace& ws, int tiles, cudaStream_t s) {
  std::vector<int> ones(tiles, 1);
  WM_CUDA(cudaMemcpyAsync(ws.tile_active.p, ones.data(), tiles * sizeof(int), cudaMemcpyHostToDevice, s));
  WM_CUDA(cudaStreamSynchronize(s));
  return WM_OK;
}

// Batched flexible CG with float64 residual replacement on the systems of
// `bt` (metadata already uploaded).
template <typename T>
static int fcg(const wm_hier* h, WorkSpace& ws, const Batch& bt, const double* rhs_tiled, BatchResult* res,
               cudaStream_t s) {
  const wm_level& L0 = h->lv[0];
  const int N = L0.N, tiles = bt.tiles;
  const int ch = bt.chunks_for(N);
  const dim3 grid(ch, tiles), ggrid(ch, groups(tiles));
  const int nsys_pad = tiles * WM_LANES;
  const unsigned sb = nblk(nsys_pad, 128);
  const double Tb = (double)sizeof(T);
  // partial-sum chunks of the operator kernels (stencil: one per spatial block)
  const int ch_op = L0.sten ? wm_sten_chunks(L0, h->np) : ch;
  T* r = vb<T>(ws.r);
  T* p = vb<T>(ws.p);
  T* q = vb<T>(ws.q);
  int* cnt = ws.counters.p;
  WM_TRY(build_cheb_table(h, ws, bt, s));
  WM_CUDA(cudaMemsetAsync(ws.flags.p, 0, 4 * sizeof(int), s));
  WM_LAUNCH(WM_PC_CGVEC, s, k_gather_rhs<T><<<grid, kBlk, 0, s>>>(N, ch, tiles, rhs_tiled, ws.src_of.p, r, ws.x.p,
                                                                  ws.part[0].p));
  WM_CUDA(cudaGetLastError());
  bt.active_tiles = tiles;
  units(WM_PC_CGVEC, bt, (8.0 + 8.0 + Tb) * N, 2.0 * N);
  WM_TRY(set_all_tiles_active(ws, tiles, s));
  T* z = nullptr;
  if (bt.precond == WM_PRECOND_BPX)
    WM_TRY(bpx<T>(h, ws, bt, r, &z, s));
  else
    WM_TRY(vcycle<T>(h, ws, bt, 0, r, &z, s));
  WM_LAUNCH(WM_PC_CGVEC, s, k_dots_rz_zq<T><<<grid, kBlk, 0, s>>>(N, ch, tiles, r, z, (const T*)nullptr,
                                                                  ws.tile_active.p, ws.part[1].p, ws.part[2].p,
                                                                  (const int*)nullptr));
  WM_LAUNCH(WM_PC_SCALAR, s, k_scal_init<<<tiles, kSumBlk, 0, s>>>(ch, ws.part[0].p, ws.part[1].p, ws.src_of.p,
                                                            ws.bb.p, ws.rho.p, ws.rr.p, ws.rr_ref.p, ws.active.p,
                                                            ws.restart.p, ws.flags.p));
  WM_LAUNCH(WM_PC_SCALAR, s, k_fill_tile_active<<<nblk(tiles, 128), 128, 0, s>>>(tiles, ws.tile_active.p,
                                                                                  ws.active.p));
  WM_CUDA(cudaGetLastError());
  // p = z
  WM_CUDA(cudaMemsetAsync(ws.beta.p, 0, nsys_pad * sizeof(double), s));
  WM_LAUNCH(WM_PC_CGVEC, s, k_update_p<T><<<grid, kBlk, 0, s>>>(N, ch, ws.beta.p, z, p, ws.tile_active.p));
  const double rtol2 = bt.rtol * bt.rtol;
  const double drop2 = bt.replace_drop * bt.replace_drop;
  int it = 0, n_rep_total = 0;
  bool df_res = bt.df_residual;
  for (it = 1; it <= bt.max_iter; ++it) {
    if (L0.sten) {
      WM_TRY(wm_sten_apply_pq<T>(L0, h->np, h->p, tiles, ws.sigma.p, p, q, ws.tile_active.p, uni_of(ws),
                                 ws.part[0].p, s));
    } else {
      WM_LAUNCH(WM_PC_APPLY64, s, k_apply_pq<T><<<ggrid, kBlk, 0, s>>>(N, L0.W, ch, tiles, rows_of<T>(L0),
                                                                       ws.sigma.p, p, q, ws.tile_active.p,
                                                                       ws.part[0].p));
    }
    units(WM_PC_APPLY64, bt, 2.0 * Tb * N, 4.0 * L0.nnz + 4.0 * N);
    WM_LAUNCH(WM_PC_SCALAR, s, k_scal_alpha<<<tiles, kSumBlk, 0, s>>>(ch_op, ws.part[0].p, ws.rho.p, ws.active.p,
                                                               ws.alpha.p, ws.flags.p));
    WM_LAUNCH(WM_PC_CGVEC, s, k_update_xr<T><<<grid, kBlk, 0, s>>>(N, ch, tiles, ws.alpha.p, p, q, ws.x.p, r,
                                                                   ws.tile_active.p, ws.part[0].p));
    units(WM_PC_CGVEC, bt, (16.0 + 4.0 * Tb) * N, 6.0 * N);
    WM_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(int), s));
    WM_CUDA(cudaMemsetAsync(ws.tile_active.p, 0, tiles * sizeof(int), s));
    WM_CUDA(cudaMemsetAsync(ws.tile_rep.p, 0, tiles * sizeof(int), s));
    WM_LAUNCH(WM_PC_SCALAR, s, k_scal_conv<<<tiles, kSumBlk, 0, s>>>(ch, ws.part[0].p, ws.bb.p, ws.rr_ref.p, rtol2,
                                                              drop2, ws.rr.p, ws.active.p, ws.rep.p, ws.tile_active.p,
                                                              ws.tile_rep.p, cnt, ws.flags.p));
    WM_CUDA(cudaGetLastError());
    WM_CUDA(cudaMemcpyAsync(ws.host_small, cnt, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    WM_CUDA(cudaStreamSynchronize(s));
    int n_active = ws.host_small[0];
    int n_rep = ws.host_small[1];
    int rep_tiles = ws.host_small[3];
    bt.active_tiles = ws.host_small[2];
    if (n_rep > 0) {
      // float64 true residual of the flagged systems
      n_rep_total += n_rep;
      if (L0.sten) {
        bool done = false;
        if constexpr (std::is_same<T, float>::value) {
          if (df_res) {
            WM_TRY(wm_sten_true_residual_df(L0, h->np, h->p, tiles, uni_of(ws), ws.sigma.p, ws.x.p, rhs_tiled,
                                            ws.src_of.p, ws.rep.p, ws.tile_rep.p, r, ws.part[1].p, ws.part[2].p, s));
            WM_CUDA(cudaMemsetAsync(cnt + 5, 0, sizeof(int), s));
            WM_LAUNCH(WM_PC_SCALAR, s, k_df_check<<<tiles, kSumBlk, 0, s>>>(ch_op, ws.part[2].p, ws.bb.p,
                                                                     0.01 * rtol2, ws.rep.p, cnt + 5));
            WM_CUDA(cudaGetLastError());
            WM_CUDA(cudaMemcpyAsync(ws.host_small + 8, cnt + 5, sizeof(int), cudaMemcpyDeviceToHost, s));
            WM_CUDA(cudaStreamSynchronize(s));
            if (ws.host_small[8] == 0) {
              done = true;
            } else {
              df_res = false;  // float64 residuals for the rest of this batch
              res->df_fallbacks++;
            }
          }
        }
        if (!done)
          WM_TRY(wm_sten_true_residual<T>(L0, h->np, h->p, tiles, ws.sigma.p, ws.x.p, rhs_tiled, ws.src_of.p,
                                          ws.rep.p, ws.tile_rep.p, r, ws.part[1].p, s));
      } else {
        WM_LAUNCH(WM_PC_TRUERES, s, k_true_residual<T><<<ggrid, kBlk, 0, s>>>(
                                      N, L0.W, ch, tiles, L0.d_pk64.p, ws.sigma.p, ws.x.p, rhs_tiled, ws.src_of.p,
                                      ws.rep.p, ws.tile_rep.p, r, ws.part[1].p));
      }
      {
        int keep = bt.active_tiles;
        bt.active_tiles = rep_tiles;
        units(WM_PC_TRUERES, bt, (8.0 + Tb) * N, 4.0 * L0.nnz + 4.0 * N);  // loads b_s: shared by a sample's nodes
        bt.active_tiles = keep;
      }
      WM_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(int), s));
      WM_CUDA(cudaMemsetAsync(ws.tile_active.p, 0, tiles * sizeof(int), s));
      WM_LAUNCH(WM_PC_SCALAR, s, k_scal_replace<<<tiles, kSumBlk, 0, s>>>(ch_op, ws.part[1].p, ws.bb.p, rtol2,
                                                                   ws.rep.p, ws.rr.p, ws.rr_ref.p, ws.active.p,
                                                                   ws.restart.p, ws.tile_active.p, cnt, ws.flags.p));
      WM_CUDA(cudaGetLastError());
      WM_CUDA(cudaMemcpyAsync(ws.host_small, cnt, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
      WM_CUDA(cudaStreamSynchronize(s));
      n_active = ws.host_small[0];
      bt.active_tiles = ws.host_small[2];
    }
    if (n_active == 0) break;
    // the V-cycle's last step forms (r, z) and (z, q) for the one-shift tiles
    // (chunks = its spatial blocks); the dots kernel covers the other tiles
    VDots<T> vd;
    vd.q = q;
    vd.prz = ws.part[1].p;
    vd.pzq = ws.part[2].p;
    if (bt.precond == WM_PRECOND_BPX)
      WM_TRY(bpx<T>(h, ws, bt, r, &z, s));
    else
      WM_TRY(vcycle<T>(h, ws, bt, 0, r, &z, s, &vd));
    const int ch_dots = vd.fused ? ch_op : ch;
    if (vd.fused) units(WM_PC_SMOOTH0, bt, Tb * N, 4.0 * N);  // q read and the two products
    if (!vd.fused || ws.n_uni_tiles < tiles) {
      WM_LAUNCH(WM_PC_CGVEC, s, k_dots_rz_zq<T><<<dim3(ch_dots, tiles), kBlk, 0, s>>>(
                                    N, ch_dots, tiles, r, z, q, ws.tile_active.p, ws.part[1].p, ws.part[2].p,
                                    vd.fused ? ws.tile_uni.p : (const int*)nullptr));
      if (!vd.fused) units(WM_PC_CGVEC, bt, 3.0 * Tb * N, 4.0 * N);
    }
    WM_LAUNCH(WM_PC_SCALAR, s, k_scal_beta<<<tiles, kSumBlk, 0, s>>>(ch_dots, ws.part[1].p, ws.part[2].p,
                                                              ws.alpha.p, ws.active.p, ws.restart.p, ws.rho.p,
                                                              ws.beta.p));
    WM_LAUNCH(WM_PC_CGVEC, s, k_update_p<T><<<grid, kBlk, 0, s>>>(N, ch, ws.beta.p, z, p, ws.tile_active.p));
    units(WM_PC_CGVEC, bt, 3.0 * Tb * N, 2.0 * N);
    WM_CUDA(cudaGetLastError());
  }
  res->iterations = std::min(it, bt.max_iter);
  res->replacements = n_rep_total;
  WM_LAUNCH(WM_PC_SCALAR, s, k_reduce_stats<<<1, 256, 0, s>>>(bt.nsys, ws.rr.p, ws.bb.p, ws.active.p, ws.statd.p,
                                                              cnt + 4));
  WM_CUDA(cudaMemcpyAsync(ws.host_small + 4, cnt + 4, sizeof(int), cudaMemcpyDeviceToHost, s));
  WM_CUDA(cudaMemcpyAsync(ws.host_small + 6, ws.flags.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  WM_CUDA(cudaMemcpyAsync(&ws.host_d, ws.statd.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  WM_CUDA(cudaStreamSynchronize(s));
  res->n_not_converged = ws.host_small[4];
  res->max_rel_residual = ws.host_d;
  res->flags = ws.host_small[6];
  return WM_OK;
}

int wm_solve_batch(const wm_hier* h, WorkSpace& ws, const Batch& bt, const double* rhs_tiled, BatchResult* res,
                   cudaStream_t s) {
  if (bt.precision == WM_FP64) return fcg<double>(h, ws, bt, rhs_tiled, res, s);
  return fcg<float>(h, ws, bt, rhs_tiled, res, s);
}

int wm_vcycle_apply(const wm_hier* h, WorkSpace& ws, const Batch& bt, const double* r64, double* z64,
                    cudaStream_t s) {
  size_t n = (size_t)bt.tiles * h->lv[0].N * WM_LANES;
  bt.active_tiles = bt.tiles;
  WM_TRY(build_cheb_table(h, ws, bt, s));
  WM_TRY(set_all_tiles_active(ws, bt.tiles, s));
  if (bt.precision == WM_FP64) {
    WM_TRY(wm_copy(r64, ws.r.d.p, n, s));
    double* z = nullptr;
    WM_TRY(vcycle<double>(h, ws, bt, 0, ws.r.d.p, &z, s));
    WM_TRY(wm_copy(z, z64, n, s));
  } else {
    WM_TRY(wm_convert_f32(r64, ws.r.f.p, n, s));
    float* z = nullptr;
    WM_TRY(vcycle<float>(h, ws, bt, 0, ws.r.f.p, &z, s));
    WM_TRY(wm_widen_f32(z, z64, n, s));
  }
  return WM_OK;
}

int wm_sinc_accumulate(const wm_hier* h, int ns, int g0, int g1, const double* c_dev, const double* x,
                       double* v_tiled, cudaStream_t s) {
  const wm_level& L0 = h->lv[0];
  int stiles = (ns + WM_LANES - 1) / WM_LANES;
  int gx = std::max(1, std::min(256, (L0.N + kWarps - 1) / kWarps));
  WM_LAUNCH(WM_PC_SINC, s, k_sinc_accumulate<<<dim3(gx, stiles), kBlk, 0, s>>>(L0.N, ns, g0, g1, c_dev, x, v_tiled));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_copy(const double* a, double* b, size_t n, cudaStream_t s) {
  if (n == 0) return WM_OK;
  WM_LAUNCH(WM_PC_SINC, s, k_copy_tiles<<<nblk(n, 256), 256, 0, s>>>(n, a, b));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_convert_f32(const double* a, float* b, size_t n, cudaStream_t s) {
  if (n == 0) return WM_OK;
  WM_LAUNCH(WM_PC_SINC, s, k_convert<float><<<nblk(n, 256), 256, 0, s>>>(n, a, b));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_widen_f32(const float* a, double* b, size_t n, cudaStream_t s) {
  if (n == 0) return WM_OK;
  WM_LAUNCH(WM_PC_SINC, s, k_widen<float><<<nblk(n, 256), 256, 0, s>>>(n, a, b));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_system_dots(WorkSpace& ws, int tiles, int N, const double* a, const double* b, std::vector<double>& out,
                   cudaStream_t s) {
  Batch bt;
  bt.tiles = tiles;
  const int ch = bt.chunks_for(N);
  const int nsys_pad = tiles * WM_LANES;
  WM_TRY(ws.dots.alloc(nsys_pad));
  if (ws.part[1].n < (size_t)tiles * ch * WM_LANES || ws.tile_active.n < (size_t)tiles) {
    wm_set_error("workspace too small for the system dots");
    return WM_ERR_INVALID_ARG;
  }
  WM_TRY(set_all_tiles_active(ws, tiles, s));
  WM_LAUNCH(WM_PC_SINC, s, k_dots_rz_zq<double><<<dim3(ch, tiles), kBlk, 0, s>>>(
                               N, ch, tiles, a, b, (const double*)nullptr, ws.tile_active.p, ws.part[1].p,
                               ws.part[2].p, (const int*)nullptr));
  WM_LAUNCH(WM_PC_SINC, s, k_sum_parts<<<nblk(nsys_pad, 128), 128, 0, s>>>(nsys_pad, ch, ws.part[1].p, ws.dots.p));
  WM_CUDA(cudaGetLastError());
  out.resize(nsys_pad);
  WM_CUDA(cudaMemcpyAsync(out.data(), ws.dots.p, nsys_pad * sizeof(double), cudaMemcpyDeviceToHost, s));
  WM_CUDA(cudaStreamSynchronize(s));
  return WM_OK;
}
