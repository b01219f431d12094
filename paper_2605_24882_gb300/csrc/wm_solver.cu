// Batched shifted solves (S + sigma_g M) x_g = r_g for all systems g of a pass
// (Eq. eq:beta-approx nodes x samples, or the integer-part solves of Sec. 3.4)
// by flexible preconditioned conjugate gradients whose preconditioner is one
// geometric multigrid V-cycle over the dyadic spline hierarchy (Sec. 3.5):
// Chebyshev–Jacobi smoothing, restriction P^T and knot-insertion prolongation P,
// and a dense float64 solve on the coarsest level.
//
// Precision: the outer iteration (x, r, p, q, dot products, step lengths) is
// float64; the V-cycle runs in float64 (WM_FP64) or float32 (WM_MIXED).
//
// Layout: systems are packed 32 per tile, vectors are [tiles][N][32]; grids are
// (row chunks, tiles) with one warp per row and lane = system, so per-system
// dot products are per-lane sums over rows followed by a fixed-order
// reduction over warps and chunks (deterministic, no atomics).
#include <algorithm>
#include <cmath>

#include "wm_solver.h"

namespace {

constexpr int kWarps = 8;
const dim3 kBlk(WM_LANES, kWarps);

// ------------------------------------------------------------ dot partials
// Block (chunk c, tile t) reduces rows [c*rows, (c+1)*rows) and writes
// partial[(t * chunks + c) * 32 + lane].
template <int ND>
__device__ __forceinline__ void block_reduce_store(double (&acc)[ND], double* const* partial, int chunks) {
  __shared__ double sm[ND][kWarps][WM_LANES];
#pragma unroll
  for (int d = 0; d < ND; ++d) sm[d][threadIdx.y][threadIdx.x] = acc[d];
  __syncthreads();
  if (threadIdx.y == 0) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += sm[d][w][threadIdx.x];
      partial[d][((size_t)blockIdx.y * chunks + blockIdx.x) * WM_LANES + threadIdx.x] = s;
    }
  }
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

// r = rhs(source sample), x = 0; partials (r, r)
__global__ void k_gather_rhs(int N, int chunks, const double* __restrict__ src, const int* __restrict__ src_of,
                             double* __restrict__ r, double* __restrict__ x, double* part_rr) {
  int t = blockIdx.y;
  int g = t * WM_LANES + threadIdx.x;
  int s = src_of[g];
  RowRange rr = chunk_rows(N, chunks);
  double acc[1] = {0.0};
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    double v = s >= 0 ? src[((size_t)(s / WM_LANES) * N + i) * WM_LANES + (s % WM_LANES)] : 0.0;
    r[vidx(t, N, i)] = v;
    x[vidx(t, N, i)] = 0.0;
    acc[0] += v * v;
  }
  double* parts[1] = {part_rr};
  block_reduce_store<1>(acc, parts, chunks);
}

// q = A p in float64 with partials (p, q)
__global__ void __launch_bounds__(256) k_apply_pq(int N, int W, int chunks, const int32_t* __restrict__ col,
                                                  const double* __restrict__ S, const double* __restrict__ M,
                                                  const double* __restrict__ sigma, const double* __restrict__ p,
                                                  double* __restrict__ q, const int* __restrict__ tile_active,
                                                  double* part_pq) {
  int t = blockIdx.y;
  if (!tile_active[t]) return;
  double sg = sigma[t * WM_LANES + threadIdx.x];
  const double* pt = p + (size_t)t * N * WM_LANES;
  RowRange rr = chunk_rows(N, chunks);
  double acc[1] = {0.0};
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    const int32_t* c = col + (size_t)i * W;
    const double* s = S + (size_t)i * W;
    const double* m = M + (size_t)i * W;
    double aS = 0.0, aM = 0.0;
    for (int w = 0; w < W; ++w) {
      double v = pt[(size_t)c[w] * WM_LANES + threadIdx.x];
      aS += s[w] * v;
      aM += m[w] * v;
    }
    double qv = aS + sg * aM;
    q[vidx(t, N, i)] = qv;
    acc[0] += pt[(size_t)i * WM_LANES + threadIdx.x] * qv;
  }
  double* parts[1] = {part_pq};
  block_reduce_store<1>(acc, parts, chunks);
}

// x += alpha p, r -= alpha q; partials (r, r)
__global__ void k_update_xr(int N, int chunks, const double* __restrict__ alpha, const double* __restrict__ p,
                            const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                            const int* __restrict__ tile_active, double* part_rr) {
  int t = blockIdx.y;
  if (!tile_active[t]) return;
  double a = alpha[t * WM_LANES + threadIdx.x];
  RowRange rr = chunk_rows(N, chunks);
  double acc[1] = {0.0};
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    size_t k = vidx(t, N, i);
    x[k] += a * p[k];
    double rv = r[k] - a * q[k];
    r[k] = rv;
    acc[0] += rv * rv;
  }
  double* parts[1] = {part_rr};
  block_reduce_store<1>(acc, parts, chunks);
}

// partials (r, z) and (z, q)
template <typename Tz>
__global__ void k_dots_rz_zq(int N, int chunks, const double* __restrict__ r, const Tz* __restrict__ z,
                             const double* __restrict__ q, const int* __restrict__ tile_active, double* part_rz,
                             double* part_zq) {
  int t = blockIdx.y;
  if (!tile_active[t]) return;
  RowRange rr = chunk_rows(N, chunks);
  double acc[2] = {0.0, 0.0};
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    size_t k = vidx(t, N, i);
    double zv = (double)z[k];
    acc[0] += r[k] * zv;
    if (q) acc[1] += zv * q[k];
  }
  double* parts[2] = {part_rz, part_zq};
  block_reduce_store<2>(acc, parts, chunks);
}

// p = z + beta p
template <typename Tz>
__global__ void k_update_p(int N, int chunks, const double* __restrict__ beta, const Tz* __restrict__ z,
                           double* __restrict__ p, const int* __restrict__ tile_active) {
  int t = blockIdx.y;
  if (!tile_active[t]) return;
  double b = beta[t * WM_LANES + threadIdx.x];
  RowRange rr = chunk_rows(N, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    size_t k = vidx(t, N, i);
    p[k] = (double)z[k] + b * p[k];
  }
}

// ------------------------------------------------------------ per-system scalars
__device__ __forceinline__ double sum_parts(const double* part, int chunks, int g) {
  int t = g / WM_LANES, l = g % WM_LANES;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part[((size_t)t * chunks + c) * WM_LANES + l];
  return s;
}

__global__ void k_scal_init(int nsys_pad, int chunks, const double* part_rr, const double* part_rz,
                            const int* src_of, double* bb, double* rho, double* rr, int* active, int* flags) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsys_pad) return;
  double b2 = sum_parts(part_rr, chunks, g);
  double rz = sum_parts(part_rz, chunks, g);
  bb[g] = b2;
  rr[g] = b2;
  rho[g] = rz;
  int a = (src_of[g] >= 0 && b2 > 0.0) ? 1 : 0;
  if (a && !(isfinite(b2) && isfinite(rz))) {
    atomicOr(&flags[0], 1);
    a = 0;
  }
  active[g] = a;
}

__global__ void k_scal_alpha(int nsys_pad, int chunks, const double* part_pq, const double* rho,
                             const int* active, double* alpha, int* flags) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsys_pad) return;
  double a = 0.0;
  if (active[g]) {
    double pq = sum_parts(part_pq, chunks, g);
    if (pq > 0.0 && isfinite(pq)) a = rho[g] / pq;
    else atomicOr(&flags[0], 2);
  }
  alpha[g] = a;
}

// convergence test; counts active systems and flags active tiles
__global__ void k_scal_conv(int nsys_pad, int chunks, const double* part_rr, const double* bb, double rtol2,
                            double* rr, int* active, int* tile_active, int* counters, int* flags) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsys_pad) return;
  if (active[g]) {
    double r2 = sum_parts(part_rr, chunks, g);
    rr[g] = r2;
    if (!isfinite(r2)) {
      atomicOr(&flags[0], 1);
      active[g] = 0;
    } else if (r2 <= rtol2 * bb[g]) {
      active[g] = 0;
    }
  }
  if (active[g]) {
    atomicAdd(&counters[0], 1);
    if (atomicExch(&tile_active[g / WM_LANES], 1) == 0) atomicAdd(&counters[2], 1);
  }
}

__global__ void k_scal_beta(int nsys_pad, int chunks, const double* part_rz, const double* part_zq,
                            const double* alpha, const int* active, double* rho, double* beta, int first) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsys_pad) return;
  double rz = sum_parts(part_rz, chunks, g);
  double b = 0.0;
  if (active[g] && !first) {
    double zq = sum_parts(part_zq, chunks, g);
    double r0 = rho[g];
    if (r0 != 0.0) b = -alpha[g] * zq / r0;  // Polak–Ribiere: (z, r_new - r_old) / (z_old, r_old)
  }
  beta[g] = b;
  rho[g] = rz;
}

__global__ void k_fill_tile_active(int tiles, int* tile_active, const int* active) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tiles) return;
  int a = 0;
  for (int l = 0; l < WM_LANES; ++l) a |= active[t * WM_LANES + l];
  tile_active[t] = a;
}

// ------------------------------------------------------------ V-cycle kernels
// Chebyshev coefficients for step k on [lmax/ratio, hi*lmax]:
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

// first pre-smoothing step from z = 0: d = D^{-1} r / theta, z = d
template <typename T, typename Tr>
__global__ void k_cheb_first(int N, int chunks, const Tr* __restrict__ r, const T* __restrict__ dS,
                             const T* __restrict__ dM, const double* __restrict__ sigma,
                             const double* __restrict__ lmax, const int* __restrict__ sid, double ratio,
                             T* __restrict__ d, T* __restrict__ z, const int* __restrict__ tile_active) {
  int t = blockIdx.y;
  if (!tile_active[t]) return;
  int g = t * WM_LANES + threadIdx.x;
  T sg = (T)sigma[g];
  T c2 = (T)cheb_coef(lmax[sid[g]], ratio, 0).c2;
  RowRange rr = chunk_rows(N, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    size_t k = vidx(t, N, i);
    T dv = c2 * (T)r[k] / (dS[i] + sg * dM[i]);
    d[k] = dv;
    z[k] = dv;
  }
}

// Chebyshev step k with the residual r - A z_in:
// d = c1 d + c2 D^{-1} (r - A z_in), z_out = z_in + d
template <typename T, typename Tr>
__global__ void __launch_bounds__(256) k_cheb_step(int N, int W, int chunks, int kstep, const int32_t* __restrict__ col,
                                                   const T* __restrict__ S, const T* __restrict__ M,
                                                   const T* __restrict__ dS, const T* __restrict__ dM,
                                                   const double* __restrict__ sigma, const double* __restrict__ lmax,
                                                   const int* __restrict__ sid, double ratio, const Tr* __restrict__ r,
                                                   const T* __restrict__ zin, T* __restrict__ d, T* __restrict__ zout,
                                                   const int* __restrict__ tile_active) {
  int t = blockIdx.y;
  if (!tile_active[t]) return;
  int g = t * WM_LANES + threadIdx.x;
  T sg = (T)sigma[g];
  ChebCoef cf = cheb_coef(lmax[sid[g]], ratio, kstep);
  T c1 = (T)cf.c1, c2 = (T)cf.c2;
  const T* zt = zin + (size_t)t * N * WM_LANES;
  RowRange rr = chunk_rows(N, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    const int32_t* c = col + (size_t)i * W;
    const T* s = S + (size_t)i * W;
    const T* m = M + (size_t)i * W;
    T aS = 0, aM = 0;
    for (int w = 0; w < W; ++w) {
      T v = zt[(size_t)c[w] * WM_LANES + threadIdx.x];
      aS += s[w] * v;
      aM += m[w] * v;
    }
    size_t k = vidx(t, N, i);
    T res = (T)r[k] - (aS + sg * aM);
    T dv = (kstep == 0 ? (T)0 : c1 * d[k]) + c2 * res / (dS[i] + sg * dM[i]);
    d[k] = dv;
    zout[k] = zt[(size_t)i * WM_LANES + threadIdx.x] + dv;
  }
}

// res = r - A z
template <typename T, typename Tr>
__global__ void __launch_bounds__(256) k_residual(int N, int W, int chunks, const int32_t* __restrict__ col,
                                                  const T* __restrict__ S, const T* __restrict__ M,
                                                  const double* __restrict__ sigma, const Tr* __restrict__ r,
                                                  const T* __restrict__ z, T* __restrict__ res,
                                                  const int* __restrict__ tile_active) {
  int t = blockIdx.y;
  if (!tile_active[t]) return;
  T sg = (T)sigma[t * WM_LANES + threadIdx.x];
  const T* zt = z + (size_t)t * N * WM_LANES;
  RowRange rr = chunk_rows(N, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    const int32_t* c = col + (size_t)i * W;
    const T* s = S + (size_t)i * W;
    const T* m = M + (size_t)i * W;
    T aS = 0, aM = 0;
    for (int w = 0; w < W; ++w) {
      T v = zt[(size_t)c[w] * WM_LANES + threadIdx.x];
      aS += s[w] * v;
      aM += m[w] * v;
    }
    size_t k = vidx(t, N, i);
    res[k] = (T)r[k] - (aS + sg * aM);
  }
}

// z = A_c^{-1} r on the coarsest level, in float64, with the inverse of the
// system's shift
template <typename T, typename Tr>
__global__ void k_coarse_solve(int N, const double* __restrict__ Ainv, const int* __restrict__ sid,
                               const Tr* __restrict__ r, T* __restrict__ z, const int* __restrict__ tile_active) {
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

// power iteration helpers for lambda_max(D^{-1}(S + sigma M))
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
__global__ void __launch_bounds__(256) k_power_step(int N, int W, int chunks, const int32_t* __restrict__ col,
                                                    const double* __restrict__ S, const double* __restrict__ M,
                                                    const double* __restrict__ dS, const double* __restrict__ dM,
                                                    const double* __restrict__ sigma, const double* __restrict__ v,
                                                    double* __restrict__ w, double* part_ww, double* part_vv) {
  int t = blockIdx.y;
  double sg = sigma[t * WM_LANES + threadIdx.x];
  const double* vt = v + (size_t)t * N * WM_LANES;
  RowRange rr = chunk_rows(N, chunks);
  double acc[2] = {0.0, 0.0};
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) {
    const int32_t* c = col + (size_t)i * W;
    double aS = 0.0, aM = 0.0;
    for (int k = 0; k < W; ++k) {
      double x = vt[(size_t)c[k] * WM_LANES + threadIdx.x];
      aS += S[(size_t)i * W + k] * x;
      aM += M[(size_t)i * W + k] * x;
    }
    double wv = (aS + sg * aM) / (dS[i] + sg * dM[i]);
    w[vidx(t, N, i)] = wv;
    double vv = vt[(size_t)i * WM_LANES + threadIdx.x];
    acc[0] += wv * wv;
    acc[1] += vv * vv;
  }
  double* parts[2] = {part_ww, part_vv};
  block_reduce_store<2>(acc, parts, chunks);
}

__global__ void k_power_scale(int N, int chunks, const double* part_ww, double* w) {
  int t = blockIdx.y;
  int g = t * WM_LANES + threadIdx.x;
  double nw = sqrt(sum_parts(part_ww, chunks, g));
  double inv = nw > 0 ? 1.0 / nw : 0.0;
  RowRange rr = chunk_rows(N, chunks);
  for (int i = rr.i0 + threadIdx.y; i < rr.i1; i += kWarps) w[vidx(t, N, i)] *= inv;
}

__global__ void k_power_final(int nshift, int chunks, const double* part_ww, const double* part_vv,
                              double* lmax) {
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
  int jlo = (g0 - s + ns - 1) / ns;
  if (g0 - s <= 0) jlo = 0;
  int jhi = (g1 - 1 - s) / ns;
  if (g1 - 1 - s < 0) return;
  for (int i = blockIdx.x * kWarps + threadIdx.y; i < N; i += gridDim.x * kWarps) {
    double acc = 0.0;
    for (int j = jlo; j <= jhi; ++j) {
      int gg = j * ns + s - g0;
      acc += c[j] * x[((size_t)(gg / WM_LANES) * N + i) * WM_LANES + (gg % WM_LANES)];
    }
    v[((size_t)st * N + i) * WM_LANES + threadIdx.x] += acc;
  }
}

// copy x of systems g = s (one node) into a sample-tiled buffer
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

}  // namespace

// ====================================================================== host
// algorithmic bytes/flops of a launch over the active tiles: `b` bytes and `f`
// flops per system of one tile
static inline void units(int cat, const Batch& bt, double b, double f) {
  double sys = (double)bt.active_tiles * WM_LANES;
  wm_prof_units(cat, b * sys, f * sys);
}
int Batch::chunks_for(int N) const {
  // enough blocks to cover the GPU several times, at least 64 rows per chunk
  int target = std::max(1, (152 * 8 + tiles - 1) / std::max(1, tiles));
  int maxc = std::max(1, (N + 63) / 64);
  return std::min(std::min(target, maxc), 64);
}

template <typename T>
static T* lvbuf(VBuf& b);
template <>
double* lvbuf<double>(VBuf& b) { return b.d.p; }
template <>
float* lvbuf<float>(VBuf& b) { return b.f.p; }

int VBuf::alloc(size_t n, bool dbl) {
  if (dbl) return d.alloc(n);
  return f.alloc(n);
}

int WorkSpace::reserve(const wm_hier* h, int tiles, int nshift, bool dbl) {
  const int L = (int)h->lv.size();
  size_t n0 = (size_t)tiles * h->lv[0].N * WM_LANES;
  WM_TRY(x.alloc(n0));
  WM_TRY(r.alloc(n0));
  WM_TRY(p.alloc(n0));
  WM_TRY(q.alloc(n0));
  lvl.resize(L);
  for (int l = 0; l < L; ++l) {
    size_t n = (size_t)tiles * h->lv[l].N * WM_LANES;
    WM_TRY(lvl[l].za.alloc(n, dbl));
    WM_TRY(lvl[l].zb.alloc(n, dbl));
    if (l < L - 1) {
      WM_TRY(lvl[l].d.alloc(n, dbl));
      WM_TRY(lvl[l].res.alloc(n, dbl));
    }
    if (l > 0) WM_TRY(lvl[l].r.alloc(n, dbl));
  }
  size_t ns = (size_t)tiles * WM_LANES;
  WM_TRY(sigma.alloc(ns));
  WM_TRY(sid.alloc(ns));
  WM_TRY(src_of.alloc(ns));
  WM_TRY(active.alloc(ns));
  WM_TRY(tile_active.alloc(tiles));
  WM_TRY(rho.alloc(ns));
  WM_TRY(alpha.alloc(ns));
  WM_TRY(beta.alloc(ns));
  WM_TRY(bb.alloc(ns));
  WM_TRY(rr.alloc(ns));
  size_t np = (size_t)std::max(tiles, (nshift + WM_LANES - 1) / WM_LANES) * 64 * WM_LANES;
  for (int k = 0; k < 3; ++k) WM_TRY(part[k].alloc(np));
  WM_TRY(flags.alloc(4));
  WM_TRY(counters.alloc(4));
  WM_TRY(lmax.alloc((size_t)L * std::max(1, nshift)));
  const wm_level& C = h->lv[L - 1];
  WM_TRY(ainv.alloc((size_t)std::max(1, nshift) * C.N * C.N));
  WM_TRY(shifts.alloc(std::max(1, nshift)));
  WM_TRY(statd.alloc(2));
  if (!host_small) {
    WM_CUDA(cudaMallocHost((void**)&host_small, 64));
  }
  return WM_OK;
}

void WorkSpace::release() {
  x.release(); r.release(); p.release(); q.release();
  for (auto& l : lvl) {
    l.za.d.release(); l.za.f.release(); l.zb.d.release(); l.zb.f.release();
    l.d.d.release(); l.d.f.release(); l.res.d.release(); l.res.f.release();
    l.r.d.release(); l.r.f.release();
  }
  lvl.clear();
  sigma.release(); sid.release(); src_of.release(); active.release(); tile_active.release();
  rho.release(); alpha.release(); beta.release(); bb.release(); rr.release();
  for (auto& pp : part) pp.release();
  flags.release(); counters.release(); lmax.release(); ainv.release(); shifts.release(); statd.release();
  for (auto& b : samp) b.release();
  noise_scratch.release();
  pw_v.release(); pw_w.release(); pw_sigma.release();
  if (host_small) cudaFreeHost(host_small);
  host_small = nullptr;
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
      WM_LAUNCH(WM_PC_SETUP, s, k_power_step<<<dim3(ch, tiles), kBlk, 0, s>>>(Lv.N, Lv.W, ch, Lv.d_col.p, Lv.d_S64.p, Lv.d_M64.p,
                                                    Lv.d_dS64.p, Lv.d_dM64.p, ws.pw_sigma.p, v, w, ws.part[0].p,
                                                    ws.part[1].p));
      if (it < 14) WM_LAUNCH(WM_PC_SETUP, s, k_power_scale<<<dim3(ch, tiles), kBlk, 0, s>>>(Lv.N, ch, ws.part[0].p, w));
      std::swap(v, w);
    }
    WM_LAUNCH(WM_PC_SETUP, s, k_power_final<<<nblk(nsh, 128), 128, 0, s>>>(nsh, ch, ws.part[0].p, ws.part[1].p, ws.lmax.p + (size_t)l * nsh));
    WM_CUDA(cudaGetLastError());
  }
  return WM_OK;
}

int wm_prepare_shifts(const wm_hier* h, WorkSpace& ws, const std::vector<double>& shifts, cudaStream_t s) {
  int nsh = (int)shifts.size();
  WM_TRY(ws.shifts.upload(shifts, s));
  WM_TRY(estimate_lmax(h, ws, shifts, s));
  const wm_level& C = h->lv.back();
  size_t smem = ((size_t)C.N * C.N + C.N) * sizeof(double);
  if (smem > 220 * 1024) {
    wm_set_error("coarsest level has %d DOFs; at most 160 supported (use more levels)", C.N);
    return WM_ERR_UNSUPPORTED;
  }
  WM_CUDA(cudaFuncSetAttribute(k_coarse_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  WM_LAUNCH(WM_PC_SETUP, s, k_coarse_inverse<<<nsh, 256, smem, s>>>(C.N, C.d_Sdense.p, C.d_Mdense.p, ws.shifts.p, ws.ainv.p));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// one V-cycle from level l: input residual rin (level 0: float64 outer residual
// or the level's own buffer), returns the buffer holding z
template <typename T>
static int vcycle(const wm_hier* h, WorkSpace& ws, const Batch& bt, int l, const void* rin, bool rin_double,
                  T** zout, cudaStream_t s) {
  const int L = (int)h->lv.size();
  const wm_level& Lv = h->lv[l];
  LevelBufs& B = ws.lvl[l];
  const int* ta = ws.tile_active.p;
  int tiles = bt.tiles;
  int ch = bt.chunks_for(Lv.N);
  dim3 grid(ch, tiles);
  const double* lmax = ws.lmax.p + (size_t)l * bt.nshift;
  const T* S = std::is_same<T, double>::value ? (const T*)Lv.d_S64.p : (const T*)Lv.d_S32.p;
  const T* M = std::is_same<T, double>::value ? (const T*)Lv.d_M64.p : (const T*)Lv.d_M32.p;
  const T* dS = std::is_same<T, double>::value ? (const T*)Lv.d_dS64.p : (const T*)Lv.d_dS32.p;
  const T* dM = std::is_same<T, double>::value ? (const T*)Lv.d_dM64.p : (const T*)Lv.d_dM32.p;
  T* za = lvbuf<T>(B.za);
  T* zb = lvbuf<T>(B.zb);
  const double Rb = rin_double ? 8.0 : (double)sizeof(T), Tb = (double)sizeof(T);
  const int csm = l == 0 ? WM_PC_SMOOTH0 : WM_PC_SMOOTHC;
  const int cre = l == 0 ? WM_PC_RESID0 : WM_PC_RESIDC;
  if (l == L - 1) {
    int gx = std::max(1, std::min(64, (Lv.N + kWarps - 1) / kWarps));
    if (rin_double) {
      WM_LAUNCH(WM_PC_COARSE, s, k_coarse_solve<T, double><<<dim3(gx, tiles), kBlk, 0, s>>>(
                                     Lv.N, ws.ainv.p, ws.sid.p, (const double*)rin, za, ta));
    } else {
      WM_LAUNCH(WM_PC_COARSE, s, k_coarse_solve<T, T><<<dim3(gx, tiles), kBlk, 0, s>>>(
                                     Lv.N, ws.ainv.p, ws.sid.p, (const T*)rin, za, ta));
    }
    units(WM_PC_COARSE, bt, (Rb + Tb) * Lv.N, 2.0 * Lv.N * Lv.N);
    WM_CUDA(cudaGetLastError());
    *zout = za;
    return WM_OK;
  }
  T* d = lvbuf<T>(B.d);
  T* res = lvbuf<T>(B.res);
  int nu = bt.degree;
  double ratio = bt.cheb_ratio;
  auto cheb_step = [&](int k, const T* zin, T* zo) {
    if (rin_double) {
      WM_LAUNCH(csm, s, k_cheb_step<T, double><<<grid, kBlk, 0, s>>>(Lv.N, Lv.W, ch, k, Lv.d_col.p, S, M, dS, dM,
                                                                     ws.sigma.p, lmax, ws.sid.p, ratio,
                                                                     (const double*)rin, zin, d, zo, ta));
    } else {
      WM_LAUNCH(csm, s, k_cheb_step<T, T><<<grid, kBlk, 0, s>>>(Lv.N, Lv.W, ch, k, Lv.d_col.p, S, M, dS, dM,
                                                                ws.sigma.p, lmax, ws.sid.p, ratio, (const T*)rin,
                                                                zin, d, zo, ta));
    }
    units(csm, bt, (Rb + 4.0 * Tb) * Lv.N, 4.0 * Lv.nnz + 8.0 * Lv.N);
  };
  // pre-smoothing from z = 0
  if (rin_double) {
    WM_LAUNCH(csm, s, k_cheb_first<T, double><<<grid, kBlk, 0, s>>>(Lv.N, ch, (const double*)rin, dS, dM, ws.sigma.p,
                                                                    lmax, ws.sid.p, ratio, d, za, ta));
  } else {
    WM_LAUNCH(csm, s, k_cheb_first<T, T><<<grid, kBlk, 0, s>>>(Lv.N, ch, (const T*)rin, dS, dM, ws.sigma.p, lmax,
                                                               ws.sid.p, ratio, d, za, ta));
  }
  units(csm, bt, (Rb + 2.0 * Tb) * Lv.N, 4.0 * Lv.N);
  T* cur = za;
  T* oth = zb;
  for (int k = 1; k < nu; ++k) {
    cheb_step(k, cur, oth);
    std::swap(cur, oth);
  }
  // residual, restriction, coarse correction
  if (rin_double) {
    WM_LAUNCH(cre, s, k_residual<T, double><<<grid, kBlk, 0, s>>>(Lv.N, Lv.W, ch, Lv.d_col.p, S, M, ws.sigma.p,
                                                                  (const double*)rin, cur, res, ta));
  } else {
    WM_LAUNCH(cre, s, k_residual<T, T><<<grid, kBlk, 0, s>>>(Lv.N, Lv.W, ch, Lv.d_col.p, S, M, ws.sigma.p,
                                                             (const T*)rin, cur, res, ta));
  }
  units(cre, bt, (Rb + 2.0 * Tb) * Lv.N, 4.0 * Lv.nnz + 3.0 * Lv.N);
  WM_CUDA(cudaGetLastError());
  T* rc = lvbuf<T>(ws.lvl[l + 1].r);
  WM_TRY(wm_k_restrict<T>(Lv, tiles, res, rc, ta, s));
  units(WM_PC_RESTRICT, bt, Tb * (Lv.N + h->lv[l + 1].N), 2.0 * Lv.nnzP);
  T* zc = nullptr;
  WM_TRY(vcycle<T>(h, ws, bt, l + 1, rc, false, &zc, s));
  WM_TRY(wm_k_prolong_add<T>(Lv, tiles, zc, cur, ta, s));
  units(WM_PC_PROLONG, bt, Tb * (2.0 * Lv.N + h->lv[l + 1].N), 2.0 * Lv.nnzP);
  // post-smoothing
  for (int k = 0; k < nu; ++k) {
    cheb_step(k, cur, oth);
    std::swap(cur, oth);
  }
  WM_CUDA(cudaGetLastError());
  *zout = cur;
  return WM_OK;
}

template <typename T>
static int precondition(const wm_hier* h, WorkSpace& ws, const Batch& bt, T** z, cudaStream_t s) {
  return vcycle<T>(h, ws, bt, 0, ws.r.p, true, z, s);
}

// Batched flexible CG on the systems of `bt` (metadata already uploaded).
template <typename T>
static int fcg(const wm_hier* h, WorkSpace& ws, const Batch& bt, const double* rhs_tiled, BatchResult* res,
               cudaStream_t s) {
  const wm_level& L0 = h->lv[0];
  int N = L0.N, tiles = bt.tiles;
  int ch = bt.chunks_for(N);
  dim3 grid(ch, tiles);
  int nsys_pad = tiles * WM_LANES;
  unsigned sb = nblk(nsys_pad, 128);
  WM_CUDA(cudaMemsetAsync(ws.flags.p, 0, 4 * sizeof(int), s));
  WM_LAUNCH(WM_PC_CGVEC, s, k_gather_rhs<<<grid, kBlk, 0, s>>>(N, ch, rhs_tiled, ws.src_of.p, ws.r.p, ws.x.p, ws.part[0].p));
  WM_CUDA(cudaGetLastError());
  bt.active_tiles = tiles;
  units(WM_PC_CGVEC, bt, 24.0 * N, 2.0 * N);
  // all tiles active for the first preconditioner application
  {
    std::vector<int> ones(tiles, 1);
    WM_CUDA(cudaMemcpyAsync(ws.tile_active.p, ones.data(), tiles * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  T* z = nullptr;
  WM_TRY(precondition<T>(h, ws, bt, &z, s));
  WM_LAUNCH(WM_PC_CGVEC, s, k_dots_rz_zq<T><<<grid, kBlk, 0, s>>>(N, ch, ws.r.p, z, nullptr, ws.tile_active.p, ws.part[1].p, ws.part[2].p));
  WM_LAUNCH(WM_PC_SCALAR, s, k_scal_init<<<sb, 128, 0, s>>>(nsys_pad, ch, ws.part[0].p, ws.part[1].p, ws.src_of.p, ws.bb.p, ws.rho.p, ws.rr.p,
                                 ws.active.p, ws.flags.p));
  WM_LAUNCH(WM_PC_SCALAR, s, k_fill_tile_active<<<nblk(tiles, 128), 128, 0, s>>>(tiles, ws.tile_active.p, ws.active.p));
  WM_CUDA(cudaGetLastError());
  // p = z
  WM_CUDA(cudaMemsetAsync(ws.beta.p, 0, nsys_pad * sizeof(double), s));
  WM_LAUNCH(WM_PC_CGVEC, s, k_update_p<T><<<grid, kBlk, 0, s>>>(N, ch, ws.beta.p, z, ws.p.p, ws.tile_active.p));
  double rtol2 = bt.rtol * bt.rtol;
  int it = 0;
  int n_active = nsys_pad;
  for (it = 1; it <= bt.max_iter; ++it) {
    WM_LAUNCH(WM_PC_APPLY64, s, k_apply_pq<<<grid, kBlk, 0, s>>>(N, L0.W, ch, L0.d_col.p, L0.d_S64.p, L0.d_M64.p, ws.sigma.p, ws.p.p, ws.q.p,
                                     ws.tile_active.p, ws.part[0].p));
    units(WM_PC_APPLY64, bt, 16.0 * N, 4.0 * L0.nnz + 4.0 * N);
    WM_LAUNCH(WM_PC_SCALAR, s, k_scal_alpha<<<sb, 128, 0, s>>>(nsys_pad, ch, ws.part[0].p, ws.rho.p, ws.active.p, ws.alpha.p, ws.flags.p));
    WM_LAUNCH(WM_PC_CGVEC, s, k_update_xr<<<grid, kBlk, 0, s>>>(N, ch, ws.alpha.p, ws.p.p, ws.q.p, ws.x.p, ws.r.p, ws.tile_active.p,
                                      ws.part[0].p));
    units(WM_PC_CGVEC, bt, 48.0 * N, 6.0 * N);
    WM_CUDA(cudaMemsetAsync(ws.counters.p, 0, 3 * sizeof(int), s));
    // tiles stay flagged until all their lanes have converged
    WM_CUDA(cudaMemsetAsync(ws.tile_active.p, 0, tiles * sizeof(int), s));
    WM_LAUNCH(WM_PC_SCALAR, s, k_scal_conv<<<sb, 128, 0, s>>>(nsys_pad, ch, ws.part[0].p, ws.bb.p, rtol2, ws.rr.p, ws.active.p,
                                   ws.tile_active.p, ws.counters.p, ws.flags.p));
    WM_CUDA(cudaGetLastError());
    WM_CUDA(cudaMemcpyAsync(ws.host_small, ws.counters.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    WM_CUDA(cudaStreamSynchronize(s));
    n_active = ws.host_small[0];
    bt.active_tiles = ws.host_small[2];
    if (n_active == 0) break;
    WM_TRY(precondition<T>(h, ws, bt, &z, s));
    WM_LAUNCH(WM_PC_CGVEC, s, k_dots_rz_zq<T><<<grid, kBlk, 0, s>>>(N, ch, ws.r.p, z, ws.q.p, ws.tile_active.p, ws.part[1].p, ws.part[2].p));
    units(WM_PC_CGVEC, bt, (16.0 + sizeof(T)) * N, 4.0 * N);
    WM_LAUNCH(WM_PC_SCALAR, s, k_scal_beta<<<sb, 128, 0, s>>>(nsys_pad, ch, ws.part[1].p, ws.part[2].p, ws.alpha.p, ws.active.p, ws.rho.p,
                                   ws.beta.p, 0));
    WM_LAUNCH(WM_PC_CGVEC, s, k_update_p<T><<<grid, kBlk, 0, s>>>(N, ch, ws.beta.p, z, ws.p.p, ws.tile_active.p));
    units(WM_PC_CGVEC, bt, (16.0 + sizeof(T)) * N, 2.0 * N);
    WM_CUDA(cudaGetLastError());
  }
  res->iterations = std::min(it, bt.max_iter);
  WM_LAUNCH(WM_PC_SCALAR, s, k_reduce_stats<<<1, 256, 0, s>>>(bt.nsys, ws.rr.p, ws.bb.p, ws.active.p, ws.statd.p, ws.counters.p + 1));
  WM_CUDA(cudaMemcpyAsync(ws.host_small + 2, ws.counters.p + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  WM_CUDA(cudaMemcpyAsync(ws.host_small + 4, ws.flags.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  double maxrel = 0.0;
  WM_CUDA(cudaMemcpyAsync(&ws.host_d, ws.statd.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  WM_CUDA(cudaStreamSynchronize(s));
  maxrel = ws.host_d;
  res->n_not_converged = ws.host_small[2];
  res->max_rel_residual = maxrel;
  res->flags = ws.host_small[4];
  return WM_OK;
}

int wm_solve_batch(const wm_hier* h, WorkSpace& ws, const Batch& bt, const double* rhs_tiled, BatchResult* res,
                   cudaStream_t s) {
  if (bt.precision == WM_FP64) return fcg<double>(h, ws, bt, rhs_tiled, res, s);
  return fcg<float>(h, ws, bt, rhs_tiled, res, s);
}

int wm_vcycle_apply(const wm_hier* h, WorkSpace& ws, const Batch& bt, cudaStream_t s) {
  // z of one V-cycle on ws.r into ws.q (float64)
  size_t n = (size_t)bt.tiles * h->lv[0].N * WM_LANES;
  std::vector<int> ones(bt.tiles, 1);
  WM_CUDA(cudaMemcpyAsync(ws.tile_active.p, ones.data(), bt.tiles * sizeof(int), cudaMemcpyHostToDevice, s));
  WM_CUDA(cudaStreamSynchronize(s));
  if (bt.precision == WM_FP64) {
    double* z = nullptr;
    WM_TRY(precondition<double>(h, ws, bt, &z, s));
    WM_LAUNCH(WM_PC_SINC, s, k_copy_tiles<<<nblk(n, 256), 256, 0, s>>>(n, z, ws.q.p));
  } else {
    float* z = nullptr;
    WM_TRY(precondition<float>(h, ws, bt, &z, s));
    WM_LAUNCH(WM_PC_SINC, s, k_widen<float><<<nblk(n, 256), 256, 0, s>>>(n, z, ws.q.p));
  }
  WM_CUDA(cudaGetLastError());
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
