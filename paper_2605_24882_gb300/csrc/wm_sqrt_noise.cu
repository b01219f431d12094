// White-noise loads f = sqrt(M) y by the Hale–Higham–Trefethen sum (Sec. 3.3,
// Eq. eq:sqrt):  sqrt(M) y ~= M sum_k c_k (M + w_k^2 I)^{-1} y,  y ~ N(0, I).
//
// All shifted systems of all nodes k and samples s are solved at once by
// float64 conjugate gradients with Jacobi preconditioning.  Systems are
// packed 32 to a tile, node-major: tile T = k * tc + j holds samples
// 32 j .. 32 j + 31 (of the current sample chunk) for node k, so every node's
// block of tiles has the layout of the sample tiles and the weighted sum over
// k is an elementwise pass.  The condition number of M + w^2 I is at most that
// of M (a few hundred for p <= 3), so CG converges in tens of iterations
// without a multigrid preconditioner.
//
// Row kernels: one warp per (tile, row), lane = system, rows in chunks of
// kRows per block; each block reduces its per-lane partial dot products over
// its warps in a fixed order into part[chunk][tile][lane], and the scalar
// kernels sum the chunks in order (deterministic results).
#include <cmath>
#include <vector>

#include "wm_internal.h"

namespace {

constexpr int kWarps = 8;
constexpr int kRowIters = 16;
constexpr int kRows = kWarps * kRowIters;  // rows per block
constexpr int kNormalStream = 2;           // Philox stream id of the DOF normals y

template <typename T>
struct Buf : DevBuf<T> {
  ~Buf() { this->release(); }
};

__device__ __forceinline__ void block_partial(double acc, double* __restrict__ part, size_t slot) {
  __shared__ double sh[kWarps][WM_LANES];
  sh[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += sh[w][threadIdx.x];
    part[slot + threadIdx.x] = s;
  }
}

// x = 0, r = y (of the tile's sample tile), z = D^{-1} r, p = z; partial (r, z)
__global__ void __launch_bounds__(256) k_sq_init(int N, int tc, const double* __restrict__ ybuf,
                                                 const double* __restrict__ dM, const double* __restrict__ w2node,
                                                 double* __restrict__ x, double* __restrict__ r,
                                                 double* __restrict__ z, double* __restrict__ p,
                                                 double* __restrict__ part) {
  const int T = blockIdx.y, l = threadIdx.x;
  const int j = T % tc, k = T / tc;
  const double w2 = w2node[k];
  double acc = 0.0;
  for (int it = 0; it < kRowIters; ++it) {
    const int i = blockIdx.x * kRows + it * kWarps + threadIdx.y;
    if (i >= N) break;
    const size_t o = ((size_t)T * N + i) * WM_LANES + l;
    const double yv = ybuf[((size_t)j * N + i) * WM_LANES + l];
    const double zv = yv / (dM[i] + w2);
    x[o] = 0.0;
    r[o] = yv;
    z[o] = zv;
    p[o] = zv;
    acc += yv * zv;
  }
  block_partial(acc, part, ((size_t)blockIdx.x * gridDim.y + T) * WM_LANES);
}

// q = (M + w_k^2 I) p; partial (p, q)
__global__ void __launch_bounds__(256) k_sq_apply(int N, int W, int tc, const int32_t* __restrict__ col,
                                                  const double* __restrict__ M, const double* __restrict__ w2node,
                                                  const double* __restrict__ p, double* __restrict__ q,
                                                  double* __restrict__ part) {
  const int T = blockIdx.y, l = threadIdx.x;
  const double w2 = w2node[T / tc];
  const double* pt = p + (size_t)T * N * WM_LANES;
  double acc = 0.0;
  for (int it = 0; it < kRowIters; ++it) {
    const int i = blockIdx.x * kRows + it * kWarps + threadIdx.y;
    if (i >= N) break;
    const int32_t* c = col + (size_t)i * W;
    const double* m = M + (size_t)i * W;
    double s = 0.0;
    for (int w = 0; w < W; ++w) s += m[w] * pt[(size_t)c[w] * WM_LANES + l];
    const double pv = pt[(size_t)i * WM_LANES + l];
    const double qv = s + w2 * pv;
    q[((size_t)T * N + i) * WM_LANES + l] = qv;
    acc += pv * qv;
  }
  block_partial(acc, part, ((size_t)blockIdx.x * gridDim.y + T) * WM_LANES);
}

// x += alpha p, r -= alpha q, z = D^{-1} r; partial (r, z)
__global__ void __launch_bounds__(256) k_sq_update(int N, int tc, const double* __restrict__ dM,
                                                   const double* __restrict__ w2node,
                                                   const double* __restrict__ alpha, const double* __restrict__ p,
                                                   const double* __restrict__ q, double* __restrict__ x,
                                                   double* __restrict__ r, double* __restrict__ z,
                                                   double* __restrict__ part) {
  const int T = blockIdx.y, l = threadIdx.x;
  const double w2 = w2node[T / tc];
  const double a = alpha[(size_t)T * WM_LANES + l];
  double acc = 0.0;
  for (int it = 0; it < kRowIters; ++it) {
    const int i = blockIdx.x * kRows + it * kWarps + threadIdx.y;
    if (i >= N) break;
    const size_t o = ((size_t)T * N + i) * WM_LANES + l;
    x[o] += a * p[o];
    const double rv = r[o] - a * q[o];
    const double zv = rv / (dM[i] + w2);
    r[o] = rv;
    z[o] = zv;
    acc += rv * zv;
  }
  block_partial(acc, part, ((size_t)blockIdx.x * gridDim.y + T) * WM_LANES);
}

// p = z + beta p
__global__ void k_sq_direction(size_t n, const double* __restrict__ beta, const double* __restrict__ z,
                               double* __restrict__ p, int N) {
  size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (o >= n) return;
  const size_t T = o / ((size_t)N * WM_LANES);
  const int l = (int)(o % WM_LANES);
  p[o] = z[o] + beta[T * WM_LANES + l] * p[o];
}

__device__ __forceinline__ double chunk_sum(const double* __restrict__ part, int nchunk, int nsys, int g) {
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * nsys + g];
  return s;
}

// rz0 = rz = (r, z); a system with a zero right-hand side is done at once
__global__ void k_sq_start(int nsys, int nchunk, const double* __restrict__ part, double* __restrict__ rz,
                           double* __restrict__ rz0, int* __restrict__ active, int* __restrict__ flags) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsys) return;
  const double v = chunk_sum(part, nchunk, nsys, g);
  rz[g] = v;
  rz0[g] = v;
  if (!isfinite(v)) atomicOr(flags, 1);
  active[g] = (v > 0.0 && isfinite(v)) ? 1 : 0;
}

// alpha = (r, z) / (p, q) for active systems, 0 otherwise
__global__ void k_sq_alpha(int nsys, int nchunk, const double* __restrict__ part, const double* __restrict__ rz,
                           const int* __restrict__ active, double* __restrict__ alpha, int* __restrict__ flags) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsys) return;
  const double pq = chunk_sum(part, nchunk, nsys, g);
  double a = 0.0;
  if (active[g]) {
    if (pq > 0.0 && isfinite(pq)) {
      a = rz[g] / pq;
    } else {
      atomicOr(flags, 1);
    }
  }
  alpha[g] = a;
}

// new (r, z): convergence test sqrt(rz / rz0) <= rtol, beta, count of active systems
__global__ void k_sq_beta(int nsys, int nchunk, const double* __restrict__ part, double* __restrict__ rz,
                          const double* __restrict__ rz0, double tol2, int* __restrict__ active,
                          double* __restrict__ beta, int* __restrict__ n_active, int* __restrict__ flags) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsys) return;
  const double v = chunk_sum(part, nchunk, nsys, g);
  double b = 0.0;
  if (active[g]) {
    if (!isfinite(v)) {
      atomicOr(flags, 1);
      active[g] = 0;
    } else if (v <= tol2 * rz0[g]) {
      active[g] = 0;
    } else {
      b = v / rz[g];
      atomicAdd(n_active, 1);
    }
    rz[g] = v;
  }
  beta[g] = b;
}

// acc = sum_k c_k x_k over the node blocks (same tile layout as the samples)
__global__ void k_sq_combine(size_t n_block, int n_nodes, const double* __restrict__ cnode,
                             const double* __restrict__ x, double* __restrict__ acc) {
  size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (o >= n_block) return;
  double s = 0.0;
  for (int k = 0; k < n_nodes; ++k) s += cnode[k] * x[(size_t)k * n_block + o];
  acc[o] = s;
}

inline unsigned blocks_for(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

bool on_device(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int wm_noise_loads_sqrt(wm_hier_t h, uint64_t seed, int n_samples, double lo, double hi, int n_nodes,
                                   double rtol, int max_iter, double* f, int* iterations, void* stream) {
  if (iterations) *iterations = 0;
  if (!h || h->lv.empty() || n_samples < 0 || n_nodes < 1 || !(rtol > 0.0) || max_iter < 1) {
    wm_set_error("sqrt noise needs a hierarchy, n_samples >= 0, n_nodes >= 1, rtol > 0, max_iter >= 1");
    return WM_ERR_INVALID_ARG;
  }
  if (n_samples == 0) return WM_OK;
  if (!f || !on_device(f)) {
    wm_set_error("sqrt noise writes a device buffer");
    return WM_ERR_INVALID_ARG;
  }
  std::vector<double> w2(n_nodes), c(n_nodes);
  WM_TRY(wm_hht_rule(lo, hi, n_nodes, w2.data(), c.data()));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const wm_level& L = h->lv[0];
  const int N = L.N;
  const int ts = (n_samples + WM_LANES - 1) / WM_LANES;
  // sample tiles per pass: five CG vectors per system within half the free memory
  size_t free_b = 0, total_b = 0;
  WM_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t per_tile = (size_t)n_nodes * N * WM_LANES * sizeof(double) * 5 + (size_t)N * WM_LANES * sizeof(double) * 4;
  int tc = (int)std::min<size_t>((size_t)ts, std::max<size_t>(1, (free_b / 2) / per_tile));
  tc = std::min(tc, 65535 / n_nodes);
  if (tc < 1) {
    wm_set_error("too many nodes for one launch grid");
    return WM_ERR_INVALID_ARG;
  }
  const int n_tiles = n_nodes * tc, nsys = n_tiles * WM_LANES;
  const int nchunk = (N + kRows - 1) / kRows;
  const size_t nvec = (size_t)n_tiles * N * WM_LANES, nblk = (size_t)tc * N * WM_LANES;
  Buf<double> x, r, z, p, q, ybuf, yrows, acc, ftile, part, rz, rz0, alpha, beta, d_w2, d_c;
  Buf<int> active, counters;
  WM_TRY(x.alloc(nvec));
  WM_TRY(r.alloc(nvec));
  WM_TRY(z.alloc(nvec));
  WM_TRY(p.alloc(nvec));
  WM_TRY(q.alloc(nvec));
  WM_TRY(ybuf.alloc(nblk));
  WM_TRY(yrows.alloc((size_t)tc * WM_LANES * N));
  WM_TRY(acc.alloc(nblk));
  WM_TRY(ftile.alloc(nblk));
  WM_TRY(part.alloc((size_t)nchunk * nsys));
  WM_TRY(rz.alloc(nsys));
  WM_TRY(rz0.alloc(nsys));
  WM_TRY(alpha.alloc(nsys));
  WM_TRY(beta.alloc(nsys));
  WM_TRY(active.alloc(nsys));
  WM_TRY(counters.alloc(2));  // [0] active systems after the last step, [1] non-finite flag
  WM_TRY(d_w2.upload(w2, s));
  WM_TRY(d_c.upload(c, s));
  const double tol2 = rtol * rtol;
  const dim3 rgrid((unsigned)nchunk, (unsigned)n_tiles), rblock(WM_LANES, kWarps);
  const unsigned sgrid = blocks_for((size_t)nsys, 256);
  int worst_iters = 0;
  bool not_converged = false;
  for (int t0 = 0; t0 < ts; t0 += tc) {
    const int tcur = std::min(tc, ts - t0);  // sample tiles of this pass; unused tiles get zero rhs
    const int s0 = t0 * WM_LANES, ns = std::min(n_samples - s0, tcur * WM_LANES);
    for (int si = 0; si < ns; ++si)
      WM_TRY(wm_k_normals(seed, s0 + si, kNormalStream, 0, N, yrows.p + (size_t)si * N, s));
    WM_TRY(wm_k_to_tiled(yrows.p, ns, N, ybuf.p, tc, s));
    WM_CUDA(cudaMemsetAsync(counters.p, 0, 2 * sizeof(int), s));
    WM_LAUNCH(WM_PC_NOISE, s, k_sq_init<<<rgrid, rblock, 0, s>>>(N, tc, ybuf.p, L.d_dM64.p, d_w2.p, x.p, r.p, z.p, p.p,
                                                                 part.p));
    WM_LAUNCH(WM_PC_NOISE, s, k_sq_start<<<sgrid, 256, 0, s>>>(nsys, nchunk, part.p, rz.p, rz0.p, active.p,
                                                               counters.p + 1));
    int it = 0, host_active = 1;
    while (it < max_iter && host_active > 0) {
      ++it;
      WM_LAUNCH(WM_PC_NOISE, s, k_sq_apply<<<rgrid, rblock, 0, s>>>(N, L.W, tc, L.d_col.p, L.d_M64.p, d_w2.p, p.p,
                                                                    q.p, part.p));
      WM_LAUNCH(WM_PC_NOISE, s, k_sq_alpha<<<sgrid, 256, 0, s>>>(nsys, nchunk, part.p, rz.p, active.p, alpha.p,
                                                                 counters.p + 1));
      WM_LAUNCH(WM_PC_NOISE, s, k_sq_update<<<rgrid, rblock, 0, s>>>(N, tc, L.d_dM64.p, d_w2.p, alpha.p, p.p, q.p,
                                                                     x.p, r.p, z.p, part.p));
      WM_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(int), s));
      WM_LAUNCH(WM_PC_NOISE, s, k_sq_beta<<<sgrid, 256, 0, s>>>(nsys, nchunk, part.p, rz.p, rz0.p, tol2, active.p,
                                                                beta.p, counters.p, counters.p + 1));
      WM_LAUNCH(WM_PC_NOISE, s, k_sq_direction<<<blocks_for(nvec, 256), 256, 0, s>>>(nvec, beta.p, z.p, p.p, N));
      WM_CUDA(cudaGetLastError());
      if (it % 4 == 0 || it == max_iter) {
        int hc[2] = {0, 0};
        WM_CUDA(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
        WM_CUDA(cudaStreamSynchronize(s));
        if (hc[1]) {
          wm_set_error("non-finite value in the sqrt(M) solves");
          return WM_ERR_NONFINITE;
        }
        host_active = hc[0];
      }
    }
    worst_iters = std::max(worst_iters, it);
    if (host_active > 0) not_converged = true;
    WM_LAUNCH(WM_PC_NOISE, s, k_sq_combine<<<blocks_for(nblk, 256), 256, 0, s>>>(nblk, n_nodes, d_c.p, x.p, acc.p));
    WM_CUDA(cudaGetLastError());
    WM_TRY(wm_k_apply_mass64(L, tc, acc.p, ftile.p, nullptr, s));
    WM_TRY(wm_k_from_tiled(ftile.p, tc, N, f + (size_t)s0 * N, ns, s));
  }
  int flag = 0;
  WM_CUDA(cudaMemcpyAsync(&flag, counters.p + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  WM_CUDA(cudaStreamSynchronize(s));
  if (iterations) *iterations = worst_iters;
  if (flag) {
    wm_set_error("non-finite value in the sqrt(M) solves");
    return WM_ERR_NONFINITE;
  }
  if (not_converged) {
    wm_set_error("sqrt(M) solves missed rtol within max_iter");
    return WM_ERR_NOT_CONVERGED;
  }
  return WM_OK;
}
