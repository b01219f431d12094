// White-noise loads f = sqrt(M) y by the Hale–Higham–Trefethen sum (Sec. 3.3,
// Eq. eq:sqrt):  sqrt(M) y ~= M sum_k c_k (M + w_k^2 I)^{-1} y,  y ~ N(0, I).
//
// The K shifted systems of one sample share the Krylov space of (M, y), so
// they are solved by multi-shift conjugate gradients (Jegerlehner 1996,
// Frommer 2003): one CG sequence on the seed system M x = y, whose residuals
// r_n every shifted system shares up to a scalar, r^k_n = zeta^k_n r_n.  Per
// iteration there is one float64 mass apply per sample (not per node), and
// each shift k only updates its iterate and direction:
//   zeta^k_{n+1} = zeta^k_n zeta^k_{n-1} a_{n-1} /
//                  (a_n b_{n-1} (zeta^k_{n-1} - zeta^k_n) + zeta^k_{n-1} a_{n-1} (1 + w_k^2 a_n)),
//   a^k_n = a_n zeta^k_{n+1} / zeta^k_n,  b^k_n = b_n (zeta^k_{n+1} / zeta^k_n)^2,
//   x^k += a^k_n p^k,  p^k = zeta^k_{n+1} r_{n+1} + b^k_n p^k,
// with a_n, b_n the seed's CG coefficients (a_{-1} = 1, b_{-1} = 0,
// zeta_{-1} = zeta_0 = 1).  Shift k of a sample stops once
// |zeta^k| |r| <= rtol |y|.  The shifts are positive, so every shifted system
// converges no slower than the seed.
//
// Layout: samples 32 to a tile, [tiles][N][32] (lane = sample); the shift
// vectors are node-major blocks [K][tiles][N][32], so the weighted sum over
// k is an elementwise pass.  Row kernels: one warp per (tile, row), rows in
// chunks of kRows per block; per-lane partial dot products are reduced over
// the block's warps and then over the chunks in a fixed order.
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

__device__ __forceinline__ double chunk_sum(const double* __restrict__ part, int nchunk, int nsys, int g) {
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * nsys + g];
  return s;
}

// r = p = y, p^k = y, x^k = 0 for every shift; partial (r, r)
__global__ void __launch_bounds__(256) k_ms_init(int N, int K, const double* __restrict__ ybuf,
                                                 double* __restrict__ r, double* __restrict__ p,
                                                 double* __restrict__ xs, double* __restrict__ ps,
                                                 double* __restrict__ part) {
  const int t = blockIdx.y, l = threadIdx.x;
  const size_t nblk = (size_t)gridDim.y * N * WM_LANES;
  double acc = 0.0;
  for (int it = 0; it < kRowIters; ++it) {
    const int i = blockIdx.x * kRows + it * kWarps + threadIdx.y;
    if (i >= N) break;
    const size_t o = ((size_t)t * N + i) * WM_LANES + l;
    const double yv = ybuf[o];
    r[o] = yv;
    p[o] = yv;
    for (int k = 0; k < K; ++k) {
      xs[(size_t)k * nblk + o] = 0.0;
      ps[(size_t)k * nblk + o] = yv;
    }
    acc += yv * yv;
  }
  block_partial(acc, part, ((size_t)blockIdx.x * gridDim.y + t) * WM_LANES);
}

// q = M p; partial (p, q)
__global__ void __launch_bounds__(256) k_ms_apply(int N, int W, const int32_t* __restrict__ col,
                                                  const double* __restrict__ M, const double* __restrict__ p,
                                                  double* __restrict__ q, double* __restrict__ part) {
  const int t = blockIdx.y, l = threadIdx.x;
  const double* pt = p + (size_t)t * N * WM_LANES;
  double acc = 0.0;
  for (int it = 0; it < kRowIters; ++it) {
    const int i = blockIdx.x * kRows + it * kWarps + threadIdx.y;
    if (i >= N) break;
    const int32_t* c = col + (size_t)i * W;
    const double* m = M + (size_t)i * W;
    double s = 0.0;
    for (int w = 0; w < W; ++w) s += m[w] * pt[(size_t)c[w] * WM_LANES + l];
    q[((size_t)t * N + i) * WM_LANES + l] = s;
    acc += pt[(size_t)i * WM_LANES + l] * s;
  }
  block_partial(acc, part, ((size_t)blockIdx.x * gridDim.y + t) * WM_LANES);
}

// r -= a q; partial (r, r)
__global__ void __launch_bounds__(256) k_ms_resid(int N, const double* __restrict__ a,
                                                  const double* __restrict__ q, double* __restrict__ r,
                                                  double* __restrict__ part) {
  const int t = blockIdx.y, l = threadIdx.x;
  const double av = a[(size_t)t * WM_LANES + l];
  double acc = 0.0;
  for (int it = 0; it < kRowIters; ++it) {
    const int i = blockIdx.x * kRows + it * kWarps + threadIdx.y;
    if (i >= N) break;
    const size_t o = ((size_t)t * N + i) * WM_LANES + l;
    const double rv = r[o] - av * q[o];
    r[o] = rv;
    acc += rv * rv;
  }
  block_partial(acc, part, ((size_t)blockIdx.x * gridDim.y + t) * WM_LANES);
}

struct SampleState {
  double rr, rr0, a, b, a_old, b_old;
  int active;
};

// (r, r) of y; a sample with y = 0 is done at once.  Every shift starts at zeta = 1.
__global__ void k_ms_start(int nsamp, int nchunk, int K, const double* __restrict__ part,
                           SampleState* __restrict__ st, double* __restrict__ zeta, double* __restrict__ zeta_old,
                           int* __restrict__ shift_active, int* __restrict__ flags) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsamp) return;
  const double v = chunk_sum(part, nchunk, nsamp, g);
  if (!isfinite(v)) atomicOr(flags, 1);
  const int act = (v > 0.0 && isfinite(v)) ? 1 : 0;
  SampleState s;
  s.rr = v;
  s.rr0 = v;
  s.a = 0.0;
  s.b = 0.0;
  s.a_old = 1.0;
  s.b_old = 0.0;
  s.active = act;
  st[g] = s;
  for (int k = 0; k < K; ++k) {
    zeta[(size_t)k * nsamp + g] = 1.0;
    zeta_old[(size_t)k * nsamp + g] = 1.0;
    shift_active[(size_t)k * nsamp + g] = act;
  }
}

// seed step length a_n = (r, r) / (p, M p)
__global__ void k_ms_alpha(int nsamp, int nchunk, const double* __restrict__ part, SampleState* __restrict__ st,
                           double* __restrict__ a_out, int* __restrict__ flags) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsamp) return;
  const double pq = chunk_sum(part, nchunk, nsamp, g);
  double a = 0.0;
  if (st[g].active) {
    if (pq > 0.0 && isfinite(pq)) {
      a = st[g].rr / pq;
    } else {
      atomicOr(flags, 1);
    }
  }
  st[g].a = a;
  a_out[g] = a;
}

// b_n, and for every shift zeta_{n+1}, a^k_n, b^k_n and its convergence test
__global__ void k_ms_shifts(int nsamp, int nchunk, int K, const double* __restrict__ part,
                            const double* __restrict__ w2, double rtol, SampleState* __restrict__ st,
                            double* __restrict__ zeta, double* __restrict__ zeta_old,
                            int* __restrict__ shift_active, double* __restrict__ ak, double* __restrict__ bk,
                            double* __restrict__ zk, double* __restrict__ b_out, int* __restrict__ n_active,
                            int* __restrict__ flags) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsamp) return;
  SampleState s = st[g];
  const double rr_new = chunk_sum(part, nchunk, nsamp, g);
  double b = 0.0;
  int any = 0;
  if (s.active) {
    if (!isfinite(rr_new)) {
      atomicOr(flags, 1);
    } else if (s.rr > 0.0) {
      b = rr_new / s.rr;
    }
  }
  const double rnorm = sqrt(rr_new > 0.0 ? rr_new : 0.0), goal = rtol * sqrt(s.rr0);
  for (int k = 0; k < K; ++k) {
    const size_t j = (size_t)k * nsamp + g;
    double a_k = 0.0, b_k = 0.0, z_k = 0.0;
    if (s.active && shift_active[j]) {
      const double zc = zeta[j], zo = zeta_old[j];
      const double den = s.a * s.b_old * (zo - zc) + zo * s.a_old * (1.0 + w2[k] * s.a);
      const double zn = zc * zo * s.a_old / den;
      if (!isfinite(zn) || !(den != 0.0)) {
        atomicOr(flags, 1);
        shift_active[j] = 0;
      } else {
        const double ratio = zn / zc;
        a_k = s.a * ratio;
        b_k = b * ratio * ratio;
        z_k = zn;
        zeta_old[j] = zc;
        zeta[j] = zn;
        if (fabs(zn) * rnorm <= goal) {
          shift_active[j] = 0;
        } else {
          any = 1;
        }
      }
    }
    ak[j] = a_k;
    bk[j] = b_k;
    zk[j] = z_k;
  }
  s.a_old = s.a;
  s.b_old = b;
  s.b = b;
  s.rr = rr_new;
  s.active = s.active && any;
  st[g] = s;
  b_out[g] = s.active ? b : 0.0;
  if (s.active) atomicAdd(n_active, 1);
}

// x^k += a^k p^k, p^k = zeta^k r + b^k p^k for every shift; seed p = r + b p
__global__ void k_ms_update(size_t nblk, int N, int K, int nsamp, const double* __restrict__ ak,
                            const double* __restrict__ bk, const double* __restrict__ zk,
                            const double* __restrict__ b, const double* __restrict__ r, double* __restrict__ p,
                            double* __restrict__ xs, double* __restrict__ ps) {
  size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (o >= nblk) return;
  const int g = (int)((o / ((size_t)N * WM_LANES)) * WM_LANES + (o % WM_LANES));
  const double rv = r[o];
  for (int k = 0; k < K; ++k) {
    const size_t j = (size_t)k * nsamp + g, e = (size_t)k * nblk + o;
    const double pk = ps[e];
    xs[e] += ak[j] * pk;
    ps[e] = zk[j] * rv + bk[j] * pk;
  }
  p[o] = rv + b[g] * p[o];
}

// acc = sum_k c_k x_k over the node blocks (same tile layout as the samples)
__global__ void k_ms_combine(size_t nblk, int K, const double* __restrict__ cnode, const double* __restrict__ x,
                             double* __restrict__ acc) {
  size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (o >= nblk) return;
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += cnode[k] * x[(size_t)k * nblk + o];
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
  const int K = n_nodes;
  std::vector<double> w2(K), c(K);
  WM_TRY(wm_hht_rule(lo, hi, K, w2.data(), c.data()));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const wm_level& L = h->lv[0];
  const int N = L.N;
  const int ts = (n_samples + WM_LANES - 1) / WM_LANES;
  // sample tiles per pass: 2K shift vectors and seven seed/layout vectors per
  // sample tile within half the free memory
  size_t free_b = 0, total_b = 0;
  WM_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t per_tile = (size_t)(2 * K + 7) * N * WM_LANES * sizeof(double);
  int tc = (int)std::min<size_t>((size_t)ts, std::max<size_t>(1, (free_b / 2) / per_tile));
  tc = std::min(tc, 65535);
  const int nsamp = tc * WM_LANES;
  const int nchunk = (N + kRows - 1) / kRows;
  const size_t nblk = (size_t)tc * N * WM_LANES;
  Buf<double> r, p, q, xs, ps, ybuf, yrows, acc, ftile, part, a, b, ak, bk, zk, zeta, zeta_old, d_w2, d_c;
  Buf<SampleState> st;
  Buf<int> shift_active, counters;
  WM_TRY(r.alloc(nblk));
  WM_TRY(p.alloc(nblk));
  WM_TRY(q.alloc(nblk));
  WM_TRY(xs.alloc(nblk * K));
  WM_TRY(ps.alloc(nblk * K));
  WM_TRY(ybuf.alloc(nblk));
  WM_TRY(yrows.alloc(nblk));
  WM_TRY(acc.alloc(nblk));
  WM_TRY(ftile.alloc(nblk));
  WM_TRY(part.alloc((size_t)nchunk * nsamp));
  WM_TRY(a.alloc(nsamp));
  WM_TRY(b.alloc(nsamp));
  WM_TRY(st.alloc(nsamp));
  WM_TRY(ak.alloc((size_t)K * nsamp));
  WM_TRY(bk.alloc((size_t)K * nsamp));
  WM_TRY(zk.alloc((size_t)K * nsamp));
  WM_TRY(zeta.alloc((size_t)K * nsamp));
  WM_TRY(zeta_old.alloc((size_t)K * nsamp));
  WM_TRY(shift_active.alloc((size_t)K * nsamp));
  WM_TRY(counters.alloc(2));  // [0] samples with an unconverged shift after the last step, [1] non-finite flag
  WM_TRY(d_w2.upload(w2, s));
  WM_TRY(d_c.upload(c, s));
  const dim3 rgrid((unsigned)nchunk, (unsigned)tc), rblock(WM_LANES, kWarps);
  const unsigned sgrid = blocks_for((size_t)nsamp, 128);
  const unsigned egrid = blocks_for(nblk, 256);
  int worst_iters = 0;
  bool not_converged = false;
  for (int t0 = 0; t0 < ts; t0 += tc) {
    const int tcur = std::min(tc, ts - t0);  // sample tiles of this pass; unused tiles get y = 0
    const int s0 = t0 * WM_LANES, ns = std::min(n_samples - s0, tcur * WM_LANES);
    for (int si = 0; si < ns; ++si)
      WM_TRY(wm_k_normals(seed, s0 + si, kNormalStream, 0, N, yrows.p + (size_t)si * N, s));
    WM_TRY(wm_k_to_tiled(yrows.p, ns, N, ybuf.p, tc, s));
    WM_CUDA(cudaMemsetAsync(counters.p, 0, 2 * sizeof(int), s));
    WM_LAUNCH(WM_PC_NOISE, s, k_ms_init<<<rgrid, rblock, 0, s>>>(N, K, ybuf.p, r.p, p.p, xs.p, ps.p, part.p));
    WM_LAUNCH(WM_PC_NOISE, s, k_ms_start<<<sgrid, 128, 0, s>>>(nsamp, nchunk, K, part.p, st.p, zeta.p, zeta_old.p,
                                                               shift_active.p, counters.p + 1));
    int it = 0, host_active = 1;
    while (it < max_iter && host_active > 0) {
      ++it;
      WM_LAUNCH(WM_PC_NOISE, s, k_ms_apply<<<rgrid, rblock, 0, s>>>(N, L.W, L.d_col.p, L.d_M64.p, p.p, q.p, part.p));
      WM_LAUNCH(WM_PC_NOISE, s, k_ms_alpha<<<sgrid, 128, 0, s>>>(nsamp, nchunk, part.p, st.p, a.p, counters.p + 1));
      WM_LAUNCH(WM_PC_NOISE, s, k_ms_resid<<<rgrid, rblock, 0, s>>>(N, a.p, q.p, r.p, part.p));
      WM_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(int), s));
      WM_LAUNCH(WM_PC_NOISE, s, k_ms_shifts<<<sgrid, 128, 0, s>>>(nsamp, nchunk, K, part.p, d_w2.p, rtol, st.p,
                                                                  zeta.p, zeta_old.p, shift_active.p, ak.p, bk.p,
                                                                  zk.p, b.p, counters.p, counters.p + 1));
      WM_LAUNCH(WM_PC_NOISE, s, k_ms_update<<<egrid, 256, 0, s>>>(nblk, N, K, nsamp, ak.p, bk.p, zk.p, b.p, r.p, p.p,
                                                                  xs.p, ps.p));
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
    WM_LAUNCH(WM_PC_NOISE, s, k_ms_combine<<<egrid, 256, 0, s>>>(nblk, K, d_c.p, xs.p, acc.p));
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
