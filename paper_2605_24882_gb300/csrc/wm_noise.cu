// White-noise loads from Philox4x32-10 normals at the Gauss points (Sec. 3.3).
//
// The discrete white noise b_s must have covariance M.  It is drawn at the
// Gauss points: b_s,i = sum_q sqrt(w_q a_q) xi_{s,q} phi_i(x_q), so that
// Cov(b_s) = B B^T is exactly the mass matrix of the same Gauss rule.
//
// Philox4x32-10 is written from its published definition (Salmon, Moraes,
// Dror, Shaw, SC'11): ten rounds of two 32x32->64 multiplications by
// 0xD2511F53 and 0xCD9E8D57 with the key bumped by (0x9E3779B9, 0xBB67AE85).
#include "wm_internal.h"

namespace {

struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
  }
  return c;
}

__device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo) {
  uint64_t a = (uint64_t)(hi >> 5), b = (uint64_t)(lo >> 6);
  return (double)(a * 67108864ull + b + 1ull) * 1.1102230246251565e-16;  // 2^-53
}

// The Box–Muller pair of normals with pair index `pair` of (seed, sample, stream).
__device__ __forceinline__ void normal_pair(uint64_t seed, int sample, int stream, int64_t pair, double* z0,
                                            double* z1) {
  U4 c;
  c.x = (uint32_t)(pair & 0xFFFFFFFFll);
  c.y = (uint32_t)sample;
  c.z = (uint32_t)stream;
  c.w = (uint32_t)(pair >> 32);
  U4 o = philox10(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  double u1 = uniform53(o.x, o.y);
  double u2 = uniform53(o.z, o.w);
  double rad = sqrt(-2.0 * log(u1));
  double s, co;
  sincos(2.0 * M_PI * u2, &s, &co);
  *z0 = rad * co;
  *z1 = rad * s;
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1, uint32_t* __restrict__ out,
                         int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  U4 c = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
  U4 o = philox10(c, k0, k1);
  out[4 * i] = o.x;
  out[4 * i + 1] = o.y;
  out[4 * i + 2] = o.z;
  out[4 * i + 3] = o.w;
}

__global__ void k_normals(uint64_t seed, int sample, int stream, int64_t q0, int64_t n, double* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t q = q0 + i;
  double z0, z1;
  normal_pair(seed, sample, stream, q >> 1, &z0, &z1);
  out[i] = (q & 1) ? z1 : z0;
}

// sqrt(w_q a_q) of every Gauss point, [E][nq^2] (the factor k_noise_local
// forms per sample, with the same operations)
template <int P>
__global__ void k_noise_weights(int E, int nu, int nv, const double* __restrict__ metric,
                                const double* __restrict__ gw, double* __restrict__ w) {
  constexpr int NQ = P + 1, NQ2 = NQ * NQ;
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= (int64_t)E * NQ2) return;
  const int j = (int)(q % NQ2);
  const int gv = j / NQ, gu = j % NQ;
  const double elw = 1.0 / ((double)nu * nv);
  w[q] = sqrt(gw[gu] * gw[gv] * elw * metric[4 * q]);
}

// One thread per (element e, sample s0+sl): the (p+1)^2 local load
// contributions sum_q sqrt(w_q a_q) xi_q phi_k(x_q) of the element, xi the
// Philox normals of sample s0 + sl.  bl layout [E][nk][ns].  WT: the factors
// sqrt(w_q a_q) from the table of k_noise_weights instead of per sample.
template <int P, bool WT = false>
__global__ void k_noise_local(int E, int nu, int nv, int ns, int s0, uint64_t seed,
                              const double* __restrict__ metric, const double* __restrict__ gw,
                              const double* __restrict__ bu, const double* __restrict__ bv, double* __restrict__ bl,
                              const double* __restrict__ wtab = nullptr) {
  constexpr int NQ = P + 1, NK = (P + 1) * (P + 1), NQ2 = NQ * NQ;
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)E * ns) return;
  int64_t e = tid / ns;
  int sl = (int)(tid - e * ns);
  int eu = (int)(e % nu);
  int ev = (int)((e / nu) % nv);
  double xi[NQ2 + 1];
  int64_t q0 = e * NQ2;
  int64_t pr0 = q0 >> 1, pr1 = (q0 + NQ2 - 1) >> 1;
  for (int64_t pr = pr0; pr <= pr1; ++pr) {
    double z0, z1;
    normal_pair(seed, s0 + sl, 0, pr, &z0, &z1);
    int j0 = (int)(2 * pr - q0);
    if (j0 >= 0) xi[j0] = z0;
    if (j0 + 1 < NQ2) xi[j0 + 1] = z1;
  }
  double wq[NQ2];
  if constexpr (WT) {
#pragma unroll
    for (int j = 0; j < NQ2; ++j) wq[j] = wtab[q0 + j] * xi[j];
  } else {
    double elw = 1.0 / ((double)nu * nv);
#pragma unroll
    for (int j = 0; j < NQ2; ++j) {
      int gv = j / NQ, gu = j % NQ;
      wq[j] = sqrt(gw[gu] * gw[gv] * elw * metric[4 * (q0 + j)]) * xi[j];
    }
  }
  const double* BU = bu + (size_t)eu * (P + 1) * NQ;
  const double* BV = bv + (size_t)ev * (P + 1) * NQ;
#pragma unroll
  for (int kv = 0; kv <= P; ++kv)
#pragma unroll
    for (int ku = 0; ku <= P; ++ku) {
      double acc = 0.0;
#pragma unroll
      for (int gv = 0; gv < NQ; ++gv) {
        double t = 0.0;
#pragma unroll
        for (int gu = 0; gu < NQ; ++gu) t += BU[ku * NQ + gu] * wq[gv * NQ + gu];
        acc += BV[kv * NQ + gv] * t;
      }
      bl[((size_t)e * NK + kv * (P + 1) + ku) * ns + sl] = acc;
    }
}

// One thread per (DOF i, row s0+sl): b[tile][i][lane] = sum over the element
// functions containing i of their local contributions, in element order.
__global__ void k_noise_gather(int N, int ns, int s0, const int32_t* __restrict__ ptr,
                               const int32_t* __restrict__ idx, const double* __restrict__ bl,
                               double* __restrict__ b) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)N * ns) return;
  int i = (int)(tid / ns);
  int sl = (int)(tid - (int64_t)i * ns);
  double acc = 0.0;
  for (int t = ptr[i]; t < ptr[i + 1]; ++t) acc += bl[(size_t)idx[t] * ns + sl];
  int s = s0 + sl;
  b[((size_t)(s / WM_LANES) * N + i) * WM_LANES + (s % WM_LANES)] = acc;
}

}  // namespace

int wm_k_philox(const uint32_t* ctr, uint64_t key, uint32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return WM_OK;
  WM_LAUNCH(WM_PC_NOISE, s, k_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctr, (uint32_t)(key & 0xFFFFFFFFull),
                                                       (uint32_t)(key >> 32), out, n));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_k_normals(uint64_t seed, int sample, int stream_id, int64_t q0, int64_t n, double* out, cudaStream_t s) {
  if (n <= 0) return WM_OK;
  WM_LAUNCH(WM_PC_NOISE, s, k_normals<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(seed, sample, stream_id, q0, n, out));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_k_noise_tiled(const wm_hier* h, uint64_t seed, int sample_first, int row0, int ns, double* b_tiled,
                     double* bl, cudaStream_t s) {
  const wm_level& L = h->lv[0];
  int64_t n1 = (int64_t)L.E * ns;
  unsigned g1 = (unsigned)((n1 + 127) / 128);
#define WM_NL(PP)                                                                                              \
  if (L.d_noise_w.p)                                                                                           \
    k_noise_local<PP, true><<<g1, 128, 0, s>>>(L.E, L.nu, L.nv, ns, sample_first, seed, L.d_metric.p, h->d_gw.p, \
                                               L.d_bu.p, L.d_bv.p, bl, L.d_noise_w.p);                          \
  else                                                                                                         \
    k_noise_local<PP><<<g1, 128, 0, s>>>(L.E, L.nu, L.nv, ns, sample_first, seed, L.d_metric.p, h->d_gw.p,      \
                                         L.d_bu.p, L.d_bv.p, bl)
  wm_prof_begin(WM_PC_NOISE, s);
  switch (h->p) {
    case 1: WM_NL(1); break;
    case 2: WM_NL(2); break;
    case 3: WM_NL(3); break;
    case 4: WM_NL(4); break;
    default: return WM_ERR_UNSUPPORTED;
  }
#undef WM_NL
  wm_prof_end(WM_PC_NOISE, s);
  WM_CUDA(cudaGetLastError());
  int64_t n2 = (int64_t)L.N * ns;
  WM_LAUNCH(WM_PC_NOISE, s, k_noise_gather<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(L.N, ns, row0, L.d_ng_ptr.p, L.d_ng_idx.p, bl,
                                                              b_tiled));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_k_noise_weights(const wm_hier* h, wm_level& L, cudaStream_t s) {
  const int nq2 = h->nq * h->nq;
  WM_TRY(L.d_noise_w.alloc((size_t)L.E * nq2));
  const int64_t n = (int64_t)L.E * nq2;
  const unsigned g = (unsigned)((n + 255) / 256);
  switch (h->p) {
    case 1: WM_LAUNCH(WM_PC_ASSEMBLY, s, (k_noise_weights<1><<<g, 256, 0, s>>>(L.E, L.nu, L.nv, L.d_metric.p, h->d_gw.p, L.d_noise_w.p))); break;
    case 2: WM_LAUNCH(WM_PC_ASSEMBLY, s, (k_noise_weights<2><<<g, 256, 0, s>>>(L.E, L.nu, L.nv, L.d_metric.p, h->d_gw.p, L.d_noise_w.p))); break;
    case 3: WM_LAUNCH(WM_PC_ASSEMBLY, s, (k_noise_weights<3><<<g, 256, 0, s>>>(L.E, L.nu, L.nv, L.d_metric.p, h->d_gw.p, L.d_noise_w.p))); break;
    case 4: WM_LAUNCH(WM_PC_ASSEMBLY, s, (k_noise_weights<4><<<g, 256, 0, s>>>(L.E, L.nu, L.nv, L.d_metric.p, h->d_gw.p, L.d_noise_w.p))); break;
    default: return WM_ERR_UNSUPPORTED;
  }
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// ---------------------------------------------------------------- no-alloc entry
// White-noise loads for callers that cannot allocate device memory: a host
// framework whose caching allocator owns the device memory, or code that may
// not call cudaMalloc because it synchronises the device.  The element-local
// contributions go to a fixed file-scope device array instead of workspace
// memory; the loads are gathered straight into the caller's [n][N] output.
#include <mutex>

#define WM_NOALLOC_SCRATCH_DOUBLES (1 << 22) /* 32 MiB, resident on every device that loads the library */

static __device__ __align__(256) double g_noalloc_scratch[WM_NOALLOC_SCRATCH_DOUBLES];

namespace {

// b[s][i] = sum over the element functions containing i of their contributions
__global__ void k_noise_gather_rows(int N, int ns, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                    const double* __restrict__ bl, double* __restrict__ b) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)N * ns) return;
  int s = (int)(tid / N);
  int i = (int)(tid - (int64_t)s * N);
  double acc = 0.0;
  for (int t = ptr[i]; t < ptr[i + 1]; ++t) acc += bl[(size_t)idx[t] * ns + s];
  b[(size_t)s * N + i] = acc;
}

// Device address of the scratch array, looked up once per device with that
// device current (a host-side name of a __device__ array is not its address).
int noalloc_scratch(int dev, double** out) {
  static std::mutex mu;
  static double* addr[256] = {};
  if (dev < 0 || dev >= 256) return WM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    WM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[dev] = static_cast<double*>(p);
  }
  *out = addr[dev];
  return WM_OK;
}

// device (or managed) memory the kernels may write
bool device_writable(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int wm_noise_loads_noalloc(wm_hier_t h, uint64_t seed, int n_samples, double* b, void* stream) {
  if (!h || n_samples < 0 || (n_samples > 0 && !b)) return WM_ERR_INVALID_ARG;
  if (n_samples == 0) return WM_OK;
  int dev = 0;
  WM_CUDA(cudaGetDevice(&dev));
  if (dev != h->device) {
    wm_set_error("wm_noise_loads_noalloc: the hierarchy lives on device %d but device %d is current", h->device, dev);
    return WM_ERR_INVALID_ARG;
  }
  if (!device_writable(b)) {
    wm_set_error("wm_noise_loads_noalloc: b must be device memory");
    return WM_ERR_INVALID_ARG;
  }
  const wm_level& L = h->lv[0];
  int64_t need = (int64_t)L.E * L.nk * n_samples;
  if (need > (int64_t)WM_NOALLOC_SCRATCH_DOUBLES) {
    wm_set_error("wm_noise_loads_noalloc: elements x (p+1)^2 x samples = %lld exceeds the fixed scratch of %d "
                 "doubles; use fewer samples per call",
                 (long long)need, WM_NOALLOC_SCRATCH_DOUBLES);
    return WM_ERR_INVALID_ARG;
  }
  double* bl = nullptr;
  WM_TRY(noalloc_scratch(dev, &bl));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int64_t n1 = (int64_t)L.E * n_samples;
  unsigned g1 = (unsigned)((n1 + 127) / 128);
  switch (h->p) {
    case 1: WM_LAUNCH(WM_PC_NOISE, s, k_noise_local<1><<<g1, 128, 0, s>>>(L.E, L.nu, L.nv, n_samples, 0, seed, L.d_metric.p, h->d_gw.p, L.d_bu.p, L.d_bv.p, bl)); break;
    case 2: WM_LAUNCH(WM_PC_NOISE, s, k_noise_local<2><<<g1, 128, 0, s>>>(L.E, L.nu, L.nv, n_samples, 0, seed, L.d_metric.p, h->d_gw.p, L.d_bu.p, L.d_bv.p, bl)); break;
    case 3: WM_LAUNCH(WM_PC_NOISE, s, k_noise_local<3><<<g1, 128, 0, s>>>(L.E, L.nu, L.nv, n_samples, 0, seed, L.d_metric.p, h->d_gw.p, L.d_bu.p, L.d_bv.p, bl)); break;
    case 4: WM_LAUNCH(WM_PC_NOISE, s, k_noise_local<4><<<g1, 128, 0, s>>>(L.E, L.nu, L.nv, n_samples, 0, seed, L.d_metric.p, h->d_gw.p, L.d_bu.p, L.d_bv.p, bl)); break;
    default: return WM_ERR_UNSUPPORTED;
  }
  WM_CUDA(cudaGetLastError());
  int64_t n2 = (int64_t)L.N * n_samples;
  WM_LAUNCH(WM_PC_NOISE, s, k_noise_gather_rows<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(
                                L.N, n_samples, L.d_ng_ptr.p, L.d_ng_idx.p, bl, b));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}
