// Batched operator kernels over the tiled layout [tiles][N][32].
//
// Every kernel maps one warp to one DOF row of one tile: lane l handles
// system 32 t + l, so the row's column indices and matrix values are warp
// uniform (one broadcast load serves 32 systems) and every vector access is
// one coalesced 128/256-byte row.
#include "wm_internal.h"

namespace {

constexpr int kRowsPerBlock = 8;

// y = (S + sigma M) x on the rows of one level, one warp per (tile, row).
template <typename T>
__global__ void __launch_bounds__(256) k_apply(int N, int W, const int32_t* __restrict__ col,
                                               const T* __restrict__ S, const T* __restrict__ M,
                                               const double* __restrict__ sigma, const T* __restrict__ x,
                                               T* __restrict__ y, const int* __restrict__ tile_active) {
  int t = blockIdx.y;
  if (tile_active && !tile_active[t]) return;
  int i = blockIdx.x * kRowsPerBlock + threadIdx.y;
  if (i >= N) return;
  int l = threadIdx.x;
  T sg = (T)sigma[t * WM_LANES + l];
  const T* xt = x + (size_t)t * N * WM_LANES;
  const int32_t* c = col + (size_t)i * W;
  const T* s = S + (size_t)i * W;
  const T* m = M + (size_t)i * W;
  T accS = 0, accM = 0;
  for (int w = 0; w < W; ++w) {
    T xv = xt[(size_t)c[w] * WM_LANES + l];
    accS += s[w] * xv;
    accM += m[w] * xv;
  }
  y[((size_t)t * N + i) * WM_LANES + l] = accS + sg * accM;
}

__global__ void __launch_bounds__(256) k_apply_mass(int N, int W, const int32_t* __restrict__ col,
                                                    const double* __restrict__ M, const double* __restrict__ x,
                                                    double* __restrict__ y, const int* __restrict__ tile_active) {
  int t = blockIdx.y;
  if (tile_active && !tile_active[t]) return;
  int i = blockIdx.x * kRowsPerBlock + threadIdx.y;
  if (i >= N) return;
  int l = threadIdx.x;
  const double* xt = x + (size_t)t * N * WM_LANES;
  const int32_t* c = col + (size_t)i * W;
  const double* m = M + (size_t)i * W;
  double acc = 0;
  for (int w = 0; w < W; ++w) acc += m[w] * xt[(size_t)c[w] * WM_LANES + l];
  y[((size_t)t * N + i) * WM_LANES + l] = acc;
}

// xf += P xc (CSR over fine rows)
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(int Nf, int Nc, const int32_t* __restrict__ ptr,
                                                     const int32_t* __restrict__ idx, const T* __restrict__ val,
                                                     const T* __restrict__ xc, T* __restrict__ xf,
                                                     const int* __restrict__ tile_active) {
  int t = blockIdx.y;
  if (tile_active && !tile_active[t]) return;
  int i = blockIdx.x * kRowsPerBlock + threadIdx.y;
  if (i >= Nf) return;
  int l = threadIdx.x;
  const T* xt = xc + (size_t)t * Nc * WM_LANES;
  T acc = 0;
  for (int k = ptr[i]; k < ptr[i + 1]; ++k) acc += val[k] * xt[(size_t)idx[k] * WM_LANES + l];
  xf[((size_t)t * Nf + i) * WM_LANES + l] += acc;
}

// rc = R rf (CSR over coarse rows, R = P^T)
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(int Nc, int Nf, const int32_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ idx, const T* __restrict__ val,
                                                  const T* __restrict__ rf, T* __restrict__ rc,
                                                  const int* __restrict__ tile_active) {
  int t = blockIdx.y;
  if (tile_active && !tile_active[t]) return;
  int I = blockIdx.x * kRowsPerBlock + threadIdx.y;
  if (I >= Nc) return;
  int l = threadIdx.x;
  const T* rt = rf + (size_t)t * Nf * WM_LANES;
  T acc = 0;
  for (int k = ptr[I]; k < ptr[I + 1]; ++k) acc += val[k] * rt[(size_t)idx[k] * WM_LANES + l];
  rc[((size_t)t * Nc + I) * WM_LANES + l] = acc;
}

// [n][N] -> [tiles][N][32] through a 32x32 shared-memory transpose; lanes
// beyond n are zero.
__global__ void k_to_tiled(const double* __restrict__ src, int n, int N, double* __restrict__ dst) {
  __shared__ double tileb[32][33];
  int t = blockIdx.y;
  int i0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int v = t * 32 + r, i = i0 + threadIdx.x;
    tileb[r][threadIdx.x] = (v < n && i < N) ? src[(size_t)v * N + i] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = i0 + r;
    if (i < N) dst[((size_t)t * N + i) * WM_LANES + threadIdx.x] = tileb[threadIdx.x][r];
  }
}

__global__ void k_from_tiled(const double* __restrict__ src, int N, double* __restrict__ dst, int n) {
  __shared__ double tileb[32][33];
  int t = blockIdx.y;
  int i0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = i0 + r;
    tileb[r][threadIdx.x] = i < N ? src[((size_t)t * N + i) * WM_LANES + threadIdx.x] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int v = t * 32 + r, i = i0 + threadIdx.x;
    if (v < n && i < N) dst[(size_t)v * N + i] = tileb[threadIdx.x][r];
  }
}

inline dim3 row_grid(int rows, int tiles) { return dim3((unsigned)((rows + kRowsPerBlock - 1) / kRowsPerBlock), tiles); }
const dim3 kBlock(WM_LANES, kRowsPerBlock);

}  // namespace

template <typename T>
static const T* rowsS(const wm_level& L);
template <>
const double* rowsS<double>(const wm_level& L) { return L.d_S64.p; }
template <>
const float* rowsS<float>(const wm_level& L) { return L.d_S32.p; }
template <typename T>
static const T* rowsM(const wm_level& L);
template <>
const double* rowsM<double>(const wm_level& L) { return L.d_M64.p; }
template <>
const float* rowsM<float>(const wm_level& L) { return L.d_M32.p; }
template <typename T>
static const T* pval(const wm_level& L);
template <>
const double* pval<double>(const wm_level& L) { return L.d_Pval64.p; }
template <>
const float* pval<float>(const wm_level& L) { return L.d_Pval32.p; }
template <typename T>
static const T* rval(const wm_level& L);
template <>
const double* rval<double>(const wm_level& L) { return L.d_Rval64.p; }
template <>
const float* rval<float>(const wm_level& L) { return L.d_Rval32.p; }

template <typename T>
int wm_k_apply(const wm_level& L, int tiles, const double* sigma, const T* x, T* y, const int* tile_active,
               cudaStream_t s) {
  if (tiles <= 0) return WM_OK;
  WM_LAUNCH(WM_PC_APPLY, s, k_apply<T><<<row_grid(L.N, tiles), kBlock, 0, s>>>(L.N, L.W, L.d_col.p, rowsS<T>(L), rowsM<T>(L), sigma, x, y,
                                                     tile_active));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}
template int wm_k_apply<double>(const wm_level&, int, const double*, const double*, double*, const int*,
                                cudaStream_t);
template int wm_k_apply<float>(const wm_level&, int, const double*, const float*, float*, const int*,
                               cudaStream_t);

int wm_k_apply_mass64(const wm_level& L, int tiles, const double* x, double* y, const int* tile_active,
                      cudaStream_t s) {
  if (tiles <= 0) return WM_OK;
  WM_LAUNCH(WM_PC_SINC, s, k_apply_mass<<<row_grid(L.N, tiles), kBlock, 0, s>>>(L.N, L.W, L.d_col.p, L.d_M64.p, x, y, tile_active));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// `fine` is the finer level; its P maps the next coarser level's vectors to it
template <typename T>
int wm_k_prolong_add(const wm_level& fine, int tiles, const T* xc, T* xf, const int* tile_active, cudaStream_t s) {
  if (tiles <= 0) return WM_OK;
  WM_LAUNCH(WM_PC_PROLONG, s, k_prolong_add<T><<<row_grid(fine.nP, tiles), kBlock, 0, s>>>(fine.nP, fine.nR, fine.d_Pptr.p, fine.d_Pcol.p,
                                                               pval<T>(fine), xc, xf, tile_active));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}
template int wm_k_prolong_add<double>(const wm_level&, int, const double*, double*, const int*, cudaStream_t);
template int wm_k_prolong_add<float>(const wm_level&, int, const float*, float*, const int*, cudaStream_t);

template <typename T>
int wm_k_restrict(const wm_level& fine, int tiles, const T* rf, T* rc, const int* tile_active, cudaStream_t s) {
  if (tiles <= 0) return WM_OK;
  WM_LAUNCH(WM_PC_RESTRICT, s, k_restrict<T><<<row_grid(fine.nR, tiles), kBlock, 0, s>>>(fine.nR, fine.nP, fine.d_Rptr.p, fine.d_Rcol.p,
                                                            rval<T>(fine), rf, rc, tile_active));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}
template int wm_k_restrict<double>(const wm_level&, int, const double*, double*, const int*, cudaStream_t);
template int wm_k_restrict<float>(const wm_level&, int, const float*, float*, const int*, cudaStream_t);

int wm_k_to_tiled(const double* src, int n, int N, double* dst, int tiles, cudaStream_t s) {
  if (tiles <= 0 || N <= 0) return WM_OK;
  WM_LAUNCH(WM_PC_LAYOUT, s, k_to_tiled<<<dim3((N + 31) / 32, tiles), dim3(32, 8), 0, s>>>(src, n, N, dst));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_k_from_tiled(const double* src, int tiles, int N, double* dst, int n, cudaStream_t s) {
  if (tiles <= 0 || N <= 0) return WM_OK;
  WM_LAUNCH(WM_PC_LAYOUT, s, k_from_tiled<<<dim3((N + 31) / 32, tiles), dim3(32, 8), 0, s>>>(src, N, dst, n));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}
