// Geometry, metric terms and operator assembly on the GPU (Sec. 3.2).
//
//  * k_metric: F_m, d_uF, d_vF at every Gauss point -> K_m, a_m = sqrt(det K_m),
//    G = a_m K_m^{-1} in float64 (Eqs. eq:mass, eq:stiffness).
//  * k_element_matrices: element mass and stiffness matrices by sum
//    factorisation over the tensor Gauss rule (the g_u sums are shared by all
//    k_v' of a row).
//  * k_assemble_rows: the glued rows of S and M gathered from the element
//    matrices in a fixed order (deterministic, no atomics).
#include "wm_internal.h"

namespace {

__constant__ int c_face[6][4] = {{1, 2, 0, +1}, {2, 1, 0, -1}, {2, 0, 1, +1},
                                 {0, 2, 1, -1}, {0, 1, 2, +1}, {1, 0, 2, -1}};

struct GeoArgs {
  int kind, np, nu, nv, nq;
  double R, r;
};

__device__ void surface_derivs(const GeoArgs& g, int m, double u, double v, double Fu[3], double Fv[3]) {
  if (g.kind == WM_SPHERE6) {
    double c[3], cu[3] = {0, 0, 0}, cv[3] = {0, 0, 0};
    int ax = c_face[m][0], bx = c_face[m][1], nx = c_face[m][2];
    c[ax] = 2.0 * u - 1.0;
    c[bx] = 2.0 * v - 1.0;
    c[nx] = (double)c_face[m][3];
    cu[ax] = 2.0;
    cv[bx] = 2.0;
    double n2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    double inv = rsqrt(n2);
    double inv3 = inv * inv * inv;
    double ccu = c[ax] * 2.0, ccv = c[bx] * 2.0;
    for (int d = 0; d < 3; ++d) {
      Fu[d] = cu[d] * inv - c[d] * ccu * inv3;
      Fv[d] = cv[d] * inv - c[d] * ccv * inv3;
    }
  } else {
    double su, cu_, sv, cv_;
    sincospi(2.0 * u, &su, &cu_);
    sincospi(2.0 * v, &sv, &cv_);
    double rho = g.R + g.r * cv_;
    const double tp = 2.0 * M_PI;
    Fu[0] = -tp * rho * su;
    Fu[1] = tp * rho * cu_;
    Fu[2] = 0.0;
    Fv[0] = -tp * g.r * sv * cu_;
    Fv[1] = -tp * g.r * sv * su;
    Fv[2] = tp * g.r * cv_;
  }
}

__global__ void k_metric(GeoArgs g, const double* __restrict__ gx, int64_t nQ, double* __restrict__ out) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nQ) return;
  int nq2 = g.nq * g.nq;
  int64_t e = q / nq2;
  int loc = (int)(q - e * nq2);
  int gv = loc / g.nq, gu = loc % g.nq;
  int eu = (int)(e % g.nu);
  int64_t t = e / g.nu;
  int ev = (int)(t % g.nv);
  int m = (int)(t / g.nv);
  double u = (eu + gx[gu]) / g.nu;
  double v = (ev + gx[gv]) / g.nv;
  double Fu[3], Fv[3];
  surface_derivs(g, m, u, v, Fu, Fv);
  double K11 = Fu[0] * Fu[0] + Fu[1] * Fu[1] + Fu[2] * Fu[2];
  double K12 = Fu[0] * Fv[0] + Fu[1] * Fv[1] + Fu[2] * Fv[2];
  double K22 = Fv[0] * Fv[0] + Fv[1] * Fv[1] + Fv[2] * Fv[2];
  double a = sqrt(K11 * K22 - K12 * K12);
  double* o = out + 4 * q;
  o[0] = a;
  o[1] = K22 / a;
  o[2] = -K12 / a;
  o[3] = K11 / a;
}

// One thread per (element, local row k): row k of the element mass and
// stiffness matrices.  Sum factorisation: for each g_v the g_u sums over the
// 1D factors are formed once per k_u', then combined with the g_v factors for
// all k_v'.
template <int P>
__global__ void k_element_matrices(int E, int nu, int nv, const double* __restrict__ metric,
                                   const double* __restrict__ gw, const double* __restrict__ bu,
                                   const double* __restrict__ du, const double* __restrict__ bv,
                                   const double* __restrict__ dv, double* __restrict__ Se,
                                   double* __restrict__ Me) {
  constexpr int NQ = P + 1, NK = (P + 1) * (P + 1);
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)E * NK) return;
  int64_t e = tid / NK;
  int k = (int)(tid - e * NK);
  int kv = k / (P + 1), ku = k % (P + 1);
  int eu = (int)(e % nu);
  int ev = (int)((e / nu) % nv);
  const double* BU = bu + (size_t)eu * (P + 1) * NQ;
  const double* DU = du + (size_t)eu * (P + 1) * NQ;
  const double* BV = bv + (size_t)ev * (P + 1) * NQ;
  const double* DV = dv + (size_t)ev * (P + 1) * NQ;
  double S[NK], M[NK];
#pragma unroll
  for (int t = 0; t < NK; ++t) S[t] = M[t] = 0.0;
  double elw = 1.0 / ((double)nu * nv);
  for (int gv = 0; gv < NQ; ++gv) {
    double mu[P + 1], s11[P + 1], s12[P + 1], s21[P + 1], s22[P + 1];
#pragma unroll
    for (int kk = 0; kk <= P; ++kk) mu[kk] = s11[kk] = s12[kk] = s21[kk] = s22[kk] = 0.0;
    for (int gu = 0; gu < NQ; ++gu) {
      const double* mt = metric + 4 * ((size_t)e * NQ * NQ + gv * NQ + gu);
      double w = gw[gu] * gw[gv] * elw;
      double wa = w * mt[0], w11 = w * mt[1], w12 = w * mt[2], w22 = w * mt[3];
      double b_k = BU[ku * NQ + gu], d_k = DU[ku * NQ + gu];
#pragma unroll
      for (int kk = 0; kk <= P; ++kk) {
        double b2 = BU[kk * NQ + gu], d2 = DU[kk * NQ + gu];
        mu[kk] += wa * b_k * b2;
        s11[kk] += w11 * d_k * d2;
        s12[kk] += w12 * d_k * b2;
        s21[kk] += w12 * b_k * d2;
        s22[kk] += w22 * b_k * b2;
      }
    }
    double bvk = BV[kv * NQ + gv], dvk = DV[kv * NQ + gv];
#pragma unroll
    for (int kv2 = 0; kv2 <= P; ++kv2) {
      double bv2 = BV[kv2 * NQ + gv], dv2 = DV[kv2 * NQ + gv];
#pragma unroll
      for (int ku2 = 0; ku2 <= P; ++ku2) {
        int t = kv2 * (P + 1) + ku2;
        M[t] += bvk * bv2 * mu[ku2];
        S[t] += bvk * bv2 * s11[ku2] + bvk * dv2 * s12[ku2] + dvk * bv2 * s21[ku2] + dvk * dv2 * s22[ku2];
      }
    }
  }
  double* so = Se + ((size_t)e * NK + k) * NK;
  double* mo = Me + ((size_t)e * NK + k) * NK;
#pragma unroll
  for (int t = 0; t < NK; ++t) {
    so[t] = S[t];
    mo[t] = M[t];
  }
}

// One thread per (row i, slot w): sum the element-matrix entries (i, col[i][w])
// over the element functions containing i, in element order.  A slot whose
// column already appeared earlier in the row (the padding) stays zero.
__global__ void k_assemble_rows(int N, int W, int nk, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ ng_ptr, const int32_t* __restrict__ ng_idx,
                                const int32_t* __restrict__ conn, const double* __restrict__ Se,
                                const double* __restrict__ Me, double* __restrict__ S, double* __restrict__ M,
                                float* __restrict__ S32, float* __restrict__ M32) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)N * W) return;
  int i = (int)(tid / W);
  int w = (int)(tid - (int64_t)i * W);
  int j = col[(size_t)i * W + w];
  bool dup = false;
  for (int w2 = 0; w2 < w; ++w2)
    if (col[(size_t)i * W + w2] == j) dup = true;
  double s = 0.0, m = 0.0;
  if (!dup) {
    for (int t = ng_ptr[i]; t < ng_ptr[i + 1]; ++t) {
      int ek = ng_idx[t];  // e * nk + k
      int e = ek / nk, k = ek - (ek / nk) * nk;
      const int32_t* ce = conn + (size_t)e * nk;
      for (int k2 = 0; k2 < nk; ++k2)
        if (ce[k2] == j) {
          s += Se[((size_t)e * nk + k) * nk + k2];
          m += Me[((size_t)e * nk + k) * nk + k2];
        }
    }
  }
  S[tid] = s;
  M[tid] = m;
  S32[tid] = (float)s;
  M32[tid] = (float)m;
}

__global__ void k_diagonals(int N, int W, const int32_t* __restrict__ slot, const double* __restrict__ S,
                            const double* __restrict__ M, double* dS, double* dM, float* dS32, float* dM32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = S[(size_t)i * W + slot[i]], m = M[(size_t)i * W + slot[i]];
  dS[i] = s;
  dM[i] = m;
  dS32[i] = (float)s;
  dM32[i] = (float)m;
}

__global__ void k_dense(int N, int W, const int32_t* __restrict__ col, const double* __restrict__ S,
                        const double* __restrict__ M, double* Sd, double* Md) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)N * W) return;
  int i = (int)(tid / W);
  int w = (int)(tid - (int64_t)i * W);
  int j = col[tid];
  for (int w2 = 0; w2 < w; ++w2)
    if (col[(size_t)i * W + w2] == j) return;
  Sd[(size_t)i * N + j] = S[tid];
  Md[(size_t)i * N + j] = M[tid];
}

__global__ void k_pack_rows(int64_t n, const int32_t* __restrict__ col, const double* __restrict__ S,
                            const double* __restrict__ M, PkRow32* __restrict__ p32, PkRow64* __restrict__ p64) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  PkRow32 a;
  a.col = col[t];
  a.s = (float)S[t];
  a.m = (float)M[t];
  a.pad = 0;
  p32[t] = a;
  PkRow64 b;
  b.s = S[t];
  b.m = M[t];
  b.col = col[t];
  b.pad = 0;
  p64[t] = b;
}

}  // namespace

static GeoArgs geo_args(const wm_hier* h, const wm_level& L) {
  GeoArgs g;
  g.kind = h->g.kind;
  g.np = h->np;
  g.nu = L.nu;
  g.nv = L.nv;
  g.nq = h->nq;
  g.R = h->g.R;
  g.r = h->g.r;
  return g;
}

int wm_k_metric(const wm_hier* h, const wm_level& L, cudaStream_t s) {
  int64_t nQ = (int64_t)L.E * h->nq * h->nq;
  int bs = 256;
  WM_LAUNCH(WM_PC_ASSEMBLY, s, k_metric<<<(unsigned)((nQ + bs - 1) / bs), bs, 0, s>>>(geo_args(h, L), h->d_gx.p, nQ, L.d_metric.p));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_k_element_matrices(const wm_hier* h, wm_level& L, cudaStream_t s) {
  int64_t n = (int64_t)L.E * L.nk;
  int bs = 128;
  unsigned grid = (unsigned)((n + bs - 1) / bs);
#define WM_EM(PP)                                                                                    \
  k_element_matrices<PP><<<grid, bs, 0, s>>>(L.E, L.nu, L.nv, L.d_metric.p, h->d_gw.p, L.d_bu.p,      \
                                             L.d_du.p, L.d_bv.p, L.d_dv.p, L.d_Se.p, L.d_Me.p)
  wm_prof_begin(WM_PC_ASSEMBLY, s);
  switch (h->p) {
    case 1: WM_EM(1); break;
    case 2: WM_EM(2); break;
    case 3: WM_EM(3); break;
    case 4: WM_EM(4); break;
    default: wm_set_error("degree %d unsupported", h->p); return WM_ERR_UNSUPPORTED;
  }
#undef WM_EM
  wm_prof_end(WM_PC_ASSEMBLY, s);
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_k_assemble_rows(const wm_hier* h, wm_level& L, cudaStream_t s) {
  (void)h;
  int64_t n = (int64_t)L.N * L.W;
  int bs = 256;
  WM_LAUNCH(WM_PC_ASSEMBLY, s, k_assemble_rows<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(
      L.N, L.W, L.nk, L.d_col.p, L.d_ng_ptr.p, L.d_ng_idx.p, L.d_conn.p, L.d_Se.p, L.d_Me.p, L.d_S64.p,
      L.d_M64.p, L.d_S32.p, L.d_M32.p));
  WM_CUDA(cudaGetLastError());
  WM_LAUNCH(WM_PC_ASSEMBLY, s, k_diagonals<<<(L.N + 255) / 256, 256, 0, s>>>(L.N, L.W, L.d_diag_slot.p, L.d_S64.p, L.d_M64.p, L.d_dS64.p,
                                                L.d_dM64.p, L.d_dS32.p, L.d_dM32.p));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_k_dense_coarse(const wm_level& L, cudaStream_t s) {
  WM_CUDA(cudaMemsetAsync(L.d_Sdense.p, 0, sizeof(double) * (size_t)L.N * L.N, s));
  WM_CUDA(cudaMemsetAsync(L.d_Mdense.p, 0, sizeof(double) * (size_t)L.N * L.N, s));
  int64_t n = (int64_t)L.N * L.W;
  WM_LAUNCH(WM_PC_ASSEMBLY, s, k_dense<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L.N, L.W, L.d_col.p, L.d_S64.p, L.d_M64.p, L.d_Sdense.p,
                                                      L.d_Mdense.p));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int wm_k_pack_rows(wm_level& L, cudaStream_t s) {
  int64_t n = (int64_t)L.N * L.W;
  WM_TRY(L.d_pk32.alloc(n));
  WM_TRY(L.d_pk64.alloc(n));
  WM_LAUNCH(WM_PC_ASSEMBLY, s, k_pack_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, L.d_col.p, L.d_S64.p,
                                                                                      L.d_M64.p, L.d_pk32.p,
                                                                                      L.d_pk64.p));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}
