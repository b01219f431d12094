// Shared-memory stencil kernels for the operator-type steps of the solver.
//
// A block owns a BU x BV tile of one patch's local DOF grid for TPB system
// tiles.  It stages the (BU + 2p) x (BV + 2p) window of the input vector
// (through the extended grid map: halo cells come from the neighbouring
// patch, or wrap on the torus) into shared memory, once per block, and every
// warp then sweeps one column of BV outputs with a (2p+1)-row register window,
// so each staged value is read from shared memory 2p+1 times instead of each
// neighbour being fetched from L1/L2 (2p+1)^2 times.  Lane = system, so every
// staged row is one coalesced 128/256-byte transaction and the row's stencil
// coefficients (S, M) are warp-uniform loads shared by TPB x 32 systems.
// Only the owner patch of a shared DOF computes its row.
#include <algorithm>

#include "wm_solver.h"
#include "wm_stencil.h"

namespace {

constexpr int BU = 8;   // outputs per block along u (one warp each)
// outputs per warp along v: for p = 2 the patches have 2^l + 2 local DOFs per
// side, which a height of 6 covers with less waste than 8 (66 and 18 exactly;
// coarse-level smoothing 33.9 -> 32.0 ms per bench step)
#ifndef WM_BV_P2
#define WM_BV_P2 6
#endif
template <int P>
struct BvOf {
  static constexpr int value = P == 2 ? WM_BV_P2 : 8;
  static_assert(value % 2 == 0 && value >= 2, "row pairs of the double-float residual");
};

template <typename T>
struct V2;
template <>
struct V2<float> {
  using type = float2;
};
template <>
struct V2<double> {
  using type = double2;
};

struct StenGeo {
  int nlu, nlv, ELU, ELV, nbu, nbv, N;
  const int32_t* ext;
  const int32_t* own;
};

// per-thread dot accumulator (products in T, flushed into double every 16)
template <typename T>
struct DAcc {
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

// per-block partial sums of the TPB tiles (tiles not in `act` are left untouched:
// another kernel owns them)
template <int TPB>
__device__ __forceinline__ void block_reduce(double (&acc)[TPB], double* part, int t0, int tiles, const bool* act) {
  __shared__ double red[TPB][BU][32];
#pragma unroll
  for (int k = 0; k < TPB; ++k) red[k][threadIdx.y][threadIdx.x] = acc[k];
  __syncthreads();
  if (threadIdx.y == 0) {
#pragma unroll
    for (int k = 0; k < TPB; ++k) {
      if (t0 + k >= tiles || !act[k]) continue;
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < BU; ++w) s += red[k][w][threadIdx.x];
      part[((size_t)(t0 + k) * gridDim.x + blockIdx.x) * 32 + threadIdx.x] = s;
    }
  }
}

// ---------------------------------------------------------------- epilogues
// Chebyshev step in three-term form (tiles with per-lane shifts):
// z_next = z + c1 (z - z_prev) + c2 D^{-1} (r - A z), with c1 = 0 at step 0
// and z_prev = 0 where has_prev is false; out may alias z_prev
template <typename T, int TPB>
struct ChebEpi {
  static constexpr int NIN = 2;  // r and z_prev of the output rows are staged
  const T* in[2];                // in[1] = nullptr: z_prev = 0
  int N, kstep;
  const T *dS, *dM;
  T* out;
  const double* sigma;
  const typename V2<T>::type* ctab;  // (c1, c2) per [shift][step] of this level
  const int* sid;
  T sg[TPB], c1[TPB], c2[TPB];
  __device__ __forceinline__ void init(int t0, const bool* act) {
#pragma unroll
    for (int k = 0; k < TPB; ++k) {
      int g = (t0 + k) * 32 + threadIdx.x;
      sg[k] = c1[k] = c2[k] = 0;
      if (!act[k]) continue;
      typename V2<T>::type c = ctab[sid[g] * WM_MAX_CHEB + kstep];
      c1[k] = kstep == 0 ? (T)0 : c.x;
      c2[k] = c.y;
      sg[k] = (T)sigma[g];
    }
  }
  // staged[a][k]: input a of tile k at this output row and lane
  __device__ __forceinline__ void row(int t0, const bool* act, int i, const T* aS, const T* aM, const T* zc,
                                      const T (*staged)[TPB]) {
    T ds = dS[i], dm = dM[i];
#pragma unroll
    for (int k = 0; k < TPB; ++k)
      if (act[k]) {
        size_t o = ((size_t)(t0 + k) * N + i) * 32 + threadIdx.x;
        T res = staged[0][k] - (aS[k] + sg[k] * aM[k]);
        T zp = in[1] ? staged[1][k] : (T)0;
        out[o] = zc[k] + c1[k] * (zc[k] - zp) + c2[k] * res / (ds + sg[k] * dm);
      }
  }
  __device__ __forceinline__ void finish(int, int, const bool*) {}
};

// residual: res = r - A z
template <typename T, int TPB>
struct ResidEpi {
  static constexpr int NIN = 1;  // r staged
  const T* in[1];
  int N;
  const T* r;
  T* res;
  const double* sigma;
  T sg[TPB];
  __device__ __forceinline__ void init(int t0, const bool* act) {
#pragma unroll
    for (int k = 0; k < TPB; ++k) sg[k] = act[k] ? (T)sigma[(t0 + k) * 32 + threadIdx.x] : (T)0;
  }
  __device__ __forceinline__ void row(int t0, const bool* act, int i, const T* aS, const T* aM, const T*,
                                      const T (*staged)[TPB]) {
#pragma unroll
    for (int k = 0; k < TPB; ++k)
      if (act[k]) {
        size_t o = ((size_t)(t0 + k) * N + i) * 32 + threadIdx.x;
        res[o] = staged[0][k] - (aS[k] + sg[k] * aM[k]);
      }
  }
  __device__ __forceinline__ void finish(int, int, const bool*) {}
};

// outer apply: q = A p, partial (p, q)
template <typename T, int TPB>
struct ApplyEpi {
  static constexpr int NIN = 0;
  const T* in[1];
  int N;
  T* q;
  const double* sigma;
  double* part;
  T sg[TPB];
  DAcc<T> acc[TPB];
  __device__ __forceinline__ void init(int t0, const bool* act) {
#pragma unroll
    for (int k = 0; k < TPB; ++k) sg[k] = act[k] ? (T)sigma[(t0 + k) * 32 + threadIdx.x] : (T)0;
  }
  __device__ __forceinline__ void row(int t0, const bool* act, int i, const T* aS, const T* aM, const T* zc,
                                      const T (*)[TPB]) {
#pragma unroll
    for (int k = 0; k < TPB; ++k)
      if (act[k]) {
        size_t o = ((size_t)(t0 + k) * N + i) * 32 + threadIdx.x;
        T qv = aS[k] + sg[k] * aM[k];
        q[o] = qv;
        acc[k].add(zc[k] * qv);
      }
  }
  __device__ __forceinline__ void finish(int t0, int tiles, const bool* act) {
    double a[TPB];
#pragma unroll
    for (int k = 0; k < TPB; ++k) a[k] = acc[k].get();
    block_reduce<TPB>(a, part, t0, tiles, act);
  }
};

// float64 true residual of flagged systems: r = b - A x, partial ||r||^2
template <typename Tr, int TPB>
struct TrueResEpi {
  static constexpr int NIN = 0;
  const double* in[1];
  int N;
  const double* rhs;
  const int *src_of, *rep;
  Tr* r;
  const double* sigma;
  double* part;
  double sg[TPB];
  int src[TPB];
  bool mine[TPB];
  double acc[TPB];
  __device__ __forceinline__ void init(int t0, const bool* act) {
#pragma unroll
    for (int k = 0; k < TPB; ++k) {
      int g = (t0 + k) * 32 + threadIdx.x;
      sg[k] = act[k] ? sigma[g] : 0.0;
      src[k] = act[k] ? src_of[g] : -1;
      mine[k] = act[k] && rep[g];
      acc[k] = 0.0;
    }
  }
  __device__ __forceinline__ void row(int t0, const bool*, int i, const double* aS, const double* aM, const double*,
                                      const double (*)[TPB]) {
#pragma unroll
    for (int k = 0; k < TPB; ++k)
      if (mine[k]) {
        int s = src[k];
        double b = s >= 0 ? rhs[((size_t)(s / 32) * N + i) * 32 + (s % 32)] : 0.0;
        double rt = b - (aS[k] + sg[k] * aM[k]);
        r[((size_t)(t0 + k) * N + i) * 32 + threadIdx.x] = (Tr)rt;
        acc[k] += rt * rt;
      }
  }
  __device__ __forceinline__ void finish(int t0, int tiles, const bool* act) {
    block_reduce<TPB>(acc, part, t0, tiles, act);
  }
};

// ---------------------------------------------------------------- the kernel
// 16-byte asynchronous global->shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// coefficient row stride in V2 elements, padded to 16-byte multiples
template <typename T, int P>
struct CoefStride {
  static constexpr int S2 = (2 * P + 1) * (2 * P + 1);
  static constexpr int value = sizeof(typename V2<T>::type) == 8 ? (S2 + 1) / 2 * 2 : S2;
};

template <typename T, int P, int TPB, int NIN>
struct SmemLayout {
  static constexpr int BV = BvOf<P>::value;
  static constexpr int CU = BU + 2 * P, CV = BV + 2 * P, NC = CU * CV;
  static constexpr int CS = CoefStride<T, P>::value;
  static constexpr size_t win = (size_t)TPB * NC * 32 * sizeof(T);
  static constexpr size_t coef = (size_t)BU * BV * CS * sizeof(typename V2<T>::type);
  static constexpr size_t rows = (size_t)NIN * TPB * BU * BV * 32 * sizeof(T);
  static constexpr size_t ids = (size_t)(NC + BU * BV) * sizeof(int);
  static constexpr size_t total = win + coef + rows + ids;
};

template <typename T, int P, int TPB, typename Epi>
__global__ void __launch_bounds__(BU * 32, sizeof(T) == 4 ? 2 : 1) k_sten(StenGeo G, const typename V2<T>::type* __restrict__ csm,
                                                  const T* __restrict__ src, int tiles,
                                                  const int* __restrict__ tile_active, const Epi epi_arg,
                                                  const int* __restrict__ skip_uni) {
  constexpr int BV = BvOf<P>::value;
  static_assert(TPB == 1 || TPB == 2, "tile selection below assumes at most two tiles per block");
  using C2 = typename V2<T>::type;
  using LY = SmemLayout<T, P, TPB, Epi::NIN>;
  constexpr int NIN = Epi::NIN;
  constexpr int SW = 2 * P + 1;
  constexpr int CU = LY::CU, NC = LY::NC, CS = LY::CS;
  constexpr int ROWCH = 32 * sizeof(T) / 16;  // 16-byte chunks per staged row
  constexpr int COEFCH = CS * sizeof(C2) / 16;  // 16-byte chunks per coefficient row
  Epi epi = epi_arg;  // per-thread copy (its per-tile fields live in registers)
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  C2* scf = reinterpret_cast<C2*>(smraw + LY::win);
  T* srw = reinterpret_cast<T*>(smraw + LY::win + LY::coef);      // [NIN][TPB][BU*BV][32] epilogue inputs
  int* sid = reinterpret_cast<int*>(smraw + LY::win + LY::coef + LY::rows);  // [NC] cells, then [BU*BV] rows
  int* srow = sid + NC;
  const int lane = threadIdx.x, w = threadIdx.y;
  const int tid = w * 32 + lane;
  int b = blockIdx.x;
  const int bu = b % G.nbu;
  b /= G.nbu;
  const int bv = b % G.nbv;
  const int m = b / G.nbv;
  const int t0 = blockIdx.y * TPB;
  bool act[TPB];
  bool any = false;
#pragma unroll
  for (int k = 0; k < TPB; ++k) {
    // skip_uni: tiles with a single shift are done by k_sten_uni
    act[k] = t0 + k < tiles && tile_active[t0 + k] && !(skip_uni && skip_uni[t0 + k]);
    any |= act[k];
  }
  if (!any) return;
  epi.init(t0, act);
  // phase 0: global DOF of every window cell and every output row of the block
  const int32_t* E = G.ext + (size_t)m * G.ELV * G.ELU;
  const int32_t* OWN = G.own + (size_t)m * G.nlv * G.nlu;
  for (int c = tid; c < NC + BU * BV; c += BU * 32) {
    int v = -1;
    if (c < NC) {
      int eu = bu * BU + c % CU, ev = bv * BV + c / CU;
      if (eu < G.ELU && ev < G.ELV) v = E[(size_t)ev * G.ELU + eu];
    } else {
      int o = c - NC;
      int iu = bu * BU + o % BU, iv = bv * BV + o / BU;
      if (iu < G.nlu && iv < G.nlv) v = OWN[(size_t)iv * G.nlu + iu];
    }
    sid[c] = v;
  }
  __syncthreads();
  // phase 1: asynchronous copies of the window rows and the coefficient rows
  for (int c = tid; c < TPB * NC * ROWCH; c += BU * 32) {
    int part = c % ROWCH, cell = (c / ROWCH) % NC, k = c / (ROWCH * NC);
    int gi = sid[cell];
    bool ok = gi >= 0 && (TPB == 1 ? act[0] : (k == 0 ? act[0] : act[TPB - 1]));
    const T* gp = ok ? src + ((size_t)(t0 + k) * G.N + gi) * 32 + part * (16 / sizeof(T)) : src;
    cp_async16(sm + ((size_t)k * NC + cell) * 32 + part * (16 / sizeof(T)), gp, ok ? 16 : 0);
  }
  for (int c = tid; c < BU * BV * COEFCH; c += BU * 32) {
    int part = c % COEFCH, o = c / COEFCH;
    int gi = srow[o];
    const unsigned char* gp = reinterpret_cast<const unsigned char*>(csm) +
                              (gi >= 0 ? ((size_t)gi * CS * sizeof(C2) + part * 16) : 0);
    cp_async16(reinterpret_cast<unsigned char*>(scf) + ((size_t)o * CS * sizeof(C2) + part * 16), gp,
               gi >= 0 ? 16 : 0);
  }
#pragma unroll
  for (int a = 0; a < NIN; ++a) {  // compile-time input index keeps epi in registers
    const T* base = epi.in[a];
    if (!base) continue;
    for (int c = tid; c < TPB * BU * BV * ROWCH; c += BU * 32) {
      int part = c % ROWCH, o = (c / ROWCH) % (BU * BV), k = c / (ROWCH * BU * BV);
      int gi = srow[o];
      bool ok = gi >= 0 && (TPB == 1 ? act[0] : (k == 0 ? act[0] : act[TPB - 1]));
      const T* gp = ok ? base + ((size_t)(t0 + k) * G.N + gi) * 32 + part * (16 / sizeof(T)) : src;
      cp_async16(srw + (((size_t)a * TPB + k) * BU * BV + o) * 32 + part * (16 / sizeof(T)), gp, ok ? 16 : 0);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // phase 2: each warp sweeps the column iu with a ring of SW staged rows
  const int iu = bu * BU + w;
  if (iu < G.nlu) {
    T win[TPB][SW][SW];
#pragma unroll
    for (int r = 0; r < SW - 1; ++r)
#pragma unroll
      for (int du = 0; du < SW; ++du)
#pragma unroll
        for (int k = 0; k < TPB; ++k) win[k][r][du] = sm[((size_t)k * NC + r * CU + w + du) * 32 + lane];
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      const int rn = j + SW - 1;  // staged row entering the window
#pragma unroll
      for (int du = 0; du < SW; ++du)
#pragma unroll
        for (int k = 0; k < TPB; ++k) win[k][rn % SW][du] = sm[((size_t)k * NC + rn * CU + w + du) * 32 + lane];
      const int i = srow[j * BU + w];
      if (i >= 0) {
        const C2* cf = scf + (size_t)(j * BU + w) * CS;
        T aS[TPB], aM[TPB], zc[TPB];
#pragma unroll
        for (int k = 0; k < TPB; ++k) aS[k] = aM[k] = 0;
#pragma unroll
        for (int dv = 0; dv < SW; ++dv)
#pragma unroll
          for (int du = 0; du < SW; ++du) {
            C2 c = cf[dv * SW + du];
#pragma unroll
            for (int k = 0; k < TPB; ++k) {
              T z = win[k][(j + dv) % SW][du];
              aS[k] += c.x * z;
              aM[k] += c.y * z;
            }
          }
#pragma unroll
        for (int k = 0; k < TPB; ++k) zc[k] = win[k][(j + P) % SW][P];
        T stg[NIN > 0 ? NIN : 1][TPB];
#pragma unroll
        for (int a = 0; a < NIN; ++a)
#pragma unroll
          for (int k = 0; k < TPB; ++k) stg[a][k] = srw[(((size_t)a * TPB + k) * BU * BV + j * BU + w) * 32 + lane];
        epi.row(t0, act, i, aS, aM, zc, stg);
      }
    }
  }
  epi.finish(t0, tiles, act);
}

// ------------------------------------------- operator steps, one shift per tile
// Operator-type steps for runs of consecutive tiles whose 32 systems share one
// shift sigma (sample-major packing puts the 32 samples of one sinc node in a
// tile, and the ns / 32 tiles of a node next to each other):
//   UNI_CHEB     three-term Chebyshev step  out = z + c1 (z - z_prev) + w (r - A z)
//   UNI_RESID    residual                   out = r - A z
//   UNI_APPLY    outer apply                out = A z, per-block partial (z, A z)
//   UNI_CHEBDOT  the Chebyshev step that ends a V-cycle, also forming the
//                per-block partials (r, z_new) and (z_new, q) of the outer CG
//                (q staged as a third row)
//   UNI_CHEB1    the first two pre-smoothing steps from z = 0 in one pass:
//                z1 = c2_0 Dinv r (written to out1), out = z1 + c1 z1 + c2 Dinv (r - A z1),
//                A z1 formed from the window of r with c2_0 Dinv folded into the rows
// A block owns one spatial block of one patch and a group of at most
// kUniGroup consecutive tiles of one shift (a host-built list of (first tile,
// count); `split` blocks share a group when the grid would be too small).
// Everything that depends only on the spatial block and the shift is done
// once for the group: the DOF ids of the window and of the output rows and the
// combined rows
// A = S + sigma M (with the Chebyshev weights w = c2 / (dS + sigma dM)), so an
// output costs one FMA per stencil entry and no division.  The group's tiles
// then stream through shared-memory stage buffers (cp.async copies of the
// window and the output rows).  Float p = 2 takes two (the next tile copied
// while the current one is computed) at the three blocks per SM they allow
// (measured 153.7 against 154.5 ms per bench step with one buffer at four
// blocks); p = 3 takes one (two would allow only two blocks per SM, which
// measured slower).
enum { UNI_CHEB = 0, UNI_RESID = 1, UNI_APPLY = 2, UNI_CHEBDOT = 3, UNI_CHEB1 = 4 };
// schedule constants of the one-shift kernel: stage buffers in float, output
// rows per step of a warp (0: two where the register budget allows), partial
// sums per output
#ifndef WM_UNI_NST_F32
#define WM_UNI_NST_F32 1
#endif
#ifndef WM_UNI_NST_F32_P2
#define WM_UNI_NST_F32_P2 2
#endif
#ifndef WM_UNI_RPS
#define WM_UNI_RPS 1
#endif
#ifndef WM_UNI_NACC
#define WM_UNI_NACC 1
#endif
#ifndef WM_UNI_MAXB_F32
#define WM_UNI_MAXB_F32 4
#endif
#ifndef WM_UNI_MAXB_F32_P3
#define WM_UNI_MAXB_F32_P3 4
#endif
// tiles per warp pass of the float p = 2 kernels: 0 = two for the residual and
// the outer apply (measured faster there, 5.5 vs 6.3 and 5.6 vs 5.8 ms per bench
// step) and one for the Chebyshev modes (two: 66 vs 62 ms); 1 or 2 = all modes
#ifndef WM_UNI_TPW
#define WM_UNI_TPW 0
#endif
template <int MODE>
struct UniCheb {
  static constexpr bool value = MODE == UNI_CHEB || MODE == UNI_CHEBDOT;
};
template <int MODE>
struct UniRows {  // staged 32-system rows per output row
  static constexpr int value = MODE == UNI_CHEBDOT ? 3 : (MODE == UNI_CHEB ? 2 : (MODE == UNI_RESID ? 1 : 0));
};
template <typename T, int P, int MODE>
struct UniLayout {
  static constexpr int BV = BvOf<P>::value;
  static constexpr int CU = BU + 2 * P, CV = BV + 2 * P, NC = CU * CV, S2 = (2 * P + 1) * (2 * P + 1);
  static constexpr int VEC = 16 / sizeof(T);                  // values per 16-byte load
  static constexpr int S2P = (S2 + VEC - 1) / VEC * VEC;      // padded combined row length
  static constexpr int CS = CoefStride<T, P>::value;          // (S, M) row stride of the level tables
  static constexpr int NR = UniRows<MODE>::value;
  static constexpr int ND = UniCheb<MODE>::value ? 2 : 0;     // staged diagonals dS, dM
  // tiles per warp pass (one stage buffer each) and stage buffers
  static constexpr int TPW =
      (sizeof(T) == 4 && P == 2)
          ? (WM_UNI_TPW == 0 ? ((MODE == UNI_RESID || MODE == UNI_APPLY) ? 2 : 1) : WM_UNI_TPW)
          : 1;
  static constexpr int NST = TPW == 2 ? 2 : (sizeof(T) == 4 ? (P == 2 ? WM_UNI_NST_F32_P2 : WM_UNI_NST_F32) : 1);
  static constexpr size_t win = (size_t)NC * 32 * sizeof(T);  // window of the input vector
  static constexpr size_t rows = (size_t)NR * BU * BV * 32 * sizeof(T);  // staged rows of the outputs
  static constexpr size_t stage = win + rows;
  // raw (S, M) rows, needed at set-up only: they sit in the last stage buffer
  static constexpr size_t raw = (size_t)BU * BV * CS * sizeof(typename V2<T>::type);
  static constexpr size_t last = stage > raw ? stage : raw;
  static constexpr size_t stages = (NST - 1) * stage + last;
  static constexpr size_t coef = (size_t)BU * BV * S2P * sizeof(T);  // combined rows
  static constexpr size_t diag = MODE == UNI_CHEB1 ? (size_t)3 * NC * sizeof(T)  // dS, dM, Dinv of the cells
                                                   : (size_t)(ND + 1) * BU * BV * sizeof(T);  // dS, dM, w
  static constexpr size_t diag16 = (diag + 15) / 16 * 16;
  static constexpr size_t ids = (size_t)(NC + BU * BV) * sizeof(int);
  // float Chebyshev modes: (row id, weight) of every output as one 8-byte entry
  static constexpr bool PACK_IW = UniCheb<MODE>::value && sizeof(T) == 4;
  static constexpr size_t iw = PACK_IW ? (size_t)BU * BV * sizeof(int2) : 0;
  static constexpr size_t total = stages + coef + diag16 + ids + iw;
  // 16-byte copies of one staged tile: window chunks and row chunks, and per thread
  static constexpr int ROWCH = 32 * sizeof(T) / 16;
  static constexpr int WCH = NC * ROWCH, RCH = BU * BV * ROWCH;
  static constexpr int WPT = (WCH + BU * 32 - 1) / (BU * 32), RPT = (RCH + BU * 32 - 1) / (BU * 32);
  static_assert(stage % 16 == 0 && raw % 16 == 0 && coef % 16 == 0, "16-byte aligned regions");
  static_assert(!PACK_IW || (stages + coef + diag16 + ids) % 8 == 0, "8-byte aligned (row id, weight) entries");
};
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static __device__ __forceinline__ float at(const float4& v, int k) {
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
  }
};
template <>
struct Vec16<double> {
  using type = double2;
  static __device__ __forceinline__ double at(const double2& v, int k) { return k == 0 ? v.x : v.y; }
};
// blocks per SM that the shared memory allows (with the 2 KB of the partial-sum
// reduction and the 1 KB the runtime reserves per block), at most four (float)
// or two (double: its copy offsets and window need the registers); this is
// also the register budget
template <typename T, int P, int MODE>
struct UniMinBlocks {
  static constexpr size_t per = UniLayout<T, P, MODE>::total + 3 * 1024;
  static constexpr int fit = (int)((228 * 1024) / per);
  static constexpr int cap = sizeof(T) == 4 ? (P == 3 ? WM_UNI_MAXB_F32_P3 : (UniLayout<T, P, MODE>::TPW == 2 ? 3 : WM_UNI_MAXB_F32)) : 2;
  static constexpr int value = fit >= cap ? cap : (fit < 1 ? 1 : fit);
};
// 4- or 8-byte asynchronous copy through L1 (diagonal entries)
template <int BYTES>
__device__ __forceinline__ void cp_async_ca(void* smem, const void* gmem, int src_bytes) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(gmem), "n"(BYTES), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T, int P, int MODE>
__global__ void __launch_bounds__(BU * 32, UniMinBlocks<T, P, MODE>::value)
    k_sten_uni(StenGeo G, const typename V2<T>::type* __restrict__ csm, const T* __restrict__ dS,
               const T* __restrict__ dM, const double* __restrict__ sigma, const typename V2<T>::type* __restrict__ ctab,
               const int* __restrict__ sid, int kstep, const T* __restrict__ z, const T* __restrict__ r, const T* prev,
               T* out, int tiles, const int* __restrict__ tile_active, const int2* __restrict__ groups, int split,
               double* __restrict__ part, const T* __restrict__ qd, double* __restrict__ part2,
               T* __restrict__ out1) {
  constexpr int BV = BvOf<P>::value;
  using C2 = typename V2<T>::type;
  using LY = UniLayout<T, P, MODE>;
  constexpr bool CHEB = UniCheb<MODE>::value;
  using VT = typename Vec16<T>::type;
  constexpr int SW = 2 * P + 1, CU = LY::CU, NC = LY::NC, S2 = LY::S2, S2P = LY::S2P, VEC = LY::VEC, CS = LY::CS;
  constexpr int NR = LY::NR, NST = LY::NST, ROWCH = LY::ROWCH, TPW = LY::TPW;
  constexpr int RPS = WM_UNI_RPS > 0 ? WM_UNI_RPS : (UniMinBlocks<T, P, MODE>::value >= 3 ? 1 : 2);
  constexpr int NACC = WM_UNI_NACC;
  constexpr int RW = SW + RPS - 1;     // rows of the register ring
  static_assert(BV % RPS == 0, "rows per step divide the block height");
  constexpr int EPT = 16 / sizeof(T);  // values per 16-byte chunk
  constexpr int NT = BU * 32;          // threads per block
  constexpr size_t STAGE = LY::stage / sizeof(T);  // stage buffer length in T
  extern __shared__ __align__(16) unsigned char smraw[];
  T* const stg = reinterpret_cast<T*>(smraw);  // [NST] x ([NC][32] window, [NR][64][32] rows)
  C2* const sraw = reinterpret_cast<C2*>(smraw + (NST - 1) * LY::stage);  // [64][CS], set-up only
  T* const scf = reinterpret_cast<T*>(smraw + LY::stages);                // [64][S2P]
  T* const sdg = reinterpret_cast<T*>(smraw + LY::stages + LY::coef);     // [ND][64], then w [64]
  T* const swt = sdg + LY::ND * BU * BV;
  int* const sid_ = reinterpret_cast<int*>(smraw + LY::stages + LY::coef + LY::diag16);
  int* const srow = sid_ + NC;
  int2* const siw = reinterpret_cast<int2*>(smraw + LY::stages + LY::coef + LY::diag16 + LY::ids);  // PACK_IW
  const int lane = threadIdx.x, w = threadIdx.y;
  const int tid = w * 32 + lane;
  int b = blockIdx.x;
  const int bu = b % G.nbu;
  b /= G.nbu;
  const int bv = b % G.nbv;
  const int m = b / G.nbv;
  // this block's tiles [ta, tb): part `sp` of group blockIdx.y / split
  const int2 gr = groups[blockIdx.y / split];
  const int sp = blockIdx.y % split;
  const int per = (gr.y + split - 1) / split;
  const int ta = gr.x + sp * per;
  const int tb = min(min(gr.x + gr.y, ta + per), tiles);
  unsigned todo = 0;  // active tiles of the range, bit t - ta (at most kUniGroup bits)
  for (int t = ta; t < tb; ++t)
    if (tile_active[t]) todo |= 1u << (t - ta);
  if (todo == 0) return;
  T sg, c1 = 0, c2 = 0, c20 = 0;
  {
    const int g = gr.x * 32;  // every system of the group has this shift
    if constexpr (CHEB) {
      const C2 c = ctab[sid[g] * WM_MAX_CHEB + kstep];
      c1 = kstep == 0 ? (T)0 : c.x;
      c2 = c.y;
    }
    if constexpr (MODE == UNI_CHEB1) {  // steps 0 and 1
      const C2 c0 = ctab[sid[g] * WM_MAX_CHEB], c = ctab[sid[g] * WM_MAX_CHEB + 1];
      c20 = c0.y;
      c1 = c.x;
      c2 = c.y;
    }
    sg = (T)sigma[g];
  }
  // set-up 1: global DOF of every window cell and every output row
  const int32_t* E = G.ext + (size_t)m * G.ELV * G.ELU;
  const int32_t* OWN = G.own + (size_t)m * G.nlv * G.nlu;
  for (int c = tid; c < NC + BU * BV; c += NT) {
    int v = -1;
    if (c < NC) {
      int eu = bu * BU + c % CU, ev = bv * BV + c / CU;
      if (eu < G.ELU && ev < G.ELV) v = E[ev * G.ELU + eu];
    } else {
      int o = c - NC;
      int iu = bu * BU + o % BU, iv = bv * BV + o / BU;
      if (iu < G.nlu && iv < G.nlv) v = OWN[iv * G.nlu + iu];
    }
    sid_[c] = v;
  }
  __syncthreads();
  // set-up 2: (S, M) rows and diagonals, copy offsets
  constexpr int RAWCH = CS * (int)sizeof(C2) / 16;  // 16-byte chunks per (S, M) row
  for (int c = tid; c < BU * BV * RAWCH; c += NT) {
    const int part16 = c % RAWCH, o = c / RAWCH;
    const int gi = srow[o];
    cp_async16(reinterpret_cast<unsigned char*>(sraw) + o * (CS * sizeof(C2)) + part16 * 16,
               gi >= 0 ? reinterpret_cast<const unsigned char*>(csm + (size_t)gi * CS) + part16 * 16
                       : reinterpret_cast<const unsigned char*>(csm),
               gi >= 0 ? 16 : 0);
  }
  if constexpr (MODE == UNI_CHEB1) {  // diagonals of every window cell
    for (int c = tid; c < 2 * NC; c += NT) {
      const int gi = sid_[c % NC];
      const T* base = c < NC ? dS : dM;
      cp_async_ca<sizeof(T)>(sdg + c, gi >= 0 ? base + gi : dS, gi >= 0 ? (int)sizeof(T) : 0);
    }
  }
  if constexpr (CHEB) {
    for (int c = tid; c < 2 * BU * BV; c += NT) {
      const int gi = srow[c % (BU * BV)];
      const T* base = c < BU * BV ? dS : dM;
      cp_async_ca<sizeof(T)>(sdg + c, gi >= 0 ? base + gi : dS, gi >= 0 ? (int)sizeof(T) : 0);
    }
  }
  cp_async_commit();
  // each thread's source offsets (within a tile) of its window and row
  // chunks: -1 zero-fills a cell outside the surface, -2 marks no chunk
  int woff[LY::WPT];
#pragma unroll
  for (int k = 0; k < LY::WPT; ++k) {
    const int c = tid + k * NT;
    int o = -2;
    if (c < LY::WCH) {
      const int gi = sid_[c / ROWCH];
      o = gi >= 0 ? gi * 32 + (c % ROWCH) * EPT : -1;
    }
    woff[k] = o;
  }
  int roff[NR > 0 ? LY::RPT : 1];
#pragma unroll
  for (int k = 0; k < (NR > 0 ? LY::RPT : 1); ++k) {
    const int c = tid + k * NT;
    int o = -2;
    if (NR > 0 && c < LY::RCH) {
      const int gi = srow[c / ROWCH];
      o = gi >= 0 ? gi * 32 + (c % ROWCH) * EPT : -1;
    }
    roff[k] = o;
  }
  // the 16-byte copies of tile t into stage buffer `buf` (chunk c of the
  // window lands at element c * EPT, chunk c of row input a at NC * 32 +
  // a * 64 * 32 + c * EPT); absent inputs (z_prev, q) are not copied
  auto issue = [&](int t, T* buf) {
    const size_t to = (size_t)t * G.N * 32;
#pragma unroll
    for (int k = 0; k < LY::WPT; ++k) {
      const int o = woff[k];
      if (o != -2) cp_async16(buf + (tid + k * NT) * EPT, o >= 0 ? z + to + o : z, o >= 0 ? 16 : 0);
    }
#pragma unroll
    for (int a = 0; a < NR; ++a) {
      const T* base = a == 0 ? r : (a == 1 ? prev : qd);
      if (base == nullptr) continue;
#pragma unroll
      for (int k = 0; k < LY::RPT; ++k) {
        const int o = roff[k];
        if (o != -2)
          cp_async16(buf + NC * 32 + a * BU * BV * 32 + (tid + k * NT) * EPT, o >= 0 ? base + to + o : base,
                     o >= 0 ? 16 : 0);
      }
    }
    cp_async_commit();
  };
  // tiles go through the stage buffers TPW at a time (a pair shares every load
  // of the combined rows); with PREFETCH the next tile is copied while the
  // current one is computed
  constexpr bool PREFETCH = NST == 2 && TPW == 1;
  int cur = __ffs(todo) - 1;
  todo &= todo - 1;
  if constexpr (PREFETCH) {  // the first tile goes to buffer 0 (the raw rows sit in buffer 1)
    issue(ta + cur, stg);
    cp_async_wait<1>();
  } else {
    cp_async_wait<0>();
  }
  __syncthreads();
  T* sdc = sdg + 2 * NC;  // UNI_CHEB1: Dinv of every window cell
  if constexpr (MODE == UNI_CHEB1) {
    for (int c = tid; c < NC; c += NT) sdc[c] = sid_[c] >= 0 ? (T)1 / (sdg[c] + sg * sdg[NC + c]) : (T)0;
    __syncthreads();
  }
  // set-up 3: combined rows and the Chebyshev diagonal weights
  for (int c = tid; c < BU * BV * S2P; c += NT) {
    const int o = c / S2P, sl = c - o * S2P;
    T a = 0;
    if (sl < S2) {
      const C2 q = sraw[o * CS + sl];
      a = q.x + sg * q.y;
      if constexpr (MODE == UNI_CHEB1)  // times c2_0 Dinv of the neighbour's cell: A z1 from r
        a *= c20 * sdc[((o / BU) + sl / SW) * CU + (o % BU) + sl % SW];
    }
    scf[c] = a;
  }
  if constexpr (CHEB)
    for (int c = tid; c < BU * BV; c += NT) {
      const T wc = srow[c] >= 0 ? c2 / (sdg[c] + sg * sdg[BU * BV + c]) : (T)0;
      swt[c] = wc;
      if constexpr (LY::PACK_IW) siw[c] = make_int2(srow[c], __float_as_int((float)wc));
    }
  __syncthreads();  // the raw rows are dead from here on (buffer 1 may be refilled)
  const int iu = bu * BU + w;
  int bsel = 0;
  for (;;) {
    // the tiles of this pass: tt[u] in buffer u (with PREFETCH, buffer bsel)
    int tt[TPW];
    bool ok[TPW];
    tt[0] = ta + cur;
    ok[0] = true;
    if constexpr (TPW == 2) {
      ok[1] = todo != 0;
      const int c1 = ok[1] ? __ffs(todo) - 1 : cur;
      if (ok[1]) todo &= todo - 1;
      tt[1] = ta + c1;
    }
    const bool more = todo != 0;
    const int nxt = more ? __ffs(todo) - 1 : 0;
    if constexpr (PREFETCH) {
      if (more) {
        issue(ta + nxt, stg + (bsel ^ 1) * STAGE);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
    } else {
      issue(tt[0], stg);
      if constexpr (TPW == 2)
        if (ok[1]) issue(tt[1], stg + STAGE);
      cp_async_wait<0>();
    }
    __syncthreads();
    // each warp sweeps the column iu, RPS output rows per step, with a ring of
    // RW staged rows in registers per tile; every output sums its stencil in
    // NACC partial sums (stencil rows dv mod NACC), and each combined-row load
    // serves the TPW tiles of the pass
    const T* smv[TPW];
    const T* srwv[TPW];
#pragma unroll
    for (int u = 0; u < TPW; ++u) {
      smv[u] = PREFETCH ? stg + bsel * STAGE : stg + ((TPW == 2 && !ok[u]) ? 0 : u) * STAGE;
      srwv[u] = smv[u] + NC * 32;
    }
    DAcc<T> dot[TPW];   // UNI_APPLY: (z, A z); UNI_CHEBDOT: (r, z_new) over this thread's outputs
    DAcc<T> dot2[TPW];  // UNI_CHEBDOT: (z_new, q)
    if (iu < G.nlu) {
      T win[TPW][RW][SW];
#pragma unroll
      for (int u = 0; u < TPW; ++u)
#pragma unroll
        for (int rr = 0; rr < SW - 1; ++rr)
#pragma unroll
          for (int du = 0; du < SW; ++du) win[u][rr][du] = smv[u][(rr * CU + w + du) * 32 + lane];
#pragma unroll
      for (int j = 0; j < BV; j += RPS) {
#pragma unroll
        for (int e = 0; e < RPS; ++e) {
          const int rn = j + SW - 1 + e;  // staged rows entering the window
#pragma unroll
          for (int u = 0; u < TPW; ++u)
#pragma unroll
            for (int du = 0; du < SW; ++du) win[u][rn % RW][du] = smv[u][(rn * CU + w + du) * 32 + lane];
        }
        T acc[TPW][RPS][NACC];
#pragma unroll
        for (int u = 0; u < TPW; ++u)
#pragma unroll
          for (int k = 0; k < RPS; ++k)
#pragma unroll
            for (int h = 0; h < NACC; ++h) acc[u][k][h] = 0;
#pragma unroll
        for (int q = 0; q < S2P / VEC; ++q) {
          VT a[RPS];
#pragma unroll
          for (int k = 0; k < RPS; ++k) a[k] = reinterpret_cast<const VT*>(scf + ((j + k) * BU + w) * S2P)[q];
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const int sl = q * VEC + e;
            if (sl < S2) {
              const int dv = sl / SW, du = sl % SW;
#pragma unroll
              for (int k = 0; k < RPS; ++k)
#pragma unroll
                for (int u = 0; u < TPW; ++u)
                  acc[u][k][dv % NACC] =
                      fma(Vec16<T>::at(a[k], e), win[u][(j + k + dv) % RW][du], acc[u][k][dv % NACC]);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < RPS; ++k) {
          const int jj = j + k;
          const int o = jj * BU + w;
          int i;
          T wo = 0;  // the output's Chebyshev weight (one 8-byte load with its row id in float)
          if constexpr (LY::PACK_IW) {
            const int2 iw = siw[o];
            i = iw.x;
            wo = __int_as_float(iw.y);
          } else {
            i = srow[o];
            if constexpr (CHEB) wo = swt[o];
          }
          if (i < 0) continue;
#pragma unroll
          for (int u = 0; u < TPW; ++u) {
            if (!ok[u]) continue;
            const T* const srw = srwv[u];
            const int t = tt[u];
            T az = acc[u][k][0];
#pragma unroll
            for (int h = 1; h < NACC; ++h) az += acc[u][k][h];
            const T zc = win[u][(jj + P) % RW][P];
            T res;
            if constexpr (CHEB) {
              const T rv = srw[o * 32 + lane];
              const T zp = prev ? srw[(BU * BV + o) * 32 + lane] : (T)0;
              res = zc + c1 * (zc - zp) + wo * (rv - az);
              if constexpr (MODE == UNI_CHEBDOT) {
                dot[u].add(rv * res);
                if (qd) dot2[u].add(res * srw[(2 * BU * BV + o) * 32 + lane]);
              }
            } else if constexpr (MODE == UNI_CHEB1) {
              const T dc = sdc[(jj + P) * CU + w + P];  // Dinv of the output row
              const T z1 = c20 * dc * zc;               // zc is r here
              out1[((size_t)t * G.N + i) * 32 + lane] = z1;
              res = z1 + c1 * z1 + c2 * dc * (zc - az);
            } else if constexpr (MODE == UNI_RESID) {
              res = srw[o * 32 + lane] - az;
            } else {
              res = az;
              dot[u].add(zc * az);
            }
            out[((size_t)t * G.N + i) * 32 + lane] = res;
          }
        }
      }
    }
    if constexpr (MODE == UNI_APPLY || MODE == UNI_CHEBDOT) {
      const bool one[1] = {true};
#pragma unroll
      for (int u = 0; u < TPW; ++u) {
        if (!ok[u]) continue;  // uniform over the block
        if (u > 0) __syncthreads();
        double a1[1] = {dot[u].get()};
        block_reduce<1>(a1, part, tt[u], tiles, one);
        if (MODE == UNI_CHEBDOT && qd) {
          __syncthreads();
          a1[0] = dot2[u].get();
          block_reduce<1>(a1, part2, tt[u], tiles, one);
        }
      }
    }
    __syncthreads();  // the stage buffers (and the reduction buffer) may be refilled
    if (!more) break;
    todo &= todo - 1;
    cur = nxt;
    if constexpr (PREFETCH) bsel ^= 1;
  }
}

template <typename T, int P, int TPB, int NIN>
constexpr size_t smem_bytes() {
  return SmemLayout<T, P, TPB, NIN>::total;
}

StenGeo geo_of(const wm_level& L) {
  StenGeo G;
  G.nlu = L.nlu;
  G.nlv = L.nlv;
  G.ELU = L.ELU;
  G.ELV = L.ELV;
  G.nbu = L.nbu;
  G.nbv = L.nbv;
  G.N = L.N;
  G.ext = L.d_ext.p;
  G.own = L.d_own.p;
  return G;
}

template <typename T>
const typename V2<T>::type* csm_of(const wm_level& L);
template <>
const float2* csm_of<float>(const wm_level& L) { return L.d_csm32.p; }
template <>
const double2* csm_of<double>(const wm_level& L) { return L.d_csm64.p; }

// tiles per block: two float tiles for p <= 2 (register window 2 x 25), one otherwise
template <typename T, int P>
struct Tpb {
  static constexpr int value = (sizeof(T) == 4 && P <= 2) ? 2 : 1;
};

template <typename T, int P, typename Epi>
int launch(const wm_level& L, int np, int tiles, const T* src, const int* tile_active, Epi epi, int cat,
           cudaStream_t s, const int* skip_uni = nullptr) {
  constexpr int TPB = Tpb<T, P>::value;
  constexpr size_t sm = smem_bytes<T, P, TPB, Epi::NIN>();
  static bool configured = false;
  if (!configured) {
    WM_CUDA(cudaFuncSetAttribute(k_sten<T, P, TPB, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    configured = true;
  }
  dim3 grid(np * L.nbu * L.nbv, (tiles + TPB - 1) / TPB);
  WM_LAUNCH(cat, s, k_sten<T, P, TPB, Epi><<<grid, dim3(32, BU), sm, s>>>(geo_of(L), csm_of<T>(L), src, tiles,
                                                                           tile_active, epi, skip_uni));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// ------------------------------------------- double-float true residual
// r = b - (S x + sigma M x) of the systems flagged for residual replacement,
// with every operation on the FP32 pipes: the FP64 rate of this part is
// about 1/60 of its FP32 rate (conversions to and from float64 run there
// too), so the kernel never touches a float64 register in its loops.
//  * float64 inputs (x, b, sigma) are split into float pairs hi + lo with
//    integer operations on their bits (relative error at most 2^-47);
//  * each product a*x is the rounded hi*hi plus its exact rounding error
//    (FMA) plus the two cross terms; the rounded products are summed with
//    Knuth's two-sum and all errors gathered in a float tail (about 48
//    significant bits for the stencil sum);
//  * where the 32 shifts of a tile are equal (sample-major packing) each
//    coefficient row is combined once per block into A = S + sigma M in the
//    same arithmetic and one sum is formed, two output rows at a time on the
//    packed FP32 instructions (FMUL2/FFMA2/FADD2, rounding per component as
//    the scalar ones); otherwise S x and M x are summed separately and
//    combined per output.
// Each output also accumulates B_i = sum_j |a_ij x_j| (float, from the rounded
// hi products, within a factor 1 + 2^-22 of the exact sum): the entry's
// rounding error stays below 2^-42 B_i (operand splits 2^-47 and 2^-48,
// dropped lo*lo and cross-term roundings 2^-47, float tail 25 x 2^-47), and the
// caller checks 2^-42 ||B|| against the convergence tolerance before it
// trusts the residuals, recomputing them in float64 otherwise (also when a
// value of the system is below 2^-102, where float pairs lose precision).
// The squared norms are accumulated in float over the 8 outputs of a thread
// (entries of r below about 1e-22 in magnitude lose their contribution).

// v = hi + lo with hi = v rounded to 24 significant bits and lo the rest
// rounded to float: |v - hi - lo| <= 2^-47 |v| (2^-48 while lo is a normal
// float), using integer operations on
// the bits of v and one int->float conversion.  Non-finite v or |v| >= 2^128
// gives hi = +-inf; 0 < |v| < 2^-102 (lo would be subnormal) sets `tiny` and
// returns (+-0, 0).
__device__ __forceinline__ float2 split_bits(double v, bool& tiny) {
  // 32-bit halves only (no 64-bit integer or float64 instructions)
  const unsigned hi32 = (unsigned)__double2hiint(v), lo32 = (unsigned)__double2loint(v);
  const unsigned sign = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7FFu);
  if (e < 921) {
    tiny |= ((hi32 & 0x7FFFFFFFu) | lo32) != 0u;
    return make_float2(__int_as_float((int)sign), 0.f);
  }
  if (e >= 1151) return make_float2(__int_as_float((int)(sign | 0x7F800000u)), 0.f);
  // round the magnitude to the nearest multiple of 2^29 units (24 significant
  // bits; a carry into the exponent is the correct rounding)
  const unsigned lr = lo32 + 0x10000000u;
  const unsigned hr = (hi32 & 0x7FFFFFFFu) + (lr < lo32 ? 1u : 0u);
  const unsigned hl = lr & 0xE0000000u;
  const int rem = (int)(lo32 - hl);  // |rem| <= 2^28 units of 2^(e-1075)
  const int efh = (int)(hr >> 20) - 896;
  if (efh >= 255) return make_float2(__int_as_float((int)(sign | 0x7F800000u)), 0.f);
  const float h = __int_as_float((int)(sign | ((unsigned)efh << 23) | ((hr & 0xFFFFFu) << 3) | (hl >> 29)));
  const float l = __fmul_rn(__fmul_rn(__int2float_rn(rem), 3.7252902984619141e-09f /* 2^-28 */),
                            __int_as_float((e - 920) << 23) /* 2^(e-1047) */);
  return make_float2(h, sign ? -l : l);
}
// error-free sum: a + b = s + e exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
// (s, c) += (ah + al) * (xh + xl), dropping al * xl; bnd += |ah xh|
__device__ __forceinline__ void df_acc(float& s, float& c, float& bnd, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  bnd = __fadd_rn(bnd, fabsf(p));
  float e = fmaf(ah, xh, -p);
  e = fmaf(ah, xl, fmaf(al, xh, e));
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}
// (ah + al) + (gh + gl) * (mh + ml) as a renormalised pair
__device__ __forceinline__ float2 df_axpy(float ah, float al, float gh, float gl, float mh, float ml) {
  const float p = __fmul_rn(gh, mh);
  float e = fmaf(gh, mh, -p);
  e = fmaf(gh, ml, fmaf(gl, mh, e));
  float t, err;
  two_sum(ah, p, t, err);
  const float lo = __fadd_rn(al, __fadd_rn(e, err));
  float h, l;
  two_sum(t, lo, h, l);
  return make_float2(h, l);
}

// the same accumulation for two outputs at once on the packed FP32 pipe
// (FMUL2 / FFMA2 / FADD2: each component rounds exactly as the scalar form)
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ void df_acc2(float2& s, float2& c, float& b0, float& b1, float2 ah, float2 al, float2 xh,
                                        float2 xl) {
  const float2 p = __fmul2_rn(ah, xh);
  b0 = __fadd_rn(b0, fabsf(p.x));
  b1 = __fadd_rn(b1, fabsf(p.y));
  float2 e = __ffma2_rn(ah, xh, neg2(p));
  e = __ffma2_rn(ah, xl, __ffma2_rn(al, xh, e));
  const float2 t = __fadd2_rn(s, p);
  const float2 bp = __fadd2_rn(t, neg2(s));
  const float2 err = __fadd2_rn(__fadd2_rn(s, neg2(__fadd2_rn(t, neg2(bp)))), __fadd2_rn(p, neg2(bp)));
  s = t;
  c = __fadd2_rn(c, __fadd2_rn(err, e));
}

template <int P>
struct DfLayout {
  static constexpr int BV = BvOf<P>::value;
  static constexpr int CU = BU + 2 * P, CV = BV + 2 * P, NC = CU * CV, S2 = (2 * P + 1) * (2 * P + 1);
  static constexpr size_t win = (size_t)NC * 32 * sizeof(double);
  static constexpr size_t coef = (size_t)BU * BV * S2 * sizeof(float4);
  static constexpr size_t ids = (size_t)(NC + BU * BV) * sizeof(int);
  static constexpr size_t total = win + coef + ids;
};

template <int P>
__global__ void __launch_bounds__(BU * 32, 2)
    k_sten_trueres_df(StenGeo G, const float4* __restrict__ cdf, const double* __restrict__ x, int tiles,
                      const int* __restrict__ tile_rep, const double* __restrict__ sigma,
                      const double* __restrict__ rhs, const int* __restrict__ src_of, const int* __restrict__ rep,
                      float* __restrict__ r, double* __restrict__ part, double* __restrict__ part_bound,
                      const int* __restrict__ skip_uni) {
  constexpr int BV = BvOf<P>::value;
  using LY = DfLayout<P>;
  constexpr int SW = 2 * P + 1, CU = LY::CU, NC = LY::NC, S2 = LY::S2;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* smd = reinterpret_cast<double*>(smraw);
  float2* smf = reinterpret_cast<float2*>(smraw);  // the same cells after the split
  float4* scf = reinterpret_cast<float4*>(smraw + LY::win);
  int* sid = reinterpret_cast<int*>(smraw + LY::win + LY::coef);
  int* srow = sid + NC;
  const int lane = threadIdx.x, w = threadIdx.y;
  const int tid = w * 32 + lane;
  int b = blockIdx.x;
  const int bu = b % G.nbu;
  b /= G.nbu;
  const int bv = b % G.nbv;
  const int m = b / G.nbv;
  const int t = blockIdx.y;
  if (t >= tiles || !tile_rep[t] || (skip_uni && skip_uni[t])) return;  // skip: done by the group kernel
  const int g = t * 32 + lane;
  const double sg = sigma[g];
  bool tiny = false;  // a value of this system too small for float pairs
  const float2 sgp = split_bits(sg, tiny);
  tiny = false;       // (a tiny shift only loses its own negligible part)
  const bool mine = rep[g] != 0;
  const int src = src_of[g];
  // phase 0: global DOF of every window cell and every output row
  const int32_t* E = G.ext + (size_t)m * G.ELV * G.ELU;
  const int32_t* OWN = G.own + (size_t)m * G.nlv * G.nlu;
  for (int c = tid; c < NC + BU * BV; c += BU * 32) {
    int v = -1;
    if (c < NC) {
      int eu = bu * BU + c % CU, ev = bv * BV + c / CU;
      if (eu < G.ELU && ev < G.ELV) v = E[(size_t)ev * G.ELU + eu];
    } else {
      int o = c - NC;
      int iu = bu * BU + o % BU, iv = bv * BV + o / BU;
      if (iu < G.nlu && iv < G.nlv) v = OWN[(size_t)iv * G.nlu + iu];
    }
    sid[c] = v;
  }
  __syncthreads();
  // phase 1: window rows of x (16 chunks of 16 bytes each) and coefficient rows
  for (int c = tid; c < NC * 16; c += BU * 32) {
    int part16 = c % 16, cell = c / 16;
    int gi = sid[cell];
    const double* gp = gi >= 0 ? x + ((size_t)t * G.N + gi) * 32 + part16 * 2 : x;
    cp_async16(smd + (size_t)cell * 32 + part16 * 2, gp, gi >= 0 ? 16 : 0);
  }
  for (int c = tid; c < BU * BV * S2; c += BU * 32) {
    int o = c / S2, k = c % S2;
    int gi = srow[o];
    const float4* gp = gi >= 0 ? cdf + (size_t)gi * S2 + k : cdf;
    cp_async16(scf + c, gp, gi >= 0 ? 16 : 0);
  }
  cp_async_wait_all();
  __syncthreads();
  // split x in place; combine the rows when the tile's shifts are equal
  __shared__ int s_tiny[BU][32];
  for (int c = tid; c < NC * 32; c += BU * 32) smf[c] = split_bits(smd[c], tiny);  // lane c % 32 == lane
  s_tiny[w][lane] = tiny;
  // equal shifts compared bit for bit (the same answer in every warp of the
  // block); both shuffles run on all 32 lanes before any comparison
  const int sgh = __double2hiint(sg), sgl = __double2loint(sg);
  const int sgh0 = __shfl_sync(0xffffffffu, sgh, 0);
  const int sgl0 = __shfl_sync(0xffffffffu, sgl, 0);
  const bool uni = __all_sync(0xffffffffu, (sgh == sgh0) & (sgl == sgl0));
  if (uni) {
    // combined rows A = S + sigma M, rewritten in place as row pairs: entry
    // (pair jj*BU + w, slot) = (A_hi of rows 2jj and 2jj+1, A_lo of both), the
    // operand layout of the packed two-row loop below
    constexpr int NPS = BU * (BV / 2) * S2;            // pair-slot entries
    constexpr int KPT = (NPS + BU * 32 - 1) / (BU * 32);  // per thread
    float4 pv[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int c = tid + k * BU * 32;
      if (c < NPS) {
        const int pi = c / S2, sl = c - pi * S2;
        const int o0 = (pi / BU) * 2 * BU + pi % BU;  // rows 2jj and 2jj+1 of column w
        const float4 q0 = scf[o0 * S2 + sl], q1 = scf[(o0 + BU) * S2 + sl];
        const float2 a0 = df_axpy(q0.x, q0.y, sgp.x, sgp.y, q0.z, q0.w);
        const float2 a1 = df_axpy(q1.x, q1.y, sgp.x, sgp.y, q1.z, q1.w);
        pv[k] = make_float4(a0.x, a1.x, a0.y, a1.y);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int c = tid + k * BU * 32;
      if (c < NPS) scf[c] = pv[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < BU; ++k) tiny |= s_tiny[k][lane] != 0;
  float acc = 0.f, accb = 0.f;
  const int iu = bu * BU + w;
  auto emit = [&](int i, float s, float c, float bnd) {
    if (!mine) return;
    const float2 bp = split_bits(src >= 0 ? rhs[((size_t)(src / 32) * G.N + i) * 32 + (src % 32)] : 0.0, tiny);
    float d, de;
    two_sum(bp.x, -s, d, de);
    const float rt = __fadd_rn(d, __fadd_rn(de, __fsub_rn(bp.y, c)));
    r[((size_t)t * G.N + i) * 32 + lane] = rt;
    acc = fmaf(rt, rt, acc);
    accb = fmaf(bnd, bnd, accb);
  };
  if (iu < G.nlu && uni) {
#pragma unroll 1
    for (int j = 0; j < BV; j += 2) {
      const int i0 = srow[j * BU + w], i1 = srow[(j + 1) * BU + w];
      if (i0 < 0 && i1 < 0) continue;  // rows past the patch edge or owned by another patch
      const float4* cf = scf + (size_t)((j / 2) * BU + w) * S2;  // row pair (j, j+1)
      const float2* zw = smf + ((size_t)j * CU + w) * 32 + lane;
      float2 sp = make_float2(0.f, 0.f), cp = make_float2(0.f, 0.f);
      float b0 = 0.f, b1 = 0.f;
#pragma unroll
      for (int dv = 0; dv < SW; ++dv)
#pragma unroll
        for (int du = 0; du < SW; ++du) {
          const float4 q = cf[dv * SW + du];
          const float2 z0 = zw[(dv * CU + du) * 32], z1 = zw[((dv + 1) * CU + du) * 32];
          df_acc2(sp, cp, b0, b1, make_float2(q.x, q.y), make_float2(q.z, q.w), make_float2(z0.x, z1.x),
                  make_float2(z0.y, z1.y));
        }
      if (i0 >= 0) emit(i0, sp.x, cp.x, b0);
      if (i1 >= 0) emit(i1, sp.y, cp.y, b1);
    }
  } else if (iu < G.nlu) {
#pragma unroll 1
    for (int j = 0; j < BV; ++j) {
      const int i = srow[j * BU + w];
      if (i < 0) continue;
      const float4* cf = scf + (size_t)(j * BU + w) * S2;
      const float2* zw = smf + ((size_t)j * CU + w) * 32 + lane;
      float s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll 1  // a full unroll makes the scheduler hoist every operand load (spills)
      for (int dv = 0; dv < SW; ++dv)
#pragma unroll
        for (int du = 0; du < SW; ++du) {
          float4 q = cf[dv * SW + du];
          float2 z = zw[(dv * CU + du) * 32];
          df_acc(s1, c1, b1, q.x, q.y, z.x, z.y);
          df_acc(s2, c2, b2, q.z, q.w, z.x, z.y);
        }
      if (i >= 0) {
        // (s1, c1) + sigma (s2, c2)
        float2 a = df_axpy(s1, c1, sgp.x, sgp.y, s2, c2);
        emit(i, a.x, a.y, fmaf(sgp.x, b2, b1));
      }
    }
  }
  const bool one[1] = {true};
  double a2[1] = {(double)acc};
  block_reduce<1>(a2, part, t, tiles, one);
  __syncthreads();
  a2[0] = tiny && mine ? HUGE_VAL : (double)accb;  // fails the caller's error check
  block_reduce<1>(a2, part_bound, t, tiles, one);
}

// The same residual for groups of one-shift tiles (the list of the one-shift
// kernel): a block computes its window's DOF ids and the combined double-float
// rows A = S + sigma M of its shift once, then streams the x windows of the
// group's flagged tiles through shared memory.
template <int P>
struct DfUniLayout {
  static constexpr int BV = BvOf<P>::value;
  static constexpr int CU = BU + 2 * P, CV = BV + 2 * P, NC = CU * CV, S2 = (2 * P + 1) * (2 * P + 1);
  static constexpr size_t win = (size_t)NC * 32 * sizeof(double);          // x window (raw rows at set-up)
  static constexpr size_t raw = (size_t)BU * BV * S2 * sizeof(float4);      // (S_hi, S_lo, M_hi, M_lo) rows
  static constexpr size_t pairs = (size_t)BU * (BV / 2) * S2 * sizeof(float4);  // combined row pairs
  static constexpr size_t ids = (size_t)(NC + BU * BV) * sizeof(int);
  static constexpr size_t total = win + pairs + ids;
  static_assert(raw <= win, "the raw rows are staged in the window area");
};

template <int P>
__global__ void __launch_bounds__(BU * 32, 3)
    k_sten_trueres_df_uni(StenGeo G, const float4* __restrict__ cdf, const double* __restrict__ x, int tiles,
                          const int* __restrict__ tile_rep, const int2* __restrict__ groups, int split,
                          const double* __restrict__ sigma, const double* __restrict__ rhs,
                          const int* __restrict__ src_of, const int* __restrict__ rep, float* __restrict__ r,
                          double* __restrict__ part, double* __restrict__ part_bound) {
  constexpr int BV = BvOf<P>::value;
  using LY = DfUniLayout<P>;
  constexpr int SW = 2 * P + 1, CU = LY::CU, NC = LY::NC, S2 = LY::S2;
  constexpr int NT = BU * 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* smd = reinterpret_cast<double*>(smraw);
  float2* smf = reinterpret_cast<float2*>(smraw);  // the same cells after the split
  float4* sraw = reinterpret_cast<float4*>(smraw);  // set-up only
  float4* scf = reinterpret_cast<float4*>(smraw + LY::win);
  int* sid = reinterpret_cast<int*>(smraw + LY::win + LY::pairs);
  int* srow = sid + NC;
  __shared__ int s_tiny[BU][32];
  const int lane = threadIdx.x, w = threadIdx.y;
  const int tid = w * 32 + lane;
  int b = blockIdx.x;
  const int bu = b % G.nbu;
  b /= G.nbu;
  const int bv = b % G.nbv;
  const int m = b / G.nbv;
  const int2 gr = groups[blockIdx.y / split];
  const int sp = blockIdx.y % split;
  const int per = (gr.y + split - 1) / split;
  const int ta = gr.x + sp * per;
  const int tb = min(min(gr.x + gr.y, ta + per), tiles);
  unsigned todo = 0;  // flagged tiles of the range, bit t - ta
  for (int t = ta; t < tb; ++t)
    if (tile_rep[t]) todo |= 1u << (t - ta);
  if (todo == 0) return;
  bool tiny = false;
  const float2 sgp = split_bits(sigma[gr.x * 32], tiny);  // the group's shift (a tiny shift only loses itself)
  // set-up: global DOF of every window cell and every output row
  const int32_t* E = G.ext + (size_t)m * G.ELV * G.ELU;
  const int32_t* OWN = G.own + (size_t)m * G.nlv * G.nlu;
  for (int c = tid; c < NC + BU * BV; c += NT) {
    int v = -1;
    if (c < NC) {
      int eu = bu * BU + c % CU, ev = bv * BV + c / CU;
      if (eu < G.ELU && ev < G.ELV) v = E[(size_t)ev * G.ELU + eu];
    } else {
      int o = c - NC;
      int iu = bu * BU + o % BU, iv = bv * BV + o / BU;
      if (iu < G.nlu && iv < G.nlv) v = OWN[(size_t)iv * G.nlu + iu];
    }
    sid[c] = v;
  }
  __syncthreads();
  for (int c = tid; c < BU * BV * S2; c += NT) {
    const int o = c / S2, k = c % S2;
    const int gi = srow[o];
    cp_async16(sraw + c, gi >= 0 ? cdf + (size_t)gi * S2 + k : cdf, gi >= 0 ? 16 : 0);
  }
  cp_async_wait_all();
  __syncthreads();
  // combined rows A = S + sigma M as row pairs: entry (pair jj*BU + w, slot) =
  // (A_hi of rows 2jj and 2jj+1, A_lo of both), the operands of the packed loop
  for (int c = tid; c < BU * (BV / 2) * S2; c += NT) {
    const int pi = c / S2, sl = c - pi * S2;
    const int o0 = (pi / BU) * 2 * BU + pi % BU;  // rows 2jj and 2jj+1 of column w
    const float4 q0 = sraw[o0 * S2 + sl], q1 = sraw[(o0 + BU) * S2 + sl];
    const float2 a0 = df_axpy(q0.x, q0.y, sgp.x, sgp.y, q0.z, q0.w);
    const float2 a1 = df_axpy(q1.x, q1.y, sgp.x, sgp.y, q1.z, q1.w);
    scf[c] = make_float4(a0.x, a1.x, a0.y, a1.y);
  }
  __syncthreads();  // the raw rows are dead: the window area is free
  const int iu = bu * BU + w;
  while (todo) {
    const int t = ta + __ffs(todo) - 1;
    todo &= todo - 1;
    const int g = t * 32 + lane;
    const bool mine = rep[g] != 0;
    const int src = src_of[g];
    for (int c = tid; c < NC * 16; c += NT) {  // x window: 16 chunks of 16 bytes per cell
      const int part16 = c % 16, cell = c / 16;
      const int gi = sid[cell];
      cp_async16(smd + (size_t)cell * 32 + part16 * 2, gi >= 0 ? x + ((size_t)t * G.N + gi) * 32 + part16 * 2 : x,
                 gi >= 0 ? 16 : 0);
    }
    cp_async_wait_all();
    __syncthreads();
    tiny = false;
    for (int c = tid; c < NC * 32; c += NT) smf[c] = split_bits(smd[c], tiny);  // lane c % 32 == lane
    s_tiny[w][lane] = tiny;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BU; ++k) tiny |= s_tiny[k][lane] != 0;
    float acc = 0.f, accb = 0.f;
    auto emit = [&](int i, float s, float c, float bnd) {
      if (!mine) return;
      const float2 bp = split_bits(src >= 0 ? rhs[((size_t)(src / 32) * G.N + i) * 32 + (src % 32)] : 0.0, tiny);
      float d, de;
      two_sum(bp.x, -s, d, de);
      const float rt = __fadd_rn(d, __fadd_rn(de, __fsub_rn(bp.y, c)));
      r[((size_t)t * G.N + i) * 32 + lane] = rt;
      acc = fmaf(rt, rt, acc);
      accb = fmaf(bnd, bnd, accb);
    };
    if (iu < G.nlu) {
#pragma unroll 1
      for (int j = 0; j < BV; j += 2) {
        const int i0 = srow[j * BU + w], i1 = srow[(j + 1) * BU + w];
        if (i0 < 0 && i1 < 0) continue;  // rows past the patch edge or owned by another patch
        const float4* cf = scf + (size_t)((j / 2) * BU + w) * S2;  // row pair (j, j+1)
        const float2* zw = smf + ((size_t)j * CU + w) * 32 + lane;
        float2 spp = make_float2(0.f, 0.f), cpp = make_float2(0.f, 0.f);
        float b0 = 0.f, b1 = 0.f;
#pragma unroll
        for (int dv = 0; dv < SW; ++dv)
#pragma unroll
          for (int du = 0; du < SW; ++du) {
            const float4 q = cf[dv * SW + du];
            const float2 z0 = zw[(dv * CU + du) * 32], z1 = zw[((dv + 1) * CU + du) * 32];
            df_acc2(spp, cpp, b0, b1, make_float2(q.x, q.y), make_float2(q.z, q.w), make_float2(z0.x, z1.x),
                    make_float2(z0.y, z1.y));
          }
        if (i0 >= 0) emit(i0, spp.x, cpp.x, b0);
        if (i1 >= 0) emit(i1, spp.y, cpp.y, b1);
      }
    }
    const bool one[1] = {true};
    double a2[1] = {(double)acc};
    block_reduce<1>(a2, part, t, tiles, one);
    __syncthreads();
    a2[0] = tiny && mine ? HUGE_VAL : (double)accb;  // fails the caller's error check
    block_reduce<1>(a2, part_bound, t, tiles, one);
    __syncthreads();  // the window and the reduction buffer may be refilled
  }
}

__global__ void k_build_csm(int N, int W, int cs32, int cs64, const int16_t* __restrict__ slot,
                            const double* __restrict__ S, const double* __restrict__ M, float2* __restrict__ c32,
                            double2* __restrict__ c64, float4* __restrict__ cdf) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * W) return;
  int sl = slot[t];
  if (sl < 0) return;
  int i = (int)(t / W);
  c32[(size_t)i * cs32 + sl] = make_float2((float)S[t], (float)M[t]);
  c64[(size_t)i * cs64 + sl] = make_double2(S[t], M[t]);
  float sh = (float)S[t], mh = (float)M[t];
  cdf[(size_t)i * cs64 + sl] = make_float4(sh, (float)(S[t] - (double)sh), mh, (float)(M[t] - (double)mh));
}

}  // namespace

// ====================================================================== host
// levels whose patches have fewer local DOFs per side keep the row kernels
// (moving the 10- and 18-wide levels of the sphere to the row kernels was slower:
// 174.5 and 184.0 against 172.5 ms per bench step)
#ifndef WM_STEN_MIN_NL
#define WM_STEN_MIN_NL 8
#endif

int wm_sten_build(const wm_geom_desc& g, int np, wm_level& L, cudaStream_t s) {
  L.sten = false;
  if (g.degree < 2 || g.degree > 3 || L.nlu < WM_STEN_MIN_NL || L.nlv < WM_STEN_MIN_NL) return WM_OK;
  std::vector<int32_t> ext, own;
  std::vector<int16_t> slot;
  if (wm_host_stencil(g, np, L, ext, own, slot) != WM_OK) return WM_OK;  // row kernels only
  const int p = g.degree, S2 = (2 * p + 1) * (2 * p + 1);
  const int cs32 = (S2 + 1) / 2 * 2, cs64 = S2;  // coefficient row strides (16-byte multiples)
  L.ELU = L.nlu + 2 * p;
  L.ELV = L.nlv + 2 * p;
  L.nbu = (L.nlu + BU - 1) / BU;
  const int bv = p == 2 ? BvOf<2>::value : BvOf<3>::value;
  L.nbv = (L.nlv + bv - 1) / bv;
  WM_TRY(L.d_ext.upload(ext, s));
  WM_TRY(L.d_own.upload(own, s));
  DevBuf<int16_t> d_slot;
  WM_TRY(d_slot.upload(slot, s));
  WM_TRY(L.d_csm32.alloc((size_t)L.N * cs32));
  WM_TRY(L.d_csm64.alloc((size_t)L.N * cs64));
  WM_TRY(L.d_csmdf.alloc((size_t)L.N * cs64));
  WM_CUDA(cudaMemsetAsync(L.d_csm32.p, 0, sizeof(float2) * (size_t)L.N * cs32, s));
  WM_CUDA(cudaMemsetAsync(L.d_csm64.p, 0, sizeof(double2) * (size_t)L.N * cs64, s));
  WM_CUDA(cudaMemsetAsync(L.d_csmdf.p, 0, sizeof(float4) * (size_t)L.N * cs64, s));
  int64_t n = (int64_t)L.N * L.W;
  WM_LAUNCH(WM_PC_ASSEMBLY, s, k_build_csm<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
                                   L.N, L.W, cs32, cs64, d_slot.p, L.d_S64.p, L.d_M64.p, L.d_csm32.p, L.d_csm64.p,
                                   L.d_csmdf.p));
  WM_CUDA(cudaGetLastError());
  WM_CUDA(cudaStreamSynchronize(s));
  d_slot.release();
  L.sten = true;
  return WM_OK;
}

int wm_sten_chunks(const wm_level& L, int np) { return L.sten ? np * L.nbu * L.nbv : 0; }

#define WM_DISPATCH_P(P_, ...)                     \
  switch (P_) {                                    \
    case 2: {                                      \
      constexpr int PP = 2;                        \
      __VA_ARGS__;                                 \
    } break;                                       \
    case 3: {                                      \
      constexpr int PP = 3;                        \
      __VA_ARGS__;                                 \
    } break;                                       \
    default: return WM_ERR_UNSUPPORTED;            \
  }

// SMs of the current device (grid sizing of the one-shift kernel)
static int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  return n > 0 ? n : 152;
}

template <typename T, int P, int MODE>
static int launch_uni(const wm_level& L, int np, int tiles, const UniTiles& ut, int kstep, const double* sigma,
                      const typename V2<T>::type* ctab, const int* sid, const T* r, const T* z, const T* prev,
                      T* out, const int* tile_active, double* part, int cat, cudaStream_t s,
                      const T* qd = nullptr, double* part2 = nullptr, T* out1 = nullptr) {
  constexpr size_t sm = UniLayout<T, P, MODE>::total;
  static bool configured = false;
  if (!configured) {
    WM_CUDA(cudaFuncSetAttribute(k_sten_uni<T, P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    configured = true;
  }
  if (ut.n_groups <= 0) return WM_OK;
  static const int sms = device_sms();
  const int bx = np * L.nbu * L.nbv;
  // blocks that share a group: enough blocks for ut.waves waves
  const int64_t want = (int64_t)ut.waves * sms * UniMinBlocks<T, P, MODE>::value;
  int split = 1;
  while (split < kUniGroup && (int64_t)bx * ut.n_groups * split < want) split *= 2;
  const T* dS = std::is_same<T, double>::value ? (const T*)L.d_dS64.p : (const T*)L.d_dS32.p;
  const T* dM = std::is_same<T, double>::value ? (const T*)L.d_dM64.p : (const T*)L.d_dM32.p;
  const int gmax = 65535 / split;  // grid.y limit
  for (int g0 = 0; g0 < ut.n_groups; g0 += gmax) {
    const int ng = std::min(gmax, ut.n_groups - g0);
    dim3 grid(bx, ng * split);
    WM_LAUNCH(cat, s, k_sten_uni<T, P, MODE><<<grid, dim3(32, BU), sm, s>>>(
                          geo_of(L), csm_of<T>(L), dS, dM, sigma, ctab, sid, kstep, z, r, prev, out, tiles,
                          tile_active, ut.groups + g0, split, part, qd, part2, out1));
    WM_CUDA(cudaGetLastError());
  }
  return WM_OK;
}

template <typename T>
int wm_sten_cheb_step(const wm_level& L, int np, int p, int tiles, int kstep, const double* sigma,
                      const typename StenC2<T>::type* ctab, const int* sid, const T* r, const T* z, const T* prev,
                      T* out, const int* tile_active, const UniTiles& ut, int cat, cudaStream_t s,
                      const T* q, double* part_rz, double* part_zq, bool generic_only) {
  if (generic_only) {
    // the one-shift tiles were done elsewhere: generic kernel for the others only
  } else if (ut.n > 0 && part_rz) {
    WM_DISPATCH_P(p, { WM_TRY((launch_uni<T, PP, UNI_CHEBDOT>(L, np, tiles, ut, kstep, sigma, ctab, sid, r, z, prev,
                                                              out, tile_active, part_rz, cat, s, q, part_zq))); });
  } else if (ut.n > 0) {
    WM_DISPATCH_P(p, { WM_TRY((launch_uni<T, PP, UNI_CHEB>(L, np, tiles, ut, kstep, sigma, ctab, sid, r, z, prev,
                                                           out, tile_active, nullptr, cat, s))); });
  }
  if (ut.n >= tiles) return WM_OK;
  ChebEpi<T, 2> e2;
  ChebEpi<T, 1> e1;
  auto fill = [&](auto& e) {
    e.N = L.N;
    e.kstep = kstep;
    e.dS = std::is_same<T, double>::value ? (const T*)L.d_dS64.p : (const T*)L.d_dS32.p;
    e.dM = std::is_same<T, double>::value ? (const T*)L.d_dM64.p : (const T*)L.d_dM32.p;
    e.out = out;
    e.sigma = sigma;
    e.ctab = ctab;
    e.sid = sid;
    e.in[0] = r;
    e.in[1] = prev;
  };
  fill(e2);
  fill(e1);
  const int* skip = ut.n > 0 ? ut.flag : nullptr;
  WM_DISPATCH_P(p, {
    if constexpr (Tpb<T, PP>::value == 2)
      return launch<T, PP>(L, np, tiles, z, tile_active, e2, cat, s, skip);
    else
      return launch<T, PP>(L, np, tiles, z, tile_active, e1, cat, s, skip);
  });
  return WM_OK;
}

template <typename T>
int wm_sten_cheb_first2(const wm_level& L, int np, int p, int tiles, const double* sigma,
                        const typename StenC2<T>::type* ctab, const int* sid, const T* r, T* z1, T* z2,
                        const int* tile_active, const UniTiles& ut, int cat, cudaStream_t s) {
  WM_DISPATCH_P(p, { WM_TRY((launch_uni<T, PP, UNI_CHEB1>(L, np, tiles, ut, 1, sigma, ctab, sid, nullptr, r, nullptr,
                                                          z2, tile_active, nullptr, cat, s, nullptr, nullptr,
                                                          z1))); });
  return WM_OK;
}

template <typename T>
int wm_sten_residual(const wm_level& L, int np, int p, int tiles, const double* sigma, const T* r, const T* z,
                     T* res, const int* tile_active, const UniTiles& ut, int cat, cudaStream_t s) {
  if (ut.n > 0) {
    WM_DISPATCH_P(p, { WM_TRY((launch_uni<T, PP, UNI_RESID>(L, np, tiles, ut, 0, sigma, nullptr, nullptr, r, z,
                                                            nullptr, res, tile_active, nullptr, cat, s))); });
    if (ut.n >= tiles) return WM_OK;
  }
  ResidEpi<T, 2> e2;
  ResidEpi<T, 1> e1;
  e2.N = e1.N = L.N;
  e2.r = e1.r = r;
  e2.res = e1.res = res;
  e2.sigma = e1.sigma = sigma;
  e2.in[0] = e1.in[0] = r;
  const int* skip = ut.n > 0 ? ut.flag : nullptr;
  WM_DISPATCH_P(p, {
    if constexpr (Tpb<T, PP>::value == 2)
      return launch<T, PP>(L, np, tiles, z, tile_active, e2, cat, s, skip);
    else
      return launch<T, PP>(L, np, tiles, z, tile_active, e1, cat, s, skip);
  });
  return WM_OK;
}

template <typename T>
int wm_sten_apply_pq(const wm_level& L, int np, int p, int tiles, const double* sigma, const T* pv, T* q,
                     const int* tile_active, const UniTiles& ut, double* part, cudaStream_t s) {
  if (ut.n > 0) {
    WM_DISPATCH_P(p, { WM_TRY((launch_uni<T, PP, UNI_APPLY>(L, np, tiles, ut, 0, sigma, nullptr, nullptr, nullptr,
                                                            pv, nullptr, q, tile_active, part, WM_PC_APPLY64,
                                                            s))); });
    if (ut.n >= tiles) return WM_OK;
  }
  ApplyEpi<T, 2> e2;
  ApplyEpi<T, 1> e1;
  e2.N = e1.N = L.N;
  e2.q = e1.q = q;
  e2.sigma = e1.sigma = sigma;
  e2.part = e1.part = part;
  const int* skip = ut.n > 0 ? ut.flag : nullptr;
  WM_DISPATCH_P(p, {
    if constexpr (Tpb<T, PP>::value == 2)
      return launch<T, PP>(L, np, tiles, pv, tile_active, e2, WM_PC_APPLY64, s, skip);
    else
      return launch<T, PP>(L, np, tiles, pv, tile_active, e1, WM_PC_APPLY64, s, skip);
  });
  return WM_OK;
}

template <typename Tr>
int wm_sten_true_residual(const wm_level& L, int np, int p, int tiles, const double* sigma, const double* x,
                          const double* rhs, const int* src_of, const int* rep, const int* tile_rep, Tr* r,
                          double* part, cudaStream_t s) {
  TrueResEpi<Tr, 1> e;
  e.N = L.N;
  e.rhs = rhs;
  e.src_of = src_of;
  e.rep = rep;
  e.r = r;
  e.sigma = sigma;
  e.part = part;
  WM_DISPATCH_P(p, { return launch<double, PP>(L, np, tiles, x, tile_rep, e, WM_PC_TRUERES, s); });
  return WM_OK;
}

template <int P>
static int launch_df(const wm_level& L, int np, int tiles, const UniTiles& ut, const double* sigma, const double* x,
                     const double* rhs, const int* src_of, const int* rep, const int* tile_rep, float* r, double* part,
                     double* part_bound, cudaStream_t s) {
  constexpr size_t sm = DfLayout<P>::total;
  constexpr size_t smu = DfUniLayout<P>::total;
  static bool configured = false;
  if (!configured) {
    WM_CUDA(cudaFuncSetAttribute(k_sten_trueres_df<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    WM_CUDA(cudaFuncSetAttribute(k_sten_trueres_df_uni<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smu));
    configured = true;
  }
  const int bx = np * L.nbu * L.nbv;
  if (ut.n_groups > 0) {
    static const int sms = device_sms();
    const int64_t want = (int64_t)ut.waves * sms * 3;
    int split = 1;
    while (split < kUniGroup && (int64_t)bx * ut.n_groups * split < want) split *= 2;
    const int gmax = 65535 / split;
    for (int g0 = 0; g0 < ut.n_groups; g0 += gmax) {
      const int ng = std::min(gmax, ut.n_groups - g0);
      WM_LAUNCH(WM_PC_TRUERES, s, k_sten_trueres_df_uni<P><<<dim3(bx, ng * split), dim3(32, BU), smu, s>>>(
                                      geo_of(L), L.d_csmdf.p, x, tiles, tile_rep, ut.groups + g0, split, sigma, rhs,
                                      src_of, rep, r, part, part_bound));
      WM_CUDA(cudaGetLastError());
    }
  }
  if (ut.n < tiles) {
    dim3 grid(bx, tiles);
    WM_LAUNCH(WM_PC_TRUERES, s, k_sten_trueres_df<P><<<grid, dim3(32, BU), sm, s>>>(
                                    geo_of(L), L.d_csmdf.p, x, tiles, tile_rep, sigma, rhs, src_of, rep, r, part,
                                    part_bound, ut.n > 0 ? ut.flag : nullptr));
    WM_CUDA(cudaGetLastError());
  }
  return WM_OK;
}

int wm_sten_true_residual_df(const wm_level& L, int np, int p, int tiles, const UniTiles& ut, const double* sigma,
                             const double* x, const double* rhs, const int* src_of, const int* rep,
                             const int* tile_rep, float* r, double* part, double* part_bound, cudaStream_t s) {
  WM_DISPATCH_P(p, {
    return launch_df<PP>(L, np, tiles, ut, sigma, x, rhs, src_of, rep, tile_rep, r, part, part_bound, s);
  });
  return WM_OK;
}

template int wm_sten_cheb_step<float>(const wm_level&, int, int, int, int, const double*, const float2*,
                                      const int*, const float*, const float*, const float*, float*, const int*,
                                      const UniTiles&, int, cudaStream_t, const float*, double*, double*, bool);
template int wm_sten_cheb_step<double>(const wm_level&, int, int, int, int, const double*, const double2*,
                                       const int*, const double*, const double*, const double*, double*, const int*,
                                       const UniTiles&, int, cudaStream_t, const double*, double*, double*, bool);
template int wm_sten_cheb_first2<float>(const wm_level&, int, int, int, const double*, const float2*, const int*,
                                        const float*, float*, float*, const int*, const UniTiles&, int, cudaStream_t);
template int wm_sten_cheb_first2<double>(const wm_level&, int, int, int, const double*, const double2*, const int*,
                                         const double*, double*, double*, const int*, const UniTiles&, int,
                                         cudaStream_t);
template int wm_sten_residual<float>(const wm_level&, int, int, int, const double*, const float*, const float*, float*,
                                     const int*, const UniTiles&, int, cudaStream_t);
template int wm_sten_residual<double>(const wm_level&, int, int, int, const double*, const double*, const double*,
                                      double*, const int*, const UniTiles&, int, cudaStream_t);
template int wm_sten_apply_pq<float>(const wm_level&, int, int, int, const double*, const float*, float*, const int*,
                                     const UniTiles&, double*, cudaStream_t);
template int wm_sten_apply_pq<double>(const wm_level&, int, int, int, const double*, const double*, double*,
                                      const int*, const UniTiles&, double*, cudaStream_t);
template int wm_sten_true_residual<float>(const wm_level&, int, int, int, const double*, const double*, const double*,
                                          const int*, const int*, const int*, float*, double*, cudaStream_t);
template int wm_sten_true_residual<double>(const wm_level&, int, int, int, const double*, const double*,
                                           const double*, const int*, const int*, const int*, double*, double*,
                                           cudaStream_t);
