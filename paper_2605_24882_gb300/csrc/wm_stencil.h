// Shared-memory stencil kernels (wm_stencil.cu) for levels with a stencil form.
#pragma once

#include "wm_internal.h"

#ifndef WM_MAX_CHEB
#define WM_MAX_CHEB 8
#endif

// Tiles whose 32 systems share one shift (sample-major packing: the 32 samples
// of one sinc node), for the combined-coefficient kernel: a per-tile flag (the
// generic kernel skips those tiles) and groups of at most kUniGroup
// consecutive such tiles with the same shift index, each (first tile, count).
// A block of the one-shift kernel serves one group (or part of one).
constexpr int kUniGroup = 8;
struct UniTiles {
  const int* flag = nullptr;     // [tiles] 1 where the 32 shifts of the tile are equal
  int n = 0;                     // number of such tiles
  const int2* groups = nullptr;  // [n_groups] (first tile, count), count in 1..kUniGroup
  int n_groups = 0;
  int waves = 4;                 // grid target: runs are split until the grid has this many waves
};

// Builds the stencil form of a level (extended grids, owner map, coefficient
// slots) after its rows are assembled; leaves L.sten = false when the level
// keeps the row kernels (degree outside 2..3, patches narrower than 8).
int wm_sten_build(const wm_geom_desc& g, int np, wm_level& L, cudaStream_t s);
// number of spatial blocks of a stencil launch on the level (partial-sum chunks)
int wm_sten_chunks(const wm_level& L, int np);

template <typename T>
struct StenC2;
template <>
struct StenC2<float> {
  using type = float2;
};
template <>
struct StenC2<double> {
  using type = double2;
};
// Three-term Chebyshev step out = z + c1 (z - prev) + c2 D^{-1} (r - A z)
// (c1 = 0 at kstep 0, prev = nullptr for z_prev = 0; out may alias prev).
// ctab: (c1, c2) per [shift][step] of the level (WM_MAX_CHEB steps per shift).
// The one-shift tiles of `ut` go to the combined-coefficient kernel, the
// others to the generic one.
template <typename T>
int wm_sten_cheb_step(const wm_level& L, int np, int p, int tiles, int kstep, const double* sigma,
                      const typename StenC2<T>::type* ctab, const int* sid, const T* r, const T* z, const T* prev,
                      T* out, const int* tile_active, const UniTiles& ut, int cat, cudaStream_t s,
                      const T* q = nullptr, double* part_rz = nullptr, double* part_zq = nullptr,
                      bool generic_only = false);
// With part_rz set, the one-shift tiles of the step also leave per-block partial
// sums (r, out) in part_rz and, with q set, (out, q) in part_zq ([tile][chunk][32],
// chunk = spatial block); the other tiles get none (the caller forms them).
// generic_only: the one-shift tiles are left alone (done by another launch).
// The first two pre-smoothing steps from z = 0 for the one-shift tiles only:
// z1 = c2_0 D^{-1} r and z2 = z1 + c1_1 z1 + c2_1 D^{-1} (r - A z1) in one pass
// over the window of r (the other tiles take the row-form first step and
// wm_sten_cheb_step with generic_only).
template <typename T>
int wm_sten_cheb_first2(const wm_level& L, int np, int p, int tiles, const double* sigma,
                        const typename StenC2<T>::type* ctab, const int* sid, const T* r, T* z1, T* z2,
                        const int* tile_active, const UniTiles& ut, int cat, cudaStream_t s);
// residual res = r - A z and outer apply q = A p with per-block partial sums
// (p, q) in `part` ([tile][chunk][32], chunk = spatial block); the one-shift
// tiles of `ut` take the combined-coefficient kernel
template <typename T>
int wm_sten_residual(const wm_level& L, int np, int p, int tiles, const double* sigma, const T* r, const T* z,
                     T* res, const int* tile_active, const UniTiles& ut, int cat, cudaStream_t s);
template <typename T>
int wm_sten_apply_pq(const wm_level& L, int np, int p, int tiles, const double* sigma, const T* pv, T* q,
                     const int* tile_active, const UniTiles& ut, double* part, cudaStream_t s);
template <typename Tr>
int wm_sten_true_residual(const wm_level& L, int np, int p, int tiles, const double* sigma, const double* x,
                          const double* rhs, const int* src_of, const int* rep, const int* tile_rep, Tr* r,
                          double* part, cudaStream_t s);
// the same residual (float output) with the stencil sums in double-float
// arithmetic on the FP32 pipes; part_bound receives the per-block partial
// sums of ||B||^2 with B_i = sum_j |a_ij| |x_j| (the rounding error of entry i
// is below 2^-42 B_i), or +inf for a system with a value below 2^-102
// (one-shift tiles of `ut` by groups, the others one tile per block)
int wm_sten_true_residual_df(const wm_level& L, int np, int p, int tiles, const UniTiles& ut, const double* sigma,
                             const double* x, const double* rhs, const int* src_of, const int* rep,
                             const int* tile_rep, float* r, double* part, double* part_bound, cudaStream_t s);
