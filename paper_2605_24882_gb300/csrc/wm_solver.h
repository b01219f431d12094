// Batched solver state shared by the sampler entry points.
#pragma once

// largest Chebyshev degree of a smoothing sweep
#ifndef WM_MAX_CHEB
#define WM_MAX_CHEB 8
#endif

#include "wm_internal.h"

// float or double buffer (only the one of the solve's precision is allocated)
struct VBuf {
  DevBuf<double> d;
  DevBuf<float> f;
  int alloc(size_t n, bool dbl);
  void release() {
    d.release();
    f.release();
  }
};

struct LevelBufs {
  VBuf za, zb;  // smoother iterates (three-term recurrence: the new iterate overwrites z_prev)
  VBuf res;     // residual before restriction
  VBuf r;       // restricted residual (levels >= 1)
};

// One batched solve: `tiles` tiles of 32 systems; systems g < nsys are real.
struct Batch {
  int tiles = 0;
  int nsys = 0;
  int nshift = 0;     // distinct shifts (coarse inverses, smoother bounds)
  int precision = WM_MIXED;
  double rtol = 1e-8;
  int max_iter = 200;
  int degree = 2;     // Chebyshev degree of each smoothing sweep on the finest level
  int degree_coarse = 0;  // on the coarser levels (0: the same)
  int degree_of(int level) const { return level == 0 || degree_coarse == 0 ? degree : degree_coarse; }
  double cheb_ratio = 8.0;
  // float64 residual replacement once the recursive residual of a system has
  // fallen by this factor since its last replacement (and always before a
  // system is declared converged)
  double replace_drop = 1e-3;
  // float64 true residuals of the float-preconditioned solve evaluated in
  // double-float arithmetic (stencil levels), checked against the tolerance
  bool df_residual = false;
  int precond = WM_PRECOND_VCYCLE;  // or WM_PRECOND_BPX
  mutable int active_tiles = 0;  // host copy of the active tile count (for work accounting)
  int vec_rows = 128;     // rows per block of the CG vector kernels
  int vcycle_rows = 16;   // rows per block of the V-cycle row kernels
  bool tail_fused = true;  // float: the coarse end of the V-cycle in one kernel per tile
  int chunks_for(int N) const;
  int vcycle_chunks(int N) const;
  void schedule(const wm_schedule& s) {
    vec_rows = s.vec_rows;
    vcycle_rows = s.vcycle_rows;
    tail_fused = s.tail_fused != 0;
  }
};

struct BatchResult {
  int iterations = 0;
  int replacements = 0;
  int n_not_converged = 0;
  double max_rel_residual = 0.0;
  int flags = 0;  // bit 0: non-finite value, bit 1: CG breakdown
  int df_fallbacks = 0;  // double-float residuals rejected by the error check
};

struct WorkSpace {
  DevBuf<double> x;           // float64 solution [tiles][N0][32]
  VBuf r, p, q;               // recursion in the V-cycle precision
  std::vector<LevelBufs> lvl;
  DevBuf<double> sigma;       // per system shift
  DevBuf<int> sid;            // per system shift index
  DevBuf<int> src_of;         // per system right-hand-side sample (-1: padding)
  DevBuf<int> active, rep, restart, tile_active, tile_rep;
  DevBuf<int> tile_uni;       // 1 where the 32 shifts of a tile are equal
  int n_uni_tiles = 0;        // host count of such tiles in the current batch
  DevBuf<int2> uni_groups;    // runs of at most 8 consecutive such tiles of one shift: (first tile, count)
  int n_uni_groups = 0;
  int uni_waves = 4;          // grid target of the one-shift kernels (the hierarchy's schedule)
  DevBuf<double> rho, alpha, beta, bb, rr, rr_ref;
  DevBuf<double> part[3];
  DevBuf<int> flags, counters;
  DevBuf<double> lmax, ainv, shifts, statd;
  // Chebyshev step coefficients (c1, c2) per [level][shift][step], both precisions
  DevBuf<float2> cheb32;
  DevBuf<double2> cheb64;
  // sample-tiled float64 buffers: loads, integer iterate, field, pass rhs, staging
  DevBuf<double> samp[5];
  DevBuf<double> noise_scratch;
  DevBuf<double> pw_v, pw_w, pw_sigma;
  DevBuf<double> coef;        // sinc weights of the current pass
  DevBuf<double> ckpt, mx, dots;  // adjoint: forward solutions of a batch, M x, per-system dots
  std::vector<DevBuf<double>> chain;  // adjoint: integer-part iterates w_1..w_n (sample-tiled)
  DevBuf<double> rpass[2], xpass[2], vpass;  // adjoint: pass right-hand sides, kept pass solutions, pass result
  // Forward checkpoint for the backward (WM_CKPT_KEEP): the loads, the integer
  // iterates w_1..w_n and the pass right-hand sides (sample-tiled), and the
  // solution of every system of each fractional pass ([tiles][N][32], system
  // g = j n_s + s of the pass); valid for the descriptor `desc`.
  struct Ckpt {
    bool valid = false;
    wm_sample_desc desc{};
    DevBuf<double> b;
    std::vector<DevBuf<double>> w;
    DevBuf<double> r[2], x[2];
    void release() {
      valid = false;
      b.release();
      for (auto& v : w) v.release();
      w.clear();
      for (int k = 0; k < 2; ++k) {
        r[k].release();
        x[k].release();
      }
    }
  } ck;
  // shifts whose smoother bounds and coarse inverses are in lmax / ainv
  std::vector<double> prep_shifts;
  const double* prep_lmax = nullptr;
  const double* prep_ainv = nullptr;
  int* host_small = nullptr;  // pinned
  double host_d = 0.0;
  int reserve(const wm_hier* h, int tiles, int nshift, bool dbl);
  void release();
};

int wm_prepare_shifts(const wm_hier* h, WorkSpace& ws, const std::vector<double>& shifts, cudaStream_t s);
int wm_solve_batch(const wm_hier* h, WorkSpace& ws, const Batch& bt, const double* rhs_tiled, BatchResult* res,
                   cudaStream_t s);
// one V-cycle on the float64 tiled residual `r64` (staged through ws.r) with
// the result widened to float64 in `z64`
int wm_vcycle_apply(const wm_hier* h, WorkSpace& ws, const Batch& bt, const double* r64, double* z64,
                    cudaStream_t s);
int wm_sinc_accumulate(const wm_hier* h, int ns, int g0, int g1, const double* c_dev, const double* x,
                       double* v_tiled, cudaStream_t s);
int wm_copy(const double* a, double* b, size_t n, cudaStream_t s);
// out[g] = (a_g, b_g) for the 32*tiles systems of two tiled float64 vectors
int wm_system_dots(WorkSpace& ws, int tiles, int N, const double* a, const double* b, std::vector<double>& out,
                   cudaStream_t s);
int wm_convert_f32(const double* a, float* b, size_t n, cudaStream_t s);
int wm_widen_f32(const float* a, double* b, size_t n, cudaStream_t s);
