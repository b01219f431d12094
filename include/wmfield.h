/*
 * wmfield.h -- C ABI of the GB300 Whittle–Matérn surface field sampler.
 *
 * The library samples Gaussian random fields u on closed surfaces from the
 * fractional SPDE (kappa^2 - Delta_Gamma)^beta u = white noise (Eq. eq:PDE,
 * Sec. 1), discretised with C0-glued tensor B-splines on the patches of the
 * surface (Sec. 2.3, Eq. def::space2).  With S the stiffness and M the mass
 * matrix (Eqs. eq:FEM, eq:mass, eq:stiffness) it computes, per noise sample s,
 *   integer part (Sec. 3.4):  (S + kappa^2 M) w_1 = b_s,  (S + kappa^2 M) w_i = M w_{i-1},
 *   fractional part (Eq. eq:beta-approx, y = -2t):
 *       u_s = sum_l c_l x_{l,s},  (S + sigma_l M) x_{l,s} = M w_n   (b_s if n = 0),
 *       y_l = l k, sigma_l = e^{y_l} + kappa^2, c_l = (sin(pi beta')/pi) k e^{(1-beta') y_l},
 * and, with the improved split (Sec. 3.4), the sinc map twice.  All shifted
 * systems of all samples are solved together on the GPU by a batched
 * preconditioned conjugate gradient with a geometric multigrid V-cycle over the
 * dyadic spline hierarchy (Sec. 3.5).
 *
 * Conventions for every entry point:
 *  - Return value: WM_OK (0) or a negative WM_ERR_* code; no exception ever
 *    crosses the ABI.  wm_error_string() names a code; wm_last_error() returns
 *    a message for the calling thread's last failure.
 *  - Handles (wm_geom_t, wm_hier_t) are owned by the library and released with
 *    wm_destroy_*.  A handle may be used by one host thread at a time.
 *  - "device" pointers are caller-owned CUDA device memory of the current
 *    device; "host" pointers are caller-owned host memory.  Vectors of n
 *    samples over N degrees of freedom are row-major [n][N] float64.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is stream-ordered; entry points that return
 *    statistics or host results synchronise the stream before returning.
 *  - Levels are numbered from 0 = finest to wm_num_levels()-1 = coarsest.
 */
#ifndef WMFIELD_H
#define WMFIELD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define WM_OK 0
#define WM_ERR_INVALID_ARG (-1)   /* a size, pointer or parameter is out of range  */
#define WM_ERR_OOM (-2)           /* a device or host allocation failed            */
#define WM_ERR_CUDA (-3)          /* a CUDA call failed; see wm_last_error()       */
#define WM_ERR_NOT_CONVERGED (-4) /* some system missed rtol within max_iter       */
#define WM_ERR_NONFINITE (-5)     /* a NaN/Inf appeared in a residual norm         */
#define WM_ERR_UNSUPPORTED (-7)   /* valid request outside what is implemented     */

/* ---- enumerations --------------------------------------------------------- */
#define WM_SPHERE6 0      /* unit sphere as six gnomonic cube-face patches     */
#define WM_TORUS 1        /* one doubly periodic torus patch (R, r)            */
#define WM_NURBS_PERIODIC 2 /* one NURBS patch, periodic in u and v (torus topology)  */
#define WM_NURBS_CUBE 3     /* six NURBS patches in the cube-face arrangement          */

#define WM_FP64 0         /* every step in float64                              */
#define WM_MIXED 1        /* float64 outer CG, float32 multigrid preconditioner */

#define WM_SPLIT_STANDARD 0  /* beta = n + beta'                               */
#define WM_SPLIT_IMPROVED 1  /* Sec. 3.4 itemize: beta'' applied twice          */

#define WM_NOISE_DRAW 0   /* draw b_s from Philox with desc.seed               */
#define WM_NOISE_GIVEN 1  /* take b_s from the caller's b buffer               */

#define WM_PRECOND_VCYCLE 0  /* multiplicative: one V-cycle per CG iteration       */
#define WM_PRECOND_BPX 1     /* additive: BPX multilevel diagonal scaling           */

#define WM_CKPT_RECOMPUTE 0  /* the backward re-solves the forward systems it needs */
#define WM_CKPT_KEEP 1       /* forward solutions are kept for the backward when
                                they fit in half of the free device memory         */

/* ---- geometry ------------------------------------------------------------- */
typedef struct {
  int kind;      /* WM_SPHERE6 or WM_TORUS                                        */
  int degree;    /* spline degree p, 1 <= p <= 4                                   */
  int elems_u;   /* elements per patch side at the finest level (power of two)     */
  int elems_v;   /* sphere: must equal elems_u; torus: elements along the tube     */
  double R, r;   /* torus major / minor radius (ignored for the sphere)            */
} wm_geom_desc;

typedef struct wm_geom* wm_geom_t;
typedef struct wm_hier* wm_hier_t;

/*
 * One NURBS patch of a geometry map (Sec. 2.2): F(u, v) on [0, 1]^2 is
 * sum_ij N_i(u) M_j(v) w_ij P_ij / sum_ij N_i(u) M_j(v) w_ij with the B-splines
 * N_i, M_j of Definition 2.1 on the knot vectors.  Host memory, read during
 * wm_setup_geometry_nurbs and copied; the caller keeps ownership.
 */
typedef struct {
  int degree_u, degree_v;  /* 1 .. 8                                                */
  int n_u, n_v;            /* control points per direction (>= degree + 1)          */
  const double* knots_u;   /* n_u + degree_u + 1 knots, nondecreasing, the first    */
  const double* knots_v;   /*   degree+1 equal to 0 and the last degree+1 equal to 1 */
  const double* cpw;       /* [n_v][n_u][4]: x, y, z and weight (> 0)               */
} wm_nurbs_patch;

/*
 * Validates a surface description and builds its patch table and the C0
 * gluing of the spline space S^0_{j,p} (Eq. def::space2) by combinatorial
 * matching of patch edges.  Host only.  Global DOF numbering: patches in
 * order, local DOFs row by row (i_v outer, i_u inner); a shared DOF keeps the
 * index of its first occurrence.
 * Errors: WM_ERR_INVALID_ARG for a bad kind/degree/size or NULL out.
 */
int wm_setup_geometry(const wm_geom_desc* desc, wm_geom_t* out);

/*
 * A surface given by NURBS patches (Sec. 2.2, multi-patch NURBS
 * parametrisations).  desc->kind is WM_NURBS_PERIODIC (n_patches = 1; the
 * solution space is the torus's periodic spline space, so F must be periodic
 * in u and v) or WM_NURBS_CUBE (n_patches = 6, glued like WM_SPHERE6: patch m
 * covers the cube face whose coordinate a is 2u-1, b is 2v-1 and n is s, with
 * (a, b, n, s) = (1,2,0,+), (2,1,0,-), (2,0,1,+), (0,2,1,-), (0,1,2,+), (1,0,2,-)
 * for m = 0..5, and neighbouring patches must agree along their shared edges,
 * parameter for parameter).  degree, elems_u, elems_v as for wm_setup_geometry;
 * R and r are ignored.  The closure (periodic) or the edge agreement (cube) is
 * checked at sample points to 1e-10 of the surface's size.  The geometry map
 * is evaluated on the host at every Gauss point when a hierarchy is assembled;
 * element boundaries should fall on the knots of the patches for full
 * quadrature accuracy.
 * Errors: WM_ERR_INVALID_ARG (kind, sizes, knots, weights, closure), WM_ERR_OOM.
 */
int wm_setup_geometry_nurbs(const wm_geom_desc* desc, const wm_nurbs_patch* patches, int n_patches,
                            wm_geom_t* out);

/*
 * Host-only: the metric terms (a, G11, G12, G22) with G = a K^{-1} (Sec. 3.2)
 * of a NURBS geometry at the Gauss points of a level, float64 [n_quad][4] in
 * host memory (Gauss point order as wm_metric), exactly as the hierarchy
 * uploads them.  `cap` is the capacity of `out` in doubles.
 * Errors: WM_ERR_UNSUPPORTED for the analytic kinds (their metric is computed
 * on the GPU, see wm_metric), WM_ERR_INVALID_ARG.
 */
int wm_geom_metric(wm_geom_t g, int level, double* out, int64_t cap);

/*
 * Host-only queries of the discrete space of a geometry; no CUDA device is
 * used.  They return what wm_assemble_hierarchy builds on the host for its
 * level `level` (0 = the description's elements; each level halves the
 * elements per side) before uploading it.  A level is allowed when a hierarchy
 * of level+1 levels is (the prolongation needs level+2).
 *
 * wm_geom_level_sizes: glued DOFs N of S^0_{j,p} (Eq. def::space2), local
 *   DOFs per patch side (elems + p open, elems periodic), elements E of all
 *   patches, and the stored entries of the prolongation from level+1 to
 *   level (0 at the coarsest allowed level).  NULL outputs are skipped.
 * wm_geom_dof_map: copies the local-to-global map [np][n_loc_v][n_loc_u]
 *   (int32, same numbering rule as wm_setup_geometry) to host `l2g`, and, if
 *   `conn` is not NULL, the element connectivity [E][(p+1)^2] (element
 *   (m n_v + e_v) n_u + e_u, local function k = k_v (p+1) + k_u; periodic
 *   elements carry the functions e-p..e mod n).  Capacities are in entries.
 * wm_geom_prolongation: the prolongation from level+1 to level by dyadic
 *   knot insertion (Sec. 2.3: the nested spaces Xi_{j,p} of the refinement)
 *   as host CSR: row_ptr [N_fine + 1], col [nnz] (coarse DOF, ascending in a
 *   row), val [nnz] float64.  nnz_cap is the capacity of col and val.
 * Errors: WM_ERR_INVALID_ARG for a NULL handle or buffer, a level out of range
 * or a capacity too small; nothing is written then.
 */
int wm_geom_level_sizes(wm_geom_t g, int level, int* n_dofs, int* n_loc_u, int* n_loc_v, int* n_elems,
                        int64_t* prolong_nnz);
int wm_geom_dof_map(wm_geom_t g, int level, int32_t* l2g, int64_t l2g_cap, int32_t* conn, int64_t conn_cap);
int wm_geom_prolongation(wm_geom_t g, int level, int32_t* row_ptr, int32_t* col, double* val, int64_t nnz_cap);

/*
 * Host-only: the stencil form of a level's operator rows, as the shared-memory
 * stencil kernels read it (no device used).
 *   ext  [np][n_loc_v + 2p][n_loc_u + 2p]: global DOF of every cell of the patch
 *        grids extended by a halo of p cells (across a cube edge the adjacent
 *        patch's DOFs, periodic grids wrapped, beyond a cube corner -1);
 *   own  [np][n_loc_v][n_loc_u]: the DOF whose row this patch position computes
 *        (every DOF at its first patch), else -1;
 *   col  [N][W]: the stored columns of each row, padded with the row index;
 *   slot [N][W]: the window position (dv + p)(2p+1) + (du + p) of each stored
 *        entry in the frame of the row's owner, -1 for padding.
 * With all four arrays NULL only *W (the row width) is written.  Capacities are
 * in entries (row_cap for col and slot).
 * Errors: WM_ERR_UNSUPPORTED when the level has no stencil form (row kernels
 * serve it), WM_ERR_INVALID_ARG for a bad level or a capacity too small.
 */
int wm_geom_stencil(wm_geom_t g, int level, int32_t* ext, int64_t ext_cap, int32_t* own, int64_t own_cap,
                    int32_t* col, int16_t* slot, int64_t row_cap, int* W);

/*
 * Host-only bounds lo <= lambda_min(M) and lambda_max(M) <= hi of the
 * assembled mass matrix of a level (the spectrum bounds m, M of Sec. 3.3 that
 * the sqrt(M) rule needs).  On each patch the quadrature mass form lies
 * between the smallest and the largest area element times the flat
 * tensor-product form M_u (x) M_v; lo and hi combine the closed-form extremes of
 * the area element (cube sphere: 4 (1+a^2+b^2)^{-3/2} on [-1,1]^2; torus:
 * 4 pi^2 r (R +- r)) with the extreme eigenvalues of the 1D mass matrices and,
 * for hi, the three patches that share a cube corner.  Level as for
 * wm_geom_level_sizes.  Errors: WM_ERR_INVALID_ARG.
 */
int wm_geom_mass_bounds(wm_geom_t g, int level, double* lo, double* hi);

/*
 * Host-only: shifts w2[k] = w_k^2 and weights c[k] (host arrays [n_nodes]) of
 * the n_nodes-point rule sqrt(A) y ~= A sum_k c_k (A + w_k^2 I)^{-1} y for a
 * symmetric positive definite A with spectrum in [lo, hi] (Sec. 3.3,
 * Eq. eq:sqrt, after Hale, Higham and Trefethen): w_k = sqrt(lo) sn(t_k|q) /
 * cn(t_k|q), c_k = 2 K sqrt(lo) dn(t_k|q) / (pi n_nodes cn(t_k|q)^2),
 * t_k = (k + 1/2) K / n_nodes, q = 1 - lo/hi, K = K(q) the complete elliptic
 * integral of the first kind.  Errors: WM_ERR_INVALID_ARG unless 0 < lo < hi,
 * n_nodes >= 1 and both arrays are given.
 */
int wm_hht_rule(double lo, double hi, int n_nodes, double* w2, double* c);

/*
 * Builds the dyadic hierarchy of n_levels levels (finest = the description's
 * elements, each coarser level halves the elements per side; Sec. 2.3,
 * Xi_{j,p}) on the current CUDA device: the metric terms a_m and a_m K_m^{-1}
 * at the (p+1)^2 Gauss points of every element in float64 (Sec. 3.2), the
 * assembled mass and stiffness rows of every level (float64 and float32
 * copies), and the knot-insertion prolongations between levels.
 * Errors: WM_ERR_INVALID_ARG (n_levels < 1 or too many for the element
 * counts), WM_ERR_OOM, WM_ERR_CUDA.  The geometry handle stays owned by the
 * caller and may be destroyed afterwards.
 */
int wm_assemble_hierarchy(wm_geom_t geom, int n_levels, void* stream, wm_hier_t* out);

/*
 * Kernel schedule of a hierarchy's batched solves (a tuning knob: results
 * change at most in rounding order).  Defaults in parentheses; wm_set_schedule
 * with NULL restores them.  Errors: WM_ERR_INVALID_ARG for values out of range.
 */
typedef struct {
  int uni_run;      /* consecutive one-shift tiles one block of the stencil kernels
                       serves (window ids and combined rows built once), 1..8 (8)   */
  int uni_waves;    /* grid target of those kernels, in waves of resident blocks:
                       runs are split over more blocks until the grid reaches it,
                       1..64 (4)                                                    */
  int vec_rows;     /* rows per block of the outer CG's vector kernels, 32..4096
                       (128)                                                        */
  int vcycle_rows;  /* rows per block of the V-cycle's row kernels (levels without
                       a stencil form), 8..1024 (16)                                */
  int tail_fused;   /* float solves: the V-cycle from the first level without a
                       stencil form down to the coarse solve and back in one
                       kernel per tile (vectors in shared memory), where those
                       levels fit a block's shared memory; 0: one launch per
                       level and step.  0 or 1 (1)                                  */
} wm_schedule;
int wm_set_schedule(wm_hier_t h, const wm_schedule* sched);
int wm_get_schedule(wm_hier_t h, wm_schedule* out);

int wm_num_levels(wm_hier_t h);               /* number of levels, or < 0 on error */
int wm_num_dofs(wm_hier_t h, int level);      /* glued DOFs N of a level, or < 0    */
int wm_num_quad_points(wm_hier_t h, int level); /* Gauss points of a level, or < 0   */

/*
 * Copies the local-to-global DOF map of a level to host memory:
 * out[m][i_v][i_u] (int32), n_patches * n_loc_v * n_loc_u entries, where
 * n_loc = elems + p for open patches and elems for the periodic torus.
 * `cap` is the capacity of `out` in entries.  Returns the number of entries
 * written, or WM_ERR_INVALID_ARG when cap is too small.
 */
int wm_dof_map(wm_hier_t h, int level, int32_t* out, int64_t cap);

/*
 * Copies the float64 metric terms of a level at its Gauss points to device
 * memory `out` [n_quad][4] = (a, G11, G12, G22) with G = a K^{-1} (Sec. 3.2).
 * Gauss point index q = ((m n_v + e_v) n_u + e_u) nq^2 + g_v nq + g_u.
 */
int wm_metric(wm_hier_t h, int level, double* out, void* stream);

/* ---- operators ------------------------------------------------------------ */
/*
 * y_j = (S + sigma_j M) x_j for n_vec vectors on a level (Eqs. eq:FEM,
 * eq:var_form with t = sigma_j).  sigma: host array [n_vec]; x, y: device
 * [n_vec][N].  precision WM_FP64 applies the float64 rows, WM_MIXED the
 * float32 rows (inputs rounded to float32, result widened).  x and y must not
 * overlap.
 */
int wm_apply_shifted(wm_hier_t h, int level, int n_vec, const double* sigma,
                     const double* x, double* y, int precision, void* stream);

/* y_j = M x_j on a level in float64 (the S-term off). */
int wm_apply_mass(wm_hier_t h, int level, const double* x, double* y, int n_vec, void* stream);

/*
 * Prolongation by dyadic knot insertion from level `level`+1 (coarse) to
 * `level` (fine): the fine coefficients of the same spline (Sec. 3.5, nested
 * spaces).  xc: device [n_vec][N_coarse], xf: device [n_vec][N_fine].
 */
int wm_prolongate(wm_hier_t h, int level, const double* xc, double* xf, int n_vec, void* stream);

/* Restriction = transpose of wm_prolongate: rc = P^T rf. */
int wm_restrict(wm_hier_t h, int level, const double* rf, double* rc, int n_vec, void* stream);

/*
 * One application of the batched V-cycle preconditioner on level 0 to n_vec
 * residuals with shifts sigma (host [n_vec]); z = B_sigma r.  r, z: device
 * [n_vec][N].  Smoother: Chebyshev of degree `smoother_degree` on
 * [lambda_max/cheb_ratio, 1.1 lambda_max] of D^{-1}(S + sigma M); precision
 * as in wm_apply_shifted.
 */
int wm_vcycle(wm_hier_t h, int n_vec, const double* sigma, const double* r, double* z,
              int precision, int smoother_degree, double cheb_ratio, void* stream);

/* ---- random numbers and white noise --------------------------------------- */
/*
 * Philox4x32-10 (Salmon et al., SC'11) on n counters: ctr device [n][4]
 * uint32, key = (key mod 2^32, key div 2^32), out device [n][4].
 */
int wm_philox4x32_10(const uint32_t* ctr, uint64_t key, uint32_t* out, int64_t n, void* stream);

/*
 * Standard normals of the white noise, n consecutive Gauss-point indices from
 * q0 of one sample: out device [n].  Normal q is half (q mod 2) of a
 * Box–Muller pair drawn from the counter (q/2 mod 2^32, sample, stream_id,
 * q/2 div 2^32): u = ((x_hi >> 5) 2^26 + (x_lo >> 6) + 1) 2^-53 in (0,1].
 * stream_id 0 = noise, 1 = loss targets.
 */
int wm_normals(uint64_t seed, int sample, int stream_id, int64_t q0, int64_t n,
               double* out, void* stream);

/*
 * White-noise loads of samples 0..n_samples-1 on level 0 (Sec. 3.3):
 * b_s,i = sum_q sqrt(w_q a_q) xi_{s,q} phi_i(x_q) with xi from wm_normals,
 * so Cov(b_s) is the quadrature mass matrix.  b: device [n_samples][N].
 */
int wm_noise_loads(wm_hier_t h, uint64_t seed, int n_samples, double* b, void* stream);

/*
 * wm_noise_loads without any device allocation, for callers that cannot
 * allocate device memory: a host framework whose caching allocator owns the
 * device memory, or code that may not call cudaMalloc because cudaMalloc can
 * synchronise the device.  The paper has no counterpart: this is a packaging
 * variant of wm_noise_loads with the same result (b: device [n_samples][N],
 * caller-owned; the hierarchy's device must be the current device).  Its
 * element-local scratch is a fixed file-scope device array of 2^22 doubles
 * (32 MiB) that every GPU which loads the library holds until process exit; a
 * call needs elements x (p+1)^2 x n_samples <= 2^22 and otherwise returns
 * WM_ERR_INVALID_ARG without launching anything (so does a b that is not
 * device memory, or a current device other than the hierarchy's).  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; later calls query only the current
 * device and the pointer attributes of b before their two kernel launches
 * (with wm_profile_enable on, CUDA events are recorded around them).
 * Every call writes all the scratch it reads, so nothing needs to
 * start at zero; all calls share the array, so calls whose work overlaps on
 * the GPU (different streams, or different host threads) race.
 * Stream-ordered, no synchronisation.
 */
int wm_noise_loads_noalloc(wm_hier_t h, uint64_t seed, int n_samples, double* b, void* stream);

/*
 * White-noise loads by the matrix square root (Sec. 3.3, Eq. eq:sqrt):
 * f_s = sqrt(M) y_s for samples s = 0..n_samples-1 on the finest level, with
 * y_s[i] the Philox normal of index i (DOF) of sample s in stream 2 (counter
 * layout of wm_normals), so Cov(f_s) = M up to the rule and solver errors.
 * sqrt(M) y = M sum_k c_k (M + w_k^2 I)^{-1} y with the n_nodes-point rule of
 * wm_hht_rule on [lo, hi], which must bracket the spectrum of M (e.g.
 * wm_geom_mass_bounds of the same geometry).  The n_nodes shifted systems of
 * a sample share the Krylov space of (M, y_s) and are solved together by
 * float64 multi-shift conjugate gradients (one mass apply per sample and
 * iteration) until every shifted residual satisfies |r_k| <= rtol |y_s|, at
 * most max_iter iterations.  f: device [n_samples][N] float64, caller-owned.
 * iterations: host, may be NULL; receives the CG iterations of the slowest
 * pass.  Device scratch is allocated per call (2 n_nodes + 7 float64 vectors
 * per sample, samples processed in passes that fit half the free memory) and
 * the call returns after the stream has finished.
 * Errors: WM_ERR_INVALID_ARG (sizes, bounds, host f), WM_ERR_OOM, WM_ERR_CUDA,
 * WM_ERR_NONFINITE, WM_ERR_NOT_CONVERGED (f is still written).
 */
int wm_noise_loads_sqrt(wm_hier_t h, uint64_t seed, int n_samples, double lo, double hi, int n_nodes,
                        double rtol, int max_iter, double* f, int* iterations, void* stream);

/* ---- the sampler ------------------------------------------------------------ */
typedef struct {
  double kappa;         /* kappa > 0                                                 */
  double beta;          /* beta > 0 (nu = 2 beta - 1)                                */
  int split;            /* WM_SPLIT_STANDARD or WM_SPLIT_IMPROVED                    */
  double sinc_k;        /* node step k > 0 in y                                      */
  int l_lo, l_hi;       /* node indices l_lo..l_hi (l_lo <= l_hi)                    */
  uint64_t seed;        /* Philox key of the noise                                   */
  int n_samples;        /* samples s = 0..n_samples-1                                */
  int noise_mode;       /* WM_NOISE_DRAW or WM_NOISE_GIVEN                           */
  int precision;        /* WM_FP64 or WM_MIXED                                       */
  double rtol;          /* per-system stop: ||r|| <= rtol ||rhs|| (Euclidean)        */
  int max_iter;         /* outer CG iteration cap                                    */
  int smoother_degree;  /* Chebyshev degree of pre- and post-smoothing (>= 1)        */
  double cheb_ratio;    /* Chebyshev interval [lmax/cheb_ratio, 1.1 lmax]            */
  int max_systems;      /* systems per batched solve (0 = all at once); 1 = one
                           system at a time                                          */
  int preconditioner;   /* WM_PRECOND_VCYCLE (0): one V-cycle per CG iteration;
                           WM_PRECOND_BPX (1): additive multilevel diagonal scaling,
                           the BPX preconditioner the paper's experiments favour
                           (Sec. 3.5): sum over levels of P D^{-1} P^T with the
                           dense coarse solve on the coarsest level              */
  int sample0;          /* index of the first sample: the call computes the fields
                           of samples sample0 .. sample0 + n_samples - 1 (their
                           Philox counters), stored as rows 0 .. n_samples - 1;
                           >= 0.  Splitting one sample range over calls (or
                           GPUs) gives the loads of the whole range bit for bit */
  int ckpt;             /* WM_CKPT_RECOMPUTE or WM_CKPT_KEEP.  In wm_sample_fields,
                           KEEP keeps the per-node solutions x_{l,s} of every
                           fractional pass, the pass right-hand sides, the
                           integer iterates and the loads in the hierarchy's
                           workspace (replacing an earlier checkpoint) when they
                           fit in half of the free device memory; a following
                           wm_sample_fields_backward with the same descriptor
                           and the same loads then solves the adjoint systems
                           only.  In the backward, KEEP also keeps the solutions
                           of a first pass (improved split) between its forward
                           and adjoint sweeps when they fit, instead of solving
                           them twice                                           */
  int smoother_degree_coarse;  /* Chebyshev degree on the levels below the finest,
                           0..8; 0: smoother_degree                             */
} wm_sample_desc;

typedef struct {
  int n_systems;          /* shifted systems solved (all passes)                     */
  int n_batches;          /* batched PCG solves launched                             */
  int max_iterations;     /* largest outer iteration count of any batch             */
  int total_iterations;   /* sum over batches of their iteration counts             */
  int n_not_converged;    /* systems that missed rtol                               */
  double max_rel_residual;/* largest final ||r||/||rhs|| (recursive residual)       */
  int n_int_solves;       /* integer-part solves per sample                          */
  int n_frac_passes;      /* sinc passes (0, 1 or 2)                                 */
  int n_nodes;            /* sinc nodes per pass                                     */
  int n_replacements;     /* float64 true-residual evaluations (system count)       */
  int n_df_fallbacks;     /* batches whose double-float residual failed its error
                             check and switched to float64 (mixed precision)        */
  int ckpt_kept;          /* wm_sample_fields: 1 when the forward solutions were
                             kept (WM_CKPT_KEEP and enough memory)                   */
  int ckpt_used;          /* wm_sample_fields_backward: 1 when it took the forward
                             solutions from a matching checkpoint                   */
} wm_stats;

/*
 * The fields u_s of samples 0..n_samples-1 on level 0 (see the file header for
 * the formula).  u: [n_samples][N] float64, device or host memory (host memory
 * is staged through the library's device workspace and copied back before
 * return).  b: [n_samples][N] or NULL; with WM_NOISE_DRAW the drawn loads are
 * written there if non-NULL, with WM_NOISE_GIVEN they are read from there
 * (same memory rules as u).  stats: host, may be NULL.  The stream is
 * synchronised before return.
 * Errors: WM_ERR_INVALID_ARG, WM_ERR_OOM, WM_ERR_CUDA, WM_ERR_NOT_CONVERGED
 * (u is still written with the last iterates), WM_ERR_NONFINITE.
 */
int wm_sample_fields(wm_hier_t h, const wm_sample_desc* desc, double* u, double* b,
                     wm_stats* stats, void* stream);

/*
 * Several independent problems (surfaces, levels, kappa, beta, samples) in one
 * call: u[i] receives the fields of problem i ([n_samples_i][N_i] device memory;
 * loads drawn, WM_NOISE_DRAW).  Instances with the same hierarchy handle and the
 * same solver settings (precision, rtol, max_iter, smoother, preconditioner,
 * max_systems) form a group whose instances share every batched solve: stage k
 * (an instance's k-th integer solve, then its fractional passes; Sec. 3.4) of
 * all the group's instances is one list of shifted systems, each with its own
 * shift, sample and sinc weight, solved in memory-sized batches; the first
 * stage takes the loads, every later one M times the previous stage's result.
 * Groups run one after another on the stream; when the call has several
 * groups, each hierarchy's workspace (with any checkpoint it held) is released
 * after its last group, so later groups can size their batches to the free
 * memory.  ckpt is not used here.
 * stats: host [n_inst] or NULL; per instance: its systems, convergence and
 * largest final relative residual exactly; iterations, batches, replacements
 * and fallbacks of the batches it took part in.  The stream is synchronised
 * before return.  Errors as wm_sample_fields (the worst over the instances).
 */
int wm_sample_fields_batched(int n_inst, const wm_hier_t* h, const wm_sample_desc* desc,
                             double* const* u, wm_stats* stats, void* stream);

/*
 * Gradient of a scalar loss through the fields: given grad_u = dL/du
 * [n_samples][N] (device) for the fields of `desc` with loads b (device,
 * [n_samples][N], e.g. those returned by wm_sample_fields), returns
 * grad_b = dL/db (device [n_samples][N], may be NULL) and *grad_kappa = dL/dkappa
 * (host, may be NULL), for every split (integer beta, one fractional pass, or
 * the improved split's two passes, Sec. 3.4).  The operator is symmetric, so
 * the adjoint reuses the batched shifted solves: a pass with right-hand side
 * r and nodes (c_l, sigma_l) maps dL/d(out) to dL/dr = sum_l c_l z_l,
 * z_l = (S + sigma_l M)^{-1} dL/d(out), and adds
 * -2 kappa sum_l c_l z_l^T M x_l (x_l its forward solutions) to dL/dkappa; a
 * pass fed by M v passes M dL/dr back to v; the integer solves
 * w_i = (S + kappa^2 M)^{-1} M w_{i-1} are chained the same way.  The forward
 * solutions come from a matching WM_CKPT_KEEP checkpoint of wm_sample_fields
 * (same descriptor fields and bit-identical loads), else they are recomputed
 * per batch of max_systems.  stats: host, may be NULL (systems, iterations,
 * ckpt_used).  The stream is synchronised before return.
 * Errors as wm_sample_fields; WM_ERR_INVALID_ARG also for host buffers.
 */
int wm_sample_fields_backward(wm_hier_t h, const wm_sample_desc* desc, const double* b,
                              const double* grad_u, double* grad_b, double* grad_kappa,
                              wm_stats* stats, void* stream);

/* Integer/fractional split of beta (Sec. 3.4): n_int, beta_frac, n_passes. */
int wm_beta_plan(double beta, int split, int* n_int, double* beta_frac, int* n_passes);

/*
 * Tolerance-driven sinc node set for the fractional pass of beta under `split`
 * (Eq. eq:beta-approx in y = -2t, convergence Eq. eq:K-convergence): step
 * *sinc_k and range [*l_lo, *l_hi] such that, for every eigenvalue
 * mu >= kappa^2 of M^{-1}(S + kappa^2 M), the rule's value differs from
 * mu^{-beta'} by at most tol (absolute, per unit load).  The step comes from
 * the trapezoidal error bound in the strip |Im y| < pi/2, the range from the
 * integrand's upper and lower tails, each part at tol / 3.  Host only, no GPU
 * work.  Errors: WM_ERR_INVALID_ARG (null outputs, kappa <= 0, tol outside
 * (0, 1), beta <= 0), WM_ERR_UNSUPPORTED (integer beta: no fractional pass).
 */
int wm_sinc_nodes(double beta, int split, double kappa, double tol, double* sinc_k, int* l_lo, int* l_hi);

/* ---- live profiling --------------------------------------------------------- */
/*
 * Launch counting is always on.  wm_profile_enable(1) resets the per-category
 * timers and starts recording a CUDA event pair on the launching stream around
 * every kernel launch of the library (a diagnostic aid: about a microsecond
 * of host time per launch); wm_profile_enable(0) stops.  wm_profile_read()
 * waits for the recorded events and returns, for category c in
 * [0, wm_profile_categories()), the summed device time of its timed launches,
 * their number, the number of launches since the library was loaded, the
 * algorithmic bytes and flops of the timed launches (the minimum traffic and
 * arithmetic of each launch: every vector stream of the active systems read
 * or written once, operator rows counted per stored nonzero), and a static
 * name.  Returns 1 instead of WM_OK when the event pool (65536 pairs)
 * overflowed, after which further launches were counted but not timed.
 */
int wm_profile_enable(int on);
int wm_profile_read(int c, double* total_ms, int64_t* timed_launches, int64_t* all_launches,
                    double* alg_bytes, double* alg_flops, const char** name);
int wm_profile_categories(void);

/* ---- errors and teardown ---------------------------------------------------- */
const char* wm_error_string(int code);
const char* wm_last_error(void);
void wm_destroy_hier(wm_hier_t h);
void wm_destroy_geom(wm_geom_t g);

#ifdef __cplusplus
}
#endif
#endif /* WMFIELD_H */
