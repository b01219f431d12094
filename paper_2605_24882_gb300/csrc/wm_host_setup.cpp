// Host-side set-up of the spline hierarchy: patch topology and C0 gluing,
// element connectivity, operator row patterns, 1D basis tables at the Gauss
// points, knot-insertion prolongation and the beta split.  Integer topology
// and small 1D tables only; every floating-point quantity of the discretised
// operators is computed on the GPU (wm_assembly.cu).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <unordered_map>

#include "wm_internal.h"

static thread_local std::string g_last_error;

void wm_set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

extern "C" const char* wm_last_error(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------------ Gauss rule
// Gauss–Legendre nodes/weights on [0,1] by Newton's method on P_n.
void wm_gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  std::vector<std::pair<double, double>> xw;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      // P_n(z) and P_n'(z) by the three-term recurrence
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (n == 1) p0 = 1.0;
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    if (n == 1) p0 = 1.0;
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    // on [0,1]: x = (z+1)/2 and w = (2 / ((1-z^2) P_n'(z)^2)) / 2
    xw.push_back({0.5 * (z + 1.0), 1.0 / ((1.0 - z * z) * dp * dp)});
  }
  std::sort(xw.begin(), xw.end());
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    x[i] = xw[i].first;
    w[i] = xw[i].second;
  }
}

// --------------------------------------------------------------- B-spline 1D
// Knot t_i of the p-open uniform knot vector with n elements (Sec. 2.3).
static double open_knot(int n, int p, int i) {
  if (i <= p) return 0.0;
  if (i >= n + p) return 1.0;
  return double(i - p) / n;
}

// Values and derivatives of the p+1 functions alive on element e at x, by the
// Cox–de Boor recursion (Definition 2.1) over the functions e..e+p.
static void open_local_basis(int n, int p, int e, double x, double* val, double* der) {
  // tri[d][j]: degree d function with global index e + p - d + j, j = 0..d
  double tri[8][8];
  tri[0][0] = 1.0;
  for (int d = 1; d <= p; ++d) {
    for (int j = 0; j <= d; ++j) {
      int gi = e + p - d + j;  // global function index
      double v = 0.0;
      // term with b_{gi}^{d-1}: index j-1 in the previous row (exists if 0 <= j-1 <= d-1)
      if (j - 1 >= 0) {
        double den = open_knot(n, p, gi + d) - open_knot(n, p, gi);
        if (den > 0) v += (x - open_knot(n, p, gi)) / den * tri[d - 1][j - 1];
      }
      if (j <= d - 1) {
        double den = open_knot(n, p, gi + d + 1) - open_knot(n, p, gi + 1);
        if (den > 0) v += (open_knot(n, p, gi + d + 1) - x) / den * tri[d - 1][j];
      }
      tri[d][j] = v;
    }
  }
  for (int a = 0; a <= p; ++a) val[a] = tri[p][a];
  for (int a = 0; a <= p; ++a) {
    int gi = e + a;
    double v = 0.0;
    if (p > 0) {
      if (a - 1 >= 0) {
        double den = open_knot(n, p, gi + p) - open_knot(n, p, gi);
        if (den > 0) v += p / den * tri[p - 1][a - 1];
      }
      if (a <= p - 1) {
        double den = open_knot(n, p, gi + p + 1) - open_knot(n, p, gi + 1);
        if (den > 0) v -= p / den * tri[p - 1][a];
      }
    }
    der[a] = v;
  }
}

// Cardinal B-spline N_p(t) on knots 0..p+1 and its derivative (recursion on
// the integer knots).
static void cardinal_eval(int p, double t, double* val, double* der) {
  if (t < 0.0 || t >= p + 1.0) { *val = 0.0; *der = 0.0; return; }
  int span = (int)std::floor(t);
  // degree-d functions with index span-d..span on integer knots
  double tri[8][8];
  tri[0][0] = 1.0;
  for (int d = 1; d <= p; ++d) {
    for (int j = 0; j <= d; ++j) {
      int gi = span - d + j;
      double v = 0.0;
      if (j - 1 >= 0) v += (t - gi) / d * tri[d - 1][j - 1];
      if (j <= d - 1) v += (gi + d + 1 - t) / d * tri[d - 1][j];
      tri[d][j] = v;
    }
  }
  // N_p = function with index 0 = position j = p - span in row p
  int j = p - span;
  *val = tri[p][j];
  double dv = 0.0;
  if (p > 0) {
    // d/dt N_p^{(0)} = N_{p-1}^{(0)}(t) - N_{p-1}^{(1)}(t); row p-1 holds indices span-p+1..span
    int j0 = 0 - (span - (p - 1));  // index 0
    int j1 = 1 - (span - (p - 1));  // index 1
    if (j0 >= 0 && j0 <= p - 1) dv += tri[p - 1][j0];
    if (j1 >= 0 && j1 <= p - 1) dv -= tri[p - 1][j1];
  }
  *der = dv;
}

void wm_host_tables(const wm_geom_desc& g, const std::vector<double>& gx, wm_level& L) {
  int p = g.degree, nq = (int)gx.size();
  bool periodic = wm_periodic(g.kind);
  auto fill = [&](int n, std::vector<double>& b, std::vector<double>& d) {
    b.assign((size_t)n * (p + 1) * nq, 0.0);
    d.assign((size_t)n * (p + 1) * nq, 0.0);
    for (int e = 0; e < n; ++e)
      for (int q = 0; q < nq; ++q) {
        double val[8], der[8];
        if (periodic) {
          for (int a = 0; a <= p; ++a) {
            double v, dd;
            cardinal_eval(p, gx[q] + p - a, &v, &dd);
            val[a] = v;
            der[a] = n * dd;
          }
        } else {
          open_local_basis(n, p, e, (e + gx[q]) / n, val, der);
        }
        for (int a = 0; a <= p; ++a) {
          b[((size_t)e * (p + 1) + a) * nq + q] = val[a];
          d[((size_t)e * (p + 1) + a) * nq + q] = der[a];
        }
      }
  };
  fill(L.nu, L.bu, L.du);
  fill(L.nv, L.bv, L.dv);
}

// --------------------------------------------------------------- topology
// Cube face table, identical to the surface parametrisation: patch m maps
// (u, v) to the cube point with coordinate a_axis = 2u-1, b_axis = 2v-1 and
// n_axis fixed to n_sign.
static const int kFace[6][4] = {{1, 2, 0, +1}, {2, 1, 0, -1}, {2, 0, 1, +1},
                                {0, 2, 1, -1}, {0, 1, 2, +1}, {1, 0, 2, -1}};

int wm_host_build_level(const wm_geom_desc& g, int np, int nu, int nv, wm_level& L) {
  int p = g.degree;
  L.nu = nu;
  L.nv = nv;
  L.nk = (p + 1) * (p + 1);
  L.E = np * nu * nv;
  if (wm_periodic(g.kind)) {
    L.nlu = nu;
    L.nlv = nv;
    L.N = nu * nv;
    L.l2g.resize((size_t)nu * nv);
    for (int i = 0; i < nu * nv; ++i) L.l2g[i] = i;
  } else {
    // C0 gluing by matching DOF lattice points on the cube surface: local DOF
    // (iu, iv) of patch m sits at integer coordinates a = 2 iu - (n+p-1),
    // b = 2 iv - (n+p-1), normal = n_sign (n+p-1).  Patch edges are cube
    // edges, so the shared functions of two patches land on the same points.
    int nl = nu + p;
    L.nlu = L.nlv = nl;
    L.l2g.assign((size_t)np * nl * nl, -1);
    std::unordered_map<int64_t, int32_t> seen;
    seen.reserve((size_t)np * nl * 4 + 64);
    int32_t next = 0;
    int64_t span = 2 * nl + 1;
    for (int m = 0; m < np; ++m)
      for (int iv = 0; iv < nl; ++iv)
        for (int iu = 0; iu < nl; ++iu) {
          int c[3];
          c[kFace[m][0]] = 2 * iu - (nl - 1);
          c[kFace[m][1]] = 2 * iv - (nl - 1);
          c[kFace[m][2]] = kFace[m][3] * (nl - 1);
          bool boundary = iu == 0 || iv == 0 || iu == nl - 1 || iv == nl - 1;
          int32_t gidx;
          if (boundary) {
            int64_t key = ((int64_t)(c[0] + nl) * span + (c[1] + nl)) * span + (c[2] + nl);
            auto it = seen.find(key);
            if (it != seen.end()) {
              gidx = it->second;
            } else {
              gidx = next++;
              seen.emplace(key, gidx);
            }
          } else {
            gidx = next++;
          }
          L.l2g[((size_t)m * nl + iv) * nl + iu] = gidx;
        }
    L.N = next;
  }
  // element connectivity, local index k = kv (p+1) + ku
  L.conn.resize((size_t)L.E * L.nk);
  for (int m = 0; m < np; ++m)
    for (int ev = 0; ev < nv; ++ev)
      for (int eu = 0; eu < nu; ++eu) {
        size_t e = ((size_t)m * nv + ev) * nu + eu;
        for (int kv = 0; kv <= p; ++kv)
          for (int ku = 0; ku <= p; ++ku) {
            int iu, iv;
            if (wm_periodic(g.kind)) {
              iu = ((eu - p + ku) % nu + nu) % nu;
              iv = ((ev - p + kv) % nv + nv) % nv;
            } else {
              iu = eu + ku;
              iv = ev + kv;
            }
            L.conn[e * L.nk + kv * (p + 1) + ku] = L.l2g[((size_t)m * L.nlv + iv) * L.nlu + iu];
          }
      }
  // row patterns: union of the element DOF sets containing each row
  int cap = (2 * p + 1) * (2 * p + 1) + 16;
  std::vector<int32_t> cols((size_t)L.N * cap);
  std::vector<int32_t> cnt(L.N, 0);
  for (size_t e = 0; e < (size_t)L.E; ++e) {
    const int32_t* ce = &L.conn[e * L.nk];
    for (int k = 0; k < L.nk; ++k) {
      int32_t i = ce[k];
      int32_t* row = &cols[(size_t)i * cap];
      for (int k2 = 0; k2 < L.nk; ++k2) {
        int32_t j = ce[k2];
        bool found = false;
        for (int t = 0; t < cnt[i]; ++t)
          if (row[t] == j) { found = true; break; }
        if (!found) {
          if (cnt[i] >= cap) {
            wm_set_error("row pattern overflow at row %d", i);
            return WM_ERR_INVALID_ARG;
          }
          row[cnt[i]++] = j;
        }
      }
    }
  }
  int W = 0;
  for (int i = 0; i < L.N; ++i) W = std::max(W, (int)cnt[i]);
  L.W = W;
  L.nnz = 0;
  for (int i = 0; i < L.N; ++i) L.nnz += cnt[i];
  L.col.assign((size_t)L.N * W, 0);
  L.diag_slot.assign(L.N, 0);
  for (int i = 0; i < L.N; ++i) {
    int32_t* row = &cols[(size_t)i * cap];
    std::sort(row, row + cnt[i]);
    for (int t = 0; t < W; ++t) L.col[(size_t)i * W + t] = t < cnt[i] ? row[t] : i;
    for (int t = 0; t < cnt[i]; ++t)
      if (row[t] == i) L.diag_slot[i] = t;
  }
  return WM_OK;
}

// DOF -> list of element functions (e * nk + k) containing it, in element order.
void wm_host_noise_map(const wm_level& L, std::vector<int32_t>& ptr, std::vector<int32_t>& idx) {
  ptr.assign(L.N + 1, 0);
  for (size_t t = 0; t < L.conn.size(); ++t) ptr[L.conn[t] + 1]++;
  for (int i = 0; i < L.N; ++i) ptr[i + 1] += ptr[i];
  idx.resize(L.conn.size());
  std::vector<int32_t> pos(ptr.begin(), ptr.end() - 1);
  for (size_t t = 0; t < L.conn.size(); ++t) idx[pos[L.conn[t]]++] = (int32_t)t;
}

// ------------------------------------------------------------ knot insertion
// 1D refinement matrix (n_f = 2 n_c elements) as dense [nf_dofs][nc_dofs].
// Open knots: Boehm's algorithm, inserting the midpoints one at a time.
// Periodic: the two-scale relation of the cardinal B-spline, which is the same
// insertion of all midpoints at once: N_p(t) = sum_k 2^-p C(p+1,k) N_p(2t-k).
static void refine_1d(int nc, int p, bool periodic, std::vector<double>& P, int& nf_dofs, int& nc_dofs) {
  if (periodic) {
    nc_dofs = nc;
    nf_dofs = 2 * nc;
    P.assign((size_t)nf_dofs * nc_dofs, 0.0);
    for (int I = 0; I < nc; ++I)
      for (int k = 0; k <= p + 1; ++k) {
        double binom = 1.0;
        for (int t = 0; t < k; ++t) binom = binom * (p + 1 - t) / (t + 1);
        int f = (2 * I + k) % nf_dofs;
        P[(size_t)f * nc_dofs + I] += binom / std::pow(2.0, p);
      }
    return;
  }
  nc_dofs = nc + p;
  nf_dofs = 2 * nc + p;
  std::vector<double> knots;
  for (int i = 0; i <= p; ++i) knots.push_back(0.0);
  for (int i = 1; i < nc; ++i) knots.push_back(double(i) / nc);
  for (int i = 0; i <= p; ++i) knots.push_back(1.0);
  // current control "points" = identity columns: Q[i][I]
  std::vector<std::vector<double>> Q(nc_dofs, std::vector<double>(nc_dofs, 0.0));
  for (int i = 0; i < nc_dofs; ++i) Q[i][i] = 1.0;
  for (int el = 0; el < nc; ++el) {
    double t = (el + 0.5) / nc;
    // span s: knots[s] <= t < knots[s+1]
    int s = 0;
    for (int i = 0; i + 1 < (int)knots.size(); ++i)
      if (knots[i] <= t && t < knots[i + 1]) s = i;
    int ncp = (int)Q.size();
    std::vector<std::vector<double>> R(ncp + 1, std::vector<double>(nc_dofs, 0.0));
    for (int i = 0; i <= ncp; ++i) {
      if (i <= s - p) {
        R[i] = Q[i];
      } else if (i > s) {
        R[i] = Q[i - 1];
      } else {
        double a = (t - knots[i]) / (knots[i + p] - knots[i]);
        for (int c = 0; c < nc_dofs; ++c) R[i][c] = a * Q[i][c] + (1.0 - a) * Q[i - 1][c];
      }
    }
    knots.insert(knots.begin() + s + 1, t);
    Q.swap(R);
  }
  P.assign((size_t)nf_dofs * nc_dofs, 0.0);
  for (int f = 0; f < nf_dofs; ++f)
    for (int c = 0; c < nc_dofs; ++c) P[(size_t)f * nc_dofs + c] = Q[f][c];
}

int wm_host_prolongation(const wm_geom_desc& g, int np, const wm_level& F, const wm_level& C,
                         std::vector<int32_t>& Pptr, std::vector<int32_t>& Pcol, std::vector<double>& Pval,
                         std::vector<int32_t>& Rptr, std::vector<int32_t>& Rcol, std::vector<double>& Rval) {
  int p = g.degree;
  bool periodic = wm_periodic(g.kind);
  std::vector<double> Pu, Pv;
  int nfu, ncu, nfv, ncv;
  refine_1d(C.nu, p, periodic, Pu, nfu, ncu);
  refine_1d(C.nv, p, periodic, Pv, nfv, ncv);
  if (nfu != F.nlu || nfv != F.nlv || ncu != C.nlu || ncv != C.nlv) {
    wm_set_error("prolongation size mismatch");
    return WM_ERR_INVALID_ARG;
  }
  // per fine row: (coarse col, value), deduplicated across patches
  std::vector<std::vector<std::pair<int32_t, double>>> rows(F.N);
  for (int m = 0; m < np; ++m)
    for (int fv = 0; fv < nfv; ++fv)
      for (int fu = 0; fu < nfu; ++fu) {
        int32_t i = F.l2g[((size_t)m * F.nlv + fv) * F.nlu + fu];
        auto& row = rows[i];
        bool have = !row.empty();
        std::vector<std::pair<int32_t, double>> mine;
        for (int Iv = 0; Iv < ncv; ++Iv) {
          double a = Pv[(size_t)fv * ncv + Iv];
          if (a == 0.0) continue;
          for (int Iu = 0; Iu < ncu; ++Iu) {
            double b = Pu[(size_t)fu * ncu + Iu];
            if (b == 0.0) continue;
            mine.push_back({C.l2g[((size_t)m * C.nlv + Iv) * C.nlu + Iu], a * b});
          }
        }
        std::sort(mine.begin(), mine.end());
        if (!have) {
          row = mine;
        } else {
          // the same glued function seen from another patch: must agree
          if (mine.size() != row.size()) {
            wm_set_error("inconsistent prolongation row %d (%zu vs %zu)", i, mine.size(), row.size());
            return WM_ERR_INVALID_ARG;
          }
          for (size_t t = 0; t < mine.size(); ++t)
            if (mine[t].first != row[t].first || std::fabs(mine[t].second - row[t].second) > 1e-13) {
              wm_set_error("inconsistent prolongation entry at row %d", i);
              return WM_ERR_INVALID_ARG;
            }
        }
      }
  Pptr.assign(F.N + 1, 0);
  for (int i = 0; i < F.N; ++i) Pptr[i + 1] = Pptr[i] + (int)rows[i].size();
  Pcol.resize(Pptr[F.N]);
  Pval.resize(Pptr[F.N]);
  for (int i = 0; i < F.N; ++i)
    for (size_t t = 0; t < rows[i].size(); ++t) {
      Pcol[Pptr[i] + t] = rows[i][t].first;
      Pval[Pptr[i] + t] = rows[i][t].second;
    }
  // transpose: rows of R are coarse DOFs, entries ordered by fine index
  Rptr.assign(C.N + 1, 0);
  for (size_t t = 0; t < Pcol.size(); ++t) Rptr[Pcol[t] + 1]++;
  for (int I = 0; I < C.N; ++I) Rptr[I + 1] += Rptr[I];
  Rcol.resize(Pcol.size());
  Rval.resize(Pcol.size());
  std::vector<int32_t> pos(Rptr.begin(), Rptr.end() - 1);
  for (int i = 0; i < F.N; ++i)
    for (int t = Pptr[i]; t < Pptr[i + 1]; ++t) {
      int32_t I = Pcol[t];
      Rcol[pos[I]] = i;
      Rval[pos[I]] = Pval[t];
      pos[I]++;
    }
  return WM_OK;
}

// ------------------------------------------------------------ sqrt(M) rule
// Jacobian elliptic functions sn, cn, dn of argument u and parameter q, and the
// complete elliptic integral of the first kind K(q), by the scale of the
// arithmetic-geometric mean (Abramowitz & Stegun 16.4 and 17.6):
// a_0 = 1, b_0 = sqrt(1-q), c_0 = sqrt(q); a_n, b_n the means, c_n = (a_{n-1} - b_{n-1})/2;
// phi_N = 2^N a_N u and phi_{n-1} = (phi_n + asin(c_n sin(phi_n) / a_n)) / 2;
// sn = sin phi_0, cn = cos phi_0, dn = cos phi_0 / cos(phi_1 - phi_0); K = pi / (2 a_N).
namespace {
struct Agm {
  double a[40], c[40];
  int n = 0;
};

Agm agm_scale(double q) {
  Agm s;
  double a = 1.0, b = std::sqrt(1.0 - q);
  s.a[0] = a;
  s.c[0] = std::sqrt(q);
  while (s.n < 38 && std::fabs(a - b) > 3e-16 * a) {
    double an = 0.5 * (a + b), bn = std::sqrt(a * b);
    ++s.n;
    s.c[s.n] = 0.5 * (a - b);
    s.a[s.n] = an;
    a = an;
    b = bn;
  }
  return s;
}

void jacobi_sncndn(const Agm& s, double u, double* sn, double* cn, double* dn) {
  if (s.n == 0) {
    *sn = std::sin(u);
    *cn = std::cos(u);
    *dn = 1.0;
    return;
  }
  double phi = std::ldexp(s.a[s.n] * u, s.n), prev = phi;
  for (int k = s.n; k >= 1; --k) {
    prev = phi;
    phi = 0.5 * (phi + std::asin(s.c[k] * std::sin(phi) / s.a[k]));
  }
  *sn = std::sin(phi);
  *cn = std::cos(phi);
  *dn = *cn / std::cos(prev - phi);
}
}  // namespace

// Shifts and weights of the K^-node rule A^{1/2} y ~= A sum_k c_k (A + w_k^2 I)^{-1} y
// (Sec. 3.3, Eq. eq:sqrt): w = sqrt(lo) sn(t|q)/cn(t|q), q = 1 - lo/hi, and the
// midpoint rule t_k = (k - 1/2) K(q) / K^ on A^{-1/2} = (2/pi) int_0^inf (A + w^2 I)^{-1} dw.
// Nodes past K/2 are evaluated at the reflected argument u = K - t
// (sn(t) = cn(u)/dn(u), cn(t) = k' sn(u)/dn(u), dn(t) = k'/dn(u), k'^2 = 1 - q),
// where cn(t) would otherwise be known only to absolute accuracy.
extern "C" int wm_hht_rule(double lo, double hi, int n_nodes, double* w2, double* c) {
  if (!(lo > 0.0 && hi > lo) || n_nodes < 1 || !w2 || !c) {
    wm_set_error("hht rule needs 0 < lo < hi, n_nodes >= 1 and output arrays");
    return WM_ERR_INVALID_ARG;
  }
  double q = 1.0 - lo / hi, kp2 = 1.0 - q;
  Agm s = agm_scale(q);
  double K = 0.5 * M_PI / s.a[s.n];
  double pre = 2.0 * K / (M_PI * n_nodes);
  for (int k = 0; k < n_nodes; ++k) {
    double t = (k + 0.5) * K / n_nodes;
    double sn, cn, dn;
    if (t <= 0.5 * K) {
      jacobi_sncndn(s, t, &sn, &cn, &dn);
      w2[k] = lo * (sn / cn) * (sn / cn);
      c[k] = pre * std::sqrt(lo) * dn / (cn * cn);
    } else {
      jacobi_sncndn(s, K - t, &sn, &cn, &dn);
      w2[k] = lo / kp2 * (cn / sn) * (cn / sn);
      c[k] = pre * std::sqrt(lo / kp2) * dn / (sn * sn);
    }
  }
  return WM_OK;
}

// Extremes of the spectrum of the 1D mass matrix int_0^1 B_i B_j of the spline
// space with n elements (exact with the p+1 point Gauss rule).  Open knots: the
// matrix is banded (bandwidth p) and positive definite, and lambda_min (lambda_max)
// is located by bisection on sigma with a banded Cholesky factorisation of
// A - sigma I (sigma I - A), which exists exactly when sigma is below (above)
// the spectrum.  Periodic: the matrix is circulant, lambda_k = c_0 + 2 sum_j c_j cos(2 pi j k / n).
static void mass_1d_extremes(const wm_geom_desc& g, int n, const std::vector<double>& gx,
                             const std::vector<double>& gw, double* lmin, double* lmax) {
  int p = g.degree, nq = (int)gx.size();
  bool periodic = wm_periodic(g.kind);
  int nd = periodic ? n : n + p;
  // band storage: B[i][d] = A[i][i+d], d = 0..p (periodic: offsets mod n, c_d)
  std::vector<double> B((size_t)nd * (p + 1), 0.0);
  for (int e = 0; e < n; ++e)
    for (int qi = 0; qi < nq; ++qi) {
      double val[8], der[8];
      if (periodic) {
        for (int a = 0; a <= p; ++a) cardinal_eval(p, gx[qi] + p - a, &val[a], &der[a]);
      } else {
        open_local_basis(n, p, e, (e + gx[qi]) / n, val, der);
      }
      for (int a = 0; a <= p; ++a)
        for (int b = a; b <= p; ++b) {
          int i = periodic ? ((e - p + a) % n + n) % n : e + a;
          B[(size_t)i * (p + 1) + (b - a)] += gw[qi] / n * val[a] * val[b];
        }
    }
  if (periodic) {
    // every row of the circulant carries the same c_d; take row 0
    *lmin = 1e300;
    *lmax = -1e300;
    for (int k = 0; k < n; ++k) {
      double lam = B[0];
      for (int d = 1; d <= p; ++d) lam += 2.0 * B[d] * std::cos(2.0 * M_PI * d * k / n);
      *lmin = std::min(*lmin, lam);
      *lmax = std::max(*lmax, lam);
    }
    return;
  }
  auto chol_ok = [&](double sigma, double sign) {
    // factor sign*(A - sigma I) in band form, L[i][d] = L(i, i-d)
    std::vector<double> L((size_t)nd * (p + 1), 0.0);
    for (int i = 0; i < nd; ++i)
      for (int j = std::max(0, i - p); j <= i; ++j) {
        double v = sign * (B[(size_t)j * (p + 1) + (i - j)] - (i == j ? sigma : 0.0));
        for (int k = std::max(0, i - p); k < j; ++k) v -= L[(size_t)i * (p + 1) + (i - k)] * L[(size_t)j * (p + 1) + (j - k)];
        if (i == j) {
          if (!(v > 0.0)) return false;
          L[(size_t)i * (p + 1)] = std::sqrt(v);
        } else {
          L[(size_t)i * (p + 1) + (i - j)] = v / L[(size_t)j * (p + 1)];
        }
      }
    return true;
  };
  double rowmax = 0.0;
  for (int i = 0; i < nd; ++i) {
    double r = 0.0;
    for (int j = std::max(0, i - p); j <= std::min(nd - 1, i + p); ++j)
      r += std::fabs(i <= j ? B[(size_t)i * (p + 1) + (j - i)] : B[(size_t)j * (p + 1) + (i - j)]);
    rowmax = std::max(rowmax, r);
  }
  double a = 0.0, b = rowmax;  // chol(A - a I) succeeds, chol(A - b I) fails
  for (int it = 0; it < 200 && b - a > 1e-15 * rowmax; ++it) {
    double m = 0.5 * (a + b);
    (chol_ok(m, 1.0) ? a : b) = m;
  }
  *lmin = a;
  a = 0.0;
  b = rowmax * (1.0 + 1e-12);  // chol(b I - A) succeeds, chol(a I - A) fails
  for (int it = 0; it < 200 && b - a > 1e-15 * rowmax; ++it) {
    double m = 0.5 * (a + b);
    (chol_ok(m, -1.0) ? b : a) = m;
  }
  *lmax = b;
}

// Bounds lo <= lambda_min(M) <= lambda_max(M) <= hi of the assembled mass matrix
// of one level.  On a patch the quadrature mass form is sum_q w_q a_q (sum_i x_i phi_i)^2,
// between a_min and a_max times the flat form x^T (M_u (x) M_v) x, which the
// p+1 point rule integrates exactly; the patches' DOF vectors x_m satisfy
// |x|^2 <= sum_m |x_m|^2 <= mult |x|^2 (mult = 3 on the cube sphere, whose corner
// DOFs lie on three patches).  amin, amax bound the area element at the Gauss
// points (NURBS kinds: their extremes there).
int wm_host_mass_bounds_metric(const wm_geom_desc& g, int nu, int nv, double amin, double amax, double* lo,
                               double* hi) {
  std::vector<double> gx, gw;
  wm_gauss_legendre01(g.degree + 1, gx, gw);
  double umin, umax, vmin, vmax;
  mass_1d_extremes(g, nu, gx, gw, &umin, &umax);
  mass_1d_extremes(g, nv, gx, gw, &vmin, &vmax);
  const double mult = wm_periodic(g.kind) ? 1.0 : 3.0;
  if (!(umin > 0.0 && vmin > 0.0 && amin > 0.0)) {
    wm_set_error("mass bounds need positive 1D spectra and area elements");
    return WM_ERR_INVALID_ARG;
  }
  // relative margins cover the rounding of the bisection and of the area elements
  *lo = amin * umin * vmin * (1.0 - 1e-9);
  *hi = mult * amax * umax * vmax * (1.0 + 1e-9);
  return WM_OK;
}

// Analytic kinds, area elements in closed form: gnomonic 4 (1 + a^2 + b^2)^{-3/2},
// a, b in [-1, 1], so a in [4 / 3^{3/2}, 4]; torus 4 pi^2 r (R + r cos 2 pi v).
int wm_host_mass_bounds(const wm_geom_desc& g, int nu, int nv, double* lo, double* hi) {
  double amin, amax;
  if (g.kind == WM_TORUS) {
    amin = 4.0 * M_PI * M_PI * g.r * (g.R - g.r);
    amax = 4.0 * M_PI * M_PI * g.r * (g.R + g.r);
  } else {
    amin = 4.0 / (3.0 * std::sqrt(3.0));
    amax = 4.0;
  }
  return wm_host_mass_bounds_metric(g, nu, nv, amin, amax, lo, hi);
}

// ------------------------------------------------------------ NURBS geometry
// Span s of x in a clamped knot vector of n basis functions of degree p:
// knots[s] <= x < knots[s+1], s in [p, n-1]; x at the right end takes the last
// non-empty span.
static int nurbs_span(const std::vector<double>& kn, int p, int n, double x) {
  if (x >= kn[n]) {
    int s = n - 1;
    while (s > p && !(kn[s] < kn[s + 1])) --s;
    return s;
  }
  int lo = p, hi = n;  // kn[lo] <= x < kn[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (x < kn[mid]) hi = mid; else lo = mid;
  }
  return lo;
}

// Values N[a] and derivatives dN[a] of the p+1 B-splines s-p+a (a = 0..p) that
// are non-zero on span s, by the Cox–de Boor recursion (Definition 2.1); the
// derivative from the degree p-1 functions.
static void nurbs_basis(const std::vector<double>& kn, int p, int s, double x, double* N, double* dN) {
  double tri[9][9];
  tri[0][0] = 1.0;
  for (int d = 1; d <= p; ++d)
    for (int j = 0; j <= d; ++j) {
      int i = s - d + j;
      double v = 0.0;
      if (j >= 1) {
        double den = kn[i + d] - kn[i];
        if (den > 0) v += (x - kn[i]) / den * tri[d - 1][j - 1];
      }
      if (j <= d - 1) {
        double den = kn[i + d + 1] - kn[i + 1];
        if (den > 0) v += (kn[i + d + 1] - x) / den * tri[d - 1][j];
      }
      tri[d][j] = v;
    }
  for (int a = 0; a <= p; ++a) {
    N[a] = tri[p][a];
    int i = s - p + a;
    double v = 0.0;
    if (p > 0) {
      if (a >= 1) {
        double den = kn[i + p] - kn[i];
        if (den > 0) v += p / den * tri[p - 1][a - 1];
      }
      if (a <= p - 1) {
        double den = kn[i + p + 1] - kn[i + 1];
        if (den > 0) v -= p / den * tri[p - 1][a];
      }
    }
    dN[a] = v;
  }
}

// F, d_u F, d_v F of a patch: F = A / W with A = sum N_i M_j w_ij P_ij and
// W = sum N_i M_j w_ij; d F = (d A - F d W) / W.
static void nurbs_eval(const WmNurbs& P, double u, double v, double F[3], double Fu[3], double Fv[3]) {
  double Nu[9], dNu[9], Nv[9], dNv[9];
  int su = nurbs_span(P.ku, P.pu, P.nu, u), sv = nurbs_span(P.kv, P.pv, P.nv, v);
  nurbs_basis(P.ku, P.pu, su, u, Nu, dNu);
  nurbs_basis(P.kv, P.pv, sv, v, Nv, dNv);
  double A[3] = {0, 0, 0}, Au[3] = {0, 0, 0}, Av[3] = {0, 0, 0}, W = 0, Wu = 0, Wv = 0;
  for (int b = 0; b <= P.pv; ++b)
    for (int a = 0; a <= P.pu; ++a) {
      const double* c = &P.cpw[((size_t)(sv - P.pv + b) * P.nu + (su - P.pu + a)) * 4];
      double w = c[3];
      double f = Nu[a] * Nv[b] * w, fu = dNu[a] * Nv[b] * w, fv = Nu[a] * dNv[b] * w;
      for (int k = 0; k < 3; ++k) {
        A[k] += f * c[k];
        Au[k] += fu * c[k];
        Av[k] += fv * c[k];
      }
      W += f;
      Wu += fu;
      Wv += fv;
    }
  for (int k = 0; k < 3; ++k) {
    F[k] = A[k] / W;
    Fu[k] = (Au[k] - F[k] * Wu) / W;
    Fv[k] = (Av[k] - F[k] * Wv) / W;
  }
}

int wm_host_nurbs_metric(const std::vector<WmNurbs>& patches, int nu, int nv, const std::vector<double>& gx,
                         std::vector<double>& out) {
  const int nq = (int)gx.size(), np = (int)patches.size();
  out.assign((size_t)np * nu * nv * nq * nq * 4, 0.0);
  for (int m = 0; m < np; ++m)
    for (int ev = 0; ev < nv; ++ev)
      for (int eu = 0; eu < nu; ++eu)
        for (int gv = 0; gv < nq; ++gv)
          for (int gu = 0; gu < nq; ++gu) {
            double F[3], Fu[3], Fv[3];
            nurbs_eval(patches[m], (eu + gx[gu]) / nu, (ev + gx[gv]) / nv, F, Fu, Fv);
            double K11 = Fu[0] * Fu[0] + Fu[1] * Fu[1] + Fu[2] * Fu[2];
            double K12 = Fu[0] * Fv[0] + Fu[1] * Fv[1] + Fu[2] * Fv[2];
            double K22 = Fv[0] * Fv[0] + Fv[1] * Fv[1] + Fv[2] * Fv[2];
            double det = K11 * K22 - K12 * K12;
            if (!(det > 0.0) || !std::isfinite(det)) {
              wm_set_error("degenerate NURBS map on patch %d element (%d, %d)", m, eu, ev);
              return WM_ERR_INVALID_ARG;
            }
            double a = std::sqrt(det);
            double* o = &out[((((size_t)m * nv + ev) * nu + eu) * nq * nq + gv * nq + gu) * 4];
            o[0] = a;
            o[1] = K22 / a;
            o[2] = -K12 / a;
            o[3] = K11 / a;
          }
  return WM_OK;
}

// Knots clamped to [0, 1] and nondecreasing, weights positive, coordinates
// finite; then the closure of a periodic patch (F(0, t) = F(1, t), F(t, 0) =
// F(t, 1)) or, for six cube-arranged patches, the agreement of every patch
// edge with its neighbour at the same cube point, at 33 points per edge, to
// 1e-10 of the largest control point coordinate.
int wm_host_nurbs_check(int kind, const std::vector<WmNurbs>& P) {
  double scale = 0.0;
  for (size_t m = 0; m < P.size(); ++m) {
    const WmNurbs& q = P[m];
    for (int dir = 0; dir < 2; ++dir) {
      const std::vector<double>& kn = dir ? q.kv : q.ku;
      int p = dir ? q.pv : q.pu, n = dir ? q.nv : q.nu;
      if (p < 1 || p > 8 || n < p + 1 || (int)kn.size() != n + p + 1) {
        wm_set_error("patch %zu: degree 1..8 and n >= degree + 1 control points per direction", m);
        return WM_ERR_INVALID_ARG;
      }
      for (int i = 0; i + 1 < (int)kn.size(); ++i)
        if (!(kn[i] <= kn[i + 1])) {
          wm_set_error("patch %zu: knots must be nondecreasing", m);
          return WM_ERR_INVALID_ARG;
        }
      for (int i = 0; i <= p; ++i)
        if (kn[i] != 0.0 || kn[n + i] != 1.0) {
          wm_set_error("patch %zu: knot vectors must be clamped to [0, 1]", m);
          return WM_ERR_INVALID_ARG;
        }
    }
    for (size_t i = 0; i < q.cpw.size(); ++i) {
      if (!std::isfinite(q.cpw[i]) || (i % 4 == 3 && !(q.cpw[i] > 0.0))) {
        wm_set_error("patch %zu: control points must be finite and weights positive", m);
        return WM_ERR_INVALID_ARG;
      }
      if (i % 4 != 3) scale = std::max(scale, std::fabs(q.cpw[i]));
    }
  }
  const double tol = 1e-10 * std::max(scale, 1e-300);
  auto dist = [](const double* a, const double* b) {
    return std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
  };
  const int ns = 33;
  double F0[3], F1[3], du[3], dv[3];
  if (kind == WM_NURBS_PERIODIC) {
    for (int i = 0; i < ns; ++i) {
      double t = (double)i / (ns - 1);
      nurbs_eval(P[0], 0.0, t, F0, du, dv);
      nurbs_eval(P[0], 1.0, t, F1, du, dv);
      bool ok = dist(F0, F1) <= tol;
      nurbs_eval(P[0], t, 0.0, F0, du, dv);
      nurbs_eval(P[0], t, 1.0, F1, du, dv);
      if (!ok || dist(F0, F1) > tol) {
        wm_set_error("periodic NURBS patch is not closed (at t = %g)", t);
        return WM_ERR_INVALID_ARG;
      }
    }
    return WM_OK;
  }
  // cube arrangement: a boundary point of patch m sits at the cube point c with
  // c[a] = 2u-1, c[b] = 2v-1, c[n] = s; every other patch m' with c[n'] = s' holds
  // the same point at u' = (c[a'] + 1)/2, v' = (c[b'] + 1)/2
  for (int m = 0; m < 6; ++m)
    for (int e = 0; e < 4; ++e)
      for (int i = 0; i < ns; ++i) {
        double t = (double)i / (ns - 1);
        double u = e == 0 ? t : e == 1 ? t : e == 2 ? 0.0 : 1.0;
        double v = e == 0 ? 0.0 : e == 1 ? 1.0 : t;
        double c[3];
        c[kFace[m][0]] = 2.0 * u - 1.0;
        c[kFace[m][1]] = 2.0 * v - 1.0;
        c[kFace[m][2]] = kFace[m][3];
        nurbs_eval(P[m], u, v, F0, du, dv);
        for (int m2 = 0; m2 < 6; ++m2) {
          if (m2 == m || c[kFace[m2][2]] != (double)kFace[m2][3]) continue;
          nurbs_eval(P[m2], 0.5 * (c[kFace[m2][0]] + 1.0), 0.5 * (c[kFace[m2][1]] + 1.0), F1, du, dv);
          if (dist(F0, F1) > tol) {
            wm_set_error("NURBS patches %d and %d disagree on their shared edge (t = %g)", m, m2, t);
            return WM_ERR_INVALID_ARG;
          }
        }
      }
  return WM_OK;
}

// ------------------------------------------------------------ beta split
int wm_split_beta(double beta, int split, int* n, double* bp, int* passes) {
  if (!(beta > 0.0) || !std::isfinite(beta)) return WM_ERR_INVALID_ARG;
  int ni = (int)std::floor(beta);
  double f = beta - ni;
  if (f == 0.0) {
    *n = ni; *bp = 0.0; *passes = 0;
    return WM_OK;
  }
  if (split == WM_SPLIT_IMPROVED) {
    if (f < 1.0 / 3.0 && ni >= 1) { *n = ni - 1; *bp = (f + 1.0) / 2.0; *passes = 2; return WM_OK; }
    if (f > 2.0 / 3.0) { *n = ni; *bp = f / 2.0; *passes = 2; return WM_OK; }
  } else if (split != WM_SPLIT_STANDARD) {
    return WM_ERR_INVALID_ARG;
  }
  *n = ni; *bp = f; *passes = 1;
  return WM_OK;
}

extern "C" int wm_beta_plan(double beta, int split, int* n_int, double* beta_frac, int* n_passes) {
  if (!n_int || !beta_frac || !n_passes) return WM_ERR_INVALID_ARG;
  return wm_split_beta(beta, split, n_int, beta_frac, n_passes);
}

// Node set for an absolute error <= tol: with g the pass exponent, the sinc
// sum approximates mu^{-g} = s * integral of e^{(1-g)y} / (e^y + mu) dy,
// s = sin(pi g) / pi, mu >= kappa^2.  Step: the trapezoidal error for a
// function analytic in |Im y| < pi/2 is about 2 B e^{-pi^2/k}, with
// B = 2 s (1/g + 1/((1-g) kappa^2)) bounding the integrand's strip integral;
// tails: s e^{-g y_hi} / g above and s e^{(1-g) y_lo} / ((1-g) kappa^2) below.
// Each part is set to tol / 3.
extern "C" int wm_sinc_nodes(double beta, int split, double kappa, double tol, double* sinc_k, int* l_lo,
                             int* l_hi) {
  if (!sinc_k || !l_lo || !l_hi || !(kappa > 0.0) || !(tol > 0.0 && tol < 1.0)) return WM_ERR_INVALID_ARG;
  int n = 0, passes = 0;
  double g = 0.0;
  WM_TRY(wm_split_beta(beta, split, &n, &g, &passes));
  if (passes == 0) {
    wm_set_error("beta = %g is an integer: there is no fractional pass", beta);
    return WM_ERR_UNSUPPORTED;
  }
  const double pi = 3.14159265358979323846;
  const double s = std::sin(pi * g) / pi;
  const double mu = kappa * kappa;
  const double bound = 2.0 * s * (1.0 / g + 1.0 / ((1.0 - g) * mu));
  const double k = pi * pi / std::log(3.0 * bound / tol);
  const double y_hi = std::log(3.0 * s / (g * tol)) / g;
  const double y_lo = std::log(tol * (1.0 - g) * mu / (3.0 * s)) / (1.0 - g);
  *sinc_k = k;
  *l_lo = (int)std::floor(y_lo / k);
  *l_hi = (int)std::ceil(y_hi / k);
  return WM_OK;
}

// ------------------------------------------------------------ stencil form
// Extended patch grids for the shared-memory stencil kernels.  Each patch's
// local DOF grid is extended by a halo of width p: halo cells across a cube
// edge are the adjacent face's DOFs at the same distance from the edge (the
// integer cube lattice folded over the edge), halo cells of the periodic torus
// wrap around, and cells beyond a cube corner are empty (-1).  Every operator
// row is then a (2p+1)^2 stencil in the frame of the patch that owns the row
// (the first patch in which the DOF occurs); slot[i][w] gives the stencil slot
// of the stored entry w of row i (-1 for padding).  Returns WM_ERR_UNSUPPORTED
// if some entry falls outside its owner's stencil window.
int wm_host_stencil(const wm_geom_desc& g, int np, const wm_level& L, std::vector<int32_t>& ext,
                    std::vector<int32_t>& own, std::vector<int16_t>& slot) {
  const int p = g.degree;
  const int nlu = L.nlu, nlv = L.nlv;
  const int ELU = nlu + 2 * p, ELV = nlv + 2 * p;
  const int SW = 2 * p + 1;
  ext.assign((size_t)np * ELV * ELU, -1);
  own.assign((size_t)np * nlv * nlu, -1);
  if (wm_periodic(g.kind)) {
    for (int ev = 0; ev < ELV; ++ev)
      for (int eu = 0; eu < ELU; ++eu) {
        int iu = ((eu - p) % nlu + nlu) % nlu, iv = ((ev - p) % nlv + nlv) % nlv;
        ext[(size_t)ev * ELU + eu] = L.l2g[(size_t)iv * nlu + iu];
      }
    for (int t = 0; t < nlu * nlv; ++t) own[t] = L.l2g[t];
  } else {
    const int nl = nlu;
    const int64_t span = 2 * nl + 1;
    auto key = [&](const int c[3]) { return ((int64_t)(c[0] + nl) * span + (c[1] + nl)) * span + (c[2] + nl); };
    std::unordered_map<int64_t, int32_t> lat;
    lat.reserve((size_t)L.N * 2);
    std::vector<char> seen(L.N, 0);
    for (int m = 0; m < np; ++m)
      for (int iv = 0; iv < nl; ++iv)
        for (int iu = 0; iu < nl; ++iu) {
          int c[3];
          c[kFace[m][0]] = 2 * iu - (nl - 1);
          c[kFace[m][1]] = 2 * iv - (nl - 1);
          c[kFace[m][2]] = kFace[m][3] * (nl - 1);
          int32_t gi = L.l2g[((size_t)m * nl + iv) * nl + iu];
          lat[key(c)] = gi;
          if (!seen[gi]) {
            seen[gi] = 1;
            own[((size_t)m * nl + iv) * nl + iu] = gi;
          }
        }
    for (int m = 0; m < np; ++m)
      for (int ev = 0; ev < ELV; ++ev)
        for (int eu = 0; eu < ELU; ++eu) {
          int iu = eu - p, iv = ev - p;
          bool ou = iu < 0 || iu >= nl, ov = iv < 0 || iv >= nl;
          if (ou && ov) continue;  // beyond a cube corner
          int c[3];
          c[kFace[m][0]] = 2 * iu - (nl - 1);
          c[kFace[m][1]] = 2 * iv - (nl - 1);
          c[kFace[m][2]] = kFace[m][3] * (nl - 1);
          if (ou) {  // fold over the edge iu = 0 or iu = nl-1 onto the adjacent face
            int k = iu < 0 ? -iu : iu - (nl - 1);
            c[kFace[m][0]] = iu < 0 ? -(nl - 1) : (nl - 1);
            c[kFace[m][2]] = kFace[m][3] * (nl - 1 - 2 * k);
          }
          if (ov) {
            int k = iv < 0 ? -iv : iv - (nl - 1);
            c[kFace[m][1]] = iv < 0 ? -(nl - 1) : (nl - 1);
            c[kFace[m][2]] = kFace[m][3] * (nl - 1 - 2 * k);
          }
          auto it = lat.find(key(c));
          if (it != lat.end()) ext[((size_t)m * ELV + ev) * ELU + eu] = it->second;
        }
  }
  // owner frame of every row and the slot of each stored entry
  std::vector<int32_t> om(L.N, -1), ou(L.N, -1), ov(L.N, -1);
  for (int m = 0; m < np; ++m)
    for (int iv = 0; iv < nlv; ++iv)
      for (int iu = 0; iu < nlu; ++iu) {
        int32_t gi = own[((size_t)m * nlv + iv) * nlu + iu];
        if (gi >= 0) {
          om[gi] = m;
          ou[gi] = iu;
          ov[gi] = iv;
        }
      }
  slot.assign((size_t)L.N * L.W, -1);
  std::vector<char> used(SW * SW);
  for (int i = 0; i < L.N; ++i) {
    if (om[i] < 0) return WM_ERR_UNSUPPORTED;
    std::fill(used.begin(), used.end(), 0);
    const int32_t* E = &ext[(size_t)om[i] * ELV * ELU];
    for (int w = 0; w < L.W; ++w) {
      int32_t j = L.col[(size_t)i * L.W + w];
      bool dup = false;
      for (int w2 = 0; w2 < w; ++w2)
        if (L.col[(size_t)i * L.W + w2] == j) dup = true;
      if (dup) continue;  // padding
      int found = -1;
      for (int s = 0; s < SW * SW && found < 0; ++s) {
        int dv = s / SW - p, du = s % SW - p;
        int eu = ou[i] + p + du, ev = ov[i] + p + dv;
        if (!used[s] && E[(size_t)ev * ELU + eu] == j) found = s;
      }
      if (found < 0) return WM_ERR_UNSUPPORTED;
      used[found] = 1;
      slot[(size_t)i * L.W + w] = (int16_t)found;
    }
  }
  return WM_OK;
}
