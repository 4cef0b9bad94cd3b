// Host-side setup: see host_setup.h.  FP64 throughout.
#include "host_setup.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <iterator>
#include <numeric>
#include <omp.h>

namespace pdh {
namespace {

enum { ST_INVALID = 1, ST_BAD_MESH = 2, ST_REGION = 3, ST_NOT_SPD = 5, ST_OOM = 9 };

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Sorted, duplicate-free rows of a sparse pattern from the (row, column)
// pairs that pairs(f) reports by calling f(row, column): a counting pass, a
// filling pass, then every row sorted on its own (rows in parallel).
template <class Pairs>
void pattern_rows(int64_t nrows, Pairs pairs, std::vector<int64_t>& ptr, std::vector<int32_t>& adj) {
  std::vector<int64_t> start(nrows + 1, 0);
  pairs([&](int64_t r, int64_t) { ++start[r + 1]; });
  for (int64_t i = 0; i < nrows; ++i) start[i + 1] += start[i];
  std::vector<int32_t> tmp(start[nrows]);
  std::vector<int64_t> cur(start.begin(), start.end() - 1);
  pairs([&](int64_t r, int64_t c) { tmp[cur[r]++] = (int32_t)c; });
  std::vector<int64_t> len(nrows);
#pragma omp parallel for schedule(dynamic, 512)
  for (int64_t i = 0; i < nrows; ++i) {
    const auto b = tmp.begin() + start[i], e = tmp.begin() + start[i + 1];
    std::sort(b, e);
    len[i] = std::unique(b, e) - b;
  }
  ptr.assign(nrows + 1, 0);
  for (int64_t i = 0; i < nrows; ++i) ptr[i + 1] = ptr[i] + len[i];
  adj.resize(ptr[nrows]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nrows; ++i)
    std::copy(tmp.begin() + start[i], tmp.begin() + start[i] + len[i], adj.begin() + ptr[i]);
}

// ------------------------------------------------------------ element data
// Dm = [X1-X0, X2-X0, X3-X0] (as columns); Vol = |det Dm| / 6 (Section 2.2).
bool element_data(const Input& in, Setup& s, std::string* err) {
  s.Dminv.assign(in.E * 9, 0.0);
  s.vol.assign(in.E, 0.0);
  bool ok = true;
  int64_t bad = -1;
#pragma omp parallel for reduction(&& : ok)
  for (int64_t e = 0; e < in.E; ++e) {
    const int32_t* t = in.tets + 4 * e;
    const double* x0 = in.X + 3 * t[0];
    double D[9];  // row-major, column c = X_{c+1} - X_0
    double h = 0;
    for (int c = 0; c < 3; ++c) {
      const double* xc = in.X + 3 * t[c + 1];
      for (int r = 0; r < 3; ++r) {
        D[3 * r + c] = xc[r] - x0[r];
        h = std::max(h, std::fabs(D[3 * r + c]));
      }
    }
    double c00 = D[4] * D[8] - D[5] * D[7], c01 = D[5] * D[6] - D[3] * D[8], c02 = D[3] * D[7] - D[4] * D[6];
    double det = D[0] * c00 + D[1] * c01 + D[2] * c02;
    if (!(std::fabs(det) > 1e-14 * h * h * h) || !std::isfinite(det)) {
      ok = false;
#pragma omp critical
      bad = e;
      continue;
    }
    double id = 1.0 / det, *Mi = &s.Dminv[9 * e];
    Mi[0] = c00 * id; Mi[1] = (D[2] * D[7] - D[1] * D[8]) * id; Mi[2] = (D[1] * D[5] - D[2] * D[4]) * id;
    Mi[3] = c01 * id; Mi[4] = (D[0] * D[8] - D[2] * D[6]) * id; Mi[5] = (D[2] * D[3] - D[0] * D[5]) * id;
    Mi[6] = c02 * id; Mi[7] = (D[1] * D[6] - D[0] * D[7]) * id; Mi[8] = (D[0] * D[4] - D[1] * D[3]) * id;
    s.vol[e] = std::fabs(det) / 6.0;
  }
  if (!ok) {
    *err = "degenerate rest tet " + std::to_string(bad);
    return false;
  }
  return true;
}

// G_e = S Dm^-1 (4x3): row 0 = -(sum of the rows of Dm^-1), rows 1..3 = rows of Dm^-1.
inline void shape_grad(const double* Mi, double G[4][3]) {
  for (int c = 0; c < 3; ++c) {
    G[1][c] = Mi[c]; G[2][c] = Mi[3 + c]; G[3][c] = Mi[6 + c];
    G[0][c] = -(Mi[c] + Mi[3 + c] + Mi[6 + c]);
  }
}

// ------------------------------------------------------------ nested dissection
// Geometric recursive bisection of the x_1 graph: split at the median of the
// longest bounding-box axis and take the smaller one-sided boundary as the
// vertex separator; order = [part A, part B, separator].
struct ND {
  const std::vector<int64_t>& ptr;
  const std::vector<int32_t>& adj;
  const std::vector<double>& xyz;  // [n1][3]
  std::vector<int8_t> side;
  std::vector<int32_t> order;
  ND(const std::vector<int64_t>& p, const std::vector<int32_t>& a, const std::vector<double>& c, int64_t n)
      : ptr(p), adj(a), xyz(c), side(n, -1) { order.reserve(n); }

  void run(std::vector<int32_t> v) {
    if (v.size() <= 48) {
      for (int32_t u : v) order.push_back(u);
      return;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int32_t u : v)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], xyz[3 * u + d]);
        hi[d] = std::max(hi[d], xyz[3 * u + d]);
      }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    size_t half = v.size() / 2;
    std::nth_element(v.begin(), v.begin() + half, v.end(), [&](int32_t a, int32_t b) {
      double ca = xyz[3 * a + ax], cb = xyz[3 * b + ax];
      return ca < cb || (ca == cb && a < b);
    });
    // move the median coordinate's equal values consistently: split by value
    double cut = xyz[3 * v[half] + ax];
    std::vector<int32_t> A, B;
    for (int32_t u : v) (xyz[3 * u + ax] < cut ? A : B).push_back(u);
    if (A.empty() || B.empty()) {  // all on one plane: fall back to rank split
      A.assign(v.begin(), v.begin() + half);
      B.assign(v.begin() + half, v.end());
    }
    for (int32_t u : A) side[u] = 0;
    for (int32_t u : B) side[u] = 1;
    std::vector<int32_t> bA, bB;
    for (int32_t u : A)
      for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q)
        if (side[adj[q]] == 1) { bA.push_back(u); break; }
    for (int32_t u : B)
      for (int64_t q = ptr[u]; q < ptr[u + 1]; ++q)
        if (side[adj[q]] == 0) { bB.push_back(u); break; }
    std::vector<int32_t>& sep = (bA.size() <= bB.size()) ? bA : bB;
    int8_t sepside = (bA.size() <= bB.size()) ? 0 : 1;
    for (int32_t u : sep) side[u] = 2;
    std::vector<int32_t> A2, B2;
    for (int32_t u : A) if (side[u] == 0) A2.push_back(u);
    for (int32_t u : B) if (side[u] == 1) B2.push_back(u);
    (void)sepside;
    for (int32_t u : v) side[u] = -1;
    std::vector<int32_t> sepc = sep;
    std::vector<int32_t>().swap(A);
    std::vector<int32_t>().swap(B);
    std::vector<int32_t>().swap(v);
    run(std::move(A2));
    run(std::move(B2));
    for (int32_t u : sepc) order.push_back(u);
  }
};

// ------------------------------------------------------------ dense kernels for fronts
// Column-major front F (ld), lower triangle.
bool potrf(double* F, int64_t ld, int64_t nc) {
  for (int64_t j = 0; j < nc; ++j) {
    double d = F[j + j * ld];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    d = std::sqrt(d);
    F[j + j * ld] = d;
    double id = 1.0 / d;
    for (int64_t i = j + 1; i < nc; ++i) F[i + j * ld] *= id;
    for (int64_t k = j + 1; k < nc; ++k) {
      double lkj = F[k + j * ld];
      if (lkj == 0.0) continue;
      double* Fk = F + k * ld;
      const double* Fj = F + j * ld;
      for (int64_t i = k; i < nc; ++i) Fk[i] -= Fj[i] * lkj;
    }
  }
  return true;
}

// rows nc..nf-1 of the first nc columns: F21 <- F21 L11^-T
void trsm(double* F, int64_t ld, int64_t nc, int64_t nr) {
  const int64_t CH = 256;
  int64_t nchunk = (nr + CH - 1) / CH;
#pragma omp parallel for schedule(dynamic) if (nr * nc * nc > 2000000)
  for (int64_t ch = 0; ch < nchunk; ++ch) {
    int64_t r0 = nc + ch * CH, r1 = std::min(nc + nr, r0 + CH);
    for (int64_t j = 0; j < nc; ++j) {
      double* cj = F + j * ld;
      for (int64_t k = 0; k < j; ++k) {
        double l = F[j + k * ld];
        if (l == 0.0) continue;
        const double* ck = F + k * ld;
        for (int64_t i = r0; i < r1; ++i) cj[i] -= ck[i] * l;
      }
      double id = 1.0 / F[j + j * ld];
      for (int64_t i = r0; i < r1; ++i) cj[i] *= id;
    }
  }
}

// F22 -= F21 F21^T (lower), F21 = rows nc.. of columns 0..nc-1.
void syrk(double* F, int64_t ld, int64_t nc, int64_t nr) {
  const int64_t TB = 64;
  int64_t nt = (nr + TB - 1) / TB;
  std::vector<std::pair<int64_t, int64_t>> tiles;
  for (int64_t tj = 0; tj < nt; ++tj)
    for (int64_t ti = tj; ti < nt; ++ti) tiles.push_back({ti, tj});
#pragma omp parallel for schedule(dynamic) if (nr * nr * nc > 4000000)
  for (size_t t = 0; t < tiles.size(); ++t) {
    int64_t i0 = nc + tiles[t].first * TB, j0 = nc + tiles[t].second * TB;
    int64_t i1 = std::min(nc + nr, i0 + TB), j1 = std::min(nc + nr, j0 + TB);
    for (int64_t j = j0; j < j1; j += 4) {
      int64_t jn = std::min<int64_t>(4, j1 - j);
      int64_t ilo = std::max(i0, j);
      if (ilo >= i1) continue;
      double acc[4][TB];
      for (int jj = 0; jj < 4; ++jj)
        for (int64_t i = 0; i < TB; ++i) acc[jj][i] = 0.0;
      for (int64_t k = 0; k < nc; ++k) {
        const double* ck = F + k * ld;
        double b0 = ck[j], b1 = jn > 1 ? ck[j + 1] : 0.0, b2 = jn > 2 ? ck[j + 2] : 0.0,
               b3 = jn > 3 ? ck[j + 3] : 0.0;
        if (b0 == 0.0 && b1 == 0.0 && b2 == 0.0 && b3 == 0.0) continue;
        const double* a = ck + ilo;
        int64_t len = i1 - ilo;
#pragma omp simd
        for (int64_t i = 0; i < len; ++i) {
          double ai = a[i];
          acc[0][i] += ai * b0; acc[1][i] += ai * b1; acc[2][i] += ai * b2; acc[3][i] += ai * b3;
        }
      }
      for (int64_t jj = 0; jj < jn; ++jj) {
        double* cj = F + (j + jj) * ld;
        for (int64_t i = std::max(ilo, j + jj); i < i1; ++i) cj[i] -= acc[jj][i - ilo];
      }
    }
  }
}

// In-place inverse of the lower-triangular nc x nc block (column-major, ld).
void trinv(double* L, int64_t ld, int64_t nc) {
  std::vector<double> inv(nc * nc, 0.0);
  for (int64_t j = 0; j < nc; ++j) {
    // solve L z = e_j for rows >= j
    double* z = &inv[j * nc];
    z[j] = 1.0 / L[j + j * ld];
    for (int64_t i = j + 1; i < nc; ++i) {
      double sum = 0.0;
      for (int64_t k = j; k < i; ++k) sum += L[i + k * ld] * z[k];
      z[i] = -sum / L[i + i * ld];
    }
  }
  for (int64_t j = 0; j < nc; ++j)
    for (int64_t i = j; i < nc; ++i) L[i + j * ld] = inv[i + j * nc];
}

}  // namespace

// The numeric phase on the host: multifrontal partial Cholesky with x_2 never
// pivoted (Eq. 9), L (diagonal blocks inverted) into s.Lval and Sigma_0.
int numeric_phase(Setup& s, LowerCSC& A, double& t_num, std::string* err) {
  const int64_t n1 = s.n1, m = s.m, nf = n1 + m, nsn = s.nsn;
  try {
    s.Lval.assign(s.nnzL, 0.0);
  } catch (...) {
    *err = "host allocation of the interior factor failed";
    return ST_OOM;
  }
  // ---- numeric: multifrontal partial Cholesky, x_2 never pivoted (Eq. 9)
  std::vector<double> Sig((size_t)m * m, 0.0);   // Sigma_alpha, column-major = row-major (symmetric)
  for (int64_t j = n1; j < nf; ++j)
    for (int64_t q = A.colptr[j]; q < A.colptr[j + 1]; ++q) {
      int64_t i = A.row[q];
      Sig[(i - n1) + (j - n1) * m] += A.val[q];
      if (i != j) Sig[(j - n1) + (i - n1) * m] += A.val[q];
    }
  struct Upd { int32_t sn; std::vector<double> U; };
  std::vector<Upd> stack;
  std::vector<int32_t> loc(nf, -1);
  double flops = 0.0;
  for (int64_t k = 0; k < nsn; ++k) {
    const int64_t c0 = s.sn_col0[k], nc = s.sn_col0[k + 1] - c0;
    const int64_t nr = s.sn_rowptr[k + 1] - s.sn_rowptr[k];
    const int32_t* R = &s.rows[s.sn_rowptr[k]];
    const int64_t fsz = nc + nr;
    std::vector<double> F;
    try { F.assign(fsz * fsz, 0.0); } catch (...) { *err = "host allocation of a front failed"; return ST_OOM; }
    for (int64_t c = 0; c < nc; ++c) loc[c0 + c] = (int32_t)c;
    for (int64_t r = 0; r < nr; ++r) loc[R[r]] = (int32_t)(nc + r);
    for (int64_t c = 0; c < nc; ++c) {
      int64_t j = c0 + c;
      for (int64_t q = A.colptr[j]; q < A.colptr[j + 1]; ++q) F[loc[A.row[q]] + c * fsz] += A.val[q];
    }
    // extend-add the children's update matrices (top of the stack)
    while (!stack.empty() && s.sn_parent[stack.back().sn] == k) {
      Upd& u = stack.back();
      int64_t cn = s.sn_rowptr[u.sn + 1] - s.sn_rowptr[u.sn];
      const int32_t* CR = &s.rows[s.sn_rowptr[u.sn]];
      for (int64_t b = 0; b < cn; ++b) {
        int64_t lb = loc[CR[b]];
        double* Fc = &F[lb * fsz];
        const double* Uc = &u.U[b * cn];
        for (int64_t a = b; a < cn; ++a) Fc[loc[CR[a]]] += Uc[a];
      }
      stack.pop_back();
    }
    if (!potrf(F.data(), fsz, nc)) {
      *err = "interior matrix is not positive definite (a free part without a Dirichlet node?)";
      return ST_NOT_SPD;
    }
    trsm(F.data(), fsz, nc, nr);
    syrk(F.data(), fsz, nc, nr);
    flops += nc * nc * nc / 3.0 + (double)nr * nc * nc + (double)nr * nr * nc;
    double* P = &s.Lval[s.sn_valptr[k]];
    for (int64_t c = 0; c < nc; ++c) std::memcpy(P + c * fsz, &F[c * fsz], sizeof(double) * fsz);
    trinv(P, fsz, nc);
    if (nr > 0) {
      if (s.sn_parent[k] >= 0) {
        Upd u;
        u.sn = (int32_t)k;
        u.U.resize(nr * nr);
        for (int64_t b = 0; b < nr; ++b)
          for (int64_t a = b; a < nr; ++a) u.U[a + b * nr] = F[(nc + a) + (nc + b) * fsz];
        stack.push_back(std::move(u));
      } else {
        // every remaining row is in x_2: add into Sigma_alpha (both triangles)
        for (int64_t b = 0; b < nr; ++b) {
          int64_t gb = R[b] - n1;
          for (int64_t a = b; a < nr; ++a) {
            int64_t ga = R[a] - n1;
            double v = F[(nc + a) + (nc + b) * fsz];
            Sig[ga + gb * m] += v;
            if (ga != gb) Sig[gb + ga * m] += v;
          }
        }
      }
    }
    for (int64_t c = 0; c < nc; ++c) loc[c0 + c] = -1;
    for (int64_t r = 0; r < nr; ++r) loc[R[r]] = -1;
  }
  s.factor_flops = flops;
  t_num = now_ms();

  // Sigma_0 = Sigma_alpha + A22^beta (+ M_2/dt^2)
  s.Sigma0.swap(Sig);
  for (int64_t j = 0; j < m; ++j)
    for (int64_t q = s.B22.colptr[j]; q < s.B22.colptr[j + 1]; ++q)
      s.Sigma0[s.B22.row[q] + j * m] += s.B22.val[q];
  A = LowerCSC();   // not needed once Sigma_0 and L are formed
  return 0;
}


int build(const Input& in, Setup& s, std::string* err) {
  double t0 = now_ms();
  const int64_t n = in.n, E = in.E, m = in.m;
  if (n < 1 || E < 1 || !in.X || !in.tets || !(in.mu > 0) || in.dt < 0 || !std::isfinite(in.mu) ||
      !(in.mu_prime >= 0) || !std::isfinite(in.mu_prime) || !(in.kappa >= 0) || !std::isfinite(in.kappa)) {
    *err = "invalid mesh or material";
    return ST_INVALID;
  }
  for (int64_t i = 0; i < 4 * E; ++i)
    if (in.tets[i] < 0 || in.tets[i] >= n) {
      *err = "tet node id out of range";
      return ST_BAD_MESH;
    }
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* t = in.tets + 4 * e;
    if (t[0] == t[1] || t[0] == t[2] || t[0] == t[3] || t[1] == t[2] || t[1] == t[3] || t[2] == t[3]) {
      *err = "tet with repeated node";
      return ST_BAD_MESH;
    }
  }
  if (m < 1 || m > 16384 || !in.region) {
    *err = "region size must be in [1, 16384]";
    return ST_REGION;
  }
  if (in.dt > 0 && !(in.density > 0)) {
    *err = "backward Euler needs a positive density";
    return ST_INVALID;
  }
  s.n = n; s.m = m;
  // node classes: 0 = x_1, 1 = x_2, 2 = Dirichlet
  std::vector<int8_t> cls(n, 0);
  for (int64_t i = 0; i < in.nd; ++i) {
    int32_t v = in.dirichlet[i];
    if (v < 0 || v >= n) { *err = "Dirichlet node id out of range"; return ST_INVALID; }
    if (cls[v] == 2) { *err = "repeated Dirichlet node"; return ST_INVALID; }
    cls[v] = 2;
  }
  for (int64_t i = 0; i < m; ++i) {
    int32_t v = in.region[i];
    if (v < 0 || v >= n) { *err = "region node id out of range"; return ST_REGION; }
    if (cls[v] == 2) { *err = "region overlaps the Dirichlet set"; return ST_REGION; }
    if (cls[v] == 1) { *err = "repeated region node"; return ST_REGION; }
    cls[v] = 1;
  }
  if (!element_data(in, s, err)) return ST_BAD_MESH;

  // E_beta: tets with all four vertices in x_2 (Figure 2); E_alpha: the rest.
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* t = in.tets + 4 * e;
    bool b = cls[t[0]] == 1 && cls[t[1]] == 1 && cls[t[2]] == 1 && cls[t[3]] == 1;
    (b ? s.beta : s.alpha).push_back((int32_t)e);
  }
  if (in.dt > 0) {
    s.mass.assign(n, 0.0);
    for (int64_t e = 0; e < E; ++e)
      for (int a = 0; a < 4; ++a) s.mass[in.tets[4 * e + a]] += in.density * s.vol[e] / 4.0;
  }

  // ---- x_1 graph and nested-dissection ordering
  std::vector<int32_t> tid(n, -1), x1nodes;
  for (int64_t v = 0; v < n; ++v)
    if (cls[v] == 0) { tid[v] = (int32_t)x1nodes.size(); x1nodes.push_back((int32_t)v); }
  const int64_t n1 = (int64_t)x1nodes.size();
  s.n1 = n1;
  s.nfree = n1 + m;
  std::vector<int64_t> gptr;
  std::vector<int32_t> gadj;
  pattern_rows(n1, [&](auto f) {
    for (int32_t e : s.alpha) {
      const int32_t* t = in.tets + 4 * e;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          if (a != b && cls[t[a]] == 0 && cls[t[b]] == 0) f(tid[t[a]], tid[t[b]]);
    }
  }, gptr, gadj);
  std::vector<int32_t> ndorder;
  {
    std::vector<double> xyz(3 * n1);
    for (int64_t i = 0; i < n1; ++i)
      for (int d = 0; d < 3; ++d) xyz[3 * i + d] = in.X[3 * x1nodes[i] + d];
    ND nd(gptr, gadj, xyz, n1);
    std::vector<int32_t> all(n1);
    std::iota(all.begin(), all.end(), 0);
    nd.run(std::move(all));
    ndorder.swap(nd.order);
  }
  double t_nd = now_ms();

  // ---- positions before postordering: x_1 by ND rank, x_2 by region index
  std::vector<int32_t> rank(n1);
  for (int64_t k = 0; k < n1; ++k) rank[ndorder[k]] = (int32_t)k;
  // adjacency of x_1 columns (by rank) including x_2 neighbours (as n1 + idx)
  std::vector<int32_t> ridx(n, -1);
  for (int64_t i = 0; i < m; ++i) ridx[in.region[i]] = (int32_t)i;
  auto build_adj = [&](const std::vector<int32_t>& posx1, std::vector<int64_t>& ptr, std::vector<int32_t>& adj) {
    pattern_rows(n1, [&](auto f) {
      for (int32_t e : s.alpha) {
        const int32_t* t = in.tets + 4 * e;
        for (int a = 0; a < 4; ++a) {
          if (cls[t[a]] != 0) continue;
          const int64_t pa = posx1[tid[t[a]]];
          for (int b = 0; b < 4; ++b) {
            if (a == b || cls[t[b]] == 2) continue;
            f(pa, cls[t[b]] == 0 ? (int64_t)posx1[tid[t[b]]] : n1 + ridx[t[b]]);
          }
        }
      }
    }, ptr, adj);
  };
  // elimination tree (Liu) with all of x_2 contracted to one root
  auto etree = [&](const std::vector<int64_t>& ptr, const std::vector<int32_t>& adj) {
    std::vector<int32_t> parent(n1, -1), anc(n1, -1);
    for (int64_t j = 0; j < n1; ++j) {
      for (int64_t q = ptr[j]; q < ptr[j + 1]; ++q) {
        int64_t i = adj[q];
        if (i >= j) continue;  // neighbours before j (row j of the lower part)
        int64_t r = i;
        while (anc[r] != -1 && anc[r] != j) {
          int64_t t = anc[r];
          anc[r] = (int32_t)j;
          r = t;
        }
        if (anc[r] == -1) { anc[r] = (int32_t)j; parent[r] = (int32_t)j; }
      }
    }
    return parent;
  };
  std::vector<int32_t> pos1 = rank;
  std::vector<int64_t> aptr;
  std::vector<int32_t> aadj;
  build_adj(pos1, aptr, aadj);
  std::vector<int32_t> parent = etree(aptr, aadj);
  // postorder of the x_1 forest
  {
    std::vector<int32_t> head(n1, -1), next(n1, -1), post;
    post.reserve(n1);
    for (int64_t j = n1 - 1; j >= 0; --j)
      if (parent[j] >= 0) { next[j] = head[parent[j]]; head[parent[j]] = (int32_t)j; }
    std::vector<int32_t> stack;
    for (int64_t r = 0; r < n1; ++r) {
      if (parent[r] != -1) continue;
      stack.push_back((int32_t)r);
      while (!stack.empty()) {
        int32_t p = stack.back();
        int32_t c = head[p];
        if (c == -1) { post.push_back(p); stack.pop_back(); }
        else { head[p] = next[c]; stack.push_back(c); }
      }
    }
    std::vector<int32_t> newpos(n1);
    for (int64_t k = 0; k < n1; ++k) newpos[post[k]] = (int32_t)k;
    std::vector<int32_t> np(n1, -1);
    for (int64_t k = 0; k < n1; ++k) np[k] = parent[post[k]] < 0 ? -1 : newpos[parent[post[k]]];
    parent.swap(np);
    for (int64_t i = 0; i < n1; ++i) pos1[i] = newpos[rank[i]];
  }
  s.pos.assign(n, -1);
  s.node_of_pos.assign(n1 + m, -1);
  for (int64_t i = 0; i < n1; ++i) { s.pos[x1nodes[i]] = pos1[i]; s.node_of_pos[pos1[i]] = x1nodes[i]; }
  for (int64_t i = 0; i < m; ++i) { s.pos[in.region[i]] = (int32_t)(n1 + i); s.node_of_pos[n1 + i] = in.region[i]; }
  build_adj(pos1, aptr, aadj);  // adjacency in final positions

  // ---- assemble the alpha matrix (lower, final positions) and B22 = A22^beta (+ M2/dt^2)
  const int64_t nf = n1 + m;
  LowerCSC& A = s.A;
  {
    // entries (row pa >= column pb) bucketed by column in element order, then
    // each column sorted by row, stably so that duplicates are summed in
    // element order, and compacted; columns in parallel
    auto each = [&](auto f) {
      for (int32_t e : s.alpha) {
        const int32_t* t = in.tets + 4 * e;
        double G[4][3];
        shape_grad(&s.Dminv[9 * e], G);
        const double w = 2.0 * (in.mu + in.mu_prime + in.kappa) * s.vol[e];
        for (int a = 0; a < 4; ++a) {
          const int64_t pa = s.pos[t[a]];
          if (pa < 0) continue;
          for (int b = 0; b < 4; ++b) {
            const int64_t pb = s.pos[t[b]];
            if (pb < 0 || pb > pa) continue;
            f(pb, pa, w * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]));
          }
        }
      }
      if (in.dt > 0)
        for (int64_t i = 0; i < n1; ++i) f(pos1[i], pos1[i], s.mass[x1nodes[i]] / (in.dt * in.dt));
    };
    std::vector<int64_t> start(nf + 1, 0);
    each([&](int64_t c, int64_t, double) { ++start[c + 1]; });
    for (int64_t j = 0; j < nf; ++j) start[j + 1] += start[j];
    std::vector<std::pair<int32_t, double>> ent(start[nf]);
    std::vector<int64_t> cur(start.begin(), start.end() - 1);
    each([&](int64_t c, int64_t r, double v) { ent[cur[c]++] = {(int32_t)r, v}; });
    std::vector<int64_t> len(nf);
#pragma omp parallel for schedule(dynamic, 512)
    for (int64_t j = 0; j < nf; ++j) {
      const auto b = ent.begin() + start[j], e = ent.begin() + start[j + 1];
      std::stable_sort(b, e, [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
        return x.first < y.first;
      });
      int64_t k = 0;
      for (auto q = b; q != e; ++q) {
        if (k > 0 && b[k - 1].first == q->first) b[k - 1].second += q->second;
        else b[k++] = *q;
      }
      len[j] = k;
    }
    A.n = nf;
    A.colptr.assign(nf + 1, 0);
    for (int64_t j = 0; j < nf; ++j) A.colptr[j + 1] = A.colptr[j] + len[j];
    A.row.resize(A.colptr[nf]);
    A.val.resize(A.colptr[nf]);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nf; ++j)
      for (int64_t k = 0; k < len[j]; ++k) {
        A.row[A.colptr[j] + k] = ent[start[j] + k].first;
        A.val[A.colptr[j] + k] = ent[start[j] + k].second;
      }
  }
  {
    std::vector<std::pair<int64_t, double>> trip;
    for (int32_t e : s.beta) {
      const int32_t* t = in.tets + 4 * e;
      double G[4][3];
      shape_grad(&s.Dminv[9 * e], G);
      double w = 2.0 * (in.mu + in.mu_prime + in.kappa) * s.vol[e];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          double v = w * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
          trip.push_back({(int64_t)ridx[t[b]] * m + ridx[t[a]], v});
        }
    }
    if (in.dt > 0)
      for (int64_t i = 0; i < m; ++i) trip.push_back({i * m + i, s.mass[in.region[i]] / (in.dt * in.dt)});
    std::sort(trip.begin(), trip.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    LowerCSC& B = s.B22;
    B.n = m;
    B.colptr.assign(m + 1, 0);
    for (size_t q = 0; q < trip.size();) {
      size_t r = q;
      double v = 0.0;
      while (r < trip.size() && trip[r].first == trip[q].first) v += trip[r++].second;
      B.row.push_back((int32_t)(trip[q].first % m));
      B.val.push_back(v);
      B.colptr[trip[q].first / m + 1]++;
      q = r;
    }
    for (int64_t j = 0; j < m; ++j) B.colptr[j + 1] += B.colptr[j];
  }
  double t_asm = now_ms();

  // ---- symbolic: column structures (rows > j), supernodes with relaxed merging
  std::vector<std::vector<int32_t>> cstruct(n1);
  std::vector<int32_t> chead(n1, -1), cnext(n1, -1);
  for (int64_t j = n1 - 1; j >= 0; --j)
    if (parent[j] >= 0) { cnext[j] = chead[parent[j]]; chead[parent[j]] = (int32_t)j; }
  {
    // struct(j) = (rows of A's column j below j) U (struct(c) \ {j} for the
    // children c of j): sorted lists merged, no sort
    std::vector<int32_t> buf;
    for (int64_t j = 0; j < n1; ++j) {
      std::vector<int32_t>& st = cstruct[j];
      for (int64_t q = A.colptr[j]; q < A.colptr[j + 1]; ++q)   // rows ascend within a column
        if (A.row[q] > j) st.push_back(A.row[q]);
      for (int32_t c = chead[j]; c != -1; c = cnext[c]) {
        const std::vector<int32_t>& cs = cstruct[c];
        buf.clear();
        std::set_union(st.begin(), st.end(), std::upper_bound(cs.begin(), cs.end(), (int32_t)j), cs.end(),
                       std::back_inserter(buf));
        st.swap(buf);
      }
    }
  }
  std::vector<int64_t> cnt(n1);
  for (int64_t j = 0; j < n1; ++j) cnt[j] = (int64_t)cstruct[j].size();
  s.sn_col0.clear();
  std::vector<int32_t> col2sn(n1, -1);
  {
    int64_t j = 0;
    while (j < n1) {
      int64_t j0 = j;
      while (j + 1 < n1 && parent[j] == j + 1) {
        int64_t zeros = cnt[j + 1] + 1 - cnt[j];
        int64_t width = j - j0 + 1;
        bool fundamental = zeros == 0 && width < 1024;
        bool relaxed = zeros <= 4 + cnt[j] / 4 && width < 256;
        if (!(fundamental || relaxed)) break;
        ++j;
      }
      int32_t sid = (int32_t)s.sn_col0.size();
      s.sn_col0.push_back((int32_t)j0);
      for (int64_t c = j0; c <= j; ++c) col2sn[c] = sid;
      ++j;
    }
    s.nsn = (int64_t)s.sn_col0.size();
    s.sn_col0.push_back((int32_t)n1);
  }
  const int64_t nsn = s.nsn;
  s.sn_rowptr.assign(nsn + 1, 0);
  s.sn_valptr.assign(nsn + 1, 0);
  s.sn_parent.assign(nsn, -1);
  s.sn_level.assign(nsn, 0);
  for (int64_t k = 0; k < nsn; ++k) {
    int64_t j1 = s.sn_col0[k + 1] - 1;
    int64_t nc = s.sn_col0[k + 1] - s.sn_col0[k];
    int64_t nr = (int64_t)cstruct[j1].size();
    s.sn_rowptr[k + 1] = s.sn_rowptr[k] + nr;
    s.sn_valptr[k + 1] = s.sn_valptr[k] + (nc + nr) * nc;
    s.sn_parent[k] = parent[j1] < 0 ? -1 : col2sn[parent[j1]];
  }
  s.rows.resize(s.sn_rowptr[nsn]);
  for (int64_t k = 0; k < nsn; ++k) {
    int64_t j1 = s.sn_col0[k + 1] - 1;
    std::copy(cstruct[j1].begin(), cstruct[j1].end(), s.rows.begin() + s.sn_rowptr[k]);
  }
  std::vector<std::vector<int32_t>>().swap(cstruct);
  for (int64_t k = 0; k < nsn; ++k)
    if (s.sn_parent[k] >= 0) s.sn_level[s.sn_parent[k]] = std::max(s.sn_level[s.sn_parent[k]], s.sn_level[k] + 1);
  s.nlevels = 0;
  for (int64_t k = 0; k < nsn; ++k) s.nlevels = std::max<int64_t>(s.nlevels, s.sn_level[k] + 1);
  s.nnzL = s.sn_valptr[nsn];
  double t_sym = now_ms();

  double t_num = t_sym;
  if (in.numeric) {
    int st = numeric_phase(s, A, t_num, err);
    if (st) return st;
  }

  // ---- gather maps
  auto build_gather = [](int64_t ntarget, const std::vector<int32_t>& elems, const int32_t* tets,
                         auto target_of, std::vector<int64_t>& ptr, std::vector<int32_t>& slot) {
    ptr.assign(ntarget + 1, 0);
    for (size_t e = 0; e < elems.size(); ++e)
      for (int a = 0; a < 4; ++a) {
        int64_t t = target_of(tets[4 * elems[e] + a]);
        if (t >= 0) ptr[t + 1]++;
      }
    for (int64_t i = 0; i < ntarget; ++i) ptr[i + 1] += ptr[i];
    slot.resize(ptr[ntarget]);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (size_t e = 0; e < elems.size(); ++e)
      for (int a = 0; a < 4; ++a) {
        int64_t t = target_of(tets[4 * elems[e] + a]);
        if (t >= 0) slot[fill[t]++] = (int32_t)(4 * e + a);
      }
  };
  build_gather(nf, s.alpha, in.tets, [&](int32_t v) -> int64_t { return s.pos[v]; }, s.ga_ptr, s.ga_slot);
  build_gather(m, s.beta, in.tets, [&](int32_t v) -> int64_t { return ridx[v]; }, s.gb_ptr, s.gb_slot);
  std::vector<int32_t> alle(E);
  std::iota(alle.begin(), alle.end(), 0);
  build_gather(n, alle, in.tets, [](int32_t v) -> int64_t { return v; }, s.gall_ptr, s.gall_slot);

  s.ms_total = now_ms() - t0;
  char buf[512];
  snprintf(buf, sizeof buf,
           "n=%lld n1=%lld m=%lld alpha=%zu beta=%zu supernodes=%lld levels=%lld nnzL=%lld "
           "flops=%.3g | nd %.0f ms, assemble %.0f ms, symbolic %.0f ms, numeric %.0f ms, total %.0f ms",
           (long long)n, (long long)n1, (long long)m, s.alpha.size(), s.beta.size(), (long long)nsn,
           (long long)s.nlevels, (long long)s.nnzL, s.factor_flops, t_nd - t0, t_asm - t_nd, t_sym - t_asm,
           t_num - t_sym, s.ms_total);
  s.log = buf;
  return 0;
}

}  // namespace pdh
