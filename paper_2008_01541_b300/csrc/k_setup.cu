// Numeric phase of the setup on the device (see setup_dev.h): multifrontal
// partial Cholesky of the constant PD matrix, Section 3.1 Eq. 9, in FP64.
//
// The host's symbolic analysis gives the supernodes (nc fully-summed columns,
// nr off-diagonal rows each, rows sorted), their elimination tree and its
// levels (height above the leaves).  Every supernode owns a dense front of
// order nc + nr in one device arena.  Level by level from the leaves:
//   1. extend-add: each front adds its children's update matrices (the
//      trailing nr x nr blocks of the children's fronts), one child per
//      parent per pass, so no two writes meet and the sums are deterministic;
//   2. factor: the nc fully-summed columns are eliminated and the trailing
//      block updated (potrf, trsm and syrk of the front), by one CTA in
//      shared memory for fronts of order <= kSmallFront, else by the blocked
//      FP64 tile Cholesky of the dense collision block (a partial
//      factorisation of the front padded to 64-multiples with identity);
//      the factor panel goes to L as L_ss^-1 over L_rs L_ss^-1, so that
//      both triangular solves apply each supernode in one step;
//   3. the update of a front whose parent is x_2 itself (every row in x_2)
//      is added into Sigma_0, one front per launch in supernode order.
// Sigma_0 starts as A_22 of the alpha elements and receives A_22 of the beta
// elements (and M_2 / dt^2) last, the order of the host's factorisation.
#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "setup_dev.h"

namespace pdk {
namespace {

constexpr int TBS = 64;            // tile of the FP64 dense factor
constexpr int kSmallFront = 128;   // fronts up to this order: one CTA, shared memory

struct Front {
  int64_t off;      // first element in the arena
  int64_t valptr;   // first element of the panel in L
  int64_t rowptr;   // first off-diagonal row in rows / relind
  int32_t ld;       // leading dimension (order, padded to 64-multiples for large fronts)
  int32_t nc;       // fully-summed columns
  int32_t ncp;      // local index of the first off-diagonal row (nc, or nc rounded up to 64)
  int32_t nr;       // off-diagonal rows
};

// base[dst[i]] += val[i] (the positions of one list are distinct)
__global__ void k_scatter_add(const int64_t* __restrict__ dst, const double* __restrict__ val, int64_t n,
                              double* __restrict__ base) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) base[dst[i]] += val[i];
}

// One extend-add task: columns b0 .. b0 + nb - 1 of child u's update matrix
// into its parent's front (relind: the child's rows as local indices of the
// parent's front).
struct EaTask {
  int32_t u, p, b0, nb;
};
__global__ void __launch_bounds__(256) k_extend_add(const EaTask* __restrict__ tasks, const Front* __restrict__ fr,
                                                    const int32_t* __restrict__ relind, double* __restrict__ arena) {
  const EaTask t = tasks[blockIdx.x];
  const Front cu = fr[t.u], cp = fr[t.p];
  const int32_t* ri = relind + cu.rowptr;
  const double* U = arena + cu.off + (int64_t)cu.ncp * cu.ld + cu.ncp;   // U[a + b * ld]
  double* F = arena + cp.off;
  for (int b = t.b0; b < t.b0 + t.nb; ++b) {
    const int64_t pb = (int64_t)ri[b] * cp.ld;
    for (int a = b + (int)threadIdx.x; a < cu.nr; a += blockDim.x) F[ri[a] + pb] += U[a + (int64_t)b * cu.ld];
  }
}

// The update matrix of a front whose rows all lie in x_2 into Sigma_0 (both
// triangles): columns b0 .. b0 + nb - 1 per CTA.
__global__ void __launch_bounds__(256) k_sigma_add(Front f, int b0all, const int32_t* __restrict__ rows, int64_t n1,
                                                   const double* __restrict__ arena, double* __restrict__ S, int64_t m,
                                                   int nbcta) {
  const int b0 = b0all + blockIdx.x * nbcta;
  const int32_t* R = rows + f.rowptr;
  const double* U = arena + f.off + (int64_t)f.ncp * f.ld + f.ncp;
  for (int b = b0; b < min(b0 + nbcta, f.nr); ++b) {
    const int64_t gb = R[b] - n1;
    for (int a = b + (int)threadIdx.x; a < f.nr; a += blockDim.x) {
      const int64_t ga = R[a] - n1;
      const double v = U[a + (int64_t)b * f.ld];
      S[ga + gb * m] += v;
      if (a != b) S[gb + ga * m] += v;
    }
  }
}

// One small front per CTA, in shared memory (order n = nc + nr <=
// kSmallFront): right-looking elimination of the nc fully-summed columns
// (the trailing block receives the syrk update in the same sweep), then
// X = L_ss^-1 by forward substitution, one column per thread (X[i][c], i > c,
// kept in the front's free upper triangle), then the panel to L and the
// update matrix back to the arena.
__global__ void __launch_bounds__(256) k_front_small(const int32_t* __restrict__ list, const Front* __restrict__ fr,
                                                     double* __restrict__ arena, double* __restrict__ L,
                                                     int* __restrict__ status) {
  extern __shared__ double F[];   // [n][n] column-major
  __shared__ double dinv[kSmallFront];
  const int tid = threadIdx.x;
  const Front f = fr[list[blockIdx.x]];
  const int n = f.ld, nc = f.nc;
  double* G = arena + f.off;
  for (int i = tid; i < n * n; i += blockDim.x) F[i] = G[i];
  __syncthreads();
  for (int j = 0; j < nc; ++j) {
    double d = F[j + j * n];
    if (!(d > 0.0)) {   // not positive definite: reported, and 1 taken so the sweep stays finite
      if (tid == 0) atomicCAS(status, 0, 1);
      d = 1.0;
    }
    const double sq = sqrt(d), rs = 1.0 / sq;
    __syncthreads();   // every thread has read F[j][j]
    if (tid == 0) F[j + j * n] = sq;
    for (int i = j + 1 + tid; i < n; i += blockDim.x) F[i + j * n] *= rs;
    __syncthreads();
    const int w = n - j - 1;
    for (int idx = tid; idx < w * w; idx += blockDim.x) {
      const int c = j + 1 + idx / w, i = j + 1 + idx % w;
      if (i >= c) F[i + c * n] = fma(-F[i + j * n], F[c + j * n], F[i + c * n]);
    }
    __syncthreads();
  }
  for (int c = tid; c < nc; c += blockDim.x) dinv[c] = 1.0 / F[c + c * n];
  __syncthreads();
  for (int c = tid; c < nc; c += blockDim.x) {
    for (int i = c + 1; i < nc; ++i) {   // x_i = -(sum_{c <= k < i} L_ik x_k) / L_ii
      double t = F[i + c * n] * dinv[c];
      for (int k = c + 1; k < i; ++k) t = fma(F[i + k * n], F[c + k * n], t);
      F[c + i * n] = -t * dinv[i];
    }
  }
  __syncthreads();
  double* P = L + f.valptr;   // P[c * n + r]
  for (int idx = tid; idx < n * nc; idx += blockDim.x) {
    const int c = idx / n, r = idx % n;
    double v;
    if (r < nc) {
      v = r < c ? 0.0 : r == c ? dinv[c] : F[c + r * n];
    } else {   // (L_rs L_ss^-1)[r][c] = sum_{c <= k < nc} L_rk X_kc
      v = F[r + c * n] * dinv[c];
      for (int k = c + 1; k < nc; ++k) v = fma(F[r + k * n], F[c + k * n], v);
    }
    P[idx] = v;
  }
  for (int idx = tid; idx < f.nr * f.nr; idx += blockDim.x) {
    const int c = nc + idx / f.nr, i = nc + idx % f.nr;
    if (i >= c) G[i + c * n] = F[i + c * n];
  }
}

// Block row i of X = L_ss^-1 for a large front (tiles of 64; ncp = T * 64):
// X_ii = Z_ii (the diagonal tile inverses of the dense factor), and for
// j < i, X_ij = -Z_ii sum_{j <= t < i} L_it X_tj.  CTA j; each thread owns a
// 4 x 4 block of the 64 x 64 result.
__global__ void __launch_bounds__(256) k_binv_row(const double* __restrict__ F, int ld, const double* __restrict__ Linv,
                                                  double* __restrict__ X, int ncp, int i) {
  extern __shared__ double sm[];
  double* As = sm;                 // [64][65]: As[k * 65 + r] = left operand (r, k)
  double* Bs = sm + 64 * 65;       // [64][65]: Bs[c * 65 + k] = right operand (k, c)
  const int tid = threadIdx.x, j = blockIdx.x, r0 = 4 * (tid & 15), c0 = 4 * (tid >> 4);
  const double* Z = Linv + (int64_t)i * TBS * TBS;   // Z[c * 64 + r]
  double* Xij = X + (int64_t)TBS * i + (int64_t)TBS * j * ncp;
  if (j == i) {
    for (int idx = tid; idx < TBS * TBS; idx += blockDim.x) Xij[(idx & 63) + (int64_t)(idx >> 6) * ncp] = Z[idx];
    return;
  }
  double acc[4][4] = {};
  for (int t = j; t < i; ++t) {
    const double* Lit = F + (int64_t)TBS * i + (int64_t)TBS * t * ld;
    const double* Xtj = X + (int64_t)TBS * t + (int64_t)TBS * j * ncp;
    for (int idx = tid; idx < TBS * TBS; idx += blockDim.x) {
      const int r = idx & 63, k = idx >> 6;
      As[k * 65 + r] = Lit[r + (int64_t)k * ld];
      Bs[k * 65 + r] = Xtj[r + (int64_t)k * ncp];   // column k of X_tj: Bs[c * 65 + k'] with c = k, k' = r
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < TBS; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[k * 65 + r0 + q]; b[q] = Bs[(c0 + q) * 65 + k]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  // X_ij = -Z_ii acc: Z into As, acc into Bs
  for (int idx = tid; idx < TBS * TBS; idx += blockDim.x) As[(idx >> 6) * 65 + (idx & 63)] = Z[idx];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) Bs[(c0 + q) * 65 + r0 + p] = acc[p][q];
  __syncthreads();
  double out[4][4] = {};
#pragma unroll 4
  for (int k = 0; k < TBS; ++k) {
    double a[4], b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { a[q] = As[k * 65 + r0 + q]; b[q] = Bs[(c0 + q) * 65 + k]; }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) out[p][q] = fma(a[p], b[q], out[p][q]);
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) Xij[(r0 + p) + (int64_t)(c0 + q) * ncp] = -out[p][q];
}

// The diagonal block of a large front's panel in L: X = L_ss^-1, zero above
// the diagonal.
__global__ void k_extract_big(Front f, const double* __restrict__ X, double* __restrict__ L) {
  const int n = f.nc + f.nr;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)f.nc * f.nc) return;
  const int c = (int)(idx / f.nc), r = (int)(idx % f.nc);
  L[f.valptr + (int64_t)c * n + r] = r < c ? 0.0 : X[r + (int64_t)c * f.ncp];
}

// The off-diagonal rows of a large front's panel in L: M = L_rs X with
// X = L_ss^-1 (lower, ncp x ncp), by 64 x 64 tiles: CTA (ri, cj) forms rows
// 64 ri .. + 63 and columns 64 cj .. + 63 of M from the tiles t >= cj.
__global__ void __launch_bounds__(256) k_lrs_x(Front f, const double* __restrict__ F, const double* __restrict__ X,
                                               double* __restrict__ L) {
  extern __shared__ double sm[];
  double* As = sm;             // As[k * 65 + r] = L_rs (64 ri + r, 64 t + k)
  double* Bs = sm + 64 * 65;   // Bs[c * 65 + k] = X (64 t + k, 64 cj + c)
  const int tid = threadIdx.x, ri = blockIdx.x, cj = blockIdx.y, r0 = 4 * (tid & 15), c0 = 4 * (tid >> 4);
  const int T = f.ncp / TBS;
  double acc[4][4] = {};
  for (int t = cj; t < T; ++t) {
    for (int idx = tid; idx < TBS * TBS; idx += blockDim.x) {
      const int r = idx & 63, k = idx >> 6;
      As[k * 65 + r] = F[(f.ncp + TBS * ri + r) + (int64_t)(TBS * t + k) * f.ld];
      Bs[k * 65 + r] = X[(TBS * t + r) + (int64_t)(TBS * cj + k) * f.ncp];
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < TBS; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[k * 65 + r0 + q]; b[q] = Bs[(c0 + q) * 65 + k]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  const int n = f.nc + f.nr;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = TBS * ri + r0 + p, c = TBS * cj + c0 + q;
      if (r < f.nr && c < f.nc) L[f.valptr + (int64_t)c * n + f.nc + r] = acc[p][q];
    }
}

inline int64_t round64(int64_t x) { return (x + TBS - 1) / TBS * TBS; }

// device buffer owned for the duration of numeric_factor
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  template <class T>
  bool alloc(size_t n) { return cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1)) == cudaSuccess; }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
  template <class T>
  bool upload(const std::vector<T>& v, cudaStream_t st) {
    if (!alloc<T>(v.size())) return false;
    return v.empty() || cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st) == cudaSuccess;
  }
};

}  // namespace

int numeric_factor(const pdh::Setup& s, double* Lval, double* Sigma0, cudaStream_t st, std::string* err) {
  const int64_t n1 = s.n1, m = s.m, nsn = s.nsn;
  const pdh::LowerCSC& A = s.A;
  if ((int64_t)A.colptr.size() != n1 + m + 1) {
    *err = "device setup: the assembled matrix is missing";
    return 1;
  }
  auto cuda_fail = [&](const char* what) {
    *err = std::string("device setup: ") + what + ": " + cudaGetErrorString(cudaGetLastError());
    return 8;
  };
  // ---- front geometry and the arena
  std::vector<Front> fr(nsn);
  int64_t arena_n = 0, ncp_max = 0, ld_max = 0;
  for (int64_t k = 0; k < nsn; ++k) {
    Front& f = fr[k];
    f.nc = s.sn_col0[k + 1] - s.sn_col0[k];
    f.nr = (int32_t)(s.sn_rowptr[k + 1] - s.sn_rowptr[k]);
    const bool big = f.nc + f.nr > kSmallFront;
    f.ncp = big ? (int32_t)round64(f.nc) : f.nc;
    f.ld = big ? (int32_t)(f.ncp + round64(f.nr)) : f.nc + f.nr;
    f.off = arena_n;
    f.valptr = s.sn_valptr[k];
    f.rowptr = s.sn_rowptr[k];
    arena_n += (int64_t)f.ld * f.ld;
    if (big) { ncp_max = std::max<int64_t>(ncp_max, f.ncp); ld_max = std::max<int64_t>(ld_max, f.ld); }
  }
  // local index of global row i in front k (its structure must contain i)
  auto local = [&](int64_t k, int64_t i) -> int64_t {
    const int64_t c0 = s.sn_col0[k];
    if (i >= c0 && i < c0 + fr[k].nc) return i - c0;
    const int32_t* R = s.rows.data() + s.sn_rowptr[k];
    const int32_t* e = R + fr[k].nr;
    const int32_t* q = std::lower_bound(R, e, (int32_t)i);
    return (q == e || *q != i) ? -1 : fr[k].ncp + (q - R);
  };
  // ---- A of the alpha elements into the fronts (and the identity padding), A_22 into Sigma
  std::vector<int64_t> adst;
  std::vector<double> aval;
  std::vector<int64_t> sdst;
  std::vector<double> sval;
  adst.reserve(A.colptr[n1]);
  aval.reserve(A.colptr[n1]);
  for (int64_t k = 0; k < nsn; ++k) {
    const Front& f = fr[k];
    for (int64_t c = 0; c < f.nc; ++c) {
      const int64_t j = s.sn_col0[k] + c;
      for (int64_t q = A.colptr[j]; q < A.colptr[j + 1]; ++q) {
        const int64_t li = local(k, A.row[q]);
        if (li < 0) {
          *err = "device setup: a matrix entry outside its front's structure";
          return 1;
        }
        adst.push_back(f.off + li + c * f.ld);
        aval.push_back(A.val[q]);
      }
    }
    for (int64_t c = f.nc; c < f.ncp; ++c) {
      adst.push_back(f.off + c + c * f.ld);
      aval.push_back(1.0);
    }
  }
  for (int64_t j = n1; j < n1 + m; ++j)
    for (int64_t q = A.colptr[j]; q < A.colptr[j + 1]; ++q) {
      const int64_t i = A.row[q];
      sdst.push_back((i - n1) + (j - n1) * m);
      sval.push_back(A.val[q]);
      if (i != j) {
        sdst.push_back((j - n1) + (i - n1) * m);
        sval.push_back(A.val[q]);
      }
    }
  std::vector<int64_t> bdst;
  std::vector<double> bval;
  for (int64_t j = 0; j < m; ++j)
    for (int64_t q = s.B22.colptr[j]; q < s.B22.colptr[j + 1]; ++q) {
      bdst.push_back(s.B22.row[q] + j * m);
      bval.push_back(s.B22.val[q]);
    }
  for (int64_t k = 0; k < nsn; ++k)   // a front whose parent is x_2 has every row in x_2
    if (s.sn_parent[k] < 0 && fr[k].nr > 0 && s.rows[s.sn_rowptr[k]] < n1) {
      *err = "device setup: a root front with rows outside x_2";
      return 1;
    }
  // ---- children and their rows as local indices of the parent's front
  std::vector<std::vector<int32_t>> kids(nsn);
  std::vector<int32_t> relind(s.rows.size(), 0);
  for (int64_t u = 0; u < nsn; ++u) {
    const int64_t p = s.sn_parent[u];
    if (p < 0) continue;
    kids[p].push_back((int32_t)u);
    for (int64_t a = 0; a < fr[u].nr; ++a) {
      const int64_t li = local(p, s.rows[s.sn_rowptr[u] + a]);
      if (li < 0) {
        *err = "device setup: a child's row outside its parent's front";
        return 1;
      }
      relind[s.sn_rowptr[u] + a] = (int32_t)li;
    }
  }
  // ---- per level: extend-add passes, small fronts, large fronts, roots
  const int64_t nl = s.nlevels;
  std::vector<std::vector<int32_t>> bylevel(nl);
  for (int64_t k = 0; k < nsn; ++k) bylevel[s.sn_level[k]].push_back((int32_t)k);
  std::vector<EaTask> tasks;
  std::vector<std::vector<std::pair<int64_t, int64_t>>> passes(nl);   // [level] -> (first task, count) per pass
  std::vector<int32_t> small;
  std::vector<std::pair<int64_t, int64_t>> small_at(nl);
  std::vector<int32_t> small_ld(nl, 0);
  for (int64_t l = 0; l < nl; ++l) {
    size_t maxc = 0;
    for (int32_t p : bylevel[l]) maxc = std::max(maxc, kids[p].size());
    for (size_t r = 0; r < maxc; ++r) {
      const int64_t first = (int64_t)tasks.size();
      for (int32_t p : bylevel[l]) {
        if (r >= kids[p].size()) continue;
        const int32_t u = kids[p][r];
        const int32_t nb = std::max(1, 8192 / std::max(fr[u].nr, 1));
        for (int32_t b0 = 0; b0 < fr[u].nr; b0 += nb) tasks.push_back({u, p, b0, std::min(nb, fr[u].nr - b0)});
      }
      passes[l].push_back({first, (int64_t)tasks.size() - first});
    }
    small_at[l].first = (int64_t)small.size();
    for (int32_t k : bylevel[l])
      if (fr[k].nc + fr[k].nr <= kSmallFront) {
        small.push_back(k);
        small_ld[l] = std::max(small_ld[l], fr[k].ld);
      }
    small_at[l].second = (int64_t)small.size() - small_at[l].first;
  }
  // ---- device buffers
  DevBuf d_arena, d_fr, d_adst, d_aval, d_sdst, d_sval, d_bdst, d_bval, d_rel, d_rows, d_tasks, d_small, d_linv, d_x,
      d_status;
  if (!d_arena.alloc<double>(arena_n)) {
    cudaGetLastError();
    *err = "device setup: out of memory for the fronts (" + std::to_string(arena_n * 8 / (1 << 20)) + " MB)";
    return 9;
  }
  if (!d_fr.upload(fr, st) || !d_adst.upload(adst, st) || !d_aval.upload(aval, st) || !d_sdst.upload(sdst, st) ||
      !d_sval.upload(sval, st) || !d_bdst.upload(bdst, st) || !d_bval.upload(bval, st) || !d_rel.upload(relind, st) ||
      !d_rows.upload(s.rows, st) || !d_tasks.upload(tasks, st) || !d_small.upload(small, st) ||
      !d_linv.alloc<double>(std::max<int64_t>(ncp_max, TBS) / TBS * TBS * TBS) ||
      !d_x.alloc<double>(ncp_max * ncp_max) || !d_status.alloc<int>(1))
    return cuda_fail("upload");
  if (cudaMemsetAsync(d_arena.p, 0, sizeof(double) * std::max<int64_t>(arena_n, 1), st) != cudaSuccess ||
      cudaMemsetAsync(Sigma0, 0, sizeof(double) * m * m, st) != cudaSuccess ||
      cudaMemsetAsync(d_status.p, 0, sizeof(int), st) != cudaSuccess)
    return cuda_fail("memset");
  double* arena = d_arena.as<double>();
  int* status = d_status.as<int>();
  auto scatter = [&](const DevBuf& dst, const DevBuf& val, size_t n, double* base) {
    if (n == 0) return;
    k_scatter_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dst.as<int64_t>(), val.as<double>(), (int64_t)n, base);
    ++g_launches;
  };
  scatter(d_adst, d_aval, adst.size(), arena);
  scatter(d_sdst, d_sval, sdst.size(), Sigma0);
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(k_front_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSmallFront * kSmallFront * (int)sizeof(double));
    cudaFuncSetAttribute(k_binv_row, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 65 * (int)sizeof(double));
    cudaFuncSetAttribute(k_lrs_x, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 65 * (int)sizeof(double));
  }
  for (int64_t l = 0; l < nl; ++l) {
    for (const auto& ps : passes[l]) {
      if (ps.second == 0) continue;
      k_extend_add<<<(unsigned)ps.second, 256, 0, st>>>(d_tasks.as<EaTask>() + ps.first, d_fr.as<Front>(),
                                                         d_rel.as<int32_t>(), arena);
      ++g_launches;
    }
    if (small_at[l].second > 0) {
      k_front_small<<<(unsigned)small_at[l].second, 256, (size_t)small_ld[l] * small_ld[l] * sizeof(double), st>>>(
          d_small.as<int32_t>() + small_at[l].first, d_fr.as<Front>(), arena, Lval, status);
      ++g_launches;
    }
    for (int32_t k : bylevel[l]) {
      const Front& f = fr[k];
      if (f.nc + f.nr <= kSmallFront) continue;
      double* F = arena + f.off;
      cholesky_fp64(F, f.ld, d_linv.as<double>(), status, st, nullptr, 0, f.ncp / TBS);
      for (int i = 0; i < f.ncp / TBS; ++i) {
        k_binv_row<<<i + 1, 256, 2 * 64 * 65 * sizeof(double), st>>>(F, f.ld, d_linv.as<double>(), d_x.as<double>(),
                                                                       f.ncp, i);
        ++g_launches;
      }
      const int64_t nel = (int64_t)f.nc * f.nc;
      k_extract_big<<<(unsigned)((nel + 255) / 256), 256, 0, st>>>(f, d_x.as<double>(), Lval);
      ++g_launches;
      if (f.nr > 0) {
        k_lrs_x<<<dim3((unsigned)((f.nr + TBS - 1) / TBS), (unsigned)(f.ncp / TBS)), 256, 2 * 64 * 65 * sizeof(double),
                  st>>>(f, F, d_x.as<double>(), Lval);
        ++g_launches;
      }
    }
    for (int32_t k : bylevel[l]) {
      const Front& f = fr[k];
      if (s.sn_parent[k] >= 0 || f.nr == 0) continue;
      const int nbcta = 4;
      k_sigma_add<<<(unsigned)((f.nr + nbcta - 1) / nbcta), 256, 0, st>>>(f, 0, d_rows.as<int32_t>(), n1, arena,
                                                                          Sigma0, m, nbcta);
      ++g_launches;
    }
    if (cudaGetLastError() != cudaSuccess) return cuda_fail("launch");
  }
  scatter(d_bdst, d_bval, bdst.size(), Sigma0);
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return cuda_fail("factorisation");
  if (h_status != 0) {
    *err = "interior matrix is not positive definite (a free part without a Dirichlet node?)";
    return 5;
  }
  return 0;
}

}  // namespace pdk
