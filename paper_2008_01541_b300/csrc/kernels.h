// Launch wrappers of the CUDA kernels (plain pointers, one stream each).
#pragma once
#include <cstdint>
#include <vector>
#include <atomic>
#include <cuda_runtime.h>

namespace pdk {

// True the first time it is called with this mask on the current device (one
// bit per device): kernel attributes such as the dynamic shared-memory limit
// are set per device, so a process driving several GPUs sets them on each.
inline bool first_on_device(std::atomic<unsigned long long>& mask) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  return (mask.fetch_or(bit) & bit) == 0;
}


// Number of kernels launched by this library so far (host-side counter).
extern int64_t g_launches;

// ---- local step (Section 2.2) -------------------------------------------
// Extra local-step terms: bi-phasic strain limiting (Section 5), frac =
// mu' / (mu + mu' + kappa), singular value bounds [lo, hi]; the PD volume
// term (the lambda term of Eq. 1 in PD form), vfrac = kappa / (mu + mu' +
// kappa), determinant bounds [vlo, vhi].
struct StrainLimit {
  double frac = 0.0, lo = 0.0, hi = 0.0;
  double vfrac = 0.0, vlo = 0.0, vhi = 0.0;
};

// For each element e of a set: F = Ds Dm^-1, R = polar(F) in SO(3),
// fe[e][a][:] = forces on its four vertices, f_a = -w_e (F - P) G_a^T with
// P = R, or with the extra terms P = (1 - frac - vfrac) R + frac Q + vfrac T
// (w_e = 2 (mu + mu' + kappa) Vol_e).  R_out (optional) receives R row-major [count][9].
void polar_forces(int64_t count, const int4* tets, const double* DminvSoA, const double* w,
                  const double* x, double* fe, double* R_out, cudaStream_t st, const StrainLimit* sl = nullptr);

// out[t][:] = sum over the slots of target t of fe[slot][:]  (+ inertia if
// mass_h2 != null and t < inertia_limit: - mass_h2[t] (x[node(t)] - y[t]))
void gather_forces(int64_t ntarget, const int64_t* ptr, const int32_t* slot, const double* fe,
                   double* out, const double* add /*[ntarget][3] or null*/,
                   const double* mass_h2, const double* x, const double* y, const int32_t* node_of_t,
                   int64_t inertia_limit, cudaStream_t st);

// ---- supernodal triangular solves with L_1 / L_21 (Section 3.2, Steps 1 and 3)
struct SparseFactor {
  int64_t n1 = 0, nfree = 0, nsn = 0, nlevels = 0;
  const int32_t* col0 = nullptr;     // [nsn+1]
  const int64_t* rowptr = nullptr;   // [nsn+1]
  const int32_t* rows = nullptr;
  const int64_t* valptr = nullptr;   // [nsn+1]
  const double* L = nullptr;
  // Tasks {s | kind << 29, row offset, col offset, target-list index} in
  // forward / backward topological order; kind 0 = 64 x 64 tile of a
  // diagonal block, 1 = tile of an off-diagonal block, 2 = a whole small
  // supernode.
  int64_t n_ftasks = 0, n_btasks = 0;
  const int4* ftasks = nullptr;
  const int4* btasks = nullptr;
  const int64_t* tgt_ptr = nullptr;       // target lists: distinct supernodes owning a task's off-diagonal rows
  const int32_t* tgt = nullptr;
  int* cnt = nullptr;                     // counters, reset from cnt_init before each solve
  const int* cnt_init = nullptr;
  int64_t cnt_fin = 0, cnt_ydone = 0, cnt_next_f = 0, cnt_zpend = 0, cnt_udone = 0, cnt_next_b = 0;
  int grid_f = 0, grid_b = 0;             // persistent CTAs of the forward / backward launch
  int* status = nullptr;                  // status[1] <- 300 if a wait gave up
};
// CTAs of the persistent grid: every resident slot of the direction's build
// (four per SM forward, five backward).
int sparse_grid(bool forward);
// b [nfree][3] in: forces (factor order).  Out: y[0..n1) = L_1^-1 b_1 and
// b[n1..nfree) = b_2 - L_21 y_1.
void sparse_forward(const SparseFactor& f, double* b, double* y, cudaStream_t st);
// u[n1..nfree) must hold U_2.  Out: u[0..n1) = L_1^-T (y_1 - L_21^T U_2).
void sparse_backward(const SparseFactor& f, const double* y, double* u, double* z, cudaStream_t st);

// ---- dense collision-region block (Section 3.3) ---------------------------
// H (mp x mp, column-major, lower) = Sigma0 (m x m) padded with identity.
void copy_sigma(const double* Sigma0, int64_t m, double* H, int64_t mp, cudaStream_t st);
// Springs store ns node slots each (region indices, -1 = unused): 4 for a
// proxy embedded in one tet, 8 for a two-sided spring between two proxies.
constexpr int CSLOTS = 8;
// H[ra][rb] += c_j w_a w_b for the k springs
// perm (optional): region index -> position in a permuted H.
void contact_scatter(int64_t k, const int32_t* cidx, const double* cw, const double* cs,
                     double* H, int64_t mp, cudaStream_t st, int ns = CSLOTS, const int32_t* perm = nullptr);
// g[r][:] += -w_a c_j (p_j - t_j) with p_j = sum_a w_a x[region[r_a]]
void contact_forces(int64_t k, const int32_t* cidx, const double* cw, const double* ct,
                    const double* cs, const int32_t* region, const double* x, double* g,
                    cudaStream_t st, int ns = CSLOTS);
// Side stream and events for the look-ahead factorisation order.
struct LookAhead {
  cudaStream_t side = nullptr;
  std::vector<cudaEvent_t> ev_panel, ev_rest;   // one per tile step
};
// Blocked right-looking FP64 Cholesky of the padded H (tile 64). Linv receives
// the inverses of the diagonal tiles; status[0] = first failing column + 1.
// With la (events for mp/64 steps) the trailing update is split between st
// and la->side (depth-1 look-ahead); without it everything runs on st.
// [k_begin, k_end) restricts the work to the panels of those tiles (a partial
// factorisation leaves the Schur complement in the trailing block); Linv is
// formed for the same tiles.
void cholesky_fp64(double* H, int64_t mp, double* Linv, int* status, cudaStream_t st,
                   const LookAhead* la = nullptr, int k_begin = 0, int k_end = -1);
// H = P S P^T (mp x mp, column-major, identity padding), P given by iperm:
// factor position -> region index
void permute_sym(const double* S, int64_t m, const int32_t* iperm, double* H, int64_t mp, cudaStream_t st);
// the n x n block of H at (off, off) to (to_h) or from a dense buffer B
void block_copy(double* H, int64_t mp, int64_t off, double* B, int64_t n, bool to_h, cudaStream_t st);
// Solve (L L^T) u = g for 3 right-hand sides, g/u [m][3] (padded internally),
// one launch per block step.
void chol_solve_fp64(const double* H, int64_t mp, const double* Linv, const double* g, double* u,
                     int64_t m, double* work /*[mp][3] x 2*/, cudaStream_t st, const int32_t* perm = nullptr);
// The same solve as two persistent launches of dependency-counter tasks;
// cnt: [1 + 2 mp/64] ints of scratch, status[1] <- 302 if a wait gave up.
// A device on which the chain cluster cannot run beside an update cluster
// takes the per-step solve instead.
// perm (optional): region index -> factor position of a permuted factor.
void chol_solve_fp64_tasks(const double* H, int64_t mp, const double* Linv, const double* g, double* u,
                           int64_t m, double* work /*[mp][3] x 2*/, int* cnt, int* status, cudaStream_t st,
                           const int32_t* perm = nullptr);
// out[i][:] = sum_j S[i][j] v[j][:]  (S symmetric m x m, full storage), FP64
void symv3(const double* S, int64_t m, const double* v, double* out, cudaStream_t st);
// out[i][:] += alpha * sum_j B[i][j] v[j][:]  (CSC of a symmetric pattern)
void spmv3(int64_t m, const int64_t* ptr, const int32_t* row, const double* val, const double* v,
           double alpha, double* out, cudaStream_t st);
// Device collision detection (one spring slot per proxy / side-A proxy).
// sph: [nsph][4] centre + radius.  Region indices for the proxies.
void detect_spheres(int64_t np, const int32_t* prox_r, const int32_t* region, const double* x, int nsph,
                    const double* sph, double stiffness, int32_t* cidx, double* cw, double* ct, double* cs,
                    cudaStream_t st);
void detect_pairs(int64_t na, const int32_t* ra, int64_t nb, const int32_t* rb, const int32_t* region,
                  const double* x, double gap, double stiffness, int32_t* cidx, double* cw, double* ct, double* cs,
                  cudaStream_t st);
// Point-triangle detector: na side-A proxies then nb side-B proxies (region
// indices, prox[0 .. na + nb)), nta side-A triangles then ntb side-B
// triangles (region indices, tris[0 .. 3 (nta + ntb))), rest positions of the
// region nodes xr [m][3], bounding-sphere scratch bnd [nta + ntb].  Slots
// 0 .. na + nb of the spring arrays, one per proxy.
struct TriDetector {
  int64_t na = 0, nb = 0, nta = 0, ntb = 0;
  const int32_t* prox = nullptr;
  const int32_t* tris = nullptr;
  const double* xr = nullptr;
  float4* bnd = nullptr;
  double gap = 0.0, rest_min = 0.0, stiffness = 0.0;
};
void detect_tris(const TriDetector& d, const int32_t* region, const double* x, int32_t* cidx, double* cw, double* ct,
                 double* cs, cudaStream_t st);
// Algorithm 1, 4.6-4.7: x2 += u2, U2 += u2, ft2 -= (Su - Bu)   (Bu already in Su: Su holds Sigma_alpha u)
void inner_update(int64_t m, const double* u2, const double* Sau, const int32_t* region, double* x,
                  double* U2, double* ft2, cudaStream_t st);
// x[node_of_pos[p]] += u[p] for p < n1
void apply_interior(int64_t n1, const double* u, const int32_t* node_of_pos, double* x, cudaStream_t st);
// out[i] = x[idx[i]]  (3 doubles each)
void gather_rows(int64_t cnt, const int32_t* idx, const double* x, double* out, cudaStream_t st);
// x[idx[i]] = v[i]
void scatter_rows(int64_t cnt, const int32_t* idx, const double* v, double* x, cudaStream_t st);
// y = a*x + b*y elementwise over n doubles
void axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st);

}  // namespace pdk
