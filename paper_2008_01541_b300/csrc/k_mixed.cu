// Mixed-precision forms of the collision-region solve H u = g (Algorithm 1,
// step 4.5; Section 3.3).  H = Sigma_0 + C_22 is equilibrated by
// D = diag(H)^-1/2 and factored in low precision with a blocked right-looking
// Cholesky (128 x 128 tiles): FP32 diagonal-tile factorisation and inversion,
// FP32 panel solve, and tcgen05 trailing updates in TF32, split TF32 (three
// products, ~FP32 accuracy) or BF16, all accumulated in FP32.  Accuracy is
// recovered with FP64-accurate residuals r = g - H u (FP64 vectors; Sigma_0 u
// from Sigma_0 stored as an FP32 head + tail pair, ~48 bits, multiplied in
// double-float arithmetic; the contact term in FP64): plain iterative refinement for
// the split-TF32 factor, and refinement accelerated by preconditioned CG for
// TF32 and BF16.  PD_PCG_WARM runs PCG on H with the contact-free factor of
// Sigma_0 (computed once) as the preconditioner, started from a given guess.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include "chol_ll.h"
#include "df_arith.cuh"
#include "kernels.h"
#include "lowp_tile.cuh"
#include "mixed.h"
#include "solver.h"
#include "tc.h"

namespace pdm {


struct Factor {
  float* L = nullptr;         // [mq][mq] row-major, lower tiles hold the factor
  float* Dinv = nullptr;      // [T][128][128] row-major inverses of the diagonal tiles
  float* E = nullptr;         // [T][128][128] Dinv^T Dinv per diagonal tile
  float* Lh = nullptr;        // [mq][mq] row-major, Lh_ik = L_ik Dinv_k (i > k)
  __nv_bfloat16* Pb[2] = {nullptr, nullptr};  // [mq][128] BF16 copies of the panel, by panel parity
  double* d = nullptr;        // [mq] equilibration D (by region index)
  const int32_t* iperm = nullptr;   // factor position -> region index (nested form), else identity
  int k0 = 0;                 // nested form: tiles before k0 are fixed
  float* Sp = nullptr;        // nested form: saved trailing block
  CUtensorMap mapL{}, mapP[2]{};
  // persistent left-looking factorisation: TF32 tails / BF16 copies of the finished panels
  float* Llo = nullptr;       // [mq][mq] split TF32
  __nv_bfloat16* Lb = nullptr;   // [mq][mq] BF16
  CUtensorMap mapLo{}, mapLb{};
  bool valid = false;
};

struct MixedState {
  int64_t mq = 0, T = 0;
  int64_t ldm = 0;            // row stride of Shi / Slo / Minv0 and length / 3 of vhi / vlo / r32: m rounded up to 4
  bool nested_ready = false;  // nested form: the fixed leading tiles of f are current
  int nested_mode = -1;
  Factor f, f0;               // per-solve factor, contact-free factor (PCG_WARM)
  double *hdiag = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *u = nullptr;
  double* sig = nullptr;          // [m][3] Sigma_0 x of the last residual product's x (sig_x)
  const double* sig_x = nullptr;  // that x's buffer; null once its contents may have changed
  float *Shi = nullptr, *Slo = nullptr;   // Sigma_0 = Shi + Slo (FP32 pair, ~48-bit)
  float *vhi = nullptr, *vlo = nullptr;   // [m][3] split of the vector being multiplied
  float* Minv0 = nullptr;     // [m][m] explicit inverse of the contact-free factor (PCG form), built once
  float* r32 = nullptr;       // [m][3] float copy of a right-hand side
  bool minv_valid = false;
  double* sc = nullptr;       // device scalars: [0] r.r  [1] r.z  [2] p.q  [3] r.z old  [4] g.g
  double* sc_h = nullptr;     // pinned copy
  float *w = nullptr, *uo = nullptr;   // [mq][3] triangular-solve vectors
  int* pcnt = nullptr;        // preconditioner scratch: task counters [2 + 4T], then facc, bacc
  float *facc = nullptr, *bacc = nullptr;   // [mq][3] accumulated block products (forward / backward)
  int pc_grid = 0;            // persistent grid of the preconditioner
  int* llsync = nullptr;      // counters of the persistent left-looking factorisation
  // first non-positive pivot + 1 of the low-precision factor (the pivot is
  // replaced by 1: H is SPD, the FP32 factor of an ill-conditioned D H D can
  // still lose a pivot; the refinement against H then decides)
  int* lpiv = nullptr;
  int* lpiv_h = nullptr;      // pinned copy
  bool lookahead = false;     // PD_LOWP_SCHEDULE=lookahead: one launch per tile step instead
  int ll_ctas = 0;            // PD_LOWP_CTAS: cap on the persistent factorisation's grid (0: two thirds of the SMs)
  cudaStream_t side = nullptr;              // low-priority stream for the bulk trailing updates
  std::vector<cudaEvent_t> ev_panel, ev_rest;
  // Capacitance (Woodbury) correction of the PCG form's preconditioner: with
  // V = C^1/2 W over the active springs, P^-1 = M0^-1 - Y^T S^-1 V M0^-1,
  // Y = V M0^-1 [kact][ldm] (rows of the explicit inverse, FP32) and
  // S = I + V M0^-1 V^T [kp][kp] (FP64, column-major, identity padding,
  // factored by the FP64 blocked Cholesky); P = M0 + C_22 up to the FP32
  // inverse, so the one outlier eigenvalue per spring of M0^-1 H is removed.
  int64_t cap_rows = 0;       // spring slots the buffers below hold
  int64_t cap_kp = 0;         // order of Scap (kact rounded up to 64)
  int64_t kact = 0;           // active springs of the current solve (0: no correction)
  int* cap_act = nullptr;     // [cap_rows] slot of each active spring, in slot order
  int* cap_cnt = nullptr;     // [1] active count; cap_cnt_h its pinned copy
  int* cap_cnt_h = nullptr;
  float* Y = nullptr;
  double* ccoef = nullptr;    // [cap_rows][8] sqrt(c_j) w_js of each active spring's slots (0: unused slot)
  double *Scap = nullptr, *Slinv = nullptr;   // S and the inverses of its 64 x 64 diagonal tiles
  double *ct = nullptr, *cy = nullptr, *cwork = nullptr;   // [kp][3] V z, S^-1 V z; [kp][3] x 2 solve work
  double* cpart = nullptr;    // [kp / 64][m][3] chunk partial sums of Y^T S^-1 V z
  int *ccnt = nullptr, *cstat = nullptr;     // solve task counters; factor status
  int cg_hint = 1;            // PCG iterations of the previous solve (where the checks start)
  bool cap_pending = false;   // active springs counted (ev_cap), S not yet built
  cudaEvent_t ev_cap = nullptr;
};

namespace {

// ---------------------------------------------------------------- small kernels
__global__ void k_hdiag(const double* S, int64_t m, double* hd) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) hd[i] = S[i * m + i];
}
__global__ void k_contact_diag(int64_t k, const int32_t* cidx, const double* cw, const double* cs, double* hd) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  constexpr int NS = pdk::CSLOTS;
  if (t >= (int64_t)NS * NS * k) return;
  int64_t j = t / (NS * NS);
  int a = (int)((t / NS) % NS), b = (int)(t % NS);
  int ra = cidx[NS * j + a], rb = cidx[NS * j + b];
  if (ra < 0 || ra != rb) return;
  atomicAdd(hd + ra, cs[j] * cw[NS * j + a] * cw[NS * j + b]);
}
__global__ void k_dscale(const double* hd, int64_t m, int64_t mq, double* d, int* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= mq) return;
  if (i < m) {
    double h = hd[i];
    if (!(h > 0.0)) { atomicCAS(status, 0, (int)i + 1); h = 1.0; }
    d[i] = 1.0 / sqrt(h);
  } else {
    d[i] = 1.0;
  }
}
// L = D Sigma_0 D in FP32 (lower tiles), identity padding.
__global__ void k_cast_eq(const double* __restrict__ S, int64_t m, const double* __restrict__ d,
                          float* __restrict__ L, int64_t mq) {
  int ti = blockIdx.x, tj = blockIdx.y;
  if (ti < tj) return;
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
    int r = q / NB, c = q % NB;
    int64_t i = (int64_t)ti * NB + r, j = (int64_t)tj * NB + c;
    float v;
    if (i < m && j < m) v = (float)(S[i * m + j] * d[i] * d[j]);
    else v = (i == j) ? 1.f : 0.f;
    L[i * mq + j] = v;
  }
}
__global__ void k_contact_scatter_f32(int64_t k, const int32_t* cidx, const double* cw, const double* cs,
                                      const double* d, float* L, int64_t mq, const int32_t* perm) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  constexpr int NS = pdk::CSLOTS;
  if (t >= (int64_t)NS * NS * k) return;
  int64_t j = t / (NS * NS);
  int a = (int)((t / NS) % NS), b = (int)(t % NS);
  int ra = cidx[NS * j + a], rb = cidx[NS * j + b];
  if (ra < 0 || rb < 0) return;
  const double v = cs[j] * cw[NS * j + a] * cw[NS * j + b] * d[ra] * d[rb];
  if (perm) { ra = perm[ra]; rb = perm[rb]; }   // factor positions (d stays by region index)
  if (ra < rb) return;
  atomicAdd(L + (int64_t)ra * mq + rb, (float)v);
}
// L = D P Sigma_0 P^T D in FP32 (lower tiles, row-major), identity padding;
// factor position p holds region index iperm[p], d by region index.
__global__ void k_cast_eq_perm(const double* __restrict__ S, int64_t m, const double* __restrict__ d,
                               const int32_t* __restrict__ iperm, float* __restrict__ L, int64_t mq) {
  int ti = blockIdx.x, tj = blockIdx.y;
  if (ti < tj) return;
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
    int r = q / NB, c = q % NB;
    int64_t i = (int64_t)ti * NB + r, j = (int64_t)tj * NB + c;
    float v;
    if (i < m && j < m) {
      const int64_t a = iperm[i], b = iperm[j];
      v = (float)(S[a * m + b] * d[a] * d[b]);
    } else {
      v = (i == j) ? 1.f : 0.f;
    }
    L[i * mq + j] = v;
  }
}
// copy the trailing n x n block at (off, off) of the row-major L to (to_l) or from B
__global__ void k_block_copy_f32(float* __restrict__ L, int64_t mq, int64_t off, float* __restrict__ B, int64_t n,
                                 int to_l) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int64_t i = q / n, j = q % n;
  float* l = L + (off + i) * mq + (off + j);
  if (to_l) *l = B[q];
  else B[q] = *l;
}

// Factor the diagonal tile (kt, kt) in FP32 (L_kk), blocked in shared memory
// with 32-wide sub-blocks and a look-ahead inside the tile: while warp 0
// factors sub-block p, warps 1-7 apply the rest of panel p-1's trailing
// update; the panel below sub-block p is solved one thread per row.  Then the
// tile's inverse Dinv_k (tile_inverse) from the same shared-memory tile.  One
// 128 x 129 FP32 tile plus the four 32 x 33 diagonal inverse blocks (83 KB)
// fit on an SM beside two CTAs of the concurrent tensor-core trailing update,
// so the serial chain never waits for the whole bulk update to drain.
__global__ void __launch_bounds__(256) k_diag_f32(float* __restrict__ L, int64_t mq, int kt,
                                                  float* __restrict__ Dinv, int* __restrict__ status) {
  extern __shared__ float sm[];
  float* A = sm;                   // [128][PADW]
  float* Zd = sm + NB * PADW;      // [4][32][33] diagonal blocks of the inverse
  const int tid = threadIdx.x;
  float* Lt = L + (int64_t)kt * NB * mq + (int64_t)kt * NB;
  {
    float4 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int q = tid + 256 * k, r = q >> 5, c = 4 * (q & 31);
      v[k] = __ldcg(reinterpret_cast<const float4*>(Lt + (int64_t)r * mq + c));
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int q = tid + 256 * k, r = q >> 5, c = 4 * (q & 31);
      A[r * PADW + c] = v[k].x; A[r * PADW + c + 1] = v[k].y; A[r * PADW + c + 2] = v[k].z; A[r * PADW + c + 3] = v[k].w;
    }
  }
  __syncthreads();
  diag_factor_smem(A, kt, status);
  for (int q = tid; q < NB * NB; q += 256) {
    const int r = q / NB, c = q % NB;
    if (c <= r) Lt[(int64_t)r * mq + c] = A[r * PADW + c];
  }
  // the inverse for the panel solve and the preconditioner, from the tile in shared memory
  tile_inverse(A, Zd, Dinv + (int64_t)kt * NB * NB);
}

// E_k = Dinv_k^T Dinv_k for every diagonal tile (one CTA per tile, off the
// factorisation's critical path).
__global__ void __launch_bounds__(512) k_gram(const float* __restrict__ Dinv, float* __restrict__ E) {
  extern __shared__ float sm[];
  const float* Di = Dinv + (int64_t)blockIdx.x * NB * NB;
  float* Ek = E + (int64_t)blockIdx.x * NB * NB;
  for (int q = threadIdx.x; q < NB * NB; q += 512) sm[(q / NB) * PADW + q % NB] = Di[q];
  __syncthreads();
  for (int q = threadIdx.x; q < NB * NB; q += 512) {
    const int r = q / NB, c = q % NB;
    float e = 0.f;
    for (int t = (r > c ? r : c); t < NB; ++t) e = fmaf(sm[t * PADW + r], sm[t * PADW + c], e);
    Ek[q] = e;
  }
}

// Panel solve for the 32-row slab blockIdx.x below tile kt: L_ik = A_ik Dinv_k^T
// and Lh_ik = L_ik Dinv_k.  256 threads, 4 x 4 outputs each (warp = 4 rows);
// operands are held k-major in shared memory so every inner step is two
// 16-byte loads.
constexpr int RB = 32, AP = RB + 4, DP = NB + 4;
__global__ void __launch_bounds__(256) k_trsm_f32(float* __restrict__ L, float* __restrict__ Lh, int64_t mq, int kt,
                                               const float* __restrict__ Dinv, __nv_bfloat16* __restrict__ Pb) {
  extern __shared__ float4 sm4[];
  float* AT = reinterpret_cast<float*>(sm4);   // [NB][AP]  A^T, later L row-major
  float* DT = AT + NB * AP;                     // [NB][DP]  Dinv^T, later Dinv
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  const int64_t r0 = (int64_t)(kt + 1) * NB + (int64_t)blockIdx.x * RB;
  float* Ab = L + r0 * mq + (int64_t)kt * NB;
  float* Hb = Lh + r0 * mq + (int64_t)kt * NB;
  const float* Di = Dinv + (int64_t)kt * NB * NB;
  {
    // consecutive threads take consecutive rows, so the transposed shared
    // stores hit consecutive banks
    float4 va[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // A slab: 32 rows x 32 float4
      const int q = tid + 256 * k, r = q & 31, c = 4 * (q >> 5);
      va[k] = __ldcg(reinterpret_cast<const float4*>(Ab + (int64_t)r * mq + c));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = tid + 256 * k, r = q & 31, c = 4 * (q >> 5);
      AT[(c + 0) * AP + r] = va[k].x; AT[(c + 1) * AP + r] = va[k].y; AT[(c + 2) * AP + r] = va[k].z; AT[(c + 3) * AP + r] = va[k].w;
    }
    const int row = tid & 127, kh = 16 * (tid >> 7);
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {  // Dinv: row `row`, float4 k, stored transposed
      const int k = kh + kk;
      const float4 v = __ldcg(reinterpret_cast<const float4*>(Di + row * NB + 4 * k));
      DT[(4 * k + 0) * DP + row] = v.x; DT[(4 * k + 1) * DP + row] = v.y;
      DT[(4 * k + 2) * DP + row] = v.z; DT[(4 * k + 3) * DP + row] = v.w;
    }
  }
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
  for (int t = 0; t < NB; ++t) {
    const float4 a = *reinterpret_cast<const float4*>(AT + t * AP + 4 * ty);
    const float4 b = *reinterpret_cast<const float4*>(DT + t * DP + 4 * tx);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
  __syncthreads();
  // L to global (and its BF16 copy), L row-major into AT; Dinv (row-major) into DT
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = 4 * ty + i;
    *reinterpret_cast<float4*>(Ab + (int64_t)rr * mq + 4 * tx) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    if (Pb) {
      __nv_bfloat16 hb[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) hb[j] = __float2bfloat16_rn(acc[i][j]);
      *reinterpret_cast<uint2*>(Pb + (r0 + rr) * NB + 4 * tx) = *reinterpret_cast<const uint2*>(hb);
    }
  }
  float* LS = AT;   // L row-major [RB][DP], reusing the A^T buffer
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<float4*>(LS + (4 * ty + i) * DP + 4 * tx) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
#pragma unroll 4
  for (int k = 0; k < 16; ++k) {
    const int q = tid + 256 * k, r = q >> 5, c = 4 * (q & 31);
    *reinterpret_cast<float4*>(DT + r * DP + c) = __ldcg(reinterpret_cast<const float4*>(Di + r * NB + c));
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
  for (int t = 0; t < NB; ++t) {
    const float av[4] = {LS[(4 * ty) * DP + t], LS[(4 * ty + 1) * DP + t], LS[(4 * ty + 2) * DP + t],
                         LS[(4 * ty + 3) * DP + t]};
    const float4 b = *reinterpret_cast<const float4*>(DT + t * DP + 4 * tx);
    const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<float4*>(Hb + (int64_t)(4 * ty + i) * mq + 4 * tx) =
        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
}


// z = D L^-T L^-1 D r for 3 right-hand sides.  With Lh_ik = L_ik Dinv_k and
// E_k = Dinv_k^T Dinv_k the block substitutions need no dense diagonal solve:
//   forward : w_i = D r_i - sum_{k < i} Lh_ik w_k
//   backward: u_k = E_k w_k - sum_{i > k} Lh_ik^T u_i
// One persistent launch.  The first CTA to start is the chain: it walks the
// block rows (forward, then backward), each step applying only the adjacent
// block (Lh_i,i-1 w_i-1, resp. Lh_k+1,k^T u_k+1) to the accumulated sum,
// with the previous block's vector kept in shared memory and the next
// adjacent tile loaded into registers during the step.  The other CTAs claim,
// in list order, the non-adjacent block products (forward by block column,
// then E_k w_k for every k, then backward by block row) and add them into the
// accumulators facc / bacc with FP32 atomics.  Each task waits only on the
// chain or on tasks earlier in the list, so the grid cannot stall; every wait
// is bounded (code 301 in status[1]).
// cnt: [0] task claims, [1] chain role, [2 + k] w_k written, [2 + T + k] u_k
// written, [2 + 2T + i] products added into facc_i, [2 + 3T + k] into bacc_k.
__device__ __forceinline__ unsigned long long ptimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void wait_at_least(const int* c, int target, int* status, unsigned long long t0) {
  unsigned it = 0;
  while (*(volatile const int*)c < target) {
    if (*(volatile int*)(status + 1) != 0) return;
    if (++it > 32) __nanosleep(64);
    if ((it & 1023u) == 0 && ptimer() - t0 > 1000000000ull) {
      atomicCAS(status + 1, 0, 301);
      return;
    }
  }
}

// block b of a staircase task list over T blocks: block b holds T - 2 - b tasks
__device__ inline int pc_start(int T, int b) { return b * (T - 2) - b * (b - 1) / 2; }
__device__ inline void pc_decode(int t, int T, int& b, int& q) {
  const double dd = 2.0 * T - 3.0;
  int e = (int)floor(0.5 * (dd - sqrt(fmax(dd * dd - 8.0 * t, 0.0))));
  e = max(0, min(e, T - 3));
  while (e > 0 && pc_start(T, e) > t) --e;
  while (e < T - 3 && pc_start(T, e + 1) <= t) ++e;
  b = e;
  q = t - pc_start(T, e);
}

// Row products: thread (g = tid >> 3, c8 = tid & 7) holds rows g + 32 j
// (j < 4), columns 16 c8 .. + 15 of a row-major 128 x 128 block, so a warp's
// 16-byte loads cover four 128-byte lines.  The vector is kept per component
// with entry c at c + 4 (c >> 4) (VSW floats a component), which spreads the
// eight column groups over distinct banks.
constexpr int VSW = NB + 4 * (NB / 16);
__device__ __forceinline__ int vs_pos(int c) { return c + 4 * (c >> 4); }

__device__ __forceinline__ void load_rows4(float (&l)[64], const float* p, int64_t ld) {
  const int g = threadIdx.x >> 3, c8 = threadIdx.x & 7;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p + (int64_t)(g + 32 * j) * ld + 16 * c8) + q);
      l[16 * j + 4 * q] = v.x; l[16 * j + 4 * q + 1] = v.y; l[16 * j + 4 * q + 2] = v.z; l[16 * j + 4 * q + 3] = v.w;
    }
}

// a[j][v] = sum_c block[g + 32 j][c] x_v[c], complete in every lane of the group of 8
__device__ __forceinline__ void rows4_dot(const float (&l)[64], const float (*vs)[VSW], float (&a)[4][3]) {
  const int c8 = threadIdx.x & 7;
  const float *x0 = vs[0] + 20 * c8, *x1 = vs[1] + 20 * c8, *x2 = vs[2] + 20 * c8;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    a[j][0] = a[j][1] = a[j][2] = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      a[j][0] = fmaf(l[16 * j + c], x0[c], a[j][0]);
      a[j][1] = fmaf(l[16 * j + c], x1[c], a[j][1]);
      a[j][2] = fmaf(l[16 * j + c], x2[c], a[j][2]);
    }
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int v = 0; v < 3; ++v) a[j][v] += __shfl_xor_sync(0xffffffffu, a[j][v], o);
}

// the 128 x 3 block of x (global, interleaved) into the per-component layout
__device__ __forceinline__ void load_vs(float (*vs)[VSW], const float* x) {
  for (int e = threadIdx.x; e < NB * 3; e += 256) vs[e % 3][vs_pos(e / 3)] = __ldcg(x + e);
}

// L2 prefetch of the 128 x 128 block at p (row-major, leading dimension ld):
// thread (row tid >> 1, half tid & 1) touches the two 128-byte lines of its
// 64 entries, so a later register load of the block hits L2
__device__ __forceinline__ void prefetch_block(const float* p, int64_t ld) {
  const float* q = p + (int64_t)(threadIdx.x >> 1) * ld + 64 * (threadIdx.x & 1);
  asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
  asm volatile("prefetch.global.L2 [%0];" ::"l"(q + 32));
}

// column c of a row-major block (rows h * 64 .. + 63, leading dimension ld)
__device__ __forceinline__ void load_col64(float (&l)[64], const float* p, int64_t ld) {
#pragma unroll
  for (int q = 0; q < 64; ++q) l[q] = __ldg(p + (int64_t)q * ld);
}

// facc = D r in factor order (zero on the padding rows), bacc = 0
__global__ void k_pc_pre(int64_t mq, int64_t m, const double* __restrict__ d, const double* __restrict__ r,
                         const int32_t* __restrict__ iperm, float* __restrict__ facc, float* __restrict__ bacc) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= 3 * mq) return;
  const int64_t row = q / 3;
  float v = 0.f;
  if (row < m) {
    const int64_t ri = iperm ? iperm[row] : row;   // region index of this factor row
    v = (float)(d[ri] * r[3 * ri + q % 3]);
  }
  facc[q] = v;
  bacc[q] = 0.f;
}

// z = D u back in region order
__global__ void k_pc_post(int64_t m, const double* __restrict__ d, const float* __restrict__ uo,
                          const int32_t* __restrict__ iperm, double* __restrict__ z) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= 3 * m) return;
  const int64_t col = q / 3;
  const int64_t ci = iperm ? iperm[col] : col;
  z[3 * ci + q % 3] = d[ci] * (double)uo[q];
}

__global__ void __launch_bounds__(256) k_precond(const float* __restrict__ Lh, const float* __restrict__ E,
                                                 int64_t mq, float* w, float* uo, float* facc, float* bacc, int* cnt,
                                                 int* status) {
  __shared__ float vs[2][3][VSW];   // row products: previous / current block vector (chain), the operand (tasks)
  __shared__ float vb[2][NB][3];    // column products: the same
  __shared__ float red[2][NB][3];   // half sums of the column products
  __shared__ int cur;
  const int T = (int)(mq / NB), tid = threadIdx.x;
  const int g8 = tid >> 3, c8 = tid & 7;          // row products: rows g8 + 32 j, column group c8
  const int cc = tid & (NB - 1), hc = tid >> 7;   // column products: column, half of the rows
  if (tid == 0) cur = atomicAdd(cnt + 1, 1);
  __syncthreads();
  const bool chain = cur == 0;
  __syncthreads();
  float l[64];
  if (chain) {
    int pb = 0;   // vs[pb] / vb[pb] hold the previous block's vector
    if (T > 1) load_rows4(l, Lh + (int64_t)NB * mq, mq);
    // ---- forward: w_i = facc_i - Lh_i,i-1 w_i-1 (facc_i starts as D r_i); lane c8 = j < 4
    // of a group of 8 finishes row g8 + 32 j
    const int rj = g8 + 32 * (c8 & 3);
    for (int i = 0; i < T; ++i) {
      if (tid == 0) {
        wait_at_least(cnt + 2 + 2 * T + i, i >= 1 ? i - 1 : 0, status, ptimer());
        __threadfence();
      }
      __syncthreads();
      const float* fa = facc + 3 * ((int64_t)i * NB + rj);
      float f0 = 0.f, f1 = 0.f, f2 = 0.f;
      if (c8 < 4) { f0 = __ldcg(fa); f1 = __ldcg(fa + 1); f2 = __ldcg(fa + 2); }   // in flight during the dot
      float a[4][3];
      if (i > 0) {
        rows4_dot(l, vs[pb], a);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j][0] = a[j][1] = a[j][2] = 0.f;
      }
      if (c8 < 4) {
        // a[c8], selected without indexing a register array
        const float s0 = c8 == 0 ? a[0][0] : c8 == 1 ? a[1][0] : c8 == 2 ? a[2][0] : a[3][0];
        const float s1 = c8 == 0 ? a[0][1] : c8 == 1 ? a[1][1] : c8 == 2 ? a[2][1] : a[3][1];
        const float s2 = c8 == 0 ? a[0][2] : c8 == 1 ? a[1][2] : c8 == 2 ? a[2][2] : a[3][2];
        const float w0 = f0 - s0, w1 = f1 - s1, w2 = f2 - s2;
        float* wr = w + 3 * ((int64_t)i * NB + rj);
        wr[0] = w0; wr[1] = w1; wr[2] = w2;
        const int ps = vs_pos(rj);
        vs[pb ^ 1][0][ps] = w0; vs[pb ^ 1][1][ps] = w1; vs[pb ^ 1][2][ps] = w2;
        __threadfence();
      }
      if (i + 1 < T)   // next step's adjacent tile, in flight from here
        load_rows4(l, Lh + (int64_t)(i + 1) * NB * mq + (int64_t)i * NB, mq);
      if (i + 2 < T) prefetch_block(Lh + (int64_t)(i + 2) * NB * mq + (int64_t)(i + 1) * NB, mq);
      __syncthreads();
      if (tid == 0) atomicAdd(cnt + 2 + i, 1);
      pb ^= 1;
    }
    // ---- backward: u_k = bacc_k - Lh_k+1,k^T u_k+1 (bacc_k holds E_k w_k and the other products)
    for (int k = T - 1; k >= 0; --k) {
      if (tid == 0) {
        wait_at_least(cnt + 2 + 3 * T + k, 1 + (T - 2 - k > 0 ? T - 2 - k : 0), status, ptimer());
        __threadfence();
      }
      __syncthreads();
      const int64_t col = (int64_t)k * NB + cc;
      const float* ba = bacc + 3 * col;
      float b0 = 0.f, b1 = 0.f, b2 = 0.f;
      if (hc == 0) { b0 = __ldcg(ba); b1 = __ldcg(ba + 1); b2 = __ldcg(ba + 2); }   // in flight during the dot
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
      if (k < T - 1) {
#pragma unroll
        for (int q = 0; q < 64; ++q) {
          const float* x = vb[pb][64 * hc + q];
          a0 = fmaf(l[q], x[0], a0); a1 = fmaf(l[q], x[1], a1); a2 = fmaf(l[q], x[2], a2);
        }
      }
      red[hc][cc][0] = a0; red[hc][cc][1] = a1; red[hc][cc][2] = a2;
      __syncthreads();
      if (hc == 0) {
        const float u0 = b0 - (red[0][cc][0] + red[1][cc][0]);
        const float u1 = b1 - (red[0][cc][1] + red[1][cc][1]);
        const float u2 = b2 - (red[0][cc][2] + red[1][cc][2]);
        float* uc = uo + 3 * col;
        uc[0] = u0; uc[1] = u1; uc[2] = u2;
        vb[pb ^ 1][cc][0] = u0; vb[pb ^ 1][cc][1] = u1; vb[pb ^ 1][cc][2] = u2;
        __threadfence();
      }
      if (k > 0)   // column cc of Lh_k,k-1, rows hc * 64 .. + 63
        load_col64(l, Lh + ((int64_t)k * NB + 64 * hc) * mq + (int64_t)(k - 1) * NB + cc, mq);
      if (k > 1) prefetch_block(Lh + (int64_t)(k - 1) * NB * mq + (int64_t)(k - 2) * NB, mq);
      __syncthreads();
      if (tid == 0) atomicAdd(cnt + 2 + T + k, 1);
      pb ^= 1;
    }
    return;
  }
  const int nF = T >= 3 ? (T - 2) * (T - 1) / 2 : 0, ntask = 2 * nF + T;
  for (;;) {
    if (tid == 0) cur = atomicAdd(cnt, 1);
    __syncthreads();
    const int t = cur;
    if (t >= ntask) break;
    if (t < nF || t >= nF + T) {
      const bool fwd = t < nF;
      int b, q;
      pc_decode(fwd ? t : t - nF - T, T, b, q);
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
      if (fwd) {
        // facc_i -= Lh_ik w_k, k = b, i = k + 2 + q
        const int k = b, i = k + 2 + q;
        load_rows4(l, Lh + (int64_t)i * NB * mq + (int64_t)k * NB, mq);
        if (tid == 0) {
          wait_at_least(cnt + 2 + k, 1, status, ptimer());
          __threadfence();
        }
        __syncthreads();
        load_vs(vs[0], w + 3 * (int64_t)k * NB);
        __syncthreads();
        float a[4][3];
        rows4_dot(l, vs[0], a);
        if (c8 < 4) {
          float* fa = facc + 3 * ((int64_t)i * NB + g8 + 32 * c8);
          const float s0 = c8 == 0 ? a[0][0] : c8 == 1 ? a[1][0] : c8 == 2 ? a[2][0] : a[3][0];
          const float s1 = c8 == 0 ? a[0][1] : c8 == 1 ? a[1][1] : c8 == 2 ? a[2][1] : a[3][1];
          const float s2 = c8 == 0 ? a[0][2] : c8 == 1 ? a[1][2] : c8 == 2 ? a[2][2] : a[3][2];
          atomicAdd(fa, -s0); atomicAdd(fa + 1, -s1); atomicAdd(fa + 2, -s2);
          __threadfence();
        }
        __syncthreads();
        if (tid == 0) atomicAdd(cnt + 2 + 2 * T + i, 1);
      } else {
        // bacc_k -= Lh_ik^T u_i, i = T - 1 - b, k = i - 2 - q
        const int i = T - 1 - b, k = i - 2 - q;
        load_col64(l, Lh + ((int64_t)i * NB + 64 * hc) * mq + (int64_t)k * NB + cc, mq);
        if (tid == 0) {
          wait_at_least(cnt + 2 + T + i, 1, status, ptimer());
          __threadfence();
        }
        __syncthreads();
        for (int e = tid; e < NB * 3; e += 256) (&vb[0][0][0])[e] = __ldcg(uo + 3 * (int64_t)i * NB + e);
        __syncthreads();
#pragma unroll
        for (int q2 = 0; q2 < 64; ++q2) {
          const float* x = vb[0][64 * hc + q2];
          a0 = fmaf(l[q2], x[0], a0); a1 = fmaf(l[q2], x[1], a1); a2 = fmaf(l[q2], x[2], a2);
        }
        red[hc][cc][0] = a0; red[hc][cc][1] = a1; red[hc][cc][2] = a2;
        __syncthreads();
        if (hc == 0) {
          float* ba = bacc + 3 * ((int64_t)k * NB + cc);
          atomicAdd(ba, -(red[0][cc][0] + red[1][cc][0]));
          atomicAdd(ba + 1, -(red[0][cc][1] + red[1][cc][1]));
          atomicAdd(ba + 2, -(red[0][cc][2] + red[1][cc][2]));
          __threadfence();
        }
        __syncthreads();
        if (tid == 0) atomicAdd(cnt + 2 + 3 * T + k, 1);
      }
    } else {
      // bacc_k += E_k w_k (E_k symmetric, row-major), k = T - 1 - (t - nF)
      const int k = T - 1 - (t - nF);
      load_rows4(l, E + (int64_t)k * NB * NB, NB);
      if (tid == 0) {
        wait_at_least(cnt + 2 + k, 1, status, ptimer());
        __threadfence();
      }
      __syncthreads();
      load_vs(vs[0], w + 3 * (int64_t)k * NB);
      __syncthreads();
      float a[4][3];
      rows4_dot(l, vs[0], a);
      if (c8 < 4) {
        float* ba = bacc + 3 * ((int64_t)k * NB + g8 + 32 * c8);
        const float s0 = c8 == 0 ? a[0][0] : c8 == 1 ? a[1][0] : c8 == 2 ? a[2][0] : a[3][0];
        const float s1 = c8 == 0 ? a[0][1] : c8 == 1 ? a[1][1] : c8 == 2 ? a[2][1] : a[3][1];
        const float s2 = c8 == 0 ? a[0][2] : c8 == 1 ? a[1][2] : c8 == 2 ? a[2][2] : a[3][2];
        atomicAdd(ba, s0); atomicAdd(ba + 1, s1); atomicAdd(ba + 2, s2);
        __threadfence();
      }
      __syncthreads();
      if (tid == 0) atomicAdd(cnt + 2 + 3 * T + k, 1);
    }
    __syncthreads();
  }
}

// bytes of the preconditioner scratch: counters, then the two accumulators
inline size_t pc_scratch_bytes(int64_t T, int64_t mq) {
  return ((sizeof(int) * (2 + 4 * T) + 15) & ~(size_t)15) + 2 * sizeof(float) * 3 * mq;
}

// z = Minv0 r (FP32 dense symmetric inverse, 3 right-hand sides), one warp per row.
// Row products with a padded FP32 matrix (row stride ld, a multiple of 4,
// zero beyond column m) and an interleaved [ld][3] vector (zero beyond row
// m): one warp per row, 16-byte loads, lane j4 takes columns 4 j4 .. + 3.
// z = Minv0 r (FP32 dense symmetric inverse, 3 right-hand sides).
__global__ void k_minv_apply(const float* __restrict__ Mi, int64_t m, int64_t ld, const float* __restrict__ r,
                             double* __restrict__ z) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  const float4* row = reinterpret_cast<const float4*>(Mi + i * ld);
  const float4* rv = reinterpret_cast<const float4*>(r);
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 8
  for (int64_t j4 = lane; j4 < ld / 4; j4 += 32) {
    const float4 v = __ldg(row + j4);
    const float4 x0 = __ldg(rv + 3 * j4), x1 = __ldg(rv + 3 * j4 + 1), x2 = __ldg(rv + 3 * j4 + 2);
    // x0..x2 = (c0 v0 c1 v0 c2 v0 c0 v1) (c1 v1 c2 v1 c0 v2 c1 v2) (c2 v2 c0 v3 c1 v3 c2 v3)
    a0 = fmaf(v.x, x0.x, a0); a1 = fmaf(v.x, x0.y, a1); a2 = fmaf(v.x, x0.z, a2);
    a0 = fmaf(v.y, x0.w, a0); a1 = fmaf(v.y, x1.x, a1); a2 = fmaf(v.y, x1.y, a2);
    a0 = fmaf(v.z, x1.z, a0); a1 = fmaf(v.z, x1.w, a1); a2 = fmaf(v.z, x2.x, a2);
    a0 = fmaf(v.w, x2.y, a0); a1 = fmaf(v.w, x2.z, a1); a2 = fmaf(v.w, x2.w, a2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) { z[3 * i] = a0; z[3 * i + 1] = a1; z[3 * i + 2] = a2; }
}
__global__ void k_to_f32(const double* __restrict__ x, int64_t n, float* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}
// three unit right-hand sides e_{3q}, e_{3q+1}, e_{3q+2} as the columns of r [m][3]
__global__ void k_unit3(double* r, int64_t m, int64_t q) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int v = 0; v < 3; ++v) r[3 * i + v] = (i == 3 * q + v) ? 1.0 : 0.0;
}
// rows 3q..3q+2 of the inverse from z [m][3] (the inverse is symmetric; row stride ld)
__global__ void k_store_cols(const double* z, int64_t m, int64_t ld, int64_t q, float* Mi) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int v = 0; v < 3; ++v)
    if (3 * q + v < m) Mi[(3 * q + v) * ld + i] = (float)z[3 * i + v];
}

// Double-float products: a double split into an FP32 head and an FP32 tail.
__global__ void k_split(const double* __restrict__ x, int64_t n, float* __restrict__ hi, float* __restrict__ lo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  const float h = (float)v;
  hi[i] = h;
  lo[i] = (float)(v - (double)h);
}
// Sigma_0 split into FP32 head and tail rows with the padded stride ld (zero padding).
__global__ void k_split_rows(const double* __restrict__ S, int64_t m, int64_t ld, float* __restrict__ hi,
                             float* __restrict__ lo) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= m * ld) return;
  const int64_t i = q / ld, j = q % ld;
  const double v = j < m ? S[i * m + j] : 0.0;
  const float h = (float)v;
  hi[q] = h;
  lo[q] = (float)(v - (double)h);
}

using pddf::df_acc_lazy;
using pddf::df_add;
using pddf::df_norm;

// out = Sigma_0 v for 3 right-hand sides in double-float arithmetic on the
// FP32 pipes (Shi + Slo rows with stride ld, v = vhi + vlo interleaved [ld][3]);
// one warp takes two rows, so every vector load serves both; lanes are
// combined in double-float too, so only the final conversion is FP64.
// out2 (optional) receives a second copy.
__global__ void k_symv_df(const float* __restrict__ Shi, const float* __restrict__ Slo, int64_t m, int64_t ld,
                          const float* __restrict__ vhi, const float* __restrict__ vlo, double* __restrict__ out,
                          double* __restrict__ out2) {
  const int64_t i0 = 2 * ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i0 >= m) return;
  const int64_t i1 = i0 + 1 < m ? i0 + 1 : i0;      // an odd last row is computed twice, stored once
  float h[2][3] = {}, l[2][3] = {};
  const float4* rh0 = reinterpret_cast<const float4*>(Shi + i0 * ld);
  const float4* rl0 = reinterpret_cast<const float4*>(Slo + i0 * ld);
  const float4* rh1 = reinterpret_cast<const float4*>(Shi + i1 * ld);
  const float4* rl1 = reinterpret_cast<const float4*>(Slo + i1 * ld);
  const float4* xh = reinterpret_cast<const float4*>(vhi);
  const float4* xl = reinterpret_cast<const float4*>(vlo);
#pragma unroll 2
  for (int64_t j4 = lane; j4 < ld / 4; j4 += 32) {
    const float4 a0 = __ldg(rh0 + j4), b0 = __ldg(rl0 + j4), a1 = __ldg(rh1 + j4), b1 = __ldg(rl1 + j4);
    const float4 p0 = __ldg(xh + 3 * j4), p1 = __ldg(xh + 3 * j4 + 1), p2 = __ldg(xh + 3 * j4 + 2);
    const float4 q0 = __ldg(xl + 3 * j4), q1 = __ldg(xl + 3 * j4 + 1), q2 = __ldg(xl + 3 * j4 + 2);
    const float av[2][4] = {{a0.x, a0.y, a0.z, a0.w}, {a1.x, a1.y, a1.z, a1.w}};
    const float bv[2][4] = {{b0.x, b0.y, b0.z, b0.w}, {b1.x, b1.y, b1.z, b1.w}};
    const float ph[12] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x, p2.y, p2.z, p2.w};
    const float pl[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
#pragma unroll
    for (int w = 0; w < 2; ++w) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int c = 0; c < 3; ++c) df_acc_lazy(av[w][e], bv[w][e], ph[3 * e + c], pl[3 * e + c], h[w][c], l[w][c]);
#pragma unroll
      for (int c = 0; c < 3; ++c) df_norm(h[w][c], l[w][c]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int w = 0; w < 2; ++w)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float h2 = __shfl_xor_sync(0xffffffffu, h[w][c], o), l2 = __shfl_xor_sync(0xffffffffu, l[w][c], o);
        df_add(h[w][c], l[w][c], h2, l2);
      }
  if (lane < 6) {
    const int w = lane / 3, c = lane % 3;
    float hc = 0.f, lc = 0.f;
#pragma unroll
    for (int ww = 0; ww < 2; ++ww)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc)
        if (ww == w && cc == c) { hc = h[ww][cc]; lc = l[ww][cc]; }
    const int64_t row = w == 0 ? i0 : i1;
    if (w == 0 || i1 != i0) {
      out[3 * row + c] = (double)hc + (double)lc;
      if (out2) out2[3 * row + c] = (double)hc + (double)lc;
    }
  }
}

__global__ void k_contact_matvec(int64_t k, const int32_t* cidx, const double* cw, const double* cs,
                                 const double* p, double* q) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= k) return;
  constexpr int NS = pdk::CSLOTS;
  double s0 = 0, s1 = 0, s2 = 0;
  for (int a = 0; a < NS; ++a) {
    int ra = cidx[NS * j + a];
    if (ra < 0) continue;
    double wa = cw[NS * j + a];
    s0 += wa * p[3 * ra]; s1 += wa * p[3 * ra + 1]; s2 += wa * p[3 * ra + 2];
  }
  double c = cs[j];
  for (int a = 0; a < NS; ++a) {
    int ra = cidx[NS * j + a];
    if (ra < 0) continue;
    double f = c * cw[NS * j + a];
    atomicAdd(q + 3 * ra, f * s0); atomicAdd(q + 3 * ra + 1, f * s1); atomicAdd(q + 3 * ra + 2, f * s2);
  }
}

// out[slot] += sum x*y over n doubles
__global__ void k_dot(const double* __restrict__ x, const double* __restrict__ y, int64_t n, double* out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(out, t);
  }
}
__global__ void k_sub(const double* a, const double* b, double* out, int64_t n) {   // out = a - b
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] - b[i];
}
__global__ void k_add(double* u, const double* z, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) u[i] += z[i];
}
// Fused CG kernels; sc slots: 2 = p.q, a / b = r.z of this / the next iteration.
// u += alpha p, r -= alpha q (alpha = sc[a] / sc[2]); r32 = (float) r; sc[b] = 0 for the next r.z
__global__ void k_cg_step2(double* u, double* r, const double* p, const double* q, double* sc, int a, int b,
                           int64_t n, float* r32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double pq = sc[2], alpha = pq != 0.0 ? sc[a] / pq : 0.0;
  if (i == 0) sc[b] = 0.0;
  if (i >= n) return;
  u[i] += alpha * p[i];
  const double ri = r[i] - alpha * q[i];
  r[i] = ri;
  if (r32) r32[i] = (float)ri;
}
// p = z + beta p (beta = sc[b] / sc[a]; first: p = z), p split into head / tail for the
// next Sigma_0 product, sc[2] = 0 for the next p.q
__global__ void k_cg_dir2(double* p, const double* z, double* sc, int a, int b, int64_t n, int first,
                          float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double den = sc[a], beta = first ? 0.0 : (den != 0.0 ? sc[b] / den : 0.0);
  if (i == 0) sc[2] = 0.0;
  if (i >= n) return;
  const double v = z[i] + beta * (first ? 0.0 : p[i]);
  p[i] = v;
  const float h = (float)v;
  hi[i] = h;
  lo[i] = (float)(v - (double)h);
}
// ---- capacitance correction of the PCG preconditioner (Woodbury identity)
// Active springs (stiffness > 0 and at least one node in the region) in slot
// order, by one block scanning the slots in chunks of blockDim.x (a
// multiple of 32, at most 1024): deterministic, unlike an atomic append.
__global__ void k_cap_active(int64_t k, const int32_t* __restrict__ cidx, const double* __restrict__ cs,
                             int* __restrict__ act, int* __restrict__ cnt) {
  constexpr int NS = pdk::CSLOTS;
  __shared__ int wsum[32], woff[32];
  __shared__ int base, tot;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int64_t j0 = 0; j0 < k; j0 += blockDim.x) {
    const int64_t j = j0 + threadIdx.x;
    bool on = false;
    if (j < k && cs[j] > 0.0)
      for (int a = 0; a < NS; ++a) on |= cidx[NS * j + a] >= 0;
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    if (lane == 0) wsum[wp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int q = 0; q < nw; ++q) { woff[q] = acc; acc += wsum[q]; }
      tot = acc;
    }
    __syncthreads();
    if (on) act[base + woff[wp] + __popc(bal & ((1u << lane) - 1u))] = (int)j;
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *cnt = base;
}
// coef[a][s] = sqrt(c_j) w_js for active spring a = slot j (0 for an unused slot):
// the entries of V = C^1/2 W, formed once per refactorisation
__global__ void k_cap_coef(int64_t kact, const int* __restrict__ act, const int32_t* __restrict__ cidx,
                           const double* __restrict__ cw, const double* __restrict__ cs, double* __restrict__ coef) {
  constexpr int NS = pdk::CSLOTS;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= NS * kact) return;
  const int64_t a = t / NS;
  const int q = (int)(t % NS), j = act[a];
  coef[t] = cidx[NS * j + q] >= 0 ? sqrt(cs[j]) * cw[NS * j + q] : 0.0;
}
// Y[a][:] = sum_s coef[a][s] Minv0[node_js][:] for active spring a = slot j
// (the rows of V M0^-1; the padding columns of Minv0 are zero): one spring
// per blockIdx.y, four columns per thread.
__global__ void __launch_bounds__(256) k_cap_rows(const int* __restrict__ act, const int32_t* __restrict__ cidx,
                                                  const double* __restrict__ coef, const float* __restrict__ Mi,
                                                  int64_t ldm, float* __restrict__ Y) {
  constexpr int NS = pdk::CSLOTS;
  __shared__ float cf[NS];
  __shared__ int rw[NS];
  const int64_t a = blockIdx.y;
  if (threadIdx.x < NS) {
    const int j = act[a];
    rw[threadIdx.x] = cidx[NS * j + threadIdx.x];
    cf[threadIdx.x] = (float)coef[NS * a + threadIdx.x];
  }
  __syncthreads();
  const int64_t i4 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // ldm is a multiple of 4
  if (4 * i4 >= ldm) return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    if (rw[q] < 0) continue;
    const float4 v = __ldg(reinterpret_cast<const float4*>(Mi + (int64_t)rw[q] * ldm) + i4);
    acc.x = fmaf(cf[q], v.x, acc.x); acc.y = fmaf(cf[q], v.y, acc.y);
    acc.z = fmaf(cf[q], v.z, acc.z); acc.w = fmaf(cf[q], v.w, acc.w);
  }
  reinterpret_cast<float4*>(Y + a * ldm)[i4] = acc;
}
// S = I + V M0^-1 V^T (symmetrised), kp x kp column-major, identity padding.
__global__ void k_cap_matrix(int64_t kact, int64_t kp, const int* __restrict__ act, const int32_t* __restrict__ cidx,
                             const double* __restrict__ coef, const float* __restrict__ Y, int64_t ldm,
                             double* __restrict__ S) {
  constexpr int NS = pdk::CSLOTS;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= kp * kp) return;
  const int64_t a = t % kp, b = t / kp;
  if (a >= kact || b >= kact) {
    S[t] = a == b ? 1.0 : 0.0;
    return;
  }
  const int ja = act[a], jb = act[b];
  double h1 = 0.0, h2 = 0.0;
  for (int q = 0; q < NS; ++q) {
    const int ra = cidx[NS * ja + q];
    if (ra >= 0) h1 += coef[NS * a + q] * (double)Y[b * ldm + ra];
    const int rb = cidx[NS * jb + q];
    if (rb >= 0) h2 += coef[NS * b + q] * (double)Y[a * ldm + rb];
  }
  S[t] = (a == b ? 1.0 : 0.0) + 0.5 * (h1 + h2);
}
// t[a][:] = sqrt(c_j) sum_s w_js z[node_js][:]  (V z, 3 right-hand sides)
__global__ void k_cap_gather(int64_t kact, const int* __restrict__ act, const int32_t* __restrict__ cidx,
                             const double* __restrict__ coef, const double* __restrict__ z, double* __restrict__ t) {
  constexpr int NS = pdk::CSLOTS;
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= kact) return;
  const int j = act[a];
  double t0 = 0.0, t1 = 0.0, t2 = 0.0;
  for (int q = 0; q < NS; ++q) {
    const int r = cidx[NS * j + q];
    if (r < 0) continue;
    const double w = coef[NS * a + q];
    t0 += w * z[3 * r]; t1 += w * z[3 * r + 1]; t2 += w * z[3 * r + 2];
  }
  t[3 * a] = t0; t[3 * a + 1] = t1; t[3 * a + 2] = t2;
}
// part[ch][i][:] = sum over the springs a of chunk ch (kCapChunk of them) of
// Y[a][i] y[a][:], accumulated in FP32 like the M0^-1 r it corrects (the
// preconditioner is FP32-accurate as a whole; FP64 here ran at the FP64 rate)
constexpr int kCapChunk = 64;
__global__ void k_cap_part(int64_t m, int64_t kact, const float* __restrict__ Y, int64_t ldm,
                           const double* __restrict__ y, double* __restrict__ part) {
  __shared__ float ys[3 * kCapChunk];
  const int64_t ch = blockIdx.y, a0 = ch * kCapChunk;
  const int na = (int)(kact - a0 < kCapChunk ? kact - a0 : kCapChunk);
  for (int t = threadIdx.x; t < 3 * na; t += blockDim.x) ys[t] = (float)y[3 * a0 + t];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float* Yc = Y + a0 * ldm + i;
  float c0 = 0.f, c1 = 0.f, c2 = 0.f;
  for (int a = 0; a < na; ++a) {
    const float v = __ldg(Yc + a * ldm);
    c0 = fmaf(v, ys[3 * a], c0);
    c1 = fmaf(v, ys[3 * a + 1], c1);
    c2 = fmaf(v, ys[3 * a + 2], c2);
  }
  double* o = part + (ch * m + i) * 3;
  o[0] = c0; o[1] = c1; o[2] = c2;
}
// z -= sum over the chunks of part (in chunk order), and acc += r . z after
// the correction (one atomic per block)
__global__ void k_cap_apply(int64_t m, int nch, const double* __restrict__ part, double* __restrict__ z,
                            const double* __restrict__ r, double* __restrict__ acc) {
  __shared__ double red[8];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double rz = 0.0;
  if (i < m) {
    double c0 = 0.0, c1 = 0.0, c2 = 0.0;
    for (int ch = 0; ch < nch; ++ch) {
      const double* p = part + (ch * m + i) * 3;
      c0 += p[0]; c1 += p[1]; c2 += p[2];
    }
    const double z0 = z[3 * i] - c0, z1 = z[3 * i + 1] - c1, z2 = z[3 * i + 2] - c2;
    z[3 * i] = z0; z[3 * i + 1] = z1; z[3 * i + 2] = z2;
    rz = r[3 * i] * z0 + r[3 * i + 1] * z1 + r[3 * i + 2] * z2;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rz += __shfl_xor_sync(0xffffffffu, rz, o);
  if (lane == 0) red[wp] = rz;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    atomicAdd(acc, t);
  }
}

// z = Minv0 r32 as k_minv_apply, and sc[slot] += r . z (r in FP64; one atomic per block)
__global__ void k_minv_apply_dot(const float* __restrict__ Mi, int64_t m, int64_t ld, const float* __restrict__ r32,
                                 const double* __restrict__ r, double* __restrict__ z, double* __restrict__ acc) {
  __shared__ double red[8];
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double rz = 0.0;
  if (i < m) {
    const float4* row = reinterpret_cast<const float4*>(Mi + i * ld);
    const float4* rv = reinterpret_cast<const float4*>(r32);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 8
    for (int64_t j4 = lane; j4 < ld / 4; j4 += 32) {
      const float4 v = __ldg(row + j4);
      const float4 x0 = __ldg(rv + 3 * j4), x1 = __ldg(rv + 3 * j4 + 1), x2 = __ldg(rv + 3 * j4 + 2);
      a0 = fmaf(v.x, x0.x, a0); a1 = fmaf(v.x, x0.y, a1); a2 = fmaf(v.x, x0.z, a2);
      a0 = fmaf(v.y, x0.w, a0); a1 = fmaf(v.y, x1.x, a1); a2 = fmaf(v.y, x1.y, a2);
      a0 = fmaf(v.z, x1.z, a0); a1 = fmaf(v.z, x1.w, a1); a2 = fmaf(v.z, x2.x, a2);
      a0 = fmaf(v.w, x2.y, a0); a1 = fmaf(v.w, x2.z, a1); a2 = fmaf(v.w, x2.w, a2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
      z[3 * i] = a0; z[3 * i + 1] = a1; z[3 * i + 2] = a2;
      rz = r[3 * i] * (double)a0 + r[3 * i + 1] * (double)a1 + r[3 * i + 2] * (double)a2;
    }
  }
  if (lane == 0) red[wp] = rz;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    atomicAdd(acc, t);
  }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ------------------------------------------------------------------ host side
static pd_status ensure_state(pd_solver* s) {
  if (s->mixed) return PD_OK;
  MixedState* M = new MixedState();
  s->mixed = M;
  M->mq = ((s->m + NB - 1) / NB) * NB;
  M->T = M->mq / NB;
  M->ldm = (s->m + 3) & ~(int64_t)3;
  auto A = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e == cudaSuccess) s->allocs.push_back(*p);
    return e;
  };
  const int64_t mq = M->mq, m = s->m;
  for (Factor* f : {&M->f, &M->f0}) {
    if (A((void**)&f->L, sizeof(float) * mq * mq) || A((void**)&f->Dinv, sizeof(float) * mq * NB) ||
        A((void**)&f->E, sizeof(float) * mq * NB) || A((void**)&f->Lh, sizeof(float) * mq * mq) ||
        A((void**)&f->Pb[0], sizeof(__nv_bfloat16) * mq * NB) || A((void**)&f->Pb[1], sizeof(__nv_bfloat16) * mq * NB) ||
        A((void**)&f->d, sizeof(double) * mq)) {
      s->err = "device allocation for the mixed-precision factor failed";
      return PD_ERR_OOM;
    }
    if (!pdtc::make_map(&f->mapL, f->L, 4, mq, mq, mq, 32) || !pdtc::make_map(&f->mapP[0], f->Pb[0], 2, mq, NB, NB, 64) ||
        !pdtc::make_map(&f->mapP[1], f->Pb[1], 2, mq, NB, NB, 64)) {
      s->err = "cuTensorMapEncodeTiled failed";
      return PD_ERR_CUDA;
    }
  }
  if (A((void**)&M->hdiag, sizeof(double) * m) || A((void**)&M->r, sizeof(double) * 3 * m) ||
      A((void**)&M->z, sizeof(double) * 3 * m) || A((void**)&M->p, sizeof(double) * 3 * m) ||
      A((void**)&M->q, sizeof(double) * 3 * m) || A((void**)&M->u, sizeof(double) * 3 * m) ||
      A((void**)&M->sig, sizeof(double) * 3 * m) ||
      A((void**)&M->sc, sizeof(double) * 8) || A((void**)&M->w, sizeof(float) * 3 * mq) ||
      A((void**)&M->uo, sizeof(float) * 3 * mq) || A((void**)&M->Shi, sizeof(float) * m * M->ldm) ||
      A((void**)&M->Slo, sizeof(float) * m * M->ldm) || A((void**)&M->vhi, sizeof(float) * 3 * M->ldm) ||
      A((void**)&M->vlo, sizeof(float) * 3 * M->ldm) || A((void**)&M->r32, sizeof(float) * 3 * M->ldm) ||
      A((void**)&M->pcnt, pc_scratch_bytes(M->T, mq))) {
    s->err = "device allocation for the mixed-precision vectors failed";
    return PD_ERR_OOM;
  }
  {
    const size_t cb = (sizeof(int) * (2 + 4 * M->T) + 15) & ~(size_t)15;
    M->facc = reinterpret_cast<float*>(reinterpret_cast<char*>(M->pcnt) + cb);
    M->bacc = M->facc + 3 * mq;
  }
  if (A((void**)&M->llsync, pdll::sync_bytes((int)M->T)) || A((void**)&M->lpiv, sizeof(int))) {
    s->err = "device allocation for the factorisation counters failed";
    return PD_ERR_OOM;
  }
  {
    const char* sched = std::getenv("PD_LOWP_SCHEDULE");
    M->lookahead = sched && std::string(sched) == "lookahead";
    const char* ctas = std::getenv("PD_LOWP_CTAS");
    M->ll_ctas = ctas ? std::max(0, std::atoi(ctas)) : 0;
  }
  if (cudaMallocHost(&M->sc_h, sizeof(double) * 8) != cudaSuccess) return PD_ERR_OOM;
  if (cudaMallocHost(&M->lpiv_h, sizeof(int)) != cudaSuccess) return PD_ERR_OOM;
  cudaMemsetAsync(M->lpiv, 0, sizeof(int), s->stream);
  // vectors beyond m stay zero: the padded products need no bounds checks
  cudaMemsetAsync(M->vhi, 0, sizeof(float) * 3 * M->ldm, s->stream);
  cudaMemsetAsync(M->vlo, 0, sizeof(float) * 3 * M->ldm, s->stream);
  cudaMemsetAsync(M->r32, 0, sizeof(float) * 3 * M->ldm, s->stream);
  k_split_rows<<<nblk(m * M->ldm, 256), 256, 0, s->stream>>>(s->Sigma0, m, M->ldm, M->Shi, M->Slo);
  ++pdk::g_launches;
  int lo_prio = 0, hi_prio = 0;
  cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
  if (cudaStreamCreateWithPriority(&M->side, cudaStreamNonBlocking, lo_prio) != cudaSuccess) return PD_ERR_CUDA;
  M->ev_panel.resize(M->T);
  M->ev_rest.resize(M->T);
  for (int64_t i = 0; i < M->T; ++i) {
    cudaEventCreateWithFlags(&M->ev_panel[i], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&M->ev_rest[i], cudaEventDisableTiming);
  }
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_precond, 256, 0);
  M->pc_grid = std::max(1, nsm * std::max(1, per));
  static std::atomic<unsigned long long> attr{0};
  if (pdk::first_on_device(attr)) {
    cudaFuncSetAttribute(k_diag_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (NB * PADW + 4 * 32 * 33) * 4);
    cudaFuncSetAttribute(k_trsm_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (NB * AP + NB * DP) * 4);
    cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, NB * PADW * 4);
  }
  return PD_OK;
}

// Equilibrate Sigma_0 (+ C_22 if with_contacts) into f (Algorithm 1, 4.3).
static void factor_cast(pd_solver* s, Factor& f, bool with_contacts) {
  MixedState* M = s->mixed;
  const int64_t m = s->m, mq = M->mq, T = M->T;
  cudaStream_t st = s->stream;
  const int64_t k = with_contacts ? s->k : 0;
  k_hdiag<<<nblk(m, 256), 256, 0, st>>>(s->Sigma0, m, M->hdiag); ++pdk::g_launches;
  if (k > 0) { k_contact_diag<<<nblk((int64_t)pdk::CSLOTS * pdk::CSLOTS * k, 256), 256, 0, st>>>(k, s->c_idx, s->c_w, s->c_s, M->hdiag); ++pdk::g_launches; }
  k_dscale<<<nblk(mq, 256), 256, 0, st>>>(M->hdiag, m, mq, f.d, s->status); ++pdk::g_launches;
  k_cast_eq<<<dim3((unsigned)T, (unsigned)T), 256, 0, st>>>(s->Sigma0, m, f.d, f.L, mq); ++pdk::g_launches;
  if (k > 0) {
    k_contact_scatter_f32<<<nblk((int64_t)pdk::CSLOTS * pdk::CSLOTS * k, 256), 256, 0, st>>>(k, s->c_idx, s->c_w, s->c_s, f.d, f.L, mq, nullptr);
    ++pdk::g_launches;
  }
}

// Blocked low-precision Cholesky of f.L in place.
static void factor_panels(pd_solver* s, Factor& f, pdtc::Mode mode, int k_begin = 0, int k_end = -1) {
  MixedState* M = s->mixed;
  const int64_t mq = M->mq, T = M->T;
  if (k_end < 0 || k_end > T) k_end = (int)T;
  cudaStream_t st = s->stream;
  // Depth-1 look-ahead: the main stream factors tile kt, solves panel kt and
  // updates only block column kt+1; the low-priority side stream applies
  // panel kt to the rest of the trailing matrix meanwhile.
  cudaStream_t sb = M->side;
  for (int kt = k_begin; kt < k_end; ++kt) {
    k_diag_f32<<<1, 256, (NB * PADW + 4 * 32 * 33) * 4, st>>>(f.L, mq, kt, f.Dinv, M->lpiv);
    ++pdk::g_launches;
    const int n = (int)(T - kt - 1);
    if (n <= 0) break;
    __nv_bfloat16* pb = mode == pdtc::BF16 ? f.Pb[kt & 1] : nullptr;
    k_trsm_f32<<<(unsigned)(n * (NB / RB)), 256, (NB * AP + NB * DP) * 4, st>>>(f.L, f.Lh, mq, kt, f.Dinv, pb);
    ++pdk::g_launches;
    cudaEventRecord(M->ev_panel[kt], st);
    if (kt > k_begin) cudaStreamWaitEvent(st, M->ev_rest[kt - 1], 0);
    const CUtensorMap* map = mode == pdtc::BF16 ? &f.mapP[kt & 1] : &f.mapL;
    const int kx = mode == pdtc::BF16 ? 0 : kt * NB, kch = mode == pdtc::BF16 ? 2 : 4;
    pdtc::rank_k_update(mode, map, map, kx, kch, f.L, mq, kt + 1, kt + 1, n, 1, 0, s->status, st);
    cudaStreamWaitEvent(sb, M->ev_panel[kt], 0);
    if (n > 1) pdtc::rank_k_update(mode, map, map, kx, kch, f.L, mq, kt + 2, kt + 2, n - 1, n - 1, 1, s->status, sb);
    cudaEventRecord(M->ev_rest[kt], sb);
  }
  const int last = k_end == T ? (int)T - 2 : k_end - 1;   // the last step that recorded ev_rest
  if (last >= k_begin) cudaStreamWaitEvent(st, M->ev_rest[last], 0);
  if (k_end > k_begin) {
    k_gram<<<(unsigned)(k_end - k_begin), 512, NB * PADW * 4, st>>>(f.Dinv + (int64_t)k_begin * NB * NB,
                                                                    f.E + (int64_t)k_begin * NB * NB);
    ++pdk::g_launches;
  }
  f.valid = true;
}

// The factor of tile columns k_begin .. T-1 of f.L in one persistent launch
// (left-looking, see chol_ll.h); the panel copies its tensor-core products
// read are allocated on first use.
static pd_status factor_ll(pd_solver* s, Factor& f, pdtc::Mode mode, int k_begin = 0) {
  MixedState* M = s->mixed;
  const int64_t mq = M->mq;
  if (M->lookahead) {
    factor_panels(s, f, mode, k_begin);
    return PD_OK;
  }
  if (mode == pdtc::TF32X3 && !f.Llo) {
    if (cudaMalloc(&f.Llo, sizeof(float) * mq * mq) != cudaSuccess) {
      s->err = "device allocation of the TF32 tails failed";
      return PD_ERR_OOM;
    }
    s->allocs.push_back(f.Llo);
    if (!pdtc::make_map(&f.mapLo, f.Llo, 4, mq, mq, mq, 32)) { s->err = "cuTensorMapEncodeTiled failed"; return PD_ERR_CUDA; }
  }
  if (mode == pdtc::BF16 && !f.Lb) {
    if (cudaMalloc(&f.Lb, sizeof(__nv_bfloat16) * mq * mq) != cudaSuccess) {
      s->err = "device allocation of the BF16 panels failed";
      return PD_ERR_OOM;
    }
    s->allocs.push_back(f.Lb);
    if (!pdtc::make_map(&f.mapLb, f.Lb, 2, mq, mq, mq, 64)) { s->err = "cuTensorMapEncodeTiled failed"; return PD_ERR_CUDA; }
  }
  pdll::Args a;
  a.map_hi = mode == pdtc::BF16 ? &f.mapLb : &f.mapL;
  a.map_lo = mode == pdtc::TF32X3 ? &f.mapLo : nullptr;
  a.L = f.L; a.Llo = f.Llo; a.Lb = f.Lb; a.Lh = f.Lh; a.Dinv = f.Dinv; a.E = f.E;
  a.mq = mq; a.T = (int)M->T; a.kb = k_begin; a.sync = M->llsync; a.status = s->status; a.piv = M->lpiv;
  a.max_ctas = M->ll_ctas;
  cudaError_t e = pdll::factor(mode, a, s->stream);
  if (e != cudaSuccess) { s->err = std::string("factorisation launch: ") + cudaGetErrorString(e); return PD_ERR_CUDA; }
  f.valid = true;
  return PD_OK;
}

static cudaError_t precond(pd_solver* s, const Factor& f, const double* r, double* z) {
  MixedState* M = s->mixed;
  const int64_t T = M->T;
  cudaMemsetAsync(M->pcnt, 0, sizeof(int) * (2 + 4 * T), s->stream);
  k_pc_pre<<<nblk(3 * M->mq, 256), 256, 0, s->stream>>>(M->mq, s->m, f.d, r, f.iperm, M->facc, M->bacc);
  const int nF = T >= 3 ? (int)((T - 2) * (T - 1) / 2) : 0, ntask = 2 * nF + (int)T;
  k_precond<<<(unsigned)std::min(1 + ntask, M->pc_grid), 256, 0, s->stream>>>(
      f.Lh, f.E, M->mq, M->w, M->uo, M->facc, M->bacc, M->pcnt, s->status);
  k_pc_post<<<nblk(3 * s->m, 256), 256, 0, s->stream>>>(s->m, f.d, M->uo, f.iperm, z);
  pdk::g_launches += 3;
  return cudaGetLastError();
}

// Explicit inverse of the contact-free factor, built once from m/3 solves with
// three unit right-hand sides each; afterwards the preconditioner of the PCG
// form is one dense FP32 matrix-vector product.
static pd_status build_minv(pd_solver* s) {
  MixedState* M = s->mixed;
  if (M->minv_valid) return PD_OK;
  if (!M->Minv0) {
    cudaError_t e = cudaMalloc(&M->Minv0, sizeof(float) * s->m * M->ldm);
    if (e != cudaSuccess) { s->err = "device allocation of the explicit inverse failed"; return PD_ERR_OOM; }
    s->allocs.push_back(M->Minv0);
    cudaMemsetAsync(M->Minv0, 0, sizeof(float) * s->m * M->ldm, s->stream);   // padding columns
  }
  if (!M->f0.valid) {
    factor_cast(s, M->f0, false);
    pd_status r = factor_ll(s, M->f0, pdtc::TF32X3);
    if (r != PD_OK) return r;
  }
  const int64_t m = s->m;
  for (int64_t q = 0; 3 * q < m; ++q) {
    k_unit3<<<nblk(m, 256), 256, 0, s->stream>>>(M->p, m, q);
    cudaError_t ce = precond(s, M->f0, M->p, M->z);
    if (ce != cudaSuccess) { s->err = cudaGetErrorString(ce); return PD_ERR_CUDA; }
    k_store_cols<<<nblk(m, 256), 256, 0, s->stream>>>(M->z, m, M->ldm, q, M->Minv0);
    pdk::g_launches += 2;
  }
  M->minv_valid = true;
  return PD_OK;
}

// (Re)allocate a device buffer owned by the solver (freed in pd_destroy).
static bool dev_realloc(pd_solver* s, void** ptr, size_t bytes) {
  if (*ptr) {
    for (auto it = s->allocs.begin(); it != s->allocs.end(); ++it)
      if (*it == *ptr) { s->allocs.erase(it); break; }
    cudaFree(*ptr);
    *ptr = nullptr;
  }
  if (cudaMalloc(ptr, bytes) != cudaSuccess) { *ptr = nullptr; return false; }
  s->allocs.push_back(*ptr);
  return true;
}

// The capacitance correction for the current springs (PCG form), in two
// parts.  cap_begin (with the refactorisation, on its stream): the active
// springs in slot order and their count, copied to the host behind ev_cap.
// cap_finish (at the solve, once the host has issued the local steps and
// the substitutions, so the host never waits before they are queued): wait
// for the count, which sizes S, then on the solver stream Y = V M0^-1,
// S = I + V M0^-1 V^T and its FP64 Cholesky factor (with the depth-1
// look-ahead of the FP64 form).  Issued on the factor stream instead, to run
// beside the local step and the substitutions, it took as long in total:
// both are FP64-bound and share the same FP64 units.
static pd_status cap_begin(pd_solver* s) {
  MixedState* M = s->mixed;
  M->kact = 0;
  M->cap_pending = false;
  if (!s->pcg_capacitance || s->k <= 0) return PD_OK;
  cudaStream_t st = s->stream;
  if (s->k > M->cap_rows) {
    const int64_t rows = s->k, kp = (rows + 63) / 64 * 64;
    bool ok = dev_realloc(s, (void**)&M->cap_act, sizeof(int) * rows) &&
              dev_realloc(s, (void**)&M->Y, sizeof(float) * rows * M->ldm) &&
              dev_realloc(s, (void**)&M->ccoef, sizeof(double) * pdk::CSLOTS * rows) &&
              dev_realloc(s, (void**)&M->Scap, sizeof(double) * kp * kp) &&
              dev_realloc(s, (void**)&M->Slinv, sizeof(double) * kp * 64) &&
              dev_realloc(s, (void**)&M->ct, sizeof(double) * 3 * kp) &&
              dev_realloc(s, (void**)&M->cy, sizeof(double) * 3 * kp) &&
              dev_realloc(s, (void**)&M->cwork, sizeof(double) * 6 * kp) &&
              dev_realloc(s, (void**)&M->ccnt, sizeof(int) * (2 + 2 * (kp / 64))) &&
              dev_realloc(s, (void**)&M->cpart, sizeof(double) * 3 * s->m * (kp / kCapChunk));
    if (!M->cap_cnt) ok = ok && dev_realloc(s, (void**)&M->cap_cnt, sizeof(int)) &&
                          dev_realloc(s, (void**)&M->cstat, sizeof(int) * 4) &&
                          cudaMallocHost(&M->cap_cnt_h, sizeof(int)) == cudaSuccess &&
                          cudaEventCreateWithFlags(&M->ev_cap, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { s->err = "device allocation for the capacitance correction failed"; return PD_ERR_OOM; }
    M->cap_rows = rows;
  }
  k_cap_active<<<1, 1024, 0, st>>>(s->k, s->c_idx, s->c_s, M->cap_act, M->cap_cnt);
  ++pdk::g_launches;
  cudaMemcpyAsync(M->cap_cnt_h, M->cap_cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaEventRecord(M->ev_cap, st);
  M->cap_pending = true;
  return PD_OK;
}

static pd_status cap_finish(pd_solver* s) {
  MixedState* M = s->mixed;
  M->cap_pending = false;
  if (cudaEventSynchronize(M->ev_cap) != cudaSuccess) { s->err = "capacitance set-up failed"; return PD_ERR_CUDA; }
  const int64_t kact = *M->cap_cnt_h;
  if (kact <= 0) return PD_OK;
  const int64_t kp = (kact + 63) / 64 * 64;
  cudaStream_t st = s->stream;
  s->tbegin(8);
  k_cap_coef<<<nblk(pdk::CSLOTS * kact, 256), 256, 0, st>>>(kact, M->cap_act, s->c_idx, s->c_w, s->c_s, M->ccoef);
  k_cap_rows<<<dim3(nblk(M->ldm / 4, 256), (unsigned)kact), 256, 0, st>>>(M->cap_act, s->c_idx, M->ccoef, M->Minv0,
                                                                          M->ldm, M->Y);
  k_cap_matrix<<<nblk(kp * kp, 256), 256, 0, st>>>(kact, kp, M->cap_act, s->c_idx, M->ccoef, M->Y, M->ldm, M->Scap);
  pdk::g_launches += 3;
  cudaMemsetAsync(M->cstat, 0, sizeof(int) * 4, st);
  pdk::cholesky_fp64(M->Scap, kp, M->Slinv, M->cstat, st, s->la.side ? &s->la : nullptr);
  s->tend();
  M->kact = kact;
  M->cap_kp = kp;
  return PD_OK;
}

// z = P^-1 r with the capacitance correction, acc += r . z; r32 holds r in FP32
static void apply_cap_dot(pd_solver* s, const double* r, double* z, double* acc) {
  MixedState* M = s->mixed;
  cudaStream_t st = s->stream;
  k_minv_apply<<<nblk(32 * s->m, 256), 256, 0, st>>>(M->Minv0, s->m, M->ldm, M->r32, z);
  k_cap_gather<<<nblk(M->kact, 128), 128, 0, st>>>(M->kact, M->cap_act, s->c_idx, M->ccoef, z, M->ct);
  pdk::g_launches += 2;
  pdk::chol_solve_fp64_tasks(M->Scap, M->cap_kp, M->Slinv, M->ct, M->cy, M->kact, M->cwork, M->ccnt, s->status, st);
  const int nch = (int)((M->kact + kCapChunk - 1) / kCapChunk);
  k_cap_part<<<dim3(nblk(s->m, 256), (unsigned)nch), 256, 0, st>>>(s->m, M->kact, M->Y, M->ldm, M->cy, M->cpart);
  k_cap_apply<<<nblk(s->m, 256), 256, 0, st>>>(s->m, nch, M->cpart, z, r, acc);
  pdk::g_launches += 2;
}

static void apply_minv(pd_solver* s, const double* r, double* z) {
  MixedState* M = s->mixed;
  k_to_f32<<<nblk(3 * s->m, 256), 256, 0, s->stream>>>(r, 3 * s->m, M->r32);
  k_minv_apply<<<nblk(32 * s->m, 256), 256, 0, s->stream>>>(M->Minv0, s->m, M->ldm, M->r32, z);
  pdk::g_launches += 2;
}

// q = H p = Sigma_0 p + C_22 p  (double-float Sigma_0 product, FP64 contact term)
// q = H p; Sigma_0 p is also kept (M->sig), for the bookkeeping's Sigma_0 u
// when p is the solve's result
static void hmatvec(pd_solver* s, const double* p, double* q) {
  MixedState* M = s->mixed;
  k_split<<<nblk(3 * s->m, 256), 256, 0, s->stream>>>(p, 3 * s->m, M->vhi, M->vlo);
  k_symv_df<<<nblk(16 * (s->m + 1), 256), 256, 0, s->stream>>>(M->Shi, M->Slo, s->m, M->ldm, M->vhi, M->vlo, q,
                                                               M->sig);
  M->sig_x = p;
  pdk::g_launches += 2;
  if (s->k > 0) {
    k_contact_matvec<<<nblk(s->k, 128), 128, 0, s->stream>>>(s->k, s->c_idx, s->c_w, s->c_s, p, q);
    ++pdk::g_launches;
  }
}

static void dot(pd_solver* s, const double* x, const double* y, int slot) {
  MixedState* M = s->mixed;
  cudaMemsetAsync(M->sc + slot, 0, sizeof(double), s->stream);
  k_dot<<<148, 256, 0, s->stream>>>(x, y, 3 * s->m, M->sc + slot);
  ++pdk::g_launches;
}

static double read_slot(pd_solver* s, int slot) {
  MixedState* M = s->mixed;
  cudaMemcpyAsync(M->sc_h + slot, M->sc + slot, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  cudaStreamSynchronize(s->stream);
  return M->sc_h[slot];
}

static pdtc::Mode form_mode(const pd_solver* s) {
  return s->precision == PD_FP32_IR ? pdtc::TF32X3
         : s->precision == PD_TF32_IR ? pdtc::TF32
         : s->precision == PD_BF16_IR ? pdtc::BF16 : pdtc::TF32X3;
}

// 4.3: contact update + low-precision refactorisation on s->stream (the warm
// PCG form has no per-solve factor; its fixed preconditioner is built once).
// Nested form (pd_set_contact_nodes): D from Sigma_0's diagonal (fixed), the
// region permuted with the spring-free rows first, and the factor's leading
// k0 tiles computed once; the trailing block (the contact-free Schur
// complement) is saved so that each refactorisation starts from it.
static pd_status nested_setup(pd_solver* s, pdtc::Mode mode) {
  MixedState* M = s->mixed;
  Factor& f = M->f;
  const int64_t m = s->m, mq = M->mq, T = M->T;
  cudaStream_t st = s->stream;
  f.k0 = (int)(s->n_fixed_rows / NB);
  const int64_t ntr = mq - (int64_t)f.k0 * NB;
  if (!f.Sp) {
    if (cudaMalloc(&f.Sp, sizeof(float) * mq * mq) != cudaSuccess) {   // room for any trailing block
      s->err = "device allocation for the nested factor failed";
      return PD_ERR_OOM;
    }
    s->allocs.push_back(f.Sp);
  }
  k_hdiag<<<nblk(m, 256), 256, 0, st>>>(s->Sigma0, m, M->hdiag); ++pdk::g_launches;
  k_dscale<<<nblk(mq, 256), 256, 0, st>>>(M->hdiag, m, mq, f.d, s->status); ++pdk::g_launches;
  k_cast_eq_perm<<<dim3((unsigned)T, (unsigned)T), 256, 0, st>>>(s->Sigma0, m, f.d, s->d_iperm, f.L, mq);
  ++pdk::g_launches;
  factor_panels(s, f, mode, 0, f.k0);
  k_block_copy_f32<<<nblk(ntr * ntr, 256), 256, 0, st>>>(f.L, mq, (int64_t)f.k0 * NB, f.Sp, ntr, 0);
  ++pdk::g_launches;
  f.iperm = s->d_iperm;
  M->nested_ready = true;
  M->nested_mode = (int)mode;
  return PD_OK;
}

pd_status mixed_factor(pd_solver* s) {
  pd_status rs = ensure_state(s);
  if (rs != PD_OK) return rs;
  MixedState* M = s->mixed;
  if (s->precision == PD_PCG_WARM) {
    rs = build_minv(s);
    if (rs != PD_OK) return rs;
    return cap_begin(s);
  }
  const pdtc::Mode mode = form_mode(s);
  cudaMemsetAsync(M->lpiv, 0, sizeof(int), s->stream);
  if (s->nested) {
    if (!M->nested_ready || M->nested_mode != (int)mode) {
      rs = nested_setup(s, mode);
      if (rs != PD_OK) return rs;
    }
    Factor& f = M->f;
    const int64_t mq = M->mq, ntr = mq - (int64_t)f.k0 * NB;
    cudaStream_t st = s->stream;
    s->tbegin(2);
    k_block_copy_f32<<<nblk(ntr * ntr, 256), 256, 0, st>>>(f.L, mq, (int64_t)f.k0 * NB, f.Sp, ntr, 1);
    ++pdk::g_launches;
    if (s->k > 0) {
      k_contact_scatter_f32<<<nblk((int64_t)pdk::CSLOTS * pdk::CSLOTS * s->k, 256), 256, 0, st>>>(
          s->k, s->c_idx, s->c_w, s->c_s, f.d, f.L, mq, s->d_perm);
      ++pdk::g_launches;
    }
    s->tend();
    s->tbegin(8);
    rs = factor_ll(s, f, mode, f.k0);
    s->tend();
    return rs;
  }
  M->nested_ready = false;
  M->f.iperm = nullptr;
  s->tbegin(2);
  factor_cast(s, M->f, true);
  s->tend();
  s->tbegin(8);
  rs = factor_ll(s, M->f, mode);
  s->tend();
  return rs;
}

void mixed_nested_changed(pd_solver* s) {
  if (s->mixed) s->mixed->nested_ready = false;
}

pd_status mixed_solve(pd_solver* s, const double* g, const double* u0, double* u) {
  pd_status r = mixed_factor(s);
  if (r != PD_OK) return r;
  return mixed_iterate(s, g, u0, u);
}

// 4.5 with the factor of the last mixed_factor: refinement (split-TF32) or
// factor-preconditioned CG (TF32, BF16, warm PCG) to the relative residual tol.
pd_status mixed_iterate(pd_solver* s, const double* g, const double* u0, double* u) {
  pd_status rs = ensure_state(s);
  if (rs != PD_OK) return rs;
  MixedState* M = s->mixed;
  cudaStream_t st = s->stream;
  const int64_t n3 = 3 * s->m;
  const bool warm = s->precision == PD_PCG_WARM;
  const pdtc::Mode mode = form_mode(s);
  Factor* f = warm ? &M->f0 : &M->f;
  if (warm && M->cap_pending) {
    rs = cap_finish(s);
    if (rs != PD_OK) return rs;
  }
  M->sig_x = nullptr;   // u is about to change
  s->tbegin(4);
  // u = u0 (or 0); r = g - H u (r = g for the zero start, no product).  The
  // scalars the start needs (g.g, r.r; for a supplied start u.r and g.u)
  // come back to the host with the lost-pivot word in one synchronisation.
  if (u0) {
    cudaMemcpyAsync(u, u0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st);
    hmatvec(s, u, M->q);
    k_sub<<<nblk(n3, 256), 256, 0, st>>>(g, M->q, M->r, n3); ++pdk::g_launches;
    dot(s, M->r, M->r, 0);
    dot(s, u, M->r, 6);
    dot(s, g, u, 7);
  } else {
    cudaMemsetAsync(u, 0, sizeof(double) * n3, st);
    cudaMemcpyAsync(M->r, g, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st);
  }
  dot(s, g, g, 4);
  // PCG from zero needs none of these before its first convergence check,
  // which reads g.g with r.r (slot 4 is not reused in the loop)
  const bool defer = warm && !u0;
  double gg = 0.0, tol2 = 0.0, rr = 0.0;
  int lost_pivot = 0;
  if (!defer) {
    cudaMemcpyAsync(M->lpiv_h, M->lpiv, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(M->sc_h, M->sc, sizeof(double) * 8, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    gg = M->sc_h[4];
    lost_pivot = warm ? 0 : *M->lpiv_h;
    tol2 = s->opt.tol * s->opt.tol * (gg > 0 ? gg : 1.0);
    rr = u0 ? M->sc_h[0] : gg;
  }
  if (u0) {
    // CG decreases phi(u) = u^T H u / 2 - g^T u = -(u . r + g . u) / 2 with
    // r = g - H u, and phi(u) - phi(u*) = ||u - u*||_H^2 / 2: a start with
    // phi(u0) >= phi(0) = 0 is farther from the solution in the energy norm
    // than zero (or not finite), and is replaced by zero
    const double phi = -0.5 * (M->sc_h[6] + M->sc_h[7]);
    if (!(phi < 0.0) || !std::isfinite(rr)) {
      cudaMemsetAsync(u, 0, sizeof(double) * n3, st);
      cudaMemcpyAsync(M->r, g, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st);
      rr = gg;
      ++s->starts_rejected;
    }
  }
  int it = 0;
  bool ok = !defer && rr <= tol2;
  // classic refinement for the split-TF32 factor; factor-preconditioned CG
  // for TF32 / BF16, and for any factor that lost a pivot (CG absorbs the few
  // outlier directions a replaced pivot leaves, plain refinement stalls on them)
  const bool use_cg = warm || mode != pdtc::TF32X3 || lost_pivot;
  cudaError_t ce = cudaSuccess;
  if (!ok && !use_cg) {
    // classic refinement: u += M^-1 r; r = g - H u (FP64 vectors; Sigma_0 u in
    // double-float arithmetic from the ~48-bit FP32 pair, the contact term in FP64)
    for (it = 1; it <= s->opt.max_refine; ++it) {
      ce = precond(s, *f, M->r, M->z);
      if (ce != cudaSuccess) break;
      k_add<<<nblk(n3, 256), 256, 0, st>>>(u, M->z, n3); ++pdk::g_launches;
      hmatvec(s, u, M->q);
      k_sub<<<nblk(n3, 256), 256, 0, st>>>(g, M->q, M->r, n3); ++pdk::g_launches;
      dot(s, M->r, M->r, 0);
      rr = read_slot(s, 0);
      if (rr <= tol2 || !std::isfinite(rr)) break;
    }
    ok = rr <= tol2;
  } else if (!ok) {
    // refinement accelerated by preconditioned CG (FP64 vectors, true residual checked at the end);
    // r.z alternates between slots 1 and 5, p.q uses slot 2, each zeroed by the kernel before its use
    auto rzs = [](int64_t k) { return (k & 1) ? 1 : 5; };
    auto minv_dot = [&](int slot) {   // z = M^-1 r, sc[slot] = r.z (slot zeroed beforehand)
      if (warm && M->kact > 0) {
        apply_cap_dot(s, M->r, M->z, M->sc + slot);
      } else if (warm) {
        k_minv_apply_dot<<<nblk(32 * s->m, 256), 256, 0, st>>>(M->Minv0, s->m, M->ldm, M->r32, M->r, M->z,
                                                                M->sc + slot);
        ++pdk::g_launches;
      } else {
        ce = precond(s, *f, M->r, M->z);
        k_dot<<<148, 256, 0, st>>>(M->r, M->z, n3, M->sc + slot);
        ++pdk::g_launches;
      }
    };
    if (warm) { k_to_f32<<<nblk(n3, 256), 256, 0, st>>>(M->r, n3, M->r32); ++pdk::g_launches; }
    cudaMemsetAsync(M->sc + rzs(1), 0, sizeof(double), st);
    minv_dot(rzs(1));
    k_cg_dir2<<<nblk(n3, 256), 256, 0, st>>>(M->p, M->z, M->sc, rzs(1), rzs(1), n3, 1, M->vhi, M->vlo);
    ++pdk::g_launches;
    for (it = 1; it <= s->opt.max_refine && ce == cudaSuccess; ++it) {
      const int sa = rzs(it), sb = rzs(it + 1);
      // q = H p with p already split by k_cg_dir2
      k_symv_df<<<nblk(16 * (s->m + 1), 256), 256, 0, st>>>(M->Shi, M->Slo, s->m, M->ldm, M->vhi, M->vlo, M->q,
                                                            nullptr);
      ++pdk::g_launches;
      M->sig_x = nullptr;   // u changes in this iteration's step
      if (s->k > 0) {
        k_contact_matvec<<<nblk(s->k, 128), 128, 0, st>>>(s->k, s->c_idx, s->c_w, s->c_s, M->p, M->q);
        ++pdk::g_launches;
      }
      k_dot<<<148, 256, 0, st>>>(M->p, M->q, n3, M->sc + 2);
      k_cg_step2<<<nblk(n3, 256), 256, 0, st>>>(u, M->r, M->p, M->q, M->sc, sa, sb, n3, warm ? M->r32 : nullptr);
      pdk::g_launches += 2;
      // the host reads the residual (a stream synchronisation) every iteration
      // for the first eight, then every fourth: a long PCG run pays few round
      // trips for at most three extra iterations.  PCG from zero starts
      // checking one iteration before the count of its previous solve, at
      // most at the fourth (the iterations between cost less than the round
      // trips they save, and an easier solve wastes at most three)
      const int first = defer ? std::min(4, std::max(1, M->cg_hint - 1)) : 1;
      const bool check = (it >= first && (it <= 8 || it % 4 == 0)) || it == s->opt.max_refine;
      if (check) {
        dot(s, M->r, M->r, 0);
        cudaMemcpyAsync(M->sc_h, M->sc, sizeof(double) * 8, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        rr = M->sc_h[0];
        if (defer && gg == 0.0) {
          gg = M->sc_h[4];
          tol2 = s->opt.tol * s->opt.tol * (gg > 0 ? gg : 1.0);
        }
        if (!std::isfinite(rr)) break;
        if (rr <= tol2) {   // confirm with the true residual
          hmatvec(s, u, M->q);
          k_sub<<<nblk(n3, 256), 256, 0, st>>>(g, M->q, M->r, n3); ++pdk::g_launches;
          dot(s, M->r, M->r, 0);
          rr = read_slot(s, 0);
          if (rr <= tol2) break;
          if (warm) { k_to_f32<<<nblk(n3, 256), 256, 0, st>>>(M->r, n3, M->r32); ++pdk::g_launches; }
        }
      }
      minv_dot(sb);
      k_cg_dir2<<<nblk(n3, 256), 256, 0, st>>>(M->p, M->z, M->sc, sa, sb, n3, 0, M->vhi, M->vlo);
      ++pdk::g_launches;
    }
    ok = rr <= tol2;
  }
  s->tend();
  s->last_refine = it;
  if (warm && ok) M->cg_hint = it;
  s->last_residual = std::sqrt(rr / (gg > 0 ? gg : 1.0));
  if (ce != cudaSuccess) {
    s->err = std::string("preconditioner launch failed: ") + cudaGetErrorString(ce);
    return PD_ERR_CUDA;
  }
  if (!ok) {
    int h[4] = {0, 0, 0, 0};
    cudaMemcpy(h, s->status, sizeof h, cudaMemcpyDeviceToHost);
    if (h[0]) {
      s->err = "collision-region matrix has a non-positive diagonal entry " + std::to_string(h[0] - 1);
      return PD_ERR_NOT_SPD;
    }
    if (lost_pivot) {
      s->err = "low-precision Cholesky pivot " + std::to_string(lost_pivot - 1) +
               " was not positive and the refinement did not reach tol";
      s->mixed_escalate = true;
      return PD_ERR_NOT_SPD;
    }
    if (h[1]) {
      s->err = "a bounded device wait gave up (code " + std::to_string(h[1]) + ")";
      return PD_ERR_TIMEOUT;
    }
    char buf[160];
    std::snprintf(buf, sizeof buf, "refinement reached relative residual %.3e after %d iterations (tol %.1e)",
                  s->last_residual, it, s->opt.tol);
    s->err = buf;
    s->mixed_escalate = true;
    return PD_ERR_NO_CONVERGENCE;
  }
  return PD_OK;
}

bool sigma_product(pd_solver* s, const double* p, double* q) {
  MixedState* M = s->mixed;
  if (!M) return false;
  if (p == M->sig_x) {   // the solve's last residual product was of this vector: the same values
    cudaMemcpyAsync(q, M->sig, sizeof(double) * 3 * s->m, cudaMemcpyDeviceToDevice, s->stream);
    return true;
  }
  k_split<<<nblk(3 * s->m, 256), 256, 0, s->stream>>>(p, 3 * s->m, M->vhi, M->vlo);
  k_symv_df<<<nblk(16 * (s->m + 1), 256), 256, 0, s->stream>>>(M->Shi, M->Slo, s->m, M->ldm, M->vhi, M->vlo, q,
                                                               nullptr);
  pdk::g_launches += 2;
  return true;
}

void forget_sigma_product(pd_solver* s) {
  if (s->mixed) s->mixed->sig_x = nullptr;
}

// z = M0^-1 r with the contact-free factor of Sigma_0 (computed on first use).
pd_status apply_free(pd_solver* s, const double* r, double* z) {
  pd_status rs = ensure_state(s);
  if (rs != PD_OK) return rs;
  rs = build_minv(s);
  if (rs != PD_OK) return rs;
  apply_minv(s, r, z);
  return PD_OK;
}

// Diagnostic: a grid barrier that can never complete (the target exceeds the
// grid), with a short poll limit, to exercise the timeout path.
__global__ void k_wait_probe(unsigned* ctr, unsigned limit, int* status) {
  if (threadIdx.x == 0) {
    atomicAdd(ctr, 1u);
    unsigned it = 0;
    while (*(volatile unsigned*)ctr < gridDim.x + 1u) {   // nothing ever adds the last arrival
      if (++it > limit) { atomicExch(status + 1, 201); break; }
      __nanosleep(256);
    }
  }
}

}  // namespace pdm

extern "C" pd_status pd_debug_wait_timeout(pd_solver* s) {
  if (!s) return PD_ERR_INVALID_ARG;
  cudaMemsetAsync(s->status, 0, sizeof(int) * 4, s->stream);
  cudaMemsetAsync(s->status + 3, 0, sizeof(int), s->stream);
  pdm::k_wait_probe<<<4, 32, 0, s->stream>>>(reinterpret_cast<unsigned*>(s->status + 3), 1u << 16, s->status);
  ++pdk::g_launches;
  if (cudaGetLastError() != cudaSuccess) return PD_ERR_CUDA;
  return s->check_status();
}

namespace pdm {

void mixed_free(pd_solver* s) {
  if (!s->mixed) return;
  if (s->mixed->sc_h) cudaFreeHost(s->mixed->sc_h);
  if (s->mixed->lpiv_h) cudaFreeHost(s->mixed->lpiv_h);
  if (s->mixed->cap_cnt_h) cudaFreeHost(s->mixed->cap_cnt_h);
  if (s->mixed->ev_cap) cudaEventDestroy(s->mixed->ev_cap);
  for (auto e : s->mixed->ev_panel) cudaEventDestroy(e);
  for (auto e : s->mixed->ev_rest) cudaEventDestroy(e);
  if (s->mixed->side) cudaStreamDestroy(s->mixed->side);
  delete s->mixed;   // device buffers are in s->allocs
  s->mixed = nullptr;
}

void mixed_invalidate(pd_solver* s) {
  if (s->mixed) s->mixed->f0.valid = false;
}

}  // namespace pdm
