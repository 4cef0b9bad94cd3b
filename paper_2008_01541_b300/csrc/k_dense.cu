// Dense collision-region kernels (Section 3.3; Algorithm 1 steps 4.3-4.7):
// the additive contact update of the Schur complement, the blocked FP64
// Cholesky refactorisation with 64 x 64 tiles, the blocked triangular solves
// for three right-hand sides, and the Sigma matrix-vector products.
// H is stored column-major with leading dimension mp (a multiple of 64); rows
// and columns m..mp-1 hold an identity block, so every tile is full.
#include <algorithm>

#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace pdk {
namespace {

constexpr int TB = 64;

__global__ void k_copy_sigma(const double* __restrict__ S, int64_t m, double* __restrict__ H, int64_t mp) {
  int ti = blockIdx.x, tj = blockIdx.y;
  if (ti < tj) return;
  for (int idx = threadIdx.x; idx < TB * TB; idx += blockDim.x) {
    int r = idx % TB, c = idx / TB;
    int64_t i = (int64_t)ti * TB + r, j = (int64_t)tj * TB + c;
    double v;
    if (i < m && j < m) v = S[i + j * m];
    else v = (i == j) ? 1.0 : 0.0;
    H[i + j * mp] = v;
  }
}

__global__ void k_contact_scatter(int64_t k, int ns, const int32_t* __restrict__ cidx, const double* __restrict__ cw,
                                  const double* __restrict__ cs, double* __restrict__ H, int64_t mp,
                                  const int32_t* __restrict__ perm) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)ns * ns * k) return;
  int64_t j = t / (ns * ns);
  int a = (int)((t / ns) % ns), b = (int)(t % ns);
  int ra = cidx[ns * j + a], rb = cidx[ns * j + b];
  if (ra < 0 || rb < 0) return;
  if (perm) { ra = perm[ra]; rb = perm[rb]; }
  if (ra < rb) return;
  atomicAdd(H + ra + (int64_t)rb * mp, cs[j] * cw[ns * j + a] * cw[ns * j + b]);
}

__global__ void k_contact_forces(int64_t k, int ns, const int32_t* __restrict__ cidx, const double* __restrict__ cw,
                                 const double* __restrict__ ct, const double* __restrict__ cs,
                                 const int32_t* __restrict__ region, const double* __restrict__ x,
                                 double* __restrict__ g) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= k) return;
  double p[3] = {0, 0, 0};
  for (int a = 0; a < ns; ++a) {
    int r = cidx[ns * j + a];
    if (r < 0) continue;
    const double* xv = x + 3 * (int64_t)region[r];
    double w = cw[ns * j + a];
    p[0] += w * xv[0]; p[1] += w * xv[1]; p[2] += w * xv[2];
  }
  double c = cs[j];
  double q[3] = {c * (p[0] - ct[3 * j]), c * (p[1] - ct[3 * j + 1]), c * (p[2] - ct[3 * j + 2])};
  for (int a = 0; a < ns; ++a) {
    int r = cidx[ns * j + a];
    if (r < 0) continue;
    double w = cw[ns * j + a];
    atomicAdd(g + 3 * (int64_t)r, -w * q[0]);
    atomicAdd(g + 3 * (int64_t)r + 1, -w * q[1]);
    atomicAdd(g + 3 * (int64_t)r + 2, -w * q[2]);
  }
}

// Named barrier among the first `n` threads of the block: the producer
// arrives without waiting, the consumers wait.
__device__ __forceinline__ void bar_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_wait(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// Factor the diagonal tile (kt, kt) in shared memory (FP64), blocked by 16
// columns.  On B300 one SM retires 2 FP64 FMAs per clock, a quarter of that
// per sub-partition, and a warp's FP64 instruction holds its sub-partition's
// unit for 64 clocks whatever its active lanes; so the work is spread over
// the four sub-partitions and the serial pivot chain is kept short:
//  (a) 16 x 16 diagonal block: warps 0-3 each hold four of its columns in
//      registers (lane = row); the owner of pivot j first applies pivot j-1
//      to column j, factors it and publishes it (named barrier, the producer
//      only arrives); pivot j-1 reaches the other columns afterwards, off the
//      chain;
//  (b) panel below: two rows per warp, lane = column, forward substitution
//      on the unscaled x_j with the block's columns pre-divided by their
//      pivots (x_t -= x_j L_tj / L_jj), one scaling at the end;
//  (c) trailing update of the lower part: all threads, one entry each.
// Only L_kk is formed; the inverses for the solves come from k_chol_inv.
constexpr int LDA = TB + 1;   // padded column stride of a shared 64 x 64 tile
__global__ void __launch_bounds__(256) k_chol_diag(double* __restrict__ H, int64_t mp, int kt,
                                                   int* __restrict__ status) {
  __shared__ double A[TB * LDA];   // column-major, A[c * LDA + r]
  __shared__ double colb[16][16];  // published columns of the current block: colb[j][i] = L(c0 + i, c0 + j)
  __shared__ double lt[16][16];    // lt[j][t] = L(c0 + t, c0 + j) / L(c0 + j, c0 + j) for t > j, else 0
  __shared__ double rinv[TB];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double* Ht = H + (int64_t)kt * TB + (int64_t)kt * TB * mp;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int idx = tid + 256 * k, r = idx % TB, c = idx / TB;
    A[c * LDA + r] = Ht[r + (int64_t)c * mp];
  }
  __syncthreads();
#pragma unroll 1
  for (int p = 0; p < 4; ++p) {
    const int c0 = 16 * p;
    if (w < 4) {
      // (a) columns w, w + 4, w + 8, w + 12 of the block; lanes 16-31 mirror rows 0-15
      const int i = lane & 15;
      double a[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) a[s] = A[(c0 + w + 4 * s) * LDA + c0 + i];
      unsigned bad = 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int sj = j >> 2;
        if (w == (j & 3)) {
          // register-only selection of slot sj (no local-memory array)
          double cur = sj == 0 ? a[0] : sj == 1 ? a[1] : sj == 2 ? a[2] : a[3];
          if (j > 0) cur = fma(-colb[j - 1][i], colb[j - 1][j], cur);
          double d = __shfl_sync(0xffffffffu, cur, j);
          // positive and finite, tested on the exponent bits (integer unit,
          // not the FP64 pipe); a zero or subnormal pivot counts as failed
          const int hi = __double2hiint(d);
          const bool b = hi < 0x00100000 || hi >= 0x7ff00000;
          bad |= (unsigned)b << j;
          d = b ? 1.0 : d;
          const double rs = rsqrt(d);
          const double v = i >= j ? (b && i == j ? 1.0 : cur) * rs : 0.0;   // row j: cur = d, so L_jj = d / sqrt(d)
#pragma unroll
          for (int s2 = 0; s2 < 4; ++s2) a[s2] = s2 == sj ? v : a[s2];
          if (lane < 16) {
            colb[j][i] = v;
            if (i == j) rinv[c0 + j] = rs;
          }
          __syncwarp();
          bar_arrive(1 + (j & 7), 128);
        }
        if (j > 0) {
          // pivot j - 1 on this warp's columns after j
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int c = w + 4 * s;
            if (c > j) a[s] = fma(-colb[j - 1][i], colb[j - 1][c], a[s]);
          }
        }
        if (w != (j & 3)) bar_wait(1 + (j & 7), 128);
      }
      if (lane < 16) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int c = w + 4 * s;
          if (i >= c) A[(c0 + c) * LDA + c0 + i] = a[s];
        }
      }
      if (bad && lane == 0) atomicCAS(status, 0, kt * TB + c0 + __ffs(bad));
    }
    __syncthreads();
    const int nb = TB - c0 - 16;
    if (nb > 0) {
      // (b) rows c0 + 16 .. 63: X L_D^T = A_panel
      lt[tid >> 4][tid & 15] = (tid & 15) > (tid >> 4) ? colb[tid >> 4][tid & 15] * rinv[c0 + (tid >> 4)] : 0.0;
      __syncthreads();
      const int t = lane & 15, h = lane >> 4;
      for (int pr = w; 2 * pr < nb; pr += 8) {
        const int row = c0 + 16 + 2 * pr + h;
        double x = A[(c0 + t) * LDA + row];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const double xj = __shfl_sync(0xffffffffu, x, (h << 4) + j);
          x = fma(-xj, lt[j][t], x);
        }
        A[(c0 + t) * LDA + row] = x * rinv[c0 + t];
      }
      __syncthreads();
      // (c) trailing update of rows / columns >= c0 + 16 (lower part), one
      // entry per thread step: q runs over the nb (nb + 1) / 2 lower entries
      for (int q = tid; q < nb * (nb + 1) / 2; q += 256) {
        int c = (int)((sqrtf((float)(8 * q + 1)) - 1.f) * 0.5f);   // row of the triangle (entry q)
        while (c * (c + 1) / 2 > q) --c;
        while ((c + 1) * (c + 2) / 2 <= q) ++c;
        const int r = c0 + 16 + c, cc = c0 + 16 + (q - c * (c + 1) / 2);
        double acc = 0.0;
#pragma unroll
        for (int t2 = 0; t2 < 16; ++t2) acc = fma(A[(c0 + t2) * LDA + r], A[(c0 + t2) * LDA + cc], acc);
        A[cc * LDA + r] -= acc;
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int idx = tid + 256 * k, r = idx % TB, c = idx / TB;
    if (r >= c) Ht[r + (int64_t)c * mp] = A[c * LDA + r];
  }
}

// Linv_kk = L_kk^-1 for every diagonal tile (blockIdx.x = k), column-major;
// thread c solves L z = e_c with precomputed reciprocals of the diagonal.
__global__ void __launch_bounds__(64) k_chol_inv(const double* __restrict__ H, int64_t mp,
                                                 double* __restrict__ Linv, int k0) {
  __shared__ double A[TB * LDA];
  __shared__ double rinv[TB];
  const int kt = k0 + blockIdx.x, c = threadIdx.x;
  const double* Ht = H + (int64_t)kt * TB + (int64_t)kt * TB * mp;
  for (int idx = c; idx < TB * TB; idx += TB) {
    const int r = idx % TB, cc = idx / TB;
    A[cc * LDA + r] = r >= cc ? Ht[r + (int64_t)cc * mp] : 0.0;
  }
  __syncthreads();
  rinv[c] = 1.0 / A[c * LDA + c];
  __syncthreads();
  double* Z = Linv + (int64_t)kt * TB * TB + (int64_t)c * TB;   // column c
  for (int i = 0; i < c; ++i) Z[i] = 0.0;
  // right-looking: z_i final after scaling, then eliminated from rows below
  double z[TB];
#pragma unroll
  for (int i = 0; i < TB; ++i) z[i] = (i == c) ? 1.0 : 0.0;
#pragma unroll
  for (int i = 0; i < TB; ++i) {
    if (i >= c) {
      z[i] *= rinv[i];
#pragma unroll
      for (int t = i + 1; t < TB; ++t) z[t] = fma(-z[i], A[i * LDA + t], z[t]);
    }
  }
#pragma unroll
  for (int i = 0; i < TB; ++i)
    if (i >= c) Z[i] = z[i];
}

// L_ik = A_ik L_kk^-T for tiles i > kt by forward substitution: CTA
// (blockIdx.x / 16) takes tile i = kt + 1 + blockIdx.x / 16, rows
// 4 * (blockIdx.x % 16) .. + 3, one warp per row with columns lane and
// lane + 32 in registers.  Column j of L_kk is staged divided by L_jj and
// zero on and above the diagonal, so every step is the same unpredicated
// FMAs on the still unscaled x_j (x_t -= x_j L_tj / L_jj, exact in order),
// and x is scaled by 1 / L_tt once at the end.  One warp per SM sub-partition:
// on B300 a warp's FP64 instruction occupies its sub-partition's FP64 unit
// for 64 clocks whatever its active lanes, so this keeps the chain short.
__global__ void __launch_bounds__(128) k_chol_trsm(double* __restrict__ H, int64_t mp, int kt) {
  __shared__ double Ls[TB * TB];   // Ls[j * TB + t] = L_tj / L_jj for t > j, else 0
  __shared__ double rinv[TB];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const double* Lt = H + (int64_t)kt * TB + (int64_t)kt * TB * mp;
  const int64_t it = kt + 1 + blockIdx.x / 16;
  const int row = 4 * (blockIdx.x % 16) + w;
  double* Ai = H + it * TB + row + (int64_t)kt * TB * mp;   // column c of this row at c * mp
  double x0 = Ai[(int64_t)lane * mp], x1 = Ai[(int64_t)(lane + 32) * mp];
  if (tid < TB) rinv[tid] = 1.0 / Lt[tid + (int64_t)tid * mp];
  __syncthreads();
#pragma unroll 16
  for (int k = 0; k < TB * TB / 128; ++k) {
    const int q = tid + 128 * k, t = q % TB, j = q / TB;
    Ls[q] = t > j ? Lt[t + (int64_t)j * mp] * rinv[j] : 0.0;
  }
  __syncthreads();
#pragma unroll 8
  for (int j = 0; j < 32; ++j) {
    const double xj = __shfl_sync(0xffffffffu, x0, j);
    x0 = fma(-xj, Ls[j * TB + lane], x0);
    x1 = fma(-xj, Ls[j * TB + 32 + lane], x1);
  }
#pragma unroll 8
  for (int j = 32; j < TB; ++j) {
    const double xj = __shfl_sync(0xffffffffu, x1, j - 32);
    x1 = fma(-xj, Ls[j * TB + 32 + lane], x1);
  }
  Ai[(int64_t)lane * mp] = x0 * rinv[lane];
  Ai[(int64_t)(lane + 32) * mp] = x1 * rinv[lane + 32];
}

// Column update of the look-ahead: rows 4 * (blockIdx.x % 16) .. + 3 of tile
// (kt + 1 + blockIdx.x / 16, kt + 1) -= L_ik L_(kt+1)k^T; one warp per row,
// output columns lane and lane + 32.
__global__ void __launch_bounds__(128) k_chol_colupd(double* __restrict__ H, int64_t mp, int kt) {
  __shared__ double Bs[TB * LDA];  // Bs[t * LDA + c] = L_(kt+1)k (row c, column t)
  __shared__ double As[4][TB];     // the CTA's 4 rows of L_ik
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int64_t it = kt + 1 + blockIdx.x / 16, jt = kt + 1;
  const int row = 4 * (blockIdx.x % 16) + w;
  const double* Lj = H + jt * TB + (int64_t)kt * TB * mp;
  const double* Li = H + it * TB + row + (int64_t)kt * TB * mp;
#pragma unroll 16
  for (int k = 0; k < TB * TB / 128; ++k) {
    const int q = tid + 128 * k, c = q % TB, t = q / TB;
    Bs[t * LDA + c] = Lj[c + (int64_t)t * mp];
  }
  As[w][lane] = Li[(int64_t)lane * mp];
  As[w][lane + 32] = Li[(int64_t)(lane + 32) * mp];
  __syncthreads();
  double a0 = 0.0, a1 = 0.0;
#pragma unroll 8
  for (int t = 0; t < TB; ++t) {
    const double at = As[w][t];
    a0 = fma(at, Bs[t * LDA + lane], a0);
    a1 = fma(at, Bs[t * LDA + lane + 32], a1);
  }
  double* Aij = H + it * TB + row + jt * TB * mp;
  Aij[(int64_t)lane * mp] -= a0;
  Aij[(int64_t)(lane + 32) * mp] -= a1;
}

// A_ij -= L_ik L_jk^T for the tiles selected by the launch: lower != 0 ->
// tiles it0 + ii, jt0 + jj with jj <= ii (triangular numbering); else an
// n_i x n_j rectangle starting at (it0, jt0).  S CTAs share a tile, each
// taking 64 / S of its rows, so that small trailing matrices still spread
// over the SMs (one SM retires a 64 x 64 x 64 FP64 tile in ~65 us).
template <int S>
__global__ void __launch_bounds__(256) k_chol_update(double* __restrict__ H, int64_t mp, int kt, int it0, int jt0,
                                                     int n_j, int lower) {
  constexpr int R = TB / S, RA = R / 16;
  extern __shared__ double sm[];
  double* As = sm;            // As[t * R + r]: the CTA's rows of L_ik
  double* Bs = sm + TB * R;   // Bs[t * TB + c]: L_jk
  const int tid = threadIdx.x;
  int64_t idx = blockIdx.x / S, ii, jj;
  const int r0 = R * (int)(blockIdx.x % S);
  if (lower) {
    ii = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= idx) ++ii;
    while (ii * (ii + 1) / 2 > idx) --ii;
    jj = idx - ii * (ii + 1) / 2;
  } else {
    ii = idx / n_j;
    jj = idx % n_j;
  }
  const int64_t it = it0 + ii, jt = jt0 + jj;
  const double* Li = H + it * TB + r0 + (int64_t)kt * TB * mp;
  const double* Lj = H + jt * TB + (int64_t)kt * TB * mp;
  for (int q = tid; q < R * TB; q += 256) {
    const int r = q % R, t = q / R;
    As[q] = Li[r + (int64_t)t * mp];
  }
  for (int q = tid; q < TB * TB; q += 256) {
    const int c = q % TB, t = q / TB;
    Bs[q] = Lj[c + (int64_t)t * mp];
  }
  __syncthreads();
  const int tr = tid % 16, tc = tid / 16;
  double acc[RA][4] = {};
#pragma unroll 8
  for (int t = 0; t < TB; ++t) {
    double a[RA], b[4];
#pragma unroll
    for (int p = 0; p < RA; ++p) a[p] = As[t * R + tr + 16 * p];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = Bs[t * TB + tc + 16 * q];
#pragma unroll
    for (int p = 0; p < RA; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
  }
  double* Aij = H + it * TB + r0 + jt * TB * mp;
#pragma unroll
  for (int p = 0; p < RA; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) Aij[(tr + 16 * p) + (int64_t)(tc + 16 * q) * mp] -= acc[p][q];
}

// Lower-triangular trailing update of n x n tiles from (t0, t0) with panel kt.
// S CTAs per tile (S = 1, 2, 4) trade panel reloads for finer work units:
// each launch takes the S whose whole waves of resident CTAs cover its tiles
// with the least idle capacity, cost_S = ceil(S tiles / slots_S) slots_S / S
// in units of one SM's time per tile (one wave of a partly used grid leaves
// the rest of the FP64 units idle until the next launch).
void launch_update(double* H, int64_t mp, int kt, int t0, int n, cudaStream_t st) {
  const int64_t tiles = (int64_t)n * (n + 1) / 2;
  if (tiles <= 0) return;
  static int slots[64][3];   // resident CTAs per device for S = 1, 2, 4
  int dev = 0;
  cudaGetDevice(&dev);
  int* sl = slots[dev & 63];
  if (sl[0] == 0) {
    int nsm = 0, p1 = 0, p2 = 0, p4 = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_chol_update<1>, 256, 2 * TB * TB * sizeof(double));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, k_chol_update<2>, 256, (TB / 2 + TB) * TB * sizeof(double));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p4, k_chol_update<4>, 256, (TB / 4 + TB) * TB * sizeof(double));
    sl[1] = std::max(1, nsm * p2);
    sl[2] = std::max(1, nsm * p4);
    sl[0] = std::max(1, nsm * p1);
  }
  int best = 0;
  double best_cost = 0.0;
  for (int v = 0; v < 3; ++v) {
    const int S = 1 << v;
    const int64_t units = S * tiles;
    const double cost = (double)((units + sl[v] - 1) / sl[v]) * sl[v] / S;
    if (v == 0 || cost < best_cost) { best = v; best_cost = cost; }
  }
  if (best == 0) {
    k_chol_update<1><<<(unsigned)tiles, 256, 2 * TB * TB * sizeof(double), st>>>(H, mp, kt, t0, t0, 0, 1);
  } else if (best == 1) {
    k_chol_update<2><<<(unsigned)(2 * tiles), 256, (TB / 2 + TB) * TB * sizeof(double), st>>>(H, mp, kt, t0, t0,
                                                                                              0, 1);
  } else {
    k_chol_update<4><<<(unsigned)(4 * tiles), 256, (TB / 4 + TB) * TB * sizeof(double), st>>>(H, mp, kt, t0, t0,
                                                                                              0, 1);
  }
  ++g_launches;
}

// Forward step kt: y_k = Linv_kk w_k (block 0 stores it), w_i -= L_ik y_k for i = kt + blockIdx.x
__global__ void __launch_bounds__(192) k_trsv_fwd(const double* __restrict__ H, int64_t mp, int kt,
                                                  const double* __restrict__ Linv, double* __restrict__ w,
                                                  double* __restrict__ y) {
  __shared__ double yk[TB * 3];
  const int tid = threadIdx.x, r = tid / 3, v = tid % 3;
  const double* Lk = Linv + (int64_t)kt * TB * TB;
  const double* wk = w + (int64_t)kt * TB * 3;
  double s = 0.0;
  for (int c = 0; c <= r; ++c) s += Lk[r + c * TB] * wk[3 * c + v];
  yk[tid] = s;
  __syncthreads();
  if (blockIdx.x == 0) {
    y[(int64_t)kt * TB * 3 + tid] = s;
    return;
  }
  const int64_t it = kt + blockIdx.x;
  const double* Lik = H + it * TB + (int64_t)kt * TB * mp;
  double acc = 0.0;
  for (int c = 0; c < TB; ++c) acc += Lik[r + (int64_t)c * mp] * yk[3 * c + v];
  w[it * TB * 3 + tid] -= acc;
}

// Backward step kt: u_k = Linv_kk^T w_k (block 0 stores it), w_j -= L_kj^T u_k for j = blockIdx.x - 1
__global__ void __launch_bounds__(192) k_trsv_bwd(const double* __restrict__ H, int64_t mp, int kt,
                                                  const double* __restrict__ Linv, double* __restrict__ w,
                                                  double* __restrict__ u) {
  __shared__ double uk[TB * 3];
  const int tid = threadIdx.x, r = tid / 3, v = tid % 3;
  const double* Lk = Linv + (int64_t)kt * TB * TB;
  const double* wk = w + (int64_t)kt * TB * 3;
  double s = 0.0;
  for (int c = r; c < TB; ++c) s += Lk[c + r * TB] * wk[3 * c + v];
  uk[tid] = s;
  __syncthreads();
  if (blockIdx.x == 0) {
    u[(int64_t)kt * TB * 3 + tid] = s;
    return;
  }
  const int64_t jt = blockIdx.x - 1;
  const double* Lkj = H + (int64_t)kt * TB + jt * TB * mp;
  double acc = 0.0;
  for (int c = 0; c < TB; ++c) acc += Lkj[c + (int64_t)r * mp] * uk[3 * c + v];
  w[jt * TB * 3 + tid] -= acc;
}

__global__ void k_pad_rhs(const double* g, int64_t m, int64_t mp, double* w) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < 3 * mp) w[i] = i < 3 * m ? g[i] : 0.0;
}
// w[perm[r]] = g[r] (region index r -> factor position)
__global__ void k_perm_scatter(const double* g, int64_t m, const int32_t* perm, double* w) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int64_t p = perm[r];
  w[3 * p] = g[3 * r]; w[3 * p + 1] = g[3 * r + 1]; w[3 * p + 2] = g[3 * r + 2];
}
__global__ void k_perm_gather(const double* y, int64_t m, const int32_t* perm, double* u) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int64_t p = perm[r];
  u[3 * r] = y[3 * p]; u[3 * r + 1] = y[3 * p + 1]; u[3 * r + 2] = y[3 * p + 2];
}
// H (mp x mp, column-major, full) = P S P^T with identity padding: entry
// (pi, pj) of H is S[iperm[pi]][iperm[pj]] for pi, pj < m
__global__ void k_permute_sym(const double* __restrict__ S, int64_t m, const int32_t* __restrict__ iperm,
                              double* __restrict__ H, int64_t mp) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= mp * mp) return;
  const int64_t pi = q % mp, pj = q / mp;
  H[q] = (pi < m && pj < m) ? S[(int64_t)iperm[pi] * m + iperm[pj]] : (pi == pj ? 1.0 : 0.0);
}
// copy the trailing n x n block at (off, off) of H to or from a dense buffer
__global__ void k_block_copy(double* __restrict__ H, int64_t mp, int64_t off, double* __restrict__ B, int64_t n,
                             int to_h) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int64_t i = q % n, j = q / n;
  double* h = H + (off + i) + (off + j) * mp;
  if (to_h) *h = B[q];
  else B[q] = *h;
}

__global__ void k_symv3(const double* __restrict__ S, int64_t m, const double* __restrict__ v,
                        double* __restrict__ out) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= m) return;
  const double* row = S + i * m;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t j = lane; j < m; j += 32) {
    double s = row[j];
    a0 += s * v[3 * j]; a1 += s * v[3 * j + 1]; a2 += s * v[3 * j + 2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) { out[3 * i] = a0; out[3 * i + 1] = a1; out[3 * i + 2] = a2; }
}

__global__ void k_spmv3(int64_t m, const int64_t* __restrict__ ptr, const int32_t* __restrict__ row,
                        const double* __restrict__ val, const double* __restrict__ v, double alpha,
                        double* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    double s = val[q];
    int64_t j = row[q];
    a0 += s * v[3 * j]; a1 += s * v[3 * j + 1]; a2 += s * v[3 * j + 2];
  }
  out[3 * i] += alpha * a0; out[3 * i + 1] += alpha * a1; out[3 * i + 2] += alpha * a2;
}


// ---- triangular solves of L L^T u = g as dependency-counter tasks ---------
// Forward, for i = 0 .. T-1: task D(i) waits for the i updates into w_i,
// then y_i = Linv_ii w_i; tasks U(i, j), j > i, wait for D(i), then
// w_j -= L_ji y_i.  Backward mirrors it with u_i = Linv_ii^T z_i and
// z_j -= L_ij^T u_i, j < i.  Tasks are numbered block row by block row
// (D(i) first) and claimed in that order by a persistent grid, so every wait
// is on an earlier, already claimed task.  Counters: cnt[0] claim,
// cnt[1 + i] updates received by block i, cnt[1 + T + i] block i solved.
// Waits are bounded (code 302 in status[1]).
__device__ __forceinline__ unsigned long long dtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void wait_ge(const int* c, int target, int* status) {
  const unsigned long long t0 = dtimer();
  unsigned it = 0;
  while (*(volatile const int*)c < target) {
    if (*(volatile int*)(status + 1) != 0) return;
    if (++it > 32) __nanosleep(64);
    if ((it & 1023u) == 0 && dtimer() - t0 > 1000000000ull) {
      atomicCAS(status + 1, 0, 302);
      return;
    }
  }
}

// Update tasks of one triangular solve over T block rows (solve order b):
// block row b applies y_i to the block rows two or more steps ahead (the
// update into the adjacent row is done by the chain block itself).
__host__ __device__ inline int trsv_ntask(int T) { return T >= 3 ? (T - 2) * (T - 1) / 2 : 0; }
__device__ inline int trsv_start(int T, int b) { return b * (T - 2) - b * (b - 1) / 2; }
__device__ inline void trsv_decode(int t, int T, int& b, int& q) {
  const double d = 2.0 * T - 3.0;
  int e = (int)floor(0.5 * (d - sqrt(fmax(d * d - 8.0 * t, 0.0))));
  e = max(0, min(e, T - 3));
  while (e > 0 && trsv_start(T, e) > t) --e;
  while (e < T - 3 && trsv_start(T, e + 1) <= t) ++e;
  b = e;
  q = t - trsv_start(T, e);
}

// 64 x 64 FP64 tile (column-major in global, leading dimension ld) into
// shared memory as tile[row][col] with a padded row.
__device__ __forceinline__ void stage64(double (*tile)[LDA], const double* __restrict__ src, int64_t ld) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int q = threadIdx.x + 256 * k, rr = q % TB, cc = q / TB;
    tile[rr][cc] = __ldg(src + rr + (int64_t)cc * ld);
  }
}

// One direction of the dense triangular solve with the tiled factor in H
// (lower, column-major; diagonal tiles replaced by their inverses in Linv),
// three right-hand sides, in one persistent launch of 8-CTA clusters.  The
// first cluster to start becomes the chain: for every block row in solve
// order its eight CTAs (8 rows each, on eight SMs, since one SM retires only
// 2 FP64 FMAs per clock) subtract the adjacent row's contribution, exchange
// the 64 x 3 right-hand side through distributed shared memory, apply the
// diagonal inverse and exchange y_i, keeping y on chip; the next step's row
// slices are loaded into registers during the current one.  The other CTAs
// claim the remaining updates in list order, so each waits only on the chain
// or on tasks claimed before it and the schedule cannot deadlock.
//   forward : y_i = L_ii^-1 (w_i - L_i,i-1 y_i-1); update (i, j >= i+2): w_j -= L_ji y_i
//   backward: y_i = L_ii^-T (w_i - L_i+1,i^T y_i+1); update (i, j <= i-2): w_j -= L_ij^T y_i
// cnt[0] claims updates, cnt[1 + j] counts the updates applied to w_j,
// cnt[1 + T + i] counts the chain CTAs that wrote y_i, cnt[1 + 2T] assigns
// the chain.
constexpr int CK = 8;            // CTAs of the chain cluster
constexpr int CR = TB / CK;      // rows per chain CTA
template <bool FWD>
__global__ void __cluster_dims__(CK, 1, 1) __launch_bounds__(256)
    k_trsv_tasks(const double* __restrict__ H, int64_t mp, const double* __restrict__ Linv, double* w, double* y,
                 int* cnt, int* status) {
  extern __shared__ double trsv_smem[];
  __shared__ double yfull[TB][3];   // y of the previous chain step (all 64 rows)
  __shared__ double vfull[TB][3];   // right-hand side of the current diagonal step
  __shared__ int cur_t, role;
  const int T = (int)(mp / TB), tid = threadIdx.x;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  if (rank == 0 && tid == 0) role = atomicAdd(cnt + 1 + 2 * T, 1);
  cl.sync();
  const bool chain = *cl.map_shared_rank(&role, 0) == 0;
  cl.sync();    // rank 0's shared memory stays alive until every CTA has read it
  if (chain) {
    // this CTA's output rows r0 .. r0 + CR - 1 of every block row; sa / sn hold
    // the operand rows of the diagonal inverse / the adjacent tile so that
    // out[rr] = sum_c s[rr][c] vec[c] in both directions
    double (*sa)[LDA] = reinterpret_cast<double (*)[LDA]>(trsv_smem);
    double (*sn)[LDA] = reinterpret_cast<double (*)[LDA]>(trsv_smem + CR * LDA);
    const int r0 = CR * (int)rank;
    constexpr int NF = CR * TB / 256;   // operand entries per thread and tile
    double pa[NF], pn[NF];
    auto fetch = [&](int i) {
      const double* Li = Linv + (int64_t)i * TB * TB;
      const bool has = FWD ? i > 0 : i < T - 1;
      // forward: rows of L_i,i-1 and of Linv_ii; backward: columns of L_i+1,i and of Linv_ii
      const double* An = !has ? nullptr
                         : FWD ? H + (int64_t)i * TB + (int64_t)(i - 1) * TB * mp
                               : H + (int64_t)(i + 1) * TB + (int64_t)i * TB * mp;
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const int e = tid + 256 * k, rr = e % CR, c = e / CR;   // FWD: coalesced down a column
        const int f = tid + 256 * k, c2 = f % TB, rr2 = f / TB; // BWD: coalesced down a column
        if (FWD) {
          pa[k] = __ldg(Li + (r0 + rr) + c * TB);
          pn[k] = has ? __ldg(An + (r0 + rr) + (int64_t)c * mp) : 0.0;
        } else {
          pa[k] = __ldg(Li + c2 + (r0 + rr2) * TB);
          pn[k] = has ? __ldg(An + c2 + (int64_t)(r0 + rr2) * mp) : 0.0;
        }
      }
    };
    auto park = [&]() {
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const int e = tid + 256 * k;
        const int rr = FWD ? e % CR : e / TB, c = FWD ? e / CR : e % TB;
        sa[rr][c] = pa[k];
        sn[rr][c] = pn[k];
      }
    };
    // output (rr, v) of the slice, contraction quarter q4 = lanes of a group of 4
    const int g = tid >> 2, q4 = tid & 3, rr = g / 3, v = g % 3;
    const bool act = tid < 3 * CR * 4;
    fetch(FWD ? 0 : T - 1);
    park();
    __syncthreads();
    for (int b = 0; b < T; ++b) {
      const int i = FWD ? b : T - 1 - b;
      if (b + 1 < T) fetch(FWD ? i + 1 : i - 1);         // in flight during this step
      if (tid == 0) {
        wait_ge(cnt + 1 + i, b >= 1 ? b - 1 : 0, status);
        __threadfence();
      }
      __syncthreads();
      double acc = 0.0;
      if (act && b > 0) {
#pragma unroll
        for (int c = 16 * q4; c < 16 * q4 + 16; ++c) acc = fma(sn[rr][c], yfull[c][v], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (act && q4 == 0) {
        const double val = __ldcg(w + 3 * ((int64_t)i * TB + r0 + rr) + v) - acc;
#pragma unroll
        for (int d = 0; d < CK; ++d) cl.map_shared_rank(&vfull[0][0], d)[3 * (r0 + rr) + v] = val;
      }
      cl.sync();
      acc = 0.0;
      if (act) {
#pragma unroll
        for (int c = 16 * q4; c < 16 * q4 + 16; ++c) acc = fma(sa[rr][c], vfull[c][v], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (act && q4 == 0) {
        y[3 * ((int64_t)i * TB + r0 + rr) + v] = acc;
        __threadfence();
#pragma unroll
        for (int d = 0; d < CK; ++d) cl.map_shared_rank(&yfull[0][0], d)[3 * (r0 + rr) + v] = acc;
      }
      __syncthreads();
      if (tid == 0) atomicAdd(cnt + 1 + T + i, 1);
      if (b + 1 < T) park();
      cl.sync();    // yfull complete in every CTA, vfull and sa / sn free
    }
    return;
  }
  double (*ta)[LDA] = reinterpret_cast<double (*)[LDA]>(trsv_smem);
  const int r = tid / 3, v = tid % 3;          // output row / component (tid < 192)
  const int ntask = trsv_ntask(T);
  int ahead = 0;
  if (tid == 0) ahead = atomicAdd(cnt, 1);
  for (;;) {
    if (tid == 0) {
      cur_t = ahead;
      if (ahead < ntask) ahead = atomicAdd(cnt, 1);
    }
    __syncthreads();
    const int t = cur_t;
    if (t >= ntask) break;
    int b, q;
    trsv_decode(t, T, b, q);
    const int i = FWD ? b : T - 1 - b;
    const int j = FWD ? i + 2 + q : i - 2 - q;
    // forward update (i, j) reads L_ji, backward reads L_ij; staged before the wait
    stage64(ta, FWD ? H + (int64_t)j * TB + (int64_t)i * TB * mp : H + (int64_t)i * TB + (int64_t)j * TB * mp, mp);
    if (tid == 0) {
      wait_ge(cnt + 1 + T + i, CK, status);
      __threadfence();
    }
    __syncthreads();
    if (tid < TB * 3) yfull[r][v] = __ldcg(y + 3 * ((int64_t)i * TB) + tid);
    __syncthreads();
    if (tid < TB * 3) {
      double acc = 0.0;
      if (FWD) {
#pragma unroll 8
        for (int c = 0; c < TB; ++c) acc = fma(ta[r][c], yfull[c][v], acc);
      } else {
#pragma unroll 8
        for (int c = 0; c < TB; ++c) acc = fma(ta[c][r], yfull[c][v], acc);
      }
      atomicAdd(w + 3 * ((int64_t)j * TB) + tid, -acc);
      __threadfence();
    }
    __syncthreads();
    if (tid == 0) atomicAdd(cnt + 1 + j, 1);
  }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void copy_sigma(const double* S, int64_t m, double* H, int64_t mp, cudaStream_t st) {
  dim3 grid((unsigned)(mp / TB), (unsigned)(mp / TB));
  k_copy_sigma<<<grid, 256, 0, st>>>(S, m, H, mp);
  ++g_launches;
}

void permute_sym(const double* S, int64_t m, const int32_t* iperm, double* H, int64_t mp, cudaStream_t st) {
  k_permute_sym<<<nblk(mp * mp, 256), 256, 0, st>>>(S, m, iperm, H, mp);
  ++g_launches;
}

void block_copy(double* H, int64_t mp, int64_t off, double* B, int64_t n, bool to_h, cudaStream_t st) {
  if (n <= 0) return;
  k_block_copy<<<nblk(n * n, 256), 256, 0, st>>>(H, mp, off, B, n, to_h ? 1 : 0);
  ++g_launches;
}

void contact_scatter(int64_t k, const int32_t* cidx, const double* cw, const double* cs, double* H,
                     int64_t mp, cudaStream_t st, int ns, const int32_t* perm) {
  if (k > 0) {
    k_contact_scatter<<<nblk((int64_t)ns * ns * k, 256), 256, 0, st>>>(k, ns, cidx, cw, cs, H, mp, perm);
    ++g_launches;
  }
}

void contact_forces(int64_t k, const int32_t* cidx, const double* cw, const double* ct, const double* cs,
                    const int32_t* region, const double* x, double* g, cudaStream_t st, int ns) {
  if (k > 0) {
    k_contact_forces<<<nblk(k, 128), 128, 0, st>>>(k, ns, cidx, cw, ct, cs, region, x, g);
    ++g_launches;
  }
}

void cholesky_fp64(double* H, int64_t mp, double* Linv, int* status, cudaStream_t st, const LookAhead* la, int k_begin,
                   int k_end) {
  static std::atomic<unsigned long long> attr{0};
  const int smem = 2 * TB * TB * sizeof(double);
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(k_chol_update<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_chol_update<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_chol_update<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  }
  const int T = (int)(mp / TB);
  if (k_end < 0 || k_end > T) k_end = T;
  if (k_begin >= k_end) return;
  if (!la || (int64_t)la->ev_panel.size() < T) {   // plain right-looking order on one stream
    for (int k = k_begin; k < k_end; ++k) {
      k_chol_diag<<<1, 256, 0, st>>>(H, mp, k, status);
      ++g_launches;
      int n = T - k - 1;
      if (n <= 0) break;
      k_chol_trsm<<<16 * n, 128, 0, st>>>(H, mp, k);
      ++g_launches;
      launch_update(H, mp, k, k + 1, n, st);
    }
  } else {
    // Depth-1 look-ahead: the main stream factors tile k, solves panel k and
    // updates only block column k+1 (in 16-row slices, to keep this chain
    // short); the low-priority side stream applies panel k to the rest of
    // the trailing matrix while tile k+1 is being factored.
    for (int k = k_begin; k < k_end; ++k) {
      k_chol_diag<<<1, 256, 0, st>>>(H, mp, k, status);
      ++g_launches;
      int n = T - k - 1;
      if (n <= 0) break;
      k_chol_trsm<<<16 * n, 128, 0, st>>>(H, mp, k);
      ++g_launches;
      cudaEventRecord(la->ev_panel[k], st);
      if (k > k_begin) cudaStreamWaitEvent(st, la->ev_rest[k - 1], 0);
      k_chol_colupd<<<16 * n, 128, 0, st>>>(H, mp, k);
      ++g_launches;
      cudaStreamWaitEvent(la->side, la->ev_panel[k], 0);
      launch_update(H, mp, k, k + 2, n - 1, la->side);
      cudaEventRecord(la->ev_rest[k], la->side);
    }
    const int last = k_end == T ? T - 2 : k_end - 1;   // the last step that recorded ev_rest
    if (last >= k_begin) cudaStreamWaitEvent(st, la->ev_rest[last], 0);
  }
  k_chol_inv<<<(unsigned)(k_end - k_begin), 64, 0, st>>>(H, mp, Linv, k_begin);
  ++g_launches;
}

void chol_solve_fp64_tasks(const double* H, int64_t mp, const double* Linv, const double* g, double* u,
                           int64_t m, double* work, int* cnt, int* status, cudaStream_t st, const int32_t* perm) {
  static std::atomic<unsigned long long> attr{0};
  const int smem = TB * LDA * sizeof(double);
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(k_trsv_tasks<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_trsv_tasks<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  }
  // co-resident CK-CTA clusters of this kernel, cached per device (devices
  // of different kinds may hold different numbers)
  static std::atomic<int> clusters[64];
  int dev = 0;
  cudaGetDevice(&dev);
  std::atomic<int>& ncache = clusters[dev & 63];
  if (ncache.load() == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CK * 256);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_trsv_tasks<true>, &cfg) != cudaSuccess) {
      // estimate from the per-SM occupancy instead: clusters beyond those that
      // fit at once only wait to be scheduled (a CTA claims tasks once it runs)
      cudaGetLastError();
      int nsm = 0, per = 0;
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trsv_tasks<true>, 256, smem);
      nc = nsm * std::max(0, per) / CK;
    }
    ncache.store(nc >= 2 ? nc : -1);   // -1: the chain cluster could not run beside an update cluster
  }
  if (ncache.load() < 0) {
    chol_solve_fp64(H, mp, Linv, g, u, m, work, st, perm);
    return;
  }
  const int T = (int)(mp / TB);
  const int ntask = trsv_ntask(T);
  // the chain cluster plus update CTAs, all co-resident, in whole clusters
  const int want = CK + ntask;
  const unsigned grid = (unsigned)(CK * std::max(1, std::min(ncache.load(), (want + CK - 1) / CK)));
  double* w = work;
  double* y = work + 3 * mp;
  if (perm) {
    cudaMemsetAsync(w, 0, sizeof(double) * 3 * mp, st);
    k_perm_scatter<<<nblk(m, 256), 256, 0, st>>>(g, m, perm, w);
  } else {
    k_pad_rhs<<<nblk(3 * mp, 256), 256, 0, st>>>(g, m, mp, w);
  }
  ++g_launches;
  cudaMemsetAsync(cnt, 0, sizeof(int) * (2 + 2 * T), st);
  k_trsv_tasks<true><<<grid, 256, smem, st>>>(H, mp, Linv, w, y, cnt, status);
  ++g_launches;
  // backward on y (copied into w as the running right-hand side)
  cudaMemcpyAsync(w, y, sizeof(double) * 3 * mp, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(cnt, 0, sizeof(int) * (2 + 2 * T), st);
  k_trsv_tasks<false><<<grid, 256, smem, st>>>(H, mp, Linv, w, y, cnt, status);
  ++g_launches;
  if (perm) {
    k_perm_gather<<<nblk(m, 256), 256, 0, st>>>(y, m, perm, u);
    ++g_launches;
  } else {
    cudaMemcpyAsync(u, y, sizeof(double) * 3 * m, cudaMemcpyDeviceToDevice, st);
  }
}

void chol_solve_fp64(const double* H, int64_t mp, const double* Linv, const double* g, double* u, int64_t m,
                     double* work, cudaStream_t st, const int32_t* perm) {
  const int T = (int)(mp / TB);
  double* w = work;
  double* y = work + 3 * mp;
  if (perm) {
    cudaMemsetAsync(w, 0, sizeof(double) * 3 * mp, st);
    k_perm_scatter<<<nblk(m, 256), 256, 0, st>>>(g, m, perm, w);
  } else {
    k_pad_rhs<<<nblk(3 * mp, 256), 256, 0, st>>>(g, m, mp, w);
  }
  ++g_launches;
  for (int k = 0; k < T; ++k) {
    k_trsv_fwd<<<T - k, 192, 0, st>>>(H, mp, k, Linv, w, y);
    ++g_launches;
  }
  // backward on y (copied into w as the running right-hand side)
  cudaMemcpyAsync(w, y, sizeof(double) * 3 * mp, cudaMemcpyDeviceToDevice, st);
  for (int k = T - 1; k >= 0; --k) {
    k_trsv_bwd<<<k + 1, 192, 0, st>>>(H, mp, k, Linv, w, y);
    ++g_launches;
  }
  if (perm) {
    k_perm_gather<<<nblk(m, 256), 256, 0, st>>>(y, m, perm, u);
    ++g_launches;
  } else {
    cudaMemcpyAsync(u, y, sizeof(double) * 3 * m, cudaMemcpyDeviceToDevice, st);
  }
}

void symv3(const double* S, int64_t m, const double* v, double* out, cudaStream_t st) {
  if (m > 0) {
    k_symv3<<<nblk(32 * m, 256), 256, 0, st>>>(S, m, v, out);
    ++g_launches;
  }
}

void spmv3(int64_t m, const int64_t* ptr, const int32_t* row, const double* val, const double* v, double alpha,
           double* out, cudaStream_t st) {
  if (m > 0) {
    k_spmv3<<<nblk(m, 256), 256, 0, st>>>(m, ptr, row, val, v, alpha, out);
    ++g_launches;
  }
}

}  // namespace pdk
