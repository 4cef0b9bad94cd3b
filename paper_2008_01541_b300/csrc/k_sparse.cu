// Supernodal triangular solves with dependency counters instead of one launch
// per elimination-tree level (Section 3.2, Step 1 forward and Step 3 backward
// substitution; Algorithm 1 steps 3 and 5).
//
// The factor holds, per supernode s, D_s = L_ss^-1 and M_s = L_rs L_ss^-1
// (the off-diagonal rows times the inverse), so that
//   forward   y_s = D_s b_s,           b_r -= M_s b_s
//   backward  u_s = D_s^T y_s - M_s^T u_r
// and every tile of a supernode needs only inputs that are final before any
// of them starts: one dependent step per supernode along the tree.
//
// Work is listed once as tasks in a topological order (forward: leaves first;
// backward: the reverse).  A supernode of at most 64 columns and 128
// off-diagonal rows is one task; a larger one is cut into 64 x 64 tiles of D_s
// and of M_s.  A persistent grid claims tasks in list order from one atomic
// counter; a task waits only for tasks earlier in the list, which are already
// claimed by running CTAs, so the grid always makes progress whatever the
// hardware's CTA order.
//   forward  any task of s: waits until every task writing into s's rows is
//            done
//   backward off tile / small supernode s: waits until the supernodes owning
//            its off-diagonal rows are done
//            diag tile of s: waits for nothing (y is final)
// Results move through FP64 atomics in L2; producers fence before signalling,
// consumers fence after waiting and read the vectors with L1-bypassing loads.
// Three right-hand sides make 3 FP64 FMAs per 8-byte factor entry, and only
// the nonzero part of every tile is multiplied.  The time is nonetheless set
// by per-task latency rather than by the FP64 rate or the bytes: on the
// 598K-tet elbow each direction runs ~36K tasks on 592 resident CTAs, each
// ~4 us of staging and dependency wait plus 5-8 us of work that is mostly
// fixed latency (vector loads from L2, the chunk reduction, the atomics and
// the fence before the signal).  The same tasks with the products in
// double-float on the FP32 pipes (a fifth of the FP64-pipe time) ran no
// faster.  Every wait is bounded (about a second); on expiry code 300 goes to
// status[1] and all later waits are skipped.
#include <algorithm>

#include "kernels.h"

namespace pdk {
namespace {

constexpr int TT = 64;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Spin until *c <= 0; gives up (recording code 300) after about a second or
// as soon as another wait has given up.
__device__ __forceinline__ void wait_zero(const int* c, int* status, unsigned long long t0) {
  unsigned it = 0;
  while (*(volatile const int*)c > 0) {
    if (*(volatile int*)(status + 1) != 0) return;
    if (++it > 32) __nanosleep(40);
    if ((it & 1023u) == 0 && gtimer() - t0 > 1000000000ull) {
      atomicCAS(status + 1, 0, 300);
      return;
    }
  }
}

// Stage rows [r0, r0 + nrow) x cols [0, ncol) of the column-major panel P
// (leading dimension ld) into tile; entries above the diagonal of a diagonal
// block (lower = true: column > row + r0 - c0) and outside the range are zero.
__device__ __forceinline__ void stage_tile(double (*tile)[TT + 1], const double* __restrict__ P, int64_t ld, int r0,
                                           int c0, int nrow, int ncol, bool lower) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int c = warp + 8 * k;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      double v = 0.0;
      if (c < ncol && r < nrow && !(lower && r0 + r < c0 + c)) v = __ldg(P + (r0 + r) + (int64_t)(c0 + c) * ld);
      tile[r][c] = v;
    }
  }
}

// Partial sums of out[o] = sum_t T[o][t] vec[t] (trans: T[t][o]) over the
// terms t in [lo, hi) of chunk ch (thread o = tid % 64, ch = tid / 64, 16
// terms per chunk).  Only the nonzero range is visited.
__device__ __forceinline__ void partial(const double (*tile)[TT + 1], const double (*vec)[3], bool trans, int lo,
                                        int hi, double& a0, double& a1, double& a2) {
  const int o = threadIdx.x % TT, ch = threadIdx.x / TT;
  const int t0 = max(ch * 16, lo), t1 = min(ch * 16 + 16, hi);
#pragma unroll 4
  for (int t = t0; t < t1; ++t) {
    const double l = trans ? tile[t][o] : tile[o][t];
    a0 = fma(l, vec[t][0], a0); a1 = fma(l, vec[t][1], a1); a2 = fma(l, vec[t][2], a2);
  }
}

// Sum the four chunks; the result is valid in threads with ch == 0.
__device__ __forceinline__ void reduce4(double (*part)[TT][3], double& a0, double& a1, double& a2) {
  const int o = threadIdx.x % TT, ch = threadIdx.x / TT;
  part[ch][o][0] = a0; part[ch][o][1] = a1; part[ch][o][2] = a2;
  __syncthreads();
  if (ch == 0) {
#pragma unroll
    for (int q = 1; q < 4; ++q) { a0 += part[q][o][0]; a1 += part[q][o][1]; a2 += part[q][o][2]; }
  }
}

__device__ __forceinline__ void load3(double (*dst)[3], int i, const double* x) {
  dst[i][0] = __ldcg(x); dst[i][1] = __ldcg(x + 1); dst[i][2] = __ldcg(x + 2);
}

constexpr int KIND_DIAG = 0, KIND_OFF = 1, KIND_FUSED = 2;

template <bool FWD>
__global__ void __launch_bounds__(256, FWD ? 4 : 5) k_sf_solve(SparseFactor f, int64_t ntasks, const int4* __restrict__ tasks,
                                                  int* cnt, double* __restrict__ v0, double* __restrict__ v1) {
  // FWD : v0 = b (right-hand side, reduced in place by off-diagonal rows), v1 = y
  // !FWD: v0 = u (x_2 rows preset, the rest zero),                       v1 = z (= y on entry)
  __shared__ double tile[TT][TT + 1];
  __shared__ double xs[TT][3];
  __shared__ double ys[TT][3];
  __shared__ double part[4][TT][3];
  __shared__ int4 cur;
  const int tid = threadIdx.x, o = tid % TT, ch = tid / TT;
  int* next = cnt + (FWD ? f.cnt_next_f : f.cnt_next_b);
  int* cA = cnt + (FWD ? f.cnt_fin : f.cnt_zpend);
  int* cB = cnt + (FWD ? f.cnt_ydone : f.cnt_udone);
  int my_next = 0;
  if (tid == 0) {
    const int t = atomicAdd(next, 1);
    cur = t < ntasks ? tasks[t] : make_int4(-1, 0, 0, 0);
    my_next = atomicAdd(next, 1);      // claimed ahead; tasks are still claimed in order
  }
  __syncthreads();
  for (;;) {
    const int4 tk = cur;
    if (tk.x < 0) break;
    const int s = tk.x & 0x1fffffff, kind = (tk.x >> 29) & 3;
    const int rb = tk.y, cb = tk.z, oi = tk.w;
    const int64_t c0 = f.col0[s], nc = f.col0[s + 1] - c0, nr = f.rowptr[s + 1] - f.rowptr[s], ld = nc + nr;
    const double* Pd = f.L + f.valptr[s];     // diagonal block (its inverse, lower)
    const double* Po = Pd + nc;               // off-diagonal block
    const int32_t* R = f.rows + f.rowptr[s];
    // ---- the factor tile this task starts with does not depend on the
    // vectors: stage it while the inputs are awaited
    const bool diag = kind == KIND_DIAG;
    const int64_t nrows = diag ? nc : nr;
    const int rows_t = (int)min((int64_t)TT, nrows - rb), cols_t = (int)min((int64_t)TT, nc - cb);
    if (kind == KIND_FUSED) {
      if (FWD) stage_tile(tile, Pd, ld, 0, 0, (int)nc, (int)nc, true);
      else if (nr > 0) stage_tile(tile, Po, ld, 0, 0, (int)min((int64_t)TT, nr), (int)nc, false);
    } else {
      stage_tile(tile, diag ? Pd : Po, ld, rb, cb, rows_t, cols_t, diag);
    }
    // ---- wait for the inputs
    if (tid == 0) {
      const unsigned long long t0 = gtimer();
      if (FWD) {
        wait_zero(cA + s, f.status, t0);
      } else if (kind != KIND_DIAG) {
        for (int64_t q = f.tgt_ptr[oi]; q < f.tgt_ptr[oi + 1]; ++q) wait_zero(cB + f.tgt[q], f.status, t0);
      }
      __threadfence();
    }
    __syncthreads();
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    if (kind == KIND_FUSED) {
      const int n = (int)nc;
      if (FWD) {
        // y_s = D_s b_s (its tile staged before the wait), then b[rows] -= M_s b_s
        if (tid < TT) {
          if (tid < n) load3(xs, tid, v0 + 3 * (c0 + tid));
          else xs[tid][0] = xs[tid][1] = xs[tid][2] = 0.0;
        }
        __syncthreads();
        if (o < n) partial(tile, xs, false, 0, o + 1, a0, a1, a2);
        reduce4(part, a0, a1, a2);
        if (ch == 0) {
          ys[o][0] = o < n ? a0 : 0.0; ys[o][1] = o < n ? a1 : 0.0; ys[o][2] = o < n ? a2 : 0.0;
          if (o < n) { double* d = v1 + 3 * (c0 + o); d[0] = a0; d[1] = a1; d[2] = a2; }
        }
        __syncthreads();
        for (int r0 = 0; r0 < nr; r0 += TT) {
          const int nrow = (int)min((int64_t)TT, nr - r0);
          stage_tile(tile, Po, ld, r0, 0, nrow, n, false);
          __syncthreads();
          a0 = a1 = a2 = 0.0;
          if (o < nrow) partial(tile, xs, false, 0, n, a0, a1, a2);
          reduce4(part, a0, a1, a2);
          if (ch == 0 && o < nrow) {
            double* d = v0 + 3 * (int64_t)R[r0 + o];
            atomicAdd(d, -a0); atomicAdd(d + 1, -a1); atomicAdd(d + 2, -a2);
          }
          __syncthreads();
        }
      } else {
        // e = M_s^T u[rows], then u_s = D_s^T y_s - e
        for (int r0 = 0; r0 < nr; r0 += TT) {
          const int nrow = (int)min((int64_t)TT, nr - r0);
          if (r0 > 0) stage_tile(tile, Po, ld, r0, 0, nrow, n, false);   // the first was staged before the wait
          if (tid < TT) {
            if (tid < nrow) load3(xs, tid, v0 + 3 * (int64_t)R[r0 + tid]);
            else xs[tid][0] = xs[tid][1] = xs[tid][2] = 0.0;
          }
          __syncthreads();
          if (o < n) partial(tile, xs, true, 0, nrow, a0, a1, a2);
          __syncthreads();
        }
        reduce4(part, a0, a1, a2);
        const double e0 = a0, e1 = a1, e2 = a2;   // valid in threads with ch == 0
        if (ch == 0) {
          if (o < n) {
            const double* yy = v1 + 3 * (c0 + o);
            ys[o][0] = __ldcg(yy); ys[o][1] = __ldcg(yy + 1); ys[o][2] = __ldcg(yy + 2);
          } else {
            ys[o][0] = ys[o][1] = ys[o][2] = 0.0;
          }
        }
        stage_tile(tile, Pd, ld, 0, 0, n, n, true);
        __syncthreads();
        a0 = a1 = a2 = 0.0;
        if (o < n) partial(tile, ys, true, o, n, a0, a1, a2);
        reduce4(part, a0, a1, a2);
        if (ch == 0 && o < n) { double* d = v0 + 3 * (c0 + o); d[0] = a0 - e0; d[1] = a1 - e1; d[2] = a2 - e2; }
      }
    } else {
      if (tid < TT) {
        xs[tid][0] = xs[tid][1] = xs[tid][2] = 0.0;
        if (FWD) {
          // forward contracts over the tile's columns (b_s for both kinds)
          if (tid < cols_t) load3(xs, tid, v0 + 3 * (c0 + cb + tid));
        } else {
          // backward contracts over the tile's rows
          if (tid < rows_t) load3(xs, tid, diag ? v1 + 3 * (c0 + rb + tid) : v0 + 3 * (int64_t)R[rb + tid]);
        }
      }
      __syncthreads();
      // nonzero range of the contraction for output o (diag tiles are triangular)
      int lo = 0, hi = FWD ? cols_t : rows_t;
      if (diag) {
        if (FWD) hi = min(hi, o + rb - cb + 1);   // column cb + t <= row rb + o
        else lo = max(lo, o + cb - rb);           // row rb + t >= column cb + o
      }
      if (o < (FWD ? rows_t : cols_t)) partial(tile, xs, !FWD, lo, hi, a0, a1, a2);
      reduce4(part, a0, a1, a2);
      if (ch == 0 && o < (FWD ? rows_t : cols_t)) {
        double* d;
        if (FWD) d = diag ? v1 + 3 * (c0 + rb + o) : v0 + 3 * (int64_t)R[rb + o];
        else d = v0 + 3 * (c0 + cb + o);
        const double sg = diag ? 1.0 : -1.0;
        atomicAdd(d, sg * a0); atomicAdd(d + 1, sg * a1); atomicAdd(d + 2, sg * a2);
      }
    }
    __threadfence();
    __syncthreads();
    // ---- signal, and take the next task
    if (tid == 0) {
      if (FWD) {
        if (kind == KIND_DIAG) atomicSub(cB + s, 1);
        else
          for (int64_t q = f.tgt_ptr[oi]; q < f.tgt_ptr[oi + 1]; ++q) atomicSub(cA + f.tgt[q], 1);
      } else {
        atomicSub(cB + s, 1);   // every task of s counts towards u_s
      }
      cur = my_next < ntasks ? tasks[my_next] : make_int4(-1, 0, 0, 0);
      if (my_next < ntasks) my_next = atomicAdd(next, 1);
    }
    __syncthreads();
  }
}

}  // namespace

// The backward solve is built for five resident CTAs per SM (48 registers a
// thread, 42.5 KB of shared memory each), ~6% faster than four; the forward
// keeps four (64 registers): its 48-register build ran ~4% slower at four a
// SM, and five a SM slowed the low-precision factorisation it overlaps.
int sparse_grid(bool forward) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (forward) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sf_solve<true>, 256, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sf_solve<false>, 256, 0);
  return std::max(1, nsm) * std::max(1, per);
}

void sparse_forward(const SparseFactor& f, double* b, double* y, cudaStream_t st) {
  cudaMemsetAsync(y, 0, sizeof(double) * 3 * f.n1, st);
  cudaMemcpyAsync(f.cnt + f.cnt_fin, f.cnt_init + f.cnt_fin, sizeof(int) * (f.cnt_next_f + 1 - f.cnt_fin),
                  cudaMemcpyDeviceToDevice, st);
  if (f.n_ftasks > 0) {
    k_sf_solve<true><<<f.grid_f, 256, 0, st>>>(f, f.n_ftasks, f.ftasks, f.cnt, b, y);
    ++g_launches;
  }
}

void sparse_backward(const SparseFactor& f, const double* y, double* u, double* z, cudaStream_t st) {
  cudaMemcpyAsync(z, y, sizeof(double) * 3 * f.n1, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(u, 0, sizeof(double) * 3 * f.n1, st);
  cudaMemcpyAsync(f.cnt + f.cnt_zpend, f.cnt_init + f.cnt_zpend, sizeof(int) * (f.cnt_next_b + 1 - f.cnt_zpend),
                  cudaMemcpyDeviceToDevice, st);
  if (f.n_btasks > 0) {
    k_sf_solve<false><<<f.grid_b, 256, 0, st>>>(f, f.n_btasks, f.btasks, f.cnt, u, z);
    ++g_launches;
  }
}

}  // namespace pdk
