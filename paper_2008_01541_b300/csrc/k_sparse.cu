// Supernodal triangular solves with the interior factor (Section 3.2, Step 1
// forward substitution and Step 3 backward substitution; Algorithm 1 steps 3
// and 5).  Supernode s owns factor columns col0[s]..col0[s+1]-1; its panel is
// (nc + nr) x nc column-major: the first nc rows hold the inverse of the
// diagonal block (lower), the next nr rows the off-diagonal block whose row
// positions are rows[rowptr[s]..].  Rows >= n1 are x_2 rows (the L_21 part).
//
// Supernodes are processed level by level (height in the supernodal
// elimination tree).  Within a level the work is cut into 64 x 64 tiles of
// the panels; one CTA per tile accumulates its partial products into the
// destination vector with FP64 atomics, so a large separator is spread over
// many SMs instead of a few long per-row loops.
#include "kernels.h"

namespace pdk {
namespace {

constexpr int TT = 64;

// Forward tile: dst[...] += sign * sum_c P[row + c*ld] src[c0 + c]
// diag tiles: rows/cols within the diagonal block, c <= row, dst = y[c0 + row], sign +1
// off  tiles: rows within the off-diagonal block, dst = b[rows[r]], sign -1
__global__ void __launch_bounds__(256) k_fwd_tiles(const int4* __restrict__ tasks, int diag,
                                                   const int32_t* __restrict__ col0, const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ rows, const int64_t* __restrict__ valptr,
                                                   const double* __restrict__ L, const double* __restrict__ src,
                                                   double* __restrict__ dst) {
  __shared__ double part[4][TT][3];
  const int4 tk = tasks[blockIdx.x];
  const int s = tk.x, rb = tk.y, cb = tk.z;
  const int64_t c0 = col0[s], nc = col0[s + 1] - c0, nr = rowptr[s + 1] - rowptr[s], ld = nc + nr;
  const int tid = threadIdx.x, rloc = tid % TT, chunk = tid / TT;
  const int64_t r = rb + rloc;                       // row within the diag or off block
  const int64_t nrows = diag ? nc : nr;
  const double* P = L + valptr[s] + (diag ? 0 : nc);
  double a0 = 0, a1 = 0, a2 = 0;
  if (r < nrows) {
    const int64_t cend = min((int64_t)cb + TT, nc);
    for (int64_t c = cb + chunk * 16; c < cb + chunk * 16 + 16 && c < cend; ++c) {
      if (diag && c > r) break;
      const double l = P[r + c * ld];
      const double* x = src + 3 * (c0 + c);
      a0 = fma(l, x[0], a0); a1 = fma(l, x[1], a1); a2 = fma(l, x[2], a2);
    }
  }
  part[chunk][rloc][0] = a0; part[chunk][rloc][1] = a1; part[chunk][rloc][2] = a2;
  __syncthreads();
  if (chunk == 0 && r < nrows) {
    for (int q = 1; q < 4; ++q) { a0 += part[q][rloc][0]; a1 += part[q][rloc][1]; a2 += part[q][rloc][2]; }
    if (diag) {
      double* d = dst + 3 * (c0 + r);
      atomicAdd(d, a0); atomicAdd(d + 1, a1); atomicAdd(d + 2, a2);
    } else {
      double* d = dst + 3 * (int64_t)rows[rowptr[s] + r];
      atomicAdd(d, -a0); atomicAdd(d + 1, -a1); atomicAdd(d + 2, -a2);
    }
  }
}

// Backward tile (transposed), staged through shared memory so that the
// global loads stay coalesced along the panel's columns:
// off : z[c0 + j] -= sum_r P[r + j*ld] u[rows[r]]
// diag: u[c0 + j] += sum_{r >= j} Dinv[r + j*ld] z[c0 + r]
__global__ void __launch_bounds__(256) k_bwd_tiles(const int4* __restrict__ tasks, int diag,
                                                   const int32_t* __restrict__ col0, const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ rows, const int64_t* __restrict__ valptr,
                                                   const double* __restrict__ L, const double* __restrict__ src,
                                                   double* __restrict__ dst) {
  __shared__ double tile[TT][TT + 1];
  __shared__ double xs[TT][3];
  __shared__ double part[4][TT][3];
  const int4 tk = tasks[blockIdx.x];
  const int s = tk.x, rb = tk.y, cb = tk.z;
  const int64_t c0 = col0[s], nc = col0[s + 1] - c0, nr = rowptr[s + 1] - rowptr[s], ld = nc + nr;
  const int64_t nrows = diag ? nc : nr;
  const double* P = L + valptr[s] + (diag ? 0 : nc);
  const int32_t* R = rows + rowptr[s];
  const int tid = threadIdx.x;
  for (int q = tid; q < TT * TT; q += 256) {
    const int r = q % TT, j = q / TT;
    const int64_t gr = rb + r, gj = cb + j;
    double v = 0.0;
    if (gr < nrows && gj < nc && !(diag && gr < gj)) v = P[gr + gj * ld];
    tile[r][j] = v;
  }
  if (tid < TT) {
    const int64_t gr = rb + tid;
    if (gr < nrows) {
      const double* x = diag ? src + 3 * (c0 + gr) : src + 3 * (int64_t)R[gr];
      xs[tid][0] = x[0]; xs[tid][1] = x[1]; xs[tid][2] = x[2];
    } else {
      xs[tid][0] = xs[tid][1] = xs[tid][2] = 0.0;
    }
  }
  __syncthreads();
  const int j = tid % TT, rc = tid / TT;
  double a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 4
  for (int r = rc * 16; r < rc * 16 + 16; ++r) {
    const double l = tile[r][j];
    a0 = fma(l, xs[r][0], a0); a1 = fma(l, xs[r][1], a1); a2 = fma(l, xs[r][2], a2);
  }
  part[rc][j][0] = a0; part[rc][j][1] = a1; part[rc][j][2] = a2;
  __syncthreads();
  if (rc == 0 && cb + j < nc) {
    for (int q = 1; q < 4; ++q) { a0 += part[q][j][0]; a1 += part[q][j][1]; a2 += part[q][j][2]; }
    double* d = dst + 3 * (c0 + cb + j);
    const double sg = diag ? 1.0 : -1.0;
    atomicAdd(d, sg * a0); atomicAdd(d + 1, sg * a1); atomicAdd(d + 2, sg * a2);
  }
}

}  // namespace

void sparse_forward(const SparseFactor& f, double* b, double* y, cudaStream_t st) {
  cudaMemsetAsync(y, 0, sizeof(double) * 3 * f.n1, st);
  for (int64_t l = 0; l < f.nlevels; ++l) {
    int64_t d0 = f.lvl_diag_ptr[l], d1 = f.lvl_diag_ptr[l + 1];
    int64_t o0 = f.lvl_off_ptr[l], o1 = f.lvl_off_ptr[l + 1];
    if (d1 > d0) {
      k_fwd_tiles<<<(unsigned)(d1 - d0), 256, 0, st>>>(f.diag_tasks + d0, 1, f.col0, f.rowptr, f.rows, f.valptr, f.L, b, y);
      ++g_launches;
    }
    if (o1 > o0) {
      k_fwd_tiles<<<(unsigned)(o1 - o0), 256, 0, st>>>(f.off_tasks + o0, 0, f.col0, f.rowptr, f.rows, f.valptr, f.L, y, b);
      ++g_launches;
    }
  }
}

void sparse_backward(const SparseFactor& f, const double* y, double* u, double* z, cudaStream_t st) {
  cudaMemcpyAsync(z, y, sizeof(double) * 3 * f.n1, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(u, 0, sizeof(double) * 3 * f.n1, st);
  for (int64_t l = f.nlevels - 1; l >= 0; --l) {
    int64_t d0 = f.lvl_diag_ptr[l], d1 = f.lvl_diag_ptr[l + 1];
    int64_t o0 = f.lvl_off_ptr[l], o1 = f.lvl_off_ptr[l + 1];
    if (o1 > o0) {
      k_bwd_tiles<<<(unsigned)(o1 - o0), 256, 0, st>>>(f.off_tasks + o0, 0, f.col0, f.rowptr, f.rows, f.valptr, f.L, u, z);
      ++g_launches;
    }
    if (d1 > d0) {
      k_bwd_tiles<<<(unsigned)(d1 - d0), 256, 0, st>>>(f.diag_tasks + d0, 1, f.col0, f.rowptr, f.rows, f.valptr, f.L, z, u);
      ++g_launches;
    }
  }
}

}  // namespace pdk
