// Supernodal triangular solves with the interior factor (Section 3.2, Step 1
// forward substitution and Step 3 backward substitution; Algorithm 1 steps 3
// and 5).  Supernode s owns factor columns col0[s]..col0[s+1]-1; its panel is
// (nc + nr) x nc column-major: the first nc rows hold the inverse of the
// diagonal block (lower), the next nr rows the off-diagonal block whose row
// positions are rows[rowptr[s]..].  Rows >= n1 are x_2 rows (the L_21 part).
// Supernodes are processed level by level (height in the supernodal
// elimination tree), all supernodes of a level in parallel.
#include "kernels.h"

namespace pdk {
namespace {

// y_s = Dinv_s b_s  (one thread per column item of the level)
__global__ void k_fwd_diag(int64_t n_items, const int32_t* __restrict__ isn, const int32_t* __restrict__ ii,
                           const int32_t* __restrict__ col0, const int64_t* __restrict__ rowptr,
                           const int64_t* __restrict__ valptr, const double* __restrict__ L,
                           const double* __restrict__ b, double* __restrict__ y) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_items) return;
  int s = isn[t], i = ii[t];
  int64_t c0 = col0[s], nc = col0[s + 1] - c0, ld = nc + (rowptr[s + 1] - rowptr[s]);
  const double* P = L + valptr[s];
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t j = 0; j <= i; ++j) {
    double d = P[i + j * ld];
    const double* bj = b + 3 * (c0 + j);
    a0 += d * bj[0]; a1 += d * bj[1]; a2 += d * bj[2];
  }
  double* yi = y + 3 * (c0 + i);
  yi[0] = a0; yi[1] = a1; yi[2] = a2;
}

// b[rows[r]] -= L_rs y_s  (one thread per off-diagonal row item)
__global__ void k_fwd_off(int64_t n_items, const int32_t* __restrict__ isn, const int32_t* __restrict__ ir,
                          const int32_t* __restrict__ col0, const int64_t* __restrict__ rowptr,
                          const int32_t* __restrict__ rows, const int64_t* __restrict__ valptr,
                          const double* __restrict__ L, const double* __restrict__ y, double* __restrict__ b) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_items) return;
  int s = isn[t], r = ir[t];
  int64_t c0 = col0[s], nc = col0[s + 1] - c0, ld = nc + (rowptr[s + 1] - rowptr[s]);
  const double* P = L + valptr[s] + nc + r;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t j = 0; j < nc; ++j) {
    double l = P[j * ld];
    const double* yj = y + 3 * (c0 + j);
    a0 += l * yj[0]; a1 += l * yj[1]; a2 += l * yj[2];
  }
  double* br = b + 3 * (int64_t)rows[rowptr[s] + r];
  atomicAdd(br, -a0); atomicAdd(br + 1, -a1); atomicAdd(br + 2, -a2);
}

// z_j = y_j - sum_r L_rj u_{rows[r]}  (one warp per column item)
__global__ void k_bwd_off(int64_t n_items, const int32_t* __restrict__ isn, const int32_t* __restrict__ ii,
                          const int32_t* __restrict__ col0, const int64_t* __restrict__ rowptr,
                          const int32_t* __restrict__ rows, const int64_t* __restrict__ valptr,
                          const double* __restrict__ L, const double* __restrict__ y,
                          const double* __restrict__ u, double* __restrict__ z) {
  int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (t >= n_items) return;
  int s = isn[t], j = ii[t];
  int64_t c0 = col0[s], nc = col0[s + 1] - c0, nr = rowptr[s + 1] - rowptr[s], ld = nc + nr;
  const double* P = L + valptr[s] + nc + j * ld;
  const int32_t* R = rows + rowptr[s];
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t r = lane; r < nr; r += 32) {
    double l = P[r];
    const double* ur = u + 3 * (int64_t)R[r];
    a0 += l * ur[0]; a1 += l * ur[1]; a2 += l * ur[2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) {
    const double* yj = y + 3 * (c0 + j);
    double* zj = z + 3 * (c0 + j);
    zj[0] = yj[0] - a0; zj[1] = yj[1] - a1; zj[2] = yj[2] - a2;
  }
}

// u_i = sum_{j >= i} Dinv_ji z_j  (one warp per column item)
__global__ void k_bwd_diag(int64_t n_items, const int32_t* __restrict__ isn, const int32_t* __restrict__ ii,
                           const int32_t* __restrict__ col0, const int64_t* __restrict__ rowptr,
                           const int64_t* __restrict__ valptr, const double* __restrict__ L,
                           const double* __restrict__ z, double* __restrict__ u) {
  int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (t >= n_items) return;
  int s = isn[t], i = ii[t];
  int64_t c0 = col0[s], nc = col0[s + 1] - c0, ld = nc + (rowptr[s + 1] - rowptr[s]);
  const double* P = L + valptr[s] + i * ld;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t j = i + lane; j < nc; j += 32) {
    double d = P[j];
    const double* zj = z + 3 * (c0 + j);
    a0 += d * zj[0]; a1 += d * zj[1]; a2 += d * zj[2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) {
    double* ui = u + 3 * (c0 + i);
    ui[0] = a0; ui[1] = a1; ui[2] = a2;
  }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void sparse_forward(const SparseFactor& f, double* b, double* y, cudaStream_t st) {
  for (int64_t l = 0; l < f.nlevels; ++l) {
    int64_t c0 = f.lvl_col_ptr[l], c1 = f.lvl_col_ptr[l + 1];
    int64_t r0 = f.lvl_row_ptr[l], r1 = f.lvl_row_ptr[l + 1];
    if (c1 > c0) {
      k_fwd_diag<<<nblk(c1 - c0, 128), 128, 0, st>>>(c1 - c0, f.col_sn + c0, f.col_i + c0, f.col0,
                                                     f.rowptr, f.valptr, f.L, b, y);
      ++g_launches;
    }
    if (r1 > r0) {
      k_fwd_off<<<nblk(r1 - r0, 128), 128, 0, st>>>(r1 - r0, f.row_sn + r0, f.row_r + r0, f.col0, f.rowptr,
                                                    f.rows, f.valptr, f.L, y, b);
      ++g_launches;
    }
  }
}

void sparse_backward(const SparseFactor& f, const double* y, double* u, double* z, cudaStream_t st) {
  for (int64_t l = f.nlevels - 1; l >= 0; --l) {
    int64_t c0 = f.lvl_col_ptr[l], c1 = f.lvl_col_ptr[l + 1];
    if (c1 <= c0) continue;
    k_bwd_off<<<nblk((c1 - c0) * 32, 256), 256, 0, st>>>(c1 - c0, f.col_sn + c0, f.col_i + c0, f.col0,
                                                        f.rowptr, f.rows, f.valptr, f.L, y, u, z);
    ++g_launches;
    k_bwd_diag<<<nblk((c1 - c0) * 32, 256), 256, 0, st>>>(c1 - c0, f.col_sn + c0, f.col_i + c0, f.col0,
                                                         f.rowptr, f.valptr, f.L, z, u);
    ++g_launches;
  }
}

}  // namespace pdk
