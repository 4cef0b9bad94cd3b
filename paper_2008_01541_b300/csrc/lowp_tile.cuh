// Device building blocks of the low-precision (FP32) diagonal-tile Cholesky
// of the collision-region matrix H (Section 3.3, dense refactorisation),
// shared by the look-ahead factorisation (one launch per tile) and the
// persistent left-looking factorisation: the 32 x 32 warp Cholesky, the
// blocked factor of a 128 x 128 tile held in shared memory, and the tile's
// inverse.
#pragma once
#include <cstdint>

namespace pdm {

constexpr int NB = 128;      // tile of the low-precision factor
constexpr int PADW = NB + 1; // padded shared-memory row

// named barrier among n threads (id 1..15; 0 is __syncthreads)
__device__ __forceinline__ void bar_sync_n(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

namespace {

// One warp factors the 32 x 32 block at Ap (row stride PADW) in registers
// (lane i holds row i) and writes L back to Ap, and 1 / L_jj to rinv.  The
// next pivot's column is updated first, with L[j+1][j] taken by a shuffle,
// so that the chain from pivot to pivot is two shuffles, a reciprocal square
// root and two multiplies; the rest of each scaled column goes through shared
// memory (double-buffered, so one warp barrier per pivot) and is read back
// with 16-byte broadcasts.  A non-positive pivot is replaced by 1 and reported
// in *status (first bad column + 1, offset by code0).
template <int LD = PADW>
__device__ __forceinline__ void warp_chol32(float* Ap, float* rinv, int* status, int code0) {
  const int lane = threadIdx.x & 31;
  float a[32];
  if (LD % 4 == 0) {   // 16-byte aligned rows
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(Ap + lane * LD + 4 * q);
      a[4 * q] = v.x; a[4 * q + 1] = v.y; a[4 * q + 2] = v.z; a[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 32; ++c) a[c] = Ap[lane * LD + c];
  }
  __shared__ __align__(16) float col[2][32];
  unsigned bad = 0;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    float djj = __shfl_sync(0xffffffffu, a[j], j);
    const bool b = !(djj > 0.f) || !isfinite(djj);
    bad |= (unsigned)b << j;
    djj = b ? 1.f : djj;
    const float rs = rsqrtf(djj);
    // lanes above the diagonal (lane < c) update their upper entries too:
    // those are never read (a lower entry only depends on lower entries), and
    // leaving out the lane test keeps every update an unpredicated FMA
    a[j] = lane == j ? djj * rs : a[j] * rs;
    if (lane == j) rinv[j] = rs;
    if (j + 1 < 32) {   // the next pivot's column first, with L[j+1][j] by shuffle
      const float v = __shfl_sync(0xffffffffu, a[j], j + 1);
      a[j + 1] = fmaf(-a[j], v, a[j + 1]);
    }
    if (j + 2 < 32) {   // the rest of the update from the column in shared memory
      float* cb = col[j & 1];
      cb[lane] = a[j];
      __syncwarp();
      const float4* c4 = reinterpret_cast<const float4*>(cb);
#pragma unroll
      for (int q = (j + 2) / 4; q < 8; ++q) {
        const float4 v = c4[q];
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int c = 4 * q + e;
          if (c > j + 1) a[c] = fmaf(-a[j], vv[e], a[c]);
        }
      }
    }
  }
  if (bad && lane == 0) atomicCAS(status, 0, code0 + __ffs(bad));
  if (LD % 4 == 0) {   // the whole row (the part above the diagonal is never read)
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<float4*>(Ap + lane * LD + 4 * q) = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
  } else {
#pragma unroll
    for (int c = 0; c < 32; ++c) if (c <= lane) Ap[lane * LD + c] = a[c];
  }
}

// 32 x 32 block product on a group of 64 threads: thread gr = tid & 63 holds
// rows 4 (gr >> 3) .. + 3 and columns 4 (gr & 7) .. + 3 and accumulates
// o += X[rows, t] Y[t, columns] (leading dimensions ldx, ldy).
__device__ __forceinline__ void prod32_g64(const float* X, int ldx, const float* Y, int ldy, float (&o)[4][4]) {
  const int gr = threadIdx.x & 63, r = 4 * (gr >> 3), c = 4 * (gr & 7);
#pragma unroll 4
  for (int t = 0; t < 32; ++t) {
    float x[4], y[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { x[q] = X[(r + q) * ldx + t]; y[q] = Y[t * ldy + c + q]; }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) o[p][q] = fmaf(x[p], y[q], o[p][q]);
  }
}

// Dinv_k = L_kk^-1 from the factored tile in shared memory (A, row stride
// LD, lower triangle), written row-major to Di (zero above the diagonal).
// The four diagonal 32 x 32 blocks are inverted by one warp each; then, by
// block diagonals d = i - j, Z_ij = -Z_ii T_ij with T_ij = sum_{j <= t < i}
// L_it Z_tj, the (4 - d) blocks of a diagonal at once on groups of 64
// threads.  The diagonal blocks Z_ii sit in Zd (leading dimension 33); an
// off-diagonal block Z_ij (i > j) sits in the unused block (j, i) above the
// diagonal of A.  Called by all 256 threads after a barrier.
template <int LD = PADW>
__device__ __forceinline__ void tile_inverse(float* A, float* Zd, float* __restrict__ Di) {
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int LZ = 33;
  // level 0: Z_ii = L_ii^-1 (rows of Zd, leading dimension 33)
  if (warp < 4) {
    const int lane = tid & 31, c0 = 32 * warp;
    const float* Ap = A + c0 * LD + c0;
    float a[32], z[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) { a[c] = (c <= lane) ? Ap[lane * LD + c] : 0.f; z[c] = (c == lane) ? 1.f : 0.f; }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (lane == j) {
        const float ip = __frcp_rn(a[j]);
#pragma unroll
        for (int c = 0; c <= j; ++c) z[c] *= ip;
      }
#pragma unroll
      for (int c = 0; c <= j; ++c) {
        const float zjc = __shfl_sync(0xffffffffu, z[c], j);
        if (lane > j) z[c] = fmaf(-a[j], zjc, z[c]);
      }
    }
    float* Zp = Zd + warp * 32 * LZ;
#pragma unroll
    for (int c = 0; c < 32; ++c) Zp[lane * LZ + c] = z[c];
  }
  __syncthreads();
  const int grp = tid >> 6, gr = tid & 63, orr = 4 * (gr >> 3), occ = 4 * (gr & 7);
#pragma unroll 1
  for (int d = 1; d < 4; ++d) {
    const int j = grp, i = j + d;
    if (i < 4) {
      float* Zij = A + (32 * j) * LD + 32 * i;     // block (j, i) of A holds Z_ij
      float o[4][4] = {};
      for (int t = j; t < i; ++t) {                  // T_ij = sum_t L_it Z_tj
        const float* Lit = A + (32 * i) * LD + 32 * t;
        if (t == j) prod32_g64(Lit, LD, Zd + j * 32 * LZ, LZ, o);
        else prod32_g64(Lit, LD, A + (32 * j) * LD + 32 * t, LD, o);   // Z_tj in block (j, t)
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) Zij[(orr + p) * LD + occ + q] = o[p][q];
      bar_sync_n(1 + grp, 64);
      float z2[4][4] = {};
      prod32_g64(Zd + i * 32 * LZ, LZ, Zij, LD, z2);   // Z_ij = -Z_ii T_ij
      bar_sync_n(1 + grp, 64);
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) Zij[(orr + p) * LD + occ + q] = -z2[p][q];
    }
    __syncthreads();
  }
  for (int q = tid; q < NB * NB; q += 256) {
    const int r = q / NB, c = q % NB, bi = r >> 5, bj = c >> 5;
    float v = 0.f;
    if (bi == bj) v = (c <= r) ? Zd[bi * 32 * LZ + (r & 31) * LZ + (c & 31)] : 0.f;
    else if (bi > bj) v = A[(32 * bj + (r & 31)) * LD + 32 * bi + (c & 31)];
    Di[q] = v;
  }
}

// Factor the 128 x 128 tile A (shared memory, row stride PADW, lower
// triangle) in place with 256 threads, blocked in 32-wide sub-blocks with a
// look-ahead inside the tile: while warp 0 factors sub-block p, warps 1-7
// apply the rest of panel p-1's trailing update; the panel below sub-block p
// is solved one thread per row.  A non-positive pivot is replaced by 1 and
// reported in status[0] as the first bad column (of tile kt) + 1.  Called by
// all 256 threads after a barrier; ends with one.
__device__ __noinline__ void diag_factor_smem(float* A, int kt, int* status) {
  __shared__ float rinv32[32];     // 1 / L_jj of the current 32 x 32 sub-block
  const int tid = threadIdx.x, warp = tid >> 5;
#pragma unroll 1
  for (int p = 0; p < 4; ++p) {
    const int c0 = 32 * p;
    // ---- phase 1: factor block p | rest of panel p-1's update
    if (warp == 0) {
      warp_chol32(A + c0 * PADW + c0, rinv32, status, kt * NB + c0);
    } else if (p > 0) {
      // rows >= c0 + 32, columns c0 .. row (sub-block p itself was updated in phase 3)
      const int pc = c0 - 32;                      // panel columns pc .. pc + 31
      const int nbr = (NB - c0 - 32) / 2, nbc = (NB - c0) / 2;
      for (int q = tid - 32; q < nbr * nbc; q += 224) {
        const int bi = q / nbc, bj = q % nbc;
        const int r = c0 + 32 + 2 * bi, c = c0 + 2 * bj;
        if (c > r) continue;
        float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll 8
        for (int t = 0; t < 32; ++t) {
          const float a0 = A[r * PADW + pc + t], a1 = A[(r + 1) * PADW + pc + t];
          const float b0 = A[c * PADW + pc + t], b1 = A[(c + 1) * PADW + pc + t];
          s00 = fmaf(a0, b0, s00); s01 = fmaf(a0, b1, s01); s10 = fmaf(a1, b0, s10); s11 = fmaf(a1, b1, s11);
        }
        A[r * PADW + c] -= s00;
        A[(r + 1) * PADW + c] -= s10;
        A[(r + 1) * PADW + c + 1] -= s11;
        if (c + 1 <= r) A[r * PADW + c + 1] -= s01;
      }
    }
    __syncthreads();
    // ---- phase 2: panel below block p by substitution (one thread per row)
    float* Ap = A + c0 * PADW + c0;
    const int nbelow = NB - c0 - 32;
    if (tid < nbelow) {
      // right-looking: x_j is final after its own scaling, then eliminated
      // from the later entries (independent FMAs instead of a dot-product chain)
      float* row = A + (c0 + 32 + tid) * PADW + c0;
      float x[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = row[j];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        x[j] *= rinv32[j];
#pragma unroll
        for (int t = j + 1; t < 32; ++t) x[t] = fmaf(-x[j], Ap[t * PADW + j], x[t]);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) row[j] = x[j];
    }
    __syncthreads();
    // ---- phase 3: update of the next diagonal block with panel p
    if (p < 3) {
      const int b0 = c0 + 32;
      for (int q = tid; q < 16 * 16; q += 256) {
        const int bi = q / 16, bj = q % 16;
        if (bj > bi) continue;
        const int r = b0 + 2 * bi, c = b0 + 2 * bj;
        float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll 8
        for (int t = 0; t < 32; ++t) {
          const float a0 = A[r * PADW + c0 + t], a1 = A[(r + 1) * PADW + c0 + t];
          const float e0 = A[c * PADW + c0 + t], e1 = A[(c + 1) * PADW + c0 + t];
          s00 = fmaf(a0, e0, s00); s01 = fmaf(a0, e1, s01); s10 = fmaf(a1, e0, s10); s11 = fmaf(a1, e1, s11);
        }
        A[r * PADW + c] -= s00;
        A[(r + 1) * PADW + c] -= s10;
        A[(r + 1) * PADW + c + 1] -= s11;
        if (c + 1 <= r) A[r * PADW + c + 1] -= s01;
      }
      __syncthreads();
    }
  }
}

// A[r][c] -= sum_{k < 32} A[r][pc + k] A[c][pc + k] over the 32 x 32
// super-block at rows R.., columns C.. of a tile with row stride LD (a
// multiple of 4 with LD % 32 == 4), for c <= r only (so a super-block on
// the diagonal keeps its upper part).  64 threads, g = 0..63: rows
// R + bi + 8 i and columns C + bj + 8 j (bi = g & 7, bj = g >> 3), so the
// eight lanes of a quarter-warp read rows in distinct 16-byte bank groups
// (row loads) or the same row (broadcast), and the stores hit 32 banks.
template <int LD>
__device__ __forceinline__ void superblock_update(float* A, int R, int C, int pc, int g) {
  const int bi = g & 7, bj = g >> 3;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll
  for (int k4 = 0; k4 < 8; ++k4) {
    float4 a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4*>(A + (R + bi + 8 * i) * LD + pc + 4 * k4);
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = *reinterpret_cast<const float4*>(A + (C + bj + 8 * j) * LD + pc + 4 * k4);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        acc[i][j] = fmaf(a[i].w, b[j].w, fmaf(a[i].z, b[j].z, fmaf(a[i].y, b[j].y, fmaf(a[i].x, b[j].x, acc[i][j]))));
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = R + bi + 8 * i, c = C + bj + 8 * j;
      if (c <= r) A[r * LD + c] -= acc[i][j];
    }
}

// Factor the 128 x 128 tile A (shared memory, row stride NB + 4, lower
// triangle) in place with 256 threads: the same blocked order as
// diag_factor_smem (32-wide sub-blocks, warp 0 factoring sub-block p while
// warps 1-6 apply the rest of panel p-1), with every operand read as 16-byte
// rows: the trailing updates on 32 x 32 super-blocks of 64 threads, the panel
// below each sub-block by one thread per row in dot-product form.  A
// non-positive pivot is replaced by 1 and reported in status[0] as the first
// bad column (of tile kt) + 1.  Called by all 256 threads after a barrier;
// ends with one.
__device__ __noinline__ void diag_factor_f4(float* A, int kt, int* status) {
  constexpr int LD = NB + 4;
  __shared__ __align__(16) float rinv[NB];   // 1 / L_jj
  const int tid = threadIdx.x, warp = tid >> 5;
#pragma unroll 1
  for (int p = 0; p < 4; ++p) {
    const int c0 = 32 * p;
    if (warp == 0) {
      warp_chol32<LD>(A + c0 * LD + c0, rinv + c0, status, kt * NB + c0);
    } else if (p > 0 && tid < 224) {
      // rest of panel p-1: super-blocks (rb, cb), p < rb <= 3, p <= cb <= rb, on three groups of 64
      const int grp = (tid - 32) >> 6, g = (tid - 32) & 63;
      int idx = 0;
      for (int rb = p + 1; rb < 4; ++rb)
        for (int cb = p; cb <= rb; ++cb, ++idx)
          if (idx % 3 == grp) superblock_update<LD>(A, 32 * rb, 32 * cb, c0 - 32, g);
    }
    __syncthreads();
    // the panel below sub-block p: x L_pp^T = a for each row, x_k = (a_k - sum_{t<k} L_kt x_t) / L_kk
    const int nbelow = NB - c0 - 32;
    if (tid < nbelow) {
      float* row = A + (c0 + 32 + tid) * LD + c0;
      float x[32];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 v = *reinterpret_cast<const float4*>(row + 4 * q);
        x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const float4* lr = reinterpret_cast<const float4*>(A + (c0 + k) * LD + c0);
        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
        for (int t4 = 0; t4 < k / 4; ++t4) {
          const float4 l = lr[t4];
          p0 = fmaf(l.x, x[4 * t4], p0); p1 = fmaf(l.y, x[4 * t4 + 1], p1);
          p2 = fmaf(l.z, x[4 * t4 + 2], p2); p3 = fmaf(l.w, x[4 * t4 + 3], p3);
        }
        if (k & 3) {
          const float4 l = lr[k / 4];
          const int t = 4 * (k / 4);
          p0 = fmaf(l.x, x[t], p0);
          if ((k & 3) > 1) p1 = fmaf(l.y, x[t + 1], p1);
          if ((k & 3) > 2) p2 = fmaf(l.z, x[t + 2], p2);
        }
        x[k] = (x[k] - ((p0 + p1) + (p2 + p3))) * rinv[c0 + k];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4*>(row + 4 * q) = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    }
    __syncthreads();
    if (p < 3) {   // the next diagonal sub-block with panel p (its factor comes next)
      if (tid < 64) superblock_update<LD>(A, c0 + 32, c0 + 32, c0, tid);
      __syncthreads();
    }
  }
}

}  // namespace
}  // namespace pdm
