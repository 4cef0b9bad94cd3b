// Persistent left-looking low-precision Cholesky (see chol_ll.h).
//
// One CTA of 256 threads per SM, each running tasks until its list is done.
// CTA 0 factors the diagonal tiles in order (FP32, shared memory); a few CTAs
// invert them; the rest run the tensor-core tasks, in which
//   warp 0, lane 0 : producer -- waits until the panels L_ik and L_jk of the
//                    next K step are final (per-row counters), then TMA-loads
//                    their 128-byte column chunks into a ring of shared-memory
//                    stages (128B swizzle, K-major);
//   warp 1, lane 0 : issues the tcgen05 MMAs of each stage into the 128 x 128
//                    FP32 accumulator in tensor memory and frees the stage;
//   all 8 warps    : read the accumulator (warp w the TMEM lane quarter w % 4,
//                    half the columns) and form S = A_ij - acc in shared
//                    memory; then the panel products, or S_jj back to global
//                    memory for CTA 0.
// A task waits only on tasks that precede it in these orders, so the grid
// (all CTAs co-resident) always progresses.  Every wait is bounded; a wait
// that gives up writes a code to status[1], which makes every other CTA stop
// at its next wait or claim.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>

#include "chol_ll.h"
#include "kernels.h"
#include "lowp_tile.cuh"
#include "tc_dev.cuh"

namespace pdll {
namespace {

using namespace pdtc::dev;
using pdm::NB;
using pdm::PADW;

constexpr int SP = NB + 4;                // row stride of the transposed operands of the panel products
constexpr uint32_t kSpin = 1u << 22;      // bounded waits: ~1 s with back-off
constexpr int kStageBudget = 196608;      // shared memory for the pipeline stages (192 KB)
constexpr int kDiagCtas = 6;              // CTAs for the diagonal tiles: one factors, the others invert

template <int MODE>   // 0 = TF32, 1 = split TF32 (hi.hi + hi.lo + lo.hi), 2 = BF16
struct Cfg {
  static constexpr int CPP = MODE == 2 ? 2 : 4;            // 128-byte K chunks per 128-column panel
  static constexpr int NBUF = MODE == 1 ? 4 : 2;           // 16 KB operand buffers per stage
  static constexpr int STAGE = NBUF * kChunkBytes;
  static constexpr int NST = kStageBudget / STAGE;         // 3 (split TF32) or 6 stages
  static constexpr int CHUNK = MODE == 2 ? 64 : 32;        // K elements per chunk
  static constexpr int EPI = 2 * NB * SP * 4;              // panel epilogue: S^T and an operand, 132 KB
  static constexpr int SMEM = (NST * STAGE > EPI ? NST * STAGE : EPI) + 1024;
};

struct Ptrs {
  int ndiag;   // CTAs of the diagonal tiles: the factor CTA, then the inversion CTAs
  float* L;
  float* Llo;
  __nv_bfloat16* Lb;
  float* Lh;
  float* Dinv;
  float* E;
  int64_t mq;
  int T, kb;
  int* sync;
  int* status;
  int* piv;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ bool failed_globally(const int* status) {
  return *(volatile const int*)(status + 1) != 0;
}

// Bounded wait until *p >= v.  False if it gave up (code written to
// status[1]) or if another CTA has already failed.
__device__ bool wait_flag(const int* p, int v, int* status, int code) {
  for (uint32_t it = 0; it < kSpin; ++it) {
    if (ld_acquire(p) >= v) return true;
    if (failed_globally(status)) return false;
    __nanosleep(it < 64 ? 32 : 256);
  }
  atomicCAS(status + 1, 0, code);
  return false;
}

// Bounded wait for phase `parity` of an mbarrier.  Gives up early when the
// producer has stopped (*stop) before issuing chunk q (q >= *issued).
__device__ bool mbar_wait_or_stop(uint64_t* bar, uint32_t parity, volatile int* stop, volatile int* issued, int q,
                                  int* status, int code) {
  for (uint32_t it = 0; it < kSpin; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*stop && q >= *issued) return false;
    if (it > 32) __nanosleep(64);
  }
  atomicCAS(status + 1, 0, code);
  return false;
}

// FP32 value minus its TF32 head (the head keeps the top 19 bits)
__device__ __forceinline__ float tf32_tail(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// Thread (ty, tx) of the 16 x 16 grid owns rows 8 ty .. + 7 and columns
// 4 tx .. + 3 and 64 + 4 tx .. + 3 of a 128 x 128 tile (acc[p][q], q < 4 and
// q >= 4), so a half-warp's 16-byte loads of a row of Y are contiguous.
// acc[p][q] = sum_t X[t][8 ty + p] Y[t][column q] over t < 128, both
// operands with row stride SP (X holds the left factor transposed)
__device__ __forceinline__ void prod_8x8(const float* X, const float* Y, int ty, int tx, float (&acc)[8][8]) {
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[p][q] = 0.f;
#pragma unroll 2
  for (int t = 0; t < NB; ++t) {
    const float4 a0 = *reinterpret_cast<const float4*>(X + t * SP + 8 * ty);
    const float4 a1 = *reinterpret_cast<const float4*>(X + t * SP + 8 * ty + 4);
    const float4 b0 = *reinterpret_cast<const float4*>(Y + t * SP + 4 * tx);
    const float4 b1 = *reinterpret_cast<const float4*>(Y + t * SP + 64 + 4 * tx);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
  }
}

// X L^T = S for the 128 x 128 panel tile: on entry XT[t * SP + r] = S[r][t],
// on exit X[r][t]; Lj = the factored diagonal tile (row stride SP, lower),
// rinv[k] = 1 / L[k][k].  Blocked by 32 columns: thread r < 128 solves its row
// against the 32 x 32 diagonal block with its 32 unknowns in registers,
// x_k = (s_k - sum_{t < k} L_kt x_t) / L_kk, reading each row of L with
// 16-byte broadcasts; then all 256 threads remove the block's contribution
// from the later columns (rows r and r + 64, r = tid & 63, a quarter of
// those columns each), one 16-byte load per eight multiply-adds.
__device__ __forceinline__ void panel_substitution(float* XT, const float* Lj, const float* rinv) {
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int b = 0; b < 4; ++b) {
    const int c0 = 32 * b;
    if (tid < NB) {
      float x[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) x[k] = XT[(c0 + k) * SP + tid];
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const float4* lr = reinterpret_cast<const float4*>(Lj + (c0 + k) * SP + c0);
        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
        for (int t4 = 0; t4 < k / 4; ++t4) {
          const float4 l = lr[t4];
          p0 = fmaf(l.x, x[4 * t4], p0); p1 = fmaf(l.y, x[4 * t4 + 1], p1);
          p2 = fmaf(l.z, x[4 * t4 + 2], p2); p3 = fmaf(l.w, x[4 * t4 + 3], p3);
        }
        if (k & 3) {   // the last, partial group of four
          const float4 l = lr[k / 4];
          const int t = 4 * (k / 4);
          p0 = fmaf(l.x, x[t], p0);
          if ((k & 3) > 1) p1 = fmaf(l.y, x[t + 1], p1);
          if ((k & 3) > 2) p2 = fmaf(l.z, x[t + 2], p2);
        }
        x[k] = (x[k] - ((p0 + p1) + (p2 + p3))) * rinv[c0 + k];
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) XT[(c0 + k) * SP + tid] = x[k];
    }
    __syncthreads();
    const int rest = NB - c0 - 32;
    if (rest > 0) {
      // rows r and r + 64 (r = tid & 63), a quarter of the later columns
      // each: every 16-byte row of L read serves both rows
      const int r = tid & 63, n = rest / 4, cbeg = c0 + 32 + (tid >> 6) * n;
      float x[32], y[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        x[k] = XT[(c0 + k) * SP + r];
        y[k] = XT[(c0 + k) * SP + r + 64];
      }
#pragma unroll 1
      for (int c = cbeg; c < cbeg + n; ++c) {
        const float4* lr = reinterpret_cast<const float4*>(Lj + c * SP + c0);
        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f, q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
#pragma unroll
        for (int t4 = 0; t4 < 8; ++t4) {
          const float4 l = lr[t4];
          p0 = fmaf(l.x, x[4 * t4], p0); p1 = fmaf(l.y, x[4 * t4 + 1], p1);
          p2 = fmaf(l.z, x[4 * t4 + 2], p2); p3 = fmaf(l.w, x[4 * t4 + 3], p3);
          q0 = fmaf(l.x, y[4 * t4], q0); q1 = fmaf(l.y, y[4 * t4 + 1], q1);
          q2 = fmaf(l.z, y[4 * t4 + 2], q2); q3 = fmaf(l.w, y[4 * t4 + 3], q3);
        }
        XT[c * SP + r] -= (p0 + p1) + (p2 + p3);
        XT[c * SP + r + 64] -= (q0 + q1) + (q2 + q3);
      }
    }
    __syncthreads();
  }
}

// The 128 x 128 tile at src (global, row stride ld) into shared memory (row
// stride SP), sixteen 16-byte loads per thread all in flight; and back.
__device__ __forceinline__ void load_tile(float* dst, const float* src, int64_t ld) {
  const int tid = threadIdx.x;
  float4 v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int q = tid + 256 * k, r = q >> 5, c = 4 * (q & 31);
    v[k] = __ldcg(reinterpret_cast<const float4*>(src + (int64_t)r * ld + c));
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int q = tid + 256 * k, r = q >> 5, c = 4 * (q & 31);
    *reinterpret_cast<float4*>(dst + r * SP + c) = v[k];
  }
}
__device__ __forceinline__ void store_tile(float* dst, int64_t ld, const float* src) {
  const int tid = threadIdx.x;
#pragma unroll 4
  for (int k = 0; k < 16; ++k) {
    const int q = tid + 256 * k, r = q >> 5, c = 4 * (q & 31);
    *reinterpret_cast<float4*>(dst + (int64_t)r * ld + c) = *reinterpret_cast<const float4*>(src + r * SP + c);
  }
}

// the thread's 8 x 8 outputs into a row-major tile at dst (row stride ld)
__device__ __forceinline__ void store_8x8(float* dst, int64_t ld, int ty, int tx, const float (&acc)[8][8]) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    float* row = dst + (int64_t)(8 * ty + p) * ld;
    *reinterpret_cast<float4*>(row + 4 * tx) = make_float4(acc[p][0], acc[p][1], acc[p][2], acc[p][3]);
    *reinterpret_cast<float4*>(row + 64 + 4 * tx) = make_float4(acc[p][4], acc[p][5], acc[p][6], acc[p][7]);
  }
}

template <int MODE>
__global__ void __launch_bounds__(256, 1)
    k_chol_ll(const __grid_constant__ CUtensorMap thi, const __grid_constant__ CUtensorMap tlo, const Ptrs P) {
  using C = Cfg<MODE>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[C::NST], empty[C::NST], accf;
  __shared__ uint32_t tmem_base;
  __shared__ int s_task;
  __shared__ volatile int s_stop, s_issued;
  uint8_t* sm = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int T = P.T, kb = P.kb;
  const int64_t mq = P.mq;
  // Roles.  CTA 0 factors the diagonal tiles, in order, and does nothing
  // else: the factor is long unrolled code on the critical path, and it runs
  // from a cold instruction cache on an SM (or beside a TPC partner) that
  // streams operands through TMA.  The grid is launched as CTA pairs
  // (clusters of two, one TPC each), so CTA 0 shares its TPC with CTA 1.
  // CTAs 1 .. NDIAG-1 invert the factored diagonal tiles (Dinv_j, E_j),
  // claiming them in order.  The others run the tensor-core tasks in
  // column-major order: the panels (i, j), and after the first panel of
  // column j the accumulation S_j+1,j+1 = A - sum L L^T of the next diagonal
  // tile, which they write back to its tile of L for CTA 0.  Each task waits
  // only on tasks earlier in these orders, so all progress.
  int* claim = P.sync;            // [0] inversions, [1] tensor-core tasks
  int* rowcnt = P.sync + 2;       // [T] finished tiles of row i among columns kb..
  int* dcnt = P.sync + 2 + T;     // [T] Dinv_j written
  int* scnt = P.sync + 2 + 2 * T; // [T] S_jj formed (the factor of tile j may start)
  const int nt = T - kb;
  const int role = blockIdx.x == 0 ? 0 : (int)blockIdx.x < P.ndiag ? 1 : 2;   // factor, inversion, tensor core
  const int ntask = role < 2 ? nt : nt * (nt + 1) / 2 - 1;
  int fnext = 0;   // the factor CTA's next tile (thread 0)

  constexpr int KIND = MODE == 2 ? 1 : 0;
  constexpr uint32_t ID = idesc(MODE == 2 ? 1u : 2u);

  if (tid == 0) {
    for (int s = 0; s < C::NST; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(&accf, 1);
    s_stop = 0;
    s_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(NB));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t g = 0;      // chunks through the stage ring so far (the producer and the MMA thread agree)
  uint32_t nacc = 0;   // tasks that used the accumulator so far
  float* A = reinterpret_cast<float*>(sm);    // diagonal task: the tile [128][SP]
  float* Zd = A + NB * SP;                    //   and the diagonal blocks of its inverse [4][32][33]
  float* ST = reinterpret_cast<float*>(sm);   // panel task: S transposed [128][SP]
  float* DT = ST + NB * SP;                   //   and the right operand [128][SP]

  for (;;) {
    if (tid == 0)
      s_task = (s_stop || failed_globally(P.status)) ? ntask : role == 0 ? fnext++ : atomicAdd(claim + role - 1, 1);
    __syncthreads();
    const int t = s_task;
    if (t >= ntask) break;
    int i, j;
    if (role < 2) {
      i = j = kb + t;
    } else {   // column j = kb .. T-2: panel (j+1, j), the accumulation of tile j+1, panels (j+2 .., j)
      int rem = t;
      j = kb;
      while (rem >= T - j) { rem -= T - j; ++j; }
      if (rem == 1) i = j = j + 1;
      else i = j + (rem == 0 ? 1 : rem);
    }
    const bool diag = i == j;
    const int nchunk = role == 2 ? (j - kb) * C::CPP : 0;
    float* Lt = P.L + (int64_t)i * NB * mq + (int64_t)j * NB;

    if (role == 0) {
      // ---- L_jj from S_jj (written by the accumulation task; A_jj itself
      // for the first column), published at once
      if (j > kb && tid == 0 && !wait_flag(scnt + j, 1, P.status, 318)) s_stop = 1;
      __syncthreads();
      if (s_stop) continue;
      load_tile(A, Lt, mq);
      __syncthreads();
      pdm::diag_factor_f4(A, j, P.piv);
      store_tile(Lt, mq, A);   // whole rows: the strict upper triangle of a diagonal tile of L is scratch
      __syncthreads();
      if (tid == 0) {   // the panels of column j solve against L_jj
        __threadfence();
        st_release(rowcnt + j, j - kb + 1);
      }
      continue;
    }
    if (role == 1) {
      // ---- Dinv_j (the panels' Lh products wait for it), then E_j for the preconditioner
      if (tid == 0 && !wait_flag(rowcnt + j, j - kb + 1, P.status, 319)) s_stop = 1;
      __syncthreads();
      if (s_stop) continue;
      load_tile(A, Lt, mq);
      __syncthreads();
      float* Di = P.Dinv + (int64_t)j * NB * NB;
      pdm::tile_inverse<SP>(A, Zd, Di);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(dcnt + j, 1);
      }
      float* Dsm = A;   // Dinv_j again, padded rows
#pragma unroll 4
      for (int k = 0; k < 16; ++k) {
        const int q = tid + 256 * k, r = q >> 5, c = 4 * (q & 31);
        const float4 v = __ldcg(reinterpret_cast<const float4*>(Di + r * NB + c));
        Dsm[r * PADW + c] = v.x; Dsm[r * PADW + c + 1] = v.y; Dsm[r * PADW + c + 2] = v.z; Dsm[r * PADW + c + 3] = v.w;
      }
      __syncthreads();
      float* Ej = P.E + (int64_t)j * NB * NB;
      for (int q = tid; q < NB * NB; q += 256) {   // E[r][c] = sum_{t >= max(r, c)} Dinv[t][r] Dinv[t][c]
        const int r = q / NB, c = q % NB;
        float e = 0.f;
        for (int t2 = (r > c ? r : c); t2 < NB; ++t2) e = fmaf(Dsm[t2 * PADW + r], Dsm[t2 * PADW + c], e);
        Ej[q] = e;
      }
      __syncthreads();
      continue;
    }

    // ---- acc = sum_{kb <= k < j} L_ik L_jk^T on the tensor cores
    if (nchunk > 0) {
      if (warp == 0) {
        if (lane == 0) {   // producer
          int issued = 0;
          bool ok = true;
          for (int k = kb; k < j && ok; ++k) {
            ok = wait_flag(rowcnt + i, k - kb + 1, P.status, 311) && wait_flag(rowcnt + j, k - kb + 1, P.status, 312);
            if (!ok) break;
            asm volatile("fence.proxy.async.global;" ::: "memory");   // the panels were written by other CTAs
            for (int c = 0; c < C::CPP; ++c) {
              const uint32_t gg = g + (uint32_t)issued;
              const int s = (int)(gg % C::NST);
              const uint32_t u = gg / C::NST;
              if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1)) {   // the stage's previous chunk was consumed
                atomicCAS(P.status + 1, 0, 313);
                ok = false;
                break;
              }
              uint8_t* st = sm + s * C::STAGE;
              mbar_expect_tx(&full[s], C::STAGE);
              const int x = k * NB + c * C::CHUNK;
              tma_load_2d(st, &thi, &full[s], x, i * NB);
              tma_load_2d(st + kChunkBytes, &thi, &full[s], x, j * NB);
              if (MODE == 1) {
                tma_load_2d(st + 2 * kChunkBytes, &tlo, &full[s], x, i * NB);
                tma_load_2d(st + 3 * kChunkBytes, &tlo, &full[s], x, j * NB);
              }
              ++issued;
            }
          }
          if (!ok) {
            s_issued = issued;
            __threadfence_block();
            s_stop = 1;
          }
        }
        __syncwarp();
      } else if (warp == 1) {
        if (lane == 0) {   // MMA issue: A = rows of tile i, B = rows of tile j, K-major
          for (int q = 0; q < nchunk; ++q) {
            const uint32_t gg = g + (uint32_t)q;
            const int s = (int)(gg % C::NST);
            const uint32_t u = gg / C::NST;
            if (!mbar_wait_or_stop(&full[s], u & 1, &s_stop, &s_issued, q, P.status, 314)) break;
            fence_after();
            const uint32_t sa = su32(sm + s * C::STAGE), sb = sa + kChunkBytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              mma<KIND>(tmem, sdesc(sa + 32 * kk), sdesc(sb + 32 * kk), ID, (q > 0 || kk > 0) ? 1u : 0u);
              if (MODE == 1) {   // hi.lo + lo.hi
                mma<KIND>(tmem, sdesc(sa + 32 * kk), sdesc(sb + 2 * kChunkBytes + 32 * kk), ID, 1u);
                mma<KIND>(tmem, sdesc(sa + 2 * kChunkBytes + 32 * kk), sdesc(sb + 32 * kk), ID, 1u);
              }
            }
            mma_commit(&empty[s]);   // frees the stage once these MMAs have read it
          }
          mma_commit(&accf);         // arrives when every MMA of the task is done
        }
        __syncwarp();
      }
      if (!mbar_wait(&accf, nacc & 1)) atomicCAS(P.status + 1, 0, 315);
      ++nacc;
      g += (uint32_t)nchunk;
      fence_after();
    }
    __syncthreads();
    if (s_stop) continue;

    // ---- S = A_ij - acc into shared memory (row-major for the diagonal
    // factor, transposed for the panel products)
    if (nchunk > 0) {
      // all eight warps: warp w reads the accumulator lanes of its
      // sub-partition, 32 (w & 3) .. + 31, in columns 64 (w >> 2) .. + 63
      const int r = 32 * (warp & 3) + lane;
      const float* arow = Lt + (int64_t)r * mq;
#pragma unroll 1
      for (int c0 = 64 * (warp >> 2); c0 < 64 * (warp >> 2) + 64; c0 += 32) {
        float4 a[8];
#pragma unroll
        for (int q4 = 0; q4 < 8; ++q4) a[q4] = __ldcg(reinterpret_cast<const float4*>(arow + c0 + 4 * q4));
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int q4 = 0; q4 < 8; ++q4) {
          const float e[4] = {a[q4].x - v[4 * q4], a[q4].y - v[4 * q4 + 1], a[q4].z - v[4 * q4 + 2],
                              a[q4].w - v[4 * q4 + 3]};
          const int c = c0 + 4 * q4;
          if (diag) {
            *reinterpret_cast<float4*>(A + r * SP + c) = make_float4(e[0], e[1], e[2], e[3]);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) ST[(c + u) * SP + r] = e[u];
          }
        }
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < 16; ++k) {
        const int q = tid + 256 * k;
        if (diag) {
          const int r = q >> 5, c = 4 * (q & 31);
          const float4 a = __ldcg(reinterpret_cast<const float4*>(Lt + (int64_t)r * mq + c));
          *reinterpret_cast<float4*>(A + r * SP + c) = a;
        } else {
          const int r = q & 127, c = 4 * (q >> 7);
          const float4 a = __ldcg(reinterpret_cast<const float4*>(Lt + (int64_t)r * mq + c));
          ST[c * SP + r] = a.x; ST[(c + 1) * SP + r] = a.y; ST[(c + 2) * SP + r] = a.z; ST[(c + 3) * SP + r] = a.w;
        }
      }
    }
    fence_before();   // the accumulator reads precede the barrier (the next task overwrites it)
    __syncthreads();

    if (diag) {
      // ---- accumulation task: S_jj back into its tile of L, for the factor CTA
      store_tile(Lt, mq, A);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(scnt + j, 1);
      }
    } else {
      // ---- L_ij from L_ij L_jj^T = S once L_jj is final; then Lh_ij = L_ij Dinv_j
      float* Lj = DT;                      // L_jj, rows of SP
      __shared__ float rinv[NB];
      if (tid == 0 && !wait_flag(rowcnt + j, j - kb + 1, P.status, 316)) s_stop = 1;
      __syncthreads();
      if (s_stop) continue;
      load_tile(Lj, P.L + (int64_t)j * NB * mq + (int64_t)j * NB, mq);
      __syncthreads();
      if (tid < NB) rinv[tid] = 1.f / Lj[tid * SP + tid];
      __syncthreads();
      panel_substitution(ST, Lj, rinv);
      // X (in ST, transposed) -> row-major with padded rows in the L_jj buffer, then coalesced stores
      float* XR = DT;
      for (int q = tid; q < NB * NB; q += 256) {
        const int r = q & 127, c = q >> 7;
        XR[r * PADW + c] = ST[c * SP + r];
      }
      __syncthreads();
      const int64_t off = (int64_t)i * NB * mq + (int64_t)j * NB;
      for (int q = tid; q < NB * NB; q += 256) {
        const int r = q >> 7, c = q & 127;
        const float v = XR[r * PADW + c];
        const int64_t o = off + (int64_t)r * mq + c;
        P.L[o] = v;
        if (MODE == 1) P.Llo[o] = tf32_tail(v);   // TF32 tails for the split products of later tasks
        if (MODE == 2) P.Lb[o] = __float2bfloat16_rn(v);   // BF16 copy for the BF16 products
      }
      asm volatile("fence.proxy.async.global;" ::: "memory");   // later TMA reads of this tile
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(rowcnt + i, j - kb + 1);
      }
      if (tid == 0 && !wait_flag(dcnt + j, 1, P.status, 317)) s_stop = 1;
      __syncthreads();
      if (s_stop) continue;
      const float* Di = P.Dinv + (int64_t)j * NB * NB;
#pragma unroll 4
      for (int k = 0; k < 16; ++k) {   // DT[t][n] = Dinv_j[t][n]
        const int q = tid + 256 * k, t2 = q >> 5, n4 = 4 * (q & 31);
        *reinterpret_cast<float4*>(DT + t2 * SP + n4) = __ldcg(reinterpret_cast<const float4*>(Di + t2 * NB + n4));
      }
      __syncthreads();
      const int ty = tid >> 4, tx = tid & 15;
      float acc[8][8];
      prod_8x8(ST, DT, ty, tx, acc);   // Lh_ij[r][n] = sum_t X[r][t] Dinv_j[t][n]
      store_8x8(P.Lh + off, mq, ty, tx, acc);
    }
    // generic shared-memory accesses of this task precede the next task's TMA writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NB));
  }
}

template <int MODE>
cudaError_t launch(const Args& a, Ptrs p, int ntask, cudaStream_t st) {
  static std::atomic<unsigned long long> attr{0};
  static int per_dev[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (pdk::first_on_device(attr)) {
    cudaFuncSetAttribute(k_chol_ll<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<MODE>::SMEM);
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chol_ll<MODE>, 256, Cfg<MODE>::SMEM);
    per_dev[dev & 63] = nsm * std::max(per, 1);   // one persistent CTA per SM
    // and no more CTA pairs than fit at once (every CTA must be resident)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)per_dev[dev & 63]);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = Cfg<MODE>::SMEM;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_chol_ll<MODE>, &cfg) == cudaSuccess && ncl > 0)
      per_dev[dev & 63] = std::min(per_dev[dev & 63], 2 * ncl);
  }
  // By default two thirds of the SMs: the chain of diagonal tiles, not the
  // tensor-core work, sets the time, and the remaining SMs run the main
  // stream's local step and sparse substitution concurrently.
  int cap = a.max_ctas > 0 ? std::min(per_dev[dev & 63], a.max_ctas) : std::max(8, 2 * per_dev[dev & 63] / 3);
  // one factor CTA, a few inversion CTAs (each inversion is off the
  // critical chain), the rest tensor-core CTAs
  const int nt = a.T - a.kb;
  p.ndiag = 1 + std::min(nt, kDiagCtas - 1);   // the factor CTA and the inversion CTAs
  int grid = std::max(p.ndiag + 1, std::min(p.ndiag + ntask, cap));
  grid += grid & 1;
  const CUtensorMap& lo = a.map_lo ? *a.map_lo : *a.map_hi;
  // Clusters of two: CTA 0 (the factor) shares its TPC with CTA 1 (an
  // inversion CTA, no TMA traffic) rather than with a tensor-core CTA.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = Cfg<MODE>::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_chol_ll<MODE>, *a.map_hi, lo, p);
  ++pdk::g_launches;
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

cudaError_t factor(pdtc::Mode mode, const Args& a, cudaStream_t st) {
  const int nt = a.T - a.kb;
  if (nt <= 0) return cudaSuccess;
  if (!a.map_hi || !a.L || !a.Lh || !a.Dinv || !a.E || !a.sync || !a.status || !a.piv ||
      (mode == pdtc::TF32X3 && (!a.Llo || !a.map_lo)) || (mode == pdtc::BF16 && !a.Lb))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.sync, 0, sync_bytes(a.T), st);
  if (e != cudaSuccess) return e;
  const Ptrs p{0, a.L, a.Llo, a.Lb, a.Lh, a.Dinv, a.E, a.mq, a.T, a.kb, a.sync, a.status, a.piv};
  const int ntask = nt * (nt + 1) / 2 - 1;   // panel and accumulation tasks
  switch (mode) {
    case pdtc::TF32X3: return launch<1>(a, p, ntask, st);
    case pdtc::BF16: return launch<2>(a, p, ntask, st);
    default: return launch<0>(a, p, ntask, st);
  }
}

}  // namespace pdll
