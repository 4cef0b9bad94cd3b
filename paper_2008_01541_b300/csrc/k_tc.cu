// tcgen05 rank-K tile update (see tc.h).  One CTA of 128 threads per 128x128
// output tile: thread 0 issues the TMA loads and the MMAs (M = N = 128), the
// accumulator lives in 128 TMEM columns, and all four warps run the epilogue
// (tcgen05.ld of their 32 TMEM lanes, then C -= acc in global memory).
// Every mbarrier wait is bounded; on timeout the CTA records a code in
// status[1], frees its TMEM and returns.
#include <cudaTypedefs.h>

#include <cstdio>

#include <cuda_bf16.h>

#include "kernels.h"
#include "pd.h"
#include "tc.h"
#include "tc_dev.cuh"

namespace pdtc {
namespace {
using namespace dev;

// MODE: 0 = TF32, 1 = 3xTF32 (hi*hi + hi*lo + lo*hi), 2 = BF16.  NSTAGE: stages
// resident in shared memory (0: the default that keeps three CTAs per SM; a
// one-wave launch such as the look-ahead column takes two stages instead, so
// the next chunk's loads overlap the current chunk's MMAs).
template <int MODE, int NSTAGE>
__global__ void __launch_bounds__(128, 3)
    k_rank_k(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int kx0, int kchunks,
             float* __restrict__ C, int64_t ldc, int ti0, int tj0, int n_j, int lower, int* __restrict__ status) {
  constexpr int NST = NSTAGE > 0 ? NSTAGE : ((MODE == 1) ? 1 : 2);
  constexpr int STAGE = (MODE == 1) ? 4 * kChunkBytes : 2 * kChunkBytes;  // A, B (+ A_lo, B_lo)
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[NST], done[NST];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  uint8_t* smem = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // tile of this CTA
  int ti, tj;
  if (lower) {
    int64_t idx = blockIdx.x;
    int64_t i = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= idx) ++i;
    while (i * (i + 1) / 2 > idx) --i;
    ti = (int)i;
    tj = (int)(idx - i * (i + 1) / 2);
  } else {
    ti = blockIdx.x / n_j;
    tj = blockIdx.x % n_j;
  }
  const int rowA = (ti0 + ti) * kTile, rowB = (tj0 + tj) * kTile;

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) { mbar_init(&full[s], 1); mbar_init(&done[s], 1); }
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(kTile));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  constexpr int KIND = (MODE == 2) ? 1 : 0;
  constexpr uint32_t ID = idesc(MODE == 2 ? 1u : 2u);
  const int chunk_elems = (MODE == 2) ? 64 : 32;   // 128 B of K per chunk

  auto issue = [&](int c) {
    int s = c % NST;
    uint8_t* st = smem + s * STAGE;
    mbar_expect_tx(&full[s], 2 * kChunkBytes);
    tma_load_2d(st, &ta, &full[s], kx0 + c * chunk_elems, rowA);
    tma_load_2d(st + kChunkBytes, &tb, &full[s], kx0 + c * chunk_elems, rowB);
  };
  if (tid == 0)
    for (int c = 0; c < kchunks && c < NST; ++c) issue(c);

  for (int c = 0; c < kchunks; ++c) {
    const int s = c % NST;
    const uint32_t ph = (uint32_t)((c / NST) & 1);
    uint8_t* st = smem + s * STAGE;
    if (!mbar_wait(&full[s], ph)) failed = 1;
    __syncthreads();
    if (failed) break;
    if (MODE == 1) {   // split each FP32 operand into a TF32 head and an FP32 remainder
      const float* a = reinterpret_cast<const float*>(st);
      const float* b = reinterpret_cast<const float*>(st + kChunkBytes);
      float* alo = reinterpret_cast<float*>(st + 2 * kChunkBytes);
      float* blo = reinterpret_cast<float*>(st + 3 * kChunkBytes);
      for (int q = tid; q < kChunkBytes / 4; q += 128) {
        float x = a[q], y = b[q];
        float xh = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
        float yh = __uint_as_float(__float_as_uint(y) & 0xFFFFE000u);
        alo[q] = x - xh;
        blo[q] = y - yh;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
    }
    if (tid == 0) {
      fence_after();
      const uint32_t sa = su32(st), sb = su32(st + kChunkBytes);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
        mma<KIND>(tmem, sdesc(sa + 32 * k), sdesc(sb + 32 * k), ID, acc);
        if (MODE == 1) {
          const uint32_t salo = su32(st + 2 * kChunkBytes), sblo = su32(st + 3 * kChunkBytes);
          mma<KIND>(tmem, sdesc(sa + 32 * k), sdesc(sblo + 32 * k), ID, 1u);
          mma<KIND>(tmem, sdesc(salo + 32 * k), sdesc(sb + 32 * k), ID, 1u);
        }
      }
      mma_commit(&done[s]);
      if (c + NST < kchunks) {   // refill this stage once its MMAs have read it
        if (!mbar_wait(&done[s], ph)) failed = 1;
        else issue(c + NST);
      }
    }
  }
  __syncthreads();
  if (!failed && kchunks > 0) {
    const int last = kchunks - 1;
    if (!mbar_wait(&done[last % NST], (uint32_t)((last / NST) & 1))) failed = 1;
  }
  __syncthreads();
  fence_after();
  if (!failed) {
    const int r = warp * 32 + lane;
    float* crow = C + (int64_t)(rowA + r) * ldc + rowB;
#pragma unroll 1
    for (int c0 = 0; c0 < kTile; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      float4* p = reinterpret_cast<float4*>(crow + c0);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float4 x = p[q];
        x.x -= v[4 * q]; x.y -= v[4 * q + 1]; x.z -= v[4 * q + 2]; x.w -= v[4 * q + 3];
        p[q] = x;
      }
    }
  } else if (tid == 0) {
    atomicExch(status + 1, 100 + MODE);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTile));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

template <int MODE, int NSTAGE = 0>
constexpr int smem_bytes() {
  return (NSTAGE > 0 ? NSTAGE : ((MODE == 1) ? 1 : 2)) * ((MODE == 1) ? 4 : 2) * kChunkBytes + 1024;
}

}  // namespace

bool make_map(CUtensorMap* map, const void* base, int esize, uint64_t rows, uint64_t cols, uint64_t ld_elems,
              uint32_t box_cols) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld_elems * (uint64_t)esize};
  cuuint32_t box[2] = {box_cols, (cuuint32_t)kTile};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

void rank_k_update(Mode mode, const CUtensorMap* a, const CUtensorMap* b, int kx0, int kchunks, float* C,
                   int64_t ldc, int ti0, int tj0, int n_i, int n_j, int lower, int* status, cudaStream_t st) {
  static std::atomic<unsigned long long> attr[4];
  unsigned grid = lower ? (unsigned)((int64_t)n_i * (n_i + 1) / 2) : (unsigned)(n_i * n_j);
  if (grid == 0 || kchunks <= 0) return;
  switch (mode) {
    case TF32:
      if (pdk::first_on_device(attr[0])) cudaFuncSetAttribute(k_rank_k<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<0>());
      k_rank_k<0, 0><<<grid, 128, smem_bytes<0>(), st>>>(*a, *b, kx0, kchunks, C, ldc, ti0, tj0, n_j, lower, status);
      break;
    case TF32X3:
      if (grid <= 148 && kchunks > 1) {   // one wave: two stages, one CTA per SM
        if (pdk::first_on_device(attr[3])) cudaFuncSetAttribute(k_rank_k<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<1, 2>());
        k_rank_k<1, 2><<<grid, 128, smem_bytes<1, 2>(), st>>>(*a, *b, kx0, kchunks, C, ldc, ti0, tj0, n_j, lower, status);
      } else {
        if (pdk::first_on_device(attr[1])) cudaFuncSetAttribute(k_rank_k<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<1>());
        k_rank_k<1, 0><<<grid, 128, smem_bytes<1>(), st>>>(*a, *b, kx0, kchunks, C, ldc, ti0, tj0, n_j, lower, status);
      }
      break;
    default:
      if (pdk::first_on_device(attr[2])) cudaFuncSetAttribute(k_rank_k<2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<2>());
      k_rank_k<2, 0><<<grid, 128, smem_bytes<2>(), st>>>(*a, *b, kx0, kchunks, C, ldc, ti0, tj0, n_j, lower, status);
      break;
  }
  ++pdk::g_launches;
}

}  // namespace pdtc

namespace {
__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}
}  // namespace

// Diagnostic entry point: C -= A B^T on the tensor cores (see pd.h).
extern "C" pd_status pd_tc_rank_k(int mode, const float* A, const float* B, float* C, int64_t M, int64_t N,
                                  int64_t K, void* stream) {
  if (!A || !B || !C || M <= 0 || N <= 0 || M % 128 || N % 128 || K != 128 || mode < 0 || mode > 2)
    return PD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const void* a = A;
  const void* b = B;
  __nv_bfloat16 *ab = nullptr, *bb = nullptr;
  int* status = nullptr;
  pd_status ret = PD_OK;
  if (cudaMalloc(&status, 4 * sizeof(int)) != cudaSuccess) return PD_ERR_OOM;
  cudaMemsetAsync(status, 0, 4 * sizeof(int), st);
  if (mode == 2) {
    if (cudaMalloc(&ab, M * K * 2) != cudaSuccess || cudaMalloc(&bb, N * K * 2) != cudaSuccess) {
      cudaFree(ab); cudaFree(bb); cudaFree(status);
      return PD_ERR_OOM;
    }
    k_to_bf16<<<(unsigned)((M * K + 255) / 256), 256, 0, st>>>(A, ab, M * K);
    k_to_bf16<<<(unsigned)((N * K + 255) / 256), 256, 0, st>>>(B, bb, N * K);
    a = ab;
    b = bb;
  }
  CUtensorMap ma, mb;
  const int esize = mode == 2 ? 2 : 4, box = mode == 2 ? 64 : 32;
  if (!pdtc::make_map(&ma, a, esize, M, K, K, box) || !pdtc::make_map(&mb, b, esize, N, K, K, box)) {
    ret = PD_ERR_CUDA;
  } else {
    pdtc::rank_k_update((pdtc::Mode)mode, &ma, &mb, 0, mode == 2 ? 2 : 4, C, N, 0, 0, (int)(M / 128),
                        (int)(N / 128), 0, status, st);
    int h[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(h, status, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      ret = PD_ERR_CUDA;
    else if (h[1])
      ret = PD_ERR_TIMEOUT;
  }
  cudaStreamSynchronize(st);
  cudaFree(ab); cudaFree(bb); cudaFree(status);
  return ret;
}
