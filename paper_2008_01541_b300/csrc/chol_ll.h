// Persistent left-looking low-precision Cholesky of the equilibrated
// collision-region matrix D H D (Section 3.3: the dense refactorisation of
// Algorithm 1, step 4.5), one launch for the whole factor.
//
// Tile (i, j), i >= j, of 128 x 128 is one task: S = A_ij - sum_{kb <= k < j}
// L_ik L_jk^T is accumulated on the tensor cores (tcgen05, TF32 / split TF32
// / BF16 operands, FP32 accumulator in tensor memory) from TMA loads that
// start as soon as the panels they read are final; then either the panel
// tile solves L_ij L_jj^T = S by blocked substitution (published at once) and
// then forms Lh_ij = L_ij Dinv_j, or, for a diagonal tile, S_jj goes back to
// global memory, where one CTA that does nothing else factors it in FP32
// (L_jj, published at once) and a few others invert it (Dinv_j = L_jj^-1,
// E_j = Dinv_j^T Dinv_j).  The tensor-core tasks run in column-major order;
// each task waits only on earlier ones, through per-row counters in global
// memory; every wait is bounded.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tc.h"

namespace pdll {

struct Args {
  const CUtensorMap* map_hi = nullptr;   // L (FP32, box 32 x 128) or, for BF16, Lb (box 64 x 128)
  const CUtensorMap* map_lo = nullptr;   // Llo (FP32, box 32 x 128); split TF32 only
  float* L = nullptr;                    // [mq][mq] row-major: lower tiles in = D H D, out = the factor
  float* Llo = nullptr;                  // [mq][mq] split TF32: L - tf32(L) of the finished panel tiles
  __nv_bfloat16* Lb = nullptr;           // [mq][mq] BF16: the finished panel tiles rounded to BF16
  float* Lh = nullptr;                   // [mq][mq] Lh_ij = L_ij Dinv_j (i > j)
  float* Dinv = nullptr;                 // [T][128][128] inverses of the diagonal tiles
  float* E = nullptr;                    // [T][128][128] Dinv_j^T Dinv_j
  int64_t mq = 0;                        // padded order, T * 128
  int T = 0;
  int kb = 0;                            // first tile column factored (earlier panels are final and unused)
  int* sync = nullptr;                   // sync_bytes(T) of scratch (zeroed by factor())
  int max_ctas = 0;                      // cap on the persistent grid (0: two thirds of the SMs)
  int* status = nullptr;                 // [1] receives a wait failure code
  int* piv = nullptr;                    // [0] first non-positive pivot + 1 (replaced by 1 in the factor)
};

inline size_t sync_bytes(int T) { return sizeof(int) * (2 + 3 * (size_t)T); }

// Launch the factorisation of tile columns kb .. T-1 on st.
cudaError_t factor(pdtc::Mode mode, const Args& a, cudaStream_t st);

}  // namespace pdll
