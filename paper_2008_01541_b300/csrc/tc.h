// tcgen05 (5th-generation tensor core) rank-K update: C -= A B^T on 128x128
// tiles, operands fed by TMA into 128B-swizzled shared memory, accumulator in
// tensor memory.  Used for the trailing updates of the low-precision
// Cholesky of the collision-region matrix.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace pdtc {

enum Mode { TF32 = 0, TF32X3 = 1, BF16 = 2 };

// 2-D row-major tensor map (cols contiguous) with a box of box_cols x 128 rows
// and 128B swizzle.  esize = 4 (FP32) or 2 (BF16).  Returns false on failure.
bool make_map(CUtensorMap* map, const void* base, int esize, uint64_t rows, uint64_t cols, uint64_t ld_elems,
              uint32_t box_cols);

// For every 128x128 tile (ti, tj) of C selected by the launch, C_tile -= A_i B_j^T,
// A_i = rows (ti0 + ti)*128.. of map a, B_j = rows (tj0 + tj)*128.. of map b,
// K = 128 columns starting at column kx0 of the maps (element units).
// lower != 0: tiles tj <= ti of an n x n block (n*(n+1)/2 CTAs); else n_i x n_j.
// status[1] receives a nonzero code if a bounded wait gives up.
void rank_k_update(Mode mode, const CUtensorMap* a, const CUtensorMap* b, int kx0, int kchunks, float* C,
                   int64_t ldc, int ti0, int tj0, int n_i, int n_j, int lower, int* status, cudaStream_t st);

}  // namespace pdtc
