// Learned warm start (see mlp.h).  Every matrix product of the forward and
// backward passes is a tcgen05 GEMM with BF16 operands and FP32 accumulation
// in tensor memory; the epilogues fuse bias, ReLU and the ReLU mask and also
// write the transposed activations, so that every later product again reads
// K-major operands.  Minibatches are drawn on the device from the (features,
// solution) pairs the solver records from its own region solves.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "mixed.h"
#include "mlp.h"
#include "solver.h"
#include "tc.h"
#include "tc_dev.cuh"

namespace pdn {

using bf16 = __nv_bfloat16;

struct Layer {
  int N = 0, K = 0;                       // padded output / input widths
  float *W = nullptr, *b = nullptr;       // FP32 master [N][K], [N]
  float *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
  float *gW = nullptr, *gb = nullptr;
  bf16 *Wb = nullptr, *Wt = nullptr;      // [N][K] and [K][N]
  CUtensorMap mapW{}, mapWt{};
};

struct Net {
  Layer L[4];
  int64_t Bmax = 0, mq = 0;
  bf16 *X = nullptr, *Xt = nullptr, *H[3] = {}, *Ht[3] = {}, *dZ[4] = {}, *dZt[4] = {};
  float *pred = nullptr, *tgt = nullptr;
  CUtensorMap mapX{}, mapXt{}, mapH[3]{}, mapHt[3]{}, mapdZ[4]{}, mapdZt[4]{};
  double* scal = nullptr;     // [0] rms(g), [1] u scale
  double* z0 = nullptr;       // [m][3] contact-free response M0^-1 g
  float* cacc = nullptr;      // [m][4] contact accumulation
  float* Xr = nullptr;        // [m][3] normalised rest positions
  double hbar = 1.0, lscale = 1.0;
  bool have_params = false;
  int64_t rec_cap = 0, rec_rows = 0;
  bf16* recX = nullptr;       // [rec_cap][IN_PAD]
  float* recT = nullptr;      // [rec_cap][3]
  float* recW = nullptr;      // [rec_cap] row weight H_ii / mean diag(Sigma_0) of the recorded solve
  float* wgt = nullptr;       // [Bmax] weights of the current batch
  int loss_kind = 0;          // 0: mean squared error; 1: rows weighted by H_ii (diagonal energy norm)
  int64_t adam_t = 0;
  double* loss_d = nullptr;
  double* loss_h = nullptr;
};

namespace {

using namespace pdtc::dev;

enum { EPI_RELU = 0, EPI_LIN = 1, EPI_MASK = 2, EPI_F32 = 3 };

struct EpiArgs {
  const float* bias;
  const bf16* mask;
  int64_t ldm;
  float* out32;
  int64_t ld32;
  bf16* outb;
  int64_t ldb;
  bf16* outt;
  int64_t ldt;
};

// C[M][N] = A[M][K] B[N][K]^T on 128 x 128 tiles, K in chunks of 64 (BF16).
template <int EPI>
__global__ void __launch_bounds__(128, 1) k_gemm(const __grid_constant__ CUtensorMap ta,
                                                 const __grid_constant__ CUtensorMap tb, int kchunks, int n_tj,
                                                 EpiArgs ep, int* __restrict__ status) {
  constexpr int NST = 4, STAGE = 2 * kChunkBytes;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[NST], done[NST];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  uint8_t* smem = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ti = blockIdx.x / n_tj, tj = blockIdx.x % n_tj;
  const int rowA = ti * kTile, rowB = tj * kTile;
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) { mbar_init(&full[s], 1); mbar_init(&done[s], 1); }
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)), "r"(kTile));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t ID = idesc(1u);
  auto issue = [&](int c) {
    const int s = c % NST;
    uint8_t* st = smem + s * STAGE;
    mbar_expect_tx(&full[s], 2 * kChunkBytes);
    tma_load_2d(st, &ta, &full[s], c * 64, rowA);
    tma_load_2d(st + kChunkBytes, &tb, &full[s], c * 64, rowB);
  };
  if (tid == 0)
    for (int c = 0; c < kchunks && c < NST; ++c) issue(c);
  for (int c = 0; c < kchunks; ++c) {
    const int s = c % NST;
    const uint32_t ph = (uint32_t)((c / NST) & 1);
    if (!mbar_wait(&full[s], ph)) failed = 1;
    __syncthreads();
    if (failed) break;
    if (tid == 0) {
      fence_after();
      const uint32_t sa = su32(smem + s * STAGE), sb = sa + kChunkBytes;
#pragma unroll
      for (int k = 0; k < 4; ++k) mma<1>(tmem, sdesc(sa + 32 * k), sdesc(sb + 32 * k), ID, (c > 0 || k > 0) ? 1u : 0u);
      mma_commit(&done[s]);
      if (c + NST < kchunks) {
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
    const int64_t row = rowA + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < kTile; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      const int64_t col0 = rowB + c0;
      if (EPI == EPI_LIN || EPI == EPI_F32) {
        float* o = ep.out32 + row * ep.ld32 + col0;
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
          float4 x;
          x.x = v[q]; x.y = v[q + 1]; x.z = v[q + 2]; x.w = v[q + 3];
          if (EPI == EPI_LIN) {
            x.x += ep.bias[col0 + q]; x.y += ep.bias[col0 + q + 1];
            x.z += ep.bias[col0 + q + 2]; x.w += ep.bias[col0 + q + 3];
          }
          *reinterpret_cast<float4*>(o + q) = x;
        }
      } else {
        __nv_bfloat162 pk[16];
#pragma unroll
        for (int q = 0; q < 32; q += 2) {
          float x0 = v[q], x1 = v[q + 1];
          if (EPI == EPI_RELU) {
            x0 = fmaxf(x0 + ep.bias[col0 + q], 0.f);
            x1 = fmaxf(x1 + ep.bias[col0 + q + 1], 0.f);
          } else {  // EPI_MASK: ReLU derivative of the layer input
            const bf16* mk = ep.mask + row * ep.ldm + col0;
            if (!(__bfloat162float(mk[q]) > 0.f)) x0 = 0.f;
            if (!(__bfloat162float(mk[q + 1]) > 0.f)) x1 = 0.f;
          }
          pk[q / 2] = __floats2bfloat162_rn(x0, x1);
        }
        uint4* o = reinterpret_cast<uint4*>(ep.outb + row * ep.ldb + col0);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = reinterpret_cast<const uint4*>(pk)[q];
        if (ep.outt) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            ep.outt[(col0 + 2 * q) * ep.ldt + row] = pk[q].x;
            ep.outt[(col0 + 2 * q + 1) * ep.ldt + row] = pk[q].y;
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(status + 1, 110 + EPI);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTile));
  }
}

constexpr int kGemmSmem = 4 * 2 * kChunkBytes + 1024;

// ---- small kernels ----------------------------------------------------------
__global__ void k_sumsq(const double* __restrict__ g, int64_t n, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += g[i] * g[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    out[0] = sqrt(t / (double)(n > 0 ? n : 1));
  }
}
__global__ void k_uscale(double* scal, double hbar) {
  double r = scal[0] > 0.0 ? scal[0] : 1.0;
  scal[0] = r;
  scal[1] = r / hbar;
}
__global__ void k_contact_feat(int64_t k, const int32_t* cidx, const double* cw, const double* ct,
                               const double* cs, const int32_t* region, const double* x, float* cacc) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= k) return;
  const double cs_j = cs[j];
  constexpr int NS = pdk::CSLOTS;
  double p[3] = {0, 0, 0};
  for (int a = 0; a < NS; ++a) {
    int r = cidx[NS * j + a];
    if (r < 0) continue;
    const double* xv = x + 3 * (int64_t)region[r];
    double w = cw[NS * j + a];
    p[0] += w * xv[0]; p[1] += w * xv[1]; p[2] += w * xv[2];
  }
  const double d[3] = {ct[3 * j] - p[0], ct[3 * j + 1] - p[1], ct[3 * j + 2] - p[2]};
  for (int a = 0; a < NS; ++a) {
    int r = cidx[NS * j + a];
    if (r < 0) continue;
    float w = (float)cw[NS * j + a];
    atomicAdd(cacc + 4 * r, w * (float)d[0]);
    atomicAdd(cacc + 4 * r + 1, w * (float)d[1]);
    atomicAdd(cacc + 4 * r + 2, w * (float)d[2]);
    atomicAdd(cacc + 4 * r + 3, (float)(cs_j * cw[NS * j + a] * cw[NS * j + a]));
  }
}
// Features of region node i, linear in g where they are vectors:
// g_i / rms(g), z0_i / s (contact-free response), |g_i| / rms(g), |z0_i| / s,
// contact flag, log(1 + contact stiffness / mean diag Sigma_0), spring
// direction (unit), normalised rest position.  s = rms(g) / mean(diag Sigma_0).
__global__ void k_features(int64_t m, int64_t rows, const double* __restrict__ g, const double* __restrict__ z0,
                           const float* __restrict__ cacc, const float* __restrict__ Xr,
                           const double* __restrict__ scal, double hbar, bf16* __restrict__ X) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows) return;
  float f[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) f[c] = 0.f;
  if (i < m) {
    const double rg = scal[0], us = scal[1];
    float ng = 0.f, nz = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      f[c] = (float)(g[3 * i + c] / rg);
      f[3 + c] = (float)(z0[3 * i + c] / us);
      ng += f[c] * f[c];
      nz += f[3 + c] * f[3 + c];
    }
    f[6] = sqrtf(ng);
    f[7] = sqrtf(nz);
    const float cst = cacc[4 * i + 3];
    f[8] = cst > 0.f ? 1.f : 0.f;
    f[9] = log1pf(cst / (float)hbar);
    const float a0 = cacc[4 * i], a1 = cacc[4 * i + 1], a2 = cacc[4 * i + 2];
    const float dn = sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
    if (dn > 0.f) { f[10] = a0 / dn; f[11] = a1 / dn; f[12] = a2 / dn; }
    f[13] = Xr[3 * i + 2];
  }
  uint4* o = reinterpret_cast<uint4*>(X + i * IN_PAD);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    __nv_bfloat162 p[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) p[t] = __floats2bfloat162_rn(f[8 * q + 2 * t], f[8 * q + 2 * t + 1]);
    o[q] = *reinterpret_cast<uint4*>(p);
  }
  const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int q = 2; q < IN_PAD / 8; ++q) o[q] = z;
}

__global__ void k_transpose_in(const bf16* __restrict__ X, int64_t rows, bf16* __restrict__ Xt, int64_t ldt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows * IN_PAD) return;
  int64_t r = i / IN_PAD, c = i % IN_PAD;
  Xt[c * ldt + r] = X[i];
}
__global__ void k_predict(int64_t m, const float* __restrict__ pred, const double* __restrict__ scal,
                          const double* __restrict__ z0, double* __restrict__ u0) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int c = 0; c < 3; ++c) u0[3 * i + c] = z0[3 * i + c] + (double)pred[i * OUT_PAD + c] * scal[1];
}
// One solve's rows: features, target (u - z0) / s, and the row weight
// H_ii / hbar = (Sigma_0[i][i] + C_22[i][i]) / mean diag(Sigma_0).
__global__ void k_record(int64_t m, const bf16* __restrict__ X, const double* __restrict__ u,
                         const double* __restrict__ z0, const double* __restrict__ scal,
                         const double* __restrict__ S0, const float* __restrict__ cacc, double hbar,
                         bf16* __restrict__ recX, float* __restrict__ recT, float* __restrict__ recW) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint4* src = reinterpret_cast<const uint4*>(X + i * IN_PAD);
  uint4* dst = reinterpret_cast<uint4*>(recX + i * IN_PAD);
  for (int q = 0; q < IN_PAD / 8; ++q) dst[q] = src[q];
  for (int c = 0; c < 3; ++c) recT[3 * i + c] = (float)((u[3 * i + c] - z0[3 * i + c]) / scal[1]);
  recW[i] = (float)((S0[i * m + i] + (double)cacc[4 * i + 3]) / hbar);
}
__device__ __forceinline__ uint64_t mix64(uint64_t z) {   // splitmix64 finaliser
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void k_gather_batch(const bf16* __restrict__ recX, const float* __restrict__ recT,
                               const float* __restrict__ recW, int64_t nrows, int64_t B, uint64_t seed, int64_t step,
                               bf16* __restrict__ X, float* __restrict__ T, float* __restrict__ W) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int64_t r = (int64_t)(mix64(seed ^ mix64((uint64_t)step * 0x100000001B3ull + (uint64_t)b)) % (uint64_t)nrows);
  const uint4* src = reinterpret_cast<const uint4*>(recX + r * IN_PAD);
  uint4* dst = reinterpret_cast<uint4*>(X + b * IN_PAD);
  for (int q = 0; q < IN_PAD / 8; ++q) dst[q] = src[q];
  for (int c = 0; c < 3; ++c) T[3 * b + c] = recT[3 * r + c];
  W[b] = recW[r];
}
// Mean over the first nvalid rows of w_b |pred_b - T_b|^2 / 3 (w = 1 without
// weights); dZ = d loss / d pred (BF16, plus transpose).
__global__ void k_loss(int64_t B, int64_t nvalid, const float* __restrict__ pred, const float* __restrict__ T,
                       const float* __restrict__ wgt, bf16* __restrict__ dZ, bf16* __restrict__ dZt, int64_t ldt,
                       double* __restrict__ loss) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double scale = 1.0 / (3.0 * (double)nvalid);
  const float w = (wgt && b < nvalid) ? wgt[b] : 1.f;
  double l = 0.0;
  for (int c = 0; c < OUT_PAD; ++c) {
    float d = 0.f;
    if (c < OUT && b < nvalid) {
      const float e = pred[b * OUT_PAD + c] - T[3 * b + c];
      l += (double)w * e * e;
      d = (float)(2.0 * scale) * w * e;
    }
    const bf16 v = __float2bfloat16_rn(d);
    dZ[b * OUT_PAD + c] = v;
    dZt[c * ldt + b] = v;
  }
  if (l != 0.0) atomicAdd(loss, l * scale);
}
// gb[n] = sum_b dZt[n][b]
__global__ void k_bias_grad(const bf16* __restrict__ dZt, int64_t ldt, int64_t B, float* __restrict__ gb) {
  const int n = blockIdx.x;
  float s = 0.f;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) s += __bfloat162float(dZt[n * ldt + b]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    gb[n] = t;
  }
}
// Adam on one weight matrix [N][K] (+ BF16 copies) or a bias vector (K == 1, no copies).
__global__ void k_adam(float* __restrict__ p, float* __restrict__ mm, float* __restrict__ vv,
                       const float* __restrict__ gr, int64_t n, int64_t K, float lr, float c1, float c2,
                       bf16* __restrict__ Wb, bf16* __restrict__ Wt, int64_t N) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gr[i];
  const float m1 = 0.9f * mm[i] + 0.1f * g;
  const float v1 = 0.999f * vv[i] + 0.001f * g * g;
  mm[i] = m1;
  vv[i] = v1;
  const float w = p[i] - lr * (m1 / c1) / (sqrtf(v1 / c2) + 1e-8f);
  p[i] = w;
  if (Wb) {
    const bf16 wb = __float2bfloat16_rn(w);
    Wb[i] = wb;
    Wt[(i % K) * N + i / K] = wb;
  }
}
__global__ void k_to_bf16_wt(const float* __restrict__ W, int64_t N, int64_t K, bf16* __restrict__ Wb,
                             bf16* __restrict__ Wt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N * K) return;
  const bf16 wb = __float2bfloat16_rn(W[i]);
  Wb[i] = wb;
  Wt[(i % K) * N + i / K] = wb;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

bool map_bf16(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld) {
  return pdtc::make_map(m, base, 2, (uint64_t)rows, (uint64_t)cols, (uint64_t)ld, 64);
}

template <int EPI>
void gemm(pd_solver* s, const CUtensorMap& a, const CUtensorMap& b, int64_t M, int64_t N, int64_t K,
          const EpiArgs& ep) {
  static std::atomic<unsigned long long> attr{0};
  if (pdk::first_on_device(attr)) cudaFuncSetAttribute(k_gemm<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  const int n_tj = (int)(N / 128);
  k_gemm<EPI><<<(unsigned)((M / 128) * n_tj), 128, kGemmSmem, s->stream>>>(a, b, (int)(K / 64), n_tj, ep, s->status);
  ++pdk::g_launches;
}

EpiArgs epi() {
  EpiArgs e;
  std::memset(&e, 0, sizeof e);
  return e;
}

pd_status ensure_net(pd_solver* s) {
  if (s->net) return PD_OK;
  Net* n = new Net();
  s->net = n;
  auto A = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e == cudaSuccess) { s->allocs.push_back(*p); cudaMemsetAsync(*p, 0, bytes, s->stream); }
    return e != cudaSuccess;
  };
  const int dims[4][2] = {{HID, IN_PAD}, {HID, HID}, {HID, HID}, {OUT_PAD, HID}};
  for (int l = 0; l < 4; ++l) {
    Layer& L = n->L[l];
    L.N = dims[l][0];
    L.K = dims[l][1];
    const size_t nw = (size_t)L.N * L.K;
    if (A((void**)&L.W, 4 * nw) || A((void**)&L.b, 4 * L.N) || A((void**)&L.mW, 4 * nw) || A((void**)&L.vW, 4 * nw) ||
        A((void**)&L.mb, 4 * L.N) || A((void**)&L.vb, 4 * L.N) || A((void**)&L.gW, 4 * nw) || A((void**)&L.gb, 4 * L.N) ||
        A((void**)&L.Wb, 2 * nw) || A((void**)&L.Wt, 2 * nw))
      return PD_ERR_OOM;
    if (!map_bf16(&L.mapW, L.Wb, L.N, L.K, L.K) || !map_bf16(&L.mapWt, L.Wt, L.K, L.N, L.N)) return PD_ERR_CUDA;
  }
  n->mq = ((s->m + 127) / 128) * 128;
  n->Bmax = n->mq > 8192 ? n->mq : 8192;
  const int64_t B = n->Bmax;
  if (A((void**)&n->X, 2 * B * IN_PAD) || A((void**)&n->Xt, 2 * B * IN_PAD) || A((void**)&n->pred, 4 * B * OUT_PAD) ||
      A((void**)&n->tgt, 4 * B * 3) || A((void**)&n->wgt, 4 * B) || A((void**)&n->scal, 8 * 4) ||
      A((void**)&n->cacc, 4 * 4 * s->m) ||
      A((void**)&n->Xr, 4 * 3 * s->m) || A((void**)&n->loss_d, 8) ||
      A((void**)&n->z0, 8 * 3 * s->m))
    return PD_ERR_OOM;
  for (int l = 0; l < 3; ++l)
    if (A((void**)&n->H[l], 2 * B * HID) || A((void**)&n->Ht[l], 2 * B * HID)) return PD_ERR_OOM;
  for (int l = 0; l < 4; ++l) {
    const int w = l == 3 ? OUT_PAD : HID;
    if (A((void**)&n->dZ[l], 2 * B * w) || A((void**)&n->dZt[l], 2 * B * w)) return PD_ERR_OOM;
  }
  if (cudaMallocHost(&n->loss_h, sizeof(double)) != cudaSuccess) return PD_ERR_OOM;
  bool ok = map_bf16(&n->mapX, n->X, B, IN_PAD, IN_PAD) && map_bf16(&n->mapXt, n->Xt, IN_PAD, B, B);
  for (int l = 0; l < 3; ++l)
    ok = ok && map_bf16(&n->mapH[l], n->H[l], B, HID, HID) && map_bf16(&n->mapHt[l], n->Ht[l], HID, B, B);
  for (int l = 0; l < 4; ++l) {
    const int w = l == 3 ? OUT_PAD : HID;
    ok = ok && map_bf16(&n->mapdZ[l], n->dZ[l], B, w, w) && map_bf16(&n->mapdZt[l], n->dZt[l], w, B, B);
  }
  if (!ok) return PD_ERR_CUDA;
  // normalised rest positions of the region and the mean diagonal of Sigma_0
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  const std::vector<double>& Xall = s->X_rest_h;
  for (int64_t i = 0; i < s->m; ++i)
    for (int c = 0; c < 3; ++c) {
      const double v = Xall[3 * (int64_t)s->region_h[i] + c];
      lo[c] = std::min(lo[c], v);
      hi[c] = std::max(hi[c], v);
    }
  double ext = 1e-300;
  for (int c = 0; c < 3; ++c) ext = std::max(ext, hi[c] - lo[c]);
  std::vector<float> Xr_f(3 * s->m);
  for (int64_t i = 0; i < s->m; ++i)
    for (int c = 0; c < 3; ++c)
      Xr_f[3 * i + c] = (float)(2.0 * (Xall[3 * (int64_t)s->region_h[i] + c] - 0.5 * (lo[c] + hi[c])) / ext);
  cudaMemcpy(n->Xr, Xr_f.data(), sizeof(float) * 3 * s->m, cudaMemcpyHostToDevice);
  std::vector<double> dg(s->m);
  cudaMemcpy2D(dg.data(), sizeof(double), s->Sigma0, sizeof(double) * (s->m + 1), sizeof(double), s->m,
               cudaMemcpyDeviceToHost);
  double hb = 0.0;
  for (double v : dg) hb += v;
  n->hbar = hb / (double)s->m;
  n->lscale = 1.0 / std::max(ext / std::cbrt((double)s->m), 1e-12);
  return PD_OK;
}

// forward pass on the first B rows of X; output in pred
void forward(pd_solver* s, Net* n, int64_t B) {
  EpiArgs e = epi();
  e.bias = n->L[0].b; e.outb = n->H[0]; e.ldb = HID; e.outt = n->Ht[0]; e.ldt = n->Bmax;
  gemm<EPI_RELU>(s, n->mapX, n->L[0].mapW, B, HID, IN_PAD, e);
  for (int l = 1; l < 3; ++l) {
    e = epi();
    e.bias = n->L[l].b; e.outb = n->H[l]; e.ldb = HID; e.outt = n->Ht[l]; e.ldt = n->Bmax;
    gemm<EPI_RELU>(s, n->mapH[l - 1], n->L[l].mapW, B, HID, HID, e);
  }
  e = epi();
  e.bias = n->L[3].b; e.out32 = n->pred; e.ld32 = OUT_PAD;
  gemm<EPI_LIN>(s, n->mapH[2], n->L[3].mapW, B, OUT_PAD, HID, e);
}

// loss on the first nvalid rows of a B-row batch, gradients into L[l].gW / gb
// backward pass of the loss of rows 0 .. nvalid-1 (row weights w, or none)
void backward(pd_solver* s, Net* n, int64_t B, int64_t nvalid, const float* w) {
  cudaMemsetAsync(n->loss_d, 0, sizeof(double), s->stream);
  k_loss<<<nblk(B, 128), 128, 0, s->stream>>>(B, nvalid, n->pred, n->tgt, w, n->dZ[3], n->dZt[3], n->Bmax, n->loss_d);
  ++pdk::g_launches;
  for (int l = 3; l >= 0; --l) {
    Layer& L = n->L[l];
    const CUtensorMap& actT = l == 0 ? n->mapXt : n->mapHt[l - 1];
    EpiArgs e = epi();
    e.out32 = L.gW; e.ld32 = L.K;
    gemm<EPI_F32>(s, n->mapdZt[l], actT, L.N, L.K, B, e);     // gW = dZ^T act
    k_bias_grad<<<L.N, 256, 0, s->stream>>>(n->dZt[l], n->Bmax, B, L.gb);
    ++pdk::g_launches;
    if (l > 0) {
      e = epi();
      e.mask = n->H[l - 1]; e.ldm = HID; e.outb = n->dZ[l - 1]; e.ldb = HID; e.outt = n->dZt[l - 1]; e.ldt = n->Bmax;
      gemm<EPI_MASK>(s, n->mapdZ[l], L.mapWt, B, L.K, L.N, e);  // dZ_{l-1} = (dZ_l W_l) * [H_{l-1} > 0]
    }
  }
}

pd_status build_features(pd_solver* s, Net* n, const double* g) {
  cudaStream_t st = s->stream;
  pd_status r = pdm::apply_free(s, g, n->z0);
  if (r != PD_OK) return r;
  k_sumsq<<<1, 1024, 0, st>>>(g, 3 * s->m, n->scal);
  k_uscale<<<1, 1, 0, st>>>(n->scal, n->hbar);
  cudaMemsetAsync(n->cacc, 0, sizeof(float) * 4 * s->m, st);
  if (s->k > 0) {
    k_contact_feat<<<nblk(s->k, 128), 128, 0, st>>>(s->k, s->c_idx, s->c_w, s->c_t, s->c_s, s->d_region, s->x, n->cacc);
    ++pdk::g_launches;
  }
  k_features<<<nblk(n->mq, 128), 128, 0, st>>>(s->m, n->mq, g, n->z0, n->cacc, n->Xr, n->scal, n->hbar, n->X);
  pdk::g_launches += 3;
  return PD_OK;
}

}  // namespace

// ------------------------------------------------------------------ API pieces
pd_status set_params(pd_solver* s, const float* p) {
  pd_status r = ensure_net(s);
  if (r != PD_OK) return r;
  Net* n = s->net;
  // logical layout -> padded master weights
  std::vector<float> buf;
  const float* q = p;
  for (int l = 0; l < 4; ++l) {
    Layer& L = n->L[l];
    const int rows = l == 3 ? OUT : HID, cols = l == 0 ? IN : HID;
    buf.assign((size_t)L.N * L.K, 0.f);
    for (int i = 0; i < rows; ++i)
      for (int j = 0; j < cols; ++j) buf[(size_t)i * L.K + j] = *q++;
    cudaMemcpyAsync(L.W, buf.data(), 4 * buf.size(), cudaMemcpyHostToDevice, s->stream);
    cudaStreamSynchronize(s->stream);
    buf.assign(L.N, 0.f);
    for (int i = 0; i < rows; ++i) buf[i] = *q++;
    cudaMemcpyAsync(L.b, buf.data(), 4 * buf.size(), cudaMemcpyHostToDevice, s->stream);
    cudaStreamSynchronize(s->stream);
    cudaMemsetAsync(L.mW, 0, 4 * (size_t)L.N * L.K, s->stream);
    cudaMemsetAsync(L.vW, 0, 4 * (size_t)L.N * L.K, s->stream);
    cudaMemsetAsync(L.mb, 0, 4 * L.N, s->stream);
    cudaMemsetAsync(L.vb, 0, 4 * L.N, s->stream);
    k_to_bf16_wt<<<nblk((int64_t)L.N * L.K, 256), 256, 0, s->stream>>>(L.W, L.N, L.K, L.Wb, L.Wt);
    ++pdk::g_launches;
  }
  n->adam_t = 0;
  n->have_params = true;
  return cudaStreamSynchronize(s->stream) == cudaSuccess ? PD_OK : PD_ERR_CUDA;
}

static void grads_to_logical(pd_solver* s, Net* n, float* out) {
  std::vector<float> buf;
  float* q = out;
  for (int l = 0; l < 4; ++l) {
    Layer& L = n->L[l];
    const int rows = l == 3 ? OUT : HID, cols = l == 0 ? IN : HID;
    buf.resize((size_t)L.N * L.K);
    cudaMemcpy(buf.data(), L.gW, 4 * buf.size(), cudaMemcpyDeviceToHost);
    for (int i = 0; i < rows; ++i)
      for (int j = 0; j < cols; ++j) *q++ = buf[(size_t)i * L.K + j];
    buf.resize(L.N);
    cudaMemcpy(buf.data(), L.gb, 4 * L.N, cudaMemcpyDeviceToHost);
    for (int i = 0; i < rows; ++i) *q++ = buf[i];
  }
}

pd_status get_params(pd_solver* s, float* out) {
  if (!s->net || !s->net->have_params) { s->err = "network parameters not set"; return PD_ERR_INVALID_ARG; }
  Net* n = s->net;
  cudaStreamSynchronize(s->stream);
  std::vector<float> buf;
  float* q = out;
  for (int l = 0; l < 4; ++l) {
    Layer& L = n->L[l];
    const int rows = l == 3 ? OUT : HID, cols = l == 0 ? IN : HID;
    buf.resize((size_t)L.N * L.K);
    cudaMemcpy(buf.data(), L.W, 4 * buf.size(), cudaMemcpyDeviceToHost);
    for (int i = 0; i < rows; ++i)
      for (int j = 0; j < cols; ++j) *q++ = buf[(size_t)i * L.K + j];
    buf.resize(L.N);
    cudaMemcpy(buf.data(), L.b, 4 * L.N, cudaMemcpyDeviceToHost);
    for (int i = 0; i < rows; ++i) *q++ = buf[i];
  }
  return PD_OK;
}

pd_status record(pd_solver* s, int64_t max_solves) {
  pd_status r = ensure_net(s);
  if (r != PD_OK) return r;
  Net* n = s->net;
  const int64_t cap = max_solves * s->m;
  if (cap > n->rec_cap) {
    bf16* x = nullptr;
    float *t = nullptr, *w = nullptr;
    if (cudaMalloc(&x, 2 * cap * IN_PAD) != cudaSuccess) return PD_ERR_OOM;
    if (cudaMalloc(&t, 4 * cap * 3) != cudaSuccess) { cudaFree(x); return PD_ERR_OOM; }
    if (cudaMalloc(&w, 4 * cap) != cudaSuccess) { cudaFree(x); cudaFree(t); return PD_ERR_OOM; }
    cudaFree(n->recX);
    cudaFree(n->recT);
    cudaFree(n->recW);
    n->recX = x;
    n->recT = t;
    n->recW = w;
    n->rec_cap = cap;
  }
  n->rec_rows = 0;
  s->mlp_recording = max_solves > 0;
  return PD_OK;
}

pd_status train(pd_solver* s, int64_t steps, int64_t batch, double lr, uint64_t seed, double* loss) {
  Net* n = s->net;
  if (!n || !n->have_params) { s->err = "network parameters not set"; return PD_ERR_INVALID_ARG; }
  if (n->rec_rows < 1) { s->err = "no recorded solves to train on"; return PD_ERR_INVALID_ARG; }
  if (batch < 128 || batch % 128 || batch > n->Bmax) { s->err = "batch must be a multiple of 128 and <= 8192"; return PD_ERR_INVALID_ARG; }
  double acc = 0.0;
  int64_t cnt = 0;
  for (int64_t it = 0; it < steps; ++it) {
    k_gather_batch<<<nblk(batch, 128), 128, 0, s->stream>>>(n->recX, n->recT, n->recW, n->rec_rows, batch, seed,
                                                            n->adam_t, n->X, n->tgt, n->wgt);
    k_transpose_in<<<nblk(batch * IN_PAD, 256), 256, 0, s->stream>>>(n->X, batch, n->Xt, n->Bmax);
    pdk::g_launches += 2;
    forward(s, n, batch);
    backward(s, n, batch, batch, n->loss_kind == 1 ? n->wgt : nullptr);
    ++n->adam_t;
    const float c1 = 1.f - powf(0.9f, (float)n->adam_t), c2 = 1.f - powf(0.999f, (float)n->adam_t);
    for (int l = 0; l < 4; ++l) {
      Layer& L = n->L[l];
      const int64_t nw = (int64_t)L.N * L.K;
      k_adam<<<nblk(nw, 256), 256, 0, s->stream>>>(L.W, L.mW, L.vW, L.gW, nw, L.K, (float)lr, c1, c2, L.Wb, L.Wt, L.N);
      k_adam<<<nblk(L.N, 256), 256, 0, s->stream>>>(L.b, L.mb, L.vb, L.gb, L.N, 1, (float)lr, c1, c2, nullptr, nullptr, 1);
      pdk::g_launches += 2;
    }
    if (it + 20 >= steps) {   // average the loss of the last steps
      cudaMemcpyAsync(n->loss_h, n->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
      cudaStreamSynchronize(s->stream);
      acc += *n->loss_h;
      ++cnt;
    }
  }
  if (loss) *loss = cnt ? acc / cnt : 0.0;
  return cudaStreamSynchronize(s->stream) == cudaSuccess ? PD_OK : PD_ERR_CUDA;
}

// Mean squared error of the network over all recorded rows, and of the zero
// prediction (the mean squared target), both in the scaled units; with the
// weighted loss both are weighted by the rows' H_ii.
__global__ void k_sq_targets(const float* __restrict__ T, const float* __restrict__ W, int64_t n, double* out) {
  __shared__ double red[32];
  double s2 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s2 += (W ? (double)W[i / 3] : 1.0) * T[i] * T[i];
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(out, t);
  }
}

pd_status eval(pd_solver* s, double* mse_net, double* mse_zero) {
  Net* n = s->net;
  if (!n || !n->have_params || n->rec_rows < 1) { s->err = "need parameters and recorded solves"; return PD_ERR_INVALID_ARG; }
  double net_sum = 0.0;
  const int64_t Bt = 8192;
  for (int64_t r0 = 0; r0 < n->rec_rows; r0 += Bt) {
    const int64_t nv = std::min(Bt, n->rec_rows - r0);
    const int64_t Bp = ((nv + 127) / 128) * 128;
    cudaMemsetAsync(n->X, 0, 2 * Bp * IN_PAD, s->stream);
    cudaMemcpyAsync(n->X, n->recX + r0 * IN_PAD, 2 * nv * IN_PAD, cudaMemcpyDeviceToDevice, s->stream);
    cudaMemcpyAsync(n->tgt, n->recT + r0 * 3, 4 * nv * 3, cudaMemcpyDeviceToDevice, s->stream);
    cudaMemcpyAsync(n->wgt, n->recW + r0, 4 * nv, cudaMemcpyDeviceToDevice, s->stream);
    forward(s, n, Bp);
    cudaMemsetAsync(n->loss_d, 0, sizeof(double), s->stream);
    k_loss<<<nblk(Bp, 128), 128, 0, s->stream>>>(Bp, nv, n->pred, n->tgt, n->loss_kind == 1 ? n->wgt : nullptr,
                                                  n->dZ[3], n->dZt[3], n->Bmax, n->loss_d);
    ++pdk::g_launches;
    cudaMemcpyAsync(n->loss_h, n->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return PD_ERR_CUDA;
    net_sum += *n->loss_h * (3.0 * nv);
  }
  cudaMemsetAsync(n->loss_d, 0, sizeof(double), s->stream);
  k_sq_targets<<<148, 256, 0, s->stream>>>(n->recT, n->loss_kind == 1 ? n->recW : nullptr, 3 * n->rec_rows,
                                           n->loss_d);
  ++pdk::g_launches;
  cudaMemcpyAsync(n->loss_h, n->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return PD_ERR_CUDA;
  if (mse_net) *mse_net = net_sum / (3.0 * n->rec_rows);
  if (mse_zero) *mse_zero = *n->loss_h / (3.0 * n->rec_rows);
  return PD_OK;
}

pd_status set_loss(pd_solver* s, int kind) {
  pd_status r = ensure_net(s);
  if (r != PD_OK) return r;
  s->net->loss_kind = kind;
  return PD_OK;
}

pd_status loss_grad(pd_solver* s, const float* X, const float* T, int64_t B, double* loss, float* grad) {
  Net* n = s->net;
  if (!n || !n->have_params) { s->err = "network parameters not set"; return PD_ERR_INVALID_ARG; }
  if (B < 1 || B > n->Bmax) { s->err = "batch size out of range"; return PD_ERR_INVALID_ARG; }
  const int64_t Bp = ((B + 127) / 128) * 128;
  std::vector<bf16> xb((size_t)Bp * IN_PAD, __float2bfloat16(0.f));
  std::vector<float> tb((size_t)Bp * 3, 0.f);
  for (int64_t i = 0; i < B; ++i) {
    for (int c = 0; c < IN; ++c) xb[i * IN_PAD + c] = __float2bfloat16_rn(X[i * IN + c]);
    for (int c = 0; c < 3; ++c) tb[i * 3 + c] = T[i * 3 + c];
  }
  cudaMemcpy(n->X, xb.data(), 2 * xb.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(n->tgt, tb.data(), 4 * tb.size(), cudaMemcpyHostToDevice);
  k_transpose_in<<<nblk(Bp * IN_PAD, 256), 256, 0, s->stream>>>(n->X, Bp, n->Xt, n->Bmax);
  ++pdk::g_launches;
  forward(s, n, Bp);
  backward(s, n, Bp, B, nullptr);
  cudaMemcpyAsync(n->loss_h, n->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return PD_ERR_CUDA;
  if (loss) *loss = *n->loss_h;
  if (grad) grads_to_logical(s, n, grad);
  return PD_OK;
}

pd_status before_solve(pd_solver* s, const double* g, double* u0) {
  Net* n = s->net;
  if (!n) return PD_OK;
  const bool want_pred = u0 && n->have_params;
  if (!want_pred && !s->mlp_recording) return PD_OK;
  pd_status r = build_features(s, n, g);
  if (r != PD_OK) return r;
  if (want_pred) {
    forward(s, n, n->mq);
    k_predict<<<nblk(s->m, 128), 128, 0, s->stream>>>(s->m, n->pred, n->scal, n->z0, u0);
    ++pdk::g_launches;
  }
  return PD_OK;
}

pd_status after_solve(pd_solver* s, const double* u) {
  Net* n = s->net;
  if (!n) return PD_OK;
  if (s->mlp_recording && n->rec_rows + s->m <= n->rec_cap) {
    k_record<<<nblk(s->m, 128), 128, 0, s->stream>>>(s->m, n->X, u, n->z0, n->scal, s->Sigma0, n->cacc, n->hbar,
                                                       n->recX + n->rec_rows * IN_PAD, n->recT + n->rec_rows * 3,
                                                       n->recW + n->rec_rows);
    ++pdk::g_launches;
    n->rec_rows += s->m;
  }
  return PD_OK;
}

void free_net(pd_solver* s) {
  if (!s->net) return;
  cudaFree(s->net->recX);
  cudaFree(s->net->recT);
  cudaFree(s->net->recW);
  if (s->net->loss_h) cudaFreeHost(s->net->loss_h);
  delete s->net;
  s->net = nullptr;
}

}  // namespace pdn
