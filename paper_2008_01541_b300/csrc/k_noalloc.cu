// Allocation-free variant of the FP64 Schur refactor + solve.
//
// Some callers cannot allocate device memory while they run: an engine that
// reserves every byte of the GPU up front and forbids cudaMalloc/cudaFree
// during a frame, a memory-pool or arena integration, or a real-time loop that
// cannot afford the implicit device synchronisation an allocation can cause.
// They can still call pd_schur_solve_noalloc(): its working memory (the
// padded matrix being factored, the inverses of the diagonal tiles, the
// triangular-solve workspace and the status words) lives in one file-scope
// __device__ array that the driver creates when it loads this library, and
// that every device which loads the library keeps until the process exits.
#include <cstdio>
#include <cstring>

#include "kernels.h"
#include "pd.h"

namespace {

constexpr int64_t kMaxM = 1024;                  // largest supported collision region
constexpr int64_t kHElems = kMaxM * kMaxM;       // padded H, column-major
constexpr int64_t kLinvElems = kMaxM * 64;       // inverses of the 64x64 diagonal tiles
constexpr int64_t kWorkElems = 6 * kMaxM;        // blocked triangular-solve workspace
constexpr int64_t kStatusElems = 4;              // 4 doubles = room for the int status words
constexpr int64_t kScratchElems = kHElems + kLinvElems + kWorkElems + kStatusElems;

// About 8.5 MB of device memory per device that loads the library.
static __device__ __align__(256) double noalloc_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
double* g_scratch_dev[kMaxDevices] = {nullptr};

void set_err(char* err, int64_t len, const char* msg) {
  if (!err || len <= 0) return;
  std::snprintf(err, (size_t)len, "%s", msg);
}

}  // namespace

extern "C" pd_status pd_schur_solve_noalloc(const double* sigma_dev, int64_t m, int64_t k,
                                            const int32_t* cidx_dev, const double* cw_dev,
                                            const double* cs_dev, const double* g_dev, double* u_dev,
                                            void* cuda_stream, char* err, int64_t err_len) {
  set_err(err, err_len, "");
  if (m < 1 || m > kMaxM) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "pd_schur_solve_noalloc: m = %lld is outside [1, %lld]",
                  (long long)m, (long long)kMaxM);
    set_err(err, err_len, msg);
    return PD_ERR_INVALID_ARG;
  }
  if (!sigma_dev || !g_dev || !u_dev || k < 0 || (k > 0 && (!cidx_dev || !cw_dev || !cs_dev))) {
    set_err(err, err_len, "pd_schur_solve_noalloc: null pointer or negative k");
    return PD_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_err(err, err_len, "pd_schur_solve_noalloc: no usable current device");
    return PD_ERR_CUDA;
  }
  // One-time set-up per device (the first call on each device): look up the
  // device address of the scratch array with that device current.
  if (!g_scratch_dev[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_err(err, err_len, cudaGetErrorString(e));
      return PD_ERR_CUDA;
    }
    g_scratch_dev[dev] = p;
  }
  // Contact indices must name region rows: check them on the host in
  // fixed-size chunks (no allocation).
  int32_t chunk[1024];
  for (int64_t q = 0; q < 4 * k; q += 1024) {
    int64_t len = (4 * k - q) < 1024 ? (4 * k - q) : 1024;
    e = cudaMemcpyAsync(chunk, cidx_dev + q, sizeof(int32_t) * len, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_err(err, err_len, cudaGetErrorString(e));
      return PD_ERR_CUDA;
    }
    for (int64_t i = 0; i < len; ++i)
      if (chunk[i] < -1 || chunk[i] >= m) {
        set_err(err, err_len, "pd_schur_solve_noalloc: contact index outside [-1, m)");
        return PD_ERR_CONTACT_OUTSIDE_REGION;
      }
  }
  const int64_t mp = ((m + 63) / 64) * 64;
  double* H = g_scratch_dev[dev];
  double* Linv = H + kHElems;
  double* work = Linv + kLinvElems;
  int* status = reinterpret_cast<int*>(work + kWorkElems);
  // The array keeps the previous call's contents: the status words must start at zero.
  e = cudaMemsetAsync(status, 0, sizeof(int) * 4, st);
  if (e != cudaSuccess) {
    set_err(err, err_len, cudaGetErrorString(e));
    return PD_ERR_CUDA;
  }
  pdk::copy_sigma(sigma_dev, m, H, mp, st);
  pdk::contact_scatter(k, cidx_dev, cw_dev, cs_dev, H, mp, st, 4);
  pdk::cholesky_fp64(H, mp, Linv, status, st);
  pdk::chol_solve_fp64(H, mp, Linv, g_dev, u_dev, m, work, st);
  int status_h[4] = {0, 0, 0, 0};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(status_h, status, sizeof status_h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_err(err, err_len, cudaGetErrorString(e));
    return PD_ERR_CUDA;
  }
  if (status_h[0] != 0) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "pd_schur_solve_noalloc: pivot %d is not positive", status_h[0] - 1);
    set_err(err, err_len, msg);
    return PD_ERR_NOT_SPD;
  }
  return PD_OK;
}
