// Collision detection on the device (Algorithm 1, step 4.1 DetectCollisions),
// run at every inner iteration instead of a host callback.  Every proxy owns
// one fixed spring slot, so the spring count never has to travel back to the
// host: an inactive proxy writes an empty slot (no nodes, stiffness 0).
//   spheres: proxy inside a rigid sphere -> zero-rest-length spring to its
//            projection on the sphere surface (Section 2.3)
//   pairs  : side-A proxy within `gap` of its nearest side-B proxy -> two-sided
//            spring on x_a - x_b toward separation `gap` along their current
//            direction (self-collision)
#include "kernels.h"

namespace pdk {
namespace {

constexpr int NS = CSLOTS;

__device__ __forceinline__ void empty_slot(int64_t j, int32_t* cidx, double* cw, double* ct, double* cs) {
  for (int a = 0; a < NS; ++a) { cidx[NS * j + a] = -1; cw[NS * j + a] = 0.0; }
  ct[3 * j] = ct[3 * j + 1] = ct[3 * j + 2] = 0.0;
  cs[j] = 0.0;
}

__global__ void k_detect_spheres(int64_t np, const int32_t* __restrict__ prox_r, const int32_t* __restrict__ region,
                                 const double* __restrict__ x, int ns_sph, const double* __restrict__ sph,
                                 double stiffness, int32_t* cidx, double* cw, double* ct, double* cs) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= np) return;
  const int r = prox_r[j];
  const double* p = x + 3 * (int64_t)region[r];
  int best = -1;
  double depth = 0.0;
  for (int q = 0; q < ns_sph; ++q) {
    const double dx = p[0] - sph[4 * q], dy = p[1] - sph[4 * q + 1], dz = p[2] - sph[4 * q + 2];
    const double d = sqrt(dx * dx + dy * dy + dz * dz), rad = sph[4 * q + 3];
    if (d < rad && d > 1e-12 && rad - d > depth) { depth = rad - d; best = q; }
  }
  empty_slot(j, cidx, cw, ct, cs);
  if (best < 0) return;
  const double* c = sph + 4 * best;
  const double dx = p[0] - c[0], dy = p[1] - c[1], dz = p[2] - c[2];
  const double d = sqrt(dx * dx + dy * dy + dz * dz), s = c[3] / d;
  cidx[NS * j] = r;
  cw[NS * j] = 1.0;
  ct[3 * j] = c[0] + s * dx; ct[3 * j + 1] = c[1] + s * dy; ct[3 * j + 2] = c[2] + s * dz;
  cs[j] = stiffness;
}

__global__ void k_detect_pairs(int64_t na, const int32_t* __restrict__ ra_list, int64_t nb,
                               const int32_t* __restrict__ rb_list, const int32_t* __restrict__ region,
                               const double* __restrict__ x, double gap, double stiffness, int32_t* cidx, double* cw,
                               double* ct, double* cs) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= na) return;
  const int ra = ra_list[j];
  const double* pa = x + 3 * (int64_t)region[ra];
  double best = 1e300;
  int bi = -1;
  for (int64_t q = 0; q < nb; ++q) {   // nearest side-B proxy (first index on ties)
    const double* pb = x + 3 * (int64_t)region[rb_list[q]];
    const double dx = pa[0] - pb[0], dy = pa[1] - pb[1], dz = pa[2] - pb[2];
    const double d2 = dx * dx + dy * dy + dz * dz;
    if (d2 < best) { best = d2; bi = (int)q; }
  }
  empty_slot(j, cidx, cw, ct, cs);
  const double dist = sqrt(best);
  if (bi < 0 || !(dist < gap) || !(dist > 1e-12)) return;
  const int rb = rb_list[bi];
  const double* pb = x + 3 * (int64_t)region[rb];
  const double s = gap / dist;
  cidx[NS * j] = ra;
  cw[NS * j] = 1.0;
  cidx[NS * j + 4] = rb;
  cw[NS * j + 4] = -1.0;
  ct[3 * j] = s * (pa[0] - pb[0]); ct[3 * j + 1] = s * (pa[1] - pb[1]); ct[3 * j + 2] = s * (pa[2] - pb[2]);
  cs[j] = stiffness;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void detect_spheres(int64_t np, const int32_t* prox_r, const int32_t* region, const double* x, int nsph,
                    const double* sph, double stiffness, int32_t* cidx, double* cw, double* ct, double* cs,
                    cudaStream_t st) {
  if (np <= 0) return;
  k_detect_spheres<<<nblk(np, 128), 128, 0, st>>>(np, prox_r, region, x, nsph, sph, stiffness, cidx, cw, ct, cs);
  ++g_launches;
}

void detect_pairs(int64_t na, const int32_t* ra, int64_t nb, const int32_t* rb, const int32_t* region,
                  const double* x, double gap, double stiffness, int32_t* cidx, double* cw, double* ct, double* cs,
                  cudaStream_t st) {
  if (na <= 0) return;
  k_detect_pairs<<<nblk(na, 128), 128, 0, st>>>(na, ra, nb, rb, region, x, gap, stiffness, cidx, cw, ct, cs);
  ++g_launches;
}

}  // namespace pdk
