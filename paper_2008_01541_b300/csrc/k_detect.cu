// Collision detection on the device (Algorithm 1, step 4.1 DetectCollisions),
// run at every inner iteration instead of a host callback.  Every proxy owns
// one fixed spring slot, so the spring count never has to travel back to the
// host: an inactive proxy writes an empty slot (no nodes, stiffness 0).
//   spheres : proxy inside a rigid sphere -> zero-rest-length spring to its
//             projection on the sphere surface (Section 2.3)
//   pairs   : side-A proxy within `gap` of its nearest side-B proxy -> two-sided
//             spring on x_a - x_b toward separation `gap` along their current
//             direction (self-collision)
//   triangles: proxy node of one side against the surface triangles of the
//             other side (pairs already within rest_min of each other in the
//             rest pose are skipped); the nearest triangle, if nearer than
//             `gap`, gives a two-sided spring on x_a - q (q its closest point,
//             a barycentric combination of the triangle's nodes, Eq. 5) toward
//             gap * u, u the unit vector from q to the node turned to the
//             triangle's front side (its winding's normal n; n itself if the
//             node lies on the triangle)
// Every quantity that decides which obstacle is nearest or whether a proxy is
// active is computed with explicitly rounded operations (no fused
// multiply-add) in a fixed order, so the decision is reproducible operation
// for operation by any IEEE double implementation that follows that order.
#include "kernels.h"

namespace pdk {
namespace {

constexpr int NS = CSLOTS;

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 ld3(const double* p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return {__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)}; }
// (u.x v.x + u.y v.y) + u.z v.z, each operation rounded
__device__ __forceinline__ double dot(V3 u, V3 v) {
  return __dadd_rn(__dadd_rn(__dmul_rn(u.x, v.x), __dmul_rn(u.y, v.y)), __dmul_rn(u.z, v.z));
}

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
  const V3 p = ld3(x + 3 * (int64_t)region[r]);
  int best = -1;
  double depth = 0.0;
  for (int q = 0; q < ns_sph; ++q) {
    const V3 d3 = sub(p, ld3(sph + 4 * q));
    const double d = sqrt(dot(d3, d3)), rad = sph[4 * q + 3];
    if (d < rad && d > 1e-12 && __dsub_rn(rad, d) > depth) { depth = __dsub_rn(rad, d); best = q; }
  }
  empty_slot(j, cidx, cw, ct, cs);
  if (best < 0) return;
  const double* c = sph + 4 * best;
  const V3 d3 = sub(p, ld3(c));
  const double s = __ddiv_rn(c[3], sqrt(dot(d3, d3)));
  cidx[NS * j] = r;
  cw[NS * j] = 1.0;
  ct[3 * j] = __dadd_rn(c[0], __dmul_rn(s, d3.x));
  ct[3 * j + 1] = __dadd_rn(c[1], __dmul_rn(s, d3.y));
  ct[3 * j + 2] = __dadd_rn(c[2], __dmul_rn(s, d3.z));
  cs[j] = stiffness;
}

__global__ void k_detect_pairs(int64_t na, const int32_t* __restrict__ ra_list, int64_t nb,
                               const int32_t* __restrict__ rb_list, const int32_t* __restrict__ region,
                               const double* __restrict__ x, double gap, double stiffness, int32_t* cidx, double* cw,
                               double* ct, double* cs) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= na) return;
  const int ra = ra_list[j];
  const V3 pa = ld3(x + 3 * (int64_t)region[ra]);
  double best = 1e300;
  int bi = -1;
  for (int64_t q = 0; q < nb; ++q) {   // nearest side-B proxy (first index on ties)
    const V3 d3 = sub(pa, ld3(x + 3 * (int64_t)region[rb_list[q]]));
    const double d2 = dot(d3, d3);
    if (d2 < best) { best = d2; bi = (int)q; }
  }
  empty_slot(j, cidx, cw, ct, cs);
  const double dist = sqrt(best);
  if (bi < 0 || !(dist < gap) || !(dist > 1e-12)) return;
  const int rb = rb_list[bi];
  const V3 d3 = sub(pa, ld3(x + 3 * (int64_t)region[rb]));
  const double s = __ddiv_rn(gap, dist);
  cidx[NS * j] = ra;
  cw[NS * j] = 1.0;
  cidx[NS * j + 4] = rb;
  cw[NS * j + 4] = -1.0;
  ct[3 * j] = __dmul_rn(s, d3.x); ct[3 * j + 1] = __dmul_rn(s, d3.y); ct[3 * j + 2] = __dmul_rn(s, d3.z);
  cs[j] = stiffness;
}

// Closest point q of the triangle (a, b, c) to p: returns |p - q|^2, the
// barycentric weights of q, and q.  The projection on the triangle's plane if its
// barycentric coordinates lie in [0, 1]; otherwise the nearest of the three
// segment projections (edges ab, bc, ca; the first on ties).  A zero-area
// triangle goes through its edges.
__device__ double closest_on_triangle(V3 p, V3 a, V3 b, V3 c, double* w, V3* qout) {
  const V3 e0 = sub(b, a), e1 = sub(c, a), pw = sub(p, a);
  const double d00 = dot(e0, e0), d01 = dot(e0, e1), d11 = dot(e1, e1), d20 = dot(pw, e0), d21 = dot(pw, e1);
  const double den = __dsub_rn(__dmul_rn(d00, d11), __dmul_rn(d01, d01));
  if (den > 0.0) {
    const double s = __ddiv_rn(__dsub_rn(__dmul_rn(d11, d20), __dmul_rn(d01, d21)), den);
    const double t = __ddiv_rn(__dsub_rn(__dmul_rn(d00, d21), __dmul_rn(d01, d20)), den);
    if (s >= 0.0 && t >= 0.0 && __dadd_rn(s, t) <= 1.0) {
      const V3 q = {__dadd_rn(__dadd_rn(a.x, __dmul_rn(s, e0.x)), __dmul_rn(t, e1.x)),
                    __dadd_rn(__dadd_rn(a.y, __dmul_rn(s, e0.y)), __dmul_rn(t, e1.y)),
                    __dadd_rn(__dadd_rn(a.z, __dmul_rn(s, e0.z)), __dmul_rn(t, e1.z))};
      const V3 r = sub(p, q);
      w[0] = __dsub_rn(__dsub_rn(1.0, s), t);
      w[1] = s;
      w[2] = t;
      *qout = q;
      return dot(r, r);
    }
  }
  double best = 0.0;
  const V3 us[3] = {a, b, c};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const V3 u = us[k], v = us[(k + 1) % 3];
    const V3 e = sub(v, u);
    const double ee = dot(e, e);
    double f = ee > 0.0 ? __ddiv_rn(dot(sub(p, u), e), ee) : 0.0;
    f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
    const V3 q = {__dadd_rn(u.x, __dmul_rn(f, e.x)), __dadd_rn(u.y, __dmul_rn(f, e.y)),
                  __dadd_rn(u.z, __dmul_rn(f, e.z))};
    const V3 r = sub(p, q);
    const double d2 = dot(r, r);
    if (k == 0 || d2 < best) {
      best = d2;
      w[0] = w[1] = w[2] = 0.0;
      w[k] = __dsub_rn(1.0, f);
      w[(k + 1) % 3] = f;
      *qout = q;
    }
  }
  return best;
}

// FP32 distance from p to the triangle (a, b, c), for classifying a pair
// before the exact FP64 test; negative if the triangle is too close to
// degenerate for FP32 to be trusted (its smallest angle below ~2 degrees).
__device__ __forceinline__ float dist_f32(float3 p, float3 a, float3 b, float3 c) {
  const float3 e0 = make_float3(b.x - a.x, b.y - a.y, b.z - a.z), e1 = make_float3(c.x - a.x, c.y - a.y, c.z - a.z);
  const float3 w = make_float3(p.x - a.x, p.y - a.y, p.z - a.z);
  const float d00 = e0.x * e0.x + e0.y * e0.y + e0.z * e0.z, d11 = e1.x * e1.x + e1.y * e1.y + e1.z * e1.z;
  const float d01 = e0.x * e1.x + e0.y * e1.y + e0.z * e1.z;
  const float den = d00 * d11 - d01 * d01;
  if (!(den > 1e-3f * d00 * d11)) return -1.f;
  const float d20 = w.x * e0.x + w.y * e0.y + w.z * e0.z, d21 = w.x * e1.x + w.y * e1.y + w.z * e1.z;
  float s = (d11 * d20 - d01 * d21) / den, t = (d00 * d21 - d01 * d20) / den;
  float best;
  if (s >= 0.f && t >= 0.f && s + t <= 1.f) {
    const float qx = a.x + s * e0.x + t * e1.x, qy = a.y + s * e0.y + t * e1.y, qz = a.z + s * e0.z + t * e1.z;
    best = (p.x - qx) * (p.x - qx) + (p.y - qy) * (p.y - qy) + (p.z - qz) * (p.z - qz);
  } else {
    best = 3.4e38f;
    const float3 us[3] = {a, b, c};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float3 u = us[k], v = us[(k + 1) % 3];
      const float ex = v.x - u.x, ey = v.y - u.y, ez = v.z - u.z;
      const float ee = ex * ex + ey * ey + ez * ez;
      float f = ((p.x - u.x) * ex + (p.y - u.y) * ey + (p.z - u.z) * ez) / ee;
      f = fminf(fmaxf(f, 0.f), 1.f);
      const float rx = p.x - (u.x + f * ex), ry = p.y - (u.y + f * ey), rz = p.z - (u.z + f * ez);
      best = fminf(best, rx * rx + ry * ry + rz * rz);
    }
  }
  return sqrtf(best);
}

// Bounding sphere of each triangle at the current positions, in FP32 and
// enlarged so that it is never smaller than the exact one.
__global__ void k_tri_bounds(int64_t nt, const int32_t* __restrict__ tri, const int32_t* __restrict__ region,
                             const double* __restrict__ x, float4* __restrict__ bnd) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const V3 a = ld3(x + 3 * (int64_t)region[tri[3 * t]]), b = ld3(x + 3 * (int64_t)region[tri[3 * t + 1]]),
           c = ld3(x + 3 * (int64_t)region[tri[3 * t + 2]]);
  const double cx = (a.x + b.x + c.x) / 3.0, cy = (a.y + b.y + c.y) / 3.0, cz = (a.z + b.z + c.z) / 3.0;
  double r2 = 0.0;
  for (const V3& v : {a, b, c}) {
    const double dx = v.x - cx, dy = v.y - cy, dz = v.z - cz;
    r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
  }
  bnd[t] = make_float4((float)cx, (float)cy, (float)cz, (float)(sqrt(r2) * (1.0 + 1e-5) + 1e-6));
}

// One warp per proxy: lanes scan the triangles q = lane, lane + 32, ... with a
// conservative FP32 bounding-sphere test, then classify the survivors with
// FP32 closest points (rest-pose exclusion, then farther than gap) whenever
// a wide margin settles the question, and take the exact FP64 closest point
// for the rest; the warp keeps the smallest exact distance, the lowest
// triangle index on ties.  A triangle skipped by the FP32 tests is either
// excluded or farther than gap, so it can never be the active choice: the
// result is the same as a scan of every triangle in index order with the
// exact test.  Slot j of the spring arrays.
// One warp per proxy of either side (side-A proxies against side-B triangles,
// then side-B proxies against side-A triangles; slot j = proxy j).  Pass 1:
// each lane screens its triangles in FP32 (bounding sphere, then the rest and
// current distances with the margins of dist_f32) and the survivors go to a
// per-warp list; pass 2: the lanes take the listed candidates side by side
// for the exact FP64 tests, so a proxy with several candidates pays for the
// FP64 work about once instead of once per candidate.
constexpr int kCand = 64;
__global__ void __launch_bounds__(128) k_detect_tris(
    int64_t na, int64_t nb, const int32_t* __restrict__ prox, int64_t nta, int64_t ntb,
    const int32_t* __restrict__ tris, const float4* __restrict__ bnd_all, const int32_t* __restrict__ region,
    const double* __restrict__ x, const double* __restrict__ xr, double gap, double rest_min, double stiffness,
    int32_t* cidx, double* cw, double* ct, double* cs) {
  __shared__ int cand[4][kCand];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + wib;
  if (j >= na + nb) return;
  const bool side_a = j < na;
  const int64_t nt = side_a ? ntb : nta;
  const int32_t* tri = side_a ? tris + 3 * nta : tris;
  const float4* bnd = side_a ? bnd_all + nta : bnd_all;
  const int r0 = prox[j];
  const V3 p = ld3(x + 3 * (int64_t)region[r0]), P = ld3(xr + 3 * (int64_t)r0);
  const float px = (float)p.x, py = (float)p.y, pz = (float)p.z, fg = (float)gap;
  const double rm2 = __dmul_rn(rest_min, rest_min);
  double best = 1e300;
  int64_t bi = -1;
  const float3 p32 = make_float3(px, py, pz), P32 = make_float3((float)P.x, (float)P.y, (float)P.z);
  const float frm = (float)rest_min;
  int* cl = cand[wib];
  int ncand = 0;
  auto exact = [&]() {   // pass 2 on the listed candidates (ascending triangle index)
    for (int c = lane; c < ncand; c += 32) {
      const int e = cl[c];
      const int64_t q = e & 0x3fffffff;
      const int i0 = tri[3 * q], i1 = tri[3 * q + 1], i2 = tri[3 * q + 2];
      double w[3];
      V3 qp;
      if (e & 0x40000000) {   // near the rest exclusion distance: the exact rest test decides
        const V3 R0 = ld3(xr + 3 * (int64_t)i0), R1 = ld3(xr + 3 * (int64_t)i1), R2 = ld3(xr + 3 * (int64_t)i2);
        if (closest_on_triangle(P, R0, R1, R2, w, &qp) < rm2) continue;
      }
      const V3 C0 = ld3(x + 3 * (int64_t)region[i0]), C1 = ld3(x + 3 * (int64_t)region[i1]),
               C2 = ld3(x + 3 * (int64_t)region[i2]);
      const double d2 = closest_on_triangle(p, C0, C1, C2, w, &qp);
      if (d2 < best || (d2 == best && q < bi)) { best = d2; bi = q; }
    }
    ncand = 0;
    __syncwarp();
  };
  for (int64_t q0 = 0; q0 < nt; q0 += 32) {
    const int64_t q = q0 + lane;
    bool keep = false, undecided = false;
    if (q < nt) {
      const float4 b = __ldg(bnd + q);
      const float dx = px - b.x, dy = py - b.y, dz = pz - b.z;
      const float margin = 1e-4f * (fabsf(b.x) + fabsf(b.y) + fabsf(b.z) + b.w + fg) + 1e-6f;
      if (sqrtf(dx * dx + dy * dy + dz * dz) <= b.w + fg + margin) {
        const int i0 = tri[3 * q], i1 = tri[3 * q + 1], i2 = tri[3 * q + 2];
        const V3 R0 = ld3(xr + 3 * (int64_t)i0), R1 = ld3(xr + 3 * (int64_t)i1), R2 = ld3(xr + 3 * (int64_t)i2);
        const V3 C0 = ld3(x + 3 * (int64_t)region[i0]), C1 = ld3(x + 3 * (int64_t)region[i1]),
                 C2 = ld3(x + 3 * (int64_t)region[i2]);
        // FP32 classification with a margin (1% + 1e-3) far beyond its
        // rounding; only the pairs it cannot settle take the exact FP64 test
        const float dr32 = dist_f32(P32, make_float3((float)R0.x, (float)R0.y, (float)R0.z),
                                    make_float3((float)R1.x, (float)R1.y, (float)R1.z),
                                    make_float3((float)R2.x, (float)R2.y, (float)R2.z));
        const float d32 = dist_f32(p32, make_float3((float)C0.x, (float)C0.y, (float)C0.z),
                                   make_float3((float)C1.x, (float)C1.y, (float)C1.z),
                                   make_float3((float)C2.x, (float)C2.y, (float)C2.z));
        const bool excluded = dr32 >= 0.f && dr32 < 0.99f * frm - 1e-3f;   // near at rest
        const bool far = d32 >= 0.f && d32 > 1.01f * fg + 1e-3f;           // farther than gap: never the choice
        keep = !excluded && !far;
        undecided = !(dr32 >= 0.f && dr32 > 1.01f * frm + 1e-3f);
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (bal) {
      const int cnt = __popc(bal);
      if (ncand + cnt > kCand) exact();
      if (keep) cl[ncand + __popc(bal & ((1u << lane) - 1u))] = (int)q | (undecided ? 0x40000000 : 0);
      ncand += cnt;
      __syncwarp();
    }
  }
  exact();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, o);
    const long long oi = __shfl_down_sync(0xffffffffu, (long long)bi, o);
    if (oi >= 0 && (bi < 0 || ob < best || (ob == best && oi < bi))) { best = ob; bi = oi; }
  }
  if (lane != 0) return;
  const int64_t sj = j;
  empty_slot(sj, cidx, cw, ct, cs);
  if (bi < 0 || !(sqrt(best) < gap)) return;
  const int i0 = tri[3 * bi], i1 = tri[3 * bi + 1], i2 = tri[3 * bi + 2];
  const V3 A = ld3(x + 3 * (int64_t)region[i0]), B = ld3(x + 3 * (int64_t)region[i1]),
           C = ld3(x + 3 * (int64_t)region[i2]);
  double bw[3];
  V3 q;
  closest_on_triangle(p, A, B, C, bw, &q);   // the same operations as in the scan: the same q and weights
  const V3 e0 = sub(B, A), e1 = sub(C, A);
  const V3 n = {__dsub_rn(__dmul_rn(e0.y, e1.z), __dmul_rn(e0.z, e1.y)),
                __dsub_rn(__dmul_rn(e0.z, e1.x), __dmul_rn(e0.x, e1.z)),
                __dsub_rn(__dmul_rn(e0.x, e1.y), __dmul_rn(e0.y, e1.x))};
  const V3 r = sub(p, q);
  V3 tg;
  if (best > 0.0) {   // along q -> node, on the front side
    double s = __ddiv_rn(gap, sqrt(best));
    if (dot(r, n) < 0.0) s = -s;
    tg = {__dmul_rn(s, r.x), __dmul_rn(s, r.y), __dmul_rn(s, r.z)};
  } else {            // on the triangle: along its normal
    const double nn = sqrt(dot(n, n));
    if (!(nn > 0.0)) return;
    const double s = __ddiv_rn(gap, nn);
    tg = {__dmul_rn(s, n.x), __dmul_rn(s, n.y), __dmul_rn(s, n.z)};
  }
  cidx[NS * sj] = r0;
  cw[NS * sj] = 1.0;
  cidx[NS * sj + 4] = i0; cidx[NS * sj + 5] = i1; cidx[NS * sj + 6] = i2;
  cw[NS * sj + 4] = -bw[0]; cw[NS * sj + 5] = -bw[1]; cw[NS * sj + 6] = -bw[2];
  ct[3 * sj] = tg.x; ct[3 * sj + 1] = tg.y; ct[3 * sj + 2] = tg.z;
  cs[sj] = stiffness;
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

void detect_tris(const TriDetector& d, const int32_t* region, const double* x, int32_t* cidx, double* cw, double* ct,
                 double* cs, cudaStream_t st) {
  const int64_t nt = d.nta + d.ntb;
  if (nt > 0) {
    k_tri_bounds<<<nblk(nt, 128), 128, 0, st>>>(nt, d.tris, region, x, d.bnd);
    ++g_launches;
  }
  // side-A proxies against side-B triangles and side-B proxies against side-A
  // triangles, one launch
  if (d.na + d.nb > 0) {
    k_detect_tris<<<nblk(d.na + d.nb, 4), 128, 0, st>>>(d.na, d.nb, d.prox, d.nta, d.ntb, d.tris, d.bnd, region, x,
                                                         d.xr, d.gap, d.rest_min, d.stiffness, cidx, cw, ct, cs);
    ++g_launches;
  }
}

}  // namespace pdk
