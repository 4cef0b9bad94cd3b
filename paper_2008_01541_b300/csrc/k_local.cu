// Local step kernels: batched FP64 polar decomposition of the deformation
// gradients and the elemental forces (Section 2.2), plus the deterministic
// per-node gather and small vector kernels.
#include "kernels.h"

namespace pdk {

int64_t g_launches = 0;

namespace {

// X^-T = cof(X) / det(X); row-major 3x3.
__device__ __forceinline__ double cofactor(const double* X, double* C) {
  C[0] = X[4] * X[8] - X[5] * X[7];
  C[1] = X[5] * X[6] - X[3] * X[8];
  C[2] = X[3] * X[7] - X[4] * X[6];
  C[3] = X[2] * X[7] - X[1] * X[8];
  C[4] = X[0] * X[8] - X[2] * X[6];
  C[5] = X[1] * X[6] - X[0] * X[7];
  C[6] = X[1] * X[5] - X[2] * X[4];
  C[7] = X[2] * X[3] - X[0] * X[5];
  C[8] = X[0] * X[4] - X[1] * X[3];
  return X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
}

// Scaled Newton iteration for the orthogonal polar factor (Higham):
// X <- (g X + X^-T / g) / 2, Frobenius scaling g = sqrt(||X^-1|| / ||X||)
// until the update is small, then unscaled.  Valid for det F > 0, where the
// polar factor is the closest rotation.  Returns false if it cannot be used.
__device__ bool polar_newton(const double* F, double* R) {
  double X[9], C[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) X[i] = F[i];
  double nx = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) nx += X[i] * X[i];
  bool scaled = true;
  for (int it = 0; it < 40; ++it) {
    double det = cofactor(X, C);
    if (!(det > 1e-12 * nx * sqrt(nx))) return false;
    double g = 1.0;
    if (scaled) {
      double nc = 0.0;
#pragma unroll
      for (int i = 0; i < 9; ++i) nc += C[i] * C[i];
      g = sqrt(sqrt(nc / nx) / det);
    }
    double a = 0.5 * g, b = 0.5 / (g * det), d2 = 0.0, nn = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      double v = a * X[i] + b * C[i];
      double dv = v - X[i];
      d2 += dv * dv;
      nn += v * v;
      X[i] = v;
    }
    nx = nn;
    if (d2 < 1e-4) scaled = false;
    if (d2 < 1e-20) {
#pragma unroll
      for (int i = 0; i < 9; ++i) R[i] = X[i];
      return true;
    }
  }
  return false;
}

// The same scaled Newton iteration in FP32 (64 times the FP64 rate on B300),
// to FP32 accuracy; false if it cannot be used (det <= 0, no convergence).
__device__ bool polar_newton_f32(const double* F, float* X) {
  float C[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) X[i] = (float)F[i];
  float nx = 0.f;
#pragma unroll
  for (int i = 0; i < 9; ++i) nx += X[i] * X[i];
  bool scaled = true;
  for (int it = 0; it < 30; ++it) {
    C[0] = X[4] * X[8] - X[5] * X[7];
    C[1] = X[5] * X[6] - X[3] * X[8];
    C[2] = X[3] * X[7] - X[4] * X[6];
    C[3] = X[2] * X[7] - X[1] * X[8];
    C[4] = X[0] * X[8] - X[2] * X[6];
    C[5] = X[1] * X[6] - X[0] * X[7];
    C[6] = X[1] * X[5] - X[2] * X[4];
    C[7] = X[2] * X[3] - X[0] * X[5];
    C[8] = X[0] * X[4] - X[1] * X[3];
    const float det = X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
    if (!(det > 1e-6f * nx * sqrtf(nx))) return false;
    float g = 1.f;
    if (scaled) {
      float nc = 0.f;
#pragma unroll
      for (int i = 0; i < 9; ++i) nc += C[i] * C[i];
      g = sqrtf(sqrtf(nc / nx) / det);
    }
    const float a = 0.5f * g, b = 0.5f / (g * det);
    float d2 = 0.f, nn = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float v = a * X[i] + b * C[i];
      const float dv = v - X[i];
      d2 += dv * dv;
      nn += v * v;
      X[i] = v;
    }
    nx = nn;
    if (d2 < 1e-4f) scaled = false;
    if (d2 < 1e-12f) return true;
  }
  return false;
}

// Closest rotation of F (det F > 0) to FP64 accuracy from an FP32 estimate
// R0 of it.  One FP64 Newton step (X + X^-T) / 2 first makes the estimate
// orthogonal (it leaves its rotation unchanged and squares the rest); then,
// with M = X^T F = H + K (H symmetric, K small and skew), the rotation
// X exp([w]x) with w = 2 (tr(H) I - H)^-1 axial(K) makes its transpose
// times F symmetric to first order.  The error left after a pass is of the
// order of the square of its correction, so a pass whose correction is below
// ~3e-7 is the last (an FP32 estimate of a well-conditioned F needs one); at
// most three passes, else false.
__device__ bool polar_refine(const double* F, const float* X32, double* R) {
  double X[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) X[i] = (double)X32[i];
  for (int pass = 0; pass < 3; ++pass) {
    {   // orthogonalise: X = (X + X^-T) / 2
      double Cx[9];
      const double dx = cofactor(X, Cx);
      if (!(dx > 0.0)) return false;
      const double b = 0.5 / dx;
#pragma unroll
      for (int i = 0; i < 9; ++i) X[i] = 0.5 * X[i] + b * Cx[i];
    }
    double M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) M[3 * i + j] = X[i] * F[j] + X[3 + i] * F[3 + j] + X[6 + i] * F[6 + j];   // (X^T F)_ij
    // axial vector of the skew part, and A = tr(H) I - H for the symmetric part H
    const double s0 = 0.5 * (M[7] - M[5]), s1 = 0.5 * (M[2] - M[6]), s2 = 0.5 * (M[3] - M[1]);
    const double h01 = 0.5 * (M[1] + M[3]), h02 = 0.5 * (M[2] + M[6]), h12 = 0.5 * (M[5] + M[7]);
    const double tr = M[0] + M[4] + M[8];
    const double a00 = tr - M[0], a11 = tr - M[4], a22 = tr - M[8];
    // w = 2 A^-1 s from the symmetric adjugate of A (off-diagonal a_ij = -h_ij)
    const double c00 = a11 * a22 - h12 * h12, c11 = a00 * a22 - h02 * h02, c22 = a00 * a11 - h01 * h01;
    const double c01 = a22 * h01 + h02 * h12, c02 = a11 * h02 + h01 * h12, c12 = a00 * h12 + h01 * h02;
    const double det = a00 * c00 - h01 * c01 - h02 * c02;
    if (!(det > 0.0)) return false;
    const double rd = 2.0 / det;
    const double w0 = rd * (c00 * s0 + c01 * s1 + c02 * s2);
    const double w1 = rd * (c01 * s0 + c11 * s1 + c12 * s2);
    const double w2 = rd * (c02 * s0 + c12 * s1 + c22 * s2);
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    // X <- X Q with Q = exp([w]x): to first order, X + X [w]x, when the
    // correction is small enough that Q's departure from orthogonality,
    // ~th2, is below 1e-12; else Rodrigues' formula
    if (th2 < 1e-12) {
      double Y[9];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double x0 = X[3 * i], x1 = X[3 * i + 1], x2 = X[3 * i + 2];
        Y[3 * i] = x0 + (x1 * w2 - x2 * w1);
        Y[3 * i + 1] = x1 + (x2 * w0 - x0 * w2);
        Y[3 * i + 2] = x2 + (x0 * w1 - x1 * w0);
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) X[i] = Y[i];
    } else {
      const double th = sqrt(th2);
      const double c1 = sin(th) / th, c2 = (1.0 - cos(th)) / th2;   // sin(th) / th, (1 - cos(th)) / th^2
      const double K[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
      double Q[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const double kk = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
          Q[3 * i + j] = (i == j ? 1.0 : 0.0) + c1 * K[3 * i + j] + c2 * kk;
        }
      double Y[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Y[3 * i + j] = X[3 * i] * Q[j] + X[3 * i + 1] * Q[3 + j] + X[3 * i + 2] * Q[6 + j];
#pragma unroll
      for (int i = 0; i < 9; ++i) X[i] = Y[i];
    }
    if (th2 < 1e-13) {   // the next correction would be ~th2: below 1e-12 relative, X is R
#pragma unroll
      for (int i = 0; i < 9; ++i) R[i] = X[i];
      return true;
    }
  }
  return false;
}

// Closest rotation through the eigen-decomposition of F^T F (cyclic Jacobi):
// R = [u1 u2 u1 x u2] [v1 v2 v1 x v2]^T with u_i = F v_i / sigma_i.  Used for
// inverted, degenerate or badly conditioned F, where the smallest singular
// direction is the one that gets flipped.
// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix in place:
// on return S is diagonal (the eigenvalues) and S_in = V S_out V^T.
__device__ void jacobi_eig3(double S[3][3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = S[0][1] * S[0][1] + S[0][2] * S[0][2] + S[1][2] * S[1][2];
    double dia = S[0][0] * S[0][0] + S[1][1] * S[1][1] + S[2][2] * S[2][2];
    if (off <= 1e-34 * dia || off == 0.0) break;
    for (int pq = 0; pq < 3; ++pq) {
      int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      double apq = S[p][q];
      if (apq == 0.0) continue;
      double theta = (S[q][q] - S[p][p]) / (2.0 * apq);
      double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      for (int k = 0; k < 3; ++k) {  // S <- J^T S J, J = rotation in (p,q)
        double skp = S[k][p], skq = S[k][q];
        S[k][p] = c * skp - s * skq;
        S[k][q] = s * skp + c * skq;
      }
      for (int k = 0; k < 3; ++k) {
        double spk = S[p][k], sqk = S[q][k];
        S[p][k] = c * spk - s * sqk;
        S[q][k] = s * spk + c * sqk;
      }
      for (int k = 0; k < 3; ++k) {
        double vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
}

__device__ void polar_jacobi(const double* F, double* R) {
  double S[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      S[i][j] = F[0 * 3 + i] * F[0 * 3 + j] + F[1 * 3 + i] * F[1 * 3 + j] + F[2 * 3 + i] * F[2 * 3 + j];
  jacobi_eig3(S, V);
  // sort eigenvalues descending
  int o[3] = {0, 1, 2};
  double lam[3] = {S[0][0], S[1][1], S[2][2]};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2 - i; ++j)
      if (lam[o[j]] < lam[o[j + 1]]) { int t = o[j]; o[j] = o[j + 1]; o[j + 1] = t; }
  double v1[3] = {V[0][o[0]], V[1][o[0]], V[2][o[0]]};
  double v2[3] = {V[0][o[1]], V[1][o[1]], V[2][o[1]]};
  double u1[3], u2[3];
  for (int i = 0; i < 3; ++i) {
    u1[i] = F[3 * i] * v1[0] + F[3 * i + 1] * v1[1] + F[3 * i + 2] * v1[2];
    u2[i] = F[3 * i] * v2[0] + F[3 * i + 1] * v2[1] + F[3 * i + 2] * v2[2];
  }
  double n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
  if (!(n1 > 1e-300)) {
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
    return;
  }
  for (int i = 0; i < 3; ++i) u1[i] /= n1;
  double d = u1[0] * u2[0] + u1[1] * u2[1] + u1[2] * u2[2];
  for (int i = 0; i < 3; ++i) u2[i] -= d * u1[i];
  double n2 = sqrt(u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
  if (!(n2 > 1e-14 * n1)) {  // rank one: any unit vector orthogonal to u1
    double e[3] = {0, 0, 0};
    int k = fabs(u1[0]) < fabs(u1[1]) ? (fabs(u1[0]) < fabs(u1[2]) ? 0 : 2) : (fabs(u1[1]) < fabs(u1[2]) ? 1 : 2);
    e[k] = 1.0;
    double dd = u1[k];
    for (int i = 0; i < 3; ++i) u2[i] = e[i] - dd * u1[i];
    n2 = sqrt(u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
  }
  for (int i = 0; i < 3; ++i) u2[i] /= n2;
  double u3[3] = {u1[1] * u2[2] - u1[2] * u2[1], u1[2] * u2[0] - u1[0] * u2[2], u1[0] * u2[1] - u1[1] * u2[0]};
  double v3[3] = {v1[1] * v2[2] - v1[2] * v2[1], v1[2] * v2[0] - v1[0] * v2[2], v1[0] * v2[1] - v1[1] * v2[0]};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[3 * i + j] = u1[i] * v1[j] + u2[i] * v2[j] + u3[i] * v3[j];
}

// Principal branch of the volume projection: tau(c) = (s + sqrt(s^2 - 4c)) / 2
// solves (tau - s) tau = -c; for s < 0 the same root as 2c / (s - sqrt(...)),
// which has no cancellation.
__device__ __forceinline__ double vol_tau(double s, double c, double* r_out) {
  const double r = sqrt(fmax(s * s - 4.0 * c, 0.0));
  *r_out = r;
  if (s >= 0.0) return 0.5 * (s + r);
  const double d = s - r;
  return d != 0.0 ? 2.0 * c / d : 0.0;
}

// PD volume term (the lambda term of Eq. 1 in PD form): the signed singular
// values s (eigenvalues of S, any order) are moved to tau, the diagonal
// nearest s whose product is vt, on the principal branch tau_i(c).
// g(c) = log prod tau_i(c) - log vt is decreasing in c; its root is found by
// Newton steps safeguarded by bisection of a bracket [a, b] with
// g(a) >= 0 >= g(b) (a step is taken only if it stays inside the bracket and
// at least halves the step before last; near the branch end the slope grows
// without bound and bisection takes over).  If even the branch end keeps
// the product above vt (an element stretched about twofold in every
// direction), tau is the branch end.
__device__ void volume_tau(const double s[3], double vt, double tau[3]) {
  double r[3];
  const double v = s[0] * s[1] * s[2];
  const double lvt = log(vt);
  const double s2min = fmin(s[0] * s[0], fmin(s[1] * s[1], s[2] * s[2]));
  double a, b;
  if (v < vt) {
    b = 0.0;
    a = -fmax(1.0, fmax(s[0] * s[0], fmax(s[1] * s[1], s[2] * s[2])));
    for (int k = 0; k < 64; ++k) {
      if (vol_tau(s[0], a, r) * vol_tau(s[1], a, r + 1) * vol_tau(s[2], a, r + 2) >= vt) break;
      a *= 4.0;
    }
  } else {
    a = 0.0;
    b = 0.25 * s2min;
    if (vol_tau(s[0], b, r) * vol_tau(s[1], b, r + 1) * vol_tau(s[2], b, r + 2) > vt) {
      for (int i = 0; i < 3; ++i) tau[i] = vol_tau(s[i], b, r + i);
      return;
    }
  }
  double c = b, dx = b - a, dxold = dx;
  for (int it = 0; it < 200; ++it) {
    double p = 1.0, dg = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double t = vol_tau(s[i], c, r + i);
      p *= t;
      dg -= 1.0 / (r[i] * t);   // d log tau_i / dc = -1 / (r_i tau_i)
    }
    const double g = p > 0.0 ? log(p) - lvt : -INFINITY;
    if (g == 0.0) break;
    if (g > 0.0) a = c;
    else b = c;
    const double cn = c - g / dg;
    const bool newton = isfinite(cn) && cn > a && cn < b && fabs(2.0 * g) <= fabs(dxold * dg);
    dxold = dx;
    if (newton) {
      dx = c - cn;
      c = cn;
    } else {
      dx = 0.5 * (b - a);
      c = a + dx;
    }
    // converged: a step at the resolution of c where g is at rounding level
    // (a tiny step alone is not enough: near the branch end the slope is huge)
    if ((fabs(dx) <= 1e-16 * (fabs(c) + s2min) && fabs(g) <= 1e-12) || !(b > a)) break;
  }
  for (int i = 0; i < 3; ++i) tau[i] = vol_tau(s[i], c, r + i);
}

// Residuals of the extra local-step terms from one eigen-decomposition of
// S = R^T F = V diag(lambda) V^T (signed: an inverted F has one negative
// lambda, its singular values are |lambda|):
//  * bi-phasic strain limiting (Section 5): the closest matrix with singular
//    values in [lo, hi] is Q = R V diag(sign(lambda) clamp(|lambda|)) V^T;
//  * PD volume term: T = R V diag(tau) V^T with tau from volume_tau when
//    prod(lambda) = det F lies outside [vlo, vhi] (T = F inside).
// Returns D = frac (F - Q) + vfrac (F - T) = R V diag(frac (lambda - q) +
// vfrac (lambda - tau)) V^T, exactly zero when no bound is violated.
__device__ void extra_residual(const double* F, const double* R, const StrainLimit& sl, double* D) {
  double S[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double a = R[i] * F[j] + R[3 + i] * F[3 + j] + R[6 + i] * F[6 + j];   // (R^T F)_ij
      const double b = R[j] * F[i] + R[3 + j] * F[3 + i] + R[6 + j] * F[6 + i];   // (R^T F)_ji
      S[i][j] = 0.5 * (a + b);
    }
  jacobi_eig3(S, V);
  const double lam[3] = {S[0][0], S[1][1], S[2][2]};
  double dl[3] = {0.0, 0.0, 0.0};
  bool any = false;
  if (sl.frac > 0.0) {
    for (int q = 0; q < 3; ++q) {
      const double l = lam[q], al = fabs(l), c = fmin(fmax(al, sl.lo), sl.hi);
      const double d = l - (l < 0.0 ? -c : c);
      dl[q] += sl.frac * d;
      any |= d != 0.0;
    }
  }
  if (sl.vfrac > 0.0) {
    const double v = lam[0] * lam[1] * lam[2];
    if (v < sl.vlo || v > sl.vhi) {
      double tau[3];
      volume_tau(lam, v < sl.vlo ? sl.vlo : sl.vhi, tau);
      for (int q = 0; q < 3; ++q) dl[q] += sl.vfrac * (lam[q] - tau[q]);
      any = true;
    }
  }
  if (!any) {
    for (int i = 0; i < 9; ++i) D[i] = 0.0;
    return;
  }
  double M[3][3];   // V diag(dl) V^T
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = V[i][0] * dl[0] * V[j][0] + V[i][1] * dl[1] * V[j][1] + V[i][2] * dl[2] * V[j][2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) D[3 * i + j] = R[3 * i] * M[0][j] + R[3 * i + 1] * M[1][j] + R[3 * i + 2] * M[2][j];
}

// Elemental forces f_e = -Vol_e G_e-weighted (2 mu (F - R) + 2 mu' (F - Q) +
// 2 kappa (F - T)); w = 2 (mu + mu' + kappa) Vol, so the stress is
// (1 - frac - vfrac) (F - R) + frac (F - Q) + vfrac (F - T) (EXTRA = false
// compiles the extra terms out).
template <bool EXTRA>
__global__ void k_polar_forces(int64_t count, const int4* __restrict__ tets,
                               const double* __restrict__ Dm, const double* __restrict__ w,
                               const double* __restrict__ x, double* __restrict__ fe,
                               double* __restrict__ Rout, StrainLimit sl) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= count) return;
  int4 t = tets[e];
  double p0[3], D[9];
#pragma unroll
  for (int i = 0; i < 3; ++i) p0[i] = __ldg(x + 3 * (int64_t)t.x + i);
  const int vid[3] = {t.y, t.z, t.w};
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < 3; ++i) D[3 * i + c] = __ldg(x + 3 * (int64_t)vid[c] + i) - p0[i];
  double Mi[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) Mi[i] = __ldg(Dm + i * count + e);
  double F[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F[3 * i + j] = D[3 * i] * Mi[j] + D[3 * i + 1] * Mi[3 + j] + D[3 * i + 2] * Mi[6 + j];
  // R: FP32 Newton iterations refined in FP64; the FP64 Newton iteration
  // where FP32 cannot serve; the Jacobi route for inverted or degenerate F
  double R[9];
  {
    float X32[9];
    if (!(polar_newton_f32(F, X32) && polar_refine(F, X32, R)) && !polar_newton(F, R)) polar_jacobi(F, R);
  }
  double we = __ldg(w + e);
  double P[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) P[i] = F[i] - R[i];
  if (EXTRA) {
    double D[9];
    extra_residual(F, R, sl, D);
    const double keep = 1.0 - sl.frac - sl.vfrac;
#pragma unroll
    for (int i = 0; i < 9; ++i) P[i] = keep * P[i] + D[i];
  }
  double f[4][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double P0 = P[3 * i], P1 = P[3 * i + 1], P2 = P[3 * i + 2];
#pragma unroll
    for (int a = 1; a < 4; ++a)
      f[a][i] = -we * (P0 * Mi[3 * (a - 1)] + P1 * Mi[3 * (a - 1) + 1] + P2 * Mi[3 * (a - 1) + 2]);
    f[0][i] = -(f[1][i] + f[2][i] + f[3][i]);
  }
  double* o = fe + 12 * e;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) o[3 * a + i] = f[a][i];
  if (Rout) {
#pragma unroll
    for (int i = 0; i < 9; ++i) Rout[9 * e + i] = R[i];
  }
}

__global__ void k_gather(int64_t nt, const int64_t* __restrict__ ptr, const int32_t* __restrict__ slot,
                         const double* __restrict__ fe, double* __restrict__ out,
                         const double* __restrict__ add, const double* __restrict__ mass_h2,
                         const double* __restrict__ x, const double* __restrict__ y,
                         const int32_t* __restrict__ node, int64_t lim) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double s0 = 0, s1 = 0, s2 = 0;
  for (int64_t q = ptr[t]; q < ptr[t + 1]; ++q) {
    const double* p = fe + 3 * (int64_t)slot[q];
    s0 += p[0]; s1 += p[1]; s2 += p[2];
  }
  if (add) { s0 += add[3 * t]; s1 += add[3 * t + 1]; s2 += add[3 * t + 2]; }
  if (mass_h2 && t < lim) {
    int64_t v = node[t];
    double mh = mass_h2[t];
    s0 -= mh * (x[3 * v] - y[3 * t]);
    s1 -= mh * (x[3 * v + 1] - y[3 * t + 1]);
    s2 -= mh * (x[3 * v + 2] - y[3 * t + 2]);
  }
  out[3 * t] = s0; out[3 * t + 1] = s1; out[3 * t + 2] = s2;
}

__global__ void k_gather_rows(int64_t cnt, const int32_t* idx, const double* x, double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  int64_t v = idx[i];
  out[3 * i] = x[3 * v]; out[3 * i + 1] = x[3 * v + 1]; out[3 * i + 2] = x[3 * v + 2];
}

__global__ void k_scatter_rows(int64_t cnt, const int32_t* idx, const double* v, double* x) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  int64_t r = idx[i];
  x[3 * r] = v[3 * i]; x[3 * r + 1] = v[3 * i + 1]; x[3 * r + 2] = v[3 * i + 2];
}

__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void k_inner_update(int64_t m, const double* u2, const double* Sau, const int32_t* region,
                               double* x, double* U2, double* ft2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int64_t v = region[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double du = u2[3 * i + c];
    x[3 * v + c] += du;
    U2[3 * i + c] += du;
    ft2[3 * i + c] -= Sau[3 * i + c];
  }
}

__global__ void k_apply_interior(int64_t n1, const double* u, const int32_t* node, double* x) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n1) return;
  int64_t v = node[p];
  x[3 * v] += u[3 * p]; x[3 * v + 1] += u[3 * p + 1]; x[3 * v + 2] += u[3 * p + 2];
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void polar_forces(int64_t count, const int4* tets, const double* Dm, const double* w, const double* x,
                  double* fe, double* R_out, cudaStream_t st, const StrainLimit* sl) {
  if (count <= 0) return;
  if (sl && (sl->frac > 0.0 || sl->vfrac > 0.0))
    k_polar_forces<true><<<nblk(count, 128), 128, 0, st>>>(count, tets, Dm, w, x, fe, R_out, *sl);
  else
    k_polar_forces<false><<<nblk(count, 128), 128, 0, st>>>(count, tets, Dm, w, x, fe, R_out, StrainLimit{});
  ++g_launches;
}

void gather_forces(int64_t nt, const int64_t* ptr, const int32_t* slot, const double* fe, double* out,
                   const double* add, const double* mass_h2, const double* x, const double* y,
                   const int32_t* node, int64_t lim, cudaStream_t st) {
  if (nt <= 0) return;
  k_gather<<<nblk(nt, 256), 256, 0, st>>>(nt, ptr, slot, fe, out, add, mass_h2, x, y, node, lim);
  ++g_launches;
}

void gather_rows(int64_t cnt, const int32_t* idx, const double* x, double* out, cudaStream_t st) {
  if (cnt > 0) {
    k_gather_rows<<<nblk(cnt, 256), 256, 0, st>>>(cnt, idx, x, out);
    ++g_launches;
  }
}
void scatter_rows(int64_t cnt, const int32_t* idx, const double* v, double* x, cudaStream_t st) {
  if (cnt > 0) {
    k_scatter_rows<<<nblk(cnt, 256), 256, 0, st>>>(cnt, idx, v, x);
    ++g_launches;
  }
}
void axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
  if (n > 0) {
    k_axpby<<<nblk(n, 256), 256, 0, st>>>(n, a, x, b, y);
    ++g_launches;
  }
}
void inner_update(int64_t m, const double* u2, const double* Sau, const int32_t* region, double* x,
                  double* U2, double* ft2, cudaStream_t st) {
  if (m > 0) {
    k_inner_update<<<nblk(m, 256), 256, 0, st>>>(m, u2, Sau, region, x, U2, ft2);
    ++g_launches;
  }
}
void apply_interior(int64_t n1, const double* u, const int32_t* node, double* x, cudaStream_t st) {
  if (n1 > 0) {
    k_apply_interior<<<nblk(n1, 256), 256, 0, st>>>(n1, u, node, x);
    ++g_launches;
  }
}

}  // namespace pdk
