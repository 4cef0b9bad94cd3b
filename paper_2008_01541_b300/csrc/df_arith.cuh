// Double-float arithmetic on the FP32 pipes: a value carried as an FP32 head
// h and an FP32 tail l (h + l, about 48 significant bits).  Used where FP64
// accuracy is wanted but B300's FP64 rate (1/64 of FP32) would bound the
// work: the residual products of the low-precision region solves.  The
// error-free transformations are Knuth's two-sum and the FMA product
// remainder.
#pragma once

namespace pddf {

// One term of a double-float product sum: exact head product (FMA
// remainder), cross terms, and the exact rounding error of h + p, all
// collected in l without renormalising; (h, l) is renormalised by df_norm
// every four terms, which keeps |l| a few units of h's last place in between.
__device__ __forceinline__ void df_acc_lazy(float a, float b, float x, float y, float& h, float& l) {
  const float p = a * x;
  float e = fmaf(a, x, -p);
  e = fmaf(a, y, e);
  e = fmaf(b, x, e);
  const float s = h + p;
  const float bb = s - h;
  l += ((h - (s - bb)) + (p - bb)) + e;
  h = s;
}

__device__ __forceinline__ void df_norm(float& h, float& l) {   // two-sum: no magnitude assumption
  const float s = h + l;
  const float bb = s - h;
  l = (h - (s - bb)) + (l - bb);
  h = s;
}

// (h, l) += (h2, l2) in double-float arithmetic
__device__ __forceinline__ void df_add(float& h, float& l, float h2, float l2) {
  const float s = h + h2;
  const float bb = s - h;
  float t = (h - (s - bb)) + (h2 - bb);
  t += l + l2;
  h = s + t;
  l = t - (h - s);
}

}  // namespace pddf
