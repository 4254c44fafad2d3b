// Double-float arithmetic: unevaluated pairs hi + lo of FP32 numbers
// (TwoSum after Knuth and Dekker; TwoProduct with a fused multiply-add).
// Every operation uses the _rn intrinsics, which the compiler neither
// contracts into FMAs nor reorders, so the error-free transformations hold.
#pragma once

#include <cuda_runtime.h>

namespace lqcd {

struct dfl {
  float h, l;
};
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  float s = __fadd_rn(a.h, b.h);
  float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return dfl{s, __fadd_rn(__fadd_rn(a.l, b.l), e)};
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl{-a.h, -a.l}; }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  return dfl{p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e))};
}
__device__ __forceinline__ dfl df_norm(dfl a) {  // Fast2Sum renormalisation
  float s = __fadd_rn(a.h, a.l);
  return dfl{s, __fsub_rn(a.l, __fsub_rn(s, a.h))};
}

struct cdf {  // complex double-float; .x = real, .y = imaginary
  dfl x, y;
};

}  // namespace lqcd
