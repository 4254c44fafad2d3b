// Types shared by the mixed-precision kernels (sloppy.cu).
#pragma once

#include "internal.cuh"

namespace lqcd {

constexpr int ST = 128;  // threads per block of the site-tiled kernels (one site each)

enum { EPI_PLAIN = 0, EPI_AXPY = 1, EPI_DOTR = 2, EPI_TS = 3, EPI_RES = 4 };
enum { FLAG_ACTIVE = 1, FLAG_RU = 2 };

struct D4S {
  double a, b, c, d;
};

// FP32 parity field, one right-hand side per slot: [rhs][6][vh] float4
struct F32F {
  float4 *d;
  int vh;
  __device__ void load(int r, int i, float2 v[12]) const;
  __device__ void store(int r, int i, const float2 v[12]) const;
};

// A complex number for the two right-hand sides of a pair: re = (re_even, re_odd).
struct CP {
  float2 re, im;
};

// Reduced-precision parity field storing right-hand sides in pairs: for pair
// P = rhs / 2 and site i, the 24 reals of both members are 24 16-bit pairs
// (even member in the low half) in 6 uint4: [P][6][vh] uint4.  FP16 fields also
// keep one FP32 norm per member and site, [P][vh] float2: the stored halves are
// the values divided by the largest |real| of that member's site spinor.
struct F16P {
  uint4 *d;
  float2 *n;
  int vh;
};
struct BF16P {
  uint4 *d;
  int vh;
};

// per-RHS state of the inner (sloppy) BiCGstab
struct SState {
  double2 rho, alpha, omega, beta;
  double rr, rmax, rr_ru, target2;
  int iters, status, restart, ru_count, stall, pad0;
};

}  // namespace lqcd
