// Types shared by the mixed-precision kernels (sloppy.cu, sloppy_host.cu).
#pragma once

#include "internal.cuh"

namespace lqcd {

constexpr int ST = 128;  // threads per block of the site-tiled kernels (one site each)

enum { EPI_PLAIN = 0, EPI_AXPY = 1, EPI_DOTR = 2, EPI_TS = 3, EPI_RES = 4 };
enum { FLAG_ACTIVE = 1, FLAG_RU = 2 };

struct D4S {
  double a, b, c, d;
};

// FP32 parity field [rhs][6][vh] float4
struct F32F {
  float4 *d;
  int vh;
  __device__ void load(int r, int i, float2 v[12]) const;
  __device__ void store(int r, int i, const float2 v[12]) const;
};
// FP16 parity field [rhs][3][vh] uint4 + per-site norm [rhs][vh]
struct F16F {
  uint4 *d;
  float *n;
  int vh;
  __device__ void load(int r, int i, float2 v[12]) const;
  __device__ void store(int r, int i, const float2 v[12]) const;
};
// BF16 parity field [rhs][3][vh] uint4
struct BF16F {
  uint4 *d;
  int vh;
  __device__ void load(int r, int i, float2 v[12]) const;
  __device__ void store(int r, int i, const float2 v[12]) const;
};

// per-RHS state of the inner (sloppy) BiCGstab
struct SState {
  double2 rho, alpha, omega, beta;
  double rr, rmax, rr_ru, target2;
  int iters, status, restart, ru_count, stall, pad0;
};

}  // namespace lqcd
