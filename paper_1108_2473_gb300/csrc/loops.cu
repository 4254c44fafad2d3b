// Loop contraction (Eq. loop; Eq. loop stochastic):
//   L_Gamma(x) += w * sum_i src_i(x)^+ Gamma sol_i(x)
// per site and per time slice, FP64 accumulation in a fixed order.
#include <vector>

#include "internal.cuh"

namespace lqcd {

__device__ __forceinline__ double2 gamma_phase(int ph, double2 v) {
  switch (ph) {
    case 0: return v;
    case 1: return make_double2(-v.x, -v.y);
    case 2: return make_double2(-v.y, v.x);   // +i v
    default: return make_double2(v.y, -v.x);  // -i v
  }
}

#define LOOP_THREADS 128

// grid: (ceil(Vs / LOOP_THREADS), Lt).  Each thread owns one site of slice t,
// sums over RHS, updates per_site, and the block writes its slice partial.
__global__ void __launch_bounds__(LOOP_THREADS) k_loops(Geom g, const double2 *__restrict__ src,
                                                        const double2 *__restrict__ sol, int nrhs, double weight,
                                                        double2 *per_site, double2 *part) {
  int vs = g.L[0] * g.L[1] * g.L[2];
  int t = blockIdx.y;
  int xs = blockIdx.x * blockDim.x + threadIdx.x;
  double2 acc[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) acc[k] = make_double2(0.0, 0.0);
  if (xs < vs) {
    size_t s = (size_t)t * vs + xs;
    for (int i = 0; i < nrhs; ++i) {
      const double2 *a = src + ((size_t)i * g.V + s) * 12;
      const double2 *b = sol + ((size_t)i * g.V + s) * 12;
      double2 ea[12], eb[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        ea[k] = a[k];
        eb[k] = b[k];
      }
#pragma unroll
      for (int gi = 0; gi < 6; ++gi) {
        double2 sum = make_double2(0.0, 0.0);
#pragma unroll
        for (int al = 0; al < 4; ++al) {
          int be = kGammaPerm[gi][al];
          int ph = kGammaPhase[gi][al];
#pragma unroll
          for (int c = 0; c < 3; ++c) sum = cadd(sum, cmulc(ea[al * 3 + c], gamma_phase(ph, eb[be * 3 + c])));
        }
        acc[gi] = cadd(acc[gi], sum);
      }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = cscale(acc[k], weight);
    if (per_site) {
#pragma unroll
      for (int k = 0; k < 6; ++k) per_site[s * 6 + k] = cadd(per_site[s * 6 + k], acc[k]);
    }
  }
  if (!part) return;
  // fixed-order block reduction of the 6 complex sums
  __shared__ double2 sh[LOOP_THREADS / 32][6];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double re = acc[k].x, im = acc[k].y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) sh[w][k] = make_double2(re, im);
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double2 tot = make_double2(0.0, 0.0);
    for (int ww = 0; ww < LOOP_THREADS / 32; ++ww) tot = cadd(tot, sh[ww][threadIdx.x]);
    part[((size_t)t * gridDim.x + blockIdx.x) * 6 + threadIdx.x] = tot;
  }
}

__global__ void k_loops_fin(int nbx, const double2 *part, double2 *per_t) {
  int t = blockIdx.x, k = threadIdx.x;
  if (k >= 6) return;
  double2 tot = make_double2(0.0, 0.0);
  for (int b = 0; b < nbx; ++b) tot = cadd(tot, part[((size_t)t * nbx + b) * 6 + k]);
  per_t[t * 6 + k] = cadd(per_t[t * 6 + k], tot);
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_loops_batch(lqcd_ctx *ctx, const double *src, const double *sol, int nrhs, double weight,
                                double *per_site, double *per_t, lqcd_stream_t stream) {
  if (!ctx || nrhs < 0 || (nrhs > 0 && (!src || !sol)))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_loops_batch: bad argument");
  if (nrhs == 0 || (!per_site && !per_t)) return LQCD_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Geom &g = ctx->geom;
  int vs = g.L[0] * g.L[1] * g.L[2], lt = g.L[3];
  int nbx = (vs + LOOP_THREADS - 1) / LOOP_THREADS;
  int rc = LQCD_OK;
  double2 *part = nullptr, *dpt = nullptr;
  bool host_pt = per_t && !is_device_ptr(per_t);
  if (per_t) {
    char *w = (char *)workspace(ctx, WS_LOOP_PART, ((size_t)lt * nbx * 6 + (size_t)lt * 6) * sizeof(double2), &rc);
    if (!w) return rc;
    part = (double2 *)w;
    dpt = host_pt ? part + (size_t)lt * nbx * 6 : (double2 *)per_t;
    if (host_pt)
      LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(dpt, per_t, (size_t)lt * 6 * sizeof(double2), cudaMemcpyHostToDevice, st));
  }
  KL k_loops<<<dim3(nbx, lt), LOOP_THREADS, 0, st>>>(g, (const double2 *)src, (const double2 *)sol, nrhs, weight,
                                                  (double2 *)per_site, part);
  LQCD_LAUNCH_CHECK(ctx, "k_loops");
  if (per_t) {
    KL k_loops_fin<<<lt, 32, 0, st>>>(nbx, part, dpt);
    LQCD_LAUNCH_CHECK(ctx, "k_loops_fin");
    if (host_pt) {
      LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(per_t, dpt, (size_t)lt * 6 * sizeof(double2), cudaMemcpyDeviceToHost, st));
      LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    }
  }
  return LQCD_OK;
}
