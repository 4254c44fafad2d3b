// True residual b - D x of the mixed solver in double-float arithmetic.
//
// GB300 runs FP32 FMAs ~73x faster than FP64 ones, so the residual that
// certifies |M x - b| / |b| (Sec. III) is evaluated on the FP32 units with
// unevaluated pairs hi + lo of FP32 numbers (a 48-bit significand):
//   sum:     TwoSum (Knuth; Dekker) for the high parts, low parts added,
//   product: TwoProduct with an FMA for hi*hi, cross terms added to the low part,
// everything with the _rn intrinsics, which the compiler never contracts or
// reorders.  Gauge links and the iterate x are held as such pairs (the links
// split once from FP64); the FP64 source b is split where it is read; the
// residual goes out in FP32 (it only seeds
// the next inner solve) together with FP64-accumulated norms |r|^2, |b|^2.
// The rounding error of one evaluation is a few 1e-14 of |x|, far below the
// 1e-10 residual it certifies (tests compare it with the IEEE FP64 residual).
#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "df.cuh"
#include "fpconv.cuh"

namespace lqcd {

__device__ __forceinline__ cdf load_cdf(const float4 *p) {
  float4 q = *p;
  return cdf{dfl{q.x, q.z}, dfl{q.y, q.w}};
}
// FP64 -> double-float: hi = fl32(v), lo = fl32(v - hi)
__device__ __forceinline__ cdf split_cdf(double2 v) {
  const float hx = (float)v.x, hy = (float)v.y;
  return cdf{dfl{hx, (float)(v.x - (double)hx)}, dfl{hy, (float)(v.y - (double)hy)}};
}

// Shared-projection variant: the three threads of a site (lanes base .. base + 2
// of one warp) each project only their own colour a of the neighbour spinor and
// fetch the other two colours' half spinors from their neighbours by shuffles.
__device__ __forceinline__ cdf shfl_cdf(const cdf &v, int src) {
  return cdf{dfl{__shfl_sync(0xffffffffu, v.x.h, src), __shfl_sync(0xffffffffu, v.x.l, src)},
             dfl{__shfl_sync(0xffffffffu, v.y.h, src), __shfl_sync(0xffffffffu, v.y.l, src)}};
}
template <int MU, int SIGMA, bool DAG>
__device__ __forceinline__ void hop_row_df_sh(const float4 *__restrict__ xs, const float4 *__restrict__ u, int a,
                                              int base, bool act, float sgn, cdf acc[4]) {
  cdf p[4];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) p[sp] = act ? load_cdf(xs + sp * 3 + a) : cdf{dfl{0.f, 0.f}, dfl{0.f, 0.f}};
  cdf h0, h1;  // spin projection of colour a (as spin_project)
  if (MU == 0) {
    h0 = caddi(p[0], p[3], SIGMA);
    h1 = caddi(p[1], p[2], SIGMA);
  } else if (MU == 1) {
    h0 = SIGMA > 0 ? csub(p[0], p[3]) : cadd(p[0], p[3]);
    h1 = SIGMA > 0 ? cadd(p[1], p[2]) : csub(p[1], p[2]);
  } else if (MU == 2) {
    h0 = caddi(p[0], p[2], SIGMA);
    h1 = caddi(p[1], p[3], -SIGMA);
  } else {
    h0 = SIGMA > 0 ? cadd(p[0], p[2]) : csub(p[0], p[2]);
    h1 = SIGMA > 0 ? cadd(p[1], p[3]) : csub(p[1], p[3]);
  }
  cdf h[2][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    h[0][b] = shfl_cdf(h0, base + b);
    h[1][b] = shfl_cdf(h1, base + b);
  }
  cdf ur[3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
    ur[b] = act ? load_cdf(u + (DAG ? b * 3 + a : a * 3 + b)) : cdf{dfl{0.f, 0.f}, dfl{0.f, 0.f}};
  cdf x[2];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    cdf t = DAG ? cmulc(ur[0], h[sp][0]) : cmul(ur[0], h[sp][0]);
#pragma unroll
    for (int b = 1; b < 3; ++b) t = cadd(t, DAG ? cmulc(ur[b], h[sp][b]) : cmul(ur[b], h[sp][b]));
    x[sp] = sgn < 0.f ? cdf{-t.x, -t.y} : t;
  }
  acc[0] = cadd(acc[0], x[0]);
  acc[1] = cadd(acc[1], x[1]);
  if (MU == 0) {
    acc[2] = caddi(acc[2], x[1], -SIGMA);
    acc[3] = caddi(acc[3], x[0], -SIGMA);
  } else if (MU == 1) {
    acc[2] = SIGMA > 0 ? cadd(acc[2], x[1]) : csub(acc[2], x[1]);
    acc[3] = SIGMA > 0 ? csub(acc[3], x[0]) : cadd(acc[3], x[0]);
  } else if (MU == 2) {
    acc[2] = caddi(acc[2], x[0], -SIGMA);
    acc[3] = caddi(acc[3], x[1], SIGMA);
  } else {
    acc[2] = SIGMA > 0 ? cadd(acc[2], x[0]) : csub(acc[2], x[0]);
    acc[3] = SIGMA > 0 ? cadd(acc[3], x[1]) : csub(acc[3], x[1]);
  }
}

template <int MU>
__device__ __forceinline__ void hop_dir_df_sh(const Geom &g, const int c[4], int s, int a, int base, bool act,
                                              const float4 *__restrict__ x, const float4 *__restrict__ U, cdf acc[4]) {
  {
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
    const int sn = site_of(g, cn);
    const float sgn = (MU == 3 && c[3] == g.L[3] - 1) ? -1.f : 1.f;
    hop_row_df_sh<MU, -1, false>(x + (size_t)sn * 12, U + ((size_t)s * 4 + MU) * 9, a, base, act, sgn, acc);
  }
  {
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
    const int sn = site_of(g, cn);
    const float sgn = (MU == 3 && c[3] == 0) ? -1.f : 1.f;
    hop_row_df_sh<MU, +1, true>(x + (size_t)sn * 12, U + ((size_t)sn * 4 + MU) * 9, a, base, act, sgn, acc);
  }
}

struct D4R {
  double a, b, c, d;
};

// Three threads per site (one per output colour, sharing the spin projection
// by shuffles): r = b - x + kappa H x at the sites of parity p_out.  A warp
// takes 10 sites (lanes 0..29; lanes 30, 31 only take part in the shuffles), a
// block 6 warps.  Blocks are ordered (chunk of DF3_CHUNK listed right-hand
// sides, site block, right-hand side in the chunk): blocks issued together
// share their sites' links across the chunk, while the time neighbours of a
// site block stay a few hundred blocks away (both reused from L2).
// Partials |r|^2 (.c) and |b|^2 (.d) per block.
constexpr int DF3_WARP_SITES = 10;
constexpr int DF3_WARPS = 6;
constexpr int DF3_SITES = DF3_WARP_SITES * DF3_WARPS;
constexpr int DF3_CHUNK = 8;
__global__ void __launch_bounds__(32 * DF3_WARPS, 4) k_resid_df3(Geom g, int p_out, const float4 *__restrict__ U,
                                                               const float4 *__restrict__ x,
                                                               const double2 *__restrict__ b, float2 *r, float kh,
                                                               float kl, const int *list, int n, D4R *part,
                                                               int nblk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sl = lane / 3, a = lane - 3 * sl;  // site within the warp, output colour
  const int in_chunk = blockIdx.x % DF3_CHUNK, rest = blockIdx.x / DF3_CHUNK;
  const int blk = rest % nblk, slot = (rest / nblk) * DF3_CHUNK + in_chunk;
  if (slot >= n) return;  // ragged last chunk: the whole block leaves together
  const int i = blk * DF3_SITES + warp * DF3_WARP_SITES + sl;
  const bool act = sl < DF3_WARP_SITES && i < g.Vh;
  const int base = 3 * sl;
  const int rhs = list[slot];
  const size_t stride = (size_t)g.V * 12;
  float rn = 0.f, bn = 0.f;
  int c[4];
  coords_of(g, p_out, act ? i : 0, c);
  const int s = site_of(g, c);
  cdf acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = cdf{dfl{0.f, 0.f}, dfl{0.f, 0.f}};
  const float4 *xr = x + (size_t)rhs * stride;
  hop_dir_df_sh<0>(g, c, s, a, base, act, xr, U, acc);
  hop_dir_df_sh<1>(g, c, s, a, base, act, xr, U, acc);
  hop_dir_df_sh<2>(g, c, s, a, base, act, xr, U, acc);
  hop_dir_df_sh<3>(g, c, s, a, base, act, xr, U, acc);
  if (act) {
    const dfl kd{kh, kl};
    const size_t o = (size_t)rhs * stride + (size_t)s * 12;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
      const int k = sp * 3 + a;
      const cdf bk = split_cdf(b[o + k]), xk = load_cdf(xr + (size_t)s * 12 + k);
      const dfl re = df_norm((bk.x - xk.x) + kd * df_norm(acc[sp].x));
      const dfl im = df_norm((bk.y - xk.y) + kd * df_norm(acc[sp].y));
      const float2 v = make_float2(__fadd_rn(re.h, re.l), __fadd_rn(im.h, im.l));
      r[o + k] = v;
      rn = fmaf(v.x, v.x, fmaf(v.y, v.y, rn));
      bn = fmaf(bk.x.h, bk.x.h, fmaf(bk.y.h, bk.y.h, bn));
    }
  }
  __shared__ double sh[2][32 * DF3_WARPS];
  sh[0][threadIdx.x] = rn;
  sh[1][threadIdx.x] = bn;
  __syncthreads();
  if (threadIdx.x < 64) {  // fold 192 -> 64, then a tree
    sh[0][threadIdx.x] += sh[0][threadIdx.x + 64] + sh[0][threadIdx.x + 128];
    sh[1][threadIdx.x] += sh[1][threadIdx.x + 64] + sh[1][threadIdx.x + 128];
  }
  __syncthreads();
  for (int w = 32; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    part[(size_t)slot * 2 * nblk + (size_t)p_out * nblk + blk] =
        D4R{0.0, 0.0, sh[0][0], sh[1][0]};
}

__global__ void k_df_fin(const D4R *part, int nb, double *rr, double *bb) {
  const int rhs = blockIdx.x;
  double a = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < nb; k += 32) {
    a += part[(size_t)rhs * nb + k].c;
    c += part[(size_t)rhs * nb + k].d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  if (threadIdx.x == 0) {
    rr[rhs] = a;
    bb[rhs] = c;
  }
}

// double-float canonical -> FP64 canonical; four independent elements per thread
// and iteration keep enough loads in flight to stream at the HBM rate.  The
// exact binary32 -> binary64 widenings run on the integer units, leaving one
// FP64 add per value for the narrow FP64 pipe (same result as the casts).
__device__ __forceinline__ double2 join_df(float4 q) {
  return make_double2(lqcd::f32_to_f64_bits(q.x) + lqcd::f32_to_f64_bits(q.z),
                      lqcd::f32_to_f64_bits(q.y) + lqcd::f32_to_f64_bits(q.w));
}

__global__ void k_join_df(const float4 *__restrict__ in, double2 *out, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; k + 3 * stride < n; k += 4 * stride) {
    float4 q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) q[u] = in[k + u * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u) out[k + u * stride] = join_df(q[u]);
  }
  for (; k < n; k += stride) out[k] = join_df(in[k]);
}

int df_join(lqcd_ctx *ctx, const float4 *in, double2 *out, size_t n, cudaStream_t st) {
  unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
  KL k_join_df<<<blocks, 256, 0, st>>>(in, out, n);
  LQCD_LAUNCH_CHECK(ctx, "k_join_df");
  return LQCD_OK;
}

// r = b - D x in double-float; per-RHS |r|^2, |b|^2 to the host arrays
int df_residual(lqcd_ctx *ctx, const float4 *x, const double2 *b, float2 *r, const int *list, int n, double *rr,
                double *bb, cudaStream_t st) {
  if (n <= 0) return LQCD_OK;
  const Geom &g = ctx->geom;
  const int nblk = (g.Vh + DF3_SITES - 1) / DF3_SITES;
  int rc = LQCD_OK;
  Carver sizing(nullptr);
  sizing.take<D4R>((size_t)n * 2 * nblk);
  sizing.take<double>(2 * (size_t)n);
  sizing.take<int>((size_t)n);
  void *w = workspace(ctx, WS_F64_PART, sizing.size(), &rc);
  if (!w) return rc;
  Carver cv(w);
  D4R *part = cv.take<D4R>((size_t)n * 2 * nblk);
  double *d_rr = cv.take<double>(2 * (size_t)n);
  double *d_bb = d_rr + n;
  int *d_list = cv.take<int>((size_t)n);
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(d_list, list, n * sizeof(int), cudaMemcpyHostToDevice, st));
  const float kh = (float)ctx->kappa, kl = (float)(ctx->kappa - (double)kh);
  for (int p = 0; p < 2; ++p) {
    const long long blocks = (long long)((n + DF3_CHUNK - 1) / DF3_CHUNK) * nblk * DF3_CHUNK;
    KL k_resid_df3<<<(unsigned)blocks, 32 * DF3_WARPS, 0, st>>>(g, p, ctx->Udf, x, b, r, kh, kl, d_list, n, part, nblk);
    LQCD_LAUNCH_CHECK(ctx, "k_resid_df3");
  }
  KL k_df_fin<<<n, 32, 0, st>>>(part, 2 * nblk, d_rr, d_bb);
  LQCD_LAUNCH_CHECK(ctx, "k_df_fin");
  std::vector<double> h(2 * (size_t)n);
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), d_rr, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  for (int j = 0; j < n; ++j) {
    rr[list[j]] = h[j];
    bb[list[j]] = h[n + j];
  }
  return LQCD_OK;
}

}  // namespace lqcd
