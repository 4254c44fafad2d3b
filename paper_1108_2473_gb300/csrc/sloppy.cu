// Mixed-precision many-RHS solver (Sec. II: QUDA-style mixed-precision
// BiCGstab for the all-to-all inversions; Sec. III: stop on the true
// relative residual |M x - b| / |b| of the full operator).
//
// Three precision levels:
//   * sloppy  -- Krylov vectors stored as FP16 with one FP32 norm per site
//               (values scaled into [-1, 1]) or as BF16; links as FP16
//               reconstruct-12; all arithmetic in FP32;
//   * FP32    -- the iterate x and the reliable-update residual
//               r = b - D_hat x, with FP32 reconstruct-12 links;
//   * FP64    -- the outer defect correction: r = b - D x on the full lattice
//               in FP64, inner solve D e = r, x += e, until |r| / |b| <= tol.
//
// Vectors are parity-compact, structure-of-arrays per RHS:
//   sloppy: [rhs][3][Vh] uint4 (8 x 16-bit reals each) + [rhs][Vh] float norm
//   FP32:   [rhs][6][Vh] float4
// A spinor's 24 reals are ordered ((spin * 3 + colour) * 2 + re/im).
//
// Kernels walk a device-side list of RHS: work item w = (list[w / nbx],
// site block w % nbx), grid-stride over a fixed grid, so converged or idle
// right-hand sides cost nothing.  Every reduction is written as one partial
// per (RHS, site block) and summed by one warp per RHS in a fixed order, so a
// right-hand side's arithmetic does not depend on which others share the batch.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "sloppy.cuh"

namespace lqcd {

// ============================================================ accessors
__device__ __forceinline__ float2 h2f(unsigned w) {
  __half2 h = *reinterpret_cast<__half2 *>(&w);
  return __half22float2(h);
}
__device__ __forceinline__ unsigned f2h(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<unsigned *>(&h);
}
__device__ __forceinline__ float2 b2f(unsigned w) {
  // bf16 -> f32 is exact: the bf16 bits are the high half of the f32
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ unsigned f2b(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<unsigned *>(&h);
}

__device__ __forceinline__ void F32F::load(int r, int i, float2 v[12]) const {
  const float4 *p = d + (size_t)r * 6 * vh + i;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float4 q = p[(size_t)k * vh];
    v[2 * k] = make_float2(q.x, q.y);
    v[2 * k + 1] = make_float2(q.z, q.w);
  }
}
__device__ __forceinline__ void F32F::store(int r, int i, const float2 v[12]) const {
  float4 *p = d + (size_t)r * 6 * vh + i;
#pragma unroll
  for (int k = 0; k < 6; ++k) p[(size_t)k * vh] = make_float4(v[2 * k].x, v[2 * k].y, v[2 * k + 1].x, v[2 * k + 1].y);
}

__device__ __forceinline__ void F16F::load(int r, int i, float2 v[12]) const {
  const uint4 *p = d + (size_t)r * 3 * vh + i;
  float s = n[(size_t)r * vh + i];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint4 q = p[(size_t)k * vh];
    float2 a = h2f(q.x), b = h2f(q.y), c = h2f(q.z), e = h2f(q.w);
    v[4 * k] = make_float2(a.x * s, a.y * s);
    v[4 * k + 1] = make_float2(b.x * s, b.y * s);
    v[4 * k + 2] = make_float2(c.x * s, c.y * s);
    v[4 * k + 3] = make_float2(e.x * s, e.y * s);
  }
}
__device__ __forceinline__ void F16F::store(int r, int i, const float2 v[12]) const {
  float m = 0.0f;
#pragma unroll
  for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].x), fabsf(v[k].y)));
  float inv = m > 0.0f ? 1.0f / m : 0.0f;
  uint4 *p = d + (size_t)r * 3 * vh + i;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint4 q;
    q.x = f2h(v[4 * k].x * inv, v[4 * k].y * inv);
    q.y = f2h(v[4 * k + 1].x * inv, v[4 * k + 1].y * inv);
    q.z = f2h(v[4 * k + 2].x * inv, v[4 * k + 2].y * inv);
    q.w = f2h(v[4 * k + 3].x * inv, v[4 * k + 3].y * inv);
    p[(size_t)k * vh] = q;
  }
  n[(size_t)r * vh + i] = m;
}

__device__ __forceinline__ void BF16F::load(int r, int i, float2 v[12]) const {
  const uint4 *p = d + (size_t)r * 3 * vh + i;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint4 q = p[(size_t)k * vh];
    v[4 * k] = b2f(q.x);
    v[4 * k + 1] = b2f(q.y);
    v[4 * k + 2] = b2f(q.z);
    v[4 * k + 3] = b2f(q.w);
  }
}
__device__ __forceinline__ void BF16F::store(int r, int i, const float2 v[12]) const {
  uint4 *p = d + (size_t)r * 3 * vh + i;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint4 q;
    q.x = f2b(v[4 * k].x, v[4 * k].y);
    q.y = f2b(v[4 * k + 1].x, v[4 * k + 1].y);
    q.z = f2b(v[4 * k + 2].x, v[4 * k + 2].y);
    q.w = f2b(v[4 * k + 3].x, v[4 * k + 3].y);
    p[(size_t)k * vh] = q;
  }
}

// reconstruct-12 link: rows 0, 1 stored, row 2 = (row0 x row1)^*
template <bool L32>
__device__ __forceinline__ void load_link(const void *links, int p, int mu, int i, int vh, float2 u[3][3]) {
  size_t base = ((size_t)(p * 4 + mu) * 3) * vh + i;
  if (L32) {
    const float4 *U = (const float4 *)links;
    float4 q0 = U[base], q1 = U[base + vh], q2 = U[base + 2 * (size_t)vh];
    u[0][0] = make_float2(q0.x, q0.y);
    u[0][1] = make_float2(q0.z, q0.w);
    u[0][2] = make_float2(q1.x, q1.y);
    u[1][0] = make_float2(q1.z, q1.w);
    u[1][1] = make_float2(q2.x, q2.y);
    u[1][2] = make_float2(q2.z, q2.w);
  } else {
    const uint2 *U = (const uint2 *)links;
    uint2 w0 = U[base], w1 = U[base + vh], w2 = U[base + 2 * (size_t)vh];
    u[0][0] = h2f(w0.x);
    u[0][1] = h2f(w0.y);
    u[0][2] = h2f(w1.x);
    u[1][0] = h2f(w1.y);
    u[1][1] = h2f(w2.x);
    u[1][2] = h2f(w2.y);
  }
  float2 c0 = csub(cmul(u[0][1], u[1][2]), cmul(u[0][2], u[1][1]));
  float2 c1 = csub(cmul(u[0][2], u[1][0]), cmul(u[0][0], u[1][2]));
  float2 c2 = csub(cmul(u[0][0], u[1][1]), cmul(u[0][1], u[1][0]));
  u[2][0] = make_float2(c0.x, -c0.y);
  u[2][1] = make_float2(c1.x, -c1.y);
  u[2][2] = make_float2(c2.x, -c2.y);
}

// ============================================================ hopping term
template <int MU, class IN, bool L32>
__device__ __forceinline__ void hop_dir_s(const Geom &g, int p_out, const int c[4], int i, const IN &in, int rhs,
                                          const void *links, float2 acc[4][3]) {
  float2 v[12], h[2][3], x[2][3], u[3][3];
  float2 ps[4][3];
  {  // forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
    int sn = site_of(g, cn);
    in.load(rhs, sn >> 1, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) ps[k / 3][k % 3] = v[k];
    load_link<L32>(links, p_out, MU, i, g.Vh, u);
    spin_project<MU, -1>(ps, h);
    su3_mul<false>(u, h, x);
    if (MU == 3 && c[3] == g.L[3] - 1) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) x[a][b] = make_float2(-x[a][b].x, -x[a][b].y);
    }
    spin_accum<MU, -1>(acc, x);
  }
  {  // backward: (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu)
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
    int sn = site_of(g, cn);
    in.load(rhs, sn >> 1, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) ps[k / 3][k % 3] = v[k];
    load_link<L32>(links, 1 - p_out, MU, sn >> 1, g.Vh, u);
    spin_project<MU, +1>(ps, h);
    su3_mul<true>(u, h, x);
    if (MU == 3 && c[3] == 0) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) x[a][b] = make_float2(-x[a][b].x, -x[a][b].y);
    }
    spin_accum<MU, +1>(acc, x);
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// fixed-order block reduction of a D4 (all ST threads participate)
__device__ __forceinline__ void block_reduce_store(D4S v, D4S *dst) {
  __shared__ D4S sh[ST / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v.a = warp_sum_d(v.a);
  v.b = warp_sum_d(v.b);
  v.c = warp_sum_d(v.c);
  v.d = warp_sum_d(v.d);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    D4S t = sh[0];
#pragma unroll
    for (int k = 1; k < ST / 32; ++k) {
      t.a += sh[k].a;
      t.b += sh[k].b;
      t.c += sh[k].c;
      t.d += sh[k].d;
    }
    *dst = t;
  }
  __syncthreads();
}

// out = cA A + cB B + cH (H in) at the sites of parity p_out.
// EPI_PLAIN: A, B unused.  EPI_AXPY: B unused.  EPI_DOTR: partial <B, out>.
// EPI_TS: partials <out, A> and |out|^2.  EPI_RES: partial |out|^2.
template <class IN, class OUT, bool L32, int EPI>
__global__ void __launch_bounds__(ST) k_hop_s(Geom g, int p_out, const void *links, IN in, OUT out, OUT A, OUT B,
                                              float cA, float cB, float cH, const int *list, const int *count,
                                              D4S *part, int nbx, unsigned long long *prof) {
  const int n_items = *count * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int rhs = list[w / nbx], sb = w % nbx;
    const int i = sb * ST + threadIdx.x;
    if (prof && threadIdx.x == 0) atomicAdd(prof + EPI, (unsigned long long)min(ST, g.Vh - sb * ST));
    D4S red = {0, 0, 0, 0};
    if (i < g.Vh) {
      int c[4];
      coords_of(g, p_out, i, c);
      float2 acc[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) acc[a][b] = make_float2(0.f, 0.f);
      hop_dir_s<0, IN, L32>(g, p_out, c, i, in, rhs, links, acc);
      hop_dir_s<1, IN, L32>(g, p_out, c, i, in, rhs, links, acc);
      hop_dir_s<2, IN, L32>(g, p_out, c, i, in, rhs, links, acc);
      hop_dir_s<3, IN, L32>(g, p_out, c, i, in, rhs, links, acc);
      float2 o[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) o[k] = make_float2(cH * acc[k / 3][k % 3].x, cH * acc[k / 3][k % 3].y);
      float2 a[12];
      if (EPI != EPI_PLAIN) {
        A.load(rhs, i, a);
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = make_float2(fmaf(cA, a[k].x, o[k].x), fmaf(cA, a[k].y, o[k].y));
      }
      if (EPI == EPI_RES) {
        float2 b[12];
        B.load(rhs, i, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = make_float2(fmaf(cB, b[k].x, o[k].x), fmaf(cB, b[k].y, o[k].y));
      }
      out.store(rhs, i, o);
      if (EPI == EPI_DOTR) {
        float2 r[12];
        B.load(rhs, i, r);
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          re += r[k].x * o[k].x + r[k].y * o[k].y;
          im += r[k].x * o[k].y - r[k].y * o[k].x;
        }
        red.a = re;
        red.b = im;
      } else if (EPI == EPI_TS) {
        float re = 0.f, im = 0.f, nn = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          re += o[k].x * a[k].x + o[k].y * a[k].y;
          im += o[k].x * a[k].y - o[k].y * a[k].x;
          nn += o[k].x * o[k].x + o[k].y * o[k].y;
        }
        red.a = re;
        red.b = im;
        red.d = nn;
      } else if (EPI == EPI_RES) {
        float nn = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) nn += o[k].x * o[k].x + o[k].y * o[k].y;
        red.c = nn;
      }
    }
    if (EPI == EPI_DOTR || EPI == EPI_TS || EPI == EPI_RES) block_reduce_store(red, part + (size_t)rhs * nbx + sb);
  }
}

// ============================================================ BLAS kernels
__device__ __forceinline__ float2 f2(double2 a) { return make_float2((float)a.x, (float)a.y); }

// p = r + beta (p - omega v); on restart rhat = r, p = r.
template <class S>
__global__ void __launch_bounds__(ST) k_blas_p(int vh, const SState *sc, S r, S rhat, S p, S v, const int *list,
                                               const int *count, int nbx) {
  const int n_items = *count * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int rhs = list[w / nbx];
    const int i = (w % nbx) * ST + threadIdx.x;
    if (i >= vh) continue;
    float2 rv[12];
    r.load(rhs, i, rv);
    if (sc[rhs].restart) {
      rhat.store(rhs, i, rv);
      p.store(rhs, i, rv);
    } else {
      float2 be = f2(sc[rhs].beta), om = f2(sc[rhs].omega);
      float2 pv[12], vv[12];
      p.load(rhs, i, pv);
      v.load(rhs, i, vv);
#pragma unroll
      for (int k = 0; k < 12; ++k) pv[k] = cadd(rv[k], cmul(be, csub(pv[k], cmul(om, vv[k]))));
      p.store(rhs, i, pv);
    }
  }
}

// s = r - alpha v
template <class S>
__global__ void __launch_bounds__(ST) k_blas_s(int vh, const SState *sc, S r, S v, S s, const int *list,
                                               const int *count, int nbx) {
  const int n_items = *count * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int rhs = list[w / nbx];
    const int i = (w % nbx) * ST + threadIdx.x;
    if (i >= vh) continue;
    float2 al = f2(sc[rhs].alpha);
    float2 rv[12], vv[12];
    r.load(rhs, i, rv);
    v.load(rhs, i, vv);
#pragma unroll
    for (int k = 0; k < 12; ++k) rv[k] = csub(rv[k], cmul(al, vv[k]));
    s.store(rhs, i, rv);
  }
}

// x += alpha p + omega s (FP32 x); r = s - omega t; partials <rhat, r>, |r|^2
template <class S>
__global__ void __launch_bounds__(ST) k_blas_xr(int vh, const SState *sc, F32F x, S p, S s, S t, S r, S rhat,
                                                const int *list, const int *count, D4S *part, int nbx) {
  const int n_items = *count * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int rhs = list[w / nbx], sb = w % nbx;
    const int i = sb * ST + threadIdx.x;
    D4S red = {0, 0, 0, 0};
    if (i < vh) {
      float2 al = f2(sc[rhs].alpha), om = f2(sc[rhs].omega);
      float2 xv[12], pv[12], sv[12], tv[12];
      x.load(rhs, i, xv);
      p.load(rhs, i, pv);
      s.load(rhs, i, sv);
      t.load(rhs, i, tv);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        xv[k] = cadd(xv[k], cadd(cmul(al, pv[k]), cmul(om, sv[k])));
        sv[k] = csub(sv[k], cmul(om, tv[k]));
      }
      x.store(rhs, i, xv);
      r.store(rhs, i, sv);
      rhat.load(rhs, i, pv);
      float re = 0.f, im = 0.f, nn = 0.f;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        re += pv[k].x * sv[k].x + pv[k].y * sv[k].y;
        im += pv[k].x * sv[k].y - pv[k].y * sv[k].x;
        nn += sv[k].x * sv[k].x + sv[k].y * sv[k].y;
      }
      red.a = re;
      red.b = im;
      red.c = nn;
    }
    block_reduce_store(red, part + (size_t)rhs * nbx + sb);
  }
}

// r (sloppy) = src (FP32); optionally x = 0; partials <rhat, r>, |r|^2 (rhat may alias r)
template <class S>
__global__ void __launch_bounds__(ST) k_blas_copy(int vh, F32F src, S r, S rhat, bool use_rhat, F32F x, bool zero_x,
                                                  const int *list, const int *count, D4S *part, int nbx) {
  const int n_items = *count * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int rhs = list[w / nbx], sb = w % nbx;
    const int i = sb * ST + threadIdx.x;
    D4S red = {0, 0, 0, 0};
    if (i < vh) {
      float2 v[12], h[12];
      src.load(rhs, i, v);
      r.store(rhs, i, v);
      if (zero_x) {
#pragma unroll
        for (int k = 0; k < 12; ++k) h[k] = make_float2(0.f, 0.f);
        x.store(rhs, i, h);
      }
      if (use_rhat) rhat.load(rhs, i, h);
      float re = 0.f, im = 0.f, nn = 0.f;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        float2 q = use_rhat ? h[k] : v[k];
        re += q.x * v[k].x + q.y * v[k].y;
        im += q.x * v[k].y - q.y * v[k].x;
        nn += v[k].x * v[k].x + v[k].y * v[k].y;
      }
      red.a = re;
      red.b = im;
      red.c = nn;
    }
    block_reduce_store(red, part + (size_t)rhs * nbx + sb);
  }
}

// ============================================ precision conversion kernels
// dst (FP32 parity field) = scale[rhs] * src (canonical FP64 [rhs][V][12]) on parity p
__global__ void __launch_bounds__(ST) k_cvt64to32(Geom g, int p, const double2 *__restrict__ src, F32F dst,
                                                  const double *scale, const int *list, const int *count, int nbx) {
  const int n_items = *count * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int rhs = list[w / nbx];
    const int i = (w % nbx) * ST + threadIdx.x;
    if (i >= g.Vh) continue;
    int c[4];
    coords_of(g, p, i, c);
    const double2 *q = src + ((size_t)rhs * g.V + site_of(g, c)) * 12;
    double sc = scale[rhs];
    float2 v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = make_float2((float)(q[k].x * sc), (float)(q[k].y * sc));
    dst.store(rhs, i, v);
  }
}

// x (canonical FP64) += scale[rhs] * src (FP32 parity field) on parity p
__global__ void __launch_bounds__(ST) k_accum64(Geom g, int p, F32F src, double2 *x, const double *scale,
                                                const int *list, const int *count, int nbx) {
  const int n_items = *count * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int rhs = list[w / nbx];
    const int i = (w % nbx) * ST + threadIdx.x;
    if (i >= g.Vh) continue;
    int c[4];
    coords_of(g, p, i, c);
    double2 *q = x + ((size_t)rhs * g.V + site_of(g, c)) * 12;
    double sc = scale[rhs];
    float2 v[12];
    src.load(rhs, i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = make_double2(q[k].x + sc * (double)v[k].x, q[k].y + sc * (double)v[k].y);
  }
}

// ============================================================ finalisers
__device__ __forceinline__ D4S warp_total_s(const D4S *part, int nb) {
  D4S acc = {0, 0, 0, 0};
  for (int k = threadIdx.x; k < nb; k += 32) {
    D4S v = part[k];
    acc.a += v.a;
    acc.b += v.b;
    acc.c += v.c;
    acc.d += v.d;
  }
  acc.a = warp_sum_d(acc.a);
  acc.b = warp_sum_d(acc.b);
  acc.c = warp_sum_d(acc.c);
  acc.d = warp_sum_d(acc.d);
  return acc;
}

__device__ __forceinline__ double2 cdiv_d(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// after the inner right-hand side is loaded into r (partials: |r|^2 in .c)
__global__ void k_sfin_init(SState *sc, int *flags, const int *list, const int *count, const D4S *part, int nb) {
  if (blockIdx.x >= *count) return;
  int rhs = list[blockIdx.x];
  D4S t = warp_total_s(part + (size_t)rhs * nb, nb);
  if (threadIdx.x) return;
  SState &s = sc[rhs];
  s.rr = t.c;
  s.rmax = t.c;
  s.rr_ru = t.c;
  s.rho = make_double2(t.c, 0.0);
  s.alpha = s.omega = make_double2(1.0, 0.0);
  s.beta = make_double2(0.0, 0.0);
  s.restart = 1;
  s.stall = 0;
  int f = FLAG_ACTIVE;
  if (!isfinite(t.c)) {
    s.status = LQCD_ERR_NONFINITE;
    f = 0;
  } else if (t.c <= s.target2) {
    f = 0;
  }
  flags[rhs] = f;
}

__global__ void k_sfin_alpha(SState *sc, const int *list, const int *count, const D4S *part, int nb) {
  if (blockIdx.x >= *count) return;
  int rhs = list[blockIdx.x];
  D4S t = warp_total_s(part + (size_t)rhs * nb, nb);
  if (threadIdx.x) return;
  SState &s = sc[rhs];
  double2 rv = make_double2(t.a, t.b);
  s.alpha = (rv.x == 0.0 && rv.y == 0.0) ? make_double2(0.0, 0.0) : cdiv_d(s.rho, rv);
  s.restart = 0;
}

__global__ void k_sfin_omega(SState *sc, const int *list, const int *count, const D4S *part, int nb) {
  if (blockIdx.x >= *count) return;
  int rhs = list[blockIdx.x];
  D4S t = warp_total_s(part + (size_t)rhs * nb, nb);
  if (threadIdx.x) return;
  SState &s = sc[rhs];
  s.omega = (t.d == 0.0) ? make_double2(0.0, 0.0) : make_double2(t.a / t.d, t.b / t.d);
}

// convergence / reliable-update decision after the x, r update
__global__ void k_sfin_conv(SState *sc, int *flags, const int *list, const int *count, const D4S *part, int nb,
                            double delta2, int max_iter) {
  if (blockIdx.x >= *count) return;
  int rhs = list[blockIdx.x];
  D4S t = warp_total_s(part + (size_t)rhs * nb, nb);
  if (threadIdx.x) return;
  SState &s = sc[rhs];
  double2 rho_new = make_double2(t.a, t.b);
  s.rr = t.c;
  s.iters += 1;
  if (!isfinite(t.a) || !isfinite(t.b) || !isfinite(t.c)) {
    s.status = LQCD_ERR_NONFINITE;
    flags[rhs] = 0;
    return;
  }
  int f = FLAG_ACTIVE;
  if (t.c <= s.target2 || t.c < delta2 * s.rmax) f |= FLAG_RU;  // verify / refresh with an FP32 true residual
  if (s.iters >= max_iter) f |= FLAG_RU;                          // final FP32 residual before stopping
  s.rmax = fmax(s.rmax, t.c);
  double om2 = s.omega.x * s.omega.x + s.omega.y * s.omega.y;
  double rho2 = rho_new.x * rho_new.x + rho_new.y * rho_new.y;
  if (om2 == 0.0 || rho2 == 0.0 || rho2 < 1e-60 * t.c * t.c) {
    s.restart = 1;  // breakdown: restart the shadow residual
    s.rho = make_double2(t.c, 0.0);
    s.alpha = s.omega = make_double2(1.0, 0.0);
    s.beta = make_double2(0.0, 0.0);
  } else {
    s.beta = cmul_d(cdiv_d(rho_new, s.rho), cdiv_d(s.alpha, s.omega));
    s.rho = rho_new;
  }
  flags[rhs] = f;
}

// after r32 = b32 - D_hat x32 (partials |r32|^2 in .c): accept, stop or continue
__global__ void k_sfin_ru(SState *sc, int *flags, const int *list, const int *count, const D4S *part, int nb,
                          int max_iter) {
  if (blockIdx.x >= *count) return;
  int rhs = list[blockIdx.x];
  D4S t = warp_total_s(part + (size_t)rhs * nb, nb);
  if (threadIdx.x) return;
  SState &s = sc[rhs];
  s.ru_count += 1;
  double prev = s.rr_ru;
  s.rr_ru = t.c;
  if (!isfinite(t.c)) {
    s.status = LQCD_ERR_NONFINITE;
    flags[rhs] = 0;
    return;
  }
  // FP32 residual no longer improving: the inner precision floor is reached
  if (t.c > 0.25 * prev) s.stall += 1; else s.stall = 0;
  if (t.c <= s.target2 || s.stall >= 2 || s.iters >= max_iter) {
    flags[rhs] = 0;  // inner solve finished for this cycle
    return;
  }
  s.rmax = t.c;
  flags[rhs] = FLAG_ACTIVE | FLAG_RU;  // r is replaced by r32 next
}

// after the reliable update copied r32 into r: refresh rho = <rhat, r>
__global__ void k_sfin_ru2(SState *sc, int *flags, const int *list, const int *count, const D4S *part, int nb) {
  if (blockIdx.x >= *count) return;
  int rhs = list[blockIdx.x];
  D4S t = warp_total_s(part + (size_t)rhs * nb, nb);
  if (threadIdx.x) return;
  SState &s = sc[rhs];
  s.rr = t.c;
  if (!s.restart) s.rho = make_double2(t.a, t.b);
  else s.rho = make_double2(t.c, 0.0);
  flags[rhs] = FLAG_ACTIVE;
}

// deterministic compaction of flags into the active and reliable-update lists
__global__ void k_build_lists(int n, const int *flags, int *act_list, int *act_count, int *ru_list, int *ru_count) {
  __shared__ int sa[1024], sr[1024];
  int tid = threadIdx.x, nt = blockDim.x;
  int per = (n + nt - 1) / nt;
  int b0 = tid * per, b1 = min(n, b0 + per);
  int ca = 0, cr = 0;
  for (int k = b0; k < b1; ++k) {
    ca += (flags[k] & FLAG_ACTIVE) ? 1 : 0;
    cr += (flags[k] & FLAG_RU) ? 1 : 0;
  }
  sa[tid] = ca;
  sr[tid] = cr;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {  // inclusive scan
    int va = tid >= off ? sa[tid - off] : 0, vr = tid >= off ? sr[tid - off] : 0;
    __syncthreads();
    sa[tid] += va;
    sr[tid] += vr;
    __syncthreads();
  }
  int oa = sa[tid] - ca, orr = sr[tid] - cr;
  for (int k = b0; k < b1; ++k) {
    if (flags[k] & FLAG_ACTIVE) act_list[oa++] = k;
    if (flags[k] & FLAG_RU) ru_list[orr++] = k;
  }
  if (tid == nt - 1) {
    *act_count = sa[tid];
    *ru_count = sr[tid];
  }
}

}  // namespace lqcd

// ======================================================== host-side driver
namespace lqcd {

struct SloppyState {
  int cap = 0;
  uint4 *sd = nullptr;  // 7 sloppy fields
  float *sn = nullptr;  // their norms
  float4 *f32 = nullptr;  // 5 FP32 fields
  double2 *r64 = nullptr;  // canonical FP64 residual
  char *small = nullptr;
  size_t small_bytes = 0;
  int *h_counts = nullptr;  // pinned
};

void sloppy_free(lqcd_ctx *ctx) {
  SloppyState *s = ctx->sloppy;
  if (!s) return;
  cudaFree(s->sd);
  cudaFree(s->sn);
  cudaFree(s->f32);
  cudaFree(s->r64);
  cudaFree(s->small);
  if (s->h_counts) cudaFreeHost(s->h_counts);
  delete s;
  ctx->sloppy = nullptr;
}

int pack_gauge_sloppy(lqcd_ctx *, cudaStream_t) { return LQCD_OK; }  // packed by k_pack_gauge

static int num_sms(int device) {
  static int cached[64] = {0};
  if (device >= 0 && device < 64 && cached[device]) return cached[device];
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
  if (n <= 0) n = 1;
  if (device >= 0 && device < 64) cached[device] = n;
  return n;
}

// per-RHS state, flags, lists, scales and reduction partials in one buffer
struct SmallBufs {
  SState *sc;
  int *flags, *act_list, *ru_list, *cyc_list, *counts;
  double *scale, *unscale;
  D4S *part;
  size_t bytes;
  size_t size() const { return bytes; }
};
static SmallBufs small_layout(void *base, int cap, int nbx) {
  Carver cv(base);
  SmallBufs b;
  b.sc = cv.take<SState>(cap);
  b.flags = cv.take<int>(cap);
  b.act_list = cv.take<int>(cap);
  b.ru_list = cv.take<int>(cap);
  b.cyc_list = cv.take<int>(cap);
  b.counts = cv.take<int>(16);
  b.scale = cv.take<double>(cap);
  b.unscale = cv.take<double>(cap);
  b.part = cv.take<D4S>((size_t)cap * nbx);
  b.bytes = cv.size();
  return b;
}

static int sloppy_alloc(lqcd_ctx *ctx, int nrhs) {
  if (!ctx->sloppy) ctx->sloppy = new SloppyState();
  SloppyState *s = ctx->sloppy;
  if (s->cap >= nrhs) return LQCD_OK;
  cudaStreamSynchronize(0);
  cudaDeviceSynchronize();
  cudaFree(s->sd);
  cudaFree(s->sn);
  cudaFree(s->f32);
  cudaFree(s->r64);
  cudaFree(s->small);
  s->sd = nullptr; s->sn = nullptr; s->f32 = nullptr; s->r64 = nullptr; s->small = nullptr;
  s->cap = 0;
  const Geom &g = ctx->geom;
  size_t vh = g.Vh;
  int nbx = (g.Vh + ST - 1) / ST;
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->sd, 7 * (size_t)nrhs * 3 * vh * sizeof(uint4)));
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->sn, 7 * (size_t)nrhs * vh * sizeof(float)));
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->f32, 5 * (size_t)nrhs * 6 * vh * sizeof(float4)));
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->r64, (size_t)nrhs * g.V * 12 * sizeof(double2)));
  s->small_bytes = small_layout(nullptr, nrhs, nbx).size();
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->small, s->small_bytes));
  if (!s->h_counts) LQCD_CUDA_TRY(ctx, cudaMallocHost(&s->h_counts, 16 * sizeof(int)));
  s->cap = nrhs;
  return LQCD_OK;
}

int fp64_residual_into(lqcd_ctx *ctx, const double2 *b, const double2 *x, double2 *res, int nrhs, double *rr,
                       double *bb, cudaStream_t st);

template <class S>
struct SlopFields {
  S r, rhat, p, v, s, t, tmp;
};

template <class S> S make_sfield(SloppyState *st, int f, int cap, int vh);
template <> F16F make_sfield<F16F>(SloppyState *st, int f, int cap, int vh) {
  F16F x;
  x.d = st->sd + (size_t)f * cap * 3 * vh;
  x.n = st->sn + (size_t)f * cap * vh;
  x.vh = vh;
  return x;
}
template <> BF16F make_sfield<BF16F>(SloppyState *st, int f, int cap, int vh) {
  BF16F x;
  x.d = st->sd + (size_t)f * cap * 3 * vh;
  x.vh = vh;
  return x;
}

template <class S>
static int mixed_block(lqcd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const lqcd_solver_params &p,
                       lqcd_solve_stats *stats, cudaStream_t st, double t0) {
  int rc = sloppy_alloc(ctx, nrhs);
  if (rc) return rc;
  SloppyState *ss = ctx->sloppy;
  const Geom &g = ctx->geom;
  const int vh = g.Vh, cap = ss->cap;
  const int nbx = (vh + ST - 1) / ST;
  const float kappa = (float)ctx->kappa;
  const float k2 = (float)(ctx->kappa * ctx->kappa);
  const int G = num_sms(ctx->device) * 8;
  const double delta = p.delta > 0 ? p.delta : 0.1;
  const double floor2 = 4e-12;  // (2e-6)^2: inner FP32 target floor, relative to |b_inner|^2

  // measurement of the dominant kernel (sloppy hopping term), when enabled
  unsigned long long *prof = ctx->prof_on ? ctx->d_prof : nullptr;
  if (ctx->prof_on) ctx->prof_prec = p.precision;
  auto ev_begin = [&]() {
    if (!ctx->prof_on) return;
    while (ctx->prof_used + 2 > ctx->prof_ev.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { ctx->prof_on = false; return; }
      ctx->prof_ev.push_back(e);
    }
    cudaEventRecord(ctx->prof_ev[ctx->prof_used], st);
  };
  auto ev_end = [&]() {
    if (!ctx->prof_on) return;
    cudaEventRecord(ctx->prof_ev[ctx->prof_used + 1], st);
    ctx->prof_used += 2;
    ctx->prof_hop_launches++;
  };

  SlopFields<S> F;
  F.r = make_sfield<S>(ss, 0, cap, vh);
  F.rhat = make_sfield<S>(ss, 1, cap, vh);
  F.p = make_sfield<S>(ss, 2, cap, vh);
  F.v = make_sfield<S>(ss, 3, cap, vh);
  F.s = make_sfield<S>(ss, 4, cap, vh);
  F.t = make_sfield<S>(ss, 5, cap, vh);
  F.tmp = make_sfield<S>(ss, 6, cap, vh);
  auto f32 = [&](int k) { F32F f; f.d = ss->f32 + (size_t)k * cap * 6 * vh; f.vh = vh; return f; };
  F32F x32 = f32(0), b32 = f32(1), r32 = f32(2), t32 = f32(3), o32 = f32(4);

  SmallBufs sb = small_layout(ss->small, cap, nbx);
  SState *sc = sb.sc;
  int *flags = sb.flags, *act_list = sb.act_list, *ru_list = sb.ru_list, *cyc_list = sb.cyc_list;
  int *counts = sb.counts;  // [0] active, [1] reliable update, [2] this cycle
  double *scale = sb.scale, *unscale = sb.unscale;
  D4S *part = sb.part;

  std::vector<double> rr(nrhs), bb(nrhs), prev_rel(nrhs, 1e300);
  std::vector<SState> hs(nrhs);
  std::vector<int> hl, bad(nrhs, 0);
  std::vector<double> hscale(nrhs), hun(nrhs);
  for (int k = 0; k < nrhs; ++k) {
    hs[k] = SState{};
    stats[k] = lqcd_solve_stats{0, LQCD_OK, 0.0, 0, 0};
  }
  LQCD_CUDA_TRY(ctx, cudaMemsetAsync(x, 0, (size_t)nrhs * g.V * 12 * sizeof(double2), st));
  const int max_cycles = 10;
  bool timed_out = false;

#define WL(list_ptr, count_ptr) list_ptr, count_ptr
  for (int cycle = 0; cycle <= max_cycles; ++cycle) {
    rc = fp64_residual_into(ctx, b, x, ss->r64, nrhs, rr.data(), bb.data(), st);
    if (rc) return rc;
    hl.clear();
    for (int k = 0; k < nrhs; ++k) {
      double rel = bb[k] > 0 ? std::sqrt(rr[k] / bb[k]) : 0.0;
      stats[k].true_rel_residual = rel;
      stats[k].iterations = hs[k].iters;
      stats[k].reliable_updates = hs[k].ru_count;
      stats[k].restarts = cycle > 0 ? cycle - 1 : 0;
      int status = hs[k].status;
      if (status == LQCD_OK && !std::isfinite(rel)) status = LQCD_ERR_NONFINITE;
      if (status == LQCD_OK && rel > p.tol) {
        if (timed_out) status = LQCD_ERR_TIMEOUT;
        else if (cycle == max_cycles || hs[k].iters >= p.max_iter) status = LQCD_ERR_NOT_CONVERGED;
        else if (rel > 0.5 * prev_rel[k]) {
          if (++bad[k] >= 3) status = LQCD_ERR_NOT_CONVERGED;  // refinement no longer reduces the residual
        }
      }
      prev_rel[k] = rel;
      stats[k].status = status;
      hs[k].status = status;
      if (status == LQCD_OK && rel > p.tol) {
        hl.push_back(k);
        hscale[k] = 1.0 / std::sqrt(rr[k]);
        hun[k] = std::sqrt(rr[k]);
        hs[k].target2 = 0.25 * p.tol * p.tol * bb[k] / rr[k];
        hs[k].ru_count = hs[k].ru_count;
      } else {
        hscale[k] = 0.0;
        hun[k] = 0.0;
      }
    }
    if (hl.empty() || timed_out) break;
    int ncyc = (int)hl.size();
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(cyc_list, hl.data(), ncyc * sizeof(int), cudaMemcpyHostToDevice, st));
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(counts + 2, &ncyc, sizeof(int), cudaMemcpyHostToDevice, st));
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(scale, hscale.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(unscale, hun.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sc, hs.data(), nrhs * sizeof(SState), cudaMemcpyHostToDevice, st));
    // inner right-hand side: b32 = scale (r_e + kappa H_eo r_o), o32 = scale r_o
    KL k_cvt64to32<<<G, ST, 0, st>>>(g, 0, ss->r64, b32, scale, WL(cyc_list, counts + 2), nbx);
    KL k_cvt64to32<<<G, ST, 0, st>>>(g, 1, ss->r64, o32, scale, WL(cyc_list, counts + 2), nbx);
    KL k_hop_s<F32F, F32F, true, EPI_AXPY><<<G, ST, 0, st>>>(g, 0, ctx->U32, o32, b32, b32, b32, 1.f, 0.f, kappa,
                                                            WL(cyc_list, counts + 2), nullptr, nbx, nullptr);
    KL k_blas_copy<S><<<G, ST, 0, st>>>(vh, b32, F.r, F.r, false, x32, true, WL(cyc_list, counts + 2), part, nbx);
    KL k_sfin_init<<<ncyc, 32, 0, st>>>(sc, flags, WL(cyc_list, counts + 2), part, nbx);
    // floor of the inner target relative to |b32|^2
    LQCD_LAUNCH_CHECK(ctx, "mixed: cycle setup");
    {
      // apply the floor: target2 = max(target2, floor2 * |b32|^2)
      std::vector<SState> tmp(nrhs);
      LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(tmp.data(), sc, nrhs * sizeof(SState), cudaMemcpyDeviceToHost, st));
      LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
      std::vector<int> fl(nrhs, 0);
      for (int k : hl) {
        tmp[k].target2 = std::max(tmp[k].target2, floor2 * tmp[k].rr);
        fl[k] = (tmp[k].status == LQCD_OK && tmp[k].rr > tmp[k].target2) ? FLAG_ACTIVE : 0;
      }
      LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sc, tmp.data(), nrhs * sizeof(SState), cudaMemcpyHostToDevice, st));
      LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(flags, fl.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
      LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    }
    KL k_build_lists<<<1, 1024, 0, st>>>(nrhs, flags, act_list, counts, ru_list, counts + 1);
    // ---------------------------------------------------------- inner loop
    bool any = true;
    while (any) {
      for (int it = 0; it < 4; ++it) {
        KL k_blas_p<S><<<G, ST, 0, st>>>(vh, sc, F.r, F.rhat, F.p, F.v, WL(act_list, counts), nbx);
        ev_begin();
        KL k_hop_s<S, S, false, EPI_PLAIN><<<G, ST, 0, st>>>(g, 1, ctx->U16, F.p, F.tmp, F.tmp, F.tmp, 0.f, 0.f, 1.f,
                                                          WL(act_list, counts), nullptr, nbx, prof);
        ev_end();
        ev_begin();
        KL k_hop_s<S, S, false, EPI_DOTR><<<G, ST, 0, st>>>(g, 0, ctx->U16, F.tmp, F.v, F.p, F.rhat, 1.f, 0.f, -k2,
                                                         WL(act_list, counts), part, nbx, prof);
        ev_end();
        KL k_sfin_alpha<<<nrhs, 32, 0, st>>>(sc, WL(act_list, counts), part, nbx);
        KL k_blas_s<S><<<G, ST, 0, st>>>(vh, sc, F.r, F.v, F.s, WL(act_list, counts), nbx);
        ev_begin();
        KL k_hop_s<S, S, false, EPI_PLAIN><<<G, ST, 0, st>>>(g, 1, ctx->U16, F.s, F.tmp, F.tmp, F.tmp, 0.f, 0.f, 1.f,
                                                          WL(act_list, counts), nullptr, nbx, prof);
        ev_end();
        ev_begin();
        KL k_hop_s<S, S, false, EPI_TS><<<G, ST, 0, st>>>(g, 0, ctx->U16, F.tmp, F.t, F.s, F.s, 1.f, 0.f, -k2,
                                                       WL(act_list, counts), part, nbx, prof);
        ev_end();
        KL k_sfin_omega<<<nrhs, 32, 0, st>>>(sc, WL(act_list, counts), part, nbx);
        KL k_blas_xr<S><<<G, ST, 0, st>>>(vh, sc, x32, F.p, F.s, F.t, F.r, F.rhat, WL(act_list, counts), part, nbx);
        KL k_sfin_conv<<<nrhs, 32, 0, st>>>(sc, flags, WL(act_list, counts), part, nbx, delta * delta, p.max_iter);
        KL k_build_lists<<<1, 1024, 0, st>>>(nrhs, flags, act_list, counts, ru_list, counts + 1);
        // reliable update in FP32: r32 = b32 - x32 + kappa^2 H_eo H_oe x32
        KL k_hop_s<F32F, F32F, true, EPI_PLAIN><<<G, ST, 0, st>>>(g, 1, ctx->U32, x32, t32, t32, t32, 0.f, 0.f, 1.f,
                                                               WL(ru_list, counts + 1), nullptr, nbx, nullptr);
        KL k_hop_s<F32F, F32F, true, EPI_RES><<<G, ST, 0, st>>>(g, 0, ctx->U32, t32, r32, b32, x32, 1.f, -1.f, k2,
                                                             WL(ru_list, counts + 1), part, nbx, nullptr);
        KL k_sfin_ru<<<nrhs, 32, 0, st>>>(sc, flags, WL(ru_list, counts + 1), part, nbx, p.max_iter);
        KL k_build_lists<<<1, 1024, 0, st>>>(nrhs, flags, act_list, counts, ru_list, counts + 1);
        KL k_blas_copy<S><<<G, ST, 0, st>>>(vh, r32, F.r, F.rhat, true, x32, false, WL(ru_list, counts + 1), part, nbx);
        KL k_sfin_ru2<<<nrhs, 32, 0, st>>>(sc, flags, WL(ru_list, counts + 1), part, nbx);
        KL k_build_lists<<<1, 1024, 0, st>>>(nrhs, flags, act_list, counts, ru_list, counts + 1);
      }
      LQCD_LAUNCH_CHECK(ctx, "mixed: iteration");
      LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(ss->h_counts, counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
      LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
      any = ss->h_counts[0] > 0;
      if (any && p.timeout_ms > 0 && wall_ms() - t0 > p.timeout_ms) {
        timed_out = true;
        break;
      }
    }
    // odd half of the correction: e_o = o32 + kappa H_oe x32; x += |r| e
    KL k_hop_s<F32F, F32F, true, EPI_AXPY><<<G, ST, 0, st>>>(g, 1, ctx->U32, x32, o32, o32, o32, 1.f, 0.f, kappa,
                                                            WL(cyc_list, counts + 2), nullptr, nbx, nullptr);
    KL k_accum64<<<G, ST, 0, st>>>(g, 0, x32, x, unscale, WL(cyc_list, counts + 2), nbx);
    KL k_accum64<<<G, ST, 0, st>>>(g, 1, o32, x, unscale, WL(cyc_list, counts + 2), nbx);
    LQCD_LAUNCH_CHECK(ctx, "mixed: correction");
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(hs.data(), sc, nrhs * sizeof(SState), cudaMemcpyDeviceToHost, st));
    LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    for (int k = 0; k < nrhs; ++k)
      if (std::find(hl.begin(), hl.end(), k) == hl.end()) hs[k].status = stats[k].status;
  }
#undef WL
  return LQCD_OK;
}

int mixed_solve(lqcd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const lqcd_solver_params &p,
                lqcd_solve_stats *stats, cudaStream_t st) {
  int blk = p.rhs_block > 0 ? p.rhs_block : nrhs;
  if (blk > 4096) blk = 4096;
  double t0 = wall_ms();
  size_t full = (size_t)ctx->geom.V * 12;
  int worst = LQCD_OK;
  for (int k0 = 0; k0 < nrhs; k0 += blk) {
    int nk = std::min(blk, nrhs - k0);
    int rc = p.precision == LQCD_PREC_MIXED_FP16
                 ? mixed_block<F16F>(ctx, b + k0 * full, x + k0 * full, nk, p, stats + k0, st, t0)
                 : mixed_block<BF16F>(ctx, b + k0 * full, x + k0 * full, nk, p, stats + k0, st, t0);
    if (rc) return rc;
    for (int k = 0; k < nk; ++k)
      if (worst == LQCD_OK && stats[k0 + k].status != LQCD_OK) worst = stats[k0 + k].status;
  }
  if (worst != LQCD_OK) set_error(ctx, worst, "lqcd_solve_batch: some right-hand sides did not converge");
  return worst;
}

}  // namespace lqcd
