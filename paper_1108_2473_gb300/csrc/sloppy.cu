// Mixed-precision many-RHS solver (Sec. II: mixed-precision BiCGstab for the
// all-to-all inversions; Sec. III: stop on the true relative residual
// |M x - b| / |b| of the full operator).
//
// Three precision levels:
//   * sloppy  -- Krylov vectors stored as FP16 (with one FP32 norm per site
//               and RHS, values scaled into [-1, 1]) or as BF16; links FP16;
//               all arithmetic in FP32;
//   * FP32    -- the iterate x and the reliable-update residual
//               r = b - D_hat x, with FP32 reconstruct-12 links;
//   * FP64-class -- the outer defect correction: r = b - D x on the full
//               lattice in double-float arithmetic (a 48-bit significand on the
//               FP32 units), inner solve D e = r, x += e, until |r| / |b| <= tol.
//
// Sloppy vectors hold right-hand sides in pairs (RHS 2P and 2P+1): each
// 16-bit pair is the same real of both members, so after conversion every
// operation of the hopping term and of the BLAS updates is one packed FP32x2
// instruction (fma.rn.f32x2 / add / mul) working on both members at once, and
// a link load, its conversion and the neighbour indexing serve two RHS.
// The sloppy links are FP16, all 18 reals, every real stored twice, so that
// one conversion yields the (u, u) operand of the packed products (this hop
// is bound by the FMA pipe, where a reconstruction would cost more than the
// extra link bytes; the FP32 reliable-update hop, bound by its loads, keeps
// reconstruct-12 links).
//
// Layouts (parity-compact, per pair / per RHS):
//   sloppy: [P][6][Vh] uint4 (24 16-bit pairs) + FP16 norms [P][Vh] float2
//   FP32:   [rhs][6][Vh] float4
//   links:  FP16 [2 parity][4 mu][5][Vh] uint4 (18 reals, duplicated);
//           FP32 [2][4][3][Vh] float4 (rows 0-1)
// A spinor's 24 reals are ordered ((spin * 3 + colour) * 2 + re/im).
//
// Kernels walk device-side lists (of RHS or of pairs): work item w =
// (list[w / nbx], site block w % nbx), grid-stride over a fixed grid, so
// converged right-hand sides cost nothing.  Every reduction is written as one
// partial per (RHS, site block) and summed by one warp per RHS in a fixed
// order: a right-hand side's arithmetic does not depend on its batch mates.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <memory>
#include <type_traits>
#include <vector>

#include "internal.cuh"
#include "df.cuh"
#include "fpconv.cuh"

#include "sloppy.cuh"
#include "tile_api.cuh"

namespace lqcd {

// ============================================================ conversions
__device__ __forceinline__ float2 h2f(unsigned w) {
  __half2 h = *reinterpret_cast<__half2 *>(&w);
  return __half22float2(h);
}
__device__ __forceinline__ unsigned f2h(float2 v) {
  __half2 h = __float22half2_rn(v);
  return *reinterpret_cast<unsigned *>(&h);
}
__device__ __forceinline__ float2 b2f(unsigned w) {
  // bf16 -> f32 is exact: the bf16 bits are the high half of the f32
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ unsigned f2b(float2 v) {
  __nv_bfloat162 h = __float22bfloat162_rn(v);
  return *reinterpret_cast<unsigned *>(&h);
}

// packed FP32x2 arithmetic (one instruction for both members of a pair)
__device__ __forceinline__ float2 A2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 M2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 F2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 S2(float2 a, float2 b) {  // a - b, rounded once
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 sel2(bool lo, bool hi, float2 a, float2 b) {  // per member: a where set
  return make_float2(lo ? a.x : b.x, hi ? a.y : b.y);
}

// ============================================================ FP32 field
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

// ============================================================ pair fields
// raw (unscaled) pairs and the norm pair that scales them (1, 1 for BF16)
__device__ __forceinline__ void load_raw(const F16P &f, int P, int i, float2 v[24], float2 &nrm) {
  const uint4 *p = f.d + (size_t)P * 6 * f.vh + i;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    uint4 q = p[(size_t)k * f.vh];
    v[4 * k] = h2f(q.x);
    v[4 * k + 1] = h2f(q.y);
    v[4 * k + 2] = h2f(q.z);
    v[4 * k + 3] = h2f(q.w);
  }
  nrm = f.n[(size_t)P * f.vh + i];
}
__device__ __forceinline__ void load_raw(const BF16P &f, int P, int i, float2 v[24], float2 &nrm) {
  const uint4 *p = f.d + (size_t)P * 6 * f.vh + i;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    uint4 q = p[(size_t)k * f.vh];
    v[4 * k] = b2f(q.x);
    v[4 * k + 1] = b2f(q.y);
    v[4 * k + 2] = b2f(q.z);
    v[4 * k + 3] = b2f(q.w);
  }
  nrm = make_float2(1.f, 1.f);
}
__device__ __forceinline__ void load_scaled(const F16P &f, int P, int i, float2 v[24]) {
  float2 nrm;
  load_raw(f, P, i, v, nrm);
#pragma unroll
  for (int k = 0; k < 24; ++k) v[k] = M2(v[k], nrm);
}
__device__ __forceinline__ void load_scaled(const BF16P &f, int P, int i, float2 v[24]) {
  float2 nrm;
  load_raw(f, P, i, v, nrm);
}

// FP16: the words to store and the per-member norms
__device__ __forceinline__ void encode(const F16P &, const float2 v[24], unsigned w[24], float2 &m) {
  m = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 24; ++k) {
    m.x = fmaxf(m.x, fabsf(v[k].x));
    m.y = fmaxf(m.y, fabsf(v[k].y));
  }
  float2 inv = make_float2(m.x > 0.f ? 1.f / m.x : 0.f, m.y > 0.f ? 1.f / m.y : 0.f);
#pragma unroll
  for (int k = 0; k < 24; ++k) w[k] = f2h(M2(v[k], inv));
}
__device__ __forceinline__ void encode(const BF16P &, const float2 v[24], unsigned w[24], float2 &m) {
  m = make_float2(1.f, 1.f);
#pragma unroll
  for (int k = 0; k < 24; ++k) w[k] = f2b(v[k]);
}
__device__ __forceinline__ void write_norm(const F16P &f, int P, int i, float2 m) { f.n[(size_t)P * f.vh + i] = m; }
__device__ __forceinline__ void write_norm(const BF16P &, int, int, float2) {}
__device__ __forceinline__ float2 read_norm(const F16P &f, int P, int i) { return f.n[(size_t)P * f.vh + i]; }
__device__ __forceinline__ float2 read_norm(const BF16P &, int, int) { return make_float2(1.f, 1.f); }

template <class SP>
__device__ __forceinline__ void store_pair(const SP &f, int P, int i, const float2 v[24]) {
  unsigned w[24];
  float2 m;
  encode(f, v, w, m);
  uint4 *p = f.d + (size_t)P * 6 * f.vh + i;
#pragma unroll
  for (int k = 0; k < 6; ++k) p[(size_t)k * f.vh] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
  write_norm(f, P, i, m);
}

// store only the members flagged in (lo, hi); the other member's bits are kept
template <class SP>
__device__ __forceinline__ void store_members(const SP &f, int P, int i, const float2 v[24], bool lo, bool hi) {
  if (lo && hi) {
    store_pair(f, P, i, v);
    return;
  }
  if (!lo && !hi) return;
  unsigned w[24];
  float2 m;
  encode(f, v, w, m);
  const unsigned keep = lo ? 0xffff0000u : 0x0000ffffu;
  uint4 *p = f.d + (size_t)P * 6 * f.vh + i;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    uint4 o = p[(size_t)k * f.vh];
    uint4 q;
    q.x = (o.x & keep) | (w[4 * k] & ~keep);
    q.y = (o.y & keep) | (w[4 * k + 1] & ~keep);
    q.z = (o.z & keep) | (w[4 * k + 2] & ~keep);
    q.w = (o.w & keep) | (w[4 * k + 3] & ~keep);
    p[(size_t)k * f.vh] = q;
  }
  float2 om = read_norm(f, P, i);
  write_norm(f, P, i, make_float2(lo ? m.x : om.x, hi ? m.y : om.y));
}

// ======================================================= FP32 hopping term
// reconstruct-12 FP32 link: rows 0, 1 stored, row 2 = (row0 x row1)^*
__device__ __forceinline__ void load_link32(const float4 *U, int p, int mu, int i, int vh, float2 u[3][3]) {
  size_t base = ((size_t)(p * 4 + mu) * 3) * vh + i;
  float4 q0 = U[base], q1 = U[base + vh], q2 = U[base + 2 * (size_t)vh];
  u[0][0] = make_float2(q0.x, q0.y);
  u[0][1] = make_float2(q0.z, q0.w);
  u[0][2] = make_float2(q1.x, q1.y);
  u[1][0] = make_float2(q1.z, q1.w);
  u[1][1] = make_float2(q2.x, q2.y);
  u[1][2] = make_float2(q2.z, q2.w);
  float2 c0 = csub(cmul(u[0][1], u[1][2]), cmul(u[0][2], u[1][1]));
  float2 c1 = csub(cmul(u[0][2], u[1][0]), cmul(u[0][0], u[1][2]));
  float2 c2 = csub(cmul(u[0][0], u[1][1]), cmul(u[0][1], u[1][0]));
  u[2][0] = make_float2(c0.x, -c0.y);
  u[2][1] = make_float2(c1.x, -c1.y);
  u[2][2] = make_float2(c2.x, -c2.y);
}

// FP32 hop in direction MU for NR right-hand sides of one site: each link is
// loaded and reconstructed once and applied to all of them
template <int MU, int NR>
__device__ __forceinline__ void hop_dir32n(const Geom &g, int p_out, const int c[4], int i, const F32F &in,
                                           const int rhs[NR], const float4 *links, float2 acc[NR][4][3]) {
  float2 u[3][3];
  {  // forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
    const int sn = site_of(g, cn);
    load_link32(links, p_out, MU, i, g.Vh, u);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      float2 v[12], h[2][3], x[2][3], ps[4][3];
      in.load(rhs[r], sn >> 1, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) ps[k / 3][k % 3] = v[k];
      spin_project<MU, -1>(ps, h);
      su3_mul<false>(u, h, x);
      if (MU == 3 && c[3] == g.L[3] - 1) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) x[a][b] = make_float2(-x[a][b].x, -x[a][b].y);
      }
      spin_accum<MU, -1>(acc[r], x);
    }
  }
  {  // backward: (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu)
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
    const int sn = site_of(g, cn);
    load_link32(links, 1 - p_out, MU, sn >> 1, g.Vh, u);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      float2 v[12], h[2][3], x[2][3], ps[4][3];
      in.load(rhs[r], sn >> 1, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) ps[k / 3][k % 3] = v[k];
      spin_project<MU, +1>(ps, h);
      su3_mul<true>(u, h, x);
      if (MU == 3 && c[3] == 0) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) x[a][b] = make_float2(-x[a][b].x, -x[a][b].y);
      }
      spin_accum<MU, +1>(acc[r], x);
    }
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// fixed-order block reduction of two D4S (all ST threads participate)
__device__ __forceinline__ void block_reduce_store2(D4S v0, D4S v1, D4S *dst0, D4S *dst1) {
  __shared__ D4S sh[2][ST / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v0.a = warp_sum_d(v0.a);
  v0.b = warp_sum_d(v0.b);
  v0.c = warp_sum_d(v0.c);
  v0.d = warp_sum_d(v0.d);
  v1.a = warp_sum_d(v1.a);
  v1.b = warp_sum_d(v1.b);
  v1.c = warp_sum_d(v1.c);
  v1.d = warp_sum_d(v1.d);
  if (lane == 0) {
    sh[0][w] = v0;
    sh[1][w] = v1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    D4S t = sh[threadIdx.x][0];
#pragma unroll
    for (int k = 1; k < ST / 32; ++k) {
      t.a += sh[threadIdx.x][k].a;
      t.b += sh[threadIdx.x][k].b;
      t.c += sh[threadIdx.x][k].c;
      t.d += sh[threadIdx.x][k].d;
    }
    *(threadIdx.x ? dst1 : dst0) = t;
  }
  __syncthreads();
}

// As block_reduce_store2 for each group of ST threads of a block of PPB * ST
// threads; groups with store == false only take part in the barriers.
template <int PPB>
__device__ __forceinline__ void group_reduce_store2(D4S v0, D4S v1, D4S *dst0, D4S *dst1, bool store) {
  __shared__ D4S sh[PPB][2][ST / 32];
  const int grp = threadIdx.x / ST, tid = threadIdx.x % ST;
  const int lane = tid & 31, w = tid >> 5;
  v0.a = warp_sum_d(v0.a);
  v0.b = warp_sum_d(v0.b);
  v0.c = warp_sum_d(v0.c);
  v0.d = warp_sum_d(v0.d);
  v1.a = warp_sum_d(v1.a);
  v1.b = warp_sum_d(v1.b);
  v1.c = warp_sum_d(v1.c);
  v1.d = warp_sum_d(v1.d);
  if (lane == 0) {
    sh[grp][0][w] = v0;
    sh[grp][1][w] = v1;
  }
  __syncthreads();
  if (tid < 2 && store) {
    D4S t = sh[grp][tid][0];
#pragma unroll
    for (int k = 1; k < ST / 32; ++k) {
      t.a += sh[grp][tid][k].a;
      t.b += sh[grp][tid][k].b;
      t.c += sh[grp][tid][k].c;
      t.d += sh[grp][tid][k].d;
    }
    *(tid ? dst1 : dst0) = t;
  }
  __syncthreads();
}

// FP32 hopping term: out = cA A + cB B + cH (H in) at the sites of parity p_out.
// EPI_PLAIN: A, B unused.  EPI_AXPY: B unused.  EPI_RES: partial |out|^2.
// The FP32 hopping term on two right-hand sides per thread (list entries 2j and
// 2j + 1; with an odd count the last thread recomputes entry 2j for its second
// slot and stores nothing for it), which halves the link loads and the
// reconstruction of the third link row per right-hand side.
template <int EPI>
__global__ void __launch_bounds__(ST, 4) k_hop32x2(Geom g, int p_out, const float4 *links, F32F in, F32F out, F32F A,
                                                F32F B, float cA, float cB, float cH, const int *list,
                                                const int *count, D4S *part, int nbx) {
  const int cnt = *count;
  const int n_items = (cnt + 1) / 2 * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int j = (w / nbx) * 2, sb = w % nbx;
    const bool two = j + 1 < cnt;
    const int rhs[2] = {list[j], two ? list[j + 1] : list[j]};
    const int i = sb * ST + threadIdx.x;
    D4S red[2] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    if (i < g.Vh) {
      int c[4];
      coords_of(g, p_out, i, c);
      float2 acc[2][4][3];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) acc[r][a][b] = make_float2(0.f, 0.f);
      hop_dir32n<0, 2>(g, p_out, c, i, in, rhs, links, acc);
      hop_dir32n<1, 2>(g, p_out, c, i, in, rhs, links, acc);
      hop_dir32n<2, 2>(g, p_out, c, i, in, rhs, links, acc);
      hop_dir32n<3, 2>(g, p_out, c, i, in, rhs, links, acc);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float2 o[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = make_float2(cH * acc[r][k / 3][k % 3].x, cH * acc[r][k / 3][k % 3].y);
        if (EPI != EPI_PLAIN) {
          float2 a[12];
          A.load(rhs[r], i, a);
#pragma unroll
          for (int k = 0; k < 12; ++k) o[k] = make_float2(fmaf(cA, a[k].x, o[k].x), fmaf(cA, a[k].y, o[k].y));
        }
        if (EPI == EPI_RES) {
          float2 b[12];
          B.load(rhs[r], i, b);
#pragma unroll
          for (int k = 0; k < 12; ++k) o[k] = make_float2(fmaf(cB, b[k].x, o[k].x), fmaf(cB, b[k].y, o[k].y));
        }
        if (r == 0 || two) out.store(rhs[r], i, o);
        if (EPI == EPI_RES) {
          float nn = 0.f;
#pragma unroll
          for (int k = 0; k < 12; ++k) nn += o[k].x * o[k].x + o[k].y * o[k].y;
          red[r].c = nn;
        }
      }
    }
    if (EPI == EPI_RES)
      block_reduce_store2(red[0], red[1], part + (size_t)rhs[0] * nbx + sb, part + (size_t)rhs[1] * nbx + sb);
  }
}

// ====================================================== pair hopping term
// FP16 link for both members: all nine entries from memory as (u, u) pairs,
// layout [2 parity][4 mu][5][Vh] uint4 (the fifth uint4 holds entry (2,2) only).
__device__ __forceinline__ void load_link_pair(const uint4 *U, int p, int mu, int i, int vh, CP u[3][3]) {
  const size_t base = ((size_t)(p * 4 + mu) * 5) * vh + i;
  uint4 q[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) q[k] = U[base + (size_t)k * vh];
  const unsigned w[18] = {q[0].x, q[0].y, q[0].z, q[0].w, q[1].x, q[1].y, q[1].z, q[1].w, q[2].x,
                          q[2].y, q[2].z, q[2].w, q[3].x, q[3].y, q[3].z, q[3].w, q[4].x, q[4].y};
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k / 3][k % 3] = CP{h2f(w[2 * k]), h2f(w[2 * k + 1])};
}

// Rows 0 and 1 of the same FP16 link (the first three uint4 of its layout);
// row 2 rebuilt as conj(row 0 x row 1), u[2][c] = conj(u[0][a] u[1][b] - u[0][b] u[1][a])
// for (a, b, c) cyclic, which holds for SU(3) links (the mixed solver requires
// them): two of the five loads per link traded for 30 packed FP32 operations.
__device__ __forceinline__ void load_link_pair_r12(const uint4 *U, int p, int mu, int i, int vh, CP u[3][3]) {
  const size_t base = ((size_t)(p * 4 + mu) * 5) * vh + i;
  uint4 q[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) q[k] = U[base + (size_t)k * vh];
  const unsigned w[12] = {q[0].x, q[0].y, q[0].z, q[0].w, q[1].x, q[1].y,
                          q[1].z, q[1].w, q[2].x, q[2].y, q[2].z, q[2].w};
#pragma unroll
  for (int k = 0; k < 6; ++k) u[k / 3][k % 3] = CP{h2f(w[2 * k]), h2f(w[2 * k + 1])};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    const CP &x = u[0][a], &y = u[1][b], &v = u[0][b], &z = u[1][a];
    // Re = x.re y.re - x.im y.im - v.re z.re + v.im z.im; -Im = v.re z.im + v.im z.re - x.re y.im - x.im y.re
    const float2 re = S2(F2(x.re, y.re, M2(v.im, z.im)), F2(x.im, y.im, M2(v.re, z.re)));
    const float2 mim = S2(F2(v.re, z.im, M2(v.im, z.re)), F2(x.re, y.im, M2(x.im, y.re)));
    u[2][c] = CP{re, mim};
  }
}

// a + s i b and a + s b on pairs
template <int S> __device__ __forceinline__ CP cp_addi(const CP &a, const CP &b) {
  return S > 0 ? CP{S2(a.re, b.im), A2(a.im, b.re)} : CP{A2(a.re, b.im), S2(a.im, b.re)};
}
template <int S> __device__ __forceinline__ CP cp_addpm(const CP &a, const CP &b) {
  return S > 0 ? CP{A2(a.re, b.re), A2(a.im, b.im)} : CP{S2(a.re, b.re), S2(a.im, b.im)};
}

// Spin projection (1 + SIGMA gamma_mu) of the neighbour spinor, as in
// spin_project (internal.cuh) but on pairs; then the norm pair scales h.
template <int MU, int SIGMA>
__device__ __forceinline__ void project_pair(const float2 v[24], CP h[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const CP p0{v[(0 * 3 + c) * 2], v[(0 * 3 + c) * 2 + 1]};
    const CP p1{v[(1 * 3 + c) * 2], v[(1 * 3 + c) * 2 + 1]};
    const CP p2{v[(2 * 3 + c) * 2], v[(2 * 3 + c) * 2 + 1]};
    const CP p3{v[(3 * 3 + c) * 2], v[(3 * 3 + c) * 2 + 1]};
    CP h0, h1;
    if (MU == 0) {
      h0 = cp_addi<SIGMA>(p0, p3);
      h1 = cp_addi<SIGMA>(p1, p2);
    } else if (MU == 1) {
      h0 = cp_addpm<-SIGMA>(p0, p3);
      h1 = cp_addpm<SIGMA>(p1, p2);
    } else if (MU == 2) {
      h0 = cp_addi<SIGMA>(p0, p2);
      h1 = cp_addi<-SIGMA>(p1, p3);
    } else {
      h0 = cp_addpm<SIGMA>(p0, p2);
      h1 = cp_addpm<SIGMA>(p1, p3);
    }
    h[0][c] = h0;
    h[1][c] = h1;
  }
}

// (U h)_a or (U^+ h)_a for one spin row, packed
template <bool DAG>
__device__ __forceinline__ CP su3_row_pair(const CP u[3][3], const CP h[3], int a) {
  CP r;
  if (!DAG) {  // sum_b U[a][b] h[b]
    float2 rr = M2(u[a][0].re, h[0].re), ii = M2(u[a][0].im, h[0].im);
    rr = F2(u[a][1].re, h[1].re, rr);
    ii = F2(u[a][1].im, h[1].im, ii);
    rr = F2(u[a][2].re, h[2].re, rr);
    ii = F2(u[a][2].im, h[2].im, ii);
    r.re = S2(rr, ii);
    float2 im = M2(u[a][0].re, h[0].im);
    im = F2(u[a][0].im, h[0].re, im);
    im = F2(u[a][1].re, h[1].im, im);
    im = F2(u[a][1].im, h[1].re, im);
    im = F2(u[a][2].re, h[2].im, im);
    im = F2(u[a][2].im, h[2].re, im);
    r.im = im;
  } else {  // sum_b conj(U[b][a]) h[b]
    float2 re = M2(u[0][a].re, h[0].re);
    re = F2(u[0][a].im, h[0].im, re);
    re = F2(u[1][a].re, h[1].re, re);
    re = F2(u[1][a].im, h[1].im, re);
    re = F2(u[2][a].re, h[2].re, re);
    re = F2(u[2][a].im, h[2].im, re);
    r.re = re;
    float2 ri = M2(u[0][a].re, h[0].im), ir = M2(u[0][a].im, h[0].re);
    ri = F2(u[1][a].re, h[1].im, ri);
    ir = F2(u[1][a].im, h[1].re, ir);
    ri = F2(u[2][a].re, h[2].im, ri);
    ir = F2(u[2][a].im, h[2].re, ir);
    r.im = S2(ri, ir);
  }
  return r;
}

// acc += n * (spin reconstruction of U h), colour by colour (see spin_accum);
// n is the neighbour's norm pair (with the boundary sign), folded into the FMAs
template <int S> __device__ __forceinline__ CP cp_fma_pm(const CP &acc, const CP &x, float2 n, float2 nn) {
  return S > 0 ? CP{F2(n, x.re, acc.re), F2(n, x.im, acc.im)} : CP{F2(nn, x.re, acc.re), F2(nn, x.im, acc.im)};
}
template <int S> __device__ __forceinline__ CP cp_fma_i(const CP &acc, const CP &x, float2 n, float2 nn) {
  // acc + S i n x:  re -= S n x.im, im += S n x.re
  return S > 0 ? CP{F2(nn, x.im, acc.re), F2(n, x.re, acc.im)} : CP{F2(n, x.im, acc.re), F2(nn, x.re, acc.im)};
}
template <int MU, int SIGMA, bool DAG>
__device__ __forceinline__ void su3_accum_pair(const CP u[3][3], const CP h[2][3], float2 n, CP acc[4][3]) {
  const float2 nn = make_float2(-n.x, -n.y);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const CP x0 = su3_row_pair<DAG>(u, h[0], a);
    const CP x1 = su3_row_pair<DAG>(u, h[1], a);
    acc[0][a] = cp_fma_pm<1>(acc[0][a], x0, n, nn);
    acc[1][a] = cp_fma_pm<1>(acc[1][a], x1, n, nn);
    if (MU == 0) {
      acc[2][a] = cp_fma_i<-SIGMA>(acc[2][a], x1, n, nn);
      acc[3][a] = cp_fma_i<-SIGMA>(acc[3][a], x0, n, nn);
    } else if (MU == 1) {
      acc[2][a] = cp_fma_pm<SIGMA>(acc[2][a], x1, n, nn);
      acc[3][a] = cp_fma_pm<-SIGMA>(acc[3][a], x0, n, nn);
    } else if (MU == 2) {
      acc[2][a] = cp_fma_i<-SIGMA>(acc[2][a], x0, n, nn);
      acc[3][a] = cp_fma_i<SIGMA>(acc[3][a], x1, n, nn);
    } else {
      acc[2][a] = cp_fma_pm<SIGMA>(acc[2][a], x0, n, nn);
      acc[3][a] = cp_fma_pm<SIGMA>(acc[3][a], x1, n, nn);
    }
  }
}

template <int MU, class SP, bool R12 = false>
__device__ __forceinline__ void hop_dir_pair(const Geom &g, int p_out, const int c[4], int i, const SP &in, int P,
                                             const uint4 *links, CP acc[4][3]) {
  float2 v[24], nrm;
  CP h[2][3], u[3][3];
  {  // forward: (1 - gamma_mu) U_mu(x) psi(x + mu); the t-boundary sign rides on the norm
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
    const int sn = site_of(g, cn);
    load_raw(in, P, sn >> 1, v, nrm);
    if (MU == 3 && c[3] == g.L[3] - 1) nrm = make_float2(-nrm.x, -nrm.y);
    project_pair<MU, -1>(v, h);
    if (R12) load_link_pair_r12(links, p_out, MU, i, g.Vh, u);
    else load_link_pair(links, p_out, MU, i, g.Vh, u);
    su3_accum_pair<MU, -1, false>(u, h, nrm, acc);
  }
  {  // backward: (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu)
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
    const int sn = site_of(g, cn);
    load_raw(in, P, sn >> 1, v, nrm);
    if (MU == 3 && c[3] == 0) nrm = make_float2(-nrm.x, -nrm.y);
    project_pair<MU, +1>(v, h);
    if (R12) load_link_pair_r12(links, 1 - p_out, MU, sn >> 1, g.Vh, u);
    else load_link_pair(links, 1 - p_out, MU, sn >> 1, g.Vh, u);
    su3_accum_pair<MU, +1, true>(u, h, nrm, acc);
  }
}

// Epilogue of the pair hopping term at output site i of pair P: o = cH acc
// (+ cA a unless EPI_PLAIN), stored to out; EPI_DOTR: partials <B, o> per
// member; EPI_TS: partials <o, a> and |o|^2 per member (r0, r1 untouched for
// EPI_PLAIN).
template <class SP, int EPI>
__device__ __forceinline__ void pair_epilogue(const CP acc[4][3], const float2 a[24], float2 cA2, float2 cH2,
                                              const SP &out, const SP &B, int P, int i, D4S &r0, D4S &r1) {
  float2 o[24];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    o[2 * k] = M2(acc[k / 3][k % 3].re, cH2);
    o[2 * k + 1] = M2(acc[k / 3][k % 3].im, cH2);
  }
  if (EPI != EPI_PLAIN) {
#pragma unroll
    for (int k = 0; k < 24; ++k) o[k] = F2(cA2, a[k], o[k]);
  }
  store_pair(out, P, i, o);
  if (EPI == EPI_DOTR) {  // <B, out> = sum conj(B) out
    float2 rb[24];
    load_scaled(B, P, i, rb);
    float2 re = make_float2(0.f, 0.f), ip = re, im = re;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re = F2(rb[2 * k], o[2 * k], re);
      re = F2(rb[2 * k + 1], o[2 * k + 1], re);
      ip = F2(rb[2 * k], o[2 * k + 1], ip);
      im = F2(rb[2 * k + 1], o[2 * k], im);
    }
    const float2 imag = S2(ip, im);
    r0 = D4S{re.x, imag.x, 0, 0};
    r1 = D4S{re.y, imag.y, 0, 0};
  } else if (EPI == EPI_TS) {  // <out, A> and |out|^2
    float2 re = make_float2(0.f, 0.f), ip = re, im = re, nn = re;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re = F2(o[2 * k], a[2 * k], re);
      re = F2(o[2 * k + 1], a[2 * k + 1], re);
      ip = F2(o[2 * k], a[2 * k + 1], ip);
      im = F2(o[2 * k + 1], a[2 * k], im);
      nn = F2(o[2 * k], o[2 * k], nn);
      nn = F2(o[2 * k + 1], o[2 * k + 1], nn);
    }
    const float2 imag = S2(ip, im);
    r0 = D4S{re.x, imag.x, 0, nn.x};
    r1 = D4S{re.y, imag.y, 0, nn.y};
  }
}

// Sloppy hopping term on RHS pairs: out = cA A + cH (H in) at parity p_out.
// EPI_PLAIN: out = cH H in.  EPI_DOTR: partial <B, out> per member.
// EPI_TS: partials <out, A> and |out|^2 per member.
// A block of PPB * ST threads takes PPB active pairs on the same ST sites, so
// the links those sites read are fetched from L2 once per block and then hit
// in L1 for the other pairs.  R12: links from rows 0 and 1 (load_link_pair_r12).
template <class SP, int EPI, int MINB, int PPB, bool R12 = false>
__global__ void __launch_bounds__(ST * PPB, MINB) k_hop_pair(Geom g, int p_out, const uint4 *links, SP in, SP out,
                                                       SP A, SP B, float cA, float cH, const int *plist,
                                                       const int *pcount, D4S *part, int nbx, int nrhs,
                                                       unsigned long long *prof) {
  const int count = *pcount;
  const int n_items = (count + PPB - 1) / PPB * nbx;
  const float2 cA2 = make_float2(cA, cA), cH2 = make_float2(cH, cH);
  const int grp = threadIdx.x / ST, tid = threadIdx.x % ST;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int j = (w / nbx) * PPB + grp, sb = w % nbx;
    const bool valid = j < count;
    const int P = valid ? plist[j] : 0;
    const int i = sb * ST + tid;
    if (prof && tid == 0 && valid)
      atomicAdd(prof + EPI, (unsigned long long)min(ST, g.Vh - sb * ST) * (2 * P + 1 < nrhs ? 2 : 1));
    D4S r0 = {0, 0, 0, 0}, r1 = {0, 0, 0, 0};
    if (valid && i < g.Vh) {
      int c[4];
      coords_of(g, p_out, i, c);
      CP acc[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) acc[a][b] = CP{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      hop_dir_pair<0, SP, R12>(g, p_out, c, i, in, P, links, acc);
      hop_dir_pair<1, SP, R12>(g, p_out, c, i, in, P, links, acc);
      hop_dir_pair<2, SP, R12>(g, p_out, c, i, in, P, links, acc);
      hop_dir_pair<3, SP, R12>(g, p_out, c, i, in, P, links, acc);
      float2 a[24];
      if (EPI != EPI_PLAIN) load_scaled(A, P, i, a);
      pair_epilogue<SP, EPI>(acc, a, cA2, cH2, out, B, P, i, r0, r1);
    }
    if (EPI == EPI_DOTR || EPI == EPI_TS)
      group_reduce_store2<PPB>(r0, r1, part + (size_t)(2 * P) * nbx + sb, part + (size_t)(2 * P + 1) * nbx + sb,
                               valid);
  }
}

// ============================= pair hopping term, neighbour planes in shared memory
// On lattices whose (z, t) planes hold ST sites of one parity (Lx Ly / 2 = ST),
// the parity-local indices of a plane are one aligned block of ST, so a block
// of the pair kernel covers exactly one plane of output sites.  The eight
// neighbours of those sites lie in five planes of the other parity: the plane
// itself (the x and y neighbours, wrap-arounds included), z + 1, z - 1, t + 1
// and t - 1.  The block copies those five planes of its pair (and the plane of
// the A operand) into shared memory with cp.async, which holds no registers
// while the copies are in flight, then reads every neighbour spinor from shared
// memory.  Links are loaded from global memory as in k_hop_pair, and the
// arithmetic is that of k_hop_pair, term for term in the same order.
constexpr int PLANE_VARIANT = 6;                            // its hop variant number
constexpr int R12_VARIANT = 7;                              // variant 1 with reconstruct-12 links
constexpr int PL_SLOTS = 5;                                 // own, z + 1, z - 1, t + 1, t - 1
constexpr int PL_SMEM_PLAIN = PL_SLOTS * 6 * ST * 16;       // 60 KiB
constexpr int PL_SMEM_EPI = (PL_SLOTS + 1) * 6 * ST * 16;   // + the A operand's plane: 72 KiB

__host__ __device__ inline bool planes_fit(const Geom &g) { return g.Lxh * g.L[1] == ST; }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// the 24 packed values of the site at offset loc of plane slot `slot`
__device__ __forceinline__ void load_plane(const uint4 *sm, int slot, int loc, float2 v[24]) {
  const uint4 *p = sm + slot * 6 * ST + loc;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const uint4 q = p[k * ST];
    v[4 * k] = b2f(q.x);
    v[4 * k + 1] = b2f(q.y);
    v[4 * k + 2] = b2f(q.z);
    v[4 * k + 3] = b2f(q.w);
  }
}

template <int MU>
__device__ __forceinline__ void hop_dir_plane(const Geom &g, int p_out, const int c[4], int i, const uint4 *sm,
                                              const uint4 *links, CP acc[4][3]) {
  constexpr int FWD = MU < 2 ? 0 : (MU == 2 ? 1 : 3), BWD = MU < 2 ? 0 : (MU == 2 ? 2 : 4);
  float2 v[24], nrm;
  CP h[2][3], u[3][3];
  {  // forward: (1 - gamma_mu) U_mu(x) psi(x + mu); the t-boundary sign rides on the norm
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
    const int sn = site_of(g, cn);
    load_plane(sm, FWD, (sn >> 1) & (ST - 1), v);
    nrm = (MU == 3 && c[3] == g.L[3] - 1) ? make_float2(-1.f, -1.f) : make_float2(1.f, 1.f);
    project_pair<MU, -1>(v, h);
    load_link_pair(links, p_out, MU, i, g.Vh, u);
    su3_accum_pair<MU, -1, false>(u, h, nrm, acc);
  }
  {  // backward: (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu)
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
    const int sn = site_of(g, cn);
    load_plane(sm, BWD, (sn >> 1) & (ST - 1), v);
    nrm = (MU == 3 && c[3] == 0) ? make_float2(-1.f, -1.f) : make_float2(1.f, 1.f);
    project_pair<MU, +1>(v, h);
    load_link_pair(links, 1 - p_out, MU, sn >> 1, g.Vh, u);
    su3_accum_pair<MU, +1, true>(u, h, nrm, acc);
  }
}

// BF16 pairs only; one block of ST threads per (pair, plane) item, grid-stride
// over the items pair by pair (as k_hop_pair), at most three blocks per SM
// (72 KiB of shared memory each).  Requires planes_fit(g) and nbx = Lz Lt.
template <int EPI>
__global__ void __launch_bounds__(ST, 3) k_hop_pair_pl(Geom g, int p_out, const uint4 *links, BF16P in, BF16P out,
                                                       BF16P A, BF16P B, float cA, float cH, const int *plist,
                                                       const int *pcount, D4S *part, int nbx, int nrhs,
                                                       unsigned long long *prof) {
  extern __shared__ uint4 pl_sm[];
  const int count = *pcount;
  const int n_items = count * nbx;
  const float2 cA2 = make_float2(cA, cA), cH2 = make_float2(cH, cH);
  const int tid = threadIdx.x, Lz = g.L[2], Lt = g.L[3];
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(pl_sm + tid);
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int P = plist[w / nbx], sb = w % nbx;
    const int z = sb % Lz, t = sb / Lz;
    const int pl[PL_SLOTS] = {sb, (z + 1 == Lz ? 0 : z + 1) + Lz * t, (z == 0 ? Lz - 1 : z - 1) + Lz * t,
                              z + Lz * (t + 1 == Lt ? 0 : t + 1), z + Lz * (t == 0 ? Lt - 1 : t - 1)};
    {
      const uint4 *src = in.d + (size_t)P * 6 * in.vh + tid;
#pragma unroll
      for (int s = 0; s < PL_SLOTS; ++s)
#pragma unroll
        for (int k = 0; k < 6; ++k)
          cp_async16(s_base + (uint32_t)((s * 6 + k) * ST * 16), src + (size_t)k * in.vh + (size_t)pl[s] * ST);
      if (EPI != EPI_PLAIN) {
        const uint4 *sa = A.d + (size_t)P * 6 * A.vh + (size_t)sb * ST + tid;
#pragma unroll
        for (int k = 0; k < 6; ++k)
          cp_async16(s_base + (uint32_t)(((PL_SLOTS * 6) + k) * ST * 16), sa + (size_t)k * A.vh);
      }
      asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    if (prof && tid == 0) atomicAdd(prof + EPI, (unsigned long long)ST * (2 * P + 1 < nrhs ? 2 : 1));
    const int i = sb * ST + tid;
    int c[4];
    coords_of(g, p_out, i, c);
    CP acc[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) acc[a][b] = CP{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    hop_dir_plane<0>(g, p_out, c, i, pl_sm, links, acc);
    hop_dir_plane<1>(g, p_out, c, i, pl_sm, links, acc);
    hop_dir_plane<2>(g, p_out, c, i, pl_sm, links, acc);
    hop_dir_plane<3>(g, p_out, c, i, pl_sm, links, acc);
    float2 a[24];
    if (EPI != EPI_PLAIN) load_plane(pl_sm, PL_SLOTS, tid, a);
    D4S r0 = {0, 0, 0, 0}, r1 = {0, 0, 0, 0};
    pair_epilogue<BF16P, EPI>(acc, a, cA2, cH2, out, B, P, i, r0, r1);
    if (EPI == EPI_DOTR || EPI == EPI_TS)
      group_reduce_store2<1>(r0, r1, part + (size_t)(2 * P) * nbx + sb, part + (size_t)(2 * P + 1) * nbx + sb, true);
    __syncthreads();  // the next item's copies overwrite the planes
  }
}

// ======================================== pair hopping term on tensor cores
// The SU(3) products of the hopping term are moved onto the tensor cores with
// mma.sync m16n8k8 (tf32 in, FP32 accumulate); spin projection, the norms and
// the spin reconstruction stay on the FP32 units.  A warp takes 8 pairs of one
// site; lane (g, t) = (lane / 4, lane % 4) owns pair g and colour t (t = 3
// carries zeros).  For one (site, direction, half-spinor j) the MMA computes
//   D[row][n] = sum_k A[row][k] B[k][n]
// with rows g / g + 8 = the two members of pair g, k = (Re c0, Re c1, Re c2, 0,
// Im c0, Im c1, Im c2, 0) the projected half-spinor h_j and B the real form of
// U^T (or of U^+^T backwards), columns n = (Re a0, Im a0, Re a1, ... , 0, 0):
// so each lane's operands and results are its own pair and colour, read from
// and written to the pair layout directly, with no data exchange between lanes.
__device__ __forceinline__ unsigned tf32_bits(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float d[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%10,%10,%10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f));
}
__device__ __forceinline__ float2 unpack_word(const F16P &, unsigned w) { return h2f(w); }
__device__ __forceinline__ float2 unpack_word(const BF16P &, unsigned w) { return b2f(w); }

// colour t of all four spins of pair P at site i (values as stored, unscaled)
template <class SP>
__device__ __forceinline__ void load_colour(const SP &f, int P, int i, int t, CP p[4]) {
  const uint4 *base = f.d + (size_t)P * 6 * f.vh + i;
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) {
    const int k = 6 * sp + 2 * t;  // words k (Re) and k + 1 (Im) of this colour and spin
    const uint2 q = reinterpret_cast<const uint2 *>(base + (size_t)(k >> 2) * f.vh)[(k >> 1) & 1];
    p[sp] = CP{unpack_word(f, q.x), unpack_word(f, q.y)};
  }
}
template <class SP>
__device__ __forceinline__ void store_colour(const SP &f, int P, int i, int t, const CP o[4], float2 inv) {
  uint4 *base = f.d + (size_t)P * 6 * f.vh + i;
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) {
    const int k = 6 * sp + 2 * t;
    unsigned wr, wi;
    if constexpr (std::is_same<SP, F16P>::value) {
      wr = f2h(M2(o[sp].re, inv));
      wi = f2h(M2(o[sp].im, inv));
    } else {
      wr = f2b(o[sp].re);
      wi = f2b(o[sp].im);
    }
    reinterpret_cast<uint2 *>(base + (size_t)(k >> 2) * f.vh)[(k >> 1) & 1] = make_uint2(wr, wi);
  }
}

// spin projection (1 + SIGMA gamma_mu) of one colour (cf. project_pair)
template <int MU, int SIGMA>
__device__ __forceinline__ void project_colour(const CP p[4], CP &h0, CP &h1) {
  if (MU == 0) {
    h0 = cp_addi<SIGMA>(p[0], p[3]);
    h1 = cp_addi<SIGMA>(p[1], p[2]);
  } else if (MU == 1) {
    h0 = cp_addpm<-SIGMA>(p[0], p[3]);
    h1 = cp_addpm<SIGMA>(p[1], p[2]);
  } else if (MU == 2) {
    h0 = cp_addi<SIGMA>(p[0], p[2]);
    h1 = cp_addi<-SIGMA>(p[1], p[3]);
  } else {
    h0 = cp_addpm<SIGMA>(p[0], p[2]);
    h1 = cp_addpm<SIGMA>(p[1], p[3]);
  }
}
// spin reconstruction of one colour (cf. su3_accum_pair)
template <int MU, int SIGMA>
__device__ __forceinline__ void accum_colour(CP acc[4], const CP &x0, const CP &x1, float2 n) {
  const float2 nn = make_float2(-n.x, -n.y);
  acc[0] = cp_fma_pm<1>(acc[0], x0, n, nn);
  acc[1] = cp_fma_pm<1>(acc[1], x1, n, nn);
  if (MU == 0) {
    acc[2] = cp_fma_i<-SIGMA>(acc[2], x1, n, nn);
    acc[3] = cp_fma_i<-SIGMA>(acc[3], x0, n, nn);
  } else if (MU == 1) {
    acc[2] = cp_fma_pm<SIGMA>(acc[2], x1, n, nn);
    acc[3] = cp_fma_pm<-SIGMA>(acc[3], x0, n, nn);
  } else if (MU == 2) {
    acc[2] = cp_fma_i<-SIGMA>(acc[2], x0, n, nn);
    acc[3] = cp_fma_i<SIGMA>(acc[3], x1, n, nn);
  } else {
    acc[2] = cp_fma_pm<SIGMA>(acc[2], x0, n, nn);
    acc[3] = cp_fma_pm<SIGMA>(acc[3], x1, n, nn);
  }
}

// raw operands of one neighbour, loaded before any arithmetic so that all eight
// neighbours' loads of a site are in flight together
struct MmaIn {
  uint2 w[4];  // words (Re, Im) of colour t, spins 0..3
  float2 n;    // member norms (with the time-boundary sign)
  float2 u;    // link entry for this lane (forward U[a][c], backward U[c][a])
};

template <class SP>
__device__ __forceinline__ void mma_load(const SP &in, int P, bool act, int nidx, bool flip, const float2 *lk,
                                         bool lk_ok, int t, MmaIn &r) {
  if (act) {
    const uint4 *base = in.d + (size_t)P * 6 * in.vh + nidx;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
      const int k = 6 * sp + 2 * t;
      r.w[sp] = reinterpret_cast<const uint2 *>(base + (size_t)(k >> 2) * in.vh)[(k >> 1) & 1];
    }
    r.n = read_norm(in, P, nidx);
    if (flip) r.n = make_float2(-r.n.x, -r.n.y);
  } else {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) r.w[sp] = make_uint2(0u, 0u);
    r.n = make_float2(0.f, 0.f);
  }
  r.u = lk_ok ? *lk : make_float2(0.f, 0.f);
}

// project, two MMAs (h0, h1), reconstruct into acc; SIGMA = -1 forward, +1 backward
template <int MU, int SIGMA, class SP>
__device__ __forceinline__ void mma_compute(const SP &in, const MmaIn &r, int g4, CP acc[4]) {
  CP p[4];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) p[sp] = CP{unpack_word(in, r.w[sp].x), unpack_word(in, r.w[sp].y)};
  CP h0, h1;
  project_colour<MU, SIGMA>(p, h0, h1);
  // B fragment: lane (g4, t) holds B[k = Re c_t][n = g4] and B[k = Im c_t][n = g4] of the
  // real form of M = U (forward) or U^+ (backward; the lane loaded U[c][a], M[a][c] = conj)
  const float ur = r.u.x, ui = SIGMA < 0 ? r.u.y : -r.u.y;
  unsigned b0, b1;
  if ((g4 & 1) == 0) {  // output Re a: (Re M, -Im M)
    b0 = __float_as_uint(ur);
    b1 = __float_as_uint(-ui);
  } else {  // output Im a: (Im M, Re M)
    b0 = __float_as_uint(ui);
    b1 = __float_as_uint(ur);
  }
  unsigned a[4];
  float d0[4], d1[4];
  a[0] = tf32_bits(h0.re.x);
  a[1] = tf32_bits(h0.re.y);
  a[2] = tf32_bits(h0.im.x);
  a[3] = tf32_bits(h0.im.y);
  mma_tf32(d0, a, b0, b1);
  a[0] = tf32_bits(h1.re.x);
  a[1] = tf32_bits(h1.re.y);
  a[2] = tf32_bits(h1.im.x);
  a[3] = tf32_bits(h1.im.y);
  mma_tf32(d1, a, b0, b1);
  const CP x0{make_float2(d0[0], d0[2]), make_float2(d0[1], d0[3])};
  const CP x1{make_float2(d1[0], d1[2]), make_float2(d1[1], d1[3])};
  accum_colour<MU, SIGMA>(acc, x0, x1, r.n);
}

// all eight neighbours of site i (coordinates c) for this lane's pair and colour
template <class SP>
__device__ __forceinline__ void hop_mma_site(const Geom &g, int p_out, const int c[4], int i, const SP &in, int P,
                                             bool act, const float2 *links, int g4, int t, CP acc[4]) {
  const bool lk_ok = g4 < 6 && t < 3;
  const int a = g4 >> 1;
  MmaIn r[8];  // [2 mu + (0 forward, 1 backward)]
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    int cf[4] = {c[0], c[1], c[2], c[3]}, cb[4] = {c[0], c[1], c[2], c[3]};
    cf[mu] = (c[mu] + 1 == g.L[mu]) ? 0 : c[mu] + 1;
    cb[mu] = (c[mu] == 0) ? g.L[mu] - 1 : c[mu] - 1;
    const int nf = site_of(g, cf) >> 1, nb = site_of(g, cb) >> 1;
    const float2 *lf = links + ((size_t)(p_out * 4 + mu) * g.Vh + i) * 9 + (lk_ok ? a * 3 + t : 0);
    const float2 *lb = links + ((size_t)((1 - p_out) * 4 + mu) * g.Vh + nb) * 9 + (lk_ok ? t * 3 + a : 0);
    mma_load(in, P, act, nf, mu == 3 && c[3] == g.L[3] - 1, lf, lk_ok, t, r[2 * mu]);
    mma_load(in, P, act, nb, mu == 3 && c[3] == 0, lb, lk_ok, t, r[2 * mu + 1]);
  }
  mma_compute<0, -1>(in, r[0], g4, acc);
  mma_compute<0, 1>(in, r[1], g4, acc);
  mma_compute<1, -1>(in, r[2], g4, acc);
  mma_compute<1, 1>(in, r[3], g4, acc);
  mma_compute<2, -1>(in, r[4], g4, acc);
  mma_compute<2, 1>(in, r[5], g4, acc);
  mma_compute<3, -1>(in, r[6], g4, acc);
  mma_compute<3, 1>(in, r[7], g4, acc);
}

constexpr int MMA_SITES = 128;  // sites per work item (4 warps x 32 sites), = ST
constexpr int MMA_MINB = 3;     // resident blocks per SM the register budget is cut for
// out = cA A + cH (H in) at parity p_out for groups of 8 active pairs, with the
// same epilogues and partial layout as k_hop_pair (one partial per member and
// block of ST sites).
template <class SP, int EPI>
__global__ void __launch_bounds__(128, MMA_MINB) k_hop_mma(Geom g, int p_out, const float2 *links, SP in, SP out, SP A,
                                                    SP B, float cA, float cH, const int *plist, const int *pcount,
                                                    D4S *part, int nbx, int nrhs, unsigned long long *prof) {
  const int count = *pcount;
  const int n_items = (count + 7) / 8 * nbx;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g4 = lane >> 2, t = lane & 3;
  const float2 cA2 = make_float2(cA, cA), cH2 = make_float2(cH, cH);
  __shared__ float4 red[4][8][2];  // [warp][pair][member] (re, im, |.|^2, 0)
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int j = (w / nbx) * 8 + g4, sb = w % nbx;
    const bool valid = j < count;
    const int P = valid ? plist[j] : 0;
    const bool act = valid && t < 3;
    if (prof && valid && t == 0 && warp == 0)
      atomicAdd(prof + EPI, (unsigned long long)min(MMA_SITES, g.Vh - sb * MMA_SITES) * (2 * P + 1 < nrhs ? 2 : 1));
    float2 sre = make_float2(0.f, 0.f), sim = sre, snn = sre;
    for (int k = 0; k < 32; ++k) {
      const int i = sb * MMA_SITES + warp * 32 + k;  // the same for the whole warp
      if (i >= g.Vh) break;
      int c[4];
      coords_of(g, p_out, i, c);
      CP acc[4];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp) acc[sp] = CP{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      hop_mma_site(g, p_out, c, i, in, P, act, links, g4, t, acc);
      CP o[4], av[4];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp) o[sp] = CP{M2(acc[sp].re, cH2), M2(acc[sp].im, cH2)};
      if (EPI != EPI_PLAIN) {
        if (act) {
          load_colour(A, P, i, t, av);
          const float2 an = read_norm(A, P, i);
#pragma unroll
          for (int sp = 0; sp < 4; ++sp) av[sp] = CP{M2(av[sp].re, an), M2(av[sp].im, an)};
        } else {
#pragma unroll
          for (int sp = 0; sp < 4; ++sp) av[sp] = CP{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        }
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) o[sp] = CP{F2(cA2, av[sp].re, o[sp].re), F2(cA2, av[sp].im, o[sp].im)};
      }
      // encode and store (FP16: the site norm is the largest |real| over the three colour lanes)
      float2 inv = make_float2(1.f, 1.f);
      if constexpr (std::is_same<SP, F16P>::value) {
        float2 m = make_float2(0.f, 0.f);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
          m.x = fmaxf(m.x, fmaxf(fabsf(o[sp].re.x), fabsf(o[sp].im.x)));
          m.y = fmaxf(m.y, fmaxf(fabsf(o[sp].re.y), fabsf(o[sp].im.y)));
        }
        m.x = fmaxf(m.x, __shfl_xor_sync(0xffffffffu, m.x, 1));
        m.y = fmaxf(m.y, __shfl_xor_sync(0xffffffffu, m.y, 1));
        m.x = fmaxf(m.x, __shfl_xor_sync(0xffffffffu, m.x, 2));
        m.y = fmaxf(m.y, __shfl_xor_sync(0xffffffffu, m.y, 2));
        inv = make_float2(m.x > 0.f ? 1.f / m.x : 0.f, m.y > 0.f ? 1.f / m.y : 0.f);
        if (valid && t == 0) write_norm(out, P, i, m);
      }
      if (act) store_colour(out, P, i, t, o, inv);
      if (EPI == EPI_DOTR && act) {  // <B, out>
        CP bv[4];
        load_colour(B, P, i, t, bv);
        const float2 bn = read_norm(B, P, i);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
          const float2 br = M2(bv[sp].re, bn), bi = M2(bv[sp].im, bn);
          sre = F2(br, o[sp].re, sre);
          sre = F2(bi, o[sp].im, sre);
          sim = F2(br, o[sp].im, sim);
          sim = F2(make_float2(-bi.x, -bi.y), o[sp].re, sim);
        }
      } else if (EPI == EPI_TS && act) {  // <out, A> and |out|^2
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
          sre = F2(o[sp].re, av[sp].re, sre);
          sre = F2(o[sp].im, av[sp].im, sre);
          sim = F2(o[sp].re, av[sp].im, sim);
          sim = F2(make_float2(-o[sp].im.x, -o[sp].im.y), av[sp].re, sim);
          snn = F2(o[sp].re, o[sp].re, snn);
          snn = F2(o[sp].im, o[sp].im, snn);
        }
      }
    }
    if (EPI == EPI_DOTR || EPI == EPI_TS) {
      // fixed-order reduction: colour lanes, then the four warps
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {
        sre.x += __shfl_xor_sync(0xffffffffu, sre.x, o);
        sre.y += __shfl_xor_sync(0xffffffffu, sre.y, o);
        sim.x += __shfl_xor_sync(0xffffffffu, sim.x, o);
        sim.y += __shfl_xor_sync(0xffffffffu, sim.y, o);
        snn.x += __shfl_xor_sync(0xffffffffu, snn.x, o);
        snn.y += __shfl_xor_sync(0xffffffffu, snn.y, o);
      }
      if (t == 0) {
        red[warp][g4][0] = make_float4(sre.x, sim.x, snn.x, 0.f);
        red[warp][g4][1] = make_float4(sre.y, sim.y, snn.y, 0.f);
      }
      __syncthreads();
      if (threadIdx.x < 16) {
        const int pg = threadIdx.x >> 1, mem = threadIdx.x & 1;
        const int jj = (w / nbx) * 8 + pg;
        if (jj < count) {
          double re = 0.0, im = 0.0, nn = 0.0;
#pragma unroll
          for (int ww = 0; ww < 4; ++ww) {
            re += red[ww][pg][mem].x;
            im += red[ww][pg][mem].y;
            nn += red[ww][pg][mem].z;
          }
          part[(size_t)(2 * plist[jj] + mem) * nbx + sb] = EPI == EPI_DOTR ? D4S{re, im, 0, 0} : D4S{re, im, 0, nn};
        }
      }
      __syncthreads();
    }
  }
}

// The pair-layout variants of the hopping term (0-4, 6 and 7; see HOP_VARIANTS below).
template <class SP, int EPI>
static void launch_hop_pair(int variant, int G, cudaStream_t q, const lqcd_ctx *ctx, Geom g, int p_out, SP in, SP out,
                            SP A, SP B, float cA, float cH, const int *plist, const int *pcount, D4S *part, int nbx,
                            int nrhs, unsigned long long *prof) {
  const uint4 *L16 = ctx->U16;
  switch (variant) {
    case 1:
      KL k_hop_pair<SP, EPI, 4, 1><<<G, ST, 0, q>>>(g, p_out, L16, in, out, A, B, cA, cH, plist, pcount, part, nbx,
                                                     nrhs, prof);
      break;
    case 2:
      KL k_hop_pair<SP, EPI, 2, 2><<<G, 2 * ST, 0, q>>>(g, p_out, L16, in, out, A, B, cA, cH, plist, pcount, part, nbx,
                                                         nrhs, prof);
      break;
    case 3:
      KL k_hop_pair<SP, EPI, 1, 4><<<G, 4 * ST, 0, q>>>(g, p_out, L16, in, out, A, B, cA, cH, plist, pcount, part, nbx,
                                                         nrhs, prof);
      break;
    case 4:
      KL k_hop_mma<SP, EPI><<<G, 128, 0, q>>>(g, p_out, ctx->Utf, in, out, A, B, cA, cH, plist, pcount, part, nbx, nrhs,
                                              prof);
      break;
    case PLANE_VARIANT:
      if constexpr (std::is_same<SP, BF16P>::value) {
        if (planes_fit(g)) {
          constexpr int smem = EPI == EPI_PLAIN ? PL_SMEM_PLAIN : PL_SMEM_EPI;
          static bool attr = false;  // a refused attribute makes the launch fail, which the caller reports
          if (!attr) attr = cudaFuncSetAttribute(k_hop_pair_pl<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 smem) == cudaSuccess;
          KL k_hop_pair_pl<EPI><<<G, ST, smem, q>>>(g, p_out, L16, in, out, A, B, cA, cH, plist, pcount, part, nbx,
                                                    nrhs, prof);
          break;
        }
      }
      // other precisions and geometries: the register-capped pair kernel
      KL k_hop_pair<SP, EPI, 4, 1><<<G, ST, 0, q>>>(g, p_out, L16, in, out, A, B, cA, cH, plist, pcount, part, nbx,
                                                     nrhs, prof);
      break;
    case R12_VARIANT:
      KL k_hop_pair<SP, EPI, 4, 1, true><<<G, ST, 0, q>>>(g, p_out, L16, in, out, A, B, cA, cH, plist, pcount, part,
                                                           nbx, nrhs, prof);
      break;
    default:
      KL k_hop_pair<SP, EPI, 1, 1><<<G, ST, 0, q>>>(g, p_out, L16, in, out, A, B, cA, cH, plist, pcount, part, nbx,
                                                     nrhs, prof);
      break;
  }
}

// ============================================================ BLAS kernels
__device__ __forceinline__ CP scal_pair(double2 a, double2 b) {
  return CP{make_float2((float)a.x, (float)b.x), make_float2((float)a.y, (float)b.y)};
}
// a + s * z and a - s * z
__device__ __forceinline__ CP cp_fma(const CP &s, const CP &z, const CP &a) {
  return CP{S2(F2(s.re, z.re, a.re), M2(s.im, z.im)), F2(s.re, z.im, F2(s.im, z.re, a.im))};
}
__device__ __forceinline__ CP cp_fms(const CP &s, const CP &z, const CP &a) {  // a - s z
  return CP{F2(s.im, z.im, S2(a.re, M2(s.re, z.re))), S2(a.im, F2(s.re, z.im, M2(s.im, z.re)))};
}

// p = r + beta (p - omega v); members flagged for restart take rhat = r, p = r.
template <class SP>
__global__ void __launch_bounds__(ST) k_pair_p(int vh, const SState *sc, SP r, SP rhat, SP p, SP v,
                                               const int *plist, const int *pcount, int nbx) {
  const int n_items = *pcount * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int P = plist[w / nbx];
    const int i = (w % nbx) * ST + threadIdx.x;
    if (i >= vh) continue;
    const bool re0 = sc[2 * P].restart, re1 = sc[2 * P + 1].restart;
    float2 rv[24], pv[24];
    load_scaled(r, P, i, rv);
    if (!(re0 && re1)) {
      float2 vv[24];
      load_scaled(p, P, i, pv);
      load_scaled(v, P, i, vv);
      const CP be = scal_pair(sc[2 * P].beta, sc[2 * P + 1].beta);
      const CP om = scal_pair(sc[2 * P].omega, sc[2 * P + 1].omega);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        CP t = cp_fms(om, CP{vv[2 * k], vv[2 * k + 1]}, CP{pv[2 * k], pv[2 * k + 1]});
        CP n = cp_fma(be, t, CP{rv[2 * k], rv[2 * k + 1]});
        pv[2 * k] = n.re;
        pv[2 * k + 1] = n.im;
      }
    }
    if (re0 || re1) {
#pragma unroll
      for (int k = 0; k < 24; ++k) pv[k] = sel2(re0, re1, rv[k], pv[k]);
      store_members(rhat, P, i, rv, re0, re1);
    }
    store_pair(p, P, i, pv);
  }
}

// s = r - alpha v
template <class SP>
__global__ void __launch_bounds__(ST) k_pair_s(int vh, const SState *sc, SP r, SP v, SP s, const int *plist,
                                               const int *pcount, int nbx) {
  const int n_items = *pcount * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int P = plist[w / nbx];
    const int i = (w % nbx) * ST + threadIdx.x;
    if (i >= vh) continue;
    const CP al = scal_pair(sc[2 * P].alpha, sc[2 * P + 1].alpha);
    float2 rv[24], vv[24];
    load_scaled(r, P, i, rv);
    load_scaled(v, P, i, vv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      CP n = cp_fms(al, CP{vv[2 * k], vv[2 * k + 1]}, CP{rv[2 * k], rv[2 * k + 1]});
      rv[2 * k] = n.re;
      rv[2 * k + 1] = n.im;
    }
    store_pair(s, P, i, rv);
  }
}

// x += alpha p + omega s (FP32 x, active members only); r = s - omega t;
// partials <rhat, r> and |r|^2 per member
template <class SP>
__global__ void __launch_bounds__(ST) k_pair_xr(int vh, const SState *sc, const int *flags, F32F x, SP p, SP s, SP t,
                                                SP r, SP rhat, const int *plist, const int *pcount, D4S *part,
                                                int nbx) {
  const int n_items = *pcount * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int P = plist[w / nbx], sb = w % nbx;
    const int i = sb * ST + threadIdx.x;
    D4S r0 = {0, 0, 0, 0}, r1 = {0, 0, 0, 0};
    if (i < vh) {
      const bool a0 = flags[2 * P] & FLAG_ACTIVE, a1 = flags[2 * P + 1] & FLAG_ACTIVE;
      const CP al = scal_pair(sc[2 * P].alpha, sc[2 * P + 1].alpha);
      const CP om = scal_pair(sc[2 * P].omega, sc[2 * P + 1].omega);
      float2 pv[24], sv[24], tv[24];
      load_scaled(p, P, i, pv);
      load_scaled(s, P, i, sv);
      load_scaled(t, P, i, tv);
      float2 x0[12], x1[12];
      if (a0) x.load(2 * P, i, x0);
      if (a1) x.load(2 * P + 1, i, x1);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        CP xk{make_float2(a0 ? x0[k].x : 0.f, a1 ? x1[k].x : 0.f), make_float2(a0 ? x0[k].y : 0.f, a1 ? x1[k].y : 0.f)};
        xk = cp_fma(al, CP{pv[2 * k], pv[2 * k + 1]}, xk);
        xk = cp_fma(om, CP{sv[2 * k], sv[2 * k + 1]}, xk);
        x0[k] = make_float2(xk.re.x, xk.im.x);
        x1[k] = make_float2(xk.re.y, xk.im.y);
        CP rn = cp_fms(om, CP{tv[2 * k], tv[2 * k + 1]}, CP{sv[2 * k], sv[2 * k + 1]});
        sv[2 * k] = rn.re;
        sv[2 * k + 1] = rn.im;
      }
      if (a0) x.store(2 * P, i, x0);
      if (a1) x.store(2 * P + 1, i, x1);
      store_pair(r, P, i, sv);
      load_scaled(rhat, P, i, pv);
      float2 re = make_float2(0.f, 0.f), ip = re, im = re, nn = re;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        re = F2(pv[2 * k], sv[2 * k], re);
        re = F2(pv[2 * k + 1], sv[2 * k + 1], re);
        ip = F2(pv[2 * k], sv[2 * k + 1], ip);
        im = F2(pv[2 * k + 1], sv[2 * k], im);
        nn = F2(sv[2 * k], sv[2 * k], nn);
        nn = F2(sv[2 * k + 1], sv[2 * k + 1], nn);
      }
      const float2 imag = S2(ip, im);
      r0 = D4S{re.x, imag.x, nn.x, 0};
      r1 = D4S{re.y, imag.y, nn.y, 0};
    }
    block_reduce_store2(r0, r1, part + (size_t)(2 * P) * nbx + sb, part + (size_t)(2 * P + 1) * nbx + sb);
  }
}

// members flagged FLAG_RU: r = src (FP32), optionally x = 0; partials per
// member of <rhat, r> (or <r, r>) and |r|^2
template <class SP>
__global__ void __launch_bounds__(ST) k_pair_copy(int vh, const int *flags, F32F src, SP r, SP rhat, bool use_rhat,
                                                  F32F x, bool zero_x, const int *plist, const int *pcount, D4S *part,
                                                  int nbx) {
  const int n_items = *pcount * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int P = plist[w / nbx], sb = w % nbx;
    const int i = sb * ST + threadIdx.x;
    D4S r0 = {0, 0, 0, 0}, r1 = {0, 0, 0, 0};
    if (i < vh) {
      const bool w0 = flags[2 * P] & FLAG_RU, w1 = flags[2 * P + 1] & FLAG_RU;
      float2 s0[12], s1[12], v[24];
      if (w0) src.load(2 * P, i, s0);
      if (w1) src.load(2 * P + 1, i, s1);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        v[2 * k] = make_float2(w0 ? s0[k].x : 0.f, w1 ? s1[k].x : 0.f);
        v[2 * k + 1] = make_float2(w0 ? s0[k].y : 0.f, w1 ? s1[k].y : 0.f);
      }
      store_members(r, P, i, v, w0, w1);
      if (zero_x) {
        float2 z[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = make_float2(0.f, 0.f);
        if (w0) x.store(2 * P, i, z);
        if (w1) x.store(2 * P + 1, i, z);
      }
      float2 q[24];
      if (use_rhat) load_scaled(rhat, P, i, q);
      float2 re = make_float2(0.f, 0.f), ip = re, im = re, nn = re;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float2 qr = use_rhat ? q[2 * k] : v[2 * k], qi = use_rhat ? q[2 * k + 1] : v[2 * k + 1];
        re = F2(qr, v[2 * k], re);
        re = F2(qi, v[2 * k + 1], re);
        ip = F2(qr, v[2 * k + 1], ip);
        im = F2(qi, v[2 * k], im);
        nn = F2(v[2 * k], v[2 * k], nn);
        nn = F2(v[2 * k + 1], v[2 * k + 1], nn);
      }
      const float2 imag = S2(ip, im);
      r0 = D4S{re.x, imag.x, nn.x, 0};
      r1 = D4S{re.y, imag.y, nn.y, 0};
    }
    block_reduce_store2(r0, r1, part + (size_t)(2 * P) * nbx + sb, part + (size_t)(2 * P + 1) * nbx + sb);
  }
}

// ============================================ precision conversion kernels
// Both parities at once: parity-local index i owns canonical sites 2i and 2i+1
// (one even, one odd), so each thread's canonical data is one contiguous run.
__device__ __forceinline__ int even_first(const Geom &g, int i) {  // is site 2i the even one?
  int r = i / g.Lxh;
  int y = r % g.L[1];
  r /= g.L[1];
  return ((y + r % g.L[2] + r / g.L[2]) & 1) == 0;
}

// dst_e / dst_o (FP32 parity fields) = scale[rhs] * src (canonical FP32)
__global__ void __launch_bounds__(ST) k_cvt32to32_both(Geom g, const float2 *__restrict__ src, F32F de, F32F dodd,
                                                       const double *scale, const int *list, const int *count,
                                                       int nbx) {
  const int n_items = *count * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int rhs = list[w / nbx];
    const int i = (w % nbx) * ST + threadIdx.x;
    if (i >= g.Vh) continue;
    const float2 *q = src + ((size_t)rhs * g.V + 2 * (size_t)i) * 12;
    const float sc = (float)scale[rhs];
    const int ef = even_first(g, i);
    float2 v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = make_float2(q[k].x * sc, q[k].y * sc);
    (ef ? de : dodd).store(rhs, i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = make_float2(q[12 + k].x * sc, q[12 + k].y * sc);
    (ef ? dodd : de).store(rhs, i, v);
  }
}

// dst_e / dst_o (FP32 parity fields) = scale[rhs] * src (canonical FP64)
__global__ void __launch_bounds__(ST) k_cvt64to32_both(Geom g, const double2 *__restrict__ src, F32F de, F32F dodd,
                                                       const double *scale, const int *list, const int *count,
                                                       int nbx) {
  const int n_items = *count * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int rhs = list[w / nbx];
    const int i = (w % nbx) * ST + threadIdx.x;
    if (i >= g.Vh) continue;
    const double2 *q = src + ((size_t)rhs * g.V + 2 * (size_t)i) * 12;
    const double sc = scale[rhs];
    const int ef = even_first(g, i);
    // scale = m 2^e: the power of two goes into the integer rounding to binary32,
    // m is one FP32 multiply, so the FP64 pipe does no work for a normal scale
    int e2;
    float m;
    const bool split = lqcd::split_pow2(sc, e2, m);
    float2 v[12];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (split) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const double2 a = q[12 * h + k];
          v[k] = make_float2(lqcd::f64_to_f32_bits(a.x, e2) * m, lqcd::f64_to_f32_bits(a.y, e2) * m);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const double2 a = q[12 * h + k];
          v[k] = make_float2((float)(a.x * sc), (float)(a.y * sc));
        }
      }
      ((ef != 0) == (h == 0) ? de : dodd).store(rhs, i, v);
    }
  }
}

// x (double-float canonical) += scale[rhs] * (e on even sites, o on odd sites).
// A block's ST parity-local indices own 2 ST consecutive canonical sites: that
// contiguous run (ST * 384 B) is staged through shared memory so every global
// load and store is coalesced.
constexpr int ACC_SITES = 64;  // parity-local indices per block (48 KiB of shared memory)
__global__ void __launch_bounds__(ACC_SITES * 2) k_accum_df_both(Geom g, F32F e, F32F o, float4 *x,
                                                                 const double *scale, const int *list,
                                                                 const int *count, int nbx) {
  __shared__ float4 tile[ACC_SITES * 24];
  const int n_items = *count * nbx;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int rhs = list[w / nbx];
    const int i0 = (w % nbx) * ACC_SITES;
    const int nloc = min(ACC_SITES, g.Vh - i0);
    float4 *base = x + ((size_t)rhs * g.V + 2 * (size_t)i0) * 12;
    constexpr int PER = ACC_SITES * 24 / (ACC_SITES * 2);  // elements per thread of a full tile
    if (nloc == ACC_SITES) {  // all loads issued before any store: PER requests in flight
      float4 q[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) q[u] = base[threadIdx.x + u * blockDim.x];
#pragma unroll
      for (int u = 0; u < PER; ++u) tile[threadIdx.x + u * blockDim.x] = q[u];
    } else {
      for (int k = threadIdx.x; k < nloc * 24; k += blockDim.x) tile[k] = base[k];
    }
    __syncthreads();
    // two threads per parity-local index: one per canonical site of the pair
    const int li = threadIdx.x >> 1, half = threadIdx.x & 1;
    if (li < nloc) {
      const int i = i0 + li;
      const double scd = scale[rhs];
      const float sh = (float)scd;
      const dfl sc{sh, (float)(scd - (double)sh)};
      const bool even_site = (half == 0) == (even_first(g, i) != 0);
      float2 v[12];
      (even_site ? e : o).load(rhs, i, v);
      float4 *q = tile + (size_t)li * 24 + half * 12;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        float4 old = q[k];
        dfl re = df_norm(dfl{old.x, old.z} + sc * dfl{v[k].x, 0.f});
        dfl im = df_norm(dfl{old.y, old.w} + sc * dfl{v[k].y, 0.f});
        q[k] = make_float4(re.h, im.h, re.l, im.l);
      }
    }
    __syncthreads();
    if (nloc == ACC_SITES) {
#pragma unroll
      for (int u = 0; u < PER; ++u) base[threadIdx.x + u * blockDim.x] = tile[threadIdx.x + u * blockDim.x];
    } else {
      for (int k = threadIdx.x; k < nloc * 24; k += blockDim.x) base[k] = tile[k];
    }
    __syncthreads();
  }
}

// ============================================================ finalisers
__device__ __forceinline__ D4S warp_total_s(const D4S *part, int nb) {
  D4S acc = {0, 0, 0, 0};
  for (int k = threadIdx.x & 31; k < nb; k += 32) {
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
// target2 (set by the host from the outer tolerance) is floored at floor2 * |b_inner|^2
__global__ void k_sfin_init(SState *sc, int *flags, const int *list, const int *count, const D4S *part, int nb,
                            double floor2) {
  if (blockIdx.x >= *count) return;
  int rhs = list[blockIdx.x];
  D4S t = warp_total_s(part + (size_t)rhs * nb, nb);
  if (threadIdx.x) return;
  SState &s = sc[rhs];
  s.target2 = fmax(s.target2, floor2 * t.c);
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

// One warp per member of a listed group (gs right-hand sides: 2 for the pair
// layout, 128 for tiles); a block of 64 threads takes two members, block b of
// group list entry b / (gs / 2).  Members without FLAG_ACTIVE are skipped.
#define PAIR_MEMBER(n)                                                                     \
  if (blockIdx.x / (gs >> 1) >= *pcount) return;                                           \
  const int rhs = gs * plist[blockIdx.x / (gs >> 1)] + 2 * (blockIdx.x % (gs >> 1)) + (threadIdx.x >> 5); \
  if (rhs >= (n) || !(flags[rhs] & FLAG_ACTIVE)) return;

__global__ void k_sfin_alpha(SState *sc, const int *flags, const int *plist, const int *pcount, const D4S *part,
                             int nb, int n, int gs) {
  PAIR_MEMBER(n)
  D4S t = warp_total_s(part + (size_t)rhs * nb, nb);
  if (threadIdx.x & 31) return;
  SState &s = sc[rhs];
  double2 rv = make_double2(t.a, t.b);
  s.alpha = (rv.x == 0.0 && rv.y == 0.0) ? make_double2(0.0, 0.0) : cdiv_d(s.rho, rv);
  s.restart = 0;
}

__global__ void k_sfin_omega(SState *sc, const int *flags, const int *plist, const int *pcount, const D4S *part,
                             int nb, int n, int gs) {
  PAIR_MEMBER(n)
  D4S t = warp_total_s(part + (size_t)rhs * nb, nb);
  if (threadIdx.x & 31) return;
  SState &s = sc[rhs];
  s.omega = (t.d == 0.0) ? make_double2(0.0, 0.0) : make_double2(t.a / t.d, t.b / t.d);
}

// convergence / reliable-update decision after the x, r update
__global__ void k_sfin_conv(SState *sc, int *flags, const int *plist, const int *pcount, const D4S *part, int nb,
                            int n, double delta2, int max_iter, int gs) {
  PAIR_MEMBER(n)
  D4S t = warp_total_s(part + (size_t)rhs * nb, nb);
  if (threadIdx.x & 31) return;
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

// Deterministic compaction of the per-RHS flags into: active groups (any
// member active), RHS needing a reliable update, and groups containing one.
// A group is gs consecutive right-hand sides (2: pair layout, 128: tiles).
__global__ void k_build_lists(int n, const int *flags, int gs, int *act_groups, int *ru_list, int *ru_groups,
                              int *counts) {
  __shared__ int sa[1024], sr[1024], sp[1024];
  const int ng = (n + gs - 1) / gs;
  int tid = threadIdx.x, nt = blockDim.x;
  int per = (ng + nt - 1) / nt;
  int b0 = tid * per, b1 = min(ng, b0 + per);
  int ca = 0, cr = 0, cp = 0;
  for (int P = b0; P < b1; ++P) {
    int any = 0, nru = 0;
    for (int k = P * gs; k < min(n, (P + 1) * gs); ++k) {
      any |= flags[k];
      nru += (flags[k] & FLAG_RU) ? 1 : 0;
    }
    ca += (any & FLAG_ACTIVE) ? 1 : 0;
    cp += (any & FLAG_RU) ? 1 : 0;
    cr += nru;
  }
  sa[tid] = ca;
  sr[tid] = cr;
  sp[tid] = cp;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {  // inclusive scans
    int va = tid >= off ? sa[tid - off] : 0, vr = tid >= off ? sr[tid - off] : 0, vp = tid >= off ? sp[tid - off] : 0;
    __syncthreads();
    sa[tid] += va;
    sr[tid] += vr;
    sp[tid] += vp;
    __syncthreads();
  }
  int oa = sa[tid] - ca, orr = sr[tid] - cr, op = sp[tid] - cp;
  for (int P = b0; P < b1; ++P) {
    int any = 0;
    for (int k = P * gs; k < min(n, (P + 1) * gs); ++k) {
      any |= flags[k];
      if (flags[k] & FLAG_RU) ru_list[orr++] = k;
    }
    if (any & FLAG_ACTIVE) act_groups[oa++] = P;
    if (any & FLAG_RU) ru_groups[op++] = P;
  }
  if (tid == nt - 1) {
    counts[0] = sa[tid];
    counts[1] = sr[tid];
    counts[3] = sp[tid];
  }
}

}  // namespace lqcd

// ==================================================== device-side loop control
// The inner iterations of one outer cycle run as a CUDA-graph WHILE node
// (conditional node) whose condition these kernels set on the device:
// continue while any group is active, the tile hop reported no error, the
// cycle's wall-clock budget is not spent and the iteration guard is not hit.
//   counts[0] active groups, [8] tile-hop error code, [9] set when the budget
//   ran out, [10] loop iterations run; clk[0] start (globaltimer ns), clk[1]
//   budget in ns (written by the host before each launch).
namespace lqcd {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__global__ void k_loop_init(cudaGraphConditionalHandle h, int *counts, unsigned long long *clk) {
  clk[0] = globaltimer_ns();
  counts[9] = 0;
  counts[10] = 0;
  cudaGraphSetConditional(h, (counts[0] > 0 && counts[8] == 0 && clk[1] > 0) ? 1u : 0u);
}
__global__ void k_loop_cond(cudaGraphConditionalHandle h, int *counts, const unsigned long long *clk, int max_loops) {
  const int it = ++counts[10];
  const bool late = globaltimer_ns() - clk[0] > clk[1];
  if (late && counts[0] > 0) counts[9] = 1;
  cudaGraphSetConditional(h, (counts[0] > 0 && counts[8] == 0 && !late && it < max_loops) ? 1u : 0u);
}

}  // namespace lqcd

// ======================================================== host-side driver
namespace lqcd {

struct SloppyState {
  int cap = 0;             // RHS capacity (a multiple of the layout's group size)
  int gran = 2;            // group size the buffers were laid out for (2: pairs, 128: tiles)
  uint4 *sd = nullptr;     // 7 sloppy fields (pair or tile layout; same bytes per RHS)
  float2 *sn = nullptr;    // FP16 norms of the pair layout
  float4 *f32 = nullptr;   // 5 FP32 fields
  float4 *xdf = nullptr;   // the iterate, double-float canonical [cap][V][12]
  float2 *r32 = nullptr;   // residual b - D x, FP32 canonical (seeds the next inner solve)
  char *small = nullptr;
  int *h_counts = nullptr;  // pinned
  // captured graph of four inner iterations, valid while graph_key matches
  cudaGraphExec_t graph = nullptr;
  std::vector<double> graph_key;
  long long graph_kernels = 0;  // kernel launches one replay of the graph makes
};

void sloppy_free(lqcd_ctx *ctx) {
  SloppyState *s = ctx->sloppy;
  if (!s) return;
  cudaFree(s->sd);
  cudaFree(s->sn);
  cudaFree(s->f32);
  cudaFree(s->xdf);
  cudaFree(s->r32);
  cudaFree(s->small);
  if (s->h_counts) cudaFreeHost(s->h_counts);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  delete s;
  ctx->sloppy = nullptr;
}

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
  int *flags, *act_pairs, *ru_list, *ru_pairs, *cyc_list, *cyc_pairs, *counts;
  double *scale, *unscale;
  D4S *part;
  unsigned long long *clk;  // loop start and budget (ns)
  size_t bytes;
  size_t size() const { return bytes; }
};
// partial sums per RHS: the larger of the pair kernels' blocks of ST sites and
// the tile kernels' chunks of TCH sites
static int part_blocks(int vh) { return std::max((vh + ST - 1) / ST, (vh + TCH - 1) / TCH); }
static SmallBufs small_layout(void *base, int cap, int nbp) {
  Carver cv(base);
  SmallBufs b;
  b.sc = cv.take<SState>(cap);
  b.flags = cv.take<int>(cap);
  b.act_pairs = cv.take<int>(cap / 2);
  b.ru_list = cv.take<int>(cap);
  b.ru_pairs = cv.take<int>(cap / 2);
  b.cyc_list = cv.take<int>(cap);
  b.cyc_pairs = cv.take<int>(cap / 2);
  // [0] active groups, [1] RU RHS, [2] cycle RHS, [3] RU groups, [4] cycle groups, [8] tile-hop error
  // code, [9] loop stopped by the time budget, [10] loop iterations (see k_loop_cond)
  b.counts = cv.take<int>(16);
  b.clk = cv.take<unsigned long long>(2);
  b.scale = cv.take<double>(cap);
  b.unscale = cv.take<double>(cap);
  b.part = cv.take<D4S>((size_t)cap * nbp);
  b.bytes = cv.size();
  return b;
}

// capacity for nrhs right-hand sides in groups of gran (2 or TR)
static int sloppy_alloc(lqcd_ctx *ctx, int nrhs, int gran = 2) {
  if (!ctx->sloppy) ctx->sloppy = new SloppyState();
  SloppyState *s = ctx->sloppy;
  const int cap = (nrhs + gran - 1) / gran * gran;
  if (s->cap >= cap && s->cap % gran == 0) return LQCD_OK;
  cudaDeviceSynchronize();
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
    s->graph_key.clear();
  }
  cudaFree(s->sd);
  cudaFree(s->sn);
  cudaFree(s->f32);
  cudaFree(s->xdf);
  cudaFree(s->r32);
  cudaFree(s->small);
  s->sd = nullptr; s->sn = nullptr; s->f32 = nullptr; s->xdf = nullptr; s->r32 = nullptr;
  s->small = nullptr;
  s->cap = 0;
  const Geom &g = ctx->geom;
  const size_t vh = g.Vh, pairs = cap / 2;
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->sd, 7 * pairs * 6 * vh * sizeof(uint4)));
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->sn, 7 * pairs * vh * sizeof(float2)));
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->f32, 5 * (size_t)cap * 6 * vh * sizeof(float4)));
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->xdf, (size_t)cap * g.V * 12 * sizeof(float4)));
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->r32, (size_t)cap * g.V * 12 * sizeof(float2)));
  LQCD_CUDA_TRY(ctx, cudaMalloc(&s->small, small_layout(nullptr, cap, part_blocks(g.Vh)).size()));
  // padding right-hand sides of a tile are computed alongside the real ones: start them at zero
  LQCD_CUDA_TRY(ctx, cudaMemset(s->sd, 0, 7 * pairs * 6 * vh * sizeof(uint4)));
  if (!s->h_counts) LQCD_CUDA_TRY(ctx, cudaMallocHost(&s->h_counts, 16 * sizeof(int)));
  s->cap = cap;
  s->gran = gran;
  return LQCD_OK;
}

int fp64_residual_into(lqcd_ctx *ctx, const double2 *b, const double2 *x, double2 *res, int nrhs, double *rr,
                       double *bb, cudaStream_t st);

template <class SP> SP pair_field(SloppyState *st, int f, int vh);
template <> F16P pair_field<F16P>(SloppyState *st, int f, int vh) {
  size_t pairs = st->cap / 2;
  return F16P{st->sd + (size_t)f * pairs * 6 * vh, st->sn + (size_t)f * pairs * vh, vh};
}
template <> BF16P pair_field<BF16P>(SloppyState *st, int f, int vh) {
  size_t pairs = st->cap / 2;
  return BF16P{st->sd + (size_t)f * pairs * 6 * vh, vh};
}

// Compiled variants of the sloppy hopping term, picked by the autotuner:
//   0: pair layout, one pair per block, registers as the compiler wants
//   1: pair layout, one pair per block, registers capped for four 128-thread blocks per SM
//   2: pair layout, two pairs per block (256 threads), the same register cap
//   3: pair layout, four pairs per block (512 threads), the same register cap
//   4: pair layout, SU(3) products on the tensor cores (mma.sync, k_hop_mma)
//   5: RHS-tile layout (BF16 only): neighbour blocks bulk-copied into shared memory, tcgen05.mma
//      into TMEM accumulators (k_thop)
//   6: pair layout (BF16, lattices with Lx Ly / 2 = 128): one (z, t) plane per block, the five
//      neighbour planes staged in shared memory by cp.async (k_hop_pair_pl); else variant 1
//   7: variant 1 with reconstruct-12 links (rows 0 and 1 loaded, row 2 rebuilt)
constexpr int HOP_VARIANTS = 8;
constexpr int TILE_VARIANT = 5;

// autotuned launch choice per (nrhs, precision): code = blocks_per_sm * 10 + hop variant;
// LQCD_HOP_VARIANT=0..7 in the environment overrides the variant (for tests)
static int tuned_code(const lqcd_ctx *ctx, int nrhs, int precision) {
  long long key = (long long)nrhs * 8 + precision;
  int code = 80;
  for (auto &kv : ctx->tuned)
    if (kv.first == key) code = kv.second;
  const char *force = getenv("LQCD_HOP_VARIANT");
  if (force && force[0] >= '0' && force[0] < '0' + HOP_VARIANTS && force[1] == 0)
    code = code / 10 * 10 + (force[0] - '0');
  if (precision != LQCD_PREC_MIXED_BF16 && code % 10 == TILE_VARIANT) code = code / 10 * 10 + 1;  // tiles: BF16 only
  if (code % 10 == PLANE_VARIANT && !(precision == LQCD_PREC_MIXED_BF16 && planes_fit(ctx->geom)))
    code = code / 10 * 10 + 1;  // the variant that launch_hop_pair falls back to
  return code;
}

// ---------------------------------------------------------- layout policies
// The solver below is written once against these two: the pair layout (two
// right-hand sides per 16-bit pair, FP32-unit or mma.sync hop) and the tile
// layout (128 right-hand sides per tile, tcgen05 hop).
template <class SP> struct PairOps {
  using Field = SP;
  static constexpr int GS = 2;
  static int nb(int vh) { return (vh + ST - 1) / ST; }
  static int field(lqcd_ctx *, SloppyState *ss, int f, int vh, Field &out) {
    out = pair_field<SP>(ss, f, vh);
    return LQCD_OK;
  }
  static void p(cudaStream_t q, int G, int vh, const SState *sc, const Field &r, const Field &rhat, const Field &pp,
                const Field &v, const int *gl, const int *gc, int nb) {
    KL k_pair_p<SP><<<G, ST, 0, q>>>(vh, sc, r, rhat, pp, v, gl, gc, nb);
  }
  static void s(cudaStream_t q, int G, int vh, const SState *sc, const Field &r, const Field &v, const Field &s_,
                const int *gl, const int *gc, int nb) {
    KL k_pair_s<SP><<<G, ST, 0, q>>>(vh, sc, r, v, s_, gl, gc, nb);
  }
  static void xr(cudaStream_t q, int G, int vh, const SState *sc, const int *flags, F32F x, const Field &pp,
                 const Field &s_, const Field &t, const Field &r, const Field &rhat, const int *gl, const int *gc,
                 D4S *part, int nb) {
    KL k_pair_xr<SP><<<G, ST, 0, q>>>(vh, sc, flags, x, pp, s_, t, r, rhat, gl, gc, part, nb);
  }
  static void copy(cudaStream_t q, int G, int vh, const int *flags, F32F src, const Field &r, const Field &rhat,
                   bool use_rhat, F32F x, bool zero_x, const int *gl, const int *gc, D4S *part, int nb) {
    KL k_pair_copy<SP><<<G, ST, 0, q>>>(vh, flags, src, r, rhat, use_rhat, x, zero_x, gl, gc, part, nb);
  }
  template <int EPI>
  static void hop(int variant, int G, cudaStream_t q, lqcd_ctx *ctx, int p_out, const Field &in, const Field &out,
                  const Field &A, const Field &B, float cA, float cH, const int *gl, const int *gc, D4S *part, int nb,
                  int nrhs, unsigned long long *prof, int *) {
    launch_hop_pair<SP, EPI>(variant, G, q, ctx, ctx->geom, p_out, in, out, A, B, cA, cH, gl, gc, part, nb, nrhs,
                             prof);
  }
};

struct TileOps {
  using Field = TileField;
  static constexpr int GS = TR;
  static int nb(int vh) { return (vh + TCH - 1) / TCH; }
  static int field(lqcd_ctx *, SloppyState *ss, int f, int vh, Field &out) {
    const size_t per = (size_t)ss->cap * vh * 24;  // BF16 values per field
    out.d = reinterpret_cast<__nv_bfloat16 *>(ss->sd) + (size_t)f * per;
    out.ntile = ss->cap / TR;
    out.vh = vh;
    return LQCD_OK;
  }
  static void p(cudaStream_t q, int G, int vh, const SState *sc, const Field &r, const Field &rhat, const Field &pp,
                const Field &v, const int *gl, const int *gc, int) {
    tile_p(q, G, vh, sc, r, rhat, pp, v, gl, gc);
  }
  static void s(cudaStream_t q, int G, int vh, const SState *sc, const Field &r, const Field &v, const Field &s_,
                const int *gl, const int *gc, int) {
    tile_s(q, G, vh, sc, r, v, s_, gl, gc);
  }
  static void xr(cudaStream_t q, int G, int vh, const SState *sc, const int *flags, F32F x, const Field &pp,
                 const Field &s_, const Field &t, const Field &r, const Field &rhat, const int *gl, const int *gc,
                 D4S *part, int) {
    tile_xr(q, G, vh, sc, flags, x, pp, s_, t, r, rhat, gl, gc, part);
  }
  static void copy(cudaStream_t q, int G, int vh, const int *flags, F32F src, const Field &r, const Field &rhat,
                   bool use_rhat, F32F x, bool zero_x, const int *gl, const int *gc, D4S *part, int) {
    tile_copy(q, G, vh, flags, src, r, rhat, use_rhat, x, zero_x, gl, gc, part);
  }
  template <int EPI>
  static void hop(int, int, cudaStream_t q, lqcd_ctx *ctx, int p_out, const Field &in, const Field &out,
                  const Field &A, const Field &B, float cA, float cH, const int *gl, const int *gc, D4S *part, int nb,
                  int nrhs, unsigned long long *prof, int *err) {
    // one persistent CTA per SM (it allocates all TMEM columns)
    tile_hop(EPI, q, num_sms(ctx->device), ctx, p_out, in, out, A, B, cA, cH, gl, gc, part, nb, nrhs, prof, err);
  }
};

// The part of a lattice's solve that the uneven-batch driver talks to.
struct RunIface {
  bool done = false, inner = false;
  long long loop_kernels = 0;  // kernel launches per WHILE-loop iteration (set at capture)
  virtual ~RunIface() {}
  virtual int *dev_counts() = 0;
  virtual unsigned long long *dev_clock() = 0;
  virtual int max_loops() const = 0;
  virtual int init() = 0;
  virtual int cycle_start() = 0;
  virtual void launch_iters(cudaStream_t q, int k) = 0;
  virtual int request_count(cudaStream_t q) = 0;
  virtual int poll() = 0;
  virtual int finish() = 0;
  virtual std::vector<double> graph_key() const = 0;
};

// One lattice's mixed-precision solve as a resumable state machine:
//   cycle_start()    FP64 residual b - D x, per-RHS decisions, inner source
//   launch_iters()   a fixed sequence of inner BiCGstab iterations (capturable:
//                    every kernel reads its work list and counts from device memory)
//   poll()           after the stream has drained: is the inner solve over?
//   cycle_end()      odd reconstruction and x += |r| e in FP64
template <class Ops>
struct MixedRun : RunIface {
  using SF = typename Ops::Field;
  lqcd_ctx *ctx;
  const double2 *b;
  double2 *x;
  int nrhs;
  lqcd_solver_params p;
  lqcd_solve_stats *stats;
  cudaStream_t st;
  double t0;
  SloppyState *ss = nullptr;
  Geom g;
  int vh = 0, cap = 0, nbx = 0, nb = 0, G = 0, npairs = 0, hop_variant = 0;
  float kappa = 0.f, k2 = 0.f;
  double delta = 0.05, floor2 = 4e-12;  // (2e-6)^2: inner FP32 target floor, relative to |b_inner|^2
  SF r, rhat, pp, v, s, t, tmp;
  F32F x32, b32, r32, t32, o32;
  SmallBufs sb;
  std::vector<double> rr, bb, prev_rel, hscale, hun;
  std::vector<SState> hs;
  std::vector<int> hl, hp, bad, hflags, keep_status;
  int cycle = 0;
  const int max_cycles = 10;
  bool timed_out = false;
  int force_code = -1;  // launch code (blocks per SM * 10 + hop variant) chosen by the autotuner while it times
  unsigned long long budget_ns = ~0ull;  // host copy of the value sent to the device (pinned lifetime: the run)

  MixedRun(lqcd_ctx *c, const double2 *b_, double2 *x_, int n, const lqcd_solver_params &p_, lqcd_solve_stats *s_,
           cudaStream_t st_, double t0_)
      : ctx(c), b(b_), x(x_), nrhs(n), p(p_), stats(s_), st(st_), t0(t0_) {}
  int *dev_counts() override { return sb.counts; }
  unsigned long long *dev_clock() override { return sb.clk; }
  int max_loops() const override { return p.max_iter + 1; }

  int init() override {
    int rc = sloppy_alloc(ctx, nrhs, Ops::GS);
    if (rc) return rc;
    ss = ctx->sloppy;
    g = ctx->geom;
    vh = g.Vh;
    cap = ss->cap;
    nbx = (vh + ST - 1) / ST;
    nb = Ops::nb(vh);
    kappa = (float)ctx->kappa;
    k2 = (float)(ctx->kappa * ctx->kappa);
    const int code = force_code >= 0 ? force_code : tuned_code(ctx, nrhs, p.precision);
    hop_variant = code % 10;
    // tile path: the element-wise kernels use eight 256-thread blocks per SM
    G = num_sms(ctx->device) * (Ops::GS == TR ? 8 : code / 10);
    npairs = (nrhs + 1) / 2;
    delta = p.delta > 0 ? p.delta : 0.05;
    SF *f[7] = {&r, &rhat, &pp, &v, &s, &t, &tmp};
    for (int k = 0; k < 7; ++k) {
      rc = Ops::field(ctx, ss, k, vh, *f[k]);
      if (rc) return rc;
    }
    auto f32 = [&](int k) { F32F ff; ff.d = ss->f32 + (size_t)k * cap * 6 * vh; ff.vh = vh; return ff; };
    x32 = f32(0); b32 = f32(1); r32 = f32(2); t32 = f32(3); o32 = f32(4);
    sb = small_layout(ss->small, cap, part_blocks(vh));
    rr.assign(nrhs, 0.0);
    bb.assign(nrhs, 0.0);
    prev_rel.assign(nrhs, 1e300);
    hscale.assign(cap, 0.0);
    hun.assign(cap, 0.0);
    hs.assign(cap, SState{});
    bad.assign(nrhs, 0);
    hflags.assign(cap, 0);
    keep_status.assign(nrhs, 0);
    for (int k = 0; k < nrhs; ++k) stats[k] = lqcd_solve_stats{0, LQCD_OK, 0.0, 0, 0};
    const size_t n = (size_t)nrhs * g.V * 12;
    LQCD_CUDA_TRY(ctx, cudaMemsetAsync(ss->xdf, 0, n * sizeof(float4), st));
    LQCD_CUDA_TRY(ctx, cudaMemsetAsync(sb.counts, 0, 16 * sizeof(int), st));
    return LQCD_OK;
  }

  // the FP64 solution from the double-float iterate
  int finish() override { return df_join(ctx, ss->xdf, x, (size_t)nrhs * g.V * 12, st); }

  // Autotuning: ms per inner iteration of this layout and launch code, with every
  // right-hand side kept active (zero fields; a target below zero keeps them
  // from converging and from requesting reliable updates).  *herr: tile-hop error.
  float time_iterations(int reps, int *herr) {
    for (int k = 0; k < cap; ++k) {
      SState z{};
      z.rho = make_double2(1.0, 0.0);
      z.alpha = z.omega = make_double2(1.0, 0.0);
      z.target2 = -1.0;
      hs[k] = z;
      hflags[k] = k < nrhs ? FLAG_ACTIVE : 0;
    }
    const size_t sloppy_bytes = (size_t)7 * (cap / 2) * 6 * vh * sizeof(uint4);
    if (cudaMemsetAsync(ss->sd, 0, sloppy_bytes, st) != cudaSuccess ||
        cudaMemsetAsync(ss->f32, 0, (size_t)5 * cap * 6 * vh * sizeof(float4), st) != cudaSuccess ||
        cudaMemcpyAsync(sb.sc, hs.data(), cap * sizeof(SState), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(sb.flags, hflags.data(), cap * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return -1.f;
    KL k_build_lists<<<1, 1024, 0, st>>>(nrhs, sb.flags, Ops::GS, sb.act_pairs, sb.ru_list, sb.ru_pairs, sb.counts);
    launch_iters(st, 1);  // warm-up
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    launch_iters(st, reps);
    cudaEventRecord(e1, st);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) == cudaSuccess) {
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemcpy(herr, sb.counts + 8, sizeof(int), cudaMemcpyDeviceToHost);
    return ms;
  }

  // key of the captured iteration graph: everything its kernels capture by value
  std::vector<double> graph_key() const override {
    return {(double)nrhs, (double)p.precision, (double)p.max_iter, delta, (double)kappa, (double)G, (double)hop_variant,
            (double)Ops::GS, (double)(uintptr_t)ss->sd, (double)(uintptr_t)ss->f32, (double)(uintptr_t)ss->small,
            (double)(uintptr_t)ctx->U16, (double)(uintptr_t)ctx->U32, (double)(uintptr_t)ctx->Ub16,
            (double)(uintptr_t)ss->xdf, (double)cap};
  }

  int cycle_start() override {
    // at x = 0 the residual is b itself (FP64 norms only); later: double-float
    // b - D x for the right-hand sides corrected in the previous cycle (the
    // others' iterates, and so their residuals, have not changed)
    std::vector<int> todo;
    if (cycle == 0) {
      todo.resize(nrhs);
      for (int k = 0; k < nrhs; ++k) todo[k] = k;
    } else {
      todo = hl;
    }
    int rc = cycle == 0 ? fp64_residual_into(ctx, b, nullptr, nullptr, nrhs, rr.data(), bb.data(), st)
                        : df_residual(ctx, ss->xdf, b, ss->r32, todo.data(), (int)todo.size(), rr.data(),
                                      bb.data(), st);
    if (rc) return rc;
    hl.clear();
    hp.clear();
    std::fill(hflags.begin(), hflags.end(), 0);
    std::fill(hscale.begin(), hscale.end(), 0.0);
    std::fill(hun.begin(), hun.end(), 0.0);
    for (int k : todo) {
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
        else if (rel > 0.5 * prev_rel[k] && ++bad[k] >= 3) status = LQCD_ERR_NOT_CONVERGED;
      }
      prev_rel[k] = rel;
      stats[k].status = status;
      hs[k].status = status;
      if (status == LQCD_OK && rel > p.tol) {
        hl.push_back(k);
        if (hp.empty() || hp.back() != k / Ops::GS) hp.push_back(k / Ops::GS);
        hscale[k] = 1.0 / std::sqrt(rr[k]);
        hun[k] = std::sqrt(rr[k]);
        hs[k].target2 = 0.25 * p.tol * p.tol * bb[k] / rr[k];
        hflags[k] = FLAG_RU;  // marks the members whose inner source is loaded below
      }
    }
    if (hl.empty() || timed_out) {
      done = true;
      return LQCD_OK;
    }
    int *counts = sb.counts;
    int hc[5] = {0, 0, (int)hl.size(), 0, (int)hp.size()};
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sb.cyc_list, hl.data(), hl.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sb.cyc_pairs, hp.data(), hp.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(counts, hc, sizeof(hc), cudaMemcpyHostToDevice, st));
    // wall-clock budget left for this cycle's inner loop, in ns (the loop's own check)
    budget_ns = ~0ull;
    if (p.timeout_ms > 0) {
      const double left = p.timeout_ms - (wall_ms() - t0);
      budget_ns = left > 0 ? (unsigned long long)(left * 1e6) : 0ull;
    }
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sb.clk + 1, &budget_ns, sizeof(budget_ns), cudaMemcpyHostToDevice, st));
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sb.scale, hscale.data(), cap * sizeof(double), cudaMemcpyHostToDevice, st));
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sb.unscale, hun.data(), cap * sizeof(double), cudaMemcpyHostToDevice, st));
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sb.sc, hs.data(), cap * sizeof(SState), cudaMemcpyHostToDevice, st));
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sb.flags, hflags.data(), cap * sizeof(int), cudaMemcpyHostToDevice, st));
    // inner right-hand side: b32 = scale (r_e + kappa H_eo r_o), o32 = scale r_o
    if (cycle == 0) {
      KL k_cvt64to32_both<<<G, ST, 0, st>>>(g, b, b32, o32, sb.scale, sb.cyc_list, counts + 2, nbx);
    } else {
      KL k_cvt32to32_both<<<G, ST, 0, st>>>(g, ss->r32, b32, o32, sb.scale, sb.cyc_list, counts + 2, nbx);
    }
    KL k_hop32x2<EPI_AXPY><<<G, ST, 0, st>>>(g, 0, ctx->U32, o32, b32, b32, b32, 1.f, 0.f, kappa, sb.cyc_list,
                                           counts + 2, nullptr, nbx);
    Ops::copy(st, G, vh, sb.flags, b32, r, r, false, x32, true, sb.cyc_pairs, counts + 4, sb.part, nb);
    KL k_sfin_init<<<(int)hl.size(), 32, 0, st>>>(sb.sc, sb.flags, sb.cyc_list, counts + 2, sb.part, nb, floor2);
    KL k_build_lists<<<1, 1024, 0, st>>>(nrhs, sb.flags, Ops::GS, sb.act_pairs, sb.ru_list, sb.ru_pairs, counts);
    LQCD_LAUNCH_CHECK(ctx, "mixed: cycle setup");
    inner = true;
    return LQCD_OK;
  }

  // Enqueue k inner iterations on stream q (RHS that finish simply drop out of the lists).
  void launch_iters(cudaStream_t q, int k) override {
    int *counts = sb.counts;
    const float4 *L32 = ctx->U32;
    unsigned long long *prof = ctx->prof_on ? ctx->d_prof : nullptr;
    int *herr = counts + 8;
    if (ctx->prof_on) ctx->prof_prec = p.precision;
    auto ev_begin = [&]() {
      if (!ctx->prof_on) return;
      while (ctx->prof_used + 2 > ctx->prof_ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { ctx->prof_on = false; return; }
        ctx->prof_ev.push_back(e);
      }
      cudaEventRecord(ctx->prof_ev[ctx->prof_used], q);
    };
    auto ev_end = [&]() {
      if (!ctx->prof_on) return;
      cudaEventRecord(ctx->prof_ev[ctx->prof_used + 1], q);
      ctx->prof_used += 2;
      ctx->prof_hop_launches++;
    };
    const int gs = Ops::GS;
    for (int it = 0; it < k; ++it) {
      Ops::p(q, G, vh, sb.sc, r, rhat, pp, v, sb.act_pairs, counts, nb);
      ev_begin();
      Ops::template hop<EPI_PLAIN>(hop_variant, G, q, ctx, 1, pp, tmp, tmp, tmp, 0.f, 1.f, sb.act_pairs, counts,
                                   nullptr, nb, nrhs, prof, herr);
      ev_end();
      ev_begin();
      Ops::template hop<EPI_DOTR>(hop_variant, G, q, ctx, 0, tmp, v, pp, rhat, 1.f, -k2, sb.act_pairs, counts, sb.part,
                                  nb, nrhs, prof, herr);
      ev_end();
      KL k_sfin_alpha<<<cap / 2, 64, 0, q>>>(sb.sc, sb.flags, sb.act_pairs, counts, sb.part, nb, nrhs, gs);
      Ops::s(q, G, vh, sb.sc, r, v, s, sb.act_pairs, counts, nb);
      ev_begin();
      Ops::template hop<EPI_PLAIN>(hop_variant, G, q, ctx, 1, s, tmp, tmp, tmp, 0.f, 1.f, sb.act_pairs, counts,
                                   nullptr, nb, nrhs, prof, herr);
      ev_end();
      ev_begin();
      Ops::template hop<EPI_TS>(hop_variant, G, q, ctx, 0, tmp, t, s, s, 1.f, -k2, sb.act_pairs, counts, sb.part, nb,
                                nrhs, prof, herr);
      ev_end();
      KL k_sfin_omega<<<cap / 2, 64, 0, q>>>(sb.sc, sb.flags, sb.act_pairs, counts, sb.part, nb, nrhs, gs);
      Ops::xr(q, G, vh, sb.sc, sb.flags, x32, pp, s, t, r, rhat, sb.act_pairs, counts, sb.part, nb);
      KL k_sfin_conv<<<cap / 2, 64, 0, q>>>(sb.sc, sb.flags, sb.act_pairs, counts, sb.part, nb, nrhs,
                                            delta * delta, p.max_iter, gs);
      KL k_build_lists<<<1, 1024, 0, q>>>(nrhs, sb.flags, gs, sb.act_pairs, sb.ru_list, sb.ru_pairs, counts);
      // reliable update in FP32: r32 = b32 - x32 + kappa^2 H_eo H_oe x32
      KL k_hop32x2<EPI_PLAIN><<<G, ST, 0, q>>>(g, 1, L32, x32, t32, t32, t32, 0.f, 0.f, 1.f, sb.ru_list, counts + 1,
                                             nullptr, nbx);
      KL k_hop32x2<EPI_RES><<<G, ST, 0, q>>>(g, 0, L32, t32, r32, b32, x32, 1.f, -1.f, k2, sb.ru_list, counts + 1,
                                           sb.part, nbx);
      KL k_sfin_ru<<<nrhs, 32, 0, q>>>(sb.sc, sb.flags, sb.ru_list, counts + 1, sb.part, nbx, p.max_iter);
      KL k_build_lists<<<1, 1024, 0, q>>>(nrhs, sb.flags, gs, sb.act_pairs, sb.ru_list, sb.ru_pairs, counts);
      Ops::copy(q, G, vh, sb.flags, r32, r, rhat, true, x32, false, sb.ru_pairs, counts + 3, sb.part, nb);
      KL k_sfin_ru2<<<nrhs, 32, 0, q>>>(sb.sc, sb.flags, sb.ru_list, counts + 1, sb.part, nb);
      KL k_build_lists<<<1, 1024, 0, q>>>(nrhs, sb.flags, gs, sb.act_pairs, sb.ru_list, sb.ru_pairs, counts);
    }
  }

  // enqueue the read-back of the active count, the tile hop's error code and
  // the device loop's budget flag and iteration count
  int request_count(cudaStream_t q) override {
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(ss->h_counts, sb.counts, 11 * sizeof(int), cudaMemcpyDeviceToHost, q));
    return LQCD_OK;
  }

  // with the stream drained: finish the cycle if no RHS is active any more
  int poll() override {
    if (ss->h_counts[8] != 0)
      return set_error(ctx, LQCD_ERR_CUDA,
                       "mixed: the tensor-core hop stopped after a bounded wait ran out (code %d)", ss->h_counts[8]);
    bool any = ss->h_counts[0] > 0;
    if (any && ss->h_counts[9]) {  // the device loop stopped on the time budget
      timed_out = true;
      any = false;
    }
    if (any && p.timeout_ms > 0 && wall_ms() - t0 > p.timeout_ms) {
      timed_out = true;
      any = false;
    }
    if (!any) return cycle_end();
    return LQCD_OK;
  }

  int cycle_end() {
    int *counts = sb.counts;
    // odd half of the correction: e_o = o32 + kappa H_oe x32; x += |r| e
    KL k_hop32x2<EPI_AXPY><<<G, ST, 0, st>>>(g, 1, ctx->U32, x32, o32, o32, o32, 1.f, 0.f, kappa, sb.cyc_list,
                                           counts + 2, nullptr, nbx);
    KL k_accum_df_both<<<G, ACC_SITES * 2, 0, st>>>(g, x32, o32, ss->xdf, sb.unscale, sb.cyc_list, counts + 2,
                                                    (vh + ACC_SITES - 1) / ACC_SITES);
    LQCD_LAUNCH_CHECK(ctx, "mixed: correction");
    for (int k = 0; k < nrhs; ++k) keep_status[k] = hs[k].status;
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(hs.data(), sb.sc, cap * sizeof(SState), cudaMemcpyDeviceToHost, st));
    LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    for (int k = 0; k < nrhs; ++k)
      if (!std::binary_search(hl.begin(), hl.end(), k)) hs[k].status = keep_status[k];
    inner = false;
    ++cycle;
    return LQCD_OK;
  }
};

static RunIface *make_run(lqcd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const lqcd_solver_params &p,
                          lqcd_solve_stats *stats, cudaStream_t st, double t0) {
  if (p.precision == LQCD_PREC_MIXED_FP16) return new MixedRun<PairOps<F16P>>(ctx, b, x, nrhs, p, stats, st, t0);
  if (tuned_code(ctx, nrhs, p.precision) % 10 == TILE_VARIANT)
    return new MixedRun<TileOps>(ctx, b, x, nrhs, p, stats, st, t0);
  return new MixedRun<PairOps<BF16P>>(ctx, b, x, nrhs, p, stats, st, t0);
}

// capture `body(stream)` into an executable graph on stream st; *kernels
// receives the number of kernel launches the body recorded (each replay makes
// them; the capture itself launches nothing, so the library's launch counter
// is set back)
template <class F>
static cudaError_t capture_graph(cudaStream_t st, F body, cudaGraphExec_t *exec, long long *kernels) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const long long before = g_launches.load();
  body(st);
  *kernels = g_launches.load() - before;
  g_launches -= *kernels;
  e = cudaStreamEndCapture(st, &graph);
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

constexpr int ITERS_PER_POLL = 4;  // inner iterations per host poll when launching directly (profiling)

// Append to graph g, for one lattice: k_loop_init -> WHILE node whose body is
// one inner iteration followed by k_loop_cond.  The body is recorded by
// capturing launch_iters on st into the conditional node's child graph.
static cudaError_t add_cycle_loop(cudaGraph_t g, RunIface *run, cudaStream_t st) {
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
  if (e != cudaSuccess) return e;
  int *counts = run->dev_counts();
  unsigned long long *clk = run->dev_clock();
  void *init_args[] = {&h, &counts, &clk};
  cudaKernelNodeParams kp = {};
  kp.func = (void *)k_loop_init;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.kernelParams = init_args;
  cudaGraphNode_t init_node, loop_node;
  e = cudaGraphAddKernelNode(&init_node, g, nullptr, 0, &kp);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  e = cudaGraphAddNode(&loop_node, g, &init_node, nullptr, 1, &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const long long before = g_launches.load();
  run->launch_iters(st, 1);
  KL k_loop_cond<<<1, 1, 0, st>>>(h, counts, clk, run->max_loops());
  run->loop_kernels = g_launches.load() - before;
  g_launches -= run->loop_kernels;  // recording launches nothing
  return cudaStreamEndCapture(st, &body);
}

// the library's launch counter after a replay: the init kernel plus the kernels
// of every loop iteration the device ran (read back in h_counts[10])
static void count_loop_launches(RunIface *run, const SloppyState *ss) {
  g_launches += 1 + run->loop_kernels * (long long)ss->h_counts[10];
}

// Single lattice: each outer cycle's inner loop is one launch of a CUDA graph
// holding a WHILE node (the device decides when to stop), captured once per
// configuration; the host synchronises once per cycle.  While profiling the
// iterations are launched directly, four per host poll, so that every hop
// launch gets its own events.
// Revision of the tuned layout after a solve.  The autotuner times inner
// iterations with every right-hand side active, but a layout keeps computing a
// group -- a pair (2 RHS) or a tile (TR RHS) -- until its slowest member has
// converged.  With the solve's per-RHS iteration counts, a layout's cost is its
// time per full iteration times sum_groups(size x max iterations in the group) /
// (its groups' total size); the cheaper layout becomes the choice for the key.
static void revise_layout(lqcd_ctx *ctx, int nrhs, int precision, const lqcd_solve_stats *stats) {
  const long long key = (long long)nrhs * 8 + precision;
  const lqcd_ctx::TuneRec *t = nullptr;
  for (auto &r : ctx->tune_ms)
    if (r.key == key) t = &r;
  if (!t || t->tile_ms < 0.f) return;
  auto weighted = [&](int gsz) {
    double w = 0.0;
    for (int g0 = 0; g0 < nrhs; g0 += gsz) {
      int m = 0;
      for (int i = g0; i < std::min(nrhs, g0 + gsz); ++i) m = std::max(m, stats[i].iterations);
      w += (double)gsz * m;
    }
    return w / (double)(((nrhs + gsz - 1) / gsz) * gsz);
  };
  const double pair_cost = t->pair_ms * weighted(2), tile_cost = t->tile_ms * weighted(TR);
  const int code = tile_cost < pair_cost ? 10 + TILE_VARIANT : t->pair_code;
  for (auto &kv : ctx->tuned)
    if (kv.first == key) kv.second = code;
}

static int mixed_block(lqcd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const lqcd_solver_params &p,
                       lqcd_solve_stats *stats, cudaStream_t st, double t0) {
  std::unique_ptr<RunIface> run(make_run(ctx, b, x, nrhs, p, stats, st, t0));
  int rc = run->init();
  if (rc) return rc;
  SloppyState *ss = ctx->sloppy;
  // the legacy default stream cannot be captured: launch directly there
  const bool use_graph = !ctx->prof_on && st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread &&
                         getenv("LQCD_NO_GRAPH") == nullptr;
  while (!run->done) {
    if (!run->inner) {
      rc = run->cycle_start();
      if (rc) return rc;
      continue;
    }
    if (use_graph) {
      std::vector<double> key = run->graph_key();
      if (!ss->graph || ss->graph_key != key) {
        if (ss->graph) cudaGraphExecDestroy(ss->graph);
        ss->graph = nullptr;
        cudaGraph_t g = nullptr;
        LQCD_CUDA_TRY(ctx, cudaGraphCreate(&g, 0));
        cudaError_t e = add_cycle_loop(g, run.get(), st);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ss->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          ss->graph = nullptr;
          return cuda_error(ctx, e, "mixed: capture of the inner-loop graph");
        }
        ss->graph_key = key;
        ss->graph_kernels = run->loop_kernels;
      }
      run->loop_kernels = ss->graph_kernels;
      LQCD_CUDA_TRY(ctx, cudaGraphLaunch(ss->graph, st));
    } else {
      run->launch_iters(st, ITERS_PER_POLL);
      LQCD_LAUNCH_CHECK(ctx, "mixed: iteration");
    }
    rc = run->request_count(st);
    if (rc) return rc;
    LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (use_graph) count_loop_launches(run.get(), ss);
    rc = run->poll();
    if (rc) return rc;
  }
  rc = run->finish();
  if (p.precision == LQCD_PREC_MIXED_BF16) revise_layout(ctx, nrhs, p.precision, stats);
  return rc;
}

// Uneven batch: one CUDA graph with a branch per lattice (k_loop_init -> WHILE
// node), so that one launch runs every lattice's inner loop of the current
// outer cycle concurrently; each lattice's outer refinement runs between
// launches.
static int mixed_batch(std::vector<lqcd_ctx *> &ctxs, std::vector<const double2 *> &bs, std::vector<double2 *> &xs,
                       std::vector<int> &ns, const lqcd_solver_params &p, std::vector<lqcd_solve_stats *> &stats,
                       cudaStream_t st, std::vector<cudaStream_t> &side, cudaGraphExec_t *gexec,
                       std::vector<double> *gkey, long long *gkernels) {
  (void)side;
  (void)gkernels;
  const size_t nl = ctxs.size();
  const double t0 = wall_ms();
  std::vector<std::unique_ptr<RunIface>> runs;
  for (size_t l = 0; l < nl; ++l) runs.emplace_back(make_run(ctxs[l], bs[l], xs[l], ns[l], p, stats[l], st, t0));
  for (auto &r : runs) {
    int rc = r->init();
    if (rc) return rc;
  }
  std::vector<long long> per_iter(nl, 0);
  const bool direct = getenv("LQCD_NO_GRAPH") != nullptr;  // launches visible to kernel profilers
  for (;;) {
    bool any = false;
    for (auto &r : runs) {
      while (!r->done && !r->inner) {
        int rc = r->cycle_start();
        if (rc) return rc;
      }
      any = any || !r->done;
    }
    if (!any) break;
    if (direct) {
      for (auto &r : runs)
        if (!r->done) {
          r->launch_iters(st, ITERS_PER_POLL);
          int rc = r->request_count(st);
          if (rc) return rc;
        }
      LQCD_CUDA_TRY(ctxs[0], cudaStreamSynchronize(st));
      for (auto &r : runs)
        if (!r->done && r->inner) {
          int rc = r->poll();
          if (rc) return rc;
        }
      continue;
    }
    std::vector<double> key;
    for (auto &r : runs) {
      std::vector<double> k = r->graph_key();
      key.insert(key.end(), k.begin(), k.end());
    }
    if (!*gexec || *gkey != key) {
      if (*gexec) cudaGraphExecDestroy(*gexec);
      *gexec = nullptr;
      cudaGraph_t g = nullptr;
      LQCD_CUDA_TRY(ctxs[0], cudaGraphCreate(&g, 0));
      cudaError_t e = cudaSuccess;
      for (size_t l = 0; l < nl && e == cudaSuccess; ++l) {
        e = add_cycle_loop(g, runs[l].get(), st);
        per_iter[l] = runs[l]->loop_kernels;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        *gexec = nullptr;
        return cuda_error(ctxs[0], e, "batch: capture of the inner-loop graph");
      }
      *gkey = key;
    }
    LQCD_CUDA_TRY(ctxs[0], cudaGraphLaunch(*gexec, st));
    for (auto &r : runs) {
      int rc = r->request_count(st);
      if (rc) return rc;
    }
    LQCD_CUDA_TRY(ctxs[0], cudaStreamSynchronize(st));
    for (size_t l = 0; l < nl; ++l) {
      runs[l]->loop_kernels = per_iter[l];
      count_loop_launches(runs[l].get(), ctxs[l]->sloppy);
    }
    for (auto &r : runs)
      if (!r->done && r->inner) {
        int rc = r->poll();
        if (rc) return rc;
      }
  }
  for (auto &r : runs) {
    int rc = r->finish();
    if (rc) return rc;
  }
  return LQCD_OK;
}

int mixed_solve(lqcd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const lqcd_solver_params &p,
                lqcd_solve_stats *stats, cudaStream_t st) {
  if (p.solver != LQCD_SOLVER_BICGSTAB)
    return set_error(ctx, LQCD_ERR_INVALID, "the CG solver is available with LQCD_PREC_FP64 only");
  if (!ctx->gauge_su3)
    return set_error(ctx, LQCD_ERR_INVALID,
                     "mixed precision needs SU(3) links (the FP32 copy is reconstruct-12); this gauge field was set with "
                     "lqcd_set_gauge_general: use LQCD_PREC_FP64");
  int blk = p.rhs_block > 0 ? p.rhs_block : nrhs;
  if (blk > 4096) blk = 4096;
  double t0 = wall_ms();
  size_t full = (size_t)ctx->geom.V * 12;
  int worst = LQCD_OK;
  for (int k0 = 0; k0 < nrhs; k0 += blk) {
    int nk = std::min(blk, nrhs - k0);
    int rc = mixed_block(ctx, b + k0 * full, x + k0 * full, nk, p, stats + k0, st, t0);
    if (rc) return rc;
    for (int k = 0; k < nk; ++k)
      if (worst == LQCD_OK && stats[k0 + k].status != LQCD_OK) worst = stats[k0 + k].status;
  }
  if (worst != LQCD_OK) set_error(ctx, worst, "lqcd_solve_batch: some right-hand sides did not converge");
  return worst;
}

}  // namespace lqcd

// ================================================================ batch ABI
struct lqcd_batch {
  struct Entry {
    lqcd_ctx *ctx;
    const double2 *b;
    double2 *x;
    int nrhs;
  };
  std::vector<Entry> entries;
  std::vector<cudaStream_t> side;
  cudaGraphExec_t graph = nullptr;
  std::vector<double> graph_key;
  long long graph_kernels = 0;
  std::string err;
};

using namespace lqcd;

extern "C" {

int lqcd_batch_create(lqcd_batch **out) {
  LQCD_TRACE("lqcd_batch_create");
  if (!out) return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_batch_create: null argument");
  *out = new lqcd_batch();
  return LQCD_OK;
}

int lqcd_batch_destroy(lqcd_batch *batch) {
  LQCD_TRACE("lqcd_batch_destroy");
  if (!batch) return LQCD_OK;
  if (batch->graph) cudaGraphExecDestroy(batch->graph);
  for (cudaStream_t s : batch->side) cudaStreamDestroy(s);
  delete batch;
  return LQCD_OK;
}

int lqcd_batch_add(lqcd_batch *batch, lqcd_ctx *ctx, const double *b, double *x, int nrhs) {
  LQCD_TRACE("lqcd_batch_add");
  if (!batch || !ctx || nrhs <= 0 || !b || !x) return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_batch_add: bad argument");
  if (!is_device_ptr(b) || !is_device_ptr(x))
    return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_batch_add: b and x must be device memory");
  for (auto &e : batch->entries)
    if (e.ctx == ctx) return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_batch_add: one entry per context");
  if (!batch->entries.empty() && batch->entries[0].ctx->device != ctx->device)
    return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_batch_add: all lattices must be on one device");
  batch->entries.push_back({ctx, (const double2 *)b, (double2 *)x, nrhs});
  return LQCD_OK;
}

int lqcd_batch_rhs(const lqcd_batch *batch, int *total) {
  if (!batch || !total) return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_batch_rhs: null argument");
  long long n = 0;
  for (auto &e : batch->entries) n += e.nrhs;
  *total = (int)std::min<long long>(n, 0x7fffffff);
  return LQCD_OK;
}

int lqcd_batch_run(lqcd_batch *batch, const lqcd_solver_params *params, lqcd_solve_stats *stats, int n_stats,
                   lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_batch_run");
  if (!batch || !params || (!stats && n_stats > 0))
    return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_batch_run: null argument");
  {
    long long total = 0;
    for (auto &e : batch->entries) total += e.nrhs;
    if ((long long)n_stats < total)
      return set_error(nullptr, LQCD_ERR_INVALID,
                       "lqcd_batch_run: stats holds %d records, the batch has %lld right-hand sides", n_stats, total);
  }
  if (batch->entries.empty()) return LQCD_OK;
  const lqcd_solver_params &p = *params;
  if (!(p.tol > 0.0) || p.max_iter <= 0 || p.precision < LQCD_PREC_FP64 || p.precision > LQCD_PREC_MIXED_BF16)
    return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_batch_run: bad solver parameters");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(batch->entries[0].ctx->device);
  std::vector<lqcd_ctx *> ctxs;
  std::vector<const double2 *> bs;
  std::vector<double2 *> xs;
  std::vector<int> ns;
  std::vector<lqcd_solve_stats *> sts;
  size_t off = 0;
  for (auto &e : batch->entries) {
    if (!e.ctx->have_gauge) return set_error(e.ctx, LQCD_ERR_NO_GAUGE, "lqcd_batch_run: no gauge field");
    ctxs.push_back(e.ctx);
    bs.push_back(e.b);
    xs.push_back(e.x);
    ns.push_back(e.nrhs);
    sts.push_back(stats + off);
    off += e.nrhs;
  }
  int rc = LQCD_OK;
  if (p.precision == LQCD_PREC_FP64) {
    for (size_t l = 0; l < ctxs.size() && rc == LQCD_OK; ++l) {
      rc = fp64_solve(ctxs[l], bs[l], xs[l], ns[l], p, sts[l], st);
      if (rc == LQCD_ERR_NOT_CONVERGED || rc == LQCD_ERR_NONFINITE || rc == LQCD_ERR_TIMEOUT ||
          rc == LQCD_ERR_BREAKDOWN)
        rc = LQCD_OK;  // per-RHS statuses are reported in stats
    }
  } else {
    if (p.solver != LQCD_SOLVER_BICGSTAB)
      return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_batch_run: CG is available with LQCD_PREC_FP64 only");
    for (auto *c : ctxs)
      if (!c->gauge_su3)
        return set_error(c, LQCD_ERR_INVALID, "lqcd_batch_run: mixed precision needs SU(3) links");
    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread)
      return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_batch_run: pass a created stream (the graph is captured on it)");
    while (batch->side.size() < ctxs.size()) {
      cudaStream_t s;
      LQCD_CUDA_TRY(ctxs[0], cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      batch->side.push_back(s);
    }
    rc = mixed_batch(ctxs, bs, xs, ns, p, sts, st, batch->side, &batch->graph, &batch->graph_key,
                     &batch->graph_kernels);
  }
  if (rc) {
    set_error(nullptr, rc, "lqcd_batch_run: %s", lqcd_last_error(ctxs[0]));
    return rc;
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(nullptr, e, "lqcd_batch_run: sync");
  int worst = LQCD_OK;
  for (size_t k = 0; k < off; ++k)
    if (worst == LQCD_OK && stats[k].status != LQCD_OK) worst = stats[k].status;
  return worst;
}

}  // extern "C"

// ================================================================ autotuner
namespace lqcd {

// Autotuner: every candidate layout and launch code is timed on what the solver
// runs -- inner BiCGstab iterations (the four hop launches with their epilogues,
// the layout's Krylov updates, finalisers and list builds) -- on the context's
// gauge field with nrhs right-hand sides, so that a faster hopping term that
// brings slower updates is not chosen.
template <class Ops>
static int time_code(lqcd_ctx *ctx, int nrhs, int precision, int code, float *ms_out) {
  lqcd_solver_params p{};
  p.tol = 1e-10;
  p.max_iter = 1 << 30;
  p.precision = precision;
  p.delta = 0.05;
  std::vector<lqcd_solve_stats> stats(nrhs);
  MixedRun<Ops> run(ctx, nullptr, nullptr, nrhs, p, stats.data(), (cudaStream_t)0, wall_ms());
  run.force_code = code;
  int rc = run.init();
  if (rc) return rc;
  int herr = 0;
  *ms_out = run.time_iterations(3, &herr);
  if (*ms_out < 0.f) return cuda_error(ctx, cudaGetLastError(), "lqcd_autotune: timing");
  if (herr) *ms_out = 1e30f;  // a tile hop that reported a wait that ran out is never chosen
  return LQCD_OK;
}

template <class SP>
static int autotune_hop(lqcd_ctx *ctx, int nrhs, int precision, int *best, int *best_variant) {
  const bool tiles = std::is_same<SP, BF16P>::value;
  // one allocation serves both layouts (a capacity in whole tiles is also whole pairs)
  int rc = sloppy_alloc(ctx, nrhs, tiles ? TR : 2);
  if (rc) return rc;
  const int cand[8] = {2, 4, 8, 16, 32, 64, 128, 256};
  const bool verbose = getenv("LQCD_AUTOTUNE_VERBOSE") != nullptr;  // timings to stderr
  float best_ms = 1e30f;
  int best_code = 80;
  auto consider = [&](int code, float ms) {
    if (verbose)
      fprintf(stderr, "lqcd_autotune: nrhs %d variant %d blocks/SM %d: %.4f ms per inner iteration\n", nrhs,
              code % 10, code / 10, ms);
    if (ms < best_ms) {
      best_ms = ms;
      best_code = code;
    }
  };
  for (int variant = 0; variant < HOP_VARIANTS; ++variant) {
    if (variant == TILE_VARIANT || (variant == PLANE_VARIANT && !(tiles && planes_fit(ctx->geom)))) continue;
    for (int c : cand) {
      float ms = 0.f;
      rc = time_code<PairOps<SP>>(ctx, nrhs, precision, c * 10 + variant, &ms);
      if (rc) return rc;
      consider(c * 10 + variant, ms);
    }
  }
  const int pair_code = best_code;
  const float pair_ms = best_ms;
  float tile_ms = -1.f;
  if (tiles) {
    rc = time_code<TileOps>(ctx, nrhs, precision, 10 + TILE_VARIANT, &tile_ms);
    if (rc) return rc;
    consider(10 + TILE_VARIANT, tile_ms);
  }
  long long key = (long long)nrhs * 8 + precision;
  bool rec = false;
  for (auto &t : ctx->tune_ms)
    if (t.key == key) {
      t = lqcd_ctx::TuneRec{key, pair_code, pair_ms, tile_ms};
      rec = true;
    }
  if (!rec) ctx->tune_ms.push_back(lqcd_ctx::TuneRec{key, pair_code, pair_ms, tile_ms});
  bool found = false;
  for (auto &kv : ctx->tuned)
    if (kv.first == key) {
      kv.second = best_code;
      found = true;
    }
  if (!found) ctx->tuned.push_back({key, best_code});
  if (best) *best = best_code / 10;
  if (best_variant) *best_variant = best_code % 10;
  return LQCD_OK;
}

}  // namespace lqcd

extern "C" int lqcd_tuned_choice(const lqcd_ctx *ctx, int nrhs, int precision, int *blocks_per_sm,
                                 int *hop_variant) {
  LQCD_TRACE("lqcd_tuned_choice");
  if (!ctx) return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_tuned_choice: null context");
  const int code = tuned_code(ctx, nrhs, precision);
  if (blocks_per_sm) *blocks_per_sm = code / 10;
  if (hop_variant) *hop_variant = code % 10;
  return LQCD_OK;
}

extern "C" int lqcd_autotune(lqcd_ctx *ctx, int nrhs, int precision, int *best_blocks_per_sm,
                             int *best_hop_variant) {
  LQCD_TRACE("lqcd_autotune");
  if (!ctx || nrhs <= 0 || nrhs > 4096) return set_error(ctx, LQCD_ERR_INVALID, "lqcd_autotune: bad argument");
  if (!ctx->have_gauge || !ctx->gauge_su3) return set_error(ctx, LQCD_ERR_NO_GAUGE, "lqcd_autotune: needs an SU(3) gauge field");
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (precision == LQCD_PREC_MIXED_FP16)
    return autotune_hop<F16P>(ctx, nrhs, precision, best_blocks_per_sm, best_hop_variant);
  if (precision == LQCD_PREC_MIXED_BF16)
    return autotune_hop<BF16P>(ctx, nrhs, precision, best_blocks_per_sm, best_hop_variant);
  return set_error(ctx, LQCD_ERR_INVALID, "lqcd_autotune: only the mixed-precision paths are tuned");
}
