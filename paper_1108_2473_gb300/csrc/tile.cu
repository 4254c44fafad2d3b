// RHS-tile path of the mixed-precision solver (Sec. II: mixed-precision
// BiCGstab for the all-to-all inversions): BF16 sloppy fields in 128-RHS tiles
// (layout in tile.cuh), the tensor-core hopping term, the element-wise Krylov
// updates on tiles, and the BF16 link bundle the hop reads.
#include <algorithm>
#include <cstring>

#include "tile.cuh"
#include "tile_api.cuh"

namespace lqcd {

// ============================================================ link bundle
// For output parity p and parity-local site i, the eight colour matrices C_d of
// the hopping term, d = 2 mu + (0 forward, 1 backward):
//   forward  C = U_mu(x)          (-1 if mu = t and x_t = Lt - 1)
//   backward C = U_mu(x - mu)^+   (-1 if mu = t and x_t = 0)
// stored as BF16 (re, im) pairs: [2 parity][Vh][8 d][3][3] uint32.
__global__ void k_pack_links_bf16(const double2 *__restrict__ U, Geom g, uint32_t *out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // (p, i, d)
  if (idx >= g.V * 8) return;
  const int d = idx & 7, pi = idx >> 3;
  const int p = pi / g.Vh, i = pi % g.Vh;
  int c[4];
  coords_of(g, p, i, c);
  const int mu = d >> 1;
  const bool fwd = (d & 1) == 0;
  int cl[4] = {c[0], c[1], c[2], c[3]};
  double sign = 1.0;
  if (!fwd) cl[mu] = (c[mu] == 0) ? g.L[mu] - 1 : c[mu] - 1;
  if (mu == 3 && ((fwd && c[3] == g.L[3] - 1) || (!fwd && c[3] == 0))) sign = -1.0;
  const double2 *u = U + ((size_t)site_of(g, cl) * 4 + mu) * 9;
  uint32_t *o = out + (size_t)idx * 9;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // forward: C[a][b] = U[a][b]; backward: C[a][b] = conj(U[b][a])
      const double2 v = fwd ? u[a * 3 + b] : make_double2(u[b * 3 + a].x, -u[b * 3 + a].y);
      const __nv_bfloat16 re = __double2bfloat16(sign * v.x), im = __double2bfloat16(sign * v.y);
      o[a * 3 + b] = (uint32_t)__bfloat16_as_ushort(re) | ((uint32_t)__bfloat16_as_ushort(im) << 16);
    }
}

int pack_gauge_sloppy(lqcd_ctx *ctx, cudaStream_t st) {
  const Geom &g = ctx->geom;
  if (!ctx->Ub16) LQCD_CUDA_TRY(ctx, cudaMalloc(&ctx->Ub16, (size_t)g.V * 8 * 9 * sizeof(uint32_t)));
  const int threads = 256, blocks = (g.V * 8 + threads - 1) / threads;
  KL k_pack_links_bf16<<<blocks, threads, 0, st>>>(ctx->U64, g, ctx->Ub16);
  LQCD_LAUNCH_CHECK(ctx, "k_pack_links_bf16");
  return LQCD_OK;
}

// =========================================================== host tables
// P_d = 1 - gamma_mu (forward) or 1 + gamma_mu (backward), DeGrand-Rossi basis:
// each row has the identity and one off-diagonal entry in {+-1, +-i}.
static TSpin make_spin_table() {
  // gamma_mu[s][s'] as (re, im), mu = x, y, z, t
  static const int G[4][4][4][2] = {
      {{{0, 0}, {0, 0}, {0, 0}, {0, 1}}, {{0, 0}, {0, 0}, {0, 1}, {0, 0}},
       {{0, 0}, {0, -1}, {0, 0}, {0, 0}}, {{0, -1}, {0, 0}, {0, 0}, {0, 0}}},
      {{{0, 0}, {0, 0}, {0, 0}, {-1, 0}}, {{0, 0}, {0, 0}, {1, 0}, {0, 0}},
       {{0, 0}, {1, 0}, {0, 0}, {0, 0}}, {{-1, 0}, {0, 0}, {0, 0}, {0, 0}}},
      {{{0, 0}, {0, 0}, {0, 1}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}, {0, -1}},
       {{0, -1}, {0, 0}, {0, 0}, {0, 0}}, {{0, 0}, {0, 1}, {0, 0}, {0, 0}}},
      {{{0, 0}, {0, 0}, {1, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}, {1, 0}},
       {{1, 0}, {0, 0}, {0, 0}, {0, 0}}, {{0, 0}, {1, 0}, {0, 0}, {0, 0}}}};
  TSpin t;
  memset(&t, 0, sizeof(t));
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1, sg = (d & 1) ? 1 : -1;
    for (int s = 0; s < 4; ++s)
      for (int sp = 0; sp < 4; ++sp)
        if (sp != s && (G[mu][s][sp][0] != 0 || G[mu][s][sp][1] != 0)) {
          t.so[d][s] = sp;
          t.pr[d][s] = sg * G[mu][s][sp][0];
          t.pi[d][s] = sg * G[mu][s][sp][1];
        }
  }
  return t;
}

int tile_hop(int epi, cudaStream_t q, int G, lqcd_ctx *ctx, int p_out, const TileField &in, const TileField &out,
             const TileField &A, const TileField &B, float cA, float cH, const int *tlist, const int *tcount, D4S *part,
             int nch, int nrhs, unsigned long long *prof, int *err) {
  if (!in.d || !out.d) return set_error(ctx, LQCD_ERR_INVALID, "tile hop: null field");
  THopArgs a;
  a.g = ctx->geom;
  a.p_out = p_out;
  a.links = ctx->Ub16;
  a.out = out.d;
  a.in = in.d;
  a.A = A.d;
  a.B = B.d;
  a.cA = cA;
  a.cH = cH;
  a.tlist = tlist;
  a.tcount = tcount;
  a.part = part;
  a.nch = nch;
  a.nrhs = nrhs;
  a.prof = prof;
  a.err = err;
  static const TSpin spin = make_spin_table();
  a.spin = spin;
  static bool attr_set[3] = {false, false, false};
  auto go = [&](auto kern, int slot) {
    if (!attr_set[slot]) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T_SMEM);
      if (e != cudaSuccess) return e;
      attr_set[slot] = true;
    }
    KL kern<<<G, T_THREADS, T_SMEM, q>>>(a);
    return cudaGetLastError();
  };
  cudaError_t e;
  if (epi == EPI_PLAIN) e = go(k_thop<EPI_PLAIN>, 0);
  else if (epi == EPI_DOTR) e = go(k_thop<EPI_DOTR>, 1);
  else if (epi == EPI_TS) e = go(k_thop<EPI_TS>, 2);
  else return set_error(ctx, LQCD_ERR_INVALID, "tile hop: unknown epilogue %d", epi);
  if (e != cudaSuccess) return cuda_error(ctx, e, "tile hop launch");
  return LQCD_OK;
}

// ==================================================== element-wise tile kernels
// A block takes work items (active tile T, chunk ch of TCH sites) by grid
// stride; thread (r, h) = (tid % TR, tid / TR) owns right-hand side r of the
// tile and walks the sites j0 + h, j0 + h + 2, ...  Every tile-field access of
// a warp is one 512-byte segment (chunk c of 32 consecutive right-hand sides).
constexpr int TB = 256;  // threads per block of the element-wise tile kernels
constexpr int TSB = 8;   // sites per transposition sub-block (x / FP32 side)
constexpr int TXS = TSB * 24 + 4;  // floats per RHS row of the staging buffer (padded against bank conflicts)

__device__ __forceinline__ void bf8_to_f(uint4 w, float f[8]) {
  const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    f[2 * k] = __uint_as_float(u[k] << 16);
    f[2 * k + 1] = __uint_as_float(u[k] & 0xffff0000u);
  }
}
__device__ __forceinline__ uint4 f_to_bf8(const float f[8]) {
  uint32_t u[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
    u[k] = *reinterpret_cast<uint32_t *>(&h);
  }
  return make_uint4(u[0], u[1], u[2], u[3]);
}
__device__ __forceinline__ float2 sc2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// p = r + beta (p - omega v); members flagged for restart take rhat = r, p = r
__global__ void __launch_bounds__(TB) k_tile_p(int vh, int nch, const SState *sc, const uint4 *r, uint4 *rhat, uint4 *p,
                                               const uint4 *v, const int *tlist, const int *tcount) {
  const int n_items = *tcount * nch;
  const int rr = threadIdx.x % TR, h = threadIdx.x / TR;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int T = tlist[w / nch], ch = w % nch;
    const int j0 = ch * TCH, ns = min(TCH, vh - j0);
    const SState &S = sc[T * TR + rr];
    const float2 be = sc2(S.beta), om = sc2(S.omega);
    const bool rs = S.restart != 0;
    for (int js = h; js < ns; js += TB / TR) {
      const size_t e0 = tile_chunk(T, vh, j0 + js, 0, rr);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float R[8], P[8], V[8];
        bf8_to_f(r[e0 + c * TR], R);
        bf8_to_f(p[e0 + c * TR], P);
        bf8_to_f(v[e0 + c * TR], V);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          // t = p - omega v; p = r + beta t
          const float tr = P[2 * i] - (om.x * V[2 * i] - om.y * V[2 * i + 1]);
          const float ti = P[2 * i + 1] - (om.x * V[2 * i + 1] + om.y * V[2 * i]);
          P[2 * i] = rs ? R[2 * i] : R[2 * i] + (be.x * tr - be.y * ti);
          P[2 * i + 1] = rs ? R[2 * i + 1] : R[2 * i + 1] + (be.x * ti + be.y * tr);
        }
        p[e0 + c * TR] = f_to_bf8(P);
        if (rs) rhat[e0 + c * TR] = r[e0 + c * TR];
      }
    }
  }
}

// s = r - alpha v
__global__ void __launch_bounds__(TB) k_tile_s(int vh, int nch, const SState *sc, const uint4 *r, const uint4 *v,
                                               uint4 *s, const int *tlist, const int *tcount) {
  const int n_items = *tcount * nch;
  const int rr = threadIdx.x % TR, h = threadIdx.x / TR;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int T = tlist[w / nch], ch = w % nch;
    const int j0 = ch * TCH, ns = min(TCH, vh - j0);
    const float2 al = sc2(sc[T * TR + rr].alpha);
    for (int js = h; js < ns; js += TB / TR) {
      const size_t e0 = tile_chunk(T, vh, j0 + js, 0, rr);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float R[8], V[8];
        bf8_to_f(r[e0 + c * TR], R);
        bf8_to_f(v[e0 + c * TR], V);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          R[2 * i] -= al.x * V[2 * i] - al.y * V[2 * i + 1];
          R[2 * i + 1] -= al.x * V[2 * i + 1] + al.y * V[2 * i];
        }
        s[e0 + c * TR] = f_to_bf8(R);
      }
    }
  }
}

// fixed-order reduction of the per-thread partials (one RHS and 3 values per
// thread, TB / TR threads per RHS) into part[rhs][nch] as (re, im, nn, 0)
__device__ __forceinline__ void tile_reduce_store(float *red, const float acc[3], int T, int ch, int nch, D4S *part) {
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 3; ++q) red[threadIdx.x * 3 + q] = acc[q];
  __syncthreads();
  if (threadIdx.x < TR) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int hh = 0; hh < TB / TR; ++hh) {
      s0 += red[(hh * TR + threadIdx.x) * 3];
      s1 += red[(hh * TR + threadIdx.x) * 3 + 1];
      s2 += red[(hh * TR + threadIdx.x) * 3 + 2];
    }
    part[(size_t)(T * TR + threadIdx.x) * nch + ch] = D4S{(double)s0, (double)s1, (double)s2, 0.0};
  }
  __syncthreads();
}

// x (FP32, per-RHS layout) += alpha p + omega s for active members; r = s - omega t;
// partials <rhat, r> and |r|^2.  The x increments of TSB sites are staged in
// shared memory [rhs][site][24] so that the FP32 side is read and written in
// runs of TSB consecutive sites.
__global__ void __launch_bounds__(TB) k_tile_xr(int vh, int nch, const SState *sc, const int *flags, F32F x,
                                                const uint4 *p, const uint4 *s, const uint4 *t, uint4 *r,
                                                const uint4 *rhat, const int *tlist, const int *tcount, D4S *part) {
  extern __shared__ float xsm[];  // TR * TXS floats (also the reduction scratch)
  __shared__ int act[TR];
  const int n_items = *tcount * nch;
  const int rr = threadIdx.x % TR, h = threadIdx.x / TR;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int T = tlist[w / nch], ch = w % nch;
    const int j0 = ch * TCH, ns = min(TCH, vh - j0);
    const float2 al = sc2(sc[T * TR + rr].alpha), om = sc2(sc[T * TR + rr].omega);
    __syncthreads();
    if (threadIdx.x < TR) act[threadIdx.x] = flags[T * TR + threadIdx.x] & FLAG_ACTIVE;
    float acc[3] = {0.f, 0.f, 0.f};
    for (int b0 = 0; b0 < ns; b0 += TSB) {
      const int nb = min(TSB, ns - b0);
      __syncthreads();
      for (int js = h; js < nb; js += TB / TR) {
        const size_t e0 = tile_chunk(T, vh, j0 + b0 + js, 0, rr);
        float *qrow = xsm + (size_t)rr * TXS + js * 24;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float P[8], S[8], Tt[8], H[8], dx[8];
          bf8_to_f(p[e0 + c * TR], P);
          bf8_to_f(s[e0 + c * TR], S);
          bf8_to_f(t[e0 + c * TR], Tt);
          bf8_to_f(rhat[e0 + c * TR], H);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float pr = P[2 * i], pi = P[2 * i + 1], sr = S[2 * i], si = S[2 * i + 1];
            dx[2 * i] = al.x * pr - al.y * pi + (om.x * sr - om.y * si);
            dx[2 * i + 1] = al.x * pi + al.y * pr + (om.x * si + om.y * sr);
            const float nr = sr - (om.x * Tt[2 * i] - om.y * Tt[2 * i + 1]);
            const float ni = si - (om.x * Tt[2 * i + 1] + om.y * Tt[2 * i]);
            S[2 * i] = nr;
            S[2 * i + 1] = ni;
            const float hr = H[2 * i], hi = H[2 * i + 1];
            acc[0] += hr * nr + hi * ni;
            acc[1] += hr * ni - hi * nr;
            acc[2] += nr * nr + ni * ni;
          }
          reinterpret_cast<float4 *>(qrow + 8 * c)[0] = make_float4(dx[0], dx[1], dx[2], dx[3]);
          reinterpret_cast<float4 *>(qrow + 8 * c)[1] = make_float4(dx[4], dx[5], dx[6], dx[7]);
          r[e0 + c * TR] = f_to_bf8(S);
        }
      }
      __syncthreads();
      // x side: TSB-site runs of float4 per (rhs, k4)
      for (int idx = threadIdx.x; idx < TR * 6 * TSB; idx += TB) {
        const int js = idx % TSB, k4 = (idx / TSB) % 6, r2 = idx / (TSB * 6);
        if (js >= nb || !act[r2]) continue;
        const float4 d = *reinterpret_cast<const float4 *>(xsm + (size_t)r2 * TXS + js * 24 + 4 * k4);
        float4 *xp = x.d + ((size_t)(T * TR + r2) * 6 + k4) * vh + j0 + b0 + js;
        float4 o = *xp;
        o.x += d.x;
        o.y += d.y;
        o.z += d.z;
        o.w += d.w;
        *xp = o;
      }
    }
    tile_reduce_store(xsm, acc, T, ch, nch, part);
  }
}

// members flagged FLAG_RU: r = src (FP32, per-RHS layout), optionally x = 0;
// partials per member of <rhat, r> (or <r, r>) and |r|^2
__global__ void __launch_bounds__(TB) k_tile_copy(int vh, int nch, const int *flags, F32F src, uint4 *r,
                                                  const uint4 *rhat, int use_rhat, F32F x, int zero_x,
                                                  const int *tlist, const int *tcount, D4S *part) {
  extern __shared__ float xsm[];
  __shared__ int fl[TR];
  const int n_items = *tcount * nch;
  const int rr = threadIdx.x % TR, h = threadIdx.x / TR;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int T = tlist[w / nch], ch = w % nch;
    const int j0 = ch * TCH, ns = min(TCH, vh - j0);
    __syncthreads();
    if (threadIdx.x < TR) fl[threadIdx.x] = flags[T * TR + threadIdx.x] & FLAG_RU;
    __syncthreads();
    const bool mine = fl[rr] != 0;
    float acc[3] = {0.f, 0.f, 0.f};
    for (int b0 = 0; b0 < ns; b0 += TSB) {
      const int nb = min(TSB, ns - b0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < TR * 6 * TSB; idx += TB) {
        const int js = idx % TSB, k4 = (idx / TSB) % 6, r2 = idx / (TSB * 6);
        if (js >= nb || !fl[r2]) continue;
        const size_t gi = ((size_t)(T * TR + r2) * 6 + k4) * vh + j0 + b0 + js;
        *reinterpret_cast<float4 *>(xsm + (size_t)r2 * TXS + js * 24 + 4 * k4) = src.d[gi];
        if (zero_x) x.d[gi] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncthreads();
      for (int js = h; js < nb; js += TB / TR) {
        const size_t e0 = tile_chunk(T, vh, j0 + b0 + js, 0, rr);
        const float *qrow = xsm + (size_t)rr * TXS + js * 24;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float V[8], H[8];
          if (mine) {
            const float4 a0 = reinterpret_cast<const float4 *>(qrow + 8 * c)[0];
            const float4 a1 = reinterpret_cast<const float4 *>(qrow + 8 * c)[1];
            V[0] = a0.x; V[1] = a0.y; V[2] = a0.z; V[3] = a0.w;
            V[4] = a1.x; V[5] = a1.y; V[6] = a1.z; V[7] = a1.w;
            // the stored member values are rounded to BF16; the partials use the
            // FP32 source values, as the pair path does
            r[e0 + c * TR] = f_to_bf8(V);
          } else {
            bf8_to_f(r[e0 + c * TR], V);
          }
          if (use_rhat) bf8_to_f(rhat[e0 + c * TR], H);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float vr = V[2 * i], vi = V[2 * i + 1];
            const float qr = use_rhat ? H[2 * i] : vr, qi = use_rhat ? H[2 * i + 1] : vi;
            acc[0] += qr * vr + qi * vi;
            acc[1] += qr * vi - qi * vr;
            acc[2] += vr * vr + vi * vi;
          }
        }
      }
    }
    tile_reduce_store(xsm, acc, T, ch, nch, part);
  }
}

constexpr size_t T_XR_SMEM = (size_t)TR * TXS * sizeof(float);  // 98 KiB (>= the reduction's 3 KiB)

int tile_p(cudaStream_t q, int G, int vh, const SState *sc, const TileField &r, const TileField &rhat,
           const TileField &p, const TileField &v, const int *tlist, const int *tcount) {
  const int nch = (vh + TCH - 1) / TCH;
  KL k_tile_p<<<G, TB, 0, q>>>(vh, nch, sc, (const uint4 *)r.d, (uint4 *)rhat.d, (uint4 *)p.d, (const uint4 *)v.d,
                               tlist, tcount);
  return cudaGetLastError() == cudaSuccess ? LQCD_OK : LQCD_ERR_CUDA;
}

int tile_s(cudaStream_t q, int G, int vh, const SState *sc, const TileField &r, const TileField &v,
           const TileField &s, const int *tlist, const int *tcount) {
  const int nch = (vh + TCH - 1) / TCH;
  KL k_tile_s<<<G, TB, 0, q>>>(vh, nch, sc, (const uint4 *)r.d, (const uint4 *)v.d, (uint4 *)s.d, tlist, tcount);
  return cudaGetLastError() == cudaSuccess ? LQCD_OK : LQCD_ERR_CUDA;
}

int tile_xr(cudaStream_t q, int G, int vh, const SState *sc, const int *flags, F32F x, const TileField &p,
            const TileField &s, const TileField &t, const TileField &r, const TileField &rhat, const int *tlist,
            const int *tcount, D4S *part) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_tile_xr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T_XR_SMEM) != cudaSuccess)
      return LQCD_ERR_CUDA;
    attr = true;
  }
  const int nch = (vh + TCH - 1) / TCH;
  KL k_tile_xr<<<G, TB, T_XR_SMEM, q>>>(vh, nch, sc, flags, x, (const uint4 *)p.d, (const uint4 *)s.d,
                                        (const uint4 *)t.d, (uint4 *)r.d, (const uint4 *)rhat.d, tlist, tcount, part);
  return cudaGetLastError() == cudaSuccess ? LQCD_OK : LQCD_ERR_CUDA;
}

int tile_copy(cudaStream_t q, int G, int vh, const int *flags, F32F src, const TileField &r, const TileField &rhat,
              bool use_rhat, F32F x, bool zero_x, const int *tlist, const int *tcount, D4S *part) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_tile_copy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T_XR_SMEM) != cudaSuccess)
      return LQCD_ERR_CUDA;
    attr = true;
  }
  const int nch = (vh + TCH - 1) / TCH;
  KL k_tile_copy<<<G, TB, T_XR_SMEM, q>>>(vh, nch, flags, src, (uint4 *)r.d, (const uint4 *)rhat.d, use_rhat ? 1 : 0,
                                          x, zero_x ? 1 : 0, tlist, tcount, part);
  return cudaGetLastError() == cudaSuccess ? LQCD_OK : LQCD_ERR_CUDA;
}

}  // namespace lqcd
