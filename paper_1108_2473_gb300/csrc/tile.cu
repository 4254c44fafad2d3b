// RHS-tile path of the mixed-precision solver (Sec. II: mixed-precision
// BiCGstab for the all-to-all inversions): BF16 sloppy fields in 128-RHS tiles
// (layout in tile.cuh), the tensor-core hopping term, the element-wise Krylov
// updates on tiles, and the BF16 link bundle the hop reads.
#include <cudaTypedefs.h>

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

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

int tile_field_map(lqcd_ctx *ctx, TileField &f) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return set_error(ctx, LQCD_ERR_CUDA, "tile path: cuTensorMapEncodeTiled is unavailable");
  // 2-d view: [ntile * Vh * 48 rows][64 RHS] BF16, rows of 128 bytes; boxes of
  // 64 RHS x 48 rows (one neighbour block, both halves), 128-byte swizzle
  const cuuint64_t dim[2] = {64, (cuuint64_t)f.ntile * f.vh * 48};
  const cuuint64_t stride[1] = {128};
  const cuuint32_t box[2] = {64, 48};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&f.map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)f.d, dim, stride, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(ctx, LQCD_ERR_CUDA, "tile path: cuTensorMapEncodeTiled failed (%d)", (int)r);
  const cuuint32_t sbox[2] = {32, 24};
  r = enc(&f.smap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)f.d, dim, stride, sbox, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(ctx, LQCD_ERR_CUDA, "tile path: cuTensorMapEncodeTiled (store) failed (%d)", (int)r);
  return LQCD_OK;
}

int tile_hop(int epi, cudaStream_t q, int G, lqcd_ctx *ctx, int p_out, const TileField &in, const TileField &out,
             const TileField &A, const TileField &B, float cA, float cH, const int *tlist, const int *tcount, D4S *part,
             int nch, int nrhs, unsigned long long *prof, int *err) {
  static bool attr_set[5] = {false, false, false, false, false};
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
  cudaError_t e = cudaSuccess;
#define THOP_CASE(E)                                                                                 \
  case E:                                                                                            \
    if (!attr_set[E]) {                                                                              \
      e = cudaFuncSetAttribute(k_thop<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, T_SMEM);      \
      if (e != cudaSuccess) return cuda_error(ctx, e, "tile hop: shared-memory attribute");          \
      attr_set[E] = true;                                                                            \
    }                                                                                                \
    KL k_thop<E><<<G, T_THREADS, T_SMEM, q>>>(in.map, a);                                           \
    break;
  switch (epi) {
    THOP_CASE(EPI_PLAIN)
    THOP_CASE(EPI_DOTR)
    THOP_CASE(EPI_TS)
    default:
      return set_error(ctx, LQCD_ERR_INVALID, "tile hop: unknown epilogue %d", epi);
  }
#undef THOP_CASE
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(ctx, e, "tile hop launch");
  return LQCD_OK;
}

// ==================================================== element-wise tile kernels
// A block takes work items (active tile T, chunk ch of TCH sites) by grid
// stride; thread (m, g) = (tid >> 4, tid & 15) owns the 8 right-hand sides
// 8g .. 8g+7 of the tile and walks (site, complex component) units m, m + 16, ...
constexpr int TB = 256;  // threads per block of the element-wise tile kernels
constexpr int TSB = 8;   // sites per transposition sub-block (x / FP32 side)

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
// real k of the 8 right-hand sides 8g .. 8g+7 at (tile T, site j), in uint4 units;
// real k + 1 (the imaginary part when k is even) is 64 elements = 8 uint4 further
__device__ __forceinline__ size_t trow(int T, int vh, int j, int k, int g) {
  return tile_elem(T, vh, j, k, 8 * g) / 8;
}
__device__ __forceinline__ void load_c8(const uint4 *f, size_t re_idx, float re[8], float im[8]) {
  bf8_to_f(f[re_idx], re);
  bf8_to_f(f[re_idx + 8], im);
}
__device__ __forceinline__ void store_c8(uint4 *f, size_t re_idx, const float re[8], const float im[8]) {
  f[re_idx] = f_to_bf8(re);
  f[re_idx + 8] = f_to_bf8(im);
}
__device__ __forceinline__ float2 sc2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// p = r + beta (p - omega v); members flagged for restart take rhat = r, p = r
__global__ void __launch_bounds__(TB) k_tile_p(int vh, int nch, const SState *sc, const uint4 *r, uint4 *rhat, uint4 *p,
                                               const uint4 *v, const int *tlist, const int *tcount) {
  const int n_items = *tcount * nch;
  const int g = threadIdx.x & 15, m = threadIdx.x >> 4;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int T = tlist[w / nch], ch = w % nch;
    const int j0 = ch * TCH, ns = min(TCH, vh - j0);
    float2 be[8], om[8];
    unsigned restart = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const SState &s = sc[T * TR + 8 * g + i];
      be[i] = sc2(s.beta);
      om[i] = sc2(s.omega);
      restart |= (s.restart ? 1u : 0u) << i;
    }
    for (int u = m; u < ns * 12; u += 16) {
      const int j = j0 + u / 12, c = u % 12;
      const size_t ix = trow(T, vh, j, 2 * c, g);
      float rr[8], ri[8], pr[8], pi[8], vr[8], vi[8];
      load_c8(r, ix, rr, ri);
      load_c8(p, ix, pr, pi);
      load_c8(v, ix, vr, vi);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        // t = p - omega v; p = r + beta t
        const float tr = pr[i] - (om[i].x * vr[i] - om[i].y * vi[i]);
        const float ti = pi[i] - (om[i].x * vi[i] + om[i].y * vr[i]);
        const float nr = rr[i] + (be[i].x * tr - be[i].y * ti);
        const float ni = ri[i] + (be[i].x * ti + be[i].y * tr);
        const bool rs = (restart >> i) & 1u;
        pr[i] = rs ? rr[i] : nr;
        pi[i] = rs ? ri[i] : ni;
      }
      store_c8(p, ix, pr, pi);
      if (restart) {
        float hr[8], hi[8];
        load_c8(rhat, ix, hr, hi);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if ((restart >> i) & 1u) {
            hr[i] = rr[i];
            hi[i] = ri[i];
          }
        store_c8(rhat, ix, hr, hi);
      }
    }
  }
}

// s = r - alpha v
__global__ void __launch_bounds__(TB) k_tile_s(int vh, int nch, const SState *sc, const uint4 *r, const uint4 *v,
                                               uint4 *s, const int *tlist, const int *tcount) {
  const int n_items = *tcount * nch;
  const int g = threadIdx.x & 15, m = threadIdx.x >> 4;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int T = tlist[w / nch], ch = w % nch;
    const int j0 = ch * TCH, ns = min(TCH, vh - j0);
    float2 al[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) al[i] = sc2(sc[T * TR + 8 * g + i].alpha);
    for (int u = m; u < ns * 12; u += 16) {
      const int j = j0 + u / 12, c = u % 12;
      const size_t ix = trow(T, vh, j, 2 * c, g);
      float rr[8], ri[8], vr[8], vi[8];
      load_c8(r, ix, rr, ri);
      load_c8(v, ix, vr, vi);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        rr[i] -= al[i].x * vr[i] - al[i].y * vi[i];
        ri[i] -= al[i].x * vi[i] + al[i].y * vr[i];
      }
      store_c8(s, ix, rr, ri);
    }
  }
}

// fixed-order reduction of the per-thread partials (8 RHS x 3 values per
// thread, 16 threads per RHS group) into part[rhs][nch] as (re, im, nn, 0)
__device__ __forceinline__ void tile_reduce_store(float *red, const float acc[8][3], int T, int ch, int nch, D4S *part) {
  const int g = threadIdx.x & 15, m = threadIdx.x >> 4;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 3; ++q) red[(m * TR + 8 * g + i) * 3 + q] = acc[i][q];
  __syncthreads();
  if (threadIdx.x < TR) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int mm = 0; mm < 16; ++mm) {
      s0 += red[(mm * TR + threadIdx.x) * 3];
      s1 += red[(mm * TR + threadIdx.x) * 3 + 1];
      s2 += red[(mm * TR + threadIdx.x) * 3 + 2];
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
  extern __shared__ float xsm[];  // TR * TSB * 24 floats (also the reduction scratch)
  __shared__ int act[TR];
  const int n_items = *tcount * nch;
  const int g = threadIdx.x & 15, m = threadIdx.x >> 4;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int T = tlist[w / nch], ch = w % nch;
    const int j0 = ch * TCH, ns = min(TCH, vh - j0);
    float2 al[8], om[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      al[i] = sc2(sc[T * TR + 8 * g + i].alpha);
      om[i] = sc2(sc[T * TR + 8 * g + i].omega);
    }
    if (threadIdx.x < TR) act[threadIdx.x] = flags[T * TR + threadIdx.x] & FLAG_ACTIVE;
    float acc[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0.f;
    for (int b0 = 0; b0 < ns; b0 += TSB) {
      const int nb = min(TSB, ns - b0);
      __syncthreads();
      for (int u = m; u < nb * 12; u += 16) {
        const int js = u / 12, c = u % 12, j = j0 + b0 + js;
        const size_t ix = trow(T, vh, j, 2 * c, g);
        float pr[8], pi[8], sr[8], si[8], tr[8], ti[8], hr[8], hi[8];
        load_c8(p, ix, pr, pi);
        load_c8(s, ix, sr, si);
        load_c8(t, ix, tr, ti);
        load_c8(rhat, ix, hr, hi);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float dr = al[i].x * pr[i] - al[i].y * pi[i] + (om[i].x * sr[i] - om[i].y * si[i]);
          const float di = al[i].x * pi[i] + al[i].y * pr[i] + (om[i].x * si[i] + om[i].y * sr[i]);
          float *q = xsm + ((size_t)(8 * g + i) * TSB + js) * 24 + 2 * c;
          q[0] = dr;
          q[1] = di;
          const float nr = sr[i] - (om[i].x * tr[i] - om[i].y * ti[i]);
          const float ni = si[i] - (om[i].x * ti[i] + om[i].y * tr[i]);
          sr[i] = nr;
          si[i] = ni;
          acc[i][0] += hr[i] * nr + hi[i] * ni;
          acc[i][1] += hr[i] * ni - hi[i] * nr;
          acc[i][2] += nr * nr + ni * ni;
        }
        store_c8(r, ix, sr, si);
      }
      __syncthreads();
      // x side: TSB-site runs of float4 per (rhs, k4)
      for (int idx = threadIdx.x; idx < TR * 6 * TSB; idx += TB) {
        const int js = idx % TSB, k4 = (idx / TSB) % 6, rr = idx / (TSB * 6);
        if (js >= nb || !act[rr]) continue;
        const float *q = xsm + ((size_t)rr * TSB + js) * 24 + 4 * k4;
        float4 *xp = x.d + ((size_t)(T * TR + rr) * 6 + k4) * vh + j0 + b0 + js;
        float4 o = *xp;
        o.x += q[0];
        o.y += q[1];
        o.z += q[2];
        o.w += q[3];
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
  const int g = threadIdx.x & 15, m = threadIdx.x >> 4;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int T = tlist[w / nch], ch = w % nch;
    const int j0 = ch * TCH, ns = min(TCH, vh - j0);
    __syncthreads();
    if (threadIdx.x < TR) fl[threadIdx.x] = flags[T * TR + threadIdx.x] & FLAG_RU;
    __syncthreads();
    unsigned mine = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) mine |= (fl[8 * g + i] ? 1u : 0u) << i;
    float acc[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0.f;
    for (int b0 = 0; b0 < ns; b0 += TSB) {
      const int nb = min(TSB, ns - b0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < TR * 6 * TSB; idx += TB) {
        const int js = idx % TSB, k4 = (idx / TSB) % 6, rr = idx / (TSB * 6);
        if (js >= nb || !fl[rr]) continue;
        const size_t gi = ((size_t)(T * TR + rr) * 6 + k4) * vh + j0 + b0 + js;
        const float4 v = src.d[gi];
        float *q = xsm + ((size_t)rr * TSB + js) * 24 + 4 * k4;
        q[0] = v.x;
        q[1] = v.y;
        q[2] = v.z;
        q[3] = v.w;
        if (zero_x) x.d[gi] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncthreads();
      for (int u = m; u < nb * 12; u += 16) {
        const int js = u / 12, c = u % 12, j = j0 + b0 + js;
        const size_t ix = trow(T, vh, j, 2 * c, g);
        float vr[8], vi[8], hr[8], hi[8];
        load_c8(r, ix, vr, vi);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if ((mine >> i) & 1u) {
            const float *q = xsm + ((size_t)(8 * g + i) * TSB + js) * 24 + 2 * c;
            vr[i] = q[0];
            vi[i] = q[1];
          }
        if (mine) {
          // the stored member values are rounded to BF16; the partials use the
          // FP32 source values, as the pair path does
          store_c8(r, ix, vr, vi);
        }
        if (use_rhat) load_c8(rhat, ix, hr, hi);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float qr = use_rhat ? hr[i] : vr[i], qi = use_rhat ? hi[i] : vi[i];
          acc[i][0] += qr * vr[i] + qi * vi[i];
          acc[i][1] += qr * vi[i] - qi * vr[i];
          acc[i][2] += vr[i] * vr[i] + vi[i] * vi[i];
        }
      }
    }
    tile_reduce_store(xsm, acc, T, ch, nch, part);
  }
}

constexpr size_t T_XR_SMEM = (size_t)TR * TSB * 24 * sizeof(float);  // 96 KiB (>= the reduction's 24 KiB)

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
