// Loop contraction (Eq. loop; Eq. loop stochastic):
//   L_Gamma(x) += w * sum_i src_i(x)^+ Gamma sol_i(x)
// per site and per time slice, FP64 accumulation in a fixed order.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace lqcd {

// Gamma insertion of a loop, Gamma order (1, g5, g1, g2, g3, g4), DeGrand-Rossi:
// row a of Gamma has its one non-zero entry in column gamma_col(g, a), equal to
// +1, -1, +i, -i for gamma_ph(g, a) = 0, 1, 2, 3.  Compile-time after unrolling.
__host__ __device__ constexpr int gamma_col(int g, int a) { return g < 2 ? a : (g < 4 ? 3 - a : (a + 2) & 3); }
__host__ __device__ constexpr int gamma_ph(int g, int a) {
  return g == 0 ? 0
         : g == 1 ? (a < 2 ? 0 : 1)
         : g == 2 ? (a < 2 ? 2 : 3)
         : g == 3 ? ((a == 0 || a == 3) ? 1 : 0)
         : g == 4 ? ((a == 0 || a == 3) ? 2 : 3)
                  : 0;
}

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
#pragma unroll 2
    for (int i = 0; i < nrhs; ++i) {
      const double2 *a = src + ((size_t)i * g.V + s) * 12;
      const double2 *b = sol + ((size_t)i * g.V + s) * 12;
      double2 ea[12], eb[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) ea[k] = a[k];
      // Spin rows of the source that are zero contribute exactly zero, and the
      // solution rows they would pair with are not read: a diluted source is
      // non-zero on one time slice (and spin, colour) only.
      bool nz[4];
#pragma unroll
      for (int al = 0; al < 4; ++al) {
        bool z = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) z = z && ea[al * 3 + c].x == 0.0 && ea[al * 3 + c].y == 0.0;
        nz[al] = !z;
      }
      if (!(nz[0] || nz[1] || nz[2] || nz[3])) continue;
#pragma unroll
      for (int be = 0; be < 4; ++be) {
        // rows paired with be by the three permutations: be, 3 - be, be + 2 mod 4
        const bool need = nz[be] || nz[3 - be] || nz[(be + 2) & 3];
#pragma unroll
        for (int c = 0; c < 3; ++c) eb[be * 3 + c] = need ? b[be * 3 + c] : make_double2(0.0, 0.0);
      }
      // The six Gammas use three spin permutations (identity; 3-a; a+2 mod 4):
      // colour dot products P[perm][alpha] = sum_c conj(src[alpha][c]) sol[perm(alpha)][c]
      // once, then each Gamma is a signed / i-rotated sum of four of them.
      double2 P[3][4];
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int al = 0; al < 4; ++al) {
          const int be = q == 0 ? al : (q == 1 ? 3 - al : (al + 2) & 3);
          double2 d = make_double2(0.0, 0.0);
          if (nz[al]) {
            d = cmulc(ea[al * 3], eb[be * 3]);
            d = cadd(d, cmulc(ea[al * 3 + 1], eb[be * 3 + 1]));
            d = cadd(d, cmulc(ea[al * 3 + 2], eb[be * 3 + 2]));
          }
          P[q][al] = d;
        }
#pragma unroll
      for (int gi = 0; gi < 6; ++gi) {
        const int q = gi < 2 ? 0 : (gi < 4 ? 1 : 2);
        double2 sum = make_double2(0.0, 0.0);
#pragma unroll
        for (int al = 0; al < 4; ++al) sum = cadd(sum, gamma_phase(gamma_ph(gi, al), P[q][al]));
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
  LQCD_TRACE("lqcd_loops_batch");
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

// ===================================================== no-allocation variant
// lqcd_loops_batch_noalloc: the same contraction kernels as lqcd_loops_batch,
// for callers that must not allocate device memory.  The per-time-slice
// partial sums, which lqcd_loops_batch keeps in a context workspace, live here
// in one file-scope device array of fixed size instead.  That array exists on
// every GPU that loads this library, from module load until process exit.
#include <mutex>

namespace lqcd {

// Capacity in partial blocks: Lt * ceil(Lx*Ly*Lz / LOOP_THREADS) must not exceed it.
// 8192 blocks x 6 complex128 = 768 KiB per device (e.g. 24^3 x 48 needs 5184).
#define LQCD_NOALLOC_MAX_PARTIALS 8192
static __device__ __align__(256) double2 g_noalloc_partials[LQCD_NOALLOC_MAX_PARTIALS * 6];

// Host-side record of the array's device address, looked up once per device.
// In host code the symbol g_noalloc_partials is only a host stand-in; a kernel
// must be given the address returned by cudaGetSymbolAddress.
static double2 *g_noalloc_addr[64];
static std::mutex g_noalloc_mu;

static int noalloc_scratch(double2 **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(nullptr, e, "lqcd_loops_batch_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_loops_batch_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);  // with device `dev` current
    if (e != cudaSuccess || !p)
      return cuda_error(nullptr, e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                        "lqcd_loops_batch_noalloc: cudaGetSymbolAddress");
    g_noalloc_addr[dev] = (double2 *)p;
  }
  *out = g_noalloc_addr[dev];
  return LQCD_OK;
}

}  // namespace lqcd

extern "C" int lqcd_loops_batch_noalloc(const int dims[4], const double *src, const double *sol, int nrhs,
                                        double weight, double *per_site, double *per_t, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_loops_batch_noalloc");
  if (!dims || nrhs < 0 || (nrhs > 0 && (!src || !sol)))
    return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_loops_batch_noalloc: bad argument");
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || (dims[i] & 1))
      return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_loops_batch_noalloc: extent %d = %d must be even and >= 2",
                       i, dims[i]);
  const long long vol = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  if (vol > (1LL << 30) || dims[3] > 65535)
    return set_error(nullptr, LQCD_ERR_INVALID,
                     "lqcd_loops_batch_noalloc: volume %lld (limit 2^30) or Lt = %d (limit 65535) too large", vol,
                     dims[3]);
  Geom g = make_geom(dims);
  int vs = g.L[0] * g.L[1] * g.L[2], lt = g.L[3];
  int nbx = (vs + LOOP_THREADS - 1) / LOOP_THREADS;
  long long need = (long long)lt * nbx;
  if (per_t && need > LQCD_NOALLOC_MAX_PARTIALS)
    return set_error(nullptr, LQCD_ERR_INVALID,
                     "lqcd_loops_batch_noalloc: lattice needs %lld partial blocks (Lt * ceil(Lx*Ly*Lz/%d)); the fixed "
                     "scratch holds %d -- use lqcd_loops_batch",
                     need, LOOP_THREADS, LQCD_NOALLOC_MAX_PARTIALS);
  if (nrhs == 0 || (!per_site && !per_t)) return LQCD_OK;
  // every array must be addressable by a kernel on the current device: device
  // memory of this device (or managed memory), and the stream must belong to it
  int cur = 0;
  cudaError_t ce = cudaGetDevice(&cur);
  if (ce != cudaSuccess) return cuda_error(nullptr, ce, "lqcd_loops_batch_noalloc: cudaGetDevice");
  const void *ptrs[4] = {src, sol, per_site, per_t};
  const char *names[4] = {"src", "sol", "per_site", "per_t"};
  for (int k = 0; k < 4; ++k) {
    if (!ptrs[k]) continue;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptrs[k]) != cudaSuccess) {
      cudaGetLastError();
      return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_loops_batch_noalloc: %s is not device memory", names[k]);
    }
    if (a.type == cudaMemoryTypeManaged) continue;
    if (a.type != cudaMemoryTypeDevice)
      return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_loops_batch_noalloc: %s is not device memory", names[k]);
    if (a.device != cur)
      return set_error(nullptr, LQCD_ERR_INVALID,
                       "lqcd_loops_batch_noalloc: %s is on device %d, the current device is %d", names[k], a.device,
                       cur);
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread) {
    int sdev = -1;
    ce = cudaStreamGetDevice(st, &sdev);
    if (ce != cudaSuccess) return cuda_error(nullptr, ce, "lqcd_loops_batch_noalloc: cudaStreamGetDevice");
    if (sdev != cur)
      return set_error(nullptr, LQCD_ERR_INVALID,
                       "lqcd_loops_batch_noalloc: the stream belongs to device %d, the current device is %d", sdev,
                       cur);
  }
  double2 *part = nullptr;
  if (per_t) {
    int rc = noalloc_scratch(&part);
    if (rc) return rc;
  }
  // every partial read by k_loops_fin is written by k_loops in the same call,
  // so the scratch needs no clearing
  KL k_loops<<<dim3(nbx, lt), LOOP_THREADS, 0, st>>>(g, (const double2 *)src, (const double2 *)sol, nrhs, weight,
                                                     (double2 *)per_site, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(nullptr, e, "lqcd_loops_batch_noalloc: k_loops");
  if (per_t) {
    KL k_loops_fin<<<lt, 32, 0, st>>>(nbx, part, (double2 *)per_t);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(nullptr, e, "lqcd_loops_batch_noalloc: k_loops_fin");
  }
  return LQCD_OK;
}

// ============================================== momentum projection, D_AB(p, t)
namespace lqcd {

constexpr int MOM_CHUNK = 128;  // momenta per launch (passed by value)
constexpr int MOM_THREADS = 256;
struct MomList {
  int n[MOM_CHUNK][3];
};

// out[m][t][g] = sum_{x in slice t} e^{+i p_m.x} per_site[x][g].  p.x / 2 pi is
// reduced exactly to num / (Lx Ly Lz) with integer arithmetic; the phase is
// then sincospi(2 num / (Lx Ly Lz)).  One block per (t, m); strided per-thread
// sums and a fixed tree make the result independent of scheduling.
__global__ void __launch_bounds__(MOM_THREADS) k_loops_momentum(Geom g, const double2 *__restrict__ per_site,
                                                                MomList moms, double2 *out) {
  const int t = blockIdx.x, m = blockIdx.y;
  const int lx = g.L[0], ly = g.L[1], lz = g.L[2];
  const int v3 = lx * ly * lz;
  const int nx = ((moms.n[m][0] % lx) + lx) % lx, ny = ((moms.n[m][1] % ly) + ly) % ly,
            nz = ((moms.n[m][2] % lz) + lz) % lz;
  double2 acc[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) acc[k] = make_double2(0.0, 0.0);
  for (int xs = threadIdx.x; xs < v3; xs += MOM_THREADS) {
    const int x = xs % lx, y = (xs / lx) % ly, z = xs / (lx * ly);
    const long long num = ((long long)((nx * x) % lx) * ly * lz + (long long)((ny * y) % ly) * lx * lz +
                           (long long)((nz * z) % lz) * lx * ly) % v3;
    double sn, cs;
    sincospi(2.0 * (double)num / (double)v3, &sn, &cs);
    const double2 *L = per_site + ((size_t)t * v3 + xs) * 6;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double2 l = L[k];
      acc[k].x = fma(cs, l.x, fma(-sn, l.y, acc[k].x));
      acc[k].y = fma(cs, l.y, fma(sn, l.x, acc[k].y));
    }
  }
  __shared__ double2 sh[MOM_THREADS][6];
#pragma unroll
  for (int k = 0; k < 6; ++k) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int w = MOM_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < 6; ++k) sh[threadIdx.x][k] = cadd(sh[threadIdx.x][k], sh[threadIdx.x + w][k]);
    __syncthreads();
  }
  if (threadIdx.x < 6) out[((size_t)m * gridDim.x + t) * 6 + threadIdx.x] = sh[0][threadIdx.x];
}

// D[t][a][b] for one (t, a, b) per thread:
//   sum_t' [ S_a(t + t') S'_b(t') - (unbiased ? sum_r A_r,a(t + t') B_r,b(t') : 0) ]
// with S = sum_r A_r, S' = sum_r B_r, scaled by 1 / (l3 Lt n_pairs).
__global__ void k_correlator(const double2 *__restrict__ A, const double2 *__restrict__ B, int n, int lt,
                             double scale, int unbiased, double2 *out) {
  const int t = blockIdx.x, a = threadIdx.x / 6, b = threadIdx.x % 6;
  if (threadIdx.x >= 36) return;
  double2 d = make_double2(0.0, 0.0);
  for (int tp = 0; tp < lt; ++tp) {
    const int tf = (t + tp) % lt;
    double2 sa = make_double2(0.0, 0.0), sb = sa, diag = sa;
    for (int r = 0; r < n; ++r) {
      const double2 ar = A[((size_t)r * lt + tf) * 6 + a], br = B[((size_t)r * lt + tp) * 6 + b];
      sa = cadd(sa, ar);
      sb = cadd(sb, br);
      diag = cadd(diag, cmul(ar, br));
    }
    d = cadd(d, cmul(sa, sb));
    if (unbiased) d = csub(d, diag);
  }
  out[((size_t)t * 6 + a) * 6 + b] = cscale(d, scale);
}

}  // namespace lqcd

extern "C" int lqcd_loops_momentum(lqcd_ctx *ctx, const double *per_site, int n_mom, const int *moms, double *out,
                                   lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_loops_momentum");
  if (!ctx || n_mom < 0 || (n_mom > 0 && (!per_site || !moms || !out)))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_loops_momentum: bad argument");
  if (n_mom == 0) return LQCD_OK;
  if (!is_device_ptr(per_site) || !is_device_ptr(out))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_loops_momentum: per_site and out must be device memory");
  cudaSetDevice(ctx->device);
  const Geom &g = ctx->geom;
  for (int m0 = 0; m0 < n_mom; m0 += MOM_CHUNK) {
    const int nm = std::min(MOM_CHUNK, n_mom - m0);
    MomList ml;
    for (int m = 0; m < nm; ++m)
      for (int i = 0; i < 3; ++i) ml.n[m][i] = moms[(size_t)(m0 + m) * 3 + i];
    KL k_loops_momentum<<<dim3(g.L[3], nm), MOM_THREADS, 0, (cudaStream_t)stream>>>(
        g, (const double2 *)per_site, ml, (double2 *)out + (size_t)m0 * g.L[3] * 6);
    LQCD_LAUNCH_CHECK(ctx, "k_loops_momentum");
  }
  return LQCD_OK;
}

extern "C" int lqcd_disconnected_correlator(const double *loops_p, const double *loops_mp, int n_vec, int lt, int l3,
                                            int unbiased, double *out, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_disconnected_correlator");
  if (!loops_p || !loops_mp || !out || n_vec < 1 || lt < 1 || l3 < 1 || (unbiased && n_vec < 2))
    return set_error(nullptr, LQCD_ERR_INVALID,
                     "lqcd_disconnected_correlator: bad argument (the unbiased estimator needs n_vec >= 2)");
  if (!is_device_ptr(loops_p) || !is_device_ptr(loops_mp) || !is_device_ptr(out))
    return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_disconnected_correlator: arrays must be device memory");
  const double pairs = unbiased ? (double)n_vec * (n_vec - 1) : (double)n_vec * n_vec;
  KL k_correlator<<<lt, 64, 0, (cudaStream_t)stream>>>((const double2 *)loops_p, (const double2 *)loops_mp, n_vec,
                                                      lt, 1.0 / ((double)l3 * lt * pairs), unbiased,
                                                      (double2 *)out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(nullptr, e, "lqcd_disconnected_correlator");
  return LQCD_OK;
}
