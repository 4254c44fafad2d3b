// Context management, gauge upload/packing and the C ABI entry points that
// dispatch to the FP64 and mixed-precision paths.
#include <stdarg.h>
#include <chrono>
#include <cmath>

#include "internal.cuh"

using namespace lqcd;

namespace lqcd {

static thread_local std::string g_err;  // context-free calls

double wall_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int set_error(lqcd_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf; else g_err = buf;
  return code;
}

int cuda_error(lqcd_ctx *ctx, cudaError_t e, const char *where) {
  int code = (e == cudaErrorMemoryAllocation) ? LQCD_ERR_OOM : LQCD_ERR_CUDA;
  return set_error(ctx, code, "CUDA error in %s: %s", where, cudaGetErrorString(e));
}

void *workspace(lqcd_ctx *ctx, int slot, size_t bytes, int *status) {
  *status = LQCD_OK;
  if ((int)ctx->ws.size() < WS_COUNT) ctx->ws.resize(WS_COUNT);
  DevBuf &b = ctx->ws[slot];
  if (b.bytes >= bytes && b.p) return b.p;
  if (b.p) {
    cudaDeviceSynchronize();
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *status = cuda_error(ctx, e, "workspace cudaMalloc");
    b.p = nullptr;
    return nullptr;
  }
  b.bytes = bytes;
  return b.p;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------ gauge packing
__device__ __forceinline__ double2 dmul(double2 a, double2 b) { return cmul(a, b); }

// FP32 -> tf32 with round-to-nearest (ties away), kept in an FP32 register
__device__ __forceinline__ float to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Check unitarity and unit determinant of every link; write the reduced-precision
// copies (FP32 reconstruct-12, FP16 with all 18 reals duplicated, tf32,
// double-float) in parity-split order.
__global__ void k_pack_gauge(const double2 *__restrict__ U, Geom g, float4 *U32, uint4 *U16, float4 *Udf,
                             float2 *Utf, int *flag) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.V * 4) return;
  int s = idx >> 2, mu = idx & 3;
  const double2 *u = U + (size_t)idx * 9;
  double2 m[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      m[a][b] = u[a * 3 + b];
      // double-float copy for the residual: hi = fl32(v), lo = fl32(v - hi)
      float hx = (float)m[a][b].x, hy = (float)m[a][b].y;
      Udf[(size_t)idx * 9 + a * 3 + b] =
          make_float4(hx, hy, (float)(m[a][b].x - (double)hx), (float)(m[a][b].y - (double)hy));
    }
  double dev = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < 3; ++k) acc = cadd(acc, cmulc(m[k][a], m[k][b]));
      acc.x -= (a == b) ? 1.0 : 0.0;
      dev = fmax(dev, fmax(fabs(acc.x), fabs(acc.y)));
    }
  double2 det = cadd(cadd(dmul(m[0][0], csub(dmul(m[1][1], m[2][2]), dmul(m[1][2], m[2][1]))),
                          dmul(m[0][1], csub(dmul(m[1][2], m[2][0]), dmul(m[1][0], m[2][2])))),
                     dmul(m[0][2], csub(dmul(m[1][0], m[2][1]), dmul(m[1][1], m[2][0]))));
  dev = fmax(dev, fmax(fabs(det.x - 1.0), fabs(det.y)));
  if (!(dev <= 1e-12)) atomicOr(flag, 1);
  int x = s % g.L[0], r = s / g.L[0];
  int y = r % g.L[1]; r /= g.L[1];
  int z = r % g.L[2], t = r / g.L[2];
  int p = (x + y + z + t) & 1;
  int i = s >> 1;
  size_t base = ((size_t)(p * 4 + mu) * 3) * g.Vh + i;
  float v[12];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    v[2 * k] = (float)m[k / 3][k % 3].x;
    v[2 * k + 1] = (float)m[k / 3][k % 3].y;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
    U32[base + (size_t)k * g.Vh] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  // FP16 copy for the pair kernels: all 18 reals, each stored twice (u, u), so
  // one half2 -> float2 conversion gives the operand both members of a pair use;
  // layout [2 parity][4 mu][5][Vh] uint4 (the fifth uint4 half used)
  unsigned w[20];
#pragma unroll
  for (int k = 0; k < 18; ++k) {
    const double val = (k & 1) ? m[(k / 2) / 3][(k / 2) % 3].y : m[(k / 2) / 3][(k / 2) % 3].x;
    __half2 hh = __float2half2_rn((float)val);
    w[k] = *reinterpret_cast<unsigned *>(&hh);
  }
  w[18] = w[19] = 0u;
  const size_t base16 = ((size_t)(p * 4 + mu) * 5) * g.Vh + i;
#pragma unroll
  for (int k = 0; k < 5; ++k)
    U16[base16 + (size_t)k * g.Vh] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
  // tf32 copy for the tensor-core pair kernel: the 9 entries of one link contiguous
  float2 *ut = Utf + ((size_t)(p * 4 + mu) * g.Vh + i) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) ut[k] = make_float2(to_tf32((float)m[k / 3][k % 3].x), to_tf32((float)m[k / 3][k % 3].y));
}

// Plaquette partial sums: one double per block.
__global__ void k_plaquette(const double2 *__restrict__ U, Geom g, double *partial) {
  __shared__ double red[256];
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (s < g.V) {
    int c[4];
    c[0] = s % g.L[0];
    int r = s / g.L[0];
    c[1] = r % g.L[1]; r /= g.L[1];
    c[2] = r % g.L[2]; c[3] = r / g.L[2];
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        int cm[4] = {c[0], c[1], c[2], c[3]}, cn[4] = {c[0], c[1], c[2], c[3]};
        cm[mu] = (cm[mu] + 1) % g.L[mu];
        cn[nu] = (cn[nu] + 1) % g.L[nu];
        const double2 *a = U + ((size_t)s * 4 + mu) * 9;
        const double2 *b = U + ((size_t)site_of(g, cm) * 4 + nu) * 9;
        const double2 *cc = U + ((size_t)site_of(g, cn) * 4 + mu) * 9;
        const double2 *d = U + ((size_t)s * 4 + nu) * 9;
        double2 ab[3][3], abc[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double2 t = make_double2(0, 0);
            for (int k = 0; k < 3; ++k) t = cadd(t, dmul(a[i * 3 + k], b[k * 3 + j]));
            ab[i][j] = t;
          }
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {  // ab * cc^+
            double2 t = make_double2(0, 0);
            for (int k = 0; k < 3; ++k) {
              double2 cj = cc[j * 3 + k];
              cj.y = -cj.y;
              t = cadd(t, dmul(ab[i][k], cj));
            }
            abc[i][j] = t;
          }
        for (int i = 0; i < 3; ++i)  // Re Tr(abc * d^+)
          for (int k = 0; k < 3; ++k) {
            double2 dk = d[i * 3 + k];
            dk.y = -dk.y;
            acc += dmul(abc[i][k], dk).x;
          }
      }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_point_sources(const int64_t *sites, int n_sites, int V, double2 *out) {
  size_t total = (size_t)12 * n_sites;
  size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= total) return;
  int site_k = (int)(k / 12), sc = (int)(k % 12);
  int64_t s = sites[site_k];
  out[(k * (size_t)V + (size_t)s) * 12 + sc] = make_double2(1.0, 0.0);
}

}  // namespace lqcd

// ===================================================================== C ABI
extern "C" {

int lqcd_create(lqcd_ctx **out, const int dims[4], int device) {
  LQCD_TRACE("lqcd_create");
  if (!out || !dims) return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_create: null argument");
  *out = nullptr;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || (dims[i] & 1))
      return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_create: extent %d = %d must be even and >= 2", i, dims[i]);
  long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  if (V > (1LL << 30)) return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_create: volume too large");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_error(nullptr, e, "cudaSetDevice");
  lqcd_ctx *c = new lqcd_ctx();
  c->device = device;
  for (int i = 0; i < 4; ++i) c->dims[i] = dims[i];
  c->geom = make_geom(dims);
  c->ws.resize(WS_COUNT);
  e = cudaMalloc(&c->d_flag, sizeof(int) * 16);
  if (e != cudaSuccess) {
    delete c;
    return cuda_error(nullptr, e, "cudaMalloc(flag)");
  }
  *out = c;
  return LQCD_OK;
}

int lqcd_destroy(lqcd_ctx *ctx) {
  LQCD_TRACE("lqcd_destroy");
  if (!ctx) return LQCD_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  sloppy_free(ctx);
  for (auto &b : ctx->ws)
    if (b.p) cudaFree(b.p);
  cudaFree(ctx->U64);
  cudaFree(ctx->U32);
  cudaFree(ctx->U16);
  cudaFree(ctx->Utf);
  cudaFree(ctx->Ub16);
  cudaFree(ctx->Uape);
  cudaFree(ctx->Udf);
  cudaFree(ctx->d_flag);
  cudaFree(ctx->d_prof);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  delete ctx;
  return LQCD_OK;
}

const char *lqcd_last_error(const lqcd_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

static int set_gauge_impl(lqcd_ctx *ctx, const double *U, lqcd_stream_t stream, bool require_su3);

int lqcd_set_gauge(lqcd_ctx *ctx, const double *U, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_set_gauge");
  return set_gauge_impl(ctx, U, stream, true);
}

int lqcd_set_gauge_general(lqcd_ctx *ctx, const double *U, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_set_gauge_general");
  return set_gauge_impl(ctx, U, stream, false);
}

static int set_gauge_impl(lqcd_ctx *ctx, const double *U, lqcd_stream_t stream, bool require_su3) {
  if (!ctx || !U) return set_error(ctx, LQCD_ERR_INVALID, "lqcd_set_gauge: null argument");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Geom &g = ctx->geom;
  size_t n64 = (size_t)g.V * 36;
  if (!ctx->U64) {
    LQCD_CUDA_TRY(ctx, cudaMalloc(&ctx->U64, n64 * sizeof(double2)));
    LQCD_CUDA_TRY(ctx, cudaMalloc(&ctx->U32, (size_t)g.V * 4 * 3 * sizeof(float4)));
    LQCD_CUDA_TRY(ctx, cudaMalloc(&ctx->U16, (size_t)g.Vh * 2 * 4 * 5 * sizeof(uint4)));
    LQCD_CUDA_TRY(ctx, cudaMalloc(&ctx->Utf, (size_t)g.Vh * 2 * 4 * 9 * sizeof(float2)));
    LQCD_CUDA_TRY(ctx, cudaMalloc(&ctx->Udf, n64 * sizeof(float4)));
  }
  int st_ = LQCD_OK;
  double2 *stage = (double2 *)workspace(ctx, WS_STAGE_AUX, n64 * sizeof(double2), &st_);
  if (!stage) return st_;
  cudaMemcpyKind kind = is_device_ptr(U) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(stage, U, n64 * sizeof(double2), kind, st));
  LQCD_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
  int threads = 256, blocks = (g.V * 4 + threads - 1) / threads;
  KL k_pack_gauge<<<blocks, threads, 0, st>>>(stage, g, ctx->U32, ctx->U16, ctx->Udf, ctx->Utf, ctx->d_flag);
  LQCD_LAUNCH_CHECK(ctx, "k_pack_gauge");
  int flag = 0;
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (flag && require_su3) {
    ctx->have_gauge = false;
    return set_error(ctx, LQCD_ERR_NOT_SU3, "lqcd_set_gauge: a link is not SU(3) within 1e-12");
  }
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->U64, stage, n64 * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  ctx->have_gauge = true;
  ctx->have_ape = false;  // smeared links belong to the previous field
  ctx->gauge_su3 = !flag;
  int rc = pack_gauge_sloppy(ctx, st);
  if (rc != LQCD_OK) return rc;
  LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return LQCD_OK;
}

int lqcd_set_kappa(lqcd_ctx *ctx, double kappa) {
  LQCD_TRACE("lqcd_set_kappa");
  if (!ctx) return LQCD_ERR_INVALID;
  if (!std::isfinite(kappa)) return set_error(ctx, LQCD_ERR_INVALID, "lqcd_set_kappa: non-finite kappa");
  ctx->kappa = kappa;
  return LQCD_OK;
}

int lqcd_plaquette(lqcd_ctx *ctx, double *plaq, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_plaquette");
  if (!ctx || !plaq) return set_error(ctx, LQCD_ERR_INVALID, "lqcd_plaquette: null argument");
  if (!ctx->have_gauge) return set_error(ctx, LQCD_ERR_NO_GAUGE, "lqcd_plaquette: no gauge field");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Geom &g = ctx->geom;
  int threads = 256, blocks = (g.V + threads - 1) / threads;
  int rc = LQCD_OK;
  double *part = (double *)workspace(ctx, WS_LOOP_PART, blocks * sizeof(double), &rc);
  if (!part) return rc;
  KL k_plaquette<<<blocks, threads, 0, st>>>(ctx->U64, g, part);
  LQCD_LAUNCH_CHECK(ctx, "k_plaquette");
  std::vector<double> h(blocks);
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), part, blocks * sizeof(double), cudaMemcpyDeviceToHost, st));
  LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  double s = 0.0;
  for (double v : h) s += v;
  *plaq = s / (18.0 * g.V);
  return LQCD_OK;
}

int lqcd_apply_dirac(lqcd_ctx *ctx, const double *in, double *out, int nrhs, int dagger, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_apply_dirac");
  if (!ctx || nrhs < 0 || (nrhs > 0 && (!in || !out)))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_apply_dirac: bad argument");
  if (!ctx->have_gauge) return set_error(ctx, LQCD_ERR_NO_GAUGE, "lqcd_apply_dirac: no gauge field");
  if (nrhs == 0) return LQCD_OK;
  cudaSetDevice(ctx->device);
  return fp64_apply_dirac(ctx, (const double2 *)in, (double2 *)out, nrhs, dagger != 0, (cudaStream_t)stream);
}

int lqcd_solve_batch(lqcd_ctx *ctx, const double *b, double *x, int nrhs, const lqcd_solver_params *params,
                     lqcd_solve_stats *stats, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_solve_batch");
  if (!ctx || !params || nrhs < 0 || (nrhs > 0 && (!b || !x || !stats)))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_solve_batch: bad argument");
  if (!ctx->have_gauge) return set_error(ctx, LQCD_ERR_NO_GAUGE, "lqcd_solve_batch: no gauge field");
  if (nrhs == 0) return LQCD_OK;
  lqcd_solver_params p = *params;
  if (!(p.tol > 0.0) || p.max_iter <= 0)
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_solve_batch: tol must be > 0 and max_iter > 0");
  if (p.precision < LQCD_PREC_FP64 || p.precision > LQCD_PREC_MIXED_BF16)
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_solve_batch: unknown precision %d", p.precision);
  if (p.solver != LQCD_SOLVER_BICGSTAB && p.solver != LQCD_SOLVER_CG)
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_solve_batch: unknown solver %d", p.solver);
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  size_t bytes = (size_t)nrhs * ctx->geom.V * 12 * sizeof(double2);
  bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
  const double2 *db = (const double2 *)b;
  double2 *dx = (double2 *)x;
  int rc = LQCD_OK;
  if (!bdev) {
    double2 *s = (double2 *)workspace(ctx, WS_STAGE_IN, bytes, &rc);
    if (!s) return rc;
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(s, b, bytes, cudaMemcpyHostToDevice, st));
    db = s;
  }
  if (!xdev) {
    dx = (double2 *)workspace(ctx, WS_STAGE_OUT, bytes, &rc);
    if (!dx) return rc;
  }
  if (p.precision == LQCD_PREC_FP64)
    rc = fp64_solve(ctx, db, dx, nrhs, p, stats, st);
  else
    rc = mixed_solve(ctx, db, dx, nrhs, p, stats, st);
  if (!xdev) {
    cudaError_t e = cudaMemcpyAsync(x, dx, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_error(ctx, e, "solve_batch D2H");
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(ctx, e, "solve_batch sync");
  return rc;
}

int lqcd_point_sources(lqcd_ctx *ctx, const int64_t *sites, int n_sites, double *out, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_point_sources");
  if (!ctx || n_sites < 0 || (n_sites > 0 && (!sites || !out)))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_point_sources: bad argument");
  if (n_sites == 0) return LQCD_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Geom &g = ctx->geom;
  for (int k = 0; k < n_sites; ++k)
    if (sites[k] < 0 || sites[k] >= g.V)
      return set_error(ctx, LQCD_ERR_INVALID, "lqcd_point_sources: site %lld out of range", (long long)sites[k]);
  int rc = LQCD_OK;
  int64_t *dsites = (int64_t *)workspace(ctx, WS_STAGE_AUX, n_sites * sizeof(int64_t), &rc);
  if (!dsites) return rc;
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(dsites, sites, n_sites * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  LQCD_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, (size_t)12 * n_sites * g.V * 12 * sizeof(double2), st));
  size_t total = (size_t)12 * n_sites;
  KL k_point_sources<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(dsites, n_sites, g.V, (double2 *)out);
  LQCD_LAUNCH_CHECK(ctx, "k_point_sources");
  // the staged site list must outlive the copy: synchronise before returning
  LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return LQCD_OK;
}

}  // extern "C"

// ============================================================== profiling
namespace lqcd {
std::atomic<long long> g_launches{0};
}

extern "C" {

long long lqcd_launch_count(void) { return lqcd::g_launches.load(); }

int lqcd_profile_begin(lqcd_ctx *ctx) {
  LQCD_TRACE("lqcd_profile_begin");
  if (!ctx) return LQCD_ERR_INVALID;
  cudaSetDevice(ctx->device);
  if (!ctx->d_prof) LQCD_CUDA_TRY(ctx, cudaMalloc(&ctx->d_prof, 8 * sizeof(unsigned long long)));
  LQCD_CUDA_TRY(ctx, cudaMemset(ctx->d_prof, 0, 8 * sizeof(unsigned long long)));
  ctx->prof_used = 0;
  ctx->prof_hop_launches = 0;
  ctx->prof_launch_base = lqcd::g_launches.load();
  ctx->prof_on = true;
  return LQCD_OK;
}

int lqcd_profile_end(lqcd_ctx *ctx, lqcd_profile *out) {
  LQCD_TRACE("lqcd_profile_end");
  if (!ctx || !out) return LQCD_ERR_INVALID;
  cudaSetDevice(ctx->device);
  LQCD_CUDA_TRY(ctx, cudaDeviceSynchronize());
  ctx->prof_on = false;
  double ms = 0.0;
  for (size_t k = 0; k + 1 < ctx->prof_used; k += 2) {
    float t = 0.f;
    LQCD_CUDA_TRY(ctx, cudaEventElapsedTime(&t, ctx->prof_ev[k], ctx->prof_ev[k + 1]));
    ms += t;
  }
  unsigned long long h[8] = {0};
  if (ctx->d_prof) LQCD_CUDA_TRY(ctx, cudaMemcpy(h, ctx->d_prof, sizeof(h), cudaMemcpyDeviceToHost));
  // h[EPI kind]: output (site, RHS) pairs computed by the sloppy hop with that epilogue;
  // spinor operands per pair: PLAIN 2 (in, out), DOTR 4 (in, A, B, out), TS 3 (in, A, out)
  const int operands[5] = {2, 2, 4, 3, 4};
  double spinor_bytes = ctx->prof_prec == LQCD_PREC_MIXED_FP16 ? 52.0 : 48.0;  // 24 x 16-bit (+ FP32 norm)
  double pairs = 0.0, bytes = 0.0;
  for (int e = 0; e < 5; ++e) {
    pairs += (double)h[e];
    bytes += (double)h[e] * operands[e] * spinor_bytes;
  }
  bytes += (double)ctx->prof_hop_launches * ctx->geom.Vh * 8 * 72.0;  // FP16 (u,u) links, 18 reals, once per launch
  out->launches = lqcd::g_launches.load() - ctx->prof_launch_base;
  out->hop_launches = ctx->prof_hop_launches;
  out->hop_ms = ms;
  out->hop_site_rhs = pairs;
  out->hop_bytes = bytes;
  out->hop_flops = 1320.0 * pairs;
  return LQCD_OK;
}

}  // extern "C"
