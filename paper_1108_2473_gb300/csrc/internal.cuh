// Internal declarations shared by the translation units of liblqcd.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>
#include <atomic>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lqcd.h"

namespace lqcd {

// NVTX range around one ABI call (shows up in Nsight timelines; a no-op
// without a tool attached)
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};
#define LQCD_TRACE(name) ::lqcd::TraceRange lqcd_trace_range_(name)


// ------------------------------------------------------------------ geometry
struct Geom {
  int L[4];   // Lx, Ly, Lz, Lt
  int V, Vh;  // sites, sites per parity
  int Lxh;    // Lx / 2
};

__host__ __device__ inline Geom make_geom(const int d[4]) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = d[i];
  g.V = d[0] * d[1] * d[2] * d[3];
  g.Vh = g.V / 2;
  g.Lxh = d[0] / 2;
  return g;
}

// Coordinates of parity-local index i of parity p.  Site s = 2 i + (x & 1).
// pieces of a dilution scheme (LQCD_DILUTE_* base | optional EO / CUBE flag);
// -1 for an unknown scheme or bad dims
inline int dilution_pieces(const int dims[4], int dilution) {
  if (!dims) return -1;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || (dims[i] & 1)) return -1;
  const int base = dilution & 3, spatial = dilution & ~3;
  if (spatial != 0 && spatial != LQCD_DILUTE_EO && spatial != LQCD_DILUTE_CUBE) return -1;
  const int n_sp = spatial == LQCD_DILUTE_EO ? 2 : (spatial == LQCD_DILUTE_CUBE ? 8 : 1);
  const int n_base = base == LQCD_DILUTE_NONE ? 1 : base == LQCD_DILUTE_T ? dims[3] : base == LQCD_DILUTE_TS ? 4 * dims[3] : 12 * dims[3];
  return n_base * n_sp;
}

__device__ __forceinline__ void coords_of(const Geom &g, int p, int i, int c[4]) {
  int xh = i % g.Lxh;
  int r = i / g.Lxh;
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
  c[0] = 2 * xh + ((c[1] + c[2] + c[3] + p) & 1);
}

__device__ __forceinline__ int site_of(const Geom &g, const int c[4]) {
  return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

// ------------------------------------------------------------ complex helpers
template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };

template <typename C> __device__ __forceinline__ C cmk(decltype(C().x) a, decltype(C().x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C().x) s) { return cmk<C>(a.x * s, a.y * s); }
// i * a
template <typename C> __device__ __forceinline__ C cmuli(C a) { return cmk<C>(-a.y, a.x); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return cmk<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// a + s * i * b  for s = +-1
template <typename C> __device__ __forceinline__ C caddi(C a, C b, int s) {
  return s > 0 ? cmk<C>(a.x - b.y, a.y + b.x) : cmk<C>(a.x + b.y, a.y - b.x);
}

// ------------------------------------------------ Wilson spin projection
// Projector (1 + SIGMA gamma_mu) in the DeGrand-Rossi basis on a spinor
// psi[4][3]: the upper two spin rows h0, h1 carry all information; the lower
// rows are (r2, r3) = fixed multiples of (h0, h1).  SIGMA = -1: forward hop,
// SIGMA = +1: backward hop (swapped for D^+).
template <int MU, int SIGMA, typename C>
__device__ __forceinline__ void spin_project(const C psi[4][3], C h[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) {  // h0 = psi0 + s i psi3, h1 = psi1 + s i psi2
      h[0][c] = caddi(psi[0][c], psi[3][c], SIGMA);
      h[1][c] = caddi(psi[1][c], psi[2][c], SIGMA);
    } else if (MU == 1) {  // h0 = psi0 - s psi3, h1 = psi1 + s psi2
      h[0][c] = SIGMA > 0 ? csub(psi[0][c], psi[3][c]) : cadd(psi[0][c], psi[3][c]);
      h[1][c] = SIGMA > 0 ? cadd(psi[1][c], psi[2][c]) : csub(psi[1][c], psi[2][c]);
    } else if (MU == 2) {  // h0 = psi0 + s i psi2, h1 = psi1 - s i psi3
      h[0][c] = caddi(psi[0][c], psi[2][c], SIGMA);
      h[1][c] = caddi(psi[1][c], psi[3][c], -SIGMA);
    } else {  // h0 = psi0 + s psi2, h1 = psi1 + s psi3
      h[0][c] = SIGMA > 0 ? cadd(psi[0][c], psi[2][c]) : csub(psi[0][c], psi[2][c]);
      h[1][c] = SIGMA > 0 ? cadd(psi[1][c], psi[3][c]) : csub(psi[1][c], psi[3][c]);
    }
  }
}

// out += full spinor rebuilt from the projected, colour-rotated half spinor.
template <int MU, int SIGMA, typename C>
__device__ __forceinline__ void spin_accum(C out[4][3], const C x[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    out[0][c] = cadd(out[0][c], x[0][c]);
    out[1][c] = cadd(out[1][c], x[1][c]);
    if (MU == 0) {  // r2 = -s i h1, r3 = -s i h0
      out[2][c] = caddi(out[2][c], x[1][c], -SIGMA);
      out[3][c] = caddi(out[3][c], x[0][c], -SIGMA);
    } else if (MU == 1) {  // r2 = s h1, r3 = -s h0
      out[2][c] = SIGMA > 0 ? cadd(out[2][c], x[1][c]) : csub(out[2][c], x[1][c]);
      out[3][c] = SIGMA > 0 ? csub(out[3][c], x[0][c]) : cadd(out[3][c], x[0][c]);
    } else if (MU == 2) {  // r2 = -s i h0, r3 = s i h1
      out[2][c] = caddi(out[2][c], x[0][c], -SIGMA);
      out[3][c] = caddi(out[3][c], x[1][c], SIGMA);
    } else {  // r2 = s h0, r3 = s h1
      out[2][c] = SIGMA > 0 ? cadd(out[2][c], x[0][c]) : csub(out[2][c], x[0][c]);
      out[3][c] = SIGMA > 0 ? cadd(out[3][c], x[1][c]) : csub(out[3][c], x[1][c]);
    }
  }
}

// x = U h (DAG = false) or U^+ h (DAG = true) for both spin rows.
template <bool DAG, typename C>
__device__ __forceinline__ void su3_mul(const C u[3][3], const C h[2][3], C x[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      C acc = DAG ? cmulc(u[0][a], h[s][0]) : cmul(u[a][0], h[s][0]);
#pragma unroll
      for (int b = 1; b < 3; ++b) acc = cadd(acc, DAG ? cmulc(u[b][a], h[s][b]) : cmul(u[a][b], h[s][b]));
      x[s][a] = acc;
    }
  }
}

// ------------------------------------------------------------------ context
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct SloppyState;  // mixed-precision workspace (sloppy.cu)

}  // namespace lqcd

struct lqcd_ctx {
  int device = 0;
  int dims[4] = {0, 0, 0, 0};
  lqcd::Geom geom;
  double kappa = 0.0;
  bool have_gauge = false;
  bool gauge_su3 = false;     // links checked SU(3): reconstruct-12 copies are valid
  double2 *U64 = nullptr;     // canonical [V][4][3][3]
  float4 *U32 = nullptr;      // recon-12 FP32  [2 parity][4 mu][3 float4][Vh]
  float4 *Udf = nullptr;      // double-float copy  [V][4][3][3] (hi.re, hi.im, lo.re, lo.im)
  uint4 *U16 = nullptr;       // FP16, all 18 reals, each twice  [2 parity][4 mu][5 uint4][Vh]
  float2 *Utf = nullptr;      // tf32-rounded FP32, [2 parity][4 mu][Vh][3][3] complex (tensor-core hop)
  uint32_t *Ub16 = nullptr;   // BF16 link bundle of the tile hop, [2 parity][Vh][8 dir][3][3] (re, im) pairs
  double2 *Uape = nullptr;    // APE-smeared copy (spatial links smeared) [V][4][3][3], on first use
  bool have_ape = false;
  std::vector<lqcd::DevBuf> ws;  // named workspaces, grow-only
  lqcd::SloppyState *sloppy = nullptr;
  std::string err;
  int *d_flag = nullptr;      // device error flag scratch
  // profiling of the dominant kernel (sloppy hopping term)
  bool prof_on = false;
  unsigned long long *d_prof = nullptr;  // [8] sites processed per hop epilogue kind
  std::vector<cudaEvent_t> prof_ev;       // start/stop pairs
  size_t prof_used = 0;
  long long prof_hop_launches = 0;
  long long prof_launch_base = 0;
  int prof_prec = 0;
  // autotuned launch grid (blocks per SM) per (nrhs, precision)
  std::vector<std::pair<long long, int>> tuned;
  // the autotuner's timings per key: best pair-layout code and its ms per inner
  // iteration, ms of the tile layout (< 0 if not timed); the choice is revised
  // after every solve from its per-RHS iteration counts
  struct TuneRec {
    long long key;
    int pair_code;
    float pair_ms, tile_ms;
  };
  std::vector<TuneRec> tune_ms;
};

namespace lqcd {

// Carve consecutive sub-buffers out of one allocation; every piece starts on
// a 256-byte boundary.  Use carve_size() with the same sequence to size it.
struct Carver {
  char *base;
  size_t off = 0;
  explicit Carver(void *b) : base((char *)b) {}
  template <typename T> T *take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T *p = (T *)(base ? base + off : nullptr);
    off += n * sizeof(T);
    return p;
  }
  size_t size() const { return (off + 255) & ~(size_t)255; }
};

// Kernel launches made by the library (all contexts): KL prefixes every launch.
extern std::atomic<long long> g_launches;
#define KL ++lqcd::g_launches,

// error helpers (api.cu)
int set_error(lqcd_ctx *ctx, int code, const char *fmt, ...);
int cuda_error(lqcd_ctx *ctx, cudaError_t e, const char *where);
void *workspace(lqcd_ctx *ctx, int slot, size_t bytes, int *status);
bool is_device_ptr(const void *p);

#define LQCD_CUDA_TRY(ctx, call)                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_error(ctx, e_, #call); \
  } while (0)

#define LQCD_LAUNCH_CHECK(ctx, what)                       \
  do {                                                     \
    cudaError_t e_ = cudaGetLastError();                   \
    if (e_ != cudaSuccess) return cuda_error(ctx, e_, what); \
  } while (0)

// workspace slots
enum WsSlot {
  WS_STAGE_IN = 0, WS_STAGE_OUT, WS_STAGE_AUX,
  WS_F64_VECS, WS_F64_SCAL, WS_F64_PART, WS_F64_FULL,
  WS_LOOP_PART, WS_GRAD, WS_GRAD2, WS_SMEAR, WS_SMEAR_LINKS,
  WS_COUNT
};

// FP64 kernels (fp64.cu)
int launch_hop64(lqcd_ctx *ctx, cudaStream_t st, bool dag, bool in_canon, bool out_canon, int p_out,
                 const double2 *in, size_t in_stride, double2 *out, size_t out_stride, const double2 *A, double cA,
                 const double2 *B, double cB, double cH, const int *active, int nrhs);
int df_join(lqcd_ctx *ctx, const float4 *in, double2 *out, size_t n, cudaStream_t st);
// r = b - D x in double-float for the n right-hand sides list[0..n) (host
// list); rr, bb (host, indexed by right-hand side) receive |r|^2 and |b|^2
int df_residual(lqcd_ctx *ctx, const float4 *x, const double2 *b, float2 *r, const int *list, int n, double *rr,
                double *bb, cudaStream_t st);
int fp64_true_residual(lqcd_ctx *ctx, const double2 *b, const double2 *x, int nrhs, double *rr, double *bb,
                       cudaStream_t st);
int fp64_apply_dirac(lqcd_ctx *ctx, const double2 *in, double2 *out, int nrhs, bool dagger,
                     cudaStream_t st);
int fp64_solve(lqcd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const lqcd_solver_params &p,
               lqcd_solve_stats *stats, cudaStream_t st);
// sloppy / mixed kernels (sloppy.cu)
int mixed_solve(lqcd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const lqcd_solver_params &p,
                lqcd_solve_stats *stats, cudaStream_t st);
void sloppy_free(lqcd_ctx *ctx);
int pack_gauge_sloppy(lqcd_ctx *ctx, cudaStream_t st);

double wall_ms();

}  // namespace lqcd
