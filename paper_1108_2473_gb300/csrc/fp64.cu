// FP64 path: Wilson hopping term, full-operator application, and the plain
// even-odd preconditioned BiCGstab solver (Sec. II: BiCGstab inversions;
// Sec. III: stop on |M x - b| / |b|).
//
// Layouts: canonical fields are [rhs][V][12] double2 (site-lexicographic);
// solver vectors are parity-compact [rhs][Vh][12] double2 with parity-local
// index i = site >> 1.  The gauge field is the canonical [V][4][9] copy.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace lqcd {

// ------------------------------------------------------------------ hopping
template <int MU, bool DAG, bool IN_CANON>
__device__ __forceinline__ void hop_dir64(const Geom &g, const int c[4], int s, const double2 *__restrict__ in,
                                          const double2 *__restrict__ U, double2 acc[4][3]) {
  constexpr int SF = DAG ? +1 : -1;  // projector sign of the forward hop
  constexpr int SB = -SF;
  double2 ps[4][3], h[2][3], x[2][3], u[3][3];
  // forward: (1 + SF gamma_mu) U_mu(x) psi(x + mu)
  {
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
    int sn = site_of(g, cn);
    const double2 *p = in + (size_t)(IN_CANON ? sn : (sn >> 1)) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) ps[k / 3][k % 3] = p[k];
    const double2 *up = U + ((size_t)s * 4 + MU) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k / 3][k % 3] = up[k];
    spin_project<MU, SF>(ps, h);
    su3_mul<false>(u, h, x);
    if (MU == 3 && c[3] == g.L[3] - 1) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) x[a][b] = cscale(x[a][b], -1.0);
    }
    spin_accum<MU, SF>(acc, x);
  }
  // backward: (1 + SB gamma_mu) U_mu(x - mu)^+ psi(x - mu)
  {
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
    int sn = site_of(g, cn);
    const double2 *p = in + (size_t)(IN_CANON ? sn : (sn >> 1)) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) ps[k / 3][k % 3] = p[k];
    const double2 *up = U + ((size_t)sn * 4 + MU) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k / 3][k % 3] = up[k];
    spin_project<MU, SB>(ps, h);
    su3_mul<true>(u, h, x);
    if (MU == 3 && c[3] == 0) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) x[a][b] = cscale(x[a][b], -1.0);
    }
    spin_accum<MU, SB>(acc, x);
  }
}

// out = cA*A + cB*B + cH*(H in) at the sites of parity p_out, per RHS (grid.y).
// A, B share out's layout; either may be null.  Inactive RHS are skipped.
template <bool DAG, bool IN_CANON, bool OUT_CANON>
__global__ void __launch_bounds__(128) k_hop64(Geom g, int p_out, const double2 *__restrict__ U,
                                               const double2 *__restrict__ in, size_t in_stride, double2 *out,
                                               size_t out_stride, const double2 *A, double cA, const double2 *B,
                                               double cB, double cH, const int *active) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int rhs = blockIdx.y;
  if (i >= g.Vh) return;
  if (active && !active[rhs]) return;
  int c[4];
  coords_of(g, p_out, i, c);
  int s = site_of(g, c);
  double2 acc[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) acc[a][b] = make_double2(0.0, 0.0);
  const double2 *inr = in + (size_t)rhs * in_stride;
  hop_dir64<0, DAG, IN_CANON>(g, c, s, inr, U, acc);
  hop_dir64<1, DAG, IN_CANON>(g, c, s, inr, U, acc);
  hop_dir64<2, DAG, IN_CANON>(g, c, s, inr, U, acc);
  hop_dir64<3, DAG, IN_CANON>(g, c, s, inr, U, acc);
  size_t o = (size_t)rhs * out_stride + (size_t)(OUT_CANON ? s : i) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 v = cscale(acc[k / 3][k % 3], cH);
    if (A) v = cadd(v, cscale(A[o + k], cA));
    if (B) v = cadd(v, cscale(B[o + k], cB));
    out[o + k] = v;
  }
}

int launch_hop64(lqcd_ctx *ctx, cudaStream_t st, bool dag, bool in_canon, bool out_canon, int p_out,
                 const double2 *in, size_t in_stride, double2 *out, size_t out_stride, const double2 *A, double cA,
                 const double2 *B, double cB, double cH, const int *active, int nrhs) {
  const Geom &g = ctx->geom;
  dim3 grid((g.Vh + 127) / 128, nrhs);
#define HOP64_CASE(D, IC, OC)                                                                          \
  if (dag == D && in_canon == IC && out_canon == OC) {                                                 \
    KL k_hop64<D, IC, OC><<<grid, 128, 0, st>>>(g, p_out, ctx->U64, in, in_stride, out, out_stride, A, cA, B, cB, \
                                             cH, active);                                              \
    LQCD_LAUNCH_CHECK(ctx, "k_hop64");                                                                 \
    return LQCD_OK;                                                                                    \
  }
  HOP64_CASE(false, false, false)
  HOP64_CASE(false, true, true)
  HOP64_CASE(false, true, false)
  HOP64_CASE(false, false, true)
  HOP64_CASE(true, true, true)
  HOP64_CASE(true, false, false)
#undef HOP64_CASE
  return set_error(ctx, LQCD_ERR_INVALID, "launch_hop64: unsupported layout combination");
}

int fp64_apply_dirac(lqcd_ctx *ctx, const double2 *in, double2 *out, int nrhs, bool dagger, cudaStream_t st) {
  const Geom &g = ctx->geom;
  size_t stride = (size_t)g.V * 12;
  for (int p = 0; p < 2; ++p) {
    int rc = launch_hop64(ctx, st, dagger, true, true, p, in, stride, out, stride, in, 1.0, nullptr, 0.0,
                          -ctx->kappa, nullptr, nrhs);
    if (rc) return rc;
  }
  return LQCD_OK;
}

// --------------------------------------------------------- layout changes
// canonical [rhs][V][12] -> compact parity p [rhs][Vh][12] (and back)
__global__ void k_split64(Geom g, int p, const double2 *__restrict__ full, double2 *half) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int rhs = blockIdx.y;
  if (i >= g.Vh) return;
  int c[4];
  coords_of(g, p, i, c);
  int s = site_of(g, c);
  const double2 *src = full + ((size_t)rhs * g.V + s) * 12;
  double2 *dst = half + ((size_t)rhs * g.Vh + i) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) dst[k] = src[k];
}

__global__ void k_merge64(Geom g, int p, const double2 *__restrict__ half, double2 *full, const int *active) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int rhs = blockIdx.y;
  if (i >= g.Vh) return;
  if (active && !active[rhs]) return;
  int c[4];
  coords_of(g, p, i, c);
  int s = site_of(g, c);
  const double2 *src = half + ((size_t)rhs * g.Vh + i) * 12;
  double2 *dst = full + ((size_t)rhs * g.V + s) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) dst[k] = src[k];
}

// ------------------------------------------------------------ reductions
struct D4 {
  double a, b, c, d;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of 4 doubles in a fixed order; result valid in thread 0
__device__ __forceinline__ D4 block_sum4(D4 v) {
  __shared__ D4 sh[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v.a = warp_sum(v.a);
  v.b = warp_sum(v.b);
  v.c = warp_sum(v.c);
  v.d = warp_sum(v.d);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  D4 r = {0, 0, 0, 0};
  if (w == 0) {
    int nw = blockDim.x >> 5;
    r = lane < nw ? sh[lane] : D4{0, 0, 0, 0};
    r.a = warp_sum(r.a);
    r.b = warp_sum(r.b);
    r.c = warp_sum(r.c);
    r.d = warp_sum(r.d);
  }
  __syncthreads();
  return r;
}

// per-RHS solver scalars
struct S64 {
  double2 rho, alpha, omega, beta;
  double rr, target2, bb, rel;
  int iters, status, restart, pad;
};

#define RED_THREADS 256

// p = r + beta (p - omega v); on restart: rhat = r, p = r.
__global__ void __launch_bounds__(RED_THREADS) k_bicg_p(size_t n, S64 *sc, const int *active, const double2 *r,
                                                        double2 *rhat, double2 *p, const double2 *v) {
  int rhs = blockIdx.y;
  if (!active[rhs]) return;
  const S64 s = sc[rhs];
  size_t off = (size_t)rhs * n;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double2 rk = r[off + k];
    if (s.restart) {
      rhat[off + k] = rk;
      p[off + k] = rk;
    } else {
      double2 t = csub(p[off + k], cmul(s.omega, v[off + k]));
      p[off + k] = cadd(rk, cmul(s.beta, t));
    }
  }
}

// partial <a, b> (complex) and |b|^2
__global__ void __launch_bounds__(RED_THREADS) k_dot64(size_t n, const int *active, const double2 *a, const double2 *b,
                                                       D4 *part) {
  int rhs = blockIdx.y;
  if (!active[rhs]) return;
  size_t off = (size_t)rhs * n;
  D4 acc = {0, 0, 0, 0};
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double2 x = a[off + k], y = b[off + k];
    double2 t = cmulc(x, y);
    acc.a += t.x;
    acc.b += t.y;
    acc.c += y.x * y.x + y.y * y.y;
  }
  D4 r = block_sum4(acc);
  if (threadIdx.x == 0) part[(size_t)rhs * gridDim.x + blockIdx.x] = r;
}

// s = r - alpha v
__global__ void __launch_bounds__(RED_THREADS) k_bicg_s(size_t n, const S64 *sc, const int *active, const double2 *r,
                                                        const double2 *v, double2 *s) {
  int rhs = blockIdx.y;
  if (!active[rhs]) return;
  double2 al = sc[rhs].alpha;
  size_t off = (size_t)rhs * n;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    s[off + k] = csub(r[off + k], cmul(al, v[off + k]));
}

// x += alpha p + omega s; r = s - omega t; partials <rhat, r>, |r|^2
__global__ void __launch_bounds__(RED_THREADS) k_bicg_xr(size_t n, const S64 *sc, const int *active, double2 *x,
                                                         const double2 *p, const double2 *s, const double2 *t,
                                                         double2 *r, const double2 *rhat, D4 *part) {
  int rhs = blockIdx.y;
  if (!active[rhs]) return;
  double2 al = sc[rhs].alpha, om = sc[rhs].omega;
  size_t off = (size_t)rhs * n;
  D4 acc = {0, 0, 0, 0};
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double2 sk = s[off + k];
    x[off + k] = cadd(x[off + k], cadd(cmul(al, p[off + k]), cmul(om, sk)));
    double2 rk = csub(sk, cmul(om, t[off + k]));
    r[off + k] = rk;
    double2 d = cmulc(rhat[off + k], rk);
    acc.a += d.x;
    acc.b += d.y;
    acc.c += rk.x * rk.x + rk.y * rk.y;
  }
  D4 rr = block_sum4(acc);
  if (threadIdx.x == 0) part[(size_t)rhs * gridDim.x + blockIdx.x] = rr;
}

// fixed-order sum of the nb partials of one RHS by one warp
__device__ __forceinline__ D4 warp_total(const D4 *part, int nb) {
  int lane = threadIdx.x;
  D4 acc = {0, 0, 0, 0};
  for (int k = lane; k < nb; k += 32) {
    D4 v = part[k];
    acc.a += v.a;
    acc.b += v.b;
    acc.c += v.c;
    acc.d += v.d;
  }
  acc.a = warp_sum(acc.a);
  acc.b = warp_sum(acc.b);
  acc.c = warp_sum(acc.c);
  acc.d = warp_sum(acc.d);
  return acc;
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// init: r = b_hat - A x was computed; partials hold <r, r> in .c
__global__ void k_fin_init(S64 *sc, int *active, const D4 *part, int nb, int max_iter) {
  int rhs = blockIdx.x;
  if (!active[rhs]) return;
  D4 t = warp_total(part + (size_t)rhs * nb, nb);
  if (threadIdx.x != 0) return;
  S64 &s = sc[rhs];
  s.rr = t.c;
  s.rho = make_double2(t.c, 0.0);
  s.alpha = s.omega = make_double2(1.0, 0.0);
  s.beta = make_double2(0.0, 0.0);
  s.restart = 1;
  if (!isfinite(t.c)) {
    s.status = LQCD_ERR_NONFINITE;
    active[rhs] = 0;
  } else if (t.c <= s.target2) {
    active[rhs] = 0;
  } else if (s.iters >= max_iter) {
    s.status = LQCD_ERR_NOT_CONVERGED;
    active[rhs] = 0;
  }
}

__global__ void k_fin_alpha(S64 *sc, const int *active, const D4 *part, int nb) {
  int rhs = blockIdx.x;
  if (!active[rhs]) return;
  D4 t = warp_total(part + (size_t)rhs * nb, nb);
  if (threadIdx.x != 0) return;
  S64 &s = sc[rhs];
  double2 rv = make_double2(t.a, t.b);
  s.alpha = (rv.x == 0.0 && rv.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(s.rho, rv);
  s.restart = 0;
}

__global__ void k_fin_omega(S64 *sc, const int *active, const D4 *part, int nb) {
  int rhs = blockIdx.x;
  if (!active[rhs]) return;
  D4 t = warp_total(part + (size_t)rhs * nb, nb);
  if (threadIdx.x != 0) return;
  S64 &s = sc[rhs];
  // part: a,b = <t, s>, c = |s|^2 (from k_dot64(t, s)); need |t|^2: stored in d by k_dot_ts
  double2 ts = make_double2(t.a, t.b);
  s.omega = (t.d == 0.0) ? make_double2(0.0, 0.0) : make_double2(ts.x / t.d, ts.y / t.d);
}

// partials <t, s> and |t|^2
__global__ void __launch_bounds__(RED_THREADS) k_dot_ts(size_t n, const int *active, const double2 *t, const double2 *s,
                                                        D4 *part) {
  int rhs = blockIdx.y;
  if (!active[rhs]) return;
  size_t off = (size_t)rhs * n;
  D4 acc = {0, 0, 0, 0};
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double2 x = t[off + k], y = s[off + k];
    double2 d = cmulc(x, y);
    acc.a += d.x;
    acc.b += d.y;
    acc.d += x.x * x.x + x.y * x.y;
  }
  D4 r = block_sum4(acc);
  if (threadIdx.x == 0) part[(size_t)rhs * gridDim.x + blockIdx.x] = r;
}

__global__ void k_fin_conv(S64 *sc, int *active, const D4 *part, int nb, int max_iter) {
  int rhs = blockIdx.x;
  if (!active[rhs]) return;
  D4 t = warp_total(part + (size_t)rhs * nb, nb);
  if (threadIdx.x != 0) return;
  S64 &s = sc[rhs];
  double2 rho_new = make_double2(t.a, t.b);
  s.rr = t.c;
  s.iters += 1;
  if (!isfinite(t.c) || !isfinite(t.a) || !isfinite(t.b)) {
    s.status = LQCD_ERR_NONFINITE;
    active[rhs] = 0;
    return;
  }
  if (t.c <= s.target2) {
    active[rhs] = 0;
    return;
  }
  if (s.iters >= max_iter) {
    s.status = LQCD_ERR_NOT_CONVERGED;
    active[rhs] = 0;
    return;
  }
  double om2 = s.omega.x * s.omega.x + s.omega.y * s.omega.y;
  double rho2 = rho_new.x * rho_new.x + rho_new.y * rho_new.y;
  if (om2 == 0.0 || rho2 == 0.0 || rho2 < 1e-60 * t.c * t.c) {
    // breakdown: restart the shadow residual at the current residual
    s.restart = 1;
    s.rho = make_double2(t.c, 0.0);
    s.alpha = s.omega = make_double2(1.0, 0.0);
    s.beta = make_double2(0.0, 0.0);
    return;
  }
  s.beta = cmul(cdiv(rho_new, s.rho), cdiv(s.alpha, s.omega));
  s.rho = rho_new;
}

// partial |r|^2 -> .c and |b|^2 -> .d (canonical full fields), for the true
// residual; SAME (r == b) sums once and copies, halving the FP64-pipe work
template <bool SAME>
__global__ void __launch_bounds__(RED_THREADS) k_norms64(size_t n, const double2 *r, const double2 *b, D4 *part) {
  int rhs = blockIdx.y;
  size_t off = (size_t)rhs * n;
  D4 acc = {0, 0, 0, 0};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  // four elements loaded before they are summed (in the same order as one at a time)
  for (; k + 3 * stride < n; k += 4 * stride) {
    double2 x[4], y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[u] = r[off + k + u * stride];
      if (!SAME) y[u] = b[off + k + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc.c += x[u].x * x[u].x + x[u].y * x[u].y;
      if (!SAME) acc.d += y[u].x * y[u].x + y[u].y * y[u].y;
    }
  }
  for (; k < n; k += stride) {
    double2 x = r[off + k];
    acc.c += x.x * x.x + x.y * x.y;
    if (!SAME) {
      double2 y = b[off + k];
      acc.d += y.x * y.x + y.y * y.y;
    }
  }
  if (SAME) acc.d = acc.c;
  D4 rr = block_sum4(acc);
  if (threadIdx.x == 0) part[(size_t)rhs * gridDim.x + blockIdx.x] = rr;
}

__global__ void k_fin_norms(const D4 *part, int nb, double *out_rr, double *out_bb) {
  int rhs = blockIdx.x;
  D4 t = warp_total(part + (size_t)rhs * nb, nb);
  if (threadIdx.x == 0) {
    out_rr[rhs] = t.c;
    out_bb[rhs] = t.d;
  }
}

static int red_blocks(size_t n) {
  size_t nb = (n + 2047) / 2048;
  if (nb < 1) nb = 1;
  if (nb > 304) nb = 304;
  return (int)nb;
}

// true residual |b - D x|^2 and |b|^2 per RHS (host arrays), FP64 full lattice
int fp64_true_residual(lqcd_ctx *ctx, const double2 *b, const double2 *x, int nrhs, double *rr, double *bb,
                       cudaStream_t st) {
  const Geom &g = ctx->geom;
  size_t stride = (size_t)g.V * 12;
  int rc = LQCD_OK;
  double2 *res = (double2 *)workspace(ctx, WS_F64_FULL, (size_t)nrhs * stride * sizeof(double2), &rc);
  if (!res) return rc;
  int nb = red_blocks(stride);
  Carver sizing(nullptr);
  sizing.take<D4>((size_t)nrhs * nb);
  sizing.take<double>(2 * (size_t)nrhs);
  void *pw = workspace(ctx, WS_F64_PART, sizing.size(), &rc);
  if (!pw) return rc;
  Carver cv(pw);
  D4 *part = cv.take<D4>((size_t)nrhs * nb);
  double *d_rr = cv.take<double>(2 * (size_t)nrhs);
  double *d_bb = d_rr + nrhs;
  for (int p = 0; p < 2; ++p) {
    // res = b - x + kappa H x
    rc = launch_hop64(ctx, st, false, true, true, p, x, stride, res, stride, b, 1.0, x, -1.0, ctx->kappa, nullptr,
                      nrhs);
    if (rc) return rc;
  }
  KL k_norms64<false><<<dim3(nb, nrhs), RED_THREADS, 0, st>>>(stride, res, b, part);
  LQCD_LAUNCH_CHECK(ctx, "k_norms64");
  KL k_fin_norms<<<nrhs, 32, 0, st>>>(part, nb, d_rr, d_bb);
  LQCD_LAUNCH_CHECK(ctx, "k_fin_norms");
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(rr, d_rr, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(bb, d_bb, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return LQCD_OK;
}

// res = b - x + kappa H x at the sites of parity p (canonical layout), with
// per-block partials of |res|^2 (.c) and |b|^2 (.d) at part[rhs][p * nblk + block]
__global__ void __launch_bounds__(128) k_resid64(Geom g, int p_out, const double2 *__restrict__ U,
                                                 const double2 *__restrict__ x, const double2 *__restrict__ b,
                                                 double2 *res, double kappa, D4 *part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  const size_t stride = (size_t)g.V * 12;
  D4 nrm = {0, 0, 0, 0};
  if (i < g.Vh) {
    int c[4];
    coords_of(g, p_out, i, c);
    int s = site_of(g, c);
    double2 acc[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 3; ++q) acc[a][q] = make_double2(0.0, 0.0);
    const double2 *xr = x + (size_t)rhs * stride;
    hop_dir64<0, false, true>(g, c, s, xr, U, acc);
    hop_dir64<1, false, true>(g, c, s, xr, U, acc);
    hop_dir64<2, false, true>(g, c, s, xr, U, acc);
    hop_dir64<3, false, true>(g, c, s, xr, U, acc);
    size_t o = (size_t)rhs * stride + (size_t)s * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 bk = b[o + k], xk = x[o + k];
      double2 v = cadd(csub(bk, xk), cscale(acc[k / 3][k % 3], kappa));
      res[o + k] = v;
      nrm.c += v.x * v.x + v.y * v.y;
      nrm.d += bk.x * bk.x + bk.y * bk.y;
    }
  }
  D4 t = block_sum4(nrm);
  if (threadIdx.x == 0) part[(size_t)rhs * 2 * gridDim.x + (size_t)p_out * gridDim.x + blockIdx.x] = t;
}

// res = b - D x (canonical FP64) and per-RHS |res|^2, |b|^2 (host arrays).
// With x = null the residual is b itself: only the norms are computed.
int fp64_residual_into(lqcd_ctx *ctx, const double2 *b, const double2 *x, double2 *res, int nrhs, double *rr,
                       double *bb, cudaStream_t st) {
  const Geom &g = ctx->geom;
  size_t stride = (size_t)g.V * 12;
  int rc = LQCD_OK;
  int nblk = (g.Vh + 127) / 128;
  int nb = x ? 2 * nblk : red_blocks(stride);
  Carver sizing(nullptr);
  sizing.take<D4>((size_t)nrhs * nb);
  sizing.take<double>(2 * (size_t)nrhs);
  void *pw = workspace(ctx, WS_F64_PART, sizing.size(), &rc);
  if (!pw) return rc;
  Carver cv(pw);
  D4 *part = cv.take<D4>((size_t)nrhs * nb);
  double *d_rr = cv.take<double>(2 * (size_t)nrhs);
  double *d_bb = d_rr + nrhs;
  if (x) {
    for (int p = 0; p < 2; ++p) {
      KL k_resid64<<<dim3(nblk, nrhs), 128, 0, st>>>(g, p, ctx->U64, x, b, res, ctx->kappa, part);
      LQCD_LAUNCH_CHECK(ctx, "k_resid64");
    }
  } else {
    KL k_norms64<true><<<dim3(nb, nrhs), RED_THREADS, 0, st>>>(stride, b, b, part);
    LQCD_LAUNCH_CHECK(ctx, "k_norms64");
  }
  KL k_fin_norms<<<nrhs, 32, 0, st>>>(part, nb, d_rr, d_bb);
  LQCD_LAUNCH_CHECK(ctx, "k_fin_norms");
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(rr, d_rr, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(bb, d_bb, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return LQCD_OK;
}

// ------------------------------------------------------------- the solver
// One block of nrhs right-hand sides, even-odd BiCGstab in FP64.
static int fp64_solve_block(lqcd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const lqcd_solver_params &p,
                            lqcd_solve_stats *stats, cudaStream_t st, double t_start) {
  const Geom &g = ctx->geom;
  const double kappa = ctx->kappa;
  size_t n = (size_t)g.Vh * 12;  // double2 per parity vector
  size_t full = (size_t)g.V * 12;
  const int NV = 10;
  int rc = LQCD_OK;
  double2 *vec = (double2 *)workspace(ctx, WS_F64_VECS, (size_t)NV * nrhs * n * sizeof(double2), &rc);
  if (!vec) return rc;
  double2 *xe = vec, *r = vec + (size_t)nrhs * n, *rhat = r + (size_t)nrhs * n, *pp = rhat + (size_t)nrhs * n;
  double2 *v = pp + (size_t)nrhs * n, *s = v + (size_t)nrhs * n, *t = s + (size_t)nrhs * n;
  double2 *tmp = t + (size_t)nrhs * n, *bo = tmp + (size_t)nrhs * n, *bhat = bo + (size_t)nrhs * n;
  int nb = red_blocks(n);
  Carver sizing(nullptr);
  sizing.take<S64>(nrhs);
  sizing.take<int>(nrhs);
  sizing.take<D4>((size_t)nrhs * nb);
  char *sw = (char *)workspace(ctx, WS_F64_SCAL, sizing.size(), &rc);
  if (!sw) return rc;
  Carver cv(sw);
  S64 *sc = cv.take<S64>(nrhs);
  int *active = cv.take<int>(nrhs);
  D4 *part = cv.take<D4>((size_t)nrhs * nb);

  std::vector<double> rr(nrhs), bb(nrhs), target2(nrhs);
  std::vector<S64> hs(nrhs);
  std::vector<int> hact(nrhs);
  dim3 gv((g.Vh + 127) / 128, nrhs), gr(nb, nrhs);

  // |b|^2 of the full source (FP64)
  {
    LQCD_CUDA_TRY(ctx, cudaMemsetAsync(x, 0, (size_t)nrhs * full * sizeof(double2), st));
    rc = fp64_true_residual(ctx, b, x, nrhs, rr.data(), bb.data(), st);
    if (rc) return rc;
  }
  // b_e, b_o and b_hat = b_e + kappa H_eo b_o
  KL k_split64<<<gv, 128, 0, st>>>(g, 1, b, bo);
  KL k_split64<<<gv, 128, 0, st>>>(g, 0, b, tmp);
  LQCD_LAUNCH_CHECK(ctx, "k_split64");
  rc = launch_hop64(ctx, st, false, false, false, 0, bo, n, bhat, n, tmp, 1.0, nullptr, 0.0, kappa, nullptr, nrhs);
  if (rc) return rc;
  LQCD_CUDA_TRY(ctx, cudaMemsetAsync(xe, 0, (size_t)nrhs * n * sizeof(double2), st));
  for (int k = 0; k < nrhs; ++k) {
    hs[k] = S64{};
    target2[k] = 0.25 * p.tol * p.tol * bb[k];
    hs[k].target2 = target2[k];
    hs[k].bb = bb[k];
    hact[k] = 1;
  }
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sc, hs.data(), nrhs * sizeof(S64), cudaMemcpyHostToDevice, st));
  const int max_restarts = 6;
  for (int restart = 0; restart <= max_restarts; ++restart) {
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(active, hact.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
    // r = b_hat - D_hat x_e = b_hat - x_e + kappa^2 H_eo H_oe x_e
    rc = launch_hop64(ctx, st, false, false, false, 1, xe, n, tmp, n, nullptr, 0.0, nullptr, 0.0, 1.0, active, nrhs);
    if (rc) return rc;
    rc = launch_hop64(ctx, st, false, false, false, 0, tmp, n, r, n, bhat, 1.0, xe, -1.0, kappa * kappa, active, nrhs);
    if (rc) return rc;
    KL k_dot64<<<gr, RED_THREADS, 0, st>>>(n, active, r, r, part);
    KL k_fin_init<<<nrhs, 32, 0, st>>>(sc, active, part, nb, p.max_iter);
    LQCD_LAUNCH_CHECK(ctx, "init");
    bool any = true, timed_out = false;
    while (any) {
      for (int it = 0; it < 4; ++it) {
        KL k_bicg_p<<<gr, RED_THREADS, 0, st>>>(n, sc, active, r, rhat, pp, v);
        launch_hop64(ctx, st, false, false, false, 1, pp, n, tmp, n, nullptr, 0.0, nullptr, 0.0, 1.0, active, nrhs);
        launch_hop64(ctx, st, false, false, false, 0, tmp, n, v, n, pp, 1.0, nullptr, 0.0, -kappa * kappa, active,
                     nrhs);
        KL k_dot64<<<gr, RED_THREADS, 0, st>>>(n, active, rhat, v, part);
        KL k_fin_alpha<<<nrhs, 32, 0, st>>>(sc, active, part, nb);
        KL k_bicg_s<<<gr, RED_THREADS, 0, st>>>(n, sc, active, r, v, s);
        launch_hop64(ctx, st, false, false, false, 1, s, n, tmp, n, nullptr, 0.0, nullptr, 0.0, 1.0, active, nrhs);
        launch_hop64(ctx, st, false, false, false, 0, tmp, n, t, n, s, 1.0, nullptr, 0.0, -kappa * kappa, active,
                     nrhs);
        KL k_dot_ts<<<gr, RED_THREADS, 0, st>>>(n, active, t, s, part);
        KL k_fin_omega<<<nrhs, 32, 0, st>>>(sc, active, part, nb);
        KL k_bicg_xr<<<gr, RED_THREADS, 0, st>>>(n, sc, active, xe, pp, s, t, r, rhat, part);
        KL k_fin_conv<<<nrhs, 32, 0, st>>>(sc, active, part, nb, p.max_iter);
      }
      LQCD_LAUNCH_CHECK(ctx, "bicgstab iteration");
      LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(hact.data(), active, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
      LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
      any = false;
      for (int k = 0; k < nrhs; ++k) any = any || hact[k];
      if (any && p.timeout_ms > 0 && wall_ms() - t_start > p.timeout_ms) {
        timed_out = true;
        break;
      }
    }
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(hs.data(), sc, nrhs * sizeof(S64), cudaMemcpyDeviceToHost, st));
    LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    // x_o = b_o + kappa H_oe x_e ; merge into canonical x
    rc = launch_hop64(ctx, st, false, false, false, 1, xe, n, tmp, n, bo, 1.0, nullptr, 0.0, kappa, nullptr, nrhs);
    if (rc) return rc;
    KL k_merge64<<<gv, 128, 0, st>>>(g, 0, xe, x, nullptr);
    KL k_merge64<<<gv, 128, 0, st>>>(g, 1, tmp, x, nullptr);
    LQCD_LAUNCH_CHECK(ctx, "k_merge64");
    rc = fp64_true_residual(ctx, b, x, nrhs, rr.data(), bb.data(), st);
    if (rc) return rc;
    bool again = false;
    for (int k = 0; k < nrhs; ++k) {
      double rel = bb[k] > 0 ? std::sqrt(rr[k] / bb[k]) : 0.0;
      stats[k].iterations = hs[k].iters;
      stats[k].true_rel_residual = rel;
      stats[k].reliable_updates = 0;
      stats[k].restarts = restart;
      int status = hs[k].status;
      if (timed_out && status == LQCD_OK && !(rel <= p.tol)) status = LQCD_ERR_TIMEOUT;
      if (status == LQCD_OK && !std::isfinite(rel)) status = LQCD_ERR_NONFINITE;
      stats[k].status = status;
      hact[k] = 0;
      if (status == LQCD_OK && rel > p.tol) {
        if (restart == max_restarts) {
          stats[k].status = LQCD_ERR_NOT_CONVERGED;
        } else {
          hact[k] = 1;
          again = true;
          target2[k] *= 0.01;
          hs[k].target2 = target2[k];
        }
      }
    }
    if (!again || timed_out) break;
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sc, hs.data(), nrhs * sizeof(S64), cudaMemcpyHostToDevice, st));
  }
  return LQCD_OK;
}

// ------------------------------------------------------------ CG (CGNR)
// CG on the normal equations of the Schur operator A = D_hat:
// A^+ A x = A^+ b_hat, with A^+ = gamma5 A gamma5 (the dagger hopping term),
// stopping on the Schur residual s = b_hat - A x (tracked by the recursion and
// checked against the true full-lattice FP64 residual afterwards).
struct SCG {
  double alpha, beta, rr, ss, target2;
  int iters, status, pad;
};

__global__ void k_cg_fin_init(SCG *sc, int *active, const D4 *part_r, const D4 *part_s, int nb, int max_iter) {
  int rhs = blockIdx.x;
  if (!active[rhs]) return;
  D4 tr = warp_total(part_r + (size_t)rhs * nb, nb);
  D4 ts = warp_total(part_s + (size_t)rhs * nb, nb);
  if (threadIdx.x) return;
  SCG &c = sc[rhs];
  c.rr = tr.c;
  c.ss = ts.c;
  if (!isfinite(tr.c) || !isfinite(ts.c)) {
    c.status = LQCD_ERR_NONFINITE;
    active[rhs] = 0;
  } else if (ts.c <= c.target2 || tr.c == 0.0) {
    active[rhs] = 0;
  } else if (c.iters >= max_iter) {
    c.status = LQCD_ERR_NOT_CONVERGED;
    active[rhs] = 0;
  }
}

__global__ void k_cg_fin_alpha(SCG *sc, const int *active, const D4 *part, int nb) {
  int rhs = blockIdx.x;
  if (!active[rhs]) return;
  D4 t = warp_total(part + (size_t)rhs * nb, nb);  // |A p|^2 in .c
  if (threadIdx.x) return;
  sc[rhs].alpha = t.c > 0.0 ? sc[rhs].rr / t.c : 0.0;
}

// x += alpha p; s -= alpha q; partial |s|^2
__global__ void __launch_bounds__(RED_THREADS) k_cg_xs(size_t n, const SCG *sc, const int *active, double2 *x,
                                                       const double2 *p, double2 *s, const double2 *q, D4 *part) {
  int rhs = blockIdx.y;
  if (!active[rhs]) return;
  double a = sc[rhs].alpha;
  size_t off = (size_t)rhs * n;
  D4 acc = {0, 0, 0, 0};
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    x[off + k] = cadd(x[off + k], cscale(p[off + k], a));
    double2 v = csub(s[off + k], cscale(q[off + k], a));
    s[off + k] = v;
    acc.c += v.x * v.x + v.y * v.y;
  }
  D4 r = block_sum4(acc);
  if (threadIdx.x == 0) part[(size_t)rhs * gridDim.x + blockIdx.x] = r;
}

__global__ void k_cg_fin_ss(SCG *sc, int *active, const D4 *part, int nb, int max_iter) {
  int rhs = blockIdx.x;
  if (!active[rhs]) return;
  D4 t = warp_total(part + (size_t)rhs * nb, nb);
  if (threadIdx.x) return;
  SCG &c = sc[rhs];
  c.ss = t.c;
  c.iters += 1;
  if (!isfinite(t.c)) {
    c.status = LQCD_ERR_NONFINITE;
    active[rhs] = 0;
  } else if (t.c <= c.target2) {
    active[rhs] = 0;
  } else if (c.iters >= max_iter) {
    c.status = LQCD_ERR_NOT_CONVERGED;
    active[rhs] = 0;
  }
}

__global__ void k_cg_fin_beta(SCG *sc, const int *active, const D4 *part, int nb) {
  int rhs = blockIdx.x;
  if (!active[rhs]) return;
  D4 t = warp_total(part + (size_t)rhs * nb, nb);
  if (threadIdx.x) return;
  SCG &c = sc[rhs];
  c.beta = c.rr > 0.0 ? t.c / c.rr : 0.0;
  c.rr = t.c;
}

// p = r + beta p (beta = 0 on the first use)
__global__ void __launch_bounds__(RED_THREADS) k_cg_p(size_t n, const SCG *sc, const int *active, const double2 *r,
                                                      double2 *p) {
  int rhs = blockIdx.y;
  if (!active[rhs]) return;
  double b = sc[rhs].beta;
  size_t off = (size_t)rhs * n;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    p[off + k] = cadd(r[off + k], cscale(p[off + k], b));
}

static int fp64_cg_block(lqcd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const lqcd_solver_params &p,
                         lqcd_solve_stats *stats, cudaStream_t st, double t_start) {
  const Geom &g = ctx->geom;
  const double kappa = ctx->kappa, k2 = kappa * kappa;
  size_t n = (size_t)g.Vh * 12;
  int rc = LQCD_OK;
  double2 *vec = (double2 *)workspace(ctx, WS_F64_VECS, (size_t)9 * nrhs * n * sizeof(double2), &rc);
  if (!vec) return rc;
  double2 *xe = vec, *s = vec + (size_t)nrhs * n, *r = s + (size_t)nrhs * n, *pp = r + (size_t)nrhs * n;
  double2 *q = pp + (size_t)nrhs * n, *tmp = q + (size_t)nrhs * n, *bo = tmp + (size_t)nrhs * n;
  double2 *bhat = bo + (size_t)nrhs * n, *be = bhat + (size_t)nrhs * n;
  int nb = red_blocks(n);
  Carver sizing(nullptr);
  sizing.take<SCG>(nrhs);
  sizing.take<int>(nrhs);
  sizing.take<D4>((size_t)nrhs * nb);
  sizing.take<D4>((size_t)nrhs * nb);
  char *sw = (char *)workspace(ctx, WS_F64_SCAL, sizing.size(), &rc);
  if (!sw) return rc;
  Carver cv(sw);
  SCG *sc = cv.take<SCG>(nrhs);
  int *active = cv.take<int>(nrhs);
  D4 *part = cv.take<D4>((size_t)nrhs * nb);
  D4 *part2 = cv.take<D4>((size_t)nrhs * nb);
  std::vector<double> rr(nrhs), bb(nrhs);
  std::vector<SCG> hs(nrhs);
  std::vector<int> hact(nrhs, 1);
  dim3 gv((g.Vh + 127) / 128, nrhs), gr(nb, nrhs);
  LQCD_CUDA_TRY(ctx, cudaMemsetAsync(x, 0, (size_t)nrhs * g.V * 12 * sizeof(double2), st));
  rc = fp64_true_residual(ctx, b, x, nrhs, rr.data(), bb.data(), st);  // |b|^2
  if (rc) return rc;
  KL k_split64<<<gv, 128, 0, st>>>(g, 1, b, bo);
  KL k_split64<<<gv, 128, 0, st>>>(g, 0, b, be);
  rc = launch_hop64(ctx, st, false, false, false, 0, bo, n, bhat, n, be, 1.0, nullptr, 0.0, kappa, nullptr, nrhs);
  if (rc) return rc;
  LQCD_CUDA_TRY(ctx, cudaMemsetAsync(xe, 0, (size_t)nrhs * n * sizeof(double2), st));
  for (int k = 0; k < nrhs; ++k) {
    hs[k] = SCG{};
    hs[k].target2 = 0.25 * p.tol * p.tol * bb[k];
  }
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sc, hs.data(), nrhs * sizeof(SCG), cudaMemcpyHostToDevice, st));
  const int max_restarts = 6;
  for (int restart = 0; restart <= max_restarts; ++restart) {
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(active, hact.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
    // s = b_hat - A x_e ; r = A^+ s ; p = r
    launch_hop64(ctx, st, false, false, false, 1, xe, n, tmp, n, nullptr, 0.0, nullptr, 0.0, 1.0, active, nrhs);
    launch_hop64(ctx, st, false, false, false, 0, tmp, n, s, n, bhat, 1.0, xe, -1.0, k2, active, nrhs);
    launch_hop64(ctx, st, true, false, false, 1, s, n, tmp, n, nullptr, 0.0, nullptr, 0.0, 1.0, active, nrhs);
    launch_hop64(ctx, st, true, false, false, 0, tmp, n, r, n, s, 1.0, nullptr, 0.0, -k2, active, nrhs);
    KL k_dot64<<<gr, RED_THREADS, 0, st>>>(n, active, r, r, part);
    KL k_dot64<<<gr, RED_THREADS, 0, st>>>(n, active, s, s, part2);
    KL k_cg_fin_init<<<nrhs, 32, 0, st>>>(sc, active, part, part2, nb, p.max_iter);
    LQCD_CUDA_TRY(ctx, cudaMemsetAsync(pp, 0, (size_t)nrhs * n * sizeof(double2), st));
    {  // beta = 0 for the first direction
      std::vector<SCG> tmp_h(nrhs);
      LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(tmp_h.data(), sc, nrhs * sizeof(SCG), cudaMemcpyDeviceToHost, st));
      LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
      for (auto &c : tmp_h) c.beta = 0.0;
      LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sc, tmp_h.data(), nrhs * sizeof(SCG), cudaMemcpyHostToDevice, st));
    }
    KL k_cg_p<<<gr, RED_THREADS, 0, st>>>(n, sc, active, r, pp);
    bool any = true, timed_out = false;
    while (any) {
      for (int it = 0; it < 4; ++it) {
        // q = A p
        launch_hop64(ctx, st, false, false, false, 1, pp, n, tmp, n, nullptr, 0.0, nullptr, 0.0, 1.0, active, nrhs);
        launch_hop64(ctx, st, false, false, false, 0, tmp, n, q, n, pp, 1.0, nullptr, 0.0, -k2, active, nrhs);
        KL k_dot64<<<gr, RED_THREADS, 0, st>>>(n, active, q, q, part);
        KL k_cg_fin_alpha<<<nrhs, 32, 0, st>>>(sc, active, part, nb);
        KL k_cg_xs<<<gr, RED_THREADS, 0, st>>>(n, sc, active, xe, pp, s, q, part);
        KL k_cg_fin_ss<<<nrhs, 32, 0, st>>>(sc, active, part, nb, p.max_iter);
        // r = A^+ s
        launch_hop64(ctx, st, true, false, false, 1, s, n, tmp, n, nullptr, 0.0, nullptr, 0.0, 1.0, active, nrhs);
        launch_hop64(ctx, st, true, false, false, 0, tmp, n, r, n, s, 1.0, nullptr, 0.0, -k2, active, nrhs);
        KL k_dot64<<<gr, RED_THREADS, 0, st>>>(n, active, r, r, part);
        KL k_cg_fin_beta<<<nrhs, 32, 0, st>>>(sc, active, part, nb);
        KL k_cg_p<<<gr, RED_THREADS, 0, st>>>(n, sc, active, r, pp);
      }
      LQCD_LAUNCH_CHECK(ctx, "cg iteration");
      LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(hact.data(), active, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
      LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
      any = false;
      for (int k = 0; k < nrhs; ++k) any = any || hact[k];
      if (any && p.timeout_ms > 0 && wall_ms() - t_start > p.timeout_ms) {
        timed_out = true;
        break;
      }
    }
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(hs.data(), sc, nrhs * sizeof(SCG), cudaMemcpyDeviceToHost, st));
    rc = launch_hop64(ctx, st, false, false, false, 1, xe, n, tmp, n, bo, 1.0, nullptr, 0.0, kappa, nullptr, nrhs);
    if (rc) return rc;
    KL k_merge64<<<gv, 128, 0, st>>>(g, 0, xe, x, nullptr);
    KL k_merge64<<<gv, 128, 0, st>>>(g, 1, tmp, x, nullptr);
    LQCD_LAUNCH_CHECK(ctx, "k_merge64");
    rc = fp64_true_residual(ctx, b, x, nrhs, rr.data(), bb.data(), st);
    if (rc) return rc;
    bool again = false;
    for (int k = 0; k < nrhs; ++k) {
      double rel = bb[k] > 0 ? std::sqrt(rr[k] / bb[k]) : 0.0;
      stats[k].iterations = hs[k].iters;
      stats[k].true_rel_residual = rel;
      stats[k].reliable_updates = 0;
      stats[k].restarts = restart;
      int status = hs[k].status;
      if (timed_out && status == LQCD_OK && !(rel <= p.tol)) status = LQCD_ERR_TIMEOUT;
      if (status == LQCD_OK && !std::isfinite(rel)) status = LQCD_ERR_NONFINITE;
      stats[k].status = status;
      hact[k] = 0;
      if (status == LQCD_OK && rel > p.tol) {
        if (restart == max_restarts) {
          stats[k].status = LQCD_ERR_NOT_CONVERGED;
        } else {
          hact[k] = 1;
          again = true;
          hs[k].target2 *= 0.01;
        }
      }
    }
    if (!again || timed_out) break;
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(sc, hs.data(), nrhs * sizeof(SCG), cudaMemcpyHostToDevice, st));
  }
  return LQCD_OK;
}

int fp64_solve(lqcd_ctx *ctx, const double2 *b, double2 *x, int nrhs, const lqcd_solver_params &p,
               lqcd_solve_stats *stats, cudaStream_t st) {
  int blk = p.rhs_block > 0 ? p.rhs_block : 1;  // the plain solver: one RHS at a time
  if (blk > 65535) blk = 65535;
  double t0 = wall_ms();
  size_t full = (size_t)ctx->geom.V * 12;
  int worst = LQCD_OK;
  for (int k0 = 0; k0 < nrhs; k0 += blk) {
    int nk = nrhs - k0 < blk ? nrhs - k0 : blk;
    int rc = p.solver == LQCD_SOLVER_CG ? fp64_cg_block(ctx, b + k0 * full, x + k0 * full, nk, p, stats + k0, st, t0)
                                        : fp64_solve_block(ctx, b + k0 * full, x + k0 * full, nk, p, stats + k0, st, t0);
    if (rc) return rc;
    for (int k = 0; k < nk; ++k)
      if (worst == LQCD_OK && stats[k0 + k].status != LQCD_OK) worst = stats[k0 + k].status;
  }
  if (worst != LQCD_OK) set_error(ctx, worst, "lqcd_solve_batch: some right-hand sides did not converge");
  return worst;
}

}  // namespace lqcd
