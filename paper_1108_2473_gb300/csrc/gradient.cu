// Gradients of the loop estimator by adjoint solves (the paper computes none;
// these are the derivatives of its Eq. loop stochastic for fixed noise).
//
// For a real loss of the per-time-slice loops L_g(t) with upstream gradient
// c[t][g] = d loss / d Re L_g(t) + i d loss / d Im L_g(t):
//   d loss = Re sum_d xi_d^+ M dG xi_d,  M(x) = sum_g conj(c[t(x)][g]) Gamma_g,
//   dG = kappa G dH G (links),  dG = G H G dkappa,
// so with phi_d = G xi_d (forward solutions) and
//   eta_d = gamma5 M^+ xi_d,  D y_d = eta_d,  chi_d = gamma5 y_d  (= G^+ M^+ xi_d,
//   using D^+ = gamma5 D gamma5):
//   d loss / d kappa = Re sum_d chi_d^+ H phi_d,
//   d loss / d U_mu(x) = kappa s (X^* + Y^T)   (torch complex-gradient convention),
//     X_ij = sum_ab chi(x)^*_ai (1 - gamma_mu)_ab phi(x+mu)_bj,
//     Y_ij = sum_ab chi(x+mu)^*_ai (1 + gamma_mu)_ab phi(x)_bj,
//   s = -1 on links crossing t = Lt-1 -> 0.  chi^+ H phi = sum over links of
//   s [sum_ij U_ij X_ij + sum_ij conj(U_ji) Y_ij].
#include <vector>

#include "internal.cuh"

namespace lqcd {

__device__ __forceinline__ double2 gphase(int ph, double2 v) {
  switch (ph) {
    case 0: return v;
    case 1: return make_double2(-v.x, -v.y);
    case 2: return make_double2(-v.y, v.x);
    default: return make_double2(v.y, -v.x);
  }
}
__host__ __device__ constexpr int g_col(int g, int a) { return g < 2 ? a : (g < 4 ? 3 - a : (a + 2) & 3); }
__host__ __device__ constexpr int g_ph(int g, int a) {
  return g == 0 ? 0
         : g == 1 ? (a < 2 ? 0 : 1)
         : g == 2 ? (a < 2 ? 2 : 3)
         : g == 3 ? ((a == 0 || a == 3) ? 1 : 0)
         : g == 4 ? ((a == 0 || a == 3) ? 2 : 3)
                  : 0;
}

// eta(x) = gamma5 sum_g c[t(x)][g] Gamma_g src(x)   (Gamma_g Hermitian: M^+ = sum_g c Gamma_g)
__global__ void k_adj_source(Geom g, const double2 *__restrict__ src, const double2 *__restrict__ coef,
                             double2 *eta, int nrhs) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nrhs * g.V) return;
  int s = (int)(idx % g.V);
  int t = s / (g.L[0] * g.L[1] * g.L[2]);
  const double2 *in = src + idx * 12;
  double2 v[12], o[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    v[k] = in[k];
    o[k] = make_double2(0.0, 0.0);
  }
#pragma unroll
  for (int gi = 0; gi < 6; ++gi) {
    double2 c = coef[t * 6 + gi];
    if (c.x == 0.0 && c.y == 0.0) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int col = 0; col < 3; ++col) {
        double2 gv = gphase(g_ph(gi, a), v[g_col(gi, a) * 3 + col]);
        o[a * 3 + col] = cadd(o[a * 3 + col], cmul(c, gv));
      }
  }
  double2 *out = eta + idx * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) out[k] = (k >= 6) ? make_double2(-o[k].x, -o[k].y) : o[k];  // gamma5
}

// Upper two spin components of (1 + S gamma_mu) v (DeGrand-Rossi), S = +-1.
// (1 + S gamma_mu) / 2 is a Hermitian projector whose lower two components are
// a phase times a swap of the upper two, so for any chi, phi
//   chi^+ (1 + S gamma_mu) phi = sum_{a=0,1} conj(h(chi)_a) . h(phi)_a,
// h = these upper components: half the spin sum of the full outer product.
// chi = gamma5 y flips the sign of the lower spins of y (G5 = -1 here).
template <int MU, int S, int G5>
__device__ __forceinline__ void half_proj(const double2 *__restrict__ v, double2 h[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double2 p0 = v[c], p1 = v[3 + c];
    double2 p2 = v[6 + c], p3 = v[9 + c];
    if (G5 < 0) {
      p2 = cscale(p2, -1.0);
      p3 = cscale(p3, -1.0);
    }
    double2 g0, g1;  // upper components of gamma_mu v
    if (MU == 0) {
      g0 = cmuli(p3); g1 = cmuli(p2);
    } else if (MU == 1) {
      g0 = cscale(p3, -1.0); g1 = p2;
    } else if (MU == 2) {
      g0 = cmuli(p2); g1 = cscale(cmuli(p3), -1.0);
    } else {
      g0 = p2; g1 = p3;
    }
    h[c] = S > 0 ? cadd(p0, g0) : csub(p0, g0);
    h[3 + c] = S > 0 ? cadd(p1, g1) : csub(p1, g1);
  }
}

// out_ij += sum_{a=0,1} conj(a_ai) b_aj
__device__ __forceinline__ void outer_acc2(const double2 a[6], const double2 b[6], double2 out[3][3]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) out[i][j] = cadd(out[i][j], cmulc(a[sp * 3 + i], b[sp * 3 + j]));
}

// Link (s, MU): X = sum_r chi_r(x)^+ (1 - gamma_mu) phi_r(x+mu) and
// Y = sum_r chi_r(x+mu)^+ (1 + gamma_mu) phi_r(x) as colour matrices, summed
// over the right-hand sides in order; then the d/dkappa link term and dU.
template <int MU>
__device__ __forceinline__ double force_link(const Geom &g, int s, const double2 *__restrict__ U,
                                             const double2 *__restrict__ y, const double2 *__restrict__ phi,
                                             int nrhs, double kappa, double weight, double2 *dU) {
  int c[4];
  c[0] = s % g.L[0];
  int rem = s / g.L[0];
  c[1] = rem % g.L[1];
  rem /= g.L[1];
  c[2] = rem % g.L[2];
  c[3] = rem / g.L[2];
  const double sgn = (MU == 3 && c[3] == g.L[3] - 1) ? -1.0 : 1.0;
  c[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
  const int sn = site_of(g, c);
  double2 X[3][3], Y[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) X[i][j] = Y[i][j] = make_double2(0.0, 0.0);
  const size_t stride = (size_t)g.V * 12;
  const double2 *yx = y + (size_t)s * 12, *yn = y + (size_t)sn * 12;
  const double2 *px = phi + (size_t)s * 12, *pn = phi + (size_t)sn * 12;
  for (int r = 0; r < nrhs; ++r) {
    double2 a[6], b[6];
    half_proj<MU, -1, -1>(yx + r * stride, a);
    half_proj<MU, -1, 1>(pn + r * stride, b);
    outer_acc2(a, b, X);
    half_proj<MU, 1, -1>(yn + r * stride, a);
    half_proj<MU, 1, 1>(px + r * stride, b);
    outer_acc2(a, b, Y);
  }
  const double2 *u = U + ((size_t)s * 4 + MU) * 9;
  double2 *o = dU ? dU + ((size_t)s * 4 + MU) * 9 : nullptr;
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // chi^+ H phi link terms: U_ij X_ij + conj(U_ji) Y_ij
      double2 uij = u[i * 3 + j], uji = u[j * 3 + i];
      acc += cmul(uij, X[i][j]).x + cmulc(uji, Y[i][j]).x;
      if (o) {
        double2 gx = make_double2(X[i][j].x, -X[i][j].y);  // conj(X_ij) + Y_ji
        double2 gy = Y[j][i];
        double f = weight * kappa * sgn;
        o[i * 3 + j] = cadd(o[i * 3 + j], make_double2(f * (gx.x + gy.x), f * (gx.y + gy.y)));
      }
    }
  return weight * sgn * acc;
}

// One thread per link: blocks 4 k .. 4 k + 3 hold directions 0..3 of the same
// FORCE_SITES sites, so the four read the same x-site spinors close in time;
// fixed-order block sums of d loss / d kappa.
constexpr int FORCE_SITES = 128;
__global__ void __launch_bounds__(FORCE_SITES) k_force(Geom g, const double2 *__restrict__ U,
                                                       const double2 *__restrict__ y,
                                                       const double2 *__restrict__ phi, int nrhs, double kappa,
                                                       double weight, double2 *dU, double *dk_part) {
  const int mu = blockIdx.x & 3;
  const int s = (blockIdx.x >> 2) * FORCE_SITES + threadIdx.x;
  double dk = 0.0;
  if (s < g.V) {
    switch (mu) {
      case 0: dk = force_link<0>(g, s, U, y, phi, nrhs, kappa, weight, dU); break;
      case 1: dk = force_link<1>(g, s, U, y, phi, nrhs, kappa, weight, dU); break;
      case 2: dk = force_link<2>(g, s, U, y, phi, nrhs, kappa, weight, dU); break;
      default: dk = force_link<3>(g, s, U, y, phi, nrhs, kappa, weight, dU); break;
    }
  }
  __shared__ double sh[FORCE_SITES];
  sh[threadIdx.x] = dk;
  __syncthreads();
  for (int w = FORCE_SITES / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) dk_part[blockIdx.x] = sh[0];
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_gradient(lqcd_ctx *ctx, const double *src, const double *sol, int nrhs, const double *coef,
                             double weight, const lqcd_solver_params *params, double *dkappa, double *dU,
                             lqcd_solve_stats *stats, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_gradient");
  if (!ctx || !params || nrhs < 0 || !coef || (nrhs > 0 && (!src || !sol || !stats)))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_gradient: bad argument");
  if (!ctx->have_gauge) return set_error(ctx, LQCD_ERR_NO_GAUGE, "lqcd_gradient: no gauge field");
  if (nrhs == 0) return LQCD_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Geom &g = ctx->geom;
  const int lt = g.L[3];
  const size_t field = (size_t)nrhs * g.V * 12;
  if (dU && !is_device_ptr(dU)) return set_error(ctx, LQCD_ERR_INVALID, "lqcd_gradient: dU must be device memory");
  if (!is_device_ptr(src) || !is_device_ptr(sol))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_gradient: src and sol must be device memory");
  int rc = LQCD_OK;
  const int nblk = 4 * ((g.V + FORCE_SITES - 1) / FORCE_SITES);
  Carver sizing(nullptr);
  sizing.take<double2>(field);
  sizing.take<double2>(field);
  sizing.take<double2>((size_t)lt * 6);
  sizing.take<double>(nblk);
  void *w = workspace(ctx, WS_GRAD, sizing.size(), &rc);
  if (!w) return rc;
  Carver cv(w);
  double2 *eta = cv.take<double2>(field);
  double2 *y = cv.take<double2>(field);
  double2 *dcoef = cv.take<double2>((size_t)lt * 6);
  double *dk_part = cv.take<double>(nblk);
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(dcoef, coef, (size_t)lt * 6 * sizeof(double2), cudaMemcpyHostToDevice, st));
  size_t n = (size_t)nrhs * g.V;
  KL k_adj_source<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, (const double2 *)src, dcoef, eta, nrhs);
  LQCD_LAUNCH_CHECK(ctx, "k_adj_source");
  // adjoint solves D y = eta (the same solver as the forward solves)
  int src_rc = params->precision == LQCD_PREC_FP64 ? fp64_solve(ctx, eta, y, nrhs, *params, stats, st)
                                                   : mixed_solve(ctx, eta, y, nrhs, *params, stats, st);
  if (src_rc == LQCD_ERR_CUDA || src_rc == LQCD_ERR_OOM || src_rc == LQCD_ERR_INVALID) return src_rc;
  KL k_force<<<nblk, FORCE_SITES, 0, st>>>(g, ctx->U64, y, (const double2 *)sol, nrhs, ctx->kappa, weight,
                                           (double2 *)dU, dk_part);
  LQCD_LAUNCH_CHECK(ctx, "k_force");
  std::vector<double> h(nblk);
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), dk_part, nblk * sizeof(double), cudaMemcpyDeviceToHost, st));
  LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  double tot = 0.0;
  for (double v : h) tot += v;
  if (dkappa) *dkappa += tot;
  return src_rc;
}
