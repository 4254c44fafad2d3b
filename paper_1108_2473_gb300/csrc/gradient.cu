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

// (1 + S gamma_mu) psi for a full spinor (DeGrand-Rossi), S = +-1
template <int MU, int S>
__device__ __forceinline__ void proj_full(const double2 p[12], double2 q[12]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double2 p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    double2 g0, g1, g2, g3;  // gamma_mu psi
    if (MU == 0) {
      g0 = cmuli(p3); g1 = cmuli(p2);
      g2 = cscale(cmuli(p1), -1.0); g3 = cscale(cmuli(p0), -1.0);
    } else if (MU == 1) {
      g0 = cscale(p3, -1.0); g1 = p2; g2 = p1; g3 = cscale(p0, -1.0);
    } else if (MU == 2) {
      g0 = cmuli(p2); g1 = cscale(cmuli(p3), -1.0);
      g2 = cscale(cmuli(p0), -1.0); g3 = cmuli(p1);
    } else {
      g0 = p2; g1 = p3; g2 = p0; g3 = p1;
    }
    q[c] = S > 0 ? cadd(p0, g0) : csub(p0, g0);
    q[3 + c] = S > 0 ? cadd(p1, g1) : csub(p1, g1);
    q[6 + c] = S > 0 ? cadd(p2, g2) : csub(p2, g2);
    q[9 + c] = S > 0 ? cadd(p3, g3) : csub(p3, g3);
  }
}

// out_ij += sum_a conj(a_ai) b_aj  (spin-summed colour outer product)
__device__ __forceinline__ void outer_acc(const double2 a[12], const double2 b[12], double2 out[3][3]) {
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) out[i][j] = cadd(out[i][j], cmulc(a[sp * 3 + i], b[sp * 3 + j]));
}

__device__ __forceinline__ void load_chi(const double2 *y, double2 v[12]) {  // chi = gamma5 y
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 q = y[k];
    v[k] = k >= 6 ? make_double2(-q.x, -q.y) : q;
  }
}

template <int MU>
__device__ __forceinline__ void force_link(const Geom &g, int s, const int c[4], const double2 *__restrict__ U,
                                           const double2 *__restrict__ y, const double2 *__restrict__ phi, int nrhs,
                                           double kappa, double weight, double2 *dU, double &dk) {
  int cn[4] = {c[0], c[1], c[2], c[3]};
  cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
  const int sn = site_of(g, cn);
  const double sgn = (MU == 3 && c[3] == g.L[3] - 1) ? -1.0 : 1.0;
  double2 X[3][3], Y[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) X[i][j] = Y[i][j] = make_double2(0.0, 0.0);
  const size_t stride = (size_t)g.V * 12;
  for (int r = 0; r < nrhs; ++r) {
    double2 chx[12], chn[12], pn[12], px[12], q[12];
    load_chi(y + r * stride + (size_t)s * 12, chx);
    load_chi(y + r * stride + (size_t)sn * 12, chn);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      pn[k] = phi[r * stride + (size_t)sn * 12 + k];
      px[k] = phi[r * stride + (size_t)s * 12 + k];
    }
    // X += chi(x)^+ (1 - gamma_mu) phi(x+mu);  Y += chi(x+mu)^+ (1 + gamma_mu) phi(x)
    proj_full<MU, -1>(pn, q);
    outer_acc(chx, q, X);
    proj_full<MU, +1>(px, q);
    outer_acc(chn, q, Y);
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
  dk += weight * sgn * acc;
}

// one thread per site, all four links; fixed-order block sums of d loss / d kappa
__global__ void __launch_bounds__(128) k_force(Geom g, const double2 *__restrict__ U, const double2 *__restrict__ y,
                                               const double2 *__restrict__ phi, int nrhs, double kappa, double weight,
                                               double2 *dU, double *dk_part) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double dk = 0.0;
  if (s < g.V) {
    int c[4];
    c[0] = s % g.L[0];
    int r = s / g.L[0];
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
    force_link<0>(g, s, c, U, y, phi, nrhs, kappa, weight, dU, dk);
    force_link<1>(g, s, c, U, y, phi, nrhs, kappa, weight, dU, dk);
    force_link<2>(g, s, c, U, y, phi, nrhs, kappa, weight, dU, dk);
    force_link<3>(g, s, c, U, y, phi, nrhs, kappa, weight, dU, dk);
  }
  __shared__ double sh[128];
  sh[threadIdx.x] = dk;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
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
  const int nblk = (g.V + 127) / 128;
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
  KL k_force<<<nblk, 128, 0, st>>>(g, ctx->U64, y, (const double2 *)sol, nrhs, ctx->kappa, weight, (double2 *)dU,
                                   dk_part);
  LQCD_LAUNCH_CHECK(ctx, "k_force");
  std::vector<double> h(nblk);
  LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), dk_part, nblk * sizeof(double), cudaMemcpyDeviceToHost, st));
  LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  double tot = 0.0;
  for (double v : h) tot += v;
  if (dkappa) *dkappa += tot;
  return src_rc;
}
