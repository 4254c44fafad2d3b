// Gaussian quark smearing and APE link smearing (Sec. III, smearing of the
// interpolating fields), FP64.  These act on the sources of connected
// correlators; the loops themselves are computed without smearing.
//
// Gaussian:  F = (1 + alpha H)^n within each time slice,
//   (H q)(x) = sum_{i = x, y, z} [ U_i(x) q(x + i) + U_i(x - i)^+ q(x - i) ],
// colour only (all four spins alike), optionally divided by (1 + 6 alpha) per step.
// APE:  U_i'(x) = P[ U_i(x) + alpha sum_{j != i spatial} S_ij(x) ] with the four
// spatial staples S_ij; P = unitary polar factor (scaled Newton iteration,
// Higham) divided by the principal cube root of its determinant; temporal links
// are copied unchanged.
#include <cmath>

#include "internal.cuh"

namespace lqcd {

struct M3 {
  double2 m[3][3];
};

__device__ __forceinline__ M3 load_m3(const double2 *p) {
  M3 r;
#pragma unroll
  for (int k = 0; k < 9; ++k) r.m[k / 3][k % 3] = p[k];
  return r;
}
__device__ __forceinline__ void store_m3(double2 *p, const M3 &a) {
#pragma unroll
  for (int k = 0; k < 9; ++k) p[k] = a.m[k / 3][k % 3];
}
// a b, a^+ b, a b^+
template <bool DA, bool DB>
__device__ __forceinline__ M3 mm(const M3 &a, const M3 &b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 x = DA ? make_double2(a.m[k][i].x, -a.m[k][i].y) : a.m[i][k];
        const double2 y = DB ? make_double2(b.m[j][k].x, -b.m[j][k].y) : b.m[k][j];
        acc = cadd(acc, cmul(x, y));
      }
      r.m[i][j] = acc;
    }
  return r;
}
__device__ __forceinline__ double2 det3(const M3 &a) {
  const double2 c0 = csub(cmul(a.m[1][1], a.m[2][2]), cmul(a.m[1][2], a.m[2][1]));
  const double2 c1 = csub(cmul(a.m[1][2], a.m[2][0]), cmul(a.m[1][0], a.m[2][2]));
  const double2 c2 = csub(cmul(a.m[1][0], a.m[2][1]), cmul(a.m[1][1], a.m[2][0]));
  return cadd(cadd(cmul(a.m[0][0], c0), cmul(a.m[0][1], c1)), cmul(a.m[0][2], c2));
}
// (a^{-1})^+ = conj(cofactor matrix) / conj(det)
__device__ __forceinline__ M3 inv_dag(const M3 &a, double2 det) {
  M3 cof;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      cof.m[i][j] = csub(cmul(a.m[i1][j1], a.m[i2][j2]), cmul(a.m[i1][j2], a.m[i2][j1]));
    }
  // a^{-1} = cof^T / det, so (a^{-1})^+ = conj(cof) / conj(det)
  const double n = det.x * det.x + det.y * det.y;
  const double2 inv_cdet = make_double2(det.x / n, det.y / n);  // 1 / conj(det)
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.m[i][j] = cmul(make_double2(cof.m[i][j].x, -cof.m[i][j].y), inv_cdet);
  return r;
}

// projection onto SU(3): unitary polar factor by the Newton iteration
// X <- (z X + X^{-+} / z) / 2 with z = |det X|^{-1/3}, then the det phase removed
__device__ M3 project_su3(M3 x) {
  for (int it = 0; it < 30; ++it) {
    const double2 d = det3(x);
    const double ad = sqrt(d.x * d.x + d.y * d.y);
    const double z = ad > 0.0 ? cbrt(1.0 / ad) : 1.0;
    const M3 y = inv_dag(x, d);
    double diff = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double2 nv = make_double2(0.5 * (z * x.m[i][j].x + y.m[i][j].x / z),
                                        0.5 * (z * x.m[i][j].y + y.m[i][j].y / z));
        diff = fmax(diff, fabs(nv.x - x.m[i][j].x) + fabs(nv.y - x.m[i][j].y));
        x.m[i][j] = nv;
      }
    if (diff < 1e-15 && it > 2) break;
  }
  const double2 d = det3(x);
  const double phi = atan2(d.y, d.x) / 3.0;
  double sn, cs;
  sincos(phi, &sn, &cs);
  const double2 ph = make_double2(cs, -sn);  // e^{-i phi / 3}
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) x.m[i][j] = cmul(x.m[i][j], ph);
  return x;
}

__device__ __forceinline__ int shift_site(const Geom &g, const int c[4], int mu, int step) {
  int cn[4] = {c[0], c[1], c[2], c[3]};
  cn[mu] = (c[mu] + step + g.L[mu]) % g.L[mu];
  return site_of(g, cn);
}
__device__ __forceinline__ void coords_full(const Geom &g, int s, int c[4]) {
  c[0] = s % g.L[0];
  int r = s / g.L[0];
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
}

// one APE step: thread per (site, mu); spatial links smeared, temporal copied
__global__ void k_ape_step(Geom g, const double2 *__restrict__ Uin, double2 *Uout, double alpha) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.V * 4) return;
  const int s = idx >> 2, i = idx & 3;
  const double2 *ui = Uin + (size_t)idx * 9;
  if (i == 3) {
#pragma unroll
    for (int k = 0; k < 9; ++k) Uout[(size_t)idx * 9 + k] = ui[k];
    return;
  }
  int c[4];
  coords_full(g, s, c);
  const M3 U = load_m3(ui);
  M3 S;
#pragma unroll
  for (int k = 0; k < 9; ++k) S.m[k / 3][k % 3] = make_double2(0.0, 0.0);
  for (int j = 0; j < 3; ++j) {
    if (j == i) continue;
    const int s_j = shift_site(g, c, j, 1), s_i = shift_site(g, c, i, 1), s_mj = shift_site(g, c, j, -1);
    int cmj[4] = {c[0], c[1], c[2], c[3]};
    cmj[j] = (c[j] - 1 + g.L[j]) % g.L[j];
    const int s_mj_i = shift_site(g, cmj, i, 1);
    const M3 Uj = load_m3(Uin + ((size_t)s * 4 + j) * 9);
    const M3 Ui_j = load_m3(Uin + ((size_t)s_j * 4 + i) * 9);
    const M3 Uj_i = load_m3(Uin + ((size_t)s_i * 4 + j) * 9);
    const M3 up = mm<false, true>(mm<false, false>(Uj, Ui_j), Uj_i);  // U_j(x) U_i(x+j) U_j(x+i)^+
    const M3 Uj_mj = load_m3(Uin + ((size_t)s_mj * 4 + j) * 9);
    const M3 Ui_mj = load_m3(Uin + ((size_t)s_mj * 4 + i) * 9);
    const M3 Uj_mji = load_m3(Uin + ((size_t)s_mj_i * 4 + j) * 9);
    const M3 dn = mm<false, false>(mm<true, false>(Uj_mj, Ui_mj), Uj_mji);  // U_j(x-j)^+ U_i(x-j) U_j(x-j+i)
#pragma unroll
    for (int k = 0; k < 9; ++k) S.m[k / 3][k % 3] = cadd(S.m[k / 3][k % 3], cadd(up.m[k / 3][k % 3], dn.m[k / 3][k % 3]));
  }
  M3 V;
#pragma unroll
  for (int k = 0; k < 9; ++k) V.m[k / 3][k % 3] = cadd(U.m[k / 3][k % 3], cscale(S.m[k / 3][k % 3], alpha));
  store_m3(Uout + (size_t)idx * 9, project_su3(V));
}

// one Gaussian step: out = scale * (in + alpha H in); thread per (rhs, site)
__global__ void k_gauss_step(Geom g, const double2 *__restrict__ U, const double2 *__restrict__ in, double2 *out,
                             int nrhs, double alpha, double scale) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nrhs * g.V) return;
  const int s = (int)(idx % g.V);
  const size_t base = idx - s;  // rhs * V
  int c[4];
  coords_full(g, s, c);
  double2 acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = make_double2(0.0, 0.0);
  for (int i = 0; i < 3; ++i) {
    const int sf = shift_site(g, c, i, 1), sb = shift_site(g, c, i, -1);
    const double2 *uf = U + ((size_t)s * 4 + i) * 9;   // U_i(x)
    const double2 *ub = U + ((size_t)sb * 4 + i) * 9;  // U_i(x - i)
    const double2 *qf = in + (base + sf) * 12, *qb = in + (base + sb) * 12;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double2 t = acc[sp * 3 + a];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          t = cadd(t, cmul(uf[a * 3 + b], qf[sp * 3 + b]));   // U_i(x)[a][b] q(x+i)
          t = cadd(t, cmulc(ub[b * 3 + a], qb[sp * 3 + b]));  // conj(U_i(x-i)[b][a]) q(x-i)
        }
        acc[sp * 3 + a] = t;
      }
  }
  const double2 *q = in + idx * 12;
  double2 *o = out + idx * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) o[k] = cscale(cadd(q[k], cscale(acc[k], alpha)), scale);
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_smear_ape(lqcd_ctx *ctx, double alpha, int n_iter, double *out, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_smear_ape");
  if (!ctx || n_iter < 0 || !std::isfinite(alpha)) return set_error(ctx, LQCD_ERR_INVALID, "lqcd_smear_ape: bad argument");
  if (!ctx->have_gauge) return set_error(ctx, LQCD_ERR_NO_GAUGE, "lqcd_smear_ape: no gauge field");
  if (out && !is_device_ptr(out)) return set_error(ctx, LQCD_ERR_INVALID, "lqcd_smear_ape: out must be device memory");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Geom &g = ctx->geom;
  const size_t n = (size_t)g.V * 36;
  if (!ctx->Uape) LQCD_CUDA_TRY(ctx, cudaMalloc(&ctx->Uape, n * sizeof(double2)));
  int rc = LQCD_OK;
  double2 *tmp = (double2 *)workspace(ctx, WS_SMEAR_LINKS, n * sizeof(double2), &rc);
  if (!tmp) return rc;
  // ping-pong so that the last step lands in Uape
  double2 *bufs[2] = {n_iter % 2 ? ctx->Uape : tmp, n_iter % 2 ? tmp : ctx->Uape};
  const double2 *src = ctx->U64;
  const int threads = 128, blocks = (g.V * 4 + threads - 1) / threads;
  for (int it = 0; it < n_iter; ++it) {
    double2 *dst = bufs[it % 2];
    KL k_ape_step<<<blocks, threads, 0, st>>>(g, src, dst, alpha);
    LQCD_LAUNCH_CHECK(ctx, "k_ape_step");
    src = dst;
  }
  if (n_iter == 0)
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->Uape, ctx->U64, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  if (out) LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->Uape, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  ctx->have_ape = true;
  return LQCD_OK;
}

extern "C" int lqcd_smear_gaussian(lqcd_ctx *ctx, const double *in, double *out, int nrhs, double alpha, int n_iter,
                                   int ape_links, int normalise, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_smear_gaussian");
  if (!ctx || nrhs < 0 || n_iter < 0 || !std::isfinite(alpha) || (nrhs > 0 && (!in || !out)) || (in && in == out))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_smear_gaussian: bad argument (in and out must differ)");
  if (!ctx->have_gauge) return set_error(ctx, LQCD_ERR_NO_GAUGE, "lqcd_smear_gaussian: no gauge field");
  if (ape_links && !ctx->have_ape)
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_smear_gaussian: no APE-smeared links (call lqcd_smear_ape)");
  if (nrhs == 0) return LQCD_OK;
  if (!is_device_ptr(in) || !is_device_ptr(out))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_smear_gaussian: in and out must be device memory");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Geom &g = ctx->geom;
  const size_t n = (size_t)nrhs * g.V * 12;
  if (n_iter == 0) {
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(out, in, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    return LQCD_OK;
  }
  int rc = LQCD_OK;
  double2 *tmp = (double2 *)workspace(ctx, WS_SMEAR, n * sizeof(double2), &rc);
  if (!tmp) return rc;
  const double2 *U = ape_links ? ctx->Uape : ctx->U64;
  const double scale = normalise ? 1.0 / (1.0 + 6.0 * alpha) : 1.0;
  double2 *bufs[2] = {n_iter % 2 ? (double2 *)out : tmp, n_iter % 2 ? tmp : (double2 *)out};
  const double2 *src = (const double2 *)in;
  const int threads = 128;
  const unsigned blocks = (unsigned)((nrhs * (size_t)g.V + threads - 1) / threads);
  for (int it = 0; it < n_iter; ++it) {
    double2 *dst = bufs[it % 2];
    KL k_gauss_step<<<blocks, threads, 0, st>>>(g, U, src, dst, nrhs, alpha, scale);
    LQCD_LAUNCH_CHECK(ctx, "k_gauss_step");
    src = dst;
  }
  return LQCD_OK;
}
