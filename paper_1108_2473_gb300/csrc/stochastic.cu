// Stochastic loops with dilution and the truncated solver method, driven on
// the host through the library's own entry points (Sec. II: complex Z2 noise,
// dilution, TSM; Eq. loop stochastic).  Everything numerical runs in the
// noise, solver and contraction kernels; this file only schedules them.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

using namespace lqcd;

namespace {

int n_pieces(const int dims[4], int dilution) { return dilution_pieces(dims, dilution); }

void merge(lqcd_solve_stats &acc, const lqcd_solve_stats &s) {
  acc.iterations = std::max(acc.iterations, s.iterations);
  acc.true_rel_residual = std::max(acc.true_rel_residual, s.true_rel_residual);
  acc.reliable_updates = std::max(acc.reliable_updates, s.reliable_updates);
  acc.restarts = std::max(acc.restarts, s.restarts);
  if (acc.status == LQCD_OK) acc.status = s.status;
}

}  // namespace

extern "C" int lqcd_loops_stochastic(lqcd_ctx *ctx, const lqcd_stochastic_params *sp,
                                     const lqcd_solver_params *solver, double *per_site, double *per_t,
                                     lqcd_solve_stats *summary, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_loops_stochastic");
  if (!ctx || !sp || !solver) return set_error(ctx, LQCD_ERR_INVALID, "lqcd_loops_stochastic: null argument");
  const int np = n_pieces(ctx->dims, sp->dilution);
  if (np < 0) return set_error(ctx, LQCD_ERR_INVALID, "lqcd_loops_stochastic: unknown dilution %d", sp->dilution);
  if (sp->n_lp < 1 || sp->n_hp < 0 || !(sp->tol_lp > 0) || (sp->n_hp > 0 && !(sp->tol_hp > 0)))
    return set_error(ctx, LQCD_ERR_INVALID, "lqcd_loops_stochastic: need n_lp >= 1, n_hp >= 0, tolerances > 0");
  if (!ctx->have_gauge) return set_error(ctx, LQCD_ERR_NO_GAUGE, "lqcd_loops_stochastic: no gauge field");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const Geom &g = ctx->geom;
  int chunk = sp->chunk > 0 ? sp->chunk : std::min(np, 384);
  chunk = std::min(chunk, np);
  const size_t field = (size_t)g.V * 12;
  // per_t may be host memory: accumulate on the device, copy once at the end
  const bool host_pt = per_t && !is_device_ptr(per_t);
  int rc = LQCD_OK;
  Carver sizing(nullptr);
  sizing.take<double2>((size_t)chunk * field);
  sizing.take<double2>((size_t)chunk * field);
  sizing.take<double2>((size_t)chunk * field);
  sizing.take<double2>((size_t)g.L[3] * 6);
  void *w = workspace(ctx, WS_STAGE_IN, sizing.size(), &rc);
  if (!w) return rc;
  Carver cv(w);
  double2 *src = cv.take<double2>((size_t)chunk * field);
  double2 *x_lo = cv.take<double2>((size_t)chunk * field);
  double2 *x_hi = cv.take<double2>((size_t)chunk * field);
  double2 *dpt = cv.take<double2>((size_t)g.L[3] * 6);
  double *pt = per_t;
  if (host_pt) {
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(dpt, per_t, (size_t)g.L[3] * 6 * sizeof(double2), cudaMemcpyHostToDevice, st));
    pt = (double *)dpt;
  }
  lqcd_solve_stats sum[2];
  for (auto &s : sum) s = lqcd_solve_stats{0, LQCD_OK, 0.0, 0, 0};
  std::vector<lqcd_solve_stats> stats(chunk);
  lqcd_solver_params p_lo = *solver, p_hi = *solver;
  p_lo.tol = sp->tol_lp;
  p_hi.tol = sp->tol_hp;
  int worst = LQCD_OK;
  auto note = [&](int which, int n) {
    for (int k = 0; k < n; ++k) {
      merge(sum[which], stats[k]);
      if (worst == LQCD_OK && stats[k].status != LQCD_OK) worst = stats[k].status;
    }
  };
  // low-precision (or plain) set
  const double w_lp = 1.0 / sp->n_lp;
  for (int r = 0; r < sp->n_lp; ++r) {
    for (int d0 = 0; d0 < np; d0 += chunk) {
      const int nd = std::min(chunk, np - d0);
      rc = lqcd_noise_generate(sp->seed, LQCD_STREAM_LP, sp->first_noise + r, ctx->dims, sp->dilution, d0, nd,
                               (double *)src, stream);
      if (rc) return set_error(ctx, rc, "lqcd_loops_stochastic: %s", lqcd_last_error(nullptr));
      rc = lqcd_solve_batch(ctx, (const double *)src, (double *)x_lo, nd, &p_lo, stats.data(), stream);
      if (rc == LQCD_ERR_INVALID || rc == LQCD_ERR_CUDA || rc == LQCD_ERR_OOM) return rc;
      note(0, nd);
      rc = lqcd_loops_batch(ctx, (const double *)src, (const double *)x_lo, nd, w_lp, per_site, pt, stream);
      if (rc) return rc;
    }
  }
  // high-precision correction set: the same truncated solver, then the precise one
  if (sp->n_hp > 0) {
    const double w_hp = 1.0 / sp->n_hp;
    for (int r = 0; r < sp->n_hp; ++r) {
      for (int d0 = 0; d0 < np; d0 += chunk) {
        const int nd = std::min(chunk, np - d0);
        rc = lqcd_noise_generate(sp->seed, LQCD_STREAM_HP, sp->first_noise + r, ctx->dims, sp->dilution, d0, nd,
                                 (double *)src, stream);
        if (rc) return set_error(ctx, rc, "lqcd_loops_stochastic: %s", lqcd_last_error(nullptr));
        rc = lqcd_solve_batch(ctx, (const double *)src, (double *)x_lo, nd, &p_lo, stats.data(), stream);
        if (rc == LQCD_ERR_INVALID || rc == LQCD_ERR_CUDA || rc == LQCD_ERR_OOM) return rc;
        note(0, nd);
        rc = lqcd_solve_batch(ctx, (const double *)src, (double *)x_hi, nd, &p_hi, stats.data(), stream);
        if (rc == LQCD_ERR_INVALID || rc == LQCD_ERR_CUDA || rc == LQCD_ERR_OOM) return rc;
        note(1, nd);
        rc = lqcd_loops_batch(ctx, (const double *)src, (const double *)x_hi, nd, w_hp, per_site, pt, stream);
        if (rc) return rc;
        rc = lqcd_loops_batch(ctx, (const double *)src, (const double *)x_lo, nd, -w_hp, per_site, pt, stream);
        if (rc) return rc;
      }
    }
  }
  if (host_pt)
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(per_t, dpt, (size_t)g.L[3] * 6 * sizeof(double2), cudaMemcpyDeviceToHost, st));
  LQCD_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (summary) {
    summary[0] = sum[0];
    summary[1] = sum[1];
  }
  if (worst != LQCD_OK) return set_error(ctx, worst, "lqcd_loops_stochastic: some solves did not converge");
  return LQCD_OK;
}
