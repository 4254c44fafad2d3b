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
  // pieces per batched solve; vectors with fewer pieces than a chunk are
  // grouped, several per solve (undiluted TSM vectors would otherwise be
  // solved one right-hand side at a time)
  const int chunk_req = sp->chunk > 0 ? sp->chunk : 384;
  const int chunk = std::min(chunk_req, np);
  const int vec_per_batch = std::max(1, chunk_req / np);
  const size_t field = (size_t)g.V * 12;
  // per_t may be host memory: accumulate on the device, copy once at the end
  const bool host_pt = per_t && !is_device_ptr(per_t);
  int rc = LQCD_OK;
  const size_t slots = (size_t)std::max(chunk, vec_per_batch * np);
  Carver sizing(nullptr);
  sizing.take<double2>(slots * field);
  sizing.take<double2>(slots * field);
  sizing.take<double2>(slots * field);
  sizing.take<double2>((size_t)g.L[3] * 6);
  void *w = workspace(ctx, WS_STAGE_IN, sizing.size(), &rc);
  if (!w) return rc;
  Carver cv(w);
  double2 *src = cv.take<double2>(slots * field);
  double2 *x_lo = cv.take<double2>(slots * field);
  double2 *x_hi = cv.take<double2>(slots * field);
  double2 *dpt = cv.take<double2>((size_t)g.L[3] * 6);
  double *pt = per_t;
  if (host_pt) {
    LQCD_CUDA_TRY(ctx, cudaMemcpyAsync(dpt, per_t, (size_t)g.L[3] * 6 * sizeof(double2), cudaMemcpyHostToDevice, st));
    pt = (double *)dpt;
  }
  lqcd_solve_stats sum[2];
  for (auto &s : sum) s = lqcd_solve_stats{0, LQCD_OK, 0.0, 0, 0};
  std::vector<lqcd_solve_stats> stats(slots);
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
  // a work unit: pieces d0 .. d0 + nd - 1 of each of the vectors r0 .. r0 + nv - 1
  auto generate = [&](uint64_t stream_tag, int r0, int nv, int d0, int nd) {
    for (int v = 0; v < nv; ++v) {
      int e = lqcd_noise_generate(sp->seed, stream_tag, sp->first_noise + r0 + v, ctx->dims, sp->dilution, d0, nd,
                                  (double *)(src + (size_t)v * nd * field), stream);
      if (e) return e;
    }
    return (int)LQCD_OK;
  };
  for (int r = 0; r < sp->n_lp;) {
    const int nv = np <= chunk_req ? std::min(vec_per_batch, sp->n_lp - r) : 1;
    for (int d0 = 0; d0 < np; d0 += chunk) {
      const int nd = std::min(chunk, np - d0), n = nv * nd;
      rc = generate(LQCD_STREAM_LP, r, nv, d0, nd);
      if (rc) return set_error(ctx, rc, "lqcd_loops_stochastic: %s", lqcd_last_error(nullptr));
      rc = lqcd_solve_batch(ctx, (const double *)src, (double *)x_lo, n, &p_lo, stats.data(), stream);
      if (rc == LQCD_ERR_INVALID || rc == LQCD_ERR_CUDA || rc == LQCD_ERR_OOM) return rc;
      note(0, n);
      rc = lqcd_loops_batch(ctx, (const double *)src, (const double *)x_lo, n, w_lp, per_site, pt, stream);
      if (rc) return rc;
    }
    r += nv;
  }
  // high-precision correction set: the same truncated solver, then the precise one
  if (sp->n_hp > 0) {
    const double w_hp = 1.0 / sp->n_hp;
    for (int r = 0; r < sp->n_hp;) {
      const int nv = np <= chunk_req ? std::min(vec_per_batch, sp->n_hp - r) : 1;
      for (int d0 = 0; d0 < np; d0 += chunk) {
        const int nd = std::min(chunk, np - d0), n = nv * nd;
        rc = generate(LQCD_STREAM_HP, r, nv, d0, nd);
        if (rc) return set_error(ctx, rc, "lqcd_loops_stochastic: %s", lqcd_last_error(nullptr));
        rc = lqcd_solve_batch(ctx, (const double *)src, (double *)x_lo, n, &p_lo, stats.data(), stream);
        if (rc == LQCD_ERR_INVALID || rc == LQCD_ERR_CUDA || rc == LQCD_ERR_OOM) return rc;
        note(0, n);
        rc = lqcd_solve_batch(ctx, (const double *)src, (double *)x_hi, n, &p_hi, stats.data(), stream);
        if (rc == LQCD_ERR_INVALID || rc == LQCD_ERR_CUDA || rc == LQCD_ERR_OOM) return rc;
        note(1, n);
        rc = lqcd_loops_batch(ctx, (const double *)src, (const double *)x_hi, n, w_hp, per_site, pt, stream);
        if (rc) return rc;
        rc = lqcd_loops_batch(ctx, (const double *)src, (const double *)x_lo, n, -w_hp, per_site, pt, stream);
        if (rc) return rc;
      }
      r += nv;
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
