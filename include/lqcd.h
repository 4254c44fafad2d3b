/*
 * lqcd.h -- C ABI of the GB300 disconnected-loop library.
 *
 * The library computes the hot path behind the exact and stochastic
 * evaluation of disconnected fermion loops L(x) = Tr[Gamma G(x;x)] of
 * arXiv:1108.2473 (Eq. loop, Eq. loop stochastic): many right-hand-side
 * solves of the Wilson-Dirac operator, complex Z2 noise sources with
 * dilution, the loop contraction, the truncated solver method, and gradients
 * of the loops by adjoint solves.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - dims = (Lx, Ly, Lz, Lt), all even, Lx >= 2.  V = Lx*Ly*Lz*Lt.
 *    Site index s = x + Lx*(y + Ly*(z + Lz*t)); parity (x+y+z+t) mod 2.
 *  - Wilson-Dirac operator (the operator M of the stopping rule in Sec. III):
 *      D psi(x) = psi(x) - kappa sum_mu [ (1-gamma_mu) U_mu(x) psi(x+mu)
 *                                       + (1+gamma_mu) U_mu(x-mu)^+ psi(x-mu) ]
 *    periodic in space, every hop across t = Lt-1 <-> 0 multiplied by -1.
 *    G = D^{-1}.  Gamma matrices: DeGrand-Rossi basis,
 *      g1 = [[0,0,0,i],[0,0,i,0],[0,-i,0,0],[-i,0,0,0]]
 *      g2 = [[0,0,0,-1],[0,0,1,0],[0,1,0,0],[-1,0,0,0]]
 *      g3 = [[0,0,i,0],[0,0,0,-i],[-i,0,0,0],[0,i,0,0]]
 *      g4 = [[0,0,1,0],[0,0,0,1],[1,0,0,0],[0,1,0,0]],  g5 = g1 g2 g3 g4 = diag(1,1,-1,-1).
 *  - Gauge field layout: [V][4 (mu = x,y,z,t)][3][3] complex128 (re, im
 *    interleaved), U[s][mu] is the link from s to s + mu.
 *  - Colour-spinor field layout: [nrhs][V][4 spin][3 colour] complex128.
 *  - Loop outputs: per site [V][6] and per time slice [Lt][6] complex128 with
 *    Gamma order (1, g5, g1, g2, g3, g4); per-time-slice loops are sums over
 *    the sites of the slice.
 *  - Array arguments are device pointers unless a call says otherwise; the
 *    caller owns them and the library never frees them.  Calls that accept
 *    host pointers say so; they stage through library-owned device memory and
 *    synchronise the stream before returning.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Calls that return host results synchronise that stream.
 *  - Every call returns an lqcd status (0 = LQCD_OK, < 0 = error);
 *    lqcd_last_error() describes the most recent error.  A context is not
 *    thread-safe: one host thread at a time per context.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lqcd_ctx lqcd_ctx;
typedef struct lqcd_batch lqcd_batch;
typedef struct CUstream_st *lqcd_stream_t; /* same type as cudaStream_t */

/* ---- status codes ------------------------------------------------------ */
#define LQCD_OK 0
#define LQCD_ERR_INVALID (-1)       /* bad argument (size, pointer, enum)          */
#define LQCD_ERR_CUDA (-2)          /* a CUDA runtime call failed                  */
#define LQCD_ERR_NOT_CONVERGED (-3) /* iteration cap reached above tolerance       */
#define LQCD_ERR_BREAKDOWN (-4)     /* Krylov breakdown persisted after restart    */
#define LQCD_ERR_NONFINITE (-5)     /* NaN / Inf in a source or a reduction        */
#define LQCD_ERR_TIMEOUT (-6)       /* wall-clock budget or a bounded wait expired */
#define LQCD_ERR_NO_GAUGE (-7)      /* operator used before lqcd_set_gauge         */
#define LQCD_ERR_NOT_SU3 (-8)       /* a link is not in SU(3) within 1e-12         */
#define LQCD_ERR_OOM (-9)           /* device allocation failed                    */

/* ---- enums ------------------------------------------------------------- */
#define LQCD_PREC_FP64 0        /* FP64 storage and arithmetic throughout           */
#define LQCD_PREC_MIXED_FP16 1  /* FP16 (+ per-site FP32 norm) spinors, FP16 links,
                                   FP32 arithmetic, FP64 defect correction          */
#define LQCD_PREC_MIXED_BF16 2  /* BF16 spinors, FP16 links, otherwise as above     */

#define LQCD_SOLVER_BICGSTAB 0
#define LQCD_SOLVER_CG 1 /* CG on the normal equations of the Schur operator */

#define LQCD_DILUTE_NONE 0 /* one piece: the whole vector                         */
#define LQCD_DILUTE_T 1    /* Lt pieces, piece = t                                */
#define LQCD_DILUTE_TS 2   /* 4 Lt pieces, piece = 4 t + spin                     */
#define LQCD_DILUTE_TSC 3  /* 12 Lt pieces, piece = 12 t + 3 spin + colour        */
/* Spatial partitioning (Sec. II), OR-ed onto one of the schemes above (at most
 * one of the two): the base piece b splits into n_sp pieces b * n_sp + class.
 *   EO:   n_sp = 2, class = (x + y + z) mod 2 (even-odd in space)
 *   CUBE: n_sp = 8, class = (x mod 2) + 2 (y mod 2) + 4 (z mod 2) (one source
 *         per vertex of an elementary 3-cube, repeated over the lattice)      */
#define LQCD_DILUTE_EO 4
#define LQCD_DILUTE_CUBE 8

#define LQCD_STREAM_LP 0 /* noise stream of the plain / low-precision set      */
#define LQCD_STREAM_HP 1 /* noise stream of the TSM high-precision correction  */

/* ---- parameter and statistics records ---------------------------------- */
typedef struct {
  double tol;        /* target true relative residual |b - D x| / |b| (full lattice,
                        computed in FP64), the stopping rule of Sec. III             */
  int max_iter;      /* cap on Krylov iterations per RHS, summed over restarts      */
  int precision;     /* LQCD_PREC_*                                                 */
  int solver;        /* LQCD_SOLVER_*                                               */
  double delta;      /* mixed precision: reliable update when the iterated residual
                        drops below delta * its maximum since the last update;
                        <= 0 selects 0.05 (fastest on GB300 at 16^3x32)             */
  int rhs_block;     /* RHS solved together per launch; 0 = automatic (autotuned
                        for mixed precision, 1 for FP64 = the plain solver)         */
  double timeout_ms; /* wall-clock budget of the call; <= 0 = none                  */
} lqcd_solver_params;

typedef struct {
  int iterations;           /* Krylov iterations (all restarts / refinement cycles) */
  int status;               /* LQCD_OK or the per-RHS error code                    */
  double true_rel_residual; /* |b - D x| / |b| in FP64 on the full lattice          */
  int reliable_updates;     /* mixed precision: reliable updates performed          */
  int restarts;             /* outer restarts / defect-correction cycles            */
} lqcd_solve_stats;

/* ---- context ----------------------------------------------------------- */

/* Create a context for one lattice on CUDA device `device`.  dims: host
 * array of 4 ints.  Errors: LQCD_ERR_INVALID for odd or non-positive extents,
 * LQCD_ERR_CUDA if the device cannot be selected. */
int lqcd_create(lqcd_ctx **out, const int dims[4], int device);

/* Release the context and all library-owned device memory. */
int lqcd_destroy(lqcd_ctx *ctx);

/* Text of the most recent error on ctx (NULL: of the calling thread's last
 * context-free call).  Owned by the library; valid until the next call. */
const char *lqcd_last_error(const lqcd_ctx *ctx);

/* Upload and pack the gauge field (Sec. II: the configuration the loops are
 * computed on).  U: [V][4][3][3] complex128, device or host pointer.  Keeps an
 * FP64 copy and the reduced-precision copies the mixed-precision solver reads:
 * FP32 reconstruct-12 (first two rows; the third is (row1 x row2)^*), FP16 with
 * all 18 reals duplicated, tf32 and double-float.  Errors: LQCD_ERR_NOT_SU3 if
 * a link deviates from unitarity or unit determinant by more than 1e-12
 * (nothing is kept). */
int lqcd_set_gauge(lqcd_ctx *ctx, const double *U, lqcd_stream_t stream);

/* As lqcd_set_gauge but for arbitrary complex 3x3 links (no SU(3) check).
 * The operator D is defined for any links; only the FP64 path can use such a
 * field (the reduced-precision copies rely on reconstruct-12, valid for SU(3)
 * only), and mixed-precision solves then fail with LQCD_ERR_INVALID.  Exists so
 * that gradients can be checked entry by entry (finite differences leave
 * SU(3)); the paper has no counterpart. */
int lqcd_set_gauge_general(lqcd_ctx *ctx, const double *U, lqcd_stream_t stream);

/* Set the hopping parameter kappa of D (Sec. II: kappa = 0.157 for SESAM). */
int lqcd_set_kappa(lqcd_ctx *ctx, double kappa);

/* Average plaquette (1/(18V)) sum_{x,mu<nu} Re Tr U_mu U_nu U_mu^+ U_nu^+ of
 * the current gauge field; *plaq is a host double.  Synchronises stream. */
int lqcd_plaquette(lqcd_ctx *ctx, double *plaq, lqcd_stream_t stream);

/* out = D in (dagger = 0) or D^+ in (dagger != 0) in FP64 on the full lattice,
 * for nrhs fields [nrhs][V][4][3] complex128 (device).  in and out must not
 * overlap. */
int lqcd_apply_dirac(lqcd_ctx *ctx, const double *in, double *out, int nrhs, int dagger,
                     lqcd_stream_t stream);

/* Solve D x_i = b_i for nrhs right-hand sides (Sec. II: the inversions of the
 * all-to-all propagator; Sec. III: stopping rule |M x - b| / |b| < tol).
 * b, x: [nrhs][V][4][3] complex128, device or host (host: staged, and the
 * stream is synchronised).  Even-odd preconditioned BiCGstab (or CG), in FP64
 * or mixed precision with reliable updates and FP64 defect correction.
 * stats: host array of nrhs records, always filled.  Returns LQCD_OK only if
 * every RHS reached tol; otherwise the first error status among the RHS.
 * A zero b_i gives x_i = 0.  Synchronises stream. */
int lqcd_solve_batch(lqcd_ctx *ctx, const double *b, double *x, int nrhs,
                     const lqcd_solver_params *params, lqcd_solve_stats *stats,
                     lqcd_stream_t stream);

/* Uneven batch: several lattices (each its own context: dims, gauge field and
 * kappa) solved together (Sec. II: all inversions on the GPU; here several
 * configurations / kappas at once).  lqcd_batch_add registers b, x ([nrhs][V]
 * [4][3] complex128, device) of one context (one entry per context, all on one
 * device).  lqcd_batch_run solves every entry with *params: in mixed precision
 * the inner iterations of all lattices are captured into one CUDA graph (one
 * branch per lattice) on `stream`, which must be a created stream (not the
 * legacy default); one graph launch advances every lattice by four iterations,
 * and each lattice's outer FP64 refinement runs between launches.  FP64 solves
 * the entries one after another.  stats: host array of n_stats records, one
 * per RHS in the order of lqcd_batch_add; n_stats below the batch's RHS total
 * is rejected with LQCD_ERR_INVALID before any work (lqcd_batch_rhs gives the
 * total).  Returns LQCD_OK only if every RHS converged. */
int lqcd_batch_create(lqcd_batch **out);
int lqcd_batch_add(lqcd_batch *batch, lqcd_ctx *ctx, const double *b, double *x, int nrhs);
int lqcd_batch_run(lqcd_batch *batch, const lqcd_solver_params *params, lqcd_solve_stats *stats, int n_stats,
                   lqcd_stream_t stream);
/* Total right-hand sides registered in the batch (host int).  Host only. */
int lqcd_batch_rhs(const lqcd_batch *batch, int *total);
int lqcd_batch_destroy(lqcd_batch *batch);

/* Autotuner: for nrhs right-hand sides of `precision` on this context, time
 * complete inner iterations of the mixed solver (the four hopping-term launches
 * with their epilogues and the Krylov updates of the layout) for every
 * compiled variant -- the RHS-pair layout with its hop variants (register
 * budget, pairs per block, FP32-unit or mma.sync SU(3) products, full or
 * reconstruct-12 FP16 links (variant 7); for BF16 on
 * lattices with Lx Ly / 2 = 128 also the variant that stages a block's
 * neighbour planes in shared memory, variant 6) on launch grids of 2 to 256
 * blocks per SM (powers of two), and, for BF16, the 128-RHS tile layout with the
 * tensor-core (tcgen05) hop, variant 5 -- and keep the fastest for later
 * solves of that (nrhs, precision).  *best_blocks_per_sm and *best_hop_variant
 * (host, each may be NULL) receive the choice.  Needs a gauge field.
 * Synchronises the device.  With LQCD_AUTOTUNE_VERBOSE set in the environment
 * every timing is printed to stderr; LQCD_HOP_VARIANT=<digit> overrides the
 * variant the solves use (for tests and profiling); LQCD_NO_GRAPH makes the
 * solver launch its inner iterations directly instead of through CUDA graphs
 * (kernel profilers do not see kernels inside graphs with conditional nodes).
 * The timings assume every right-hand side active in every iteration; after
 * each BF16 mixed solve of nrhs right-hand sides the choice between the two
 * layouts is revised from the solve's per-RHS iteration counts, since a layout
 * keeps computing a pair or a tile until its slowest member has converged (each
 * layout's time per iteration is weighted by the mean over its groups of the
 * group's largest iteration count). */
int lqcd_autotune(lqcd_ctx *ctx, int nrhs, int precision, int *best_blocks_per_sm, int *best_hop_variant);
/* The launch choice later solves of (nrhs, precision) will use -- after the
 * autotuner, any revision by earlier solves and the LQCD_HOP_VARIANT override --
 * as for lqcd_autotune (host ints, each may be NULL; hop variant 5 is the tile
 * layout; an override to variant 6 where it does not apply reports variant 1,
 * the kernel then launched).  Host only; LQCD_ERR_INVALID for a null ctx. */
int lqcd_tuned_choice(const lqcd_ctx *ctx, int nrhs, int precision, int *blocks_per_sm, int *hop_variant);

/* Point sources e_{x,spin,colour} (Sec. II: exact all-to-all propagator from
 * one inversion per site, spin and colour).  sites: host array of n_sites
 * site indices; out: [12 n_sites][V][4][3] complex128 (device), source
 * 12 k + 3 spin + colour = e_{sites[k], spin, colour}. */
int lqcd_point_sources(lqcd_ctx *ctx, const int64_t *sites, int n_sites, double *out,
                       lqcd_stream_t stream);

/* Complex Z2 noise (Sec. II, Eq. delta functions) with dilution.
 * Generator: Philox4x64-10 (Salmon et al., SC'11), key = (seed, noise_stream),
 * counter = (site, noise_index, 0, 0); bits 2k, 2k+1 of output word 0 give the
 * signs of Re, Im of component k = 3 spin + colour; value (+-1 +- i)/sqrt(2).
 * Writes pieces first_piece .. first_piece + n_pieces - 1 of the dilution
 * scheme (LQCD_DILUTE_*) of noise vector noise_index: out [n_pieces][V][4][3]
 * complex128 (device), zero outside each piece.  Bit-exact with the CPU
 * definition.  dims: host array of 4 ints. */
int lqcd_noise_generate(uint64_t seed, uint64_t noise_stream, uint64_t noise_index,
                        const int dims[4], int dilution, int first_piece, int n_pieces,
                        double *out, lqcd_stream_t stream);

/* Number of pieces of dilution scheme `dilution` (LQCD_DILUTE_*, optionally
 * | LQCD_DILUTE_EO or | LQCD_DILUTE_CUBE) on a lattice dims (host, 4 ints);
 * -1 for an unknown scheme or bad dims.  Host only. */
int lqcd_dilution_pieces(const int dims[4], int dilution);

/* Loop contraction (Eq. loop stochastic; with point sources Eq. loop):
 *   per_site[x][g] += weight * sum_i src_i(x)^+ Gamma_g sol_i(x)
 *   per_t[t][g]    += weight * sum_{x in slice t} sum_i src_i(x)^+ Gamma_g sol_i(x)
 * src, sol: [nrhs][V][4][3] complex128 (device).  per_site (may be NULL):
 * [V][6] complex128 device; per_t (may be NULL): [Lt][6] complex128, device
 * or host (host: the stream is synchronised).  FP64 accumulation in a fixed
 * order (bit-reproducible). */
int lqcd_loops_batch(lqcd_ctx *ctx, const double *src, const double *sol, int nrhs,
                     double weight, double *per_site, double *per_t, lqcd_stream_t stream);

/* Momentum-projected loops (the sink phase of the disconnected correlator,
 * Sec. III, and of the current insertion of the three-point function):
 *   out[m][t][g] = sum_{x in slice t} e^{+i p_m . x} per_site[x][g],
 *   p_m = 2 pi (moms[m][0] / Lx, moms[m][1] / Ly, moms[m][2] / Lz)
 * per_site: [V][6] complex128 device (as lqcd_loops_batch writes it); moms:
 * host int [n_mom][3] (any integers); out: [n_mom][Lt][6] complex128 device
 * (overwritten).  The phase is evaluated from the exact integer numerator of
 * p.x / 2 pi modulo the spatial volume; FP64 sums in a fixed order. */
int lqcd_loops_momentum(lqcd_ctx *ctx, const double *per_site, int n_mom, const int *moms, double *out,
                        lqcd_stream_t stream);

/* Disconnected two-point function (Sec. III, Eq. for D_AB), averaged over the
 * source time t':
 *   D[t][A][B] = 1/(l3 Lt) * 1/n_pairs * sum_{(r, r')} sum_t' L^r_A(p, t + t') L^{r'}_B(-p, t')
 * loops_p, loops_mp: [n_vec][Lt][6] complex128 device -- loops of n_vec noise
 * vectors (or of one exact evaluation) at momenta p and -p (the same array for
 * p = 0).  unbiased = 1: the ordered pairs r != r' (n_pairs = n_vec (n_vec - 1),
 * needs n_vec >= 2), so that no noise vector meets itself; unbiased = 0: all
 * n_vec^2 pairs (for n_vec = 1 exact loops, the plain product).  l3: spatial
 * volume.  out: [Lt][6][6] complex128 device (overwritten).  No context needed. */
int lqcd_disconnected_correlator(const double *loops_p, const double *loops_mp, int n_vec, int lt, int l3,
                                 int unbiased, double *out, lqcd_stream_t stream);

/* APE smearing of the spatial links (Sec. III: the links entering the
 * smearing hopping matrix are APE-smeared; the paper gives neither formula nor
 * parameters).  n_iter steps of
 *   U_i'(x) = P[ U_i(x) + alpha sum_{j != i spatial} S_ij(x) ],
 *   S_ij(x) = U_j(x) U_i(x+j) U_j(x+i)^+ + U_j(x-j)^+ U_i(x-j) U_j(x-j+i),
 * on the context's gauge field, temporal links unchanged; P = unitary polar
 * factor divided by the principal cube root of its determinant (FP64).  The
 * result is kept in the context (for lqcd_smear_gaussian) until the next
 * lqcd_set_gauge, and copied to out ([V][4][3][3] complex128 device, may be
 * NULL).  Errors: INVALID (negative n_iter, non-finite alpha, host out),
 * NO_GAUGE. */
int lqcd_smear_ape(lqcd_ctx *ctx, double alpha, int n_iter, double *out, lqcd_stream_t stream);

/* Gaussian smearing of quark fields (Sec. III): out = F in with
 *   F = (1 + alpha H)^n_iter,  (H q)(x) = sum_{i = x,y,z} [ U_i(x) q(x+i) + U_i(x-i)^+ q(x-i) ]
 * within each time slice, all four spins alike (the paper uses alpha = 4,
 * n = 50).  ape_links = 1 uses the links of the last lqcd_smear_ape, 0 the
 * context's links; normalise = 1 divides each factor by (1 + 6 alpha).
 * in, out: [nrhs][V][4][3] complex128 device, distinct.  FP64.  Errors:
 * INVALID (in == out, host pointers, ape_links without lqcd_smear_ape),
 * NO_GAUGE. */
int lqcd_smear_gaussian(lqcd_ctx *ctx, const double *in, double *out, int nrhs, double alpha, int n_iter,
                        int ape_links, int normalise, lqcd_stream_t stream);

/* Stochastic loops with dilution and the truncated solver method (Sec. II,
 * Eq. loop stochastic; TSM after Bali, Collins, Schafer):
 *   L += (1/n_lp) sum_{r<n_lp} sum_d xi_{r,d}^+ Gamma phi^{LP}_{r,d}
 *      + (1/n_hp) sum_{r<n_hp} sum_d eta_{r,d}^+ Gamma (phi^{HP}_{r,d} - phi^{LP}_{r,d})
 * xi: noise vectors first_noise .. of stream LQCD_STREAM_LP, eta: vectors
 * first_noise .. of stream LQCD_STREAM_HP, each split into its dilution pieces
 * d; phi^{LP} solved to tol_lp, phi^{HP} to tol_hp (true FP64 residual), both
 * with the same solver settings, so phi^{LP} of a HP vector is exactly what the
 * LP solver gives it.  n_hp = 0 gives the plain diluted estimator at tol_lp. */
typedef struct {
  uint64_t seed;
  uint64_t first_noise;
  int dilution;   /* LQCD_DILUTE_*                                        */
  int n_lp;       /* vectors of the low-precision (or plain) set, >= 1     */
  int n_hp;       /* vectors of the high-precision correction set, >= 0   */
  double tol_lp;  /* relative residual of the LP (or plain) solves         */
  double tol_hp;  /* relative residual of the HP solves                    */
  int chunk;      /* right-hand sides per batched solve: the dilution pieces
                     of one vector, or whole vectors grouped when a vector
                     has fewer pieces (undiluted TSM); 0 = 384              */
} lqcd_stochastic_params;

/* Runs the estimator above end to end on the device (noise generation,
 * batched solves with *solver's precision / iteration cap / reliable-update
 * settings, contraction) and accumulates into per_site ([V][6] complex128,
 * device, may be NULL) and per_t ([Lt][6] complex128, device or host, may be
 * NULL).  summary (host, may be NULL): [0] the LP solves, [1] the HP solves --
 * largest iteration count and true residual, worst status.  Returns LQCD_OK
 * only if every solve converged.  Synchronises stream. */
int lqcd_loops_stochastic(lqcd_ctx *ctx, const lqcd_stochastic_params *sp, const lqcd_solver_params *solver,
                          double *per_site, double *per_t, lqcd_solve_stats *summary, lqcd_stream_t stream);

/* Gradient of a real loss of the per-time-slice loops by adjoint solves (the
 * paper computes no gradients; this is the derivative of its stochastic loop
 * estimator, Eq. loop stochastic, for fixed noise).
 *   src, sol: [nrhs][V][4][3] complex128 device -- the noise pieces xi_d and
 *             their forward solutions phi_d = D^{-1} xi_d (from lqcd_solve_batch).
 *   coef:     host [Lt][6] complex128, c[t][g] = d loss / d Re L_g(t)
 *             + i d loss / d Im L_g(t) for the loops L_g(t) = sum_{x in t}
 *             sum_d xi_d(x)^+ Gamma_g phi_d(x) (Gamma order 1, g5, g1..g4).
 * Solves D y_d = gamma5 M^+ xi_d with M(x) = sum_g conj(c[t(x)][g]) Gamma_g
 * (params as for lqcd_solve_batch; D^+ = gamma5 D gamma5 makes chi_d = gamma5 y_d
 * the adjoint solution), then accumulates
 *   *dkappa (host, may be NULL) += weight * Re sum_d chi_d^+ H phi_d   (= d loss / d kappa)
 *   dU (device [V][4][3][3] complex128, may be NULL) += weight * d loss / d U
 * in the convention d loss = Re sum conj(dU_ij) dU_ij (torch's for complex
 * leaves), FP64 accumulation in a fixed order.  stats (host, nrhs) report the
 * adjoint solves; the return value is that of the adjoint solves. */
int lqcd_gradient(lqcd_ctx *ctx, const double *src, const double *sol, int nrhs, const double *coef, double weight,
                  const lqcd_solver_params *params, double *dkappa, double *dU, lqcd_solve_stats *stats,
                  lqcd_stream_t stream);

/* No-allocation variant of lqcd_loops_batch.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory -- frameworks
 * whose caching allocator already holds the GPU's memory, latency-critical
 * pipelines in which the implicit device synchronisation of cudaFree would
 * stall other streams, and services that run under a fixed memory budget.  It
 * needs no context (lqcd_create allocates) and calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 * Same result as lqcd_loops_batch (accumulating into per_site / per_t) for the
 * lattice dims (host array of 4 ints, all even, volume <= 2^30, Lt <= 65535).
 * All arrays must be device memory of the current device (or managed memory),
 * and the stream must belong to that device; otherwise LQCD_ERR_INVALID.  The
 * per-time-slice partial sums use a fixed 768 KiB device array inside the
 * library: each GPU that loads the library holds it until the process exits.
 * Limit: Lt * ceil(Lx*Ly*Lz / 128) <= 8192 when per_t is given (24^3 x 48
 * needs 5184); larger lattices are rejected with LQCD_ERR_INVALID.  The first
 * call on a device that passes per_t looks up that array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls on a device share the array, so calls
 * whose work overlaps on the GPU (different streams, or host threads) race and
 * must be serialised by the caller; every partial is rewritten by each call,
 * so nothing needs clearing in between. */
int lqcd_loops_batch_noalloc(const int dims[4], const double *src, const double *sol, int nrhs, double weight,
                             double *per_site, double *per_t, lqcd_stream_t stream);

/* ---- measurement (instrumentation, not part of the method) -------------- */

/* Work of the dominant kernel, the reduced-precision Wilson hopping term of
 * the mixed solver, between lqcd_profile_begin and lqcd_profile_end. */
typedef struct {
  long long launches;     /* kernels launched by the library on any context       */
  long long hop_launches; /* launches of the reduced-precision hopping term       */
  double hop_ms;          /* their summed CUDA-event durations on the solve stream */
  double hop_site_rhs;    /* output (site, RHS) pairs they computed               */
  double hop_bytes;       /* algorithmic bytes: one read of every input spinor and
                             epilogue operand, one write of the output, and the
                             links once per launch                                 */
  double hop_flops;       /* 1320 flops per output site and RHS                    */
} lqcd_profile;

/* Start recording: events are placed around every reduced-precision hopping
 * launch of ctx until lqcd_profile_end.  Adds a little host overhead. */
int lqcd_profile_begin(lqcd_ctx *ctx);

/* Stop recording and fill *out (host).  Synchronises the device. */
int lqcd_profile_end(lqcd_ctx *ctx, lqcd_profile *out);

/* Total kernel launches made by the library since it was loaded (kernels run
 * by a replay of a captured CUDA graph count once per replay). */
long long lqcd_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* LQCD_H */
