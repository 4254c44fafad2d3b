// RHS-tile layout of the mixed-precision solver and its tensor-core hopping
// term (Sec. II: the many-right-hand-side inversions; the Wilson hopping term
// of the operator D = 1 - kappa H).
//
// Layout.  A 16-bit (BF16) sloppy field holds its right-hand sides in tiles of
// TR = 128; one site's block of a tile is [3 chunks][128 RHS][8 reals] (6 KiB,
// tile_chunk), the 24 reals ordered ((spin * 3 + colour) * 2 + re/im).
//
// Hopping term on the tensor cores.  For an output site x of parity p,
//   (H in)(x) = sum_{d=0..7} [P_d (x) C_d(x)] in(n_d(x)),
// d = 2 mu + (0 forward, 1 backward), n_d = x +- mu, P_d = 1 -+ gamma_mu and
// C_d = U_mu(x) or U_mu(x - mu)^+ (times -1 across the time boundary).  As a
// real matrix each P_d (x) C_d is 24 x 24; stacking the eight directions along
// K gives, for the 128 right-hand sides of one tile,
//   D[rhs][n] = sum_{k < 192} A[rhs][k] W[k][n],  A = the eight neighbour
//   blocks side by side (K = 8 x 24), W = the stacked 24 x 24 blocks,
// one M = 128, N = 32 (24 used), K = 192 product per (site, tile): twelve
// tcgen05.mma kind::f16 instructions (BF16 in, FP32 accumulate in TMEM).
//
// Data flow.  In this layout a site's block of a tile is already the canonical
// K-major, no-swizzle MMA operand: core matrices of 8 right-hand sides x 16 B,
// 128 B apart, and the K-chunks of 8 reals 2 KiB apart.  The eight neighbour
// blocks of an item, copied side by side into a shared-memory stage by eight
// bulk copies (cp.async.bulk, 6 KiB each), form the whole A = [128 RHS][192],
// which the twelve MMAs address with one descriptor advanced by 4 KiB per K step.
// TNI = 4 stages keep up to 192 KiB of copies in flight per SM without holding
// registers.  Each item's MMAs end in one tcgen05.commit, to an item-done
// barrier that every reuse waits on (the stage, the W buffer, the accumulator):
// each commit costs the issuing thread ~85 cycles, so per-buffer commits (up to
// eleven per item in earlier versions) had kept the tensor core waiting.
//
// Roles inside one persistent CTA per SM (223 KiB of shared memory, 64 TMEM
// columns), all walking the same (tile, site) item sequence:
//   * warp 0: bulk-copy producer; lane d < 8 copies neighbour block d of item q
//     into stage q % TNI once item q - TNI is done, after lane 0 has announced
//     the stage's 48 KiB on its full barrier;
//   * warp 1: TMEM allocation (two FP32 accumulators of TN columns); one thread
//     issues the twelve MMAs of an item and one commit;
//   * warps 2-5: build W (K-major, no swizzle) into a ring of two W buffers
//     from the site's eight BF16 colour matrices, whose words each builder
//     thread loads T_LPF items ahead; entries of zero spin blocks are written
//     once at start;
//   * warps 6-9 (one thread per right-hand side = TMEM lane): read the 24 FP32
//     results, apply the epilogue (out = cA A + cH D, optional dot products),
//     store BF16 (streaming stores) and accumulate per-RHS partial sums over
//     chunks of TCH sites.
// Every wait on an mbarrier is bounded; a wait that runs out sets an error
// code, the other roles stop at their next wait, bulk copies in flight and
// issued MMAs are waited for (bounded by time only), and TMEM is released
// before the kernel returns.
#pragma once

#include "tile_api.cuh"

namespace lqcd {

constexpr int TK = 192;   // MMA K per site: 8 directions x 24 reals
constexpr int TN = 32;    // MMA N: 24 output reals, padded
constexpr int T_W_BYTES = (TK / 8) * 512;      // 12 KiB: 24 K-chunks x 4 N-groups x 128 B

// error codes written by the tile hop when a bounded wait runs out
enum { THOP_ERR_LOAD = 1, THOP_ERR_W = 2, THOP_ERR_MMA = 3, THOP_ERR_ACC = 4, THOP_ERR_EPI = 5 };

// Spin structure of P_d = 1 -+ gamma_mu (DeGrand-Rossi): row s has the identity
// and one off-diagonal entry at column so[d][s] with value (re, im) in {0, +-1}.
struct TSpin {
  int so[8][4];
  int pr[8][4], pi[8][4];
};

struct THopArgs {
  Geom g;
  int p_out;
  const uint32_t *links;  // [2 parity][Vh][8 d][9] BF16x2 (re low, im high), signs and daggers folded in
  __nv_bfloat16 *out;
  const __nv_bfloat16 *in; // the hop's input field
  const __nv_bfloat16 *A;  // epilogue operand (tile field), EPI != PLAIN
  const __nv_bfloat16 *B;  // <B, out> for EPI_DOTR
  float cA, cH;
  const int *tlist, *tcount;  // active tiles
  D4S *part;                  // [rhs][nch] partial sums
  int nch;                    // chunks of TCH sites per tile = ceil(Vh / TCH)
  int nrhs;                   // right-hand sides in use (rows beyond are padding)
  unsigned long long *prof;   // (site, RHS) outputs per epilogue kind, or null
  int *err;                   // device error code (0 = fine)
  TSpin spin;
};

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t s_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.u32 %0, 1, 0, P;\n}"
      : "=r"(ok)
      : "r"(s_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(b)) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// bounded wait: false when 2 s pass (every legitimate wait here is microseconds)
// or another role has aborted
constexpr uint64_t T_WAIT_NS = 2000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort) return false;
      if (global_ns() - t0 > T_WAIT_NS) return false;
    }
  }
}
// drain wait: bounded by time only, so that asynchronous work this thread
// started (MMAs) has finished before TMEM or shared memory is
// given up, even after another role has aborted
__device__ __forceinline__ bool mbar_wait_drain(uint64_t *b, uint32_t parity) {
  const uint64_t t0 = global_ns();
  while (!mbar_try(b, parity))
    if (global_ns() - t0 > T_WAIT_NS) return false;
  return true;
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(s_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor (tcgen05): start, leading / stride byte
// offsets (16-byte units), version 1, layout (0 none, 2 = 128-byte swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}
// instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, N = TN, M = TR
constexpr uint32_t T_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                             ((uint32_t)(TR >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(T_IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_ld24(uint32_t taddr, float v[24]) {
  uint32_t r[24];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
                 "=r"(r[23])
               : "r"(taddr + 16)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 24; ++k) v[k] = __uint_as_float(r[k]);
}

// byte offset of W[k][n] in the K-major, no-swizzle B buffer: core matrices of
// 8 N-rows x 16 bytes; LBO (next 8 K) = 512 B, SBO (next 8 N) = 128 B
__device__ __forceinline__ uint32_t w_off(int k, int n) {
  return (uint32_t)((k >> 3) * 512 + (n >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2);
}

// neighbour parity-local index of output site (coords c) in direction d
__device__ __forceinline__ int neighbour(const Geom &g, const int c[4], int d) {
  const int mu = d >> 1;
  int cn[4] = {c[0], c[1], c[2], c[3]};
  if ((d & 1) == 0) cn[mu] = (c[mu] + 1 == g.L[mu]) ? 0 : c[mu] + 1;
  else cn[mu] = (c[mu] == 0) ? g.L[mu] - 1 : c[mu] - 1;
  return site_of(g, cn) >> 1;
}

// Work of one CTA: units u = blockIdx.x, blockIdx.x + gridDim.x, ... of
// (active tile, chunk of TCH sites), tile-major; every role walks the same
// sequence of (tile, site) items with a TCur cursor (divisions once per unit,
// not per item).  The grid-stride order keeps the whole GPU on a window of
// gridDim.x consecutive chunks of one tile, so that the eight uses of a
// neighbour block fall close together in time and hit in L2.
struct TCur {
  int u, j, jend, T, ch;
};
struct TItems {
  int u0, u1, ustep, nch, vh;
  const int *tlist;
  __device__ void init(int count, int nch_, int vh_, const int *tlist_) {
    nch = nch_;
    vh = vh_;
    tlist = tlist_;
    u0 = blockIdx.x;
    u1 = count * nch;
    ustep = gridDim.x;
  }
  __device__ bool set(TCur &c, int u) const {
    if (u >= u1) return false;
    c.u = u;
    c.ch = u % nch;
    c.T = tlist[u / nch];
    c.j = c.ch * TCH;
    c.jend = min(c.j + TCH, vh);
    return true;
  }
  __device__ bool first(TCur &c) const { return set(c, u0); }
  // the item after c; false past the last one
  __device__ bool next(TCur &c) const { return ++c.j < c.jend || set(c, c.u + ustep); }
};
// coordinates of the parity-p site after the one with coordinates c (parity-local
// index + 1, as coords_of orders them)
__device__ __forceinline__ void coords_next(const Geom &g, int p, int c[4]) {
  int xh = c[0] >> 1;
  if (++xh == g.Lxh) {
    xh = 0;
    if (++c[1] == g.L[1]) {
      c[1] = 0;
      if (++c[2] == g.L[2]) {
        c[2] = 0;
        ++c[3];
      }
    }
  }
  c[0] = 2 * xh + ((c[1] + c[2] + c[3] + p) & 1);
}

// Stages in shared memory, one bulk copy per neighbour block, one commit per item.
constexpr int TNI = 4;                          // items in flight (shared-memory stages)
constexpr int T_BLK_BYTES = 3 * TR * 16;        // one site block of a tile: 6 KiB
constexpr int T_A_BYTES = 8 * T_BLK_BYTES;      // an item's eight neighbour blocks side by side: 48 KiB
constexpr int T_DONE = 16;                      // item-done barriers (deeper than any role lags)
constexpr int T_THREADS = 320;
constexpr int T_TMEM_COLS = 64;                 // two FP32 accumulators of TN columns
constexpr int T_LPF = 4;                        // items of link words the W builders hold in registers
constexpr int T_SMEM = 1024 + TNI * T_A_BYTES + 2 * T_W_BYTES + 1024;
static_assert(T_SMEM <= 227 * 1024, "tile hop shared memory");

template <int EPI>
__global__ void __launch_bounds__(T_THREADS, 1) k_thop(THopArgs a) {
  extern __shared__ __align__(1024) unsigned char t_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)t_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;                       // TNI x 48 KiB
  unsigned char *sW = sA + TNI * T_A_BYTES;       // 2 x 12 KiB W ring
  uint64_t *bars = (uint64_t *)(sW + 2 * T_W_BYTES);
  uint64_t *full = bars, *done = bars + TNI, *acce = done + T_DONE, *wfull = acce + 2, *drain = wfull + 2;
  uint32_t *tslot = (uint32_t *)(drain + 1);
  volatile int *abort = (volatile int *)(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Geom &g = a.g;
  const int count = *a.tcount;
  TItems it;
  it.init(count, a.nch, g.Vh, a.tlist);

  for (int i = tid; i < 2 * T_W_BYTES / 16; i += T_THREADS) reinterpret_cast<uint4 *>(sW)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < TNI; ++s) mbar_init(full + s, 1);
    for (int s = 0; s < T_DONE; ++s) mbar_init(done + s, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(acce + b, 128);
      mbar_init(wfull + b, 128);
    }
    mbar_init(drain, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(tslot)),
                 "r"(T_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ------------------------------------------------------------ bulk-copy producer
    // lane d < 8 copies neighbour block d of item q into stage q % TNI once the
    // MMAs of item q - TNI (the stage's last user) have completed; lane 0 first
    // announces the stage's 48 KiB on its full barrier.
    if (lane == 0 && a.prof)
      for (int v = it.u0; v < it.u1; v += it.ustep) {
        const int T = a.tlist[v / it.nch], ch = v % it.nch;
        atomicAdd(a.prof + EPI, (unsigned long long)(min(ch * TCH + TCH, it.vh) - ch * TCH) *
                                    (unsigned long long)min(TR, a.nrhs - T * TR));
      }
    const uint4 *in4 = reinterpret_cast<const uint4 *>(a.in);
    int q = 0, last_q = -1, cu = -1, cc[4];
    TCur cur;
    for (bool more = it.first(cur); more && !*abort; more = it.next(cur), ++q) {
      const int st = q % TNI, qr = q - TNI;
      const bool got = qr < 0 || lane > 0 || mbar_wait(done + qr % T_DONE, (qr / T_DONE) & 1, abort);
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0) atomicCAS(a.err, 0, THOP_ERR_LOAD);
        *abort = 1;
        break;
      }
      if (cur.u != cu) {
        coords_of(g, a.p_out, cur.j, cc);
        cu = cur.u;
      } else {
        coords_next(g, a.p_out, cc);
      }
      if (lane == 0) mbar_arrive_tx(full + st, T_A_BYTES);
      __syncwarp();
      if (lane < 8) {
        const size_t src = tile_chunk(cur.T, g.Vh, neighbour(g, cc, lane), 0, 0);
        bulk_load(s_u32(sA + (size_t)st * T_A_BYTES + lane * T_BLK_BYTES), in4 + src, T_BLK_BYTES, full + st);
      }
      last_q = q;
    }
    // copies in flight must land before the CTA exits (normally already consumed)
    if (lane == 0)
      for (int qq = max(0, last_q - TNI + 1); qq <= last_q; ++qq) mbar_wait_drain(full + qq % TNI, (qq / TNI) & 1);
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int q = 0;
      bool issued = false;
      TCur cur;
      for (bool more = it.first(cur); more && !*abort; more = it.next(cur), ++q) {
        const int st = q % TNI, acc = q & 1;
        if (!mbar_wait(wfull + acc, (q >> 1) & 1, abort)) {
          atomicCAS(a.err, 0, THOP_ERR_W);
          *abort = 1;
          break;
        }
        if (q >= 2 && !mbar_wait(acce + acc, ((q >> 1) - 1) & 1, abort)) {
          atomicCAS(a.err, 0, THOP_ERR_ACC);
          *abort = 1;
          break;
        }
        if (!mbar_wait(full + st, (q / TNI) & 1, abort)) {
          atomicCAS(a.err, 0, THOP_ERR_MMA);
          *abort = 1;
          break;
        }
        // K = 192 in twelve steps of 16: step k reads K-chunks 2k, 2k + 1 of the
        // eight neighbour blocks side by side (chunk c at 2 KiB c: LBO 2 KiB, SBO
        // 128 B, no swizzle) and W K-chunks 2k, 2k + 1 (LBO 512 B, SBO 128 B); the
        // descriptors' start fields advance by 4096 / 16 and 1024 / 16 per step
        const uint64_t ad = smem_desc(s_u32(sA + (size_t)st * T_A_BYTES), 2048, 128, 0);
        const uint64_t bd = smem_desc(s_u32(sW + acc * T_W_BYTES), 512, 128, 0);
        const uint32_t dacc = tmem + acc * TN;
        tc_fence_after();
#pragma unroll
        for (int k = 0; k < 12; ++k) tc_mma(dacc, ad + (uint64_t)(256 * k), bd + (uint64_t)(64 * k), k > 0);
        tc_commit(done + q % T_DONE);  // the stage, W buffer and accumulator wait on this
        issued = true;
      }
      if (issued) {
        tc_commit(drain);
        mbar_wait_drain(drain, 0);
      }
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------ W builders
    const int b = tid - 64;
    const bool active = b < 96;
    const int d = b / 12, s = (b % 12) / 3, c = b % 3;
    int so = 0, pr = 0, pi = 0;
    if (active) {
      so = a.spin.so[d][s];
      pr = a.spin.pr[d][s];
      pi = a.spin.pi[d][s];
    }
    const uint32_t *lk = a.links + (size_t)a.p_out * g.Vh * 72 + d * 9 + c * 3;
    uint32_t lw[T_LPF][3];
    TCur pf;
    bool pf_more = it.first(pf);
#pragma unroll
    for (int i = 0; i < T_LPF; ++i) {
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) lw[i][cc] = (active && pf_more) ? __ldg(lk + (size_t)pf.j * 72 + cc) : 0u;
      if (pf_more) pf_more = it.next(pf);
    }
    int q = 0;
    TCur cur;
    for (bool more = it.first(cur); more && !*abort; more = it.next(cur), ++q) {
      // W buffer q % 2 is free once the MMAs of item q - 2 are done
      const int wb = q & 1, qr = q - 2;
      if (qr >= 0 && !mbar_wait(done + qr % T_DONE, (qr / T_DONE) & 1, abort)) {
        atomicCAS(a.err, 0, THOP_ERR_W);
        *abort = 1;
        break;
      }
      uint32_t L[3] = {lw[0][0], lw[0][1], lw[0][2]};
#pragma unroll
      for (int i = 0; i + 1 < T_LPF; ++i)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) lw[i][cc] = lw[i + 1][cc];
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) lw[T_LPF - 1][cc] = (active && pf_more) ? __ldg(lk + (size_t)pf.j * 72 + cc) : 0u;
      if (pf_more) pf_more = it.next(pf);
      if (active) {
        unsigned char *W = sW + wb * T_W_BYTES;
        const int nr = (s * 3 + c) * 2;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          const uint32_t w = L[cc];
          // identity block: z = C[c][cc]
          const int kd = d * 24 + (s * 3 + cc) * 2;
          const uint32_t cr = w & 0xffffu, ci = w >> 16;
          *reinterpret_cast<uint32_t *>(W + w_off(kd, nr)) = cr | ((ci ^ 0x8000u) << 16);      // (zr, -zi)
          *reinterpret_cast<uint32_t *>(W + w_off(kd, nr + 1)) = ci | (cr << 16);             // (zi, zr)
          // off-diagonal block: z = p C[c][cc], p = pr + i pi in {+-1, +-i}
          uint32_t zr, zi;
          if (pr != 0) {
            const uint32_t sg = pr < 0 ? 0x8000u : 0u;
            zr = cr ^ sg;
            zi = ci ^ sg;
          } else {  // i pi (cr + i ci) = -pi ci + i pi cr
            const uint32_t sg = pi < 0 ? 0x8000u : 0u;
            zr = ci ^ 0x8000u ^ sg;
            zi = cr ^ sg;
          }
          const int ko = d * 24 + (so * 3 + cc) * 2;
          *reinterpret_cast<uint32_t *>(W + w_off(ko, nr)) = zr | ((zi ^ 0x8000u) << 16);
          *reinterpret_cast<uint32_t *>(W + w_off(ko, nr + 1)) = zi | (zr << 16);
        }
      }
      fence_async_smem();
      mbar_arrive(wfull + wb);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // One thread per right-hand side = TMEM lane; every step is warp-uniform
    // (the wait is agreed on with __all_sync).  The item's epilogue operands are
    // loaded before the wait for its MMAs.
    const int quarter = warp & 3;
    const int row = 32 * quarter + lane;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    const uint4 *A4 = reinterpret_cast<const uint4 *>(a.A), *B4 = reinterpret_cast<const uint4 *>(a.B);
    uint4 *O4 = reinterpret_cast<uint4 *>(a.out);
    int q = 0;
    float sre = 0.f, sim = 0.f, snn = 0.f;
    TCur cur;
    for (bool more = it.first(cur); more && !*abort;) {
      const int T = cur.T, ch = cur.ch;
      const size_t e0 = tile_chunk(T, g.Vh, cur.j, 0, row);
      const int acc = q & 1;
      uint4 ca[3], cb[3];
      if (EPI != EPI_PLAIN)
#pragma unroll
        for (int c = 0; c < 3; ++c) ca[c] = A4[e0 + c * TR];
      if (EPI == EPI_DOTR)
#pragma unroll
        for (int c = 0; c < 3; ++c) cb[c] = B4[e0 + c * TR];
      const bool got = mbar_wait(done + q % T_DONE, (q / T_DONE) & 1, abort);
      if (!__all_sync(0xffffffffu, got)) {
        atomicCAS(a.err, 0, THOP_ERR_EPI);
        *abort = 1;
        break;
      }
      tc_fence_after();
      float v[24];
      tc_ld24(tmem + lane_off + acc * TN, v);
      tc_fence_before();
      mbar_arrive(acce + acc);
#pragma unroll
      for (int k = 0; k < 24; ++k) v[k] *= a.cH;
      if (EPI != EPI_PLAIN) {
        const uint32_t *aw = reinterpret_cast<const uint32_t *>(ca);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const float a0 = __uint_as_float(aw[k] << 16), a1 = __uint_as_float(aw[k] & 0xffff0000u);
          v[2 * k] = fmaf(a.cA, a0, v[2 * k]);
          v[2 * k + 1] = fmaf(a.cA, a1, v[2 * k + 1]);
          if (EPI == EPI_TS) {  // <out, A> and |out|^2
            sre = fmaf(v[2 * k], a0, fmaf(v[2 * k + 1], a1, sre));
            sim = fmaf(v[2 * k], a1, fmaf(-v[2 * k + 1], a0, sim));
            snn = fmaf(v[2 * k], v[2 * k], fmaf(v[2 * k + 1], v[2 * k + 1], snn));
          }
        }
      }
      if (EPI == EPI_DOTR) {  // <B, out>
        const uint32_t *bw = reinterpret_cast<const uint32_t *>(cb);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const float b0 = __uint_as_float(bw[k] << 16), b1 = __uint_as_float(bw[k] & 0xffff0000u);
          sre = fmaf(b0, v[2 * k], fmaf(b1, v[2 * k + 1], sre));
          sim = fmaf(b0, v[2 * k + 1], fmaf(-b1, v[2 * k], sim));
        }
      }
      // streaming stores: the results are not read again in this launch
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          __nv_bfloat162 p2 = __floats2bfloat162_rn(v[8 * c + 2 * h], v[8 * c + 2 * h + 1]);
          w[h] = *reinterpret_cast<uint32_t *>(&p2);
        }
        __stcs(O4 + e0 + c * TR, make_uint4(w[0], w[1], w[2], w[3]));
      }
      ++q;
      const int u_prev = cur.u;
      more = it.next(cur);
      if (!more || cur.u != u_prev) {  // the unit's chunk is complete
        if (EPI == EPI_DOTR || EPI == EPI_TS)
          a.part[(size_t)(T * TR + row) * it.nch + ch] = D4S{(double)sre, (double)sim, 0.0, (double)snn};
        sre = sim = snn = 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T_TMEM_COLS) : "memory");
  }
}

}  // namespace lqcd
