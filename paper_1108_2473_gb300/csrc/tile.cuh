// RHS-tile layout of the mixed-precision solver and its tensor-core hopping
// term (Sec. II: the many-right-hand-side inversions; the Wilson hopping term
// of the operator D = 1 - kappa H).
//
// Layout.  A 16-bit (BF16) sloppy field holds its right-hand sides in tiles of
// TR = 128: [tile][Vh][2 halves][24 reals][64 RHS] (tile_elem), so one site's
// block of a tile (24 x 128 values, 6 KiB) is contiguous: 48 rows of 128 bytes,
// one TMA box.  The 24 reals are ordered ((spin * 3 + colour) * 2 + re/im).
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
// Data flow per (site, tile) item, warp-specialised inside one persistent CTA
// per SM, TNS-stage shared-memory ring:
//   * warp 0: TMA -- T_NT tiled loads (one [48 rows][128 B] box per neighbour,
//     128-byte swizzle) and one bulk copy of the site's link bundle into the
//     stage; the A buffer is [neighbour][half][24 rows][64 RHS], eight MN-major
//     SW128 blocks, which the MMAs address with per-step descriptors;
//   * warps 10-13: the other 8 - T_NT neighbour blocks by cp.async (16 bytes
//     per request, written to the same swizzled positions), so that the TMA
//     engine and the load/store units share the ~48 KiB an item needs;
//   * warps 2-5: build W (K-major, no swizzle) from the site's eight BF16 colour
//     matrices into a ring of two W buffers; entries of zero spin blocks are
//     written once at start;
//   * warp 1 (one thread): the twelve MMAs into one of two TMEM accumulators,
//     then tcgen05.commit to free the stage and to hand the accumulator on;
//   * warps 6-9 (one thread per right-hand side = TMEM lane): read the 24 FP32
//     results, apply the epilogue (out = cA A + cH D, optional dot products),
//     store BF16 (streaming stores), and accumulate per-RHS partial sums over
//     chunks of TCH sites.
// Every wait on an mbarrier is bounded; a wait that runs out sets an error
// code, the other roles stop at their next wait, TMA copies in flight are
// waited for (bounded), and TMEM is released before the kernel returns.
#pragma once

#include <cuda.h>

#include "tile_api.cuh"

namespace lqcd {

constexpr int TNS = 4;    // shared-memory stages of the hop pipeline (neighbour blocks + link bundle)
constexpr int TK = 192;   // MMA K per site: 8 directions x 24 reals
constexpr int TN = 32;    // MMA N: 24 output reals, padded
constexpr int T_A_NBR = 6144;                  // one neighbour block in a stage: [2 halves][24][64] BF16
constexpr int T_A_BYTES = 8 * T_A_NBR;         // 48 KiB
constexpr int T_W_BYTES = (TK / 8) * 512;      // 12 KiB: 24 K-chunks x 4 N-groups x 128 B
constexpr int T_NT = 0;                        // neighbours per item loaded by TMA; the rest by cp.async
constexpr int T_NL = 256;                      // cp.async loader threads (warps 10 ..)
constexpr int T_THREADS = 320 + T_NL;
constexpr int T_L_BYTES = 8 * 9 * 4;           // one site's link bundle: 288 B
constexpr int T_SMEM = 1024 + TNS * (T_A_BYTES + T_L_BYTES) + 2 * T_W_BYTES + 256;
constexpr int T_TMEM_COLS = 64;                // two FP32 accumulators of TN columns

// error codes written by the tile hop when a bounded wait runs out
enum { THOP_ERR_TMA = 1, THOP_ERR_W = 2, THOP_ERR_MMA = 3, THOP_ERR_ACC = 4, THOP_ERR_EPI = 5 };

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
  const __nv_bfloat16 *in; // the hop's input field (for the cp.async loaders)
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
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(b)), "r"(bytes) : "memory");
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
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(s_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(s_u32(bar))
               : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor (tcgen05): start, leading / stride byte
// offsets (16-byte units), version 1, layout (0 none, 2 = 128-byte swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}
// instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, A MN-major,
// B K-major, N = TN, M = TR
constexpr uint32_t T_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(TN >> 3) << 17) |
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
// sequence of (tile, site) items.  The grid-stride order keeps the whole GPU
// on a window of gridDim.x consecutive chunks of one tile, so that the eight
// uses of a neighbour block fall close together in time and hit in L2.
struct TItems {
  int u0, u1, ustep, nch, vh;
  __device__ void init(int count, int nch_, int vh_) {
    nch = nch_;
    vh = vh_;
    u0 = blockIdx.x;
    u1 = count * nch;
    ustep = gridDim.x;
  }
};
// results are stored with an L2 evict-first policy: they are not read again in
// this launch, and the neighbour blocks still to be reused should stay in L2
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, uint32_t src) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%1, %2}], [%3], %4;" ::"l"(
                   map),
               "r"(x), "r"(y), "r"(src), "l"(pol)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int EPI>
__global__ void __launch_bounds__(T_THREADS, 1) k_thop(const __grid_constant__ CUtensorMap tin, THopArgs a) {
  extern __shared__ __align__(1024) unsigned char t_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)t_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;                                  // TNS x 48 KiB neighbour blocks
  unsigned char *sW = base + TNS * T_A_BYTES;                // 2 x 12 KiB W ring
  unsigned char *sL = sW + 2 * T_W_BYTES;                    // TNS x 288 B link bundles
  uint64_t *bars = (uint64_t *)(sL + TNS * T_L_BYTES);       // full, empty, lfull [TNS]; accf, acce, wfull, wempty [2]; drain
  uint64_t *full = bars, *empty = bars + TNS, *lfull = bars + 2 * TNS;
  uint64_t *accf = bars + 3 * TNS, *acce = bars + 3 * TNS + 2;
  uint64_t *wfull = bars + 3 * TNS + 4, *wempty = bars + 3 * TNS + 6;
  uint64_t *drain = bars + 3 * TNS + 8;
  uint32_t *tslot = (uint32_t *)(drain + 1);
  volatile int *abort = (volatile int *)(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Geom &g = a.g;
  const int count = *a.tcount;
  TItems it;
  it.init(count, a.nch, g.Vh);

  // zero the W buffers (zero spin blocks stay zero), set up barriers and TMEM
  for (int i = tid; i < 2 * T_W_BYTES / 16; i += T_THREADS) reinterpret_cast<uint4 *>(sW)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < TNS; ++s) {
      mbar_init(full + s, 1 + T_NL);  // TMA producer, cp.async loaders
      mbar_init(empty + s, 1);
      mbar_init(lfull + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf + b, 1);
      mbar_init(acce + b, 128);
      mbar_init(wfull + b, 128);
      mbar_init(wempty + b, 1);
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
  if (warp == 0 && lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"(&tin) : "memory");
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    // the whole warp walks the items; lanes 0..T_NT-1 each issue one neighbour
    // block and lane 31 the link bundle
    int q = 0;
    int last_q[TNS];
    for (int s = 0; s < TNS; ++s) last_q[s] = -1;
    const int dn = lane;
    for (int u = it.u0; u < it.u1 && !*abort; u += it.ustep) {
      const int T = a.tlist[u / it.nch], ch = u % it.nch;
      const int j0 = ch * TCH, j1 = min(j0 + TCH, it.vh);
      if (a.prof && lane == 0)
        atomicAdd(a.prof + EPI, (unsigned long long)(j1 - j0) * (unsigned long long)min(TR, a.nrhs - T * TR));
      bool ok = true;
      for (int j = j0; j < j1; ++j, ++q) {
        const int s = q % TNS;
        const bool got = q < TNS || mbar_wait(empty + s, ((q / TNS) - 1) & 1, abort);
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0) atomicCAS(a.err, 0, THOP_ERR_TMA);
          *abort = 1;
          ok = false;
          break;
        }
        if (lane == 0) {
          mbar_arrive_tx(lfull + s, T_L_BYTES);
          mbar_arrive_tx(full + s, T_NT * T_A_NBR);
        }
        __syncwarp();
        if (lane < T_NT) {
          int c[4];
          coords_of(g, a.p_out, j, c);
          const int row = (T * it.vh + neighbour(g, c, dn)) * 48;
          tma_load_2d(s_u32(sA + s * T_A_BYTES) + dn * T_A_NBR, &tin, 0, row, full + s);
        } else if (lane == 31) {
          // the site's link bundle for the W builders
          bulk_load(s_u32(sL + s * T_L_BYTES), a.links + (size_t)(a.p_out * g.Vh + j) * 72, T_L_BYTES, lfull + s);
        }
        last_q[s] = q;
      }
      if (!ok) break;
    }
    // copies in flight must land before the CTA exits (normally already consumed)
    if (lane == 0)
      for (int s = 0; s < TNS; ++s)
        if (last_q[s] >= 0) {
          mbar_wait(full + s, (last_q[s] / TNS) & 1, abort);
          mbar_wait(lfull + s, (last_q[s] / TNS) & 1, abort);
        }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int q = 0;
      bool issued = false;
      for (int u = it.u0; u < it.u1 && !*abort; u += it.ustep) {
        const int ch = u % it.nch;
        const int j0 = ch * TCH, j1 = min(j0 + TCH, it.vh);
        for (int j = j0; j < j1; ++j, ++q) {
          const int s = q % TNS, acc = q & 1;
          if (!mbar_wait(full + s, (q / TNS) & 1, abort)) {
            atomicCAS(a.err, 0, THOP_ERR_MMA);
            *abort = 1;
            break;
          }
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
          tc_fence_after();
          const uint32_t aaddr = s_u32(sA + s * T_A_BYTES), waddr = s_u32(sW + acc * T_W_BYTES);
          // K = 192 = 8 neighbours x 24 reals in twelve steps of 16: rows 0..15 of
          // neighbour d (K-groups 3d, 3d+1: SBO 1 KiB), and rows 16..23 of the
          // neighbours d, d + 1 together (SBO 6 KiB); the W chunks follow the
          // same K order (LBO 512 B, resp. 3 x 512 B); LBO of A = the 3 KiB half
#pragma unroll
          for (int d = 0; d < 8; ++d) {
            tc_mma(tmem + acc * TN, smem_desc(aaddr + d * T_A_NBR, 3072, 1024, 2),
                   smem_desc(waddr + 3 * d * 512, 512, 128, 0), d > 0);
            if (d & 1)
              tc_mma(tmem + acc * TN, smem_desc(aaddr + (d - 1) * T_A_NBR + 2048, 3072, T_A_NBR, 2),
                     smem_desc(waddr + (3 * (d - 1) + 2) * 512, 3 * 512, 128, 0), 1);
          }
          tc_commit(empty + s);
          tc_commit(wempty + acc);
          tc_commit(accf + acc);
          issued = true;
        }
        if (*abort) break;
      }
      // every MMA issued must have completed before TMEM is released
      if (issued) {
        tc_commit(drain);
        mbar_wait(drain, 0, abort);
      }
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------ W builders
    const int b = tid - 64;  // 0..127; 96 of them own one (direction, spin, colour) output row pair
    const bool active = b < 96;
    const int d = b / 12, s = (b % 12) / 3, c = b % 3;
    int so = 0, pr = 0, pi = 0;
    if (active) {
      so = a.spin.so[d][s];
      pr = a.spin.pr[d][s];
      pi = a.spin.pi[d][s];
    }
    int q = 0;
    for (int u = it.u0; u < it.u1 && !*abort; u += it.ustep) {
      const int ch = u % it.nch;
      const int j0 = ch * TCH, j1 = min(j0 + TCH, it.vh);
      for (int j = j0; j < j1; ++j, ++q) {
        // W buffer q % 2 is free once the MMAs of item q - 2 are done; the link
        // bundle comes with the item's stage
        const int st = q % TNS, wb = q & 1;
        if ((q >= 2 && !mbar_wait(wempty + wb, ((q >> 1) - 1) & 1, abort)) ||
            !mbar_wait(lfull + st, (q / TNS) & 1, abort)) {
          atomicCAS(a.err, 0, THOP_ERR_W);
          *abort = 1;
          break;
        }
        if (active) {
          unsigned char *W = sW + wb * T_W_BYTES;
          const uint32_t *L = reinterpret_cast<const uint32_t *>(sL + st * T_L_BYTES) + d * 9 + c * 3;
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
    }
  } else if (warp < 10) {
    // ------------------------------------------------------------ epilogue
    // One thread per right-hand side = TMEM lane; every step is warp-uniform
    // (the accumulator wait is agreed on with __all_sync).  Each warp stages
    // its 32 right-hand sides of the BF16 result in shared memory ([24][32])
    // and writes them with one 2-d TMA store (box 32 x 24).
    const int quarter = warp & 3;
    const int row = 32 * quarter + lane;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    // epilogue operands (A, B) of item q + 1 are loaded while item q completes
    uint32_t na[12], nb[12];
    auto load_ops = [&](int T, int j) {
      const size_t e0 = tile_elem(T, g.Vh, j, 0, row);  // real k at e0 + 64 k
      if (EPI != EPI_PLAIN) {
#pragma unroll
        for (int k = 0; k < 12; ++k)
          na[k] = (uint32_t)__bfloat16_as_ushort(a.A[e0 + (size_t)(2 * k) * 64]) |
                  ((uint32_t)__bfloat16_as_ushort(a.A[e0 + (size_t)(2 * k + 1) * 64]) << 16);
      }
      if (EPI == EPI_DOTR) {
#pragma unroll
        for (int k = 0; k < 12; ++k)
          nb[k] = (uint32_t)__bfloat16_as_ushort(a.B[e0 + (size_t)(2 * k) * 64]) |
                  ((uint32_t)__bfloat16_as_ushort(a.B[e0 + (size_t)(2 * k + 1) * 64]) << 16);
      }
    };
    if (it.u0 < it.u1) load_ops(a.tlist[it.u0 / it.nch], (it.u0 % it.nch) * TCH);
    int q = 0;
    for (int u = it.u0; u < it.u1 && !*abort; u += it.ustep) {
      const int T = a.tlist[u / it.nch], ch = u % it.nch;
      const int j0 = ch * TCH, j1 = min(j0 + TCH, it.vh);
      const int rhs = T * TR + row;
      float sre = 0.f, sim = 0.f, snn = 0.f;
      bool ok = true;
      for (int j = j0; j < j1; ++j, ++q) {
        const int acc = q & 1;
        uint32_t ca[12], cb[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          ca[k] = na[k];
          cb[k] = nb[k];
        }
        // next item: the following site of this unit, else the first site of the next unit
        if (EPI != EPI_PLAIN) {
          if (j + 1 < j1) load_ops(T, j + 1);
          else if (u + it.ustep < it.u1) load_ops(a.tlist[(u + it.ustep) / it.nch], ((u + it.ustep) % it.nch) * TCH);
        }
        const bool got = mbar_wait(accf + acc, (q >> 1) & 1, abort);
        if (!__all_sync(0xffffffffu, got)) {
          atomicCAS(a.err, 0, THOP_ERR_EPI);
          *abort = 1;
          ok = false;
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
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            const float a0 = __uint_as_float(ca[k] << 16), a1 = __uint_as_float(ca[k] & 0xffff0000u);
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
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            const float b0 = __uint_as_float(cb[k] << 16), b1 = __uint_as_float(cb[k] & 0xffff0000u);
            sre = fmaf(b0, v[2 * k], fmaf(b1, v[2 * k + 1], sre));
            sim = fmaf(b0, v[2 * k + 1], fmaf(-b1, v[2 * k], sim));
          }
        }
        // streaming stores: the results are not read again in this launch
        {
          unsigned short *o = reinterpret_cast<unsigned short *>(a.out) + tile_elem(T, g.Vh, j, 0, row);
#pragma unroll
          for (int k = 0; k < 24; ++k) __stcs(o + (size_t)k * 64, __bfloat16_as_ushort(__float2bfloat16_rn(v[k])));
        }
      }
      if (!ok) break;
      if (EPI == EPI_DOTR || EPI == EPI_TS)
        a.part[(size_t)rhs * it.nch + ch] = D4S{(double)sre, (double)sim, 0.0, (double)snn};
    }
  } else {
    // ------------------------------------------------------------ cp.async loaders
    // Neighbours T_NT..7 of each item, 16 bytes per request; a thread's copies of
    // item q are fenced to the async proxy and announced on full[] once they have
    // landed, right after the copies of item q + 1 have been issued.
    const int l = tid - 320;
    constexpr int PER = (8 - T_NT) * 384 / T_NL;  // 16-byte chunks per thread and item
    int q = 0, pend = -1;
    for (int u = it.u0; u < it.u1 && !*abort; u += it.ustep) {
      const int T = a.tlist[u / it.nch], ch = u % it.nch;
      const int j0 = ch * TCH, j1 = min(j0 + TCH, it.vh);
      bool ok = true;
      for (int j = j0; j < j1; ++j, ++q) {
        const int s = q % TNS;
        const bool got = q < TNS || mbar_wait(empty + s, ((q / TNS) - 1) & 1, abort);
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0) atomicCAS(a.err, 0, THOP_ERR_TMA);
          *abort = 1;
          ok = false;
          break;
        }
        int c[4];
        coords_of(g, a.p_out, j, c);
        int nb[8 - T_NT];
#pragma unroll
        for (int d = T_NT; d < 8; ++d) nb[d - T_NT] = neighbour(g, c, d);
        const uint32_t sbase = s_u32(sA + s * T_A_BYTES);
#pragma unroll
        for (int m = 0; m < PER; ++m) {
          const int ci = l + T_NL * m, dd = ci / 384, w = ci % 384, row = w >> 3, c16 = w & 7;
          const uint4 *src = reinterpret_cast<const uint4 *>(a.in) + ((size_t)(T * it.vh + nb[dd]) * 384 + w);
          cp_async16(sbase + (T_NT + dd) * T_A_NBR + row * 128 + ((c16 ^ (row & 7)) << 4), src);
        }
        cp_async_commit();
        if (pend >= 0) {
          cp_async_wait1();
          fence_async_smem();
          mbar_arrive(full + pend);
        }
        pend = s;
      }
      if (!ok) break;
    }
    cp_async_wait_all();  // no copy may land after the CTA has left
    if (pend >= 0) {
      fence_async_smem();
      mbar_arrive(full + pend);
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
