// Host-side interface of the RHS-tile path (tile.cu) used by the solver driver
// (sloppy.cu).  Layout and kernels are described in tile.cuh.
#pragma once

#include <cuda.h>

#include "sloppy.cuh"

namespace lqcd {

constexpr int TR = 128;  // right-hand sides per tile (the MMA M of the tensor-core hop)
constexpr int TCH = 32;  // sites per reduction chunk (and work unit) of the tile kernels

// Element (real k, right-hand side r) of site j of tile T in a tile field:
// [tile][site][half = r / 64][24 reals][64 RHS], so that one site's block of a
// tile (6 KiB) is 48 rows of 128 bytes, each half a contiguous 3 KiB.
__host__ __device__ inline size_t tile_elem(int T, int vh, int j, int k, int r) {
  return ((((size_t)T * vh + j) * 2 + (r >> 6)) * 24 + k) * 64 + (r & 63);
}

// One BF16 sloppy field in 128-RHS tiles (element order of tile_elem), with the
// TMA tensor maps of the tensor-core hop (built by tile_field_map) over the 2-d
// view [ntile * vh * 48 rows][64 RHS]: `map` loads a neighbour block (64 x 48,
// 128-byte swizzle), `smap` stores an epilogue warp's share of an output block
// (32 x 24, no swizzle).
struct TileField {
  __nv_bfloat16 *d = nullptr;
  int ntile = 0, vh = 0;
  CUtensorMap map, smap;
};

int tile_field_map(lqcd_ctx *ctx, TileField &f);

// out = cA A + cH (H in) at the sites of parity p_out for the listed tiles;
// EPI_DOTR adds partials <B, out>, EPI_TS <out, A> and |out|^2 per RHS and
// chunk of TCH sites ([rhs][nch]).  *err receives a nonzero code if a bounded
// wait inside the kernel ran out.
int tile_hop(int epi, cudaStream_t q, int G, lqcd_ctx *ctx, int p_out, const TileField &in, const TileField &out,
             const TileField &A, const TileField &B, float cA, float cH, const int *tlist, const int *tcount, D4S *part,
             int nch, int nrhs, unsigned long long *prof, int *err);
int tile_p(cudaStream_t q, int G, int vh, const SState *sc, const TileField &r, const TileField &rhat,
           const TileField &p, const TileField &v, const int *tlist, const int *tcount);
int tile_s(cudaStream_t q, int G, int vh, const SState *sc, const TileField &r, const TileField &v,
           const TileField &s, const int *tlist, const int *tcount);
int tile_xr(cudaStream_t q, int G, int vh, const SState *sc, const int *flags, F32F x, const TileField &p,
            const TileField &s, const TileField &t, const TileField &r, const TileField &rhat, const int *tlist,
            const int *tcount, D4S *part);
int tile_copy(cudaStream_t q, int G, int vh, const int *flags, F32F src, const TileField &r, const TileField &rhat,
              bool use_rhat, F32F x, bool zero_x, const int *tlist, const int *tcount, D4S *part);

}  // namespace lqcd
