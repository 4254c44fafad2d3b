// Host-side interface of the RHS-tile path (tile.cu) used by the solver driver
// (sloppy.cu).  Layout and kernels are described in tile.cuh.
#pragma once

#include "sloppy.cuh"

namespace lqcd {

constexpr int TR = 128;  // right-hand sides per tile (the MMA M of the tensor-core hop)
constexpr int TCH = 32;  // sites per reduction chunk (and work unit) of the tile kernels

// A site's block of a tile is [3 chunks][TR right-hand sides][8 reals] (6 KiB):
// chunk c holds reals 8c .. 8c+7 of every right-hand side as one 16-byte row, so
// that a warp reading chunk c of 32 consecutive right-hand sides reads 512
// contiguous bytes and each thread receives 8 consecutive reals of its own RHS.
// tile_chunk is the uint4 index of (tile T, site j, chunk c, RHS r) in a field,
// tile_elem the BF16 index of (T, j, real k, r).
__host__ __device__ inline size_t tile_chunk(int T, int vh, int j, int c, int r) {
  return (((size_t)T * vh + j) * 3 + c) * TR + r;
}
__host__ __device__ inline size_t tile_elem(int T, int vh, int j, int k, int r) {
  return tile_chunk(T, vh, j, k >> 3, r) * 8 + (k & 7);
}

// One BF16 sloppy field in 128-RHS tiles (element order of tile_elem).
struct TileField {
  __nv_bfloat16 *d = nullptr;
  int ntile = 0, vh = 0;
};

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
