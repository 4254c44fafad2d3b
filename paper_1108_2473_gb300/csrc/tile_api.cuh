// Host-side interface of the RHS-tile path (tile.cu) used by the solver driver
// (sloppy.cu).  Layout and kernels are described in tile.cuh.
#pragma once

#include <cuda.h>

#include "sloppy.cuh"

namespace lqcd {

constexpr int TR = 128;  // right-hand sides per tile (the MMA M of the tensor-core hop)
constexpr int TCH = 64;  // sites per reduction chunk of the tile kernels

// One BF16 sloppy field in 128-RHS tiles: [ntile][vh][24][128] BF16, with the
// TMA tensor maps of the tensor-core hop (built by tile_field_map): `map`
// loads a neighbour half (64 RHS x 24 rows, 128-byte swizzle), `smap` stores an
// epilogue warp's share of an output block (32 RHS x 24 rows, no swizzle).
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
