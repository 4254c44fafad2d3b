// Complex Z2 noise sources (Sec. II, Eq. delta functions) from Philox4x64-10
// (Salmon, Moraes, Dror, Shaw, SC'11), with time / spin / colour dilution and
// even-odd or cubic spatial partitioning (Sec. II).
#include "internal.cuh"

namespace lqcd {

// Philox4x64 round constants and Weyl key increments (SC'11).
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t hi0 = __umul64hi(PHILOX_M0, c[0]), lo0 = PHILOX_M0 * c[0];
    uint64_t hi1 = __umul64hi(PHILOX_M1, c[2]), lo1 = PHILOX_M1 * c[2];
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// One thread per (piece, site) computes the site's Philox word and the mask of
// components its piece keeps; the warp then writes its 32 sites' 384 complex
// values as consecutive 16-byte chunks (lane l writes element 32 r + l in round
// r), with the word and mask fetched from the owning lane by shuffles.
__global__ void k_noise(Geom g, uint64_t seed, uint64_t stream_tag, uint64_t noise_index, int dilution,
                        int first_piece, int n_pieces, double2 *out) {
  const size_t total = (size_t)n_pieces * g.V;
  const size_t warp_base = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(size_t)31;
  const size_t idx = warp_base + (threadIdx.x & 31);
  const int lane = threadIdx.x & 31;
  uint64_t w = 0;
  unsigned keep = 0u;  // bit k: component k kept
  if (idx < total) {
    int piece = first_piece + (int)(idx / g.V);
    const int s = (int)(idx % g.V);
    const int t = s / (g.L[0] * g.L[1] * g.L[2]);
    // spatial partition: the piece's class among n_sp, and the site's class
    const int spatial = dilution & ~3;
    const int n_sp = spatial == LQCD_DILUTE_EO ? 2 : (spatial == LQCD_DILUTE_CUBE ? 8 : 1);
    const int x = s % g.L[0], y = (s / g.L[0]) % g.L[1], z = (s / (g.L[0] * g.L[1])) % g.L[2];
    const int site_cls = spatial == LQCD_DILUTE_EO ? (x + y + z) & 1
                         : spatial == LQCD_DILUTE_CUBE ? (x & 1) + 2 * (y & 1) + 4 * (z & 1) : 0;
    const bool in_class = piece % n_sp == site_cls;
    piece /= n_sp;
    const int base = dilution & 3;
    int pt = -1, ps = -1, pc = -1;  // kept time slice / spin / colour (-1: all)
    if (base == LQCD_DILUTE_T) {
      pt = piece;
    } else if (base == LQCD_DILUTE_TS) {
      pt = piece / 4;
      ps = piece % 4;
    } else if (base == LQCD_DILUTE_TSC) {
      pt = piece / 12;
      ps = (piece % 12) / 3;
      pc = piece % 3;
    }
    if ((pt < 0 || t == pt) && in_class) {
      uint64_t c[4] = {(uint64_t)s, noise_index, 0ULL, 0ULL};
      philox4x64_10(c, seed, stream_tag);
      w = c[0];
#pragma unroll
      for (int k = 0; k < 12; ++k)
        if ((ps < 0 || k / 3 == ps) && (pc < 0 || k % 3 == pc)) keep |= 1u << k;
    }
  }
  const double h = 0.70710678118654752440;  // 1/sqrt(2), correctly rounded
  const unsigned wlo = (unsigned)w, whi = (unsigned)(w >> 32);
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    const int e = 32 * r + lane;  // element of the warp's 32 x 12 block
    const int owner = e / 12, k = e % 12;
    const unsigned lo = __shfl_sync(0xffffffffu, wlo, owner), hi = __shfl_sync(0xffffffffu, whi, owner);
    const unsigned km = __shfl_sync(0xffffffffu, keep, owner);
    const size_t site_idx = warp_base + owner;
    if (site_idx < total) {
      const uint64_t ww = ((uint64_t)hi << 32) | lo;
      const double re = ((ww >> (2 * k)) & 1ULL) ? -h : h;
      const double im = ((ww >> (2 * k + 1)) & 1ULL) ? -h : h;
      out[site_idx * 12 + k] = ((km >> k) & 1u) ? make_double2(re, im) : make_double2(0.0, 0.0);
    }
  }
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_dilution_pieces(const int dims[4], int dilution) {
  LQCD_TRACE("lqcd_dilution_pieces"); return dilution_pieces(dims, dilution); }

extern "C" int lqcd_noise_generate(uint64_t seed, uint64_t noise_stream, uint64_t noise_index, const int dims[4],
                                   int dilution, int first_piece, int n_pieces, double *out, lqcd_stream_t stream) {
  LQCD_TRACE("lqcd_noise_generate");
  if (!dims || n_pieces < 0 || first_piece < 0 || (n_pieces > 0 && !out))
    return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_noise_generate: bad argument");
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || (dims[i] & 1)) return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_noise_generate: bad dims");
  const int npieces_total = dilution_pieces(dims, dilution);
  if (npieces_total < 0)
    return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_noise_generate: unknown dilution %d", dilution);
  if (first_piece + n_pieces > npieces_total)
    return set_error(nullptr, LQCD_ERR_INVALID, "lqcd_noise_generate: pieces %d..%d beyond %d", first_piece,
                     first_piece + n_pieces - 1, npieces_total);
  if (n_pieces == 0) return LQCD_OK;
  Geom g = make_geom(dims);
  size_t total = (size_t)n_pieces * g.V;
  KL k_noise<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(g, seed, noise_stream, noise_index,
                                                                             dilution, first_piece, n_pieces,
                                                                             (double2 *)out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(nullptr, e, "k_noise");
  return LQCD_OK;
}
