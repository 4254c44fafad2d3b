"""Counter-based complex Z2 noise (Sec. II) from Philox4x64-10.

Philox4x64-10 follows its published definition (J. K. Salmon, M. A. Moraes,
R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
ten rounds of two 64x64->128-bit multiplications, with the key bumped by the
Weyl constants between rounds.  Pinned against numpy.random.Philox, an
independent implementation of the same generator (tests/test_oracle_philox.py).

Noise definition (this library's; the paper fixes only the noise properties,
Sec. II, Eq. delta functions):

* key = (seed, stream), counter = (site, noise_index, 0, 0), where site is the
  lexicographic index x + Lx*(y + Ly*(z + Lz*t)) and stream is 0 for the
  plain / low-precision set and 1 for the TSM high-precision correction set;
* the first 64-bit output word w gives component k = 3*spin + colour the value
  ((-1)^{bit 2k of w} + i (-1)^{bit 2k+1 of w}) / sqrt(2).

Then <xi> -> 0 and <xi xi^*> -> delta as the paper requires, and |xi|^2 = 1
exactly per component.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a, b):
    """(hi, lo) 64-bit halves of the 128-bit product a*b for uint64 arrays."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _MASK32, a >> _S32
    b_lo, b_hi = b & _MASK32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _MASK32) + (hl & _MASK32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    lo = a * b
    return hi, lo


def philox4x64_10(counter, key):
    """Philox4x64 with 10 rounds.

    ``counter``: 4 uint64 arrays (broadcastable), ``key``: 2 uint64 values.
    Returns the 4 output words as uint64 arrays.
    """
    with np.errstate(over="ignore"):
        c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) for c in counter)
        k0 = np.uint64(key[0])
        k1 = np.uint64(key[1])
        m0 = np.uint64(M0)
        m1 = np.uint64(M1)
        for rnd in range(10):
            if rnd > 0:
                k0 = np.uint64((int(k0) + W0) & 0xFFFFFFFFFFFFFFFF)
                k1 = np.uint64((int(k1) + W1) & 0xFFFFFFFFFFFFFFFF)
            hi0, lo0 = _mulhilo64(m0, c0)
            hi1, lo1 = _mulhilo64(m1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        return c0, c1, c2, c3


SQRT1_2 = np.sqrt(0.5)  # correctly rounded double 1/sqrt(2)


def z2_noise(dims, seed, noise_index, stream=0):
    """Undiluted complex Z2 noise vector, shape (Lt, Lz, Ly, Lx, 4, 3)."""
    lx, ly, lz, lt = dims
    v = lx * ly * lz * lt
    site = np.arange(v, dtype=np.uint64)
    w0, _, _, _ = philox4x64_10((site, np.uint64(noise_index), np.uint64(0), np.uint64(0)),
                                (np.uint64(seed), np.uint64(stream)))
    k = np.arange(12, dtype=np.uint64)
    re_bit = (w0[:, None] >> (2 * k)[None, :]) & np.uint64(1)
    im_bit = (w0[:, None] >> (2 * k + 1)[None, :]) & np.uint64(1)
    re = np.where(re_bit == 1, -SQRT1_2, SQRT1_2)
    im = np.where(im_bit == 1, -SQRT1_2, SQRT1_2)
    xi = (re + 1j * im).reshape(lt, lz, ly, lx, 4, 3)
    return xi


# dilution schemes (Sec. II): which indices one diluted source keeps.  A base
# scheme (none, time, time+spin, time+spin+colour) may carry one spatial
# partition flag: even-odd (x+y+z mod 2, two classes) or cubic (the eight
# vertices of an elementary 3-cube, (x mod 2) + 2 (y mod 2) + 4 (z mod 2)).
DIL_NONE, DIL_T, DIL_TS, DIL_TSC = 0, 1, 2, 3
DIL_EO, DIL_CUBE = 4, 8


def _split(scheme):
    base, spatial = scheme & 3, scheme & ~3
    if spatial not in (0, DIL_EO, DIL_CUBE):
        raise ValueError("unknown dilution scheme")
    return base, {0: 1, DIL_EO: 2, DIL_CUBE: 8}[spatial], spatial


def dilution_count(dims, scheme):
    base, n_sp, _ = _split(scheme)
    lt = dims[3]
    return {DIL_NONE: 1, DIL_T: lt, DIL_TS: 4 * lt, DIL_TSC: 12 * lt}[base] * n_sp


def spatial_class(dims, scheme):
    """Spatial partition class of every site, shape (Lt, Lz, Ly, Lx) (all zero without a flag)."""
    lx, ly, lz, lt = dims
    _, _, spatial = _split(scheme)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    if spatial == DIL_EO:
        return (x + y + z) % 2
    if spatial == DIL_CUBE:
        return (x % 2) + 2 * (y % 2) + 4 * (z % 2)
    return np.zeros_like(t)


def dilute(xi, scheme, index):
    """Diluted piece ``index`` of a noise vector.

    Pieces are ordered t-major, then spin, colour, spatial class:
    index = ((t*4 + spin)*3 + colour) * n_spatial + class for TSC,
    (t*4 + spin) * n_spatial + class for TS, t * n_spatial + class for T and
    class alone without time dilution.  The pieces of one vector sum to it.
    """
    base, n_sp, _ = _split(scheme)
    dims = (xi.shape[3], xi.shape[2], xi.shape[1], xi.shape[0])
    b, cls = divmod(index, n_sp)
    keep = spatial_class(dims, scheme) == cls  # (Lt, Lz, Ly, Lx)
    out = np.zeros_like(xi)
    if base == DIL_NONE:
        out[keep] = xi[keep]
        return out
    if base == DIL_T:
        t = b
        out[t][keep[t]] = xi[t][keep[t]]
    elif base == DIL_TS:
        t, sp = divmod(b, 4)
        out[t, :, :, :, sp, :][keep[t]] = xi[t, :, :, :, sp, :][keep[t]]
    else:
        t, r = divmod(b, 12)
        sp, c = divmod(r, 3)
        out[t, :, :, :, sp, c][keep[t]] = xi[t, :, :, :, sp, c][keep[t]]
    return out


def diluted_sources(dims, seed, noise_index, scheme, stream=0):
    """All diluted pieces of noise vector ``noise_index``: (n_pieces, Lt, Lz, Ly, Lx, 4, 3)."""
    xi = z2_noise(dims, seed, noise_index, stream)
    n = dilution_count(dims, scheme)
    return np.stack([dilute(xi, scheme, i) for i in range(n)])
