"""Pins of the oracle's Philox4x64-10 and complex Z2 noise.

numpy.random.Philox is an independent implementation of the same generator;
its raw output block i is Philox(counter + i + 1, key).
"""
import numpy as np
import pytest

from oracle.philox import (philox4x64_10, z2_noise, diluted_sources, dilution_count, DIL_TSC, DIL_TS, DIL_T,
                           DIL_NONE, DIL_EO, DIL_CUBE, SQRT1_2)


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((1, 2), (5, 0, 0, 0)),
                                     ((0xDEADBEEFCAFEF00D, 0x0123456789ABCDEF), (2**64 - 3, 17, 2**63, 99)),
                                     ((2**64 - 1, 2**64 - 1), (2**64 - 2, 2**64 - 1, 2**64 - 1, 2**64 - 1))])
def test_philox_matches_numpy(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    raw = bg.random_raw(8)
    c = list(ctr)
    for blk in range(2):
        # numpy increments the 256-bit counter before producing each block
        v = (c[0] + c[1] * 2**64 + c[2] * 2**128 + c[3] * 2**192 + blk + 1) % 2**256
        cc = [(v >> (64 * k)) & (2**64 - 1) for k in range(4)]
        out = philox4x64_10(tuple(np.uint64(x) for x in cc), tuple(np.uint64(k) for k in key))
        assert [int(o) for o in out] == [int(r) for r in raw[4 * blk:4 * blk + 4]]


def test_philox_vectorised_equals_scalar():
    sites = np.arange(50, dtype=np.uint64)
    w = philox4x64_10((sites, np.uint64(3), np.uint64(0), np.uint64(0)), (np.uint64(42), np.uint64(1)))
    for s in (0, 7, 49):
        ws = philox4x64_10((np.uint64(s), np.uint64(3), np.uint64(0), np.uint64(0)), (np.uint64(42), np.uint64(1)))
        assert all(int(a[s]) == int(b) for a, b in zip(w, ws))


def test_z2_values_and_bits():
    dims = (4, 2, 2, 2)
    xi = z2_noise(dims, 1234, 5, 0)
    assert np.all(np.abs(np.abs(xi.real) - SQRT1_2) == 0) and np.all(np.abs(np.abs(xi.imag) - SQRT1_2) == 0)
    assert np.all(np.abs(xi) ** 2 - 1.0 < 1e-15)
    # site 0, component k: bit 2k of word 0 -> sign of Re
    w0 = int(philox4x64_10((np.uint64(0), np.uint64(5), np.uint64(0), np.uint64(0)), (np.uint64(1234), np.uint64(0)))[0])
    flat = xi.reshape(-1, 12)
    for k in range(12):
        assert (flat[0, k].real < 0) == bool((w0 >> (2 * k)) & 1)
        assert (flat[0, k].imag < 0) == bool((w0 >> (2 * k + 1)) & 1)


def test_z2_moments():
    """<xi> ~ 0 and <xi xi^*> ~ delta (Sec. II, Eq. delta functions), as z-tests."""
    dims = (4, 4, 4, 4)
    n = 64
    xs = np.stack([z2_noise(dims, 77, r, 0).reshape(-1) for r in range(n)])  # (n, 3072)
    mean = xs.mean(axis=0)
    # each component: Re and Im are +-1/sqrt(2) with prob 1/2 -> std of mean = 1/sqrt(2n)
    z = np.abs(mean.real) * np.sqrt(2 * n)
    assert np.mean(z) < 1.0  # E|N(0,1)| = 0.80
    corr = (xs.conj().T @ xs) / n
    assert np.allclose(np.diag(corr), 1.0, atol=1e-15)
    off = corr - np.diag(np.diag(corr))
    # off-diagonal |<xi_i^* xi_j>| ~ 1/sqrt(n)
    assert np.sqrt(np.mean(np.abs(off) ** 2)) < 1.2 / np.sqrt(n)
    # distinct streams differ
    assert not np.array_equal(z2_noise(dims, 77, 0, 0), z2_noise(dims, 77, 0, 1))


@pytest.mark.parametrize("scheme", [DIL_NONE, DIL_T, DIL_TS, DIL_TSC, DIL_EO, DIL_T | DIL_EO, DIL_TS | DIL_CUBE,
                                    DIL_TSC | DIL_EO, DIL_TSC | DIL_CUBE, DIL_CUBE])
def test_dilution_partition(scheme):
    dims = (2, 2, 2, 4)
    src = diluted_sources(dims, 9, 2, scheme)
    assert src.shape[0] == dilution_count(dims, scheme)
    assert np.array_equal(src.sum(axis=0), z2_noise(dims, 9, 2, 0))
    # pieces are disjoint
    nz = (np.abs(src) > 0).sum(axis=0)
    assert nz.max() == 1


def test_spatial_dilution_classes():
    """Even-odd: neighbouring spatial sites fall in different pieces; cubic: each
    piece holds exactly one vertex of every elementary 2^3 cube (Sec. II)."""
    dims = (4, 4, 4, 2)
    lx, ly, lz, lt = dims
    eo = diluted_sources(dims, 3, 0, DIL_T | DIL_EO)
    assert eo.shape[0] == 2 * lt
    for k in range(eo.shape[0]):
        t, cls = divmod(k, 2)
        support = np.abs(eo[k]).sum(axis=(-1, -2)) > 0  # (Lt, Lz, Ly, Lx)
        assert support.sum() == lx * ly * lz // 2
        assert support[t].sum() == support.sum()
        zz, yy, xx = np.nonzero(support[t])
        assert np.all((xx + yy + zz) % 2 == cls)
        # no two sites of a piece are nearest spatial neighbours
        for ax in range(3):
            assert not np.any(support[t] & np.roll(support[t], 1, axis=ax))
    cube = diluted_sources(dims, 3, 0, DIL_CUBE)
    assert cube.shape[0] == 8
    for k in range(8):
        support = np.abs(cube[k]).sum(axis=(-1, -2)) > 0
        for t in range(lt):
            for z0 in range(0, lz, 2):
                for y0 in range(0, ly, 2):
                    for x0 in range(0, lx, 2):
                        blk = support[t, z0:z0 + 2, y0:y0 + 2, x0:x0 + 2]
                        assert blk.sum() == 1
                        zz, yy, xx = np.nonzero(blk)
                        assert xx[0] + 2 * yy[0] + 4 * zz[0] == k


def test_spatial_dilution_counts():
    dims = (4, 4, 4, 6)
    assert dilution_count(dims, DIL_TSC | DIL_EO) == 12 * 6 * 2
    assert dilution_count(dims, DIL_TSC | DIL_CUBE) == 12 * 6 * 8
    assert dilution_count(dims, DIL_EO) == 2
    with pytest.raises(ValueError):
        dilution_count(dims, DIL_EO | DIL_CUBE)


def _golden_words():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x64_words.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    return [tuple(int(v) for v in r) for r in rows]


def test_philox_golden_words():
    """Stored words of numpy's independent Philox4x64-10 (tests/golden) for the
    noise generator's key / counter convention."""
    rows = _golden_words()
    assert len(rows) >= 10
    for seed, stream, ni, site, *w in rows:
        out = philox4x64_10((np.uint64(site), np.uint64(ni), np.uint64(0), np.uint64(0)),
                            (np.uint64(seed), np.uint64(stream)))
        assert [int(o) for o in out] == w
