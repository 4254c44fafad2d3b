"""Writes the golden fixtures of this directory.  Run from the repository root:

    python tests/golden/make_golden.py

Neither fixture comes from the GPU library:

* free_field_loops.txt -- the free-field loop per site, Tr G(x;x) with G = D^{-1} for
  U = 1, from its closed form: a momentum sum of the free Wilson propagator (periodic
  space, antiperiodic time), (12 / V) sum_p M / (M^2 + 4 kappa^2 sum_mu sin^2 p_mu)
  with M = 1 - 2 kappa sum_mu cos p_mu.  The gamma5 and gamma_mu loops vanish.
* philox4x64_words.txt -- output words of Philox4x64-10 (Salmon, Moraes, Dror, Shaw,
  SC'11) taken from numpy.random.Philox, an implementation independent of this
  repository, for the keys and counters the noise generator uses: key = (seed,
  stream), counter = (site, noise index, 0, 0).  numpy advances its 256-bit counter
  by one before each block, so the block for counter c is requested at c - 1.
"""
import itertools
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

FREE_CASES = [((4, 4, 4, 4), 0.125), ((4, 4, 4, 4), 0.1), ((6, 4, 4, 8), 0.12), ((2, 2, 2, 4), 0.13)]
PHILOX_CASES = [(0xC0FFEE, 0, 5, [0, 1, 2, 255, 1000]), (0xC0FFEE, 1, 5, [0, 17]), (1, 0, 0, [0, 1, 131071]),
                (12345678901234567, 1, 3, [42, 65535])]


def free_trace(dims, kappa):
    lx, ly, lz, lt = dims
    acc = 0.0
    for n in itertools.product(range(lx), range(ly), range(lz), range(lt)):
        p = np.array([2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
                      (2 * n[3] + 1) * np.pi / lt])
        m = 1.0 - 2.0 * kappa * np.cos(p).sum()
        acc += 12.0 * m / (m * m + 4.0 * kappa * kappa * (np.sin(p) ** 2).sum())
    return acc / (lx * ly * lz * lt)


def philox_word(seed, stream, noise_index, site):
    ctr = (site + (noise_index << 64)) - 1  # numpy increments before producing the block
    ctr %= 2 ** 256
    c = np.array([(ctr >> (64 * k)) & (2 ** 64 - 1) for k in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array([seed, stream], dtype=np.uint64), counter=c)
    return [int(v) for v in bg.random_raw(4)]


def main():
    with open(os.path.join(HERE, "free_field_loops.txt"), "w") as f:
        f.write("# Tr G(x;x) per site of the free Wilson operator D = 1 - kappa H (G = D^-1),\n")
        f.write("# periodic in space, antiperiodic in time; closed-form momentum sum (make_golden.py).\n")
        f.write("# Lx Ly Lz Lt kappa trace\n")
        for dims, kappa in FREE_CASES:
            f.write("%d %d %d %d %.6f %.17g\n" % (*dims, kappa, free_trace(dims, kappa)))
    with open(os.path.join(HERE, "philox4x64_words.txt"), "w") as f:
        f.write("# Philox4x64-10 output words from numpy.random.Philox (independent implementation).\n")
        f.write("# key = (seed, stream), counter = (site, noise_index, 0, 0)\n")
        f.write("# seed stream noise_index site w0 w1 w2 w3\n")
        for seed, stream, ni, sites in PHILOX_CASES:
            for s in sites:
                w = philox_word(seed, stream, ni, s)
                f.write("%d %d %d %d %d %d %d %d\n" % (seed, stream, ni, s, *w))


if __name__ == "__main__":
    main()
