"""The spin algebra behind the link-gradient kernel's half-spinor outer products,
checked on the CPU against the oracle's DeGrand-Rossi gamma matrices.

The kernel forms X = sum chi^+ (1 - gamma_mu) phi and Y = sum chi^+ (1 + gamma_mu) phi
from the upper two spin components h(v) = [(1 + S gamma_mu) v]_{0,1} of both
spinors.  That is exact because (1 + S gamma_mu) / 2 is a Hermitian projector
whose lower two rows are a phase times a swap of its upper two.  The kernel's
table of the upper rows of gamma_mu (in terms of v_2, v_3) is restated here and
compared with the gamma matrices entry by entry.
"""
import numpy as np
import pytest

from oracle import dirac

# upper two rows of gamma_mu as used by the kernel: (gamma_mu v)_0, (gamma_mu v)_1
# = c00 v_2 + c01 v_3, c10 v_2 + c11 v_3
KERNEL_UPPER_ROWS = {
    0: ((0, 1j), (1j, 0)),
    1: ((0, -1), (1, 0)),
    2: ((1j, 0), (0, -1j)),
    3: ((1, 0), (0, 1)),
}


@pytest.mark.parametrize("mu", range(4))
def test_kernel_upper_rows_match_gamma(mu):
    g = dirac.GAMMA[mu]
    assert np.array_equal(g[:2, :2], np.zeros((2, 2)))  # upper rows touch only v_2, v_3
    assert np.array_equal(g[:2, 2:], np.array(KERNEL_UPPER_ROWS[mu], dtype=np.complex128))


@pytest.mark.parametrize("mu", range(4))
@pytest.mark.parametrize("sign", (-1, 1))
def test_half_spinor_outer_product_identity(mu, sign):
    rng = np.random.default_rng(10 * mu + (sign > 0))
    chi = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    phi = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    P = np.eye(4) + sign * dirac.GAMMA[mu]
    # projector: (P / 2)^2 = P / 2, Hermitian
    assert np.allclose((P / 2) @ (P / 2), P / 2, atol=1e-15)
    assert np.array_equal(P, P.conj().T)
    full = np.einsum("ai,ab,bj->ij", chi.conj(), P, phi)  # colour matrix chi^+ P phi
    hc, hp = (P @ chi)[:2], (P @ phi)[:2]
    half = np.einsum("ai,aj->ij", hc.conj(), hp)
    assert np.allclose(full, half, rtol=0, atol=1e-13)
    # projecting phi alone is not enough (the check has teeth)
    assert not np.allclose(full, np.einsum("ai,aj->ij", chi[:2].conj(), hp), atol=1e-6)
