"""Pins of the oracle's gamma matrices and Wilson-Dirac operator.

Each check is fixed by mathematics, not by the oracle itself: Clifford algebra,
gamma5-hermiticity, gauge covariance, the free-field momentum-space operator,
and an entry-by-entry dense construction.
"""
import numpy as np
import pytest

from lattice_inputs import haar_su3_field, unit_gauge_field, gaussian_spinors, random_gauge_transform
from oracle import dirac
from oracle.dense import dense_D, to_vec

DIMS = (4, 4, 4, 4)


def test_gamma_clifford_algebra():
    g = dirac.GAMMA
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=0)


def test_gamma5_is_chiral_diagonal():
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]), atol=0)
    for mu in range(4):
        assert np.allclose(dirac.GAMMA5 @ dirac.GAMMA[mu] + dirac.GAMMA[mu] @ dirac.GAMMA5, 0)


def test_gamma5_hermiticity():
    U = haar_su3_field(DIMS, 0)
    u, v = gaussian_spinors(DIMS, 2, 11)
    kappa = 0.137
    lhs = dirac.inner(u, dirac.apply_D(U, kappa, v))
    rhs = dirac.inner(dirac.spin_mul(dirac.GAMMA5, dirac.apply_D(U, kappa, dirac.spin_mul(dirac.GAMMA5, u))), v)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # and D itself is not Hermitian (the check has teeth)
    herm = dirac.inner(dirac.apply_D(U, kappa, u), v)
    assert abs(lhs - herm) > 1e-3 * abs(lhs)


def test_gauge_covariance():
    U = haar_su3_field(DIMS, 3)
    g = random_gauge_transform(DIMS, 4)
    axis = (3, 2, 1, 0)
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=axis[mu])
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    psi = gaussian_spinors(DIMS, 1, 5)[0]
    gpsi = np.einsum("...ab,...sb->...sa", g, psi)
    lhs = dirac.apply_D(Ug, 0.11, gpsi)
    rhs = np.einsum("...ab,...sb->...sa", g, dirac.apply_D(U, 0.11, psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-13
    # plaquette is gauge invariant
    assert abs(dirac.plaquette(Ug) - dirac.plaquette(U)) < 1e-14


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (3, 1, 1, 2)])
def test_free_field_plane_waves(n):
    dims = (4, 6, 4, 8)
    lx, ly, lz, lt = dims
    kappa = 0.13
    U = unit_gauge_field(dims)
    p = np.array([2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz, (2 * n[3] + 1) * np.pi / lt])
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    rng = np.random.default_rng(9)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi = phase[..., None, None] * u
    Dp = (1 - 2 * kappa * np.sum(np.cos(p))) * np.eye(4) + 2j * kappa * sum(dirac.GAMMA[m] * np.sin(p[m]) for m in range(4))
    expect = phase[..., None, None] * (Dp @ u)
    got = dirac.apply_D(U, kappa, psi)
    assert np.max(np.abs(got - expect)) < 1e-13


def test_dense_matches_stencil():
    dims = (2, 2, 2, 4)
    U = haar_su3_field(dims, 7)
    psi = gaussian_spinors(dims, 1, 8)[0]
    D = dense_D(U, 0.15, dims)
    assert np.max(np.abs(D @ to_vec(psi) - to_vec(dirac.apply_D(U, 0.15, psi)))) < 1e-13


def test_plaquette_unit_and_haar():
    assert abs(dirac.plaquette(unit_gauge_field(DIMS)) - 1.0) < 1e-15
    # Haar links: <Re Tr U_p>/3 = 0, fluctuation ~ 1/sqrt(18 V)
    assert abs(dirac.plaquette(haar_su3_field((8, 8, 8, 8), 0))) < 0.02


def test_schur_complement_identity():
    """D x = b with x_o reconstructed solves the full system iff D_hat x_e = b_hat_e."""
    U = haar_su3_field(DIMS, 1)
    kappa = 0.12
    masks = dirac.parity_masks(DIMS)
    even, odd = masks
    x = gaussian_spinors(DIMS, 1, 2)[0]
    b = dirac.apply_D(U, kappa, x)
    b_hat = dirac.prepare_source(U, kappa, b, masks)
    assert np.max(np.abs(dirac.schur_apply(U, kappa, even * x, masks) - b_hat)) < 1e-12
    assert np.max(np.abs(dirac.reconstruct_odd(U, kappa, even * x, b, masks) - x)) < 1e-12
