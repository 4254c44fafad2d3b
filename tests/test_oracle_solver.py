"""Pins of the oracle's even-odd BiCGstab: dense LU (numpy.linalg.solve) and the true residual."""
import numpy as np
import pytest

from lattice_inputs import haar_su3_field, eps_su3_field, gaussian_spinors
from oracle import dirac
from oracle.dense import dense_D, to_vec, from_vec
from oracle.solver import solve


@pytest.mark.parametrize("dims,kappa,seed", [((2, 2, 2, 2), 0.125, 0), ((4, 4, 4, 4), 0.125, 0), ((4, 4, 4, 4), 0.157, 3)])
def test_solver_matches_dense_lu(dims, kappa, seed):
    U = haar_su3_field(dims, seed)
    b = gaussian_spinors(dims, 3, 100 + seed)
    x, info = solve(U, kappa, b, tol=1e-13)
    D = dense_D(U, kappa, dims)
    ref = from_vec(np.linalg.solve(D, to_vec(b).T).T, dims)
    rel = np.sqrt(dirac.norm2(x - ref) / dirac.norm2(ref))
    assert np.all(rel < 1e-11), rel
    assert np.all(info["true_rel_residual"] <= 1e-13)


def test_true_residual_definition_and_tolerance():
    dims = (4, 4, 4, 8)
    U = eps_su3_field(dims, 0.35, 1)
    b = gaussian_spinors(dims, 2, 7)
    for tol in (1e-3, 1e-8, 1e-10):
        x, info = solve(U, 0.12, b, tol=tol)
        r = np.sqrt(dirac.norm2(b - dirac.apply_D(U, 0.12, x)) / dirac.norm2(b))
        assert np.allclose(r, info["true_rel_residual"], rtol=1e-6)
        assert np.all(r <= tol)


def test_low_precision_needs_fewer_iterations():
    """The paper's observation (Sec. III): LP (1e-2) takes far fewer iterations than HP (1e-8)."""
    dims = (4, 4, 4, 8)
    U = eps_su3_field(dims, 0.35, 1)
    b = gaussian_spinors(dims, 1, 8)
    _, lp = solve(U, 0.12, b, tol=1e-2)
    _, hp = solve(U, 0.12, b, tol=1e-8)
    assert lp["iterations"][0] * 3 < hp["iterations"][0]
