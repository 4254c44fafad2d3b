"""Pins of the oracle's gradients (adjoint solves with D^+ = gamma5 D gamma5).

* the noise estimator with a complete basis of unit sources (every (x, spin,
  colour)) equals the dense reference exactly;
* central finite differences (h = 1e-5) of the oracle's own loop estimator in
  kappa and along su(3) directions of single links.
"""
import numpy as np
import pytest

from lattice_inputs import haar_su3_field, gaussian_weights
from oracle import gradient as gr
from oracle.dirac import spin_mul, GAMMA5
from oracle.philox import diluted_sources, DIL_TSC
from oracle.solver import solve

DIMS = (2, 2, 2, 2)


def _unit_basis(dims):
    lx, ly, lz, lt = dims
    n = 12 * lx * ly * lz * lt
    e = np.eye(n, dtype=np.complex128)
    return e.reshape(n, lt, lz, ly, lx, 4, 3)


@pytest.mark.parametrize("gamma_index", [0, 1, 5])
def test_dkappa_complete_basis_equals_dense(gamma_index):
    U = haar_su3_field(DIMS, 0)
    kappa = 0.13
    est = gr.dkappa_estimator(U, kappa, _unit_basis(DIMS), gamma_index, tol=1e-13)
    ref = gr.dense_dkappa(U, kappa, gamma_index)
    assert abs(est - ref) < 1e-9 * max(1.0, abs(ref))


def test_link_grad_complete_basis_equals_dense():
    U = haar_su3_field(DIMS, 1)
    kappa = 0.13
    w = gaussian_weights(DIMS[3], 2)
    est = gr.link_grad_estimator(U, kappa, _unit_basis(DIMS), w, tol=1e-13)
    ref = gr.dense_link_grad(U, kappa, w)
    assert np.max(np.abs(est - ref)) < 1e-9


def test_dkappa_finite_difference():
    dims = (2, 2, 2, 4)
    U = haar_su3_field(dims, 3)
    kappa = 0.12
    src = diluted_sources(dims, 11, 0, DIL_TSC)
    h = 1e-5
    for g in (0, 5):
        fp = gr.loop_sum_estimator(U, kappa + h, src, g, tol=1e-14)
        fm = gr.loop_sum_estimator(U, kappa - h, src, g, tol=1e-14)
        fd = (fp - fm) / (2 * h)
        an = gr.dkappa_estimator(U, kappa, src, g, tol=1e-14)
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_link_grad_finite_difference():
    dims = (2, 2, 2, 4)
    U = haar_su3_field(dims, 4)
    kappa = 0.12
    w = gaussian_weights(dims[3], 2)
    src = diluted_sources(dims, 12, 0, DIL_TSC)
    g = gr.link_grad_estimator(U, kappa, src, w, tol=1e-14)
    T = gr.su3_generators()
    h = 1e-5
    for (site, mu) in (((0, 0, 0, 0), 0), ((3, 1, 0, 1), 3), ((1, 1, 1, 0), 2)):
        F = gr.lie_derivative(U, g, site, mu)
        for a in (0, 2, 7):
            def S(eps):
                Up = U.copy()
                t, z, y, x = site
                w_, v_ = np.linalg.eigh(-1j * T[a])  # T = i H_a, exp(eps T) via H_a's eigenbasis
                Up[t, z, y, x, mu] = (v_ * np.exp(1j * eps * w_)) @ v_.conj().T @ U[t, z, y, x, mu]
                return gr.weighted_loop_estimator(Up, kappa, src, w, tol=1e-14)
            fd = (S(h) - S(-h)) / (2 * h)
            assert abs(fd - F[a]) < 1e-6 * max(1.0, abs(F[a])), (site, mu, a, fd, F[a])


def test_weighted_loop_complete_basis_equals_dense():
    U = haar_su3_field(DIMS, 5)
    w = gaussian_weights(DIMS[3], 2)
    est = gr.weighted_loop_estimator(U, 0.13, _unit_basis(DIMS), w, tol=1e-13)
    assert abs(est - gr.dense_weighted_loop(U, 0.13, w)) < 1e-10
