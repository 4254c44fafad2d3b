"""GPU parity of the adjoint-solve gradient (lqcd_gradient, LoopsFn) against
the oracle: dense references with a complete basis of unit sources, the
oracle's noise estimator with the same noise, torch.autograd.gradcheck, and
central finite differences (h = 1e-5) at the full 16^3 x 32 size."""
import numpy as np
import pytest

from lattice_inputs import haar_su3_field, eps_su3_field, gaussian_weights
from oracle import gradient as gr
from oracle.philox import diluted_sources, DIL_TSC
from tests._gpu import lattice, to_dev, rel_err, torch

pytestmark = pytest.mark.gpu


def _unit_basis(dims):
    V = int(np.prod(dims))
    n = 12 * V
    return np.eye(n, dtype=np.complex128).reshape(n, V, 4, 3)


def _coef_gamma(lt, g):
    c = np.zeros((lt, 6), dtype=np.complex128)
    c[:, g] = 1.0
    return c


def _coef_weights(w):
    c = np.zeros((len(w), 6), dtype=np.complex128)
    c[:, 0] = w
    return c


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (4, 4, 4, 4)])
def test_gradient_complete_basis_matches_dense(dims):
    U = haar_su3_field(dims, 1)
    kappa = 0.13
    V = int(np.prod(dims))
    src = _unit_basis(dims)
    w = gaussian_weights(dims[3], 2)
    with lattice(dims, U, kappa) as (L, h):
        s = to_dev(src)
        x = torch.empty_like(s)
        p = L.solver_params(tol=1e-13, precision=L.LQCD_PREC_FP64, rhs_block=len(src))
        rc, _ = L.lqcd_solve_batch(h, s, x, p)
        assert rc == 0
        for g in (0, 5):
            dk, rc, _ = L.lqcd_gradient(h, s, x, _coef_gamma(dims[3], g), p)
            assert rc == 0
            ref = gr.dense_dkappa(U, kappa, g)
            assert abs(dk - ref.real) < 1e-9 * max(1.0, abs(ref))
        dU = torch.zeros(V * 36, dtype=torch.complex128, device="cuda")
        dk, rc, _ = L.lqcd_gradient(h, s, x, _coef_weights(w), p, 1.0, dU)
        got = dU.cpu().numpy().reshape(U.shape)
    ref = gr.dense_link_grad(U, kappa, w)
    assert np.max(np.abs(got - ref)) < 1e-9 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("prec", ["fp64", "fp16", "bf16"])
def test_gradient_noise_matches_oracle_estimator(prec):
    dims = (4, 4, 4, 4)
    U = eps_su3_field(dims, 0.35, 3)
    kappa = 0.12
    V = 256
    src = diluted_sources(dims, 77, 0, DIL_TSC)  # 48 pieces
    w = gaussian_weights(dims[3], 2)
    with lattice(dims, U, kappa) as (L, h):
        pr = {"fp64": L.LQCD_PREC_FP64, "fp16": L.LQCD_PREC_MIXED_FP16, "bf16": L.LQCD_PREC_MIXED_BF16}[prec]
        p = L.solver_params(tol=1e-11, precision=pr, rhs_block=48)
        s = to_dev(src.reshape(48, V, 4, 3))
        x = torch.empty_like(s)
        assert L.lqcd_solve_batch(h, s, x, p)[0] == 0
        dk1, rc, _ = L.lqcd_gradient(h, s, x, _coef_gamma(4, 0), p)
        dk5, rc, _ = L.lqcd_gradient(h, s, x, _coef_gamma(4, 5), p)
        dU = torch.zeros(V * 36, dtype=torch.complex128, device="cuda")
        L.lqcd_gradient(h, s, x, _coef_weights(w), p, 1.0, dU)
        got = dU.cpu().numpy().reshape(U.shape)
    ref1 = gr.dkappa_estimator(U, kappa, src, 0, tol=1e-13)
    ref5 = gr.dkappa_estimator(U, kappa, src, 5, tol=1e-13)
    assert abs(dk1 - ref1.real) < 1e-8 * abs(ref1)
    assert abs(dk5 - ref5.real) < 1e-8 * max(abs(ref5), abs(ref1))
    ref = gr.link_grad_estimator(U, kappa, src, w, tol=1e-13)
    assert rel_err(got, ref) < 1e-8


def test_loopsfn_gradcheck_fp64():
    from paper_1108_2473_gb300.autograd import Lattice, loops
    from tests._gpu import require_gpu
    L = require_gpu()
    dims = (2, 2, 2, 4)
    V = 32
    U0 = haar_su3_field(dims, 4)
    src = diluted_sources(dims, 5, 0, DIL_TSC)[:12]  # time slice 0 pieces
    lat = Lattice(dims, 0)
    try:
        U = torch.from_numpy(U0.reshape(V, 4, 3, 3)).cuda().requires_grad_(True)
        kappa = torch.tensor(0.12, dtype=torch.float64, device="cuda", requires_grad=True)
        s = to_dev(src.reshape(12, V, 4, 3))
        p = L.solver_params(tol=1e-14, precision=L.LQCD_PREC_FP64)

        def f(U_, k_):
            return loops(U_, k_, lat, s, p, True)

        assert torch.autograd.gradcheck(f, (U, kappa), eps=1e-6, atol=1e-6, rtol=1e-4, fast_mode=True)
    finally:
        lat.close()


def test_loopsfn_full_size_mixed_vs_finite_differences():
    """16^3 x 32, eps = 0.35, kappa = 0.120, mixed FP16: d/dkappa of sum_x Tr[G] and
    Im sum_x Tr[g4 G] and a link derivative of Re sum_t w_t L_1(t) against central
    differences (h = 1e-5) of FP64 forward solves."""
    from paper_1108_2473_gb300.autograd import Lattice, loops
    from paper_1108_2473_gb300 import lqcd as L
    dims = (16, 16, 16, 32)
    V = int(np.prod(dims))
    Un = eps_su3_field(dims, 0.35, 1)
    w = torch.from_numpy(gaussian_weights(dims[3], 2)).cuda()
    lat = Lattice(dims, 0)
    try:
        n = 24  # pieces of time slices 0 and 1
        s = torch.empty((n, V, 4, 3), dtype=torch.complex128, device="cuda")
        L.lqcd_noise_generate(99, 0, 0, dims, L.LQCD_DILUTE_TSC, 0, n, s)
        pm = L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_FP16)
        p64 = L.solver_params(tol=1e-13, precision=L.LQCD_PREC_FP64, rhs_block=n)
        U = torch.from_numpy(Un.reshape(V, 4, 3, 3)).cuda().requires_grad_(True)
        kappa = torch.tensor(0.120, dtype=torch.float64, device="cuda", requires_grad=True)
        Lt = loops(U, kappa, lat, s, pm)
        loss = (Lt[:, 0].real * w).sum() + Lt[:, 5].imag.sum()
        loss.backward()
        h = 1e-5

        def loss64(Uv, kv):
            with torch.no_grad():
                l = loops(Uv, torch.tensor(kv, dtype=torch.float64, device="cuda"), lat, s, p64)
            return float(((l[:, 0].real * w).sum() + l[:, 5].imag.sum()).item())

        fd = (loss64(U.detach(), 0.120 + h) - loss64(U.detach(), 0.120 - h)) / (2 * h)
        assert abs(kappa.grad.item() - fd) < 1e-5 * abs(fd)
        # one link, along T = i lambda_3 / 2 (stays in SU(3))
        site, mu = 1234, 3
        T = torch.zeros((3, 3), dtype=torch.complex128, device="cuda")
        T[0, 0], T[1, 1] = 0.5j, -0.5j
        g = U.grad[site, mu]
        analytic = torch.real(torch.sum(torch.conj(g) * (T @ U.detach()[site, mu]))).item()

        def moved(e):
            Um = U.detach().clone()
            Um[site, mu] = torch.linalg.matrix_exp(e * T) @ Um[site, mu]
            return loss64(Um, 0.120)

        fdl = (moved(h) - moved(-h)) / (2 * h)
        assert abs(analytic - fdl) < 1e-4 * abs(fdl) + 1e-9
    finally:
        lat.close()


def test_dkappa_full_size_mixed_matches_oracle_sample():
    """16^3 x 32, eps = 0.35, kappa = 0.120: d/dkappa of sum_x Tr[G] and of
    sum_x Tr[g4 G] (real and imaginary parts) from the mixed-precision adjoint
    solves of two t+s+c-diluted pieces, against the oracle's estimator for the
    same pieces solved to 1e-12 (four spawned oracle processes)."""
    import multiprocessing as mp
    from tests import _oracle_pool
    from oracle.philox import DIL_TSC
    from paper_1108_2473_gb300 import lqcd as L
    dims = (16, 16, 16, 32)
    V = int(np.prod(dims))
    kappa = 0.120
    pieces = [12 * 3 + 1, 12 * 17 + 8]
    jobs = [(dims, 0.35, 1, kappa, 99, 0, DIL_TSC, pc, g, 1e-12) for g in (0, 5) for pc in pieces]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        pending = pool.map_async(_oracle_pool.dkappa_piece, jobs)
        U = eps_su3_field(dims, 0.35, 1)
        with lattice(dims, U, kappa) as (L, h):
            s = torch.empty((len(pieces), V, 4, 3), dtype=torch.complex128, device="cuda")
            for k, pc in enumerate(pieces):
                L.lqcd_noise_generate(99, 0, 0, dims, L.LQCD_DILUTE_TSC, pc, 1, s[k:k + 1])
            p = L.solver_params(tol=1e-11, precision=L.LQCD_PREC_MIXED_BF16)
            x = torch.empty_like(s)
            assert L.lqcd_solve_batch(h, s, x, p)[0] == 0
            got = {}
            for g in (0, 5):
                c = _coef_gamma(dims[3], g)
                dre, rc1, _ = L.lqcd_gradient(h, s, x, c, p)
                dim, rc2, _ = L.lqcd_gradient(h, s, x, 1j * c, p)
                assert rc1 == 0 and rc2 == 0
                got[g] = complex(dre, dim)
        ref = pending.get(timeout=1800)
    ref1 = ref[0] + ref[1]
    ref4 = ref[2] + ref[3]
    assert abs(got[0] - ref1) < 1e-8 * abs(ref1)
    assert abs(got[5] - ref4) < 1e-8 * max(abs(ref4), abs(ref1))
