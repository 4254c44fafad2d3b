"""GPU parity of the batched mixed-precision solver (FP16 / BF16 sloppy
spinors, FP16 reconstruct-12 links, FP32 arithmetic, FP32 reliable updates,
FP64 defect correction) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from lattice_inputs import haar_su3_field, eps_su3_field, gaussian_spinors
from oracle import dirac as od
from oracle.dense import dense_D, to_vec, from_vec
from oracle.solver import solve as osolve
from tests._gpu import lattice, to_dev, to_np, rel_err, torch

pytestmark = pytest.mark.gpu

PRECS = ["fp16", "bf16"]


@pytest.fixture(autouse=True, params=["0", "1", "4", "5", "7"], ids=["hop-ffma2", "hop-ffma2-capped", "hop-mma",
                                                                    "hop-tcgen05-tiles", "hop-ffma2-recon12"])
def hop_variant(request, monkeypatch):
    """Every test here runs with the FP32-unit pair hop (uncapped / register-capped,
    and register-capped with reconstruct-12 links), the mma.sync pair hop, and
    the RHS-tile solver with the tcgen05 hop (BF16 only; FP16 solves fall back
    to variant 1).  LQCD_HOP_VARIANT is read at solve setup."""
    monkeypatch.setenv("LQCD_HOP_VARIANT", request.param)
    return request.param


def _prec(L, name):
    return {"fp16": L.LQCD_PREC_MIXED_FP16, "bf16": L.LQCD_PREC_MIXED_BF16}[name]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims,kappa,seed", [((4, 4, 4, 4), 0.125, 0), ((6, 4, 2, 8), 0.13, 3)])
def test_mixed_matches_dense_lu(prec, dims, kappa, seed):
    U = haar_su3_field(dims, seed)
    n = 6
    b = gaussian_spinors(dims, n, 20 + seed)
    V = int(np.prod(dims))
    with lattice(dims, U, kappa) as (L, h):
        x = torch.empty((n, V, 4, 3), dtype=torch.complex128, device="cuda")
        rc, st = L.lqcd_solve_batch(h, to_dev(b.reshape(n, V, 4, 3)), x, L.solver_params(tol=1e-10, precision=_prec(L, prec)))
        got = to_np(x, dims)
    assert rc == 0, st
    ref = from_vec(np.linalg.solve(dense_D(U, kappa, dims), to_vec(b).T).T, dims)
    for k in range(n):
        r = np.linalg.norm((b[k] - od.apply_D(U, kappa, got[k])).ravel()) / np.linalg.norm(b[k].ravel())
        assert r <= 1e-10
        assert abs(r - st[k]["true_rel_residual"]) <= 1e-3 * r + 1e-17
        assert rel_err(got[k], ref[k]) < 1e-8


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_eps_field_against_oracle_solver(prec):
    dims = (8, 8, 8, 16)
    U = eps_su3_field(dims, 0.35, 1)
    kappa = 0.12
    n = 3
    b = gaussian_spinors(dims, n, 5)
    V = int(np.prod(dims))
    ref, info = osolve(U, kappa, b, tol=1e-12)
    with lattice(dims, U, kappa) as (L, h):
        x = torch.empty((n, V, 4, 3), dtype=torch.complex128, device="cuda")
        rc, st = L.lqcd_solve_batch(h, to_dev(b.reshape(n, V, 4, 3)), x, L.solver_params(tol=1e-10, precision=_prec(L, prec)))
        got = to_np(x, dims)
    assert rc == 0, st
    for k in range(n):
        assert st[k]["true_rel_residual"] <= 1e-10
        assert st[k]["reliable_updates"] >= 1
        assert rel_err(got[k], ref[k]) < 1e-8


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_batch_composition_is_bit_identical(prec):
    """A right-hand side's arithmetic does not depend on the others in its batch."""
    dims = (4, 4, 4, 8)
    U = eps_su3_field(dims, 0.35, 2)
    b = gaussian_spinors(dims, 5, 9).reshape(5, -1, 4, 3)
    with lattice(dims, U, 0.12) as (L, h):
        bd = to_dev(b)
        xa = torch.empty_like(bd)
        L.lqcd_solve_batch(h, bd, xa, L.solver_params(tol=1e-10, precision=_prec(L, prec)))
        xb = torch.empty_like(bd[2:3])
        L.lqcd_solve_batch(h, bd[2:3].contiguous(), xb, L.solver_params(tol=1e-10, precision=_prec(L, prec)))
        assert torch.equal(xa[2:3], xb)
        xc = torch.empty_like(bd)
        L.lqcd_solve_batch(h, bd, xc, L.solver_params(tol=1e-10, precision=_prec(L, prec), rhs_block=2))
        assert torch.equal(xa, xc)


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_low_precision_truncated_solve(prec):
    """TSM low-precision solves stop at 1e-3 (true FP64 residual), in far fewer iterations."""
    dims = (8, 8, 8, 16)
    U = eps_su3_field(dims, 0.35, 1)
    b = gaussian_spinors(dims, 2, 6).reshape(2, -1, 4, 3)
    with lattice(dims, U, 0.12) as (L, h):
        x = torch.empty_like(to_dev(b))
        rc, lp = L.lqcd_solve_batch(h, to_dev(b), x, L.solver_params(tol=1e-3, precision=_prec(L, prec)))
        assert rc == 0 and all(s["true_rel_residual"] <= 1e-3 for s in lp)
        rc, hp = L.lqcd_solve_batch(h, to_dev(b), x, L.solver_params(tol=1e-10, precision=_prec(L, prec)))
        assert rc == 0
        assert all(3 * a["iterations"] < c["iterations"] for a, c in zip(lp, hp))


def test_mixed_status_codes():
    dims = (4, 4, 4, 4)
    U = haar_su3_field(dims, 0)
    b = gaussian_spinors(dims, 3, 7).reshape(3, 256, 4, 3)
    b[1] = 0.0
    b[2, 5, 1, 1] = np.inf
    with lattice(dims, U, 0.125) as (L, h):
        x = torch.empty((3, 256, 4, 3), dtype=torch.complex128, device="cuda")
        rc, st = L.lqcd_solve_batch(h, to_dev(b), x, L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_FP16))
        assert st[0]["status"] == 0 and st[1]["status"] == 0
        assert torch.all(x[1] == 0)
        assert st[2]["status"] == L.LQCD_ERR_NONFINITE
        rc, st = L.lqcd_solve_batch(h, to_dev(b[:1]), x[:1],
                                    L.solver_params(tol=1e-10, max_iter=2, precision=L.LQCD_PREC_MIXED_FP16))
        assert rc == L.LQCD_ERR_NOT_CONVERGED
