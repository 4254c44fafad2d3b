"""Edge cases through the C ABI: empty inputs at every entry point, and the
degenerate operator kappa = 0 (D = 1, so the solution is the source itself in
every precision)."""
import numpy as np
import pytest

from lattice_inputs import haar_su3_field, gaussian_spinors
from tests._gpu import lattice, to_dev, to_np, rel_err, torch

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
V = 256


def test_empty_inputs_are_no_ops():
    U = haar_su3_field(DIMS, 1)
    with lattice(DIMS, U, 0.12) as (L, h):
        empty = torch.empty((0, V, 4, 3), dtype=torch.complex128, device="cuda")
        for prec in (L.LQCD_PREC_FP64, L.LQCD_PREC_MIXED_BF16, L.LQCD_PREC_MIXED_FP16):
            rc, st = L.lqcd_solve_batch(h, empty, empty, L.solver_params(precision=prec))
            assert rc == 0 and st == []
        ps = torch.full((V, 6), 3.0 + 1j, dtype=torch.complex128, device="cuda")
        pt = torch.full((DIMS[3], 6), 2.0, dtype=torch.complex128, device="cuda")
        L.lqcd_loops_batch(h, empty, empty, 1.0, ps, pt)
        assert torch.all(ps == 3.0 + 1j) and torch.all(pt == 2.0)
        L.lqcd_noise_generate(1, 0, 0, DIMS, L.LQCD_DILUTE_TSC, 0, 0, empty)
        L.lqcd_apply_dirac(h, empty, torch.empty_like(empty), False)
        L.lqcd_point_sources(h, [], empty)
        out = torch.empty((0, DIMS[3], 6), dtype=torch.complex128, device="cuda")
        L.lqcd_loops_momentum(h, ps, [], out)
        L.lqcd_smear_gaussian(h, empty, torch.empty_like(empty), 4.0, 3)
        dU = torch.zeros(V * 36, dtype=torch.complex128, device="cuda")
        dk, rc, st = L.lqcd_gradient(h, empty, empty, np.zeros((DIMS[3], 6)), L.solver_params(), 1.0, dU)
        assert rc == 0 and dk == 0.0 and st == [] and torch.all(dU == 0)
        # no noise vectors to correlate, or a batch too small for the unbiased estimator
        one = torch.zeros((1, DIMS[3], 6), dtype=torch.complex128, device="cuda")
        D = torch.empty((DIMS[3], 6, 6), dtype=torch.complex128, device="cuda")
        with pytest.raises(L.LqcdError):
            L.lqcd_disconnected_correlator(one, one, 64, D, True)
        with pytest.raises(L.LqcdError):
            L.lqcd_autotune(h, 0, L.LQCD_PREC_MIXED_BF16)


@pytest.mark.parametrize("prec", ["fp64", "bf16", "fp16"])
def test_kappa_zero_solution_is_the_source(prec):
    U = haar_su3_field(DIMS, 2)
    b = gaussian_spinors(DIMS, 3, 3).reshape(3, V, 4, 3)
    with lattice(DIMS, U, 0.0) as (L, h):
        p = {"fp64": L.LQCD_PREC_FP64, "bf16": L.LQCD_PREC_MIXED_BF16, "fp16": L.LQCD_PREC_MIXED_FP16}[prec]
        x = torch.empty((3, V, 4, 3), dtype=torch.complex128, device="cuda")
        rc, st = L.lqcd_solve_batch(h, to_dev(b), x, L.solver_params(tol=1e-10, precision=p))
        got = x.cpu().numpy()
    assert rc == 0
    assert rel_err(got, b) <= 1e-10
    # On D = 1 a sloppy iteration is exact up to rounding the direction to the
    # sloppy type, so each one cuts the residual by about 2^-p (p = 8 significand
    # bits for BF16, 11 for FP16): 1e-10 = 2^-33.2 takes ceil(33.2 / p) of them.
    max_it = {"fp64": 4, "bf16": 5, "fp16": 4}[prec]
    assert all(s["true_rel_residual"] <= 1e-10 and s["iterations"] <= max_it for s in st)
