"""GPU parity of the plane-staged pair hop (hop variant 6: a block takes one
(z, t) plane of output sites of one RHS pair and stages the five planes its
neighbours come from in shared memory), on lattices whose planes hold 128
sites of one parity (Lx Ly / 2 = 128).  Its arithmetic is that of the
register-capped pair hop (variant 1) term for term, so whole mixed-precision
solves must agree bit for bit; both are checked against the FP64 oracle."""
import pytest

from lattice_inputs import eps_su3_field, gaussian_spinors
from oracle.solver import solve as osolve
from tests._gpu import lattice, to_dev, to_np, rel_err, torch

pytestmark = pytest.mark.gpu


def _solve(L, h, bd, monkeypatch, variant):
    monkeypatch.setenv("LQCD_HOP_VARIANT", variant)
    x = torch.empty_like(bd)
    rc, st = L.lqcd_solve_batch(h, bd, x, L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_BF16))
    assert rc == 0, st
    assert all(s["true_rel_residual"] <= 1e-10 for s in st)
    return x, [s["iterations"] for s in st]


# (16,16,4,4): distinct z +- 1 planes; (16,16,2,6): z + 1 and z - 1 are the same
# plane; 5 and 3 right-hand sides leave the last pair with one member
@pytest.mark.parametrize("dims,n", [((16, 16, 4, 4), 5), ((16, 16, 2, 6), 3)])
def test_plane_staged_hop_solves_bit_identical_to_pair_hop(monkeypatch, dims, n):
    U = eps_su3_field(dims, 0.35, 4)
    b = gaussian_spinors(dims, n, 17)
    kappa = 0.12
    with lattice(dims, U, kappa) as (L, h):
        bd = to_dev(b.reshape(n, -1, 4, 3))
        x1, it1 = _solve(L, h, bd, monkeypatch, "1")
        x6, it6 = _solve(L, h, bd, monkeypatch, "6")
        got = to_np(x6, dims)
    assert it1 == it6
    assert torch.equal(x1, x6)
    ref, _ = osolve(U, kappa, b, tol=1e-12)
    for k in range(n):
        assert rel_err(got[k], ref[k]) < 1e-8


def test_plane_staged_variant_applies_only_where_planes_hold_128_sites(monkeypatch):
    """The override to variant 6 is reported (and launched) for BF16 on a lattice
    with Lx Ly / 2 = 128; elsewhere, and for FP16, the solver reports and
    launches the register-capped pair hop, variant 1, with the same results."""
    monkeypatch.setenv("LQCD_HOP_VARIANT", "6")
    for dims, fits in (((16, 16, 2, 4), True), ((8, 8, 2, 4), False), ((16, 8, 2, 4), False)):
        U = eps_su3_field(dims, 0.35, 5)
        b = gaussian_spinors(dims, 2, 19).reshape(2, -1, 4, 3)
        with lattice(dims, U, 0.12) as (L, h):
            assert L.lqcd_tuned_choice(h, 2, L.LQCD_PREC_MIXED_BF16)[1] == (6 if fits else 1)
            assert L.lqcd_tuned_choice(h, 2, L.LQCD_PREC_MIXED_FP16)[1] == 1
            bd = to_dev(b)
            x6, it6 = _solve(L, h, bd, monkeypatch, "6")
            x1, it1 = _solve(L, h, bd, monkeypatch, "1")
        assert it1 == it6 and torch.equal(x1, x6)
