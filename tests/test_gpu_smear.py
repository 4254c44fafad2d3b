"""GPU parity of the smearing kernels (lqcd_smear_ape, lqcd_smear_gaussian)
against the oracle (oracle/smear.py), through the C ABI."""
import numpy as np
import pytest

from lattice_inputs import eps_su3_field, haar_su3_field, gaussian_spinors
from oracle import smear as osm
from tests._gpu import lattice, to_dev, to_np, rel_err, torch

pytestmark = pytest.mark.gpu

DIMS = (4, 6, 4, 4)


@pytest.mark.parametrize("alpha,n", [(0.5, 1), (0.5, 4), (0.2, 7)])
def test_ape_matches_oracle(alpha, n):
    U = eps_su3_field(DIMS, 0.5, 3)
    V = int(np.prod(DIMS))
    with lattice(DIMS, U, 0.12) as (L, h):
        out = torch.empty(V * 36, dtype=torch.complex128, device="cuda")
        L.lqcd_smear_ape(h, alpha, n, out)
        got = out.cpu().numpy().reshape(U.shape)
    ref = osm.ape_smear(U, alpha, n)
    assert np.max(np.abs(got - ref)) < 1e-12
    assert np.array_equal(got[..., 3, :, :], U[..., 3, :, :])


@pytest.mark.parametrize("alpha,n,normalise,ape", [(0.7, 3, False, False), (4.0, 5, True, False),
                                                   (4.0, 50, True, True), (4.0, 6, False, True)])
def test_gaussian_matches_oracle(alpha, n, normalise, ape):
    U = haar_su3_field(DIMS, 4)
    q = gaussian_spinors(DIMS, 3, 5)
    V = int(np.prod(DIMS))
    with lattice(DIMS, U, 0.12) as (L, h):
        if ape:
            L.lqcd_smear_ape(h, 0.5, 10)
        src = to_dev(q.reshape(3, V, 4, 3))
        out = torch.empty_like(src)
        L.lqcd_smear_gaussian(h, src, out, alpha, n, ape_links=ape, normalise=normalise)
        got = to_np(out, DIMS)
    links = osm.ape_smear(U, 0.5, 10) if ape else U
    ref = osm.gaussian_smear(links, q, alpha, n, normalise)
    assert rel_err(got, ref) < 1e-12


def test_smearing_argument_errors_and_reset():
    U = haar_su3_field(DIMS, 6)
    V = int(np.prod(DIMS))
    with lattice(DIMS, U, 0.12) as (L, h):
        src = to_dev(gaussian_spinors(DIMS, 1, 7).reshape(1, V, 4, 3))
        out = torch.empty_like(src)
        with pytest.raises(L.LqcdError):
            L.lqcd_smear_gaussian(h, src, src, 4.0, 2)  # in == out
        with pytest.raises(L.LqcdError):
            L.lqcd_smear_gaussian(h, src, out, 4.0, 2, ape_links=True)  # no APE links yet
        L.lqcd_smear_ape(h, 0.5, 2)
        L.lqcd_smear_gaussian(h, src, out, 4.0, 2, ape_links=True)
        # a new gauge field invalidates the smeared links
        L.lqcd_set_gauge(h, torch.from_numpy(U.reshape(-1)).cuda())
        with pytest.raises(L.LqcdError):
            L.lqcd_smear_gaussian(h, src, out, 4.0, 2, ape_links=True)
        # n_iter = 0 copies
        L.lqcd_smear_gaussian(h, src, out, 4.0, 0)
        assert torch.equal(out, src)
