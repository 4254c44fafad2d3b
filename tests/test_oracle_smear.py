"""Pins of the smearing oracle (oracle/smear.py) against closed forms and
invariances: free-field plane waves, hermiticity of the 3-d hopping matrix,
gauge covariance, independence of time slices, and the SU(3) projection."""
import numpy as np
import pytest

from lattice_inputs import haar_su3_field, eps_su3_field, unit_gauge_field, gaussian_spinors, random_gauge_transform
from oracle import smear

DIMS = (4, 6, 4, 3)  # Lx, Ly, Lz, Lt: unequal extents catch axis mix-ups


def _gauge_transform(U, g):
    axis = (3, 2, 1, 0)
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=axis[mu])
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    return Ug


@pytest.mark.parametrize("n", [(0, 0, 0), (1, 2, 3), (3, 5, 1)])
@pytest.mark.parametrize("normalise", [False, True])
def test_free_field_plane_wave_eigenvalue(n, normalise):
    """U = 1: q(x) = e^{ip.x} c is an eigenvector, F(p) = (1 + 2 alpha sum_i cos p_i)^n."""
    lx, ly, lz, lt = DIMS
    alpha, steps = 0.7, 3
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    p = (2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz)
    wave = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z))
    c = gaussian_spinors((1, 1, 1, 1), 1, 3)[0, 0, 0, 0, 0]  # one (4, 3) spinor
    q = wave[..., None, None] * c
    out = smear.gaussian_smear(unit_gauge_field(DIMS), q, alpha, steps, normalise)
    lam = (1 + 2 * alpha * sum(np.cos(p))) ** steps
    if normalise:
        lam /= (1 + 6 * alpha) ** steps
    assert np.max(np.abs(out - lam * q)) < 1e-12 * max(1.0, abs(lam))


def test_hop3_hermitian_and_spatial():
    """<a, H b> = <H a, b>; H has no time hops and no spin structure."""
    U = haar_su3_field(DIMS, 2)
    a, b = gaussian_spinors(DIMS, 2, 4)
    lhs = np.vdot(a, smear.hop3(U, b))
    rhs = np.vdot(smear.hop3(U, a), b)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # a source on one time slice stays there
    q = np.zeros_like(a)
    q[1] = a[1]
    out = smear.gaussian_smear(U, q, 0.4, 4)
    assert np.max(np.abs(out[[0, 2]])) == 0.0 and np.max(np.abs(out[1])) > 0
    # spin components are smeared alike: permuting spins commutes with F
    perm = [2, 0, 3, 1]
    assert np.allclose(smear.gaussian_smear(U, a[..., perm, :], 0.4, 2),
                       smear.gaussian_smear(U, a, 0.4, 2)[..., perm, :], atol=1e-12)


def test_gaussian_smearing_gauge_covariant():
    U = haar_su3_field(DIMS, 5)
    g = random_gauge_transform(DIMS, 6)
    q = gaussian_spinors(DIMS, 1, 7)[0]
    gq = np.einsum("...ab,...sb->...sa", g, q)
    lhs = smear.gaussian_smear(_gauge_transform(U, g), gq, 0.5, 3)
    rhs = np.einsum("...ab,...sb->...sa", g, smear.gaussian_smear(U, q, 0.5, 3))
    assert np.max(np.abs(lhs - rhs)) < 1e-11 * np.max(np.abs(rhs))


def test_projection_properties():
    W = haar_su3_field((2, 2, 2, 2), 8).reshape(-1, 3, 3)[:20]
    # c W with c > 0 projects back to W; so does e^{i theta} W for |theta| < pi / 3
    assert np.max(np.abs(smear.project_su3(2.5 * W) - W)) < 1e-13
    assert np.max(np.abs(smear.project_su3(np.exp(0.4j) * W) - W)) < 1e-13
    rng = np.random.default_rng(9)
    V = rng.standard_normal((20, 3, 3)) + 1j * rng.standard_normal((20, 3, 3))
    P = smear.project_su3(V)
    eye = np.eye(3)
    assert np.max(np.abs(np.conj(np.swapaxes(P, -1, -2)) @ P - eye)) < 1e-13
    assert np.max(np.abs(np.linalg.det(P) - 1.0)) < 1e-13
    # the unitary polar factor maximises Re Tr(W^+ V) over U(3): random unitary nudges lower it
    A, _, Bh = np.linalg.svd(V)
    polar = A @ Bh
    best = np.real(np.trace(np.conj(np.swapaxes(polar, -1, -2)) @ V, axis1=-2, axis2=-1))
    for _ in range(5):
        H = rng.standard_normal((20, 3, 3)) + 1j * rng.standard_normal((20, 3, 3))
        H = 0.05 * (H + np.conj(np.swapaxes(H, -1, -2)))
        w, v = np.linalg.eigh(H)
        nudge = v @ (np.exp(1j * w)[..., None] * np.conj(np.swapaxes(v, -1, -2)))
        other = np.real(np.trace(np.conj(np.swapaxes(polar @ nudge, -1, -2)) @ V, axis1=-2, axis2=-1))
        assert np.all(other <= best + 1e-12)


def test_ape_fixed_points_su3_and_covariance():
    U = eps_su3_field(DIMS, 0.5, 10)
    # alpha = 0: the projection of an SU(3) link is the link
    assert np.max(np.abs(smear.ape_smear(U, 0.0, 2) - U)) < 1e-13
    # the free field is a fixed point (each staple sum is 4 x the identity)
    one = unit_gauge_field(DIMS)
    assert np.max(np.abs(smear.ape_smear(one, 0.5, 3) - one)) < 1e-14
    S = smear.ape_smear(U, 0.5, 3)
    # SU(3) output, temporal links untouched, spatial links changed
    L = S[..., :3, :, :]
    assert np.max(np.abs(np.conj(np.swapaxes(L, -1, -2)) @ L - np.eye(3))) < 1e-13
    assert np.max(np.abs(np.linalg.det(L) - 1.0)) < 1e-13
    assert np.array_equal(S[..., 3, :, :], U[..., 3, :, :])
    assert np.max(np.abs(L - U[..., :3, :, :])) > 1e-3
    # gauge covariance
    g = random_gauge_transform(DIMS, 11)
    lhs = smear.ape_smear(_gauge_transform(U, g), 0.5, 3)
    rhs = _gauge_transform(S, g)
    assert np.max(np.abs(lhs - rhs)) < 1e-12
    # smoothing: the spatial plaquette of the smeared field is closer to 1
    def spatial_plaq(V):
        acc = 0.0
        for i in range(3):
            for j in range(i + 1, 3):
                Vi, Vj = V[..., i, :, :], V[..., j, :, :]
                ai, aj = (3, 2, 1)[i], (3, 2, 1)[j]
                P = Vi @ np.roll(Vj, -1, axis=ai) @ np.conj(np.swapaxes(np.roll(Vi, -1, axis=aj), -1, -2)) \
                    @ np.conj(np.swapaxes(Vj, -1, -2))
                acc += np.real(np.trace(P, axis1=-2, axis2=-1)).mean() / 3
        return acc / 3
    assert spatial_plaq(S) > spatial_plaq(U) + 0.05


def test_staple_sum_on_abelian_field():
    """Diagonal U(1)-like links e^{i theta} 1: each staple is e^{i (sum of signed angles)} 1."""
    lx, ly, lz, lt = DIMS
    rng = np.random.default_rng(12)
    th = rng.uniform(-np.pi, np.pi, size=(lt, lz, ly, lx, 4))
    U = np.exp(1j * th)[..., None, None] * np.eye(3)
    i, j = 0, 1
    S = smear.staples(U, i)
    ax = {0: 3, 1: 2, 2: 1}
    tj = th[..., j]
    up = tj + np.roll(th[..., i], -1, axis=ax[j]) - np.roll(tj, -1, axis=ax[i])
    tjm = np.roll(tj, 1, axis=ax[j])
    down = -tjm + np.roll(th[..., i], 1, axis=ax[j]) + np.roll(tjm, -1, axis=ax[i])
    # the (j = 2) staples enter as well
    k = 2
    tk = th[..., k]
    up2 = tk + np.roll(th[..., i], -1, axis=ax[k]) - np.roll(tk, -1, axis=ax[i])
    tkm = np.roll(tk, 1, axis=ax[k])
    down2 = -tkm + np.roll(th[..., i], 1, axis=ax[k]) + np.roll(tkm, -1, axis=ax[i])
    expect = np.exp(1j * up) + np.exp(1j * down) + np.exp(1j * up2) + np.exp(1j * down2)
    assert np.max(np.abs(S[..., 0, 0] - expect)) < 1e-13
    assert np.max(np.abs(S[..., 0, 1])) == 0.0
