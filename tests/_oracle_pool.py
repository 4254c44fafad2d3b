"""Oracle calls run in spawned worker processes by the full-size GPU tests
(the oracle needs about a minute per 16^3 x 32 solve; several run in parallel).
Each worker regenerates its inputs from their seeds instead of receiving them."""


def dkappa_piece(args):
    """The oracle's d/dkappa estimator (complex) for one diluted piece of a
    complex Z2 noise vector on an eps-field: (dims, eps, field_seed, kappa,
    noise_seed, noise_index, scheme, piece, gamma_index, tol)."""
    dims, eps, field_seed, kappa, noise_seed, noise_index, scheme, piece, g, tol = args
    from lattice_inputs import eps_su3_field
    from oracle import gradient as gr, philox as oph
    U = eps_su3_field(dims, eps, field_seed)
    src = oph.dilute(oph.z2_noise(dims, noise_seed, noise_index, 0), scheme, piece)[None]
    return complex(gr.dkappa_estimator(U, kappa, src, g, tol=tol))
