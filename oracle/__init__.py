"""Plain, slow, FP64 CPU oracle for the disconnected-loop hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The GPU library never imports, links or runs anything here, and nothing
here imports the GPU library: the only code the two share is the seeded input
drawing in ``lattice_inputs`` (gauge fields and Gaussian vectors, none of the
method's arithmetic).

What it computes (arXiv:1108.2473):

* ``dirac``    -- the Wilson-Dirac operator D = 1 - kappa*H (the operator M of
  the stopping rule in Sec. III, in the standard Wilson form),
  gamma matrices, even-odd blocks, plaquette.
* ``solver``   -- BiCGstab (van der Vorst) on the even-odd Schur complement,
  stopped on the true relative residual |M x - b| / |b| of Sec. III.
* ``philox``   -- Philox4x64-10 (Salmon et al., SC'11) and the complex Z2
  noise built from it, with time/spin/colour dilution (Sec. II).
* ``loops``    -- exact loops L(x) = Tr[Gamma G(x;x)] (Eq. loop) from point
  sources, the stochastic estimator of Eq. (loop stochastic), and the truncated
  solver method (Sec. II, Bali et al.).
* ``gradient`` -- d/dkappa of the loops and the gauge-link gradient of a
  weighted sum of time-slice loops, via forward and gamma5-adjoint solves,
  plus dense references.
* ``dense``    -- the dense 12V x 12V matrix of D for tiny lattices.

Parity status of each function is stated in its docstring; every function
listed above is pinned by a ``-m "not gpu"`` test against closed forms,
invariants or library routines (``tests/test_oracle_*.py``).
"""
