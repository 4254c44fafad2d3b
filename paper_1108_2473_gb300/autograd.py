"""torch.autograd access to the loops and their adjoint-solve gradient.

``LoopsFn.apply(U, kappa, lattice, src, params)`` returns the per-time-slice
loops L_g(t) = sum_{x in t} sum_d src_d(x)^+ Gamma_g D^{-1} src_d(x) (Gamma order
1, g5, g1..g4; Eq. loop stochastic without the 1/N_r) as a complex128 [Lt, 6]
tensor.  Its backward runs lqcd_gradient: one adjoint solve per noise piece with
D^+ = gamma5 D gamma5, giving d loss / d U (torch's complex convention) and
d loss / d kappa.  All arithmetic is in liblqcd; this module only marshals.
"""
from __future__ import annotations

import torch

from . import lqcd as L


class Lattice:
    """A liblqcd context for one lattice shape on one device."""

    def __init__(self, dims, device=0):
        self.dims = tuple(int(d) for d in dims)
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.handle = L.lqcd_create(self.dims, self.device.index or 0)
        self.volume = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]

    def close(self):
        if self.handle is not None:
            L.lqcd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, U, kappa, general=False):
        Uc = U.detach().reshape(-1).contiguous()
        if general:
            L.lqcd_set_gauge_general(self.handle, Uc)
        else:
            L.lqcd_set_gauge(self.handle, Uc)
        L.lqcd_set_kappa(self.handle, float(kappa))


class LoopsFn(torch.autograd.Function):
    """Per-time-slice loops of the given noise pieces as a function of (U, kappa).

    U: complex128 device tensor with V*4*9 entries (canonical layout);
    kappa: float64 scalar tensor; lattice: ``Lattice``; src: complex128
    [n, V, 4, 3] device tensor of noise pieces; params: lqcd_solver_params.
    Set ``params.precision = LQCD_PREC_FP64`` and ``general=True`` to
    differentiate at non-SU(3) links (e.g. under torch.autograd.gradcheck).
    """

    @staticmethod
    def forward(ctx, U, kappa, lattice, src, params, general=False):
        lattice.set_fields(U, kappa.item(), general)
        x = torch.empty_like(src)
        rc, st = L.lqcd_solve_batch(lattice.handle, src, x, params)
        if rc != L.LQCD_OK:
            raise L.LqcdError(rc, f"forward solves failed: {st[:2]}")
        per_t = torch.zeros((lattice.dims[3], 6), dtype=torch.complex128, device=src.device)
        L.lqcd_loops_batch(lattice.handle, src, x, 1.0, None, per_t)
        ctx.lattice, ctx.params, ctx.general = lattice, params, general
        ctx.save_for_backward(U, kappa, src, x)
        return per_t

    @staticmethod
    def backward(ctx, grad_L):
        U, kappa, src, x = ctx.saved_tensors
        lat = ctx.lattice
        lat.set_fields(U, kappa.item(), ctx.general)
        dU = torch.zeros(U.numel(), dtype=torch.complex128, device=src.device)
        dk, rc, st = L.lqcd_gradient(lat.handle, src, x, grad_L.detach().to("cpu", torch.complex128), ctx.params,
                                     1.0, dU)
        if rc != L.LQCD_OK:
            raise L.LqcdError(rc, f"adjoint solves failed: {st[:2]}")
        gU = dU.reshape(U.shape) if ctx.needs_input_grad[0] else None
        gk = torch.tensor(dk, dtype=kappa.dtype, device=kappa.device) if ctx.needs_input_grad[1] else None
        return gU, gk, None, None, None, None


def loops(U, kappa, lattice, src, params, general=False):
    """Differentiable per-time-slice loops (see LoopsFn)."""
    return LoopsFn.apply(U, kappa, lattice, src, params, general)
