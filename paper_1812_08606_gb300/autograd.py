"""torch.autograd wrapper of the solve with a hand-written adjoint.

Forward: phi = A(a)^{-1} b(a, f) by the library's GMG-FGMRES solve.
Backward (the discrete adjoint of the operator of eq. (e18); not in the
paper): the operator is symmetric, so lambda = A^{-1} dL/dphi comes from the
same solver with zero plate data; then dL/df = lambda and dL/da comes from the
library's face kernel.  Only phi is kept from the forward pass (``a`` is an
input of the call, not a saved intermediate).
"""
from __future__ import annotations

import torch

from . import gmg


class PoissonSolver:
    """Holds one library context for a fixed grid and parameter set."""

    def __init__(self, shape, stream=None, **params):
        nz, ny, nx = (int(s) for s in shape)
        self.params = gmg.gmg_default_params(nx, ny, nz, **params)
        self.shape = (nz, ny, nx)
        self.stream = stream
        self.ctx = None
        self._a = None           # the tensor whose values the context holds
        self._a_version = None
        self.last_info = None
        self.last_adjoint_info = None

    def set_coefficient(self, a: torch.Tensor):
        a = a.detach()
        if self.ctx is None:
            self.ctx = gmg.gmg_setup(self.params, a.contiguous(), self.stream)
        elif a is not self._a or a._version != self._a_version:
            gmg.gmg_update_coefficient(self.ctx, a.contiguous())
        self._a, self._a_version = a, a._version

    def solve(self, a: torch.Tensor, f: torch.Tensor, phi0: torch.Tensor | None = None) -> torch.Tensor:
        return _SolveFn.apply(a, f, phi0, self)

    def field(self, phi: torch.Tensor, dtype=torch.float32):
        ex, ey, ez = (torch.empty(self.shape, dtype=dtype, device=phi.device) for _ in range(3))
        gmg.field_from_potential(self.ctx, phi.detach().contiguous(), ex, ey, ez)
        return ex, ey, ez

    def close(self):
        if self.ctx is not None:
            self.ctx.close()
            self.ctx = None


class _SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, a, f, phi0, solver):
        solver.set_coefficient(a)
        phi = phi0.detach().clone().contiguous() if phi0 is not None else torch.zeros_like(f)
        solver.last_info = gmg.fgmres_solve(solver.ctx, f.detach().contiguous(), phi)
        fctx.solver = solver
        fctx.save_for_backward(a, phi)
        return phi

    @staticmethod
    def backward(fctx, grad_phi):
        a, phi = fctx.saved_tensors
        solver = fctx.solver
        solver.set_coefficient(a)
        lam = torch.zeros_like(phi)
        solver.last_adjoint_info = gmg.fgmres_solve(solver.ctx, grad_phi.contiguous(), lam, homogeneous_bc=True)
        dlda = torch.empty_like(phi)
        gmg.adjoint_coefficient_grad(solver.ctx, phi, lam, dlda)
        return dlda, lam, None, None
