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
    """Holds one library context for a fixed grid and parameter set.

    stream: a torch.cuda.Stream for the library's work, or None to follow
    torch's current stream at every call.  With a separate stream, each call
    makes it wait for the current stream's pending work (the producers of a,
    f and dL/dphi) and makes the current stream wait for the result.
    strict: a forward or adjoint solve that stops at max_iters without
    reaching rtol raises GMGError (status GMG_ERR_NOT_CONVERGED) instead of
    returning an unconverged phi or gradient."""

    def __init__(self, shape, stream=None, strict=True, **params):
        nz, ny, nx = (int(s) for s in shape)
        self.params = gmg.gmg_default_params(nx, ny, nz, **params)
        self.shape = (nz, ny, nx)
        self.stream = stream
        self.strict = strict
        self.ctx = None
        self._a = None           # the tensor whose values the context holds
        self._a_version = None
        self.last_info = None
        self.last_adjoint_info = None

    def _enter(self):
        """Order the library's stream after torch's current stream."""
        cur = torch.cuda.current_stream()
        if self.stream is None:
            if self.ctx is not None:
                gmg.gmg_set_stream(self.ctx, cur)
        elif self.stream != cur:
            self.stream.wait_stream(cur)

    def _leave(self):
        """Order torch's current stream after the library's work."""
        cur = torch.cuda.current_stream()
        if self.stream is not None and self.stream != cur:
            cur.wait_stream(self.stream)

    def _check(self, info, what):
        if self.strict and not (info.converged and info.true_rel_residual <= self.params.rtol):
            raise gmg.GMGError(gmg.GMG_ERR_NOT_CONVERGED,
                               f"{what}: {info.iterations} iterations, true relative residual "
                               f"{info.true_rel_residual:.3e} > rtol {self.params.rtol:.1e}")
        return info

    def set_coefficient(self, a: torch.Tensor):
        self._enter()
        a = a.detach()
        if self.ctx is None:
            self.ctx = gmg.gmg_setup(self.params, a.contiguous(), self.stream)
        elif a is not self._a or a._version != self._a_version:
            gmg.gmg_update_coefficient(self.ctx, a.contiguous())
        self._a, self._a_version = a, a._version

    def solve(self, a: torch.Tensor, f: torch.Tensor, phi0: torch.Tensor | None = None) -> torch.Tensor:
        return _SolveFn.apply(a, f, phi0, self)

    def field(self, phi: torch.Tensor, dtype=torch.float32):
        self._enter()
        ex, ey, ez = (torch.empty(self.shape, dtype=dtype, device=phi.device) for _ in range(3))
        gmg.field_from_potential(self.ctx, phi.detach().contiguous(), ex, ey, ez)
        self._leave()
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
        fd = f.detach().contiguous()
        solver._enter()
        solver.last_info = gmg.fgmres_solve(solver.ctx, fd, phi)
        solver._leave()
        solver._check(solver.last_info, "forward solve")
        fctx.solver = solver
        fctx.save_for_backward(a, phi)
        return phi

    @staticmethod
    def backward(fctx, grad_phi):
        a, phi = fctx.saved_tensors
        solver = fctx.solver
        solver.set_coefficient(a)
        lam = torch.zeros_like(phi)
        g = grad_phi.contiguous()
        dlda = torch.empty_like(phi)
        solver._enter()
        solver.last_adjoint_info = gmg.fgmres_solve(solver.ctx, g, lam, homogeneous_bc=True)
        solver._check(solver.last_adjoint_info, "adjoint solve")
        gmg.adjoint_coefficient_grad(solver.ctx, phi, lam, dlda)
        solver._leave()
        return dlda, lam, None, None
