"""The second-order semi-implicit streamer time step (eqs. (e1)-(e2)) on the GPU.

A sequence of C-ABI calls, no arithmetic of its own: assemble the elliptic
coefficient and right-hand side from the densities at t_n
(``assemble_coefficient_rhs``, eq. (semi2)), renew the multigrid set-up,
solve for phi^{n+1/2} warm-started from the previous step's potential (the
first step, with a zero guess, takes full multigrid when ``params.cycle`` is
GMG_CYCLE_AUTO), then the predictor n^{n+1/2} = n^n + (tau/2) R(n^n) and the
corrector n^{n+1} = n^n + tau R(n^{n+1/2}) (``transport_step``), both in the
field E^{n+1/2}, which share the ionization rate alpha(|E|) mu_e |E|.
"""
from __future__ import annotations

import torch

from . import gmg


class SemiImplicitStepper:
    """Advances (n_e, n_p) by fixed steps tau; keeps the solver context, the
    potential (the next step's initial guess) and the work arrays."""

    def __init__(self, params: gmg.gmg_params, tau: float, mu_e: float, mu_p: float, diffusion,
                 e_over_eps0: float = gmg.E_OVER_EPS0_CM, ion_a: float = 5.7, ion_b: float = 260.0,
                 pressure: float = 760.0, device=None, stream=None):
        self.params = params
        self.tau = float(tau)
        self.mu = (float(mu_e), float(mu_p))
        self.diffusion = tuple(float(d) for d in diffusion)
        self.e_over_eps0 = float(e_over_eps0)
        self.ion = (float(ion_a), float(ion_b), float(pressure))
        self.stream = stream
        shape = (params.nz, params.ny, params.nx)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        z = lambda: torch.zeros(shape, dtype=torch.float64, device=dev)   # noqa: E731
        self.a, self.f, self.phi, self.half_e, self.half_p, self.rate = z(), z(), z(), z(), z(), z()
        self.ctx = None
        self.last_info = None

    def step(self, n_e: torch.Tensor, n_p: torch.Tensor, out_e: torch.Tensor, out_p: torch.Tensor):
        """One step from (n_e, n_p) at t_n into (out_e, out_p) at t_{n+1};
        returns the solve's info.  out_* may be n_* (in place)."""
        p, tau, s = self.params, self.tau, self.stream
        mu_e, mu_p = self.mu
        gmg.assemble_coefficient_rhs(p, n_e, n_p, self.a, self.f, tau=tau, mu_e=mu_e, mu_p=mu_p,
                                     diffusion=self.diffusion, e_over_eps0=self.e_over_eps0, stream=s)
        if self.ctx is None:
            self.ctx = gmg.gmg_setup(p, self.a, s)
        else:
            gmg.gmg_update_coefficient(self.ctx, self.a)
        info = gmg.fgmres_solve(self.ctx, self.f, self.phi)
        ion_a, ion_b, pres = self.ion
        kw = dict(mu_e=mu_e, mu_p=mu_p, diffusion=self.diffusion, ion_a=ion_a, ion_b=ion_b, pressure=pres, stream=s)
        gmg.transport_step(p, n_e, n_p, self.phi, tau, self.half_e, self.half_p, out_e, out_p, self.rate, **kw)
        self.last_info = info
        return info

    def close(self):
        if self.ctx is not None:
            self.ctx.close()
            self.ctx = None
