"""torch.autograd binding of the library's adjoint gradient.

ObservationObjective.apply(eps, solver, E0, H0, dt, nsteps, xobs, ckpt_every[, mu])
returns J = sum_{n=1..nsteps} sum_o |E^n(x_o)|^2 (a 0-d float64 tensor) for the
permittivity `eps` and, if given, the permeability `mu` (1-d tensors, one value
per element; without mu the solver's own is used); its backward gives dJ/d eps
and dJ/d mu from dgm_adjoint_grad (discrete adjoint, checkpointed
recomputation).
Marshalling only: the forward run, the adjoint run and the gradient are
computed by libdgm.so.
"""

import numpy as np
import torch

from . import _capi as capi


class ObservationObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, solver, E0, H0, dt, nsteps, xobs, ckpt_every, mu=None):
        e = np.ascontiguousarray(eps.detach().to("cpu", torch.float64).numpy())
        m = solver.mu if mu is None else np.ascontiguousarray(mu.detach().to("cpu", torch.float64).numpy())
        capi.dgm_set_materials(solver.prob, e, m)
        solver.set_fields(E0, H0)
        J, ge, gm = capi.dgm_adjoint_grad(solver.prob, dt, nsteps, xobs, ckpt_every, solver.nt, mu_grad=True)
        ctx.has_mu = mu is not None
        ctx.save_for_backward(torch.from_numpy(ge).to(eps.device, eps.dtype),
                              torch.from_numpy(gm).to(eps.device, eps.dtype))
        return torch.tensor(J, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, gJ):
        ge, gm = ctx.saved_tensors
        gmu = gJ.to(gm.dtype) * gm if ctx.has_mu else None
        return (gJ.to(ge.dtype) * ge, None, None, None, None, None, None, None, gmu)
