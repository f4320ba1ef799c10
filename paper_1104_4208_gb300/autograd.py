"""torch.autograd binding of the library's adjoint gradient.

ObservationObjective.apply(eps, solver, E0, H0, dt, nsteps, xobs, ckpt_every)
returns J = sum_{n=1..nsteps} sum_o |E^n(x_o)|^2 (a 0-d float64 tensor) for the
permittivity `eps` (1-d tensor, one value per element); its backward gives
dJ/d eps from dgm_adjoint_grad (discrete adjoint, checkpointed recomputation).
Marshalling only: the forward run, the adjoint run and the gradient are
computed by libdgm.so.
"""

import numpy as np
import torch

from . import _capi as capi


class ObservationObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, solver, E0, H0, dt, nsteps, xobs, ckpt_every):
        e = np.ascontiguousarray(eps.detach().to("cpu", torch.float64).numpy())
        capi.dgm_set_materials(solver.prob, e, solver.mu)
        solver.set_fields(E0, H0)
        J, grad = capi.dgm_adjoint_grad(solver.prob, dt, nsteps, xobs, ckpt_every, solver.nt)
        ctx.save_for_backward(torch.from_numpy(grad).to(eps.device, eps.dtype))
        return torch.tensor(J, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return (gJ.to(grad.dtype) * grad, None, None, None, None, None, None, None)
