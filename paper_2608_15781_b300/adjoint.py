"""Gradient of the column conversion through the CUDA adjoint, as a torch.autograd.Function.

``conversion(theta, u_in, lattice, f0, nsteps)`` returns the outlet conversion
J = 1 - Phi_out / Phi_in after ``nsteps`` steps from the start state ``f0``
(a (45, nz, ny, nx) float32 host array in the ``lbm_get_state`` layout) with the
per-node contact angle ``theta`` (degrees, read at solid nodes) and inlet
velocity ``u_in``.  The forward runs ``lbm_adjoint_forward`` (checkpointed
time stepping in the CUDA library); ``backward`` runs ``lbm_adjoint_backward``
(the hand-written reverse kernels) and returns dL/dtheta and dL/du_in.  This
module only marshals arguments: every step runs in the library.
"""
import numpy as np
import torch

from . import lbm


class ConversionObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, u_in, lattice, f0, nsteps, checkpoint_every):
        lattice.set_wetting(theta.detach().to("cpu", torch.float32).numpy())
        lattice.set_inlet(float(u_in.detach()))
        lattice.set_state(f0)
        J = lattice.adjoint_forward(int(nsteps), int(checkpoint_every))
        ctx.lattice = lattice
        ctx.theta_meta = (theta.dtype, theta.device)
        ctx.u_meta = (u_in.dtype, u_in.device)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        dth, du, _ = ctx.lattice.adjoint_backward(seed=float(grad_out))
        tdt, tdev = ctx.theta_meta
        udt, udev = ctx.u_meta
        return (torch.from_numpy(dth).to(tdev, tdt), torch.tensor(du, dtype=udt, device=udev),
                None, None, None, None)


def conversion(theta, u_in, lattice, f0, nsteps, checkpoint_every=0):
    """Differentiable J(theta, u_in); see the module docstring."""
    if not torch.is_tensor(u_in):
        u_in = torch.tensor(float(u_in), dtype=torch.float64)
    return ConversionObjective.apply(theta, u_in, lattice, np.ascontiguousarray(f0, dtype=np.float32),
                                     nsteps, checkpoint_every)
