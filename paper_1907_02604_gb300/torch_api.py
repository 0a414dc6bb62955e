"""autograd wrappers around md_density / md_density_adjoint.

Both functions return (rho, e) per node and differentiate through the
adjoint identity dG_jj/dV_k = -x_jp(k)^2 of the complex-symmetric resolvent
(the forward solutions, checkpointed on the device, are the adjoint
solutions), so backward needs no second solve.

* ``DensityOfPotential.apply(V, ham, z, w, nodes, halfwidth, opts)``:
  differentiable in the local potential V (float64 CUDA tensor, one value per
  grid point, x fastest); backward returns dL/dV.
* ``DensityOfAtoms.apply(R, template, z, w, opts)``: differentiable in the
  atom positions R (float64 tensor (n_atoms, 3)); the Hamiltonian is rebuilt
  from R on the device; backward returns dL/dR = -F (Hellmann-Feynman forces
  through the local Gaussian wells).  ``template`` is a workload-like object
  (grid, depths, widths, potential parameters, nodes, halfwidths).

The poles are passed in and held fixed, so the derivative is that of the
rational approximation at fixed (z_p, w_p).
"""
import numpy as np
import torch

from .api import Hamiltonian, SolverOptions, Workspace, density, density_adjoint


class DensityOfPotential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, ham, z, w, nodes, halfwidth, opts=None):
        opts = opts or SolverOptions()
        ham.set_potential(V.detach().contiguous())
        ws = Workspace(ham, nodes, halfwidth, len(z))
        rho, e, stats = density(ham, z, w, nodes, halfwidth, opts, energy=True, checkpoint=ws)
        ctx.state = (ham, z, w, nodes, halfwidth, opts, ws)
        ctx.stats = stats
        return rho, e

    @staticmethod
    def backward(ctx, grad_rho, grad_e):
        ham, z, w, nodes, halfwidth, opts, ws = ctx.state
        n = len(nodes)
        if grad_rho is None:
            grad_rho = torch.zeros(n, dtype=torch.float64, device="cuda")
        g, _ = density_adjoint(ham, z, w, nodes, halfwidth, grad_rho.contiguous(),
                               None if grad_e is None else grad_e.contiguous(), opts, checkpoint=ws)
        ws.close()
        return g, None, None, None, None, None, None


class DensityOfAtoms(torch.autograd.Function):
    @staticmethod
    def forward(ctx, R, template, z, w, opts=None):
        opts = opts or SolverOptions()
        pos = R.detach().cpu().numpy().astype(np.float64)
        ham = Hamiltonian.from_workload(template, atoms=pos)
        ws = Workspace(ham, template.nodes, template.halfwidth, len(z))
        rho, e, stats = density(ham, z, w, template.nodes, template.halfwidth, opts, energy=True,
                                checkpoint=ws)
        ctx.state = (ham, template, z, w, opts, ws, R.device)
        ctx.stats = stats
        return rho, e

    @staticmethod
    def backward(ctx, grad_rho, grad_e):
        ham, t, z, w, opts, ws, dev = ctx.state
        n = len(t.nodes)
        if grad_rho is None:
            grad_rho = torch.zeros(n, dtype=torch.float64, device="cuda")
        _, F = density_adjoint(ham, z, w, t.nodes, t.halfwidth, grad_rho.contiguous(),
                               None if grad_e is None else grad_e.contiguous(), opts,
                               checkpoint=ws, forces=True)
        ws.close()
        ham.close()
        return (-F).to(dev), None, None, None, None
