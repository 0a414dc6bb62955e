"""autograd wrappers: gradients through torch match the oracle's adjoint."""
import numpy as np
import pytest

from synthetic import make_workload
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu


def _setup(n_atoms=3):
    w = make_workload("tiny", shape=(10, 10, 10), s=3, n_nodes=5, spacing=(0.5, 0.5, 0.5), n_atoms=n_atoms)
    w.tol = 1e-12
    return w


def test_density_of_potential_gradient():
    import torch
    from oracle import density as od
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, make_poles
    from paper_1907_02604_gb300.torch_api import DensityOfPotential
    w = _setup()
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    V = ham.potential().clone().requires_grad_(True)
    rho, e = DensityOfPotential.apply(V, ham, z, wt, w.nodes, w.halfwidth, SolverOptions(tol=1e-12))
    a = torch.linspace(-1, 1, len(w.nodes), dtype=torch.float64, device="cuda")
    loss = (a * rho).sum() + 0.5 * e.sum()
    loss.backward()
    res = od.solve(w, od.build(w), z=z, wts=wt, tol=1e-13, keep_x=True)
    go = od.dL_dV(w, res, a.cpu().numpy(), 0.5 * np.ones(len(w.nodes)))
    assert rel_err(V.grad.cpu().numpy(), go) < 1e-8


def test_density_of_atoms_gradient():
    import torch
    from oracle import density as od
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, make_poles
    from paper_1907_02604_gb300.torch_api import DensityOfAtoms
    w = _setup(n_atoms=2)
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    R = torch.tensor(w.atoms, dtype=torch.float64, requires_grad=True)
    rho, e = DensityOfAtoms.apply(R, w, z, wt, SolverOptions(tol=1e-12))
    rho_t = torch.zeros_like(rho)
    loss = e.sum() + 0.5 * ((rho - rho_t) ** 2).sum()
    loss.backward()
    res = od.solve(w, od.build(w), z=z, wts=wt, tol=1e-13, keep_x=True)
    go = od.dL_dV(w, res, res.rho, np.ones(len(w.nodes)))
    Fo = od.forces(w, go)
    assert rel_err(R.grad.numpy(), -Fo) < 1e-8
