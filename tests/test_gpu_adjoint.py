"""GPU adjoint: dL/dV and forces against the oracle's gradient and against
central finite differences of the GPU forward (step 1e-4 bohr, FP64)."""
import numpy as np
import pytest

from synthetic import make_workload
from synthetic.workloads import fd_atom_choice, jittered_atoms
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu


def _loss_grads_gpu(w, a, b, checkpoint=True, forces=True):
    import torch
    from paper_1907_02604_gb300 import (Hamiltonian, SolverOptions, Workspace, density,
                                        density_adjoint, make_poles)
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    opts = SolverOptions(tol=w.tol, maxit=w.maxit, precision="fp64")
    ws = Workspace(ham, w.nodes, w.halfwidth, w.n_poles) if checkpoint else None
    rho, e, _ = density(ham, z, wt, w.nodes, w.halfwidth, opts, energy=True, checkpoint=ws)
    ta = torch.tensor(a, dtype=torch.float64, device="cuda")
    tb = torch.tensor(b, dtype=torch.float64, device="cuda")
    g, F = density_adjoint(ham, z, wt, w.nodes, w.halfwidth, ta, tb, opts, checkpoint=ws, forces=forces)
    return rho.cpu().numpy(), e.cpu().numpy(), g.cpu().numpy(), None if F is None else F.cpu().numpy(), (z, wt)


@pytest.mark.parametrize("checkpoint", [True, False])
def test_adjoint_matches_oracle_tiny(checkpoint):
    from oracle import density as od
    w = make_workload("tiny", shape=(10, 10, 10), s=3, n_nodes=5, spacing=(0.5, 0.5, 0.5), n_atoms=3)
    w.tol = 1e-12
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=5), rng.normal(size=5)
    rho, e, g, F, _ = _loss_grads_gpu(w, a, b, checkpoint=checkpoint)
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13, keep_x=True)
    go = od.dL_dV(w, res, a, b)
    Fo = od.forces(w, go)
    assert rel_err(g, go) < 1e-8
    assert rel_err(F, Fo) < 1e-8


def test_adjoint_loss_forces_vs_finite_differences():
    """Loss E_band + 1/2 ||rho - rho_target||^2 on 32 nodes of the
    128-atom, 8th-order, P = 16 cell; rho_target from the 2% jitter."""
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density, make_poles
    w = make_workload("adjoint_fp64").subset(np.arange(32))
    w.tol = 1e-12
    wj = w.with_atoms(jittered_atoms(w))
    ham_t = Hamiltonian.from_workload(wj)
    zt, wtt = make_poles(w.kT, w.mu, *ham_t.spectral_bounds(), w.n_poles)
    rho_t, _, _ = density(ham_t, zt, wtt, w.nodes, w.halfwidth, SolverOptions(tol=1e-12))
    rho_t = rho_t.cpu().numpy()

    # poles fixed at the unperturbed geometry so the FD sees only the solves
    ham0 = Hamiltonian.from_workload(w)
    z0, w0 = make_poles(w.kT, w.mu, *ham0.spectral_bounds(), w.n_poles)

    def loss(atoms):
        ham = Hamiltonian.from_workload(w, atoms=atoms)
        rho, e, _ = density(ham, z0, w0, w.nodes, w.halfwidth, SolverOptions(tol=1e-12), energy=True)
        rho, e = rho.cpu().numpy(), e.cpu().numpy()
        return e.sum() + 0.5 * np.sum((rho - rho_t) ** 2), rho

    import torch
    from paper_1907_02604_gb300 import Workspace, density_adjoint
    L0, rho0 = loss(w.atoms)
    ws = Workspace(ham0, w.nodes, w.halfwidth, w.n_poles)
    density(ham0, z0, w0, w.nodes, w.halfwidth, SolverOptions(tol=1e-12), checkpoint=ws)
    a = torch.tensor(rho0 - rho_t, device="cuda")
    b = torch.ones(len(w.nodes), dtype=torch.float64, device="cuda")
    _, F = density_adjoint(ham0, z0, w0, w.nodes, w.halfwidth, a, b, SolverOptions(tol=1e-12),
                           checkpoint=ws, forces=True)
    F = F.cpu().numpy()
    step = 1e-4
    scale = np.abs(F).max()
    for atom in fd_atom_choice(w)[:3]:
        for d in range(3):
            vals = []
            for sgn in (1, -1):
                pos = w.atoms.copy()
                pos[atom, d] += sgn * step
                vals.append(loss(pos)[0])
            fd = -(vals[0] - vals[1]) / (2 * step)
            assert abs(fd - F[atom, d]) <= 1e-6 * scale, (atom, d, fd, F[atom, d])
