"""Fused adjoint (no checkpoint): dL/dV accumulated by each system as it
converges, against the checkpointed two-pass adjoint and the oracle's
gradient (Section 2.1 forces)."""
import numpy as np
import pytest

from synthetic import make_workload
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu


def _grads_two_pass(w, a, b, precision):
    import torch
    from paper_1907_02604_gb300 import (Hamiltonian, SolverOptions, Workspace, density,
                                        density_adjoint, make_poles)
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    opts = SolverOptions(tol=w.tol, maxit=w.maxit, precision=precision)
    ws = Workspace(ham, w.nodes, w.halfwidth, w.n_poles)
    rho, e, _ = density(ham, z, wt, w.nodes, w.halfwidth, opts, energy=True, checkpoint=ws)
    ta = torch.tensor(a, dtype=torch.float64, device="cuda")
    tb = torch.tensor(b, dtype=torch.float64, device="cuda")
    g, F = density_adjoint(ham, z, wt, w.nodes, w.halfwidth, ta, tb, opts, checkpoint=ws,
                           forces=not w.nonlocal_proj)
    return ham, (z, wt), opts, rho.cpu().numpy(), e.cpu().numpy(), g.cpu().numpy(), \
        None if F is None else F.cpu().numpy()


def _fused(ham, zw, w, a, b, opts, forces):
    import torch
    from paper_1907_02604_gb300 import density_fused_adjoint
    ta = None if a is None else torch.tensor(a, dtype=torch.float64, device="cuda")
    tb = None if b is None else torch.tensor(b, dtype=torch.float64, device="cuda")
    rho, e, g, F, st = density_fused_adjoint(ham, *zw, w.nodes, w.halfwidth, ta, tb, opts, forces=forces)
    return rho.cpu().numpy(), e.cpu().numpy(), g.cpu().numpy(), None if F is None else F.cpu().numpy(), st


def test_fused_adjoint_matches_oracle_tiny():
    from oracle import density as od
    w = make_workload("tiny", shape=(10, 10, 10), s=3, n_nodes=5, spacing=(0.5, 0.5, 0.5), n_atoms=3)
    w.tol = 1e-12
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=5), rng.normal(size=5)
    ham, zw, opts, rho2, e2, g2, F2 = _grads_two_pass(w, a, b, "fp64")
    rho, e, g, F, st = _fused(ham, zw, w, a, b, opts, forces=True)
    assert st["n_converged"] == w.n_systems
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13, keep_x=True)
    go = od.dL_dV(w, res, a, b)
    Fo = od.forces(w, go)
    assert rel_err(rho, res.rho) < 1e-8
    assert rel_err(g, go) < 1e-8
    assert rel_err(F, Fo) < 1e-8
    assert rel_err(g, g2) < 1e-9
    assert rel_err(F, F2) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_adjoint_band_energy_adjoint_cell(precision):
    """Band-energy loss (a = 0, b = 1) on 24 nodes of the 128-atom cell."""
    w = make_workload("adjoint_fp64").subset(np.arange(24))
    w.tol = 1e-12 if precision == "fp64" else 1e-10
    a, b = np.zeros(24), np.ones(24)
    ham, zw, opts, rho2, e2, g2, F2 = _grads_two_pass(w, a, b, precision)
    rho, e, g, F, st = _fused(ham, zw, w, None, b, opts, forces=True)
    assert st["n_converged"] == w.n_systems
    bar = 1e-9 if precision == "fp64" else 1e-5
    assert rel_err(rho, rho2) < bar
    assert rel_err(e, e2) < bar
    assert rel_err(g, g2) < bar
    assert rel_err(F, F2) < bar


def test_fused_adjoint_nonlocal_gradient():
    """dL/dV with the nonlocal term present (forces refused there)."""
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_INVALID
    w = make_workload("bulk_mixed").subset(np.arange(2))
    w.tol = 1e-10
    rng = np.random.default_rng(2)
    a, b = rng.normal(size=2), rng.normal(size=2)
    ham, zw, opts, _, _, g2, _ = _grads_two_pass(w, a, b, "mixed")
    _, _, g, _, _ = _fused(ham, zw, w, a, b, opts, forces=False)
    assert rel_err(g, g2) < 1e-5
    with pytest.raises(MacroDFTError) as ei:
        _fused(ham, zw, w, a, b, opts, forces=True)
    assert ei.value.status == MD_ERR_INVALID


def test_fused_adjoint_refuses_shifted():
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, make_poles
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_INVALID
    w = make_workload("tiny")
    ham = Hamiltonian.from_workload(w)
    zw = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    with pytest.raises(MacroDFTError) as ei:
        _fused(ham, zw, w, None, np.ones(len(w.nodes)), SolverOptions(method="shifted"), forces=False)
    assert ei.value.status == MD_ERR_INVALID
