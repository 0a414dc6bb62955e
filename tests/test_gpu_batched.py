"""Batched uneven regions: nodes of the screw-dislocation cylinder (open x and
y axes, regions 17^3..41^3, 8th order, P = 16, mixed precision) in one
graph-captured persistent launch, against the oracle on a sample."""
import numpy as np
import pytest

from synthetic import make_workload
from tests.gpu_helpers import oracle_run, rel_err

pytestmark = pytest.mark.gpu


def test_screw_sample_mixed_vs_oracle():
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, Plan, SolverOptions, make_poles
    w = make_workload("screw_batched")
    hw = w.halfwidth
    # one node of each extreme size and two in between, all in one launch
    pick = [int(np.argmax(hw)), int(np.argmin(hw)), int(np.argsort(hw)[len(hw) // 2]),
            int(np.argsort(hw)[len(hw) // 4])]
    ws = w.subset(np.array(pick))
    ham = Hamiltonian.from_workload(ws)
    z, wt = make_poles(ws.kT, ws.mu, *ham.spectral_bounds(), ws.n_poles)
    plan = Plan(ham, z, wt, ws.nodes, ws.halfwidth, SolverOptions(tol=1e-10, precision="mixed"))
    plan.launch()
    st = plan.stats()
    assert st["n_converged"] == ws.n_systems
    rho = plan.rho.cpu().numpy()
    _, o = oracle_run(ws)
    assert rel_err(rho, o.rho) <= 1e-5
    torch.cuda.synchronize()


def test_screw_full_launch_invariants():
    """All 1,250 nodes x 16 poles in one launch: every system converges and
    the density is finite; a sample is re-checked against the oracle."""
    from paper_1907_02604_gb300 import Hamiltonian, Plan, SolverOptions, make_poles
    w = make_workload("screw_batched")
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    plan = Plan(ham, z, wt, w.nodes, w.halfwidth, SolverOptions(tol=1e-10, precision="mixed"))
    plan.launch()
    st = plan.stats(strict=False)
    assert st["n_systems"] == 20000
    assert st["n_converged"] == st["n_systems"], st
    rho = plan.rho.cpu().numpy()
    assert np.isfinite(rho).all()
    sample = np.array([0, 617, 1249])
    _, o = oracle_run(w.subset(sample))
    assert rel_err(rho[sample], o.rho) <= 1e-5
