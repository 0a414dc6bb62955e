"""Plans: the autotuned, graph-captured batched solve (uneven regions in one
launch) agrees with the oracle and replays correctly."""
import numpy as np
import pytest

from synthetic import make_workload
from tests.gpu_helpers import oracle_run, rel_err

pytestmark = pytest.mark.gpu


def _uneven():
    w = make_workload("tiny", shape=(24, 24, 24), n_nodes=10, s=2, spacing=(0.5, 0.5, 0.5), n_atoms=8)
    w.halfwidth = np.array([2, 9, 4, 7, 3, 8, 5, 6, 2, 9], dtype=np.int32)
    w.tol = 1e-11
    return w


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_plan_uneven_regions_one_launch(precision):
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, Plan, SolverOptions, make_poles
    w = _uneven()
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    plan = Plan(ham, z, wt, w.nodes, w.halfwidth, SolverOptions(tol=w.tol, precision=precision))
    block, grid = plan.launch_shape()
    assert block in (256, 512, 768, 1024) and 0 < grid <= w.n_systems
    plan.launch()
    st = plan.stats()
    assert st["n_converged"] == w.n_systems
    rho1 = plan.rho.cpu().numpy().copy()
    plan.launch()                      # graph replay
    plan.stats()
    np.testing.assert_array_equal(plan.rho.cpu().numpy(), rho1)
    _, o = oracle_run(w)
    bar = 1e-6 if precision == "fp64" else 1e-5
    assert rel_err(rho1, o.rho) <= bar
    assert rel_err(plan.e.cpu().numpy(), o.e_node) <= bar
    torch.cuda.synchronize()


def test_plan_sees_new_potential():
    from paper_1907_02604_gb300 import Hamiltonian, Plan, SolverOptions, density, make_poles
    w = _uneven()
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    plan = Plan(ham, z, wt, w.nodes, w.halfwidth, SolverOptions(tol=w.tol))
    V = ham.potential()
    ham.set_potential(V + 0.01)
    plan.launch()
    plan.stats()
    ref, _, _ = density(ham, z, wt, w.nodes, w.halfwidth, SolverOptions(tol=w.tol))
    np.testing.assert_allclose(plan.rho.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=1e-14)
