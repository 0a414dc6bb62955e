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
    # a CTA per system (generic kernels) or a cluster of CTAs per system
    assert block % 32 == 0 and 64 <= block <= 1024 and grid > 0
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


@pytest.mark.parametrize("block", [576, 384, 288])
def test_zmarch_kernel_bulk_nonlocal(block):
    """The shared-memory z-march kernel (bulk-copy staging, plane-wise
    nonlocal terms), forced with K = 2, 3, 4 columns per thread."""
    from paper_1907_02604_gb300 import Hamiltonian, Plan, SolverOptions, make_poles
    w = make_workload("bulk_mixed").subset(np.arange(2))
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    plan = Plan(ham, z, wt, w.nodes, w.halfwidth,
                SolverOptions(tol=1e-10, precision="mixed", block=block, ctas_per_sm=1, kernel="zmarch"))
    plan.launch()
    st = plan.stats()
    assert st["n_converged"] == w.n_systems
    _, o = oracle_run(w)
    assert rel_err(plan.rho.cpu().numpy(), o.rho) <= 1e-5
    assert rel_err(plan.e.cpu().numpy(), o.e_node) <= 1e-5


@pytest.mark.parametrize("case", [dict(shape=(18, 18, 18), fd_order=8, s=3, nonlocal_proj=True, n_atoms=6,
                                       spacing=(0.5, 0.5, 0.5)),
                                  dict(shape=(14, 12, 16), fd_order=4, s=3, periodic=(False, True, False)),
                                  dict(shape=(18, 20, 17), fd_order=4, s=7, nonlocal_proj=True, n_atoms=4,
                                       n_nodes=3, spacing=(0.5, 0.45, 0.55))])
def test_zmarch_kernel_tiny(case):
    from paper_1907_02604_gb300 import Hamiltonian, Plan, SolverOptions, make_poles
    w = make_workload("tiny", **case)
    c = w.node_coords()
    ok = np.ones(len(w.nodes), bool)
    for d in range(3):
        if not w.periodic[d]:
            ok &= (c[:, d] - w.halfwidth >= 0) & (c[:, d] + w.halfwidth < w.shape[d])
    w = w.subset(np.nonzero(ok)[0])
    w.tol = 1e-11
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    m = 2 * int(w.halfwidth.max()) + 1
    block = max(64, ((m * m + 1) // 2 + 31) // 32 * 32)
    plan = Plan(ham, z, wt, w.nodes, w.halfwidth,
                SolverOptions(tol=w.tol, precision="mixed", block=block, ctas_per_sm=1, kernel="zmarch"))
    plan.launch()
    plan.stats()
    _, o = oracle_run(w)
    assert rel_err(plan.rho.cpu().numpy(), o.rho) <= 1e-5
