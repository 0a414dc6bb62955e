"""Shifted COCG (one Krylov sequence per node for all poles) against the
oracle's per-pole solves: same densities within the FP64 / mixed bars, with
fewer matrix-vector products."""
import numpy as np
import pytest

from synthetic import make_workload
from tests.gpu_helpers import oracle_run, rel_err

pytestmark = pytest.mark.gpu


def _run(w, precision, method, **kw):
    from paper_1907_02604_gb300 import Hamiltonian, Plan, SolverOptions, make_poles
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    plan = Plan(ham, z, wt, w.nodes, w.halfwidth,
                SolverOptions(tol=w.tol, maxit=w.maxit, precision=precision, method=method, **kw))
    plan.launch()
    st = plan.stats()
    return plan.rho.cpu().numpy(), plan.e.cpu().numpy(), st


@pytest.mark.parametrize("name,precision,n_nodes", [("small_fp64", "fp64", 32), ("small_fp64", "mixed", 32),
                                                    ("bulk_mixed", "mixed", 3), ("bulk_mixed", "fp64", 2)])
def test_shifted_matches_oracle(name, precision, n_nodes):
    w = make_workload(name).subset(np.arange(n_nodes))
    rho, e, st = _run(w, precision, "shifted")
    assert st["n_converged"] == w.n_systems
    _, o = oracle_run(w)
    bar = 1e-6 if precision == "fp64" else 1e-5
    assert rel_err(rho, o.rho) <= bar
    assert rel_err(e, o.e_node) <= bar


def test_shifted_does_fewer_matvecs():
    w = make_workload("bulk_mixed").subset(np.arange(3))
    _, _, st_ms = _run(w, "mixed", "shifted")
    _, _, st_pp = _run(w, "mixed", "cocg")
    assert st_ms["total_point_iters"] < 0.5 * st_pp["total_point_iters"]


def test_shifted_uneven_and_ring_regions():
    w = make_workload("screw_batched")
    hw = w.halfwidth
    pick = [int(np.argmax(hw)), int(np.argmin(hw)), int(np.argsort(hw)[len(hw) // 2])]
    ws = w.subset(np.array(pick))
    rho, _, st = _run(ws, "mixed", "shifted")
    _, o = oracle_run(ws)
    assert rel_err(rho, o.rho) <= 1e-5
    wt = make_workload("tiny", shape=(6, 12, 8), fd_order=4, s=4, n_nodes=5)   # rings on x, z
    wt.tol = 1e-11
    rho, _, _ = _run(wt, "fp64", "shifted")
    _, o = oracle_run(wt)
    assert rel_err(rho, o.rho) <= 1e-6


def test_shifted_refuses_checkpoint():
    from paper_1907_02604_gb300 import Hamiltonian, Plan, SolverOptions, Workspace, make_poles
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_INVALID
    w = make_workload("tiny")
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    ws = Workspace(ham, w.nodes, w.halfwidth, w.n_poles)
    with pytest.raises(MacroDFTError) as ei:
        Plan(ham, z, wt, w.nodes, w.halfwidth, SolverOptions(method="shifted"), checkpoint=ws)
    assert ei.value.status == MD_ERR_INVALID
