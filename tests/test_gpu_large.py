"""The large configuration: a 100,000-atom hcp cylinder with a prismatic
loop and a line of Al-like wells (642 x 642 x 472 grid, 8th order, P = 16,
mixed): a sample of nodes against the oracle, a 1,000-node batch in one
launch, and band-energy forces from the fused adjoint on the sites nearest
the loop line."""
import numpy as np
import pytest

from synthetic import make_workload
from tests.gpu_helpers import rel_err
from tests.oracle_pins_helpers import golden_fd_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    from paper_1907_02604_gb300 import Hamiltonian
    w = make_workload("large_loop")
    return w, Hamiltonian.from_workload(w)


def _interval(w):
    """Spectral interval from the workload definition alone (an input to
    both sides): the FD kinetic operator of a window is positive
    semidefinite and below its Gershgorin bound
    sum_d (|w_0| + 2 sum_o |w_o|) / (2 h_d^2); V = -sum D exp(...) + noise
    lies above -4 Ha (three fully overlapping wells of the deepest kind) and
    below the noise amplitude.  The GPU's Gershgorin interval is looser below
    (negative off-diagonal sums) and must contain this one."""
    fw = golden_fd_weights()[w.fd_order]
    kin = sum((abs(fw[0]) + 2.0 * np.abs(fw[1:]).sum()) / (2.0 * h * h) for h in w.spacing)
    return -4.0, kin + 0.1


def _sample(w):
    hw = w.halfwidth
    al = w.atoms[w.meta["al_atoms"]].mean(axis=0)
    c = w.node_coords() * np.array(w.spacing)
    near_al = int(np.argmin(np.linalg.norm(c - al, axis=1)))
    return np.array(sorted({int(np.argmax(hw)), int(np.argmin(hw)), near_al, 1000}))


def test_large_sample_vs_oracle_and_fused_forces(large):
    import torch
    from oracle import density as od
    from paper_1907_02604_gb300 import Plan, SolverOptions, density_fused_adjoint, make_poles
    from oracle.poles import fermi_poles
    w, ham = large
    lo, hi = _interval(w)
    g_lo, g_hi = ham.spectral_bounds()
    assert g_lo <= lo and g_hi <= hi       # Gershgorin encloses more loosely
    ws = w.subset(_sample(w))
    z, wt = make_poles(w.kT, w.mu, lo, hi, w.n_poles)
    opts = SolverOptions(tol=1e-10, precision="mixed")
    plan = Plan(ham, z, wt, ws.nodes, ws.halfwidth, opts)
    plan.launch()
    assert plan.stats()["n_converged"] == ws.n_systems
    rho = plan.rho.cpu().numpy()
    plan.close()
    b = torch.ones(len(ws.nodes), dtype=torch.float64, device="cuda")
    _, e_f, _, F, st = density_fused_adjoint(ham, z, wt, ws.nodes, ws.halfwidth, None, b, opts, forces=True)
    assert st["n_converged"] == ws.n_systems

    H = od.build(ws, points=od.region_points(ws), bounds=(lo, hi))
    zo, wo = fermi_poles(w.kT, w.mu, lo, hi, w.n_poles)
    res = od.solve(ws, H, zo, wo, tol=1e-12, keep_x=True)
    assert np.all(res.status == 0)
    assert rel_err(rho, res.rho) <= 1e-5
    assert rel_err(e_f.cpu().numpy(), res.e_node) <= 1e-5
    atoms = w.meta["force_atoms"]
    Fo = od.forces(ws, od.dL_dV(ws, res, np.zeros(len(ws.nodes)), np.ones(len(ws.nodes))), atoms=atoms)
    Fg = F.cpu().numpy()[atoms]
    assert np.abs(Fo).max() > 0
    assert rel_err(Fg, Fo) <= 1e-5


def test_large_batch_one_launch(large):
    """1,000 nodes (16,000 systems, regions 17^3..41^3) in one graph launch."""
    from paper_1907_02604_gb300 import Plan, SolverOptions, make_poles
    w, ham = large
    ws = w.subset(np.arange(1000))
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    plan = Plan(ham, z, wt, ws.nodes, ws.halfwidth, SolverOptions(tol=1e-10, precision="mixed"))
    plan.launch()
    st = plan.stats(strict=False)
    assert st["n_systems"] == 16000
    assert st["n_converged"] == 16000, st
    rho = plan.rho.cpu().numpy()
    assert np.isfinite(rho).all()
    plan.close()
