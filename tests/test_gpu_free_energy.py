"""GPU parity of the free-energy terms and the pole-form Fermi level.

* md_free_energy: rho_j, e_j and the entropy term s_j (last term of Eq. tot,
  from the entropy weights on the same poles) per node, and the
  node-weighted totals N_e, E_band, TS and F = E_band - TS, against the FP64
  oracle (1e-6 in FP64, 1e-5 in mixed precision);
* the cluster-sampled energy of Section 3 (Eqs. free_cg, free_cg_sampling)
  end to end: the library's cluster nodes and weights feed md_free_energy,
  the oracle's feed the oracle;
* md_energy's node weights;
* md_fermi_level_poles against the oracle's bisection and, on a free-electron
  cell, against a Brent root of the closed-form count.
"""
from dataclasses import replace

import numpy as np
import pytest

from synthetic import make_workload
from synthetic.workloads import Workload
from tests.gpu_helpers import rel_err, rel_err_per_node

pytestmark = pytest.mark.gpu


def _gpu_terms(w, precision, node_weight=None, kernel="auto"):
    import torch
    from paper_1907_02604_gb300 import (Hamiltonian, SolverOptions, free_energy, make_entropy_weights,
                                        make_poles)
    ham = Hamiltonian.from_workload(w)
    lo, hi = ham.spectral_bounds()
    z, wt = make_poles(w.kT, w.mu, lo, hi, w.n_poles)
    ws = make_entropy_weights(w.kT, w.mu, lo, hi, w.n_poles)
    nu = None if node_weight is None else torch.tensor(node_weight, dtype=torch.float64, device="cuda")
    rho, e, s, terms, st = free_energy(ham, z, wt, ws, w.kT, w.nodes, w.halfwidth,
                                       SolverOptions(tol=w.tol, precision=precision, kernel=kernel),
                                       node_weight=nu)
    return rho.cpu().numpy(), e.cpu().numpy(), s.cpu().numpy(), terms, st


def _oracle_terms(w, node_weight=None):
    from oracle import density as od
    from oracle.poles import entropy_weights
    H = od.build(w)
    res = od.solve(w, H, tol=1e-12)
    ws = entropy_weights(w.kT, w.mu, H.emin, H.emax, w.n_poles)
    return res, od.free_energy_terms(w, res, ws, node_weight)


@pytest.mark.parametrize("name,precision,bar", [("small_fp64", "fp64", 1e-6), ("bulk_mixed", "mixed", 1e-5)])
def test_free_energy_matches_oracle(name, precision, bar):
    w = make_workload(name).subset(np.arange(6))
    nu = np.random.default_rng(11).uniform(0.5, 40.0, 6)
    rho, e, s, t, st = _gpu_terms(w, precision, nu)
    res, to = _oracle_terms(w, nu)
    assert st["n_converged"] == w.n_systems
    assert rel_err(rho, res.rho) <= bar
    assert rel_err(e, res.e_node) <= bar
    assert rel_err(s, to["s_node"]) <= bar
    assert rel_err_per_node(s, to["s_node"]) <= bar
    for k in ("n_electrons", "e_band", "ts", "free_energy"):
        assert abs(t[k] - to[k]) <= bar * max(abs(to[k]), abs(to["e_band"])), k
    assert t["free_energy"] == t["e_band"] - t["ts"]


def test_cluster_sampled_energy_end_to_end():
    """ESPs of the small cell with coarse-graining weights n_q; clusters of
    radius 1 bohr around each; the weighted sum over the cluster points."""
    from oracle import density as od
    from paper_1907_02604_gb300 import cluster_sampling
    w = make_workload("small_fp64")
    esp = w.nodes[:5]
    n_q = np.array([1.0, 1.0, 8.0, 27.0, 64.0])
    nodes, nu = cluster_sampling(w.shape, w.spacing, w.periodic, esp, n_q, 1.0)
    no, nuo = od.cluster_sampling(w, esp, n_q, 1.0)
    np.testing.assert_array_equal(nodes, no)
    wc = replace(w, nodes=nodes, halfwidth=np.full(len(nodes), int(w.halfwidth[0]), np.int32))
    rho, e, s, t, _ = _gpu_terms(wc, "fp64", nu)
    _, to = _oracle_terms(wc, nuo)
    for k in ("n_electrons", "e_band", "ts", "free_energy"):
        assert abs(t[k] - to[k]) <= 1e-6 * max(abs(to[k]), abs(to["e_band"])), k
    assert abs(np.sum(nu) - n_q.sum()) < 1e-12


def test_energy_node_weights():
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, energy, make_poles
    w = make_workload("small_fp64").subset(np.arange(5))
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    nu = np.array([1.0, 3.0, 0.5, 2.0, 7.0])
    e, eb, _ = energy(ham, z, wt, w.nodes, w.halfwidth, SolverOptions(tol=1e-10),
                      node_weight=torch.tensor(nu, dtype=torch.float64, device="cuda"))
    res, _ = _oracle_terms(w)
    assert abs(eb - np.sum(nu * res.e_node)) <= 1e-6 * abs(np.sum(nu * res.e_node))
    assert abs(eb - np.sum(nu * e.cpu().numpy())) <= 1e-12 * abs(eb)


def test_free_energy_cluster_kernel_mixed():
    w = make_workload("bulk_mixed").subset(np.arange(4))
    rho, e, s, t, st = _gpu_terms(w, "mixed", kernel="cluster")
    res, to = _oracle_terms(w)
    assert rel_err(s, to["s_node"]) <= 1e-5
    assert abs(t["ts"] - to["ts"]) <= 1e-5 * abs(to["ts"])


def _free_electron(shape=(4, 4, 6), spacing=(0.6, 0.6, 0.5)):
    n = int(np.prod(shape))
    return Workload(name="free", shape=shape, spacing=spacing, periodic=(True, True, True),
                    fd_order=4, atoms=np.zeros((0, 3)), depth=np.zeros(0), sigma=np.zeros(0),
                    v_ext=np.zeros(n), nodes=np.arange(n), halfwidth=np.full(n, 10, np.int32),
                    n_poles=16, tol=1e-12)


def test_fermi_level_poles_free_electron_closed_form():
    from scipy.optimize import brentq

    from oracle.poles import fermi_poles, rational
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, fermi_level_poles
    from tests.oracle_pins_helpers import fd_symbol, golden_fd_weights
    w = _free_electron()
    ham = Hamiltonian.from_workload(w)
    lo, hi = ham.spectral_bounds()
    wts = golden_fd_weights()[w.fd_order]
    eps = np.zeros(w.shape[::-1])
    for d, (n, h) in enumerate(zip(w.shape, w.spacing)):
        sh = [1, 1, 1]
        sh[2 - d] = n
        eps = eps + fd_symbol(2 * np.pi * np.fft.fftfreq(n, d=h), h, wts).reshape(sh)
    eps = eps.reshape(-1)
    target = 20.0
    mu_ref = brentq(lambda m: 2.0 * rational(eps, *fermi_poles(w.kT, m, lo, hi, w.n_poles)).sum() - target,
                    lo, hi, xtol=1e-13)
    mu, cnt, evals = fermi_level_poles(ham, w.kT, w.n_poles, w.nodes, w.halfwidth, target,
                                       SolverOptions(tol=1e-12, precision="fp64"), mu_tol=1e-11)
    assert abs(mu - mu_ref) < 1e-8
    assert abs(cnt - target) < 1e-6
    assert evals < 60


def test_fermi_level_poles_matches_oracle_bisection():
    import torch
    from oracle import density as od
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, fermi_level_poles
    w = make_workload("tiny", shape=(6, 6, 6), s=2, n_atoms=3, spacing=(0.6, 0.6, 0.6), n_nodes=12)
    w.tol = 1e-12
    nu = np.full(12, w.n_grid / 12.0)
    H = od.build(w)
    mu_o, n_o, _ = od.fermi_level_poles(w, H, 9.0, node_weight=nu, mu_tol=1e-11)
    ham = Hamiltonian.from_workload(w)
    mu, cnt, _ = fermi_level_poles(ham, w.kT, w.n_poles, w.nodes, w.halfwidth, 9.0,
                                   SolverOptions(tol=1e-12, precision="fp64"),
                                   node_weight=torch.tensor(nu, dtype=torch.float64, device="cuda"), mu_tol=1e-11)
    assert abs(mu - mu_o) < 1e-8
    assert abs(cnt - 9.0) < 1e-6


def test_fermi_level_poles_rejects_unreachable_count():
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, fermi_level_poles
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_INVALID
    w = _free_electron()
    ham = Hamiltonian.from_workload(w)
    with pytest.raises(MacroDFTError) as ei:
        fermi_level_poles(ham, w.kT, w.n_poles, w.nodes, w.halfwidth, 10.0 * w.n_grid,
                          SolverOptions(tol=1e-10, precision="fp64"))
    assert ei.value.status == MD_ERR_INVALID
