"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars: relative density error max|rho_gpu - rho_oracle| / max|rho_oracle|
<= 1e-6 in FP64 mode and <= 1e-5 in mixed mode (the stated targets); the
same bars for the band energy per node; potentials and spectral bounds to
FP64 rounding.  Inputs are the seeded synthetic workloads.
"""
import numpy as np
import pytest

from synthetic import make_workload
from tests.gpu_helpers import gpu_run, oracle_run, rel_err

pytestmark = pytest.mark.gpu

FP64_BAR = 1e-6
MIXED_BAR = 1e-5


def test_potential_matches_oracle():
    from oracle import hamiltonian as oh
    from paper_1907_02604_gb300 import Hamiltonian
    for w in [make_workload("small_fp64"), make_workload("tiny", shape=(7, 9, 11), n_atoms=5),
              make_workload("tiny", shape=(12, 10, 9), periodic=(False, True, False), s=2)]:
        ham = Hamiltonian.from_workload(w)
        V = ham.potential().cpu().numpy()
        Vo = oh.local_potential(w)
        assert np.max(np.abs(V - Vo)) < 1e-12


def test_spectral_bounds_match_oracle():
    from oracle import density as od
    from paper_1907_02604_gb300 import Hamiltonian
    w = make_workload("tiny", shape=(18, 18, 20), spacing=(0.5, 0.5, 0.45), nonlocal_proj=True,
                      n_atoms=6, fd_order=8)
    H = od.build(w)
    lo, hi = Hamiltonian.from_workload(w).spectral_bounds()
    assert abs(lo - H.emin) < 1e-10 * abs(H.emin) and abs(hi - H.emax) < 1e-10 * abs(H.emax)


def test_small_fp64_full_workload():
    """16 atoms, 24x24x40, 4th order, P = 8, 32 nodes with 21^3 regions."""
    w = make_workload("small_fp64")
    g = gpu_run(w)
    _, o = oracle_run(w)
    assert g["stats"]["n_converged"] == w.n_systems
    assert rel_err(g["rho"], o.rho) <= FP64_BAR
    assert rel_err(g["e"], o.e_node) <= FP64_BAR


TINY_CASES = [
    dict(shape=(9, 10, 11), fd_order=2, s=3),
    dict(shape=(9, 10, 11), fd_order=4, s=2, n_nodes=7),
    dict(shape=(8, 8, 8), fd_order=8, s=2, spacing=(0.5, 0.5, 0.5)),
    dict(shape=(6, 6, 8), fd_order=4, s=10, n_nodes=3),          # whole-axis rings
    dict(shape=(6, 12, 8), fd_order=4, s=4, n_nodes=5),          # rings on x, z; window on y
    dict(shape=(18, 18, 18), fd_order=8, s=3, nonlocal_proj=True, n_atoms=6, spacing=(0.5, 0.5, 0.5)),
    dict(shape=(18, 20, 17), fd_order=4, s=9, nonlocal_proj=True, n_atoms=4, n_nodes=3,
         spacing=(0.5, 0.45, 0.55)),
    dict(shape=(14, 12, 16), fd_order=4, s=3, periodic=(False, True, False)),
]


@pytest.mark.parametrize("case", range(len(TINY_CASES)))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tiny_cases(case, precision):
    kw = dict(TINY_CASES[case])
    w = make_workload("tiny", **kw)
    if not all(w.periodic):
        # keep every region inside the open axes
        c = w.node_coords()
        ok = np.ones(len(w.nodes), bool)
        for d in range(3):
            if not w.periodic[d]:
                ok &= (c[:, d] - w.halfwidth >= 0) & (c[:, d] + w.halfwidth < w.shape[d])
        w = w.subset(np.nonzero(ok)[0])
        assert len(w.nodes) > 0
    w.tol = 1e-11
    g = gpu_run(w, precision=precision)
    _, o = oracle_run(w)
    bar = FP64_BAR if precision == "fp64" else MIXED_BAR
    assert rel_err(g["rho"], o.rho) <= bar
    assert rel_err(g["e"], o.e_node) <= bar


def test_ragged_region_sizes_in_one_launch():
    w = make_workload("tiny", shape=(20, 20, 20), n_nodes=9, s=2, spacing=(0.5, 0.5, 0.5), n_atoms=6)
    w.halfwidth = np.array([1, 2, 3, 4, 5, 6, 7, 8, 0], dtype=np.int32)
    w.tol = 1e-11
    for precision in ("fp64", "mixed"):
        g = gpu_run(w, precision=precision)
        _, o = oracle_run(w)
        assert rel_err(g["rho"], o.rho) <= (FP64_BAR if precision == "fp64" else MIXED_BAR)


def test_bulk_mixed_subset_both_precisions():
    """1,024 atoms, 8th order, nonlocal projectors, 33^3 regions, P = 16."""
    w = make_workload("bulk_mixed").subset(np.arange(3))
    _, o = oracle_run(w)
    gm = gpu_run(w, precision="mixed")
    gd = gpu_run(w, precision="fp64")
    assert rel_err(gm["rho"], o.rho) <= MIXED_BAR
    assert rel_err(gd["rho"], o.rho) <= FP64_BAR
    assert rel_err(gm["e"], o.e_node) <= MIXED_BAR
    assert gm["stats"]["reliable_updates"] > 0


def test_checkpoint_does_not_change_result():
    w = make_workload("tiny", shape=(10, 10, 10), s=3, n_nodes=4, spacing=(0.5, 0.5, 0.5))
    a = gpu_run(w)
    b = gpu_run(w, checkpoint=True)
    np.testing.assert_array_equal(a["rho"], b["rho"])


def test_energy_entry_point():
    from paper_1907_02604_gb300 import energy
    w = make_workload("tiny", shape=(10, 10, 10), s=3, n_nodes=4, spacing=(0.5, 0.5, 0.5))
    g = gpu_run(w)
    e, eb, _ = energy(g["ham"], g["z"], g["w"], w.nodes, w.halfwidth, g["opts"])
    np.testing.assert_allclose(e.cpu().numpy(), g["e"], rtol=0, atol=0)
    assert abs(eb - g["e"].sum()) <= 1e-12 * abs(eb)


def test_empty_node_list():
    from paper_1907_02604_gb300 import Hamiltonian, density, make_poles
    w = make_workload("tiny")
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), 8)
    rho, _, st = density(ham, z, wt, np.zeros(0, np.int64), np.zeros(0, np.int32))
    assert rho.numel() == 0 and st["n_systems"] == 0


def test_maxit_reports_noconv_with_outputs():
    w = make_workload("tiny", shape=(10, 10, 10), s=3, n_nodes=2, spacing=(0.5, 0.5, 0.5))
    w.maxit = 3
    g = gpu_run(w, strict=False)
    assert g["stats"]["status"] == "MD_ERR_NOCONV"
    assert g["stats"]["n_noconv"] > 0 and np.all(np.isfinite(g["rho"]))


def test_device_deadline_returns_timeout():
    """The kernel's own wall-clock check ends the launch (no fault)."""
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density, make_poles
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_TIMEOUT
    w = make_workload("small_fp64")
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    opts = SolverOptions(tol=1e-14, maxit=10 ** 6, timeout_s=1e-4)
    with pytest.raises(MacroDFTError) as ei:
        density(ham, z, wt, w.nodes, w.halfwidth, opts)
    assert ei.value.status == MD_ERR_TIMEOUT
    torch.cuda.synchronize()   # the context is still usable
    rho, _, _ = density(ham, z, wt, w.nodes[:1], w.halfwidth[:1], SolverOptions(tol=1e-10))
    assert np.isfinite(rho.cpu().numpy()).all()


@pytest.mark.parametrize("bad", ["node", "open_axis", "pole", "opts"])
def test_invalid_inputs_raise(bad):
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density, make_poles
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_INVALID
    w = make_workload("tiny", shape=(12, 10, 9), periodic=(False, True, True), s=2)
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), 8)
    nodes, hw, opts = np.array([5 + 12 * 3]), np.array([2], np.int32), SolverOptions()
    if bad == "node":
        nodes = np.array([w.n_grid])
    elif bad == "open_axis":
        nodes = np.array([0])
    elif bad == "pole":
        z = z.conj()
    elif bad == "opts":
        opts = SolverOptions(tol=-1.0)
    with pytest.raises(MacroDFTError) as ei:
        density(ham, z, wt, nodes, hw, opts)
    assert ei.value.status == MD_ERR_INVALID


@pytest.mark.parametrize("n_poles", [2, 64])
def test_fewest_and_most_poles(n_poles):
    """P = 2 (one trapezoid node) and P = 64 (the shifted-COCG maximum), per
    pole and shifted, against the oracle."""
    w = make_workload("tiny", shape=(9, 10, 11), fd_order=4, s=2, n_nodes=4, n_poles=n_poles)
    w.tol = 1e-11
    _, o = oracle_run(w)
    for method in ("cocg", "shifted"):
        g = gpu_run(w, precision="fp64", method=method)
        assert rel_err(g["rho"], o.rho) <= FP64_BAR, method
        assert rel_err(g["e"], o.e_node) <= FP64_BAR, method


@pytest.mark.parametrize("method", ["cocg", "shifted"])
def test_mixed_points_over_four_projector_atoms(method):
    """Twelve atoms in a 9-bohr cell: in every 9^3 region some points lie in
    the spheres of more than four atoms (the solver's CSR path) and the rest
    in at most four (its per-point records); both meet the mixed bar."""
    w = make_workload("tiny", shape=(18, 18, 18), spacing=(0.5, 0.5, 0.5), fd_order=8, s=4,
                      nonlocal_proj=True, n_atoms=12, n_nodes=4)
    # 32 poles at kT = 0.05 resolve f on this cell's wide spectrum (the
    # densities are within 1e-3 of the dense f(H)_jj)
    w.n_poles, w.kT, w.mu, w.tol = 32, 0.05, 2.0, 1e-11
    g = gpu_run(w, precision="mixed", method=method)
    _, o = oracle_run(w)
    assert rel_err(g["rho"], o.rho) <= MIXED_BAR
    assert rel_err(g["e"], o.e_node) <= MIXED_BAR


def test_region_halfwidth_sweep_matches_oracle():
    """The locality sweep (s = 1 .. the whole cell) through the C ABI: every
    half-width agrees with the oracle, so the truncation curve the GPU
    reports is the oracle's."""
    w = make_workload("tiny", shape=(16, 16, 16), spacing=(0.5, 0.5, 0.5), fd_order=4, n_atoms=8, n_nodes=4, s=1)
    w.n_poles, w.kT, w.mu, w.tol = 32, 1.0, 2.0, 1e-11
    for s in (1, 3, 5, 8):
        w.halfwidth = np.full(len(w.nodes), s, np.int32)
        g = gpu_run(w, precision="fp64")
        _, o = oracle_run(w)
        assert rel_err(g["rho"], o.rho) <= FP64_BAR, s


@pytest.mark.slow
def test_bulk_64_nodes_both_precisions_vs_oracle():
    """The bulk workload's stated check: 64 nodes (1,024 systems, 33^3
    regions, projectors, P = 16) against the FP64 oracle, in mixed precision
    (bar 1e-5) and in the FP64 form (bar 1e-6), on the density, the band
    energy and, per node, the density of every node above 1e-3 of the
    largest."""
    from tests.gpu_helpers import rel_err_per_node
    w = make_workload("bulk_mixed").subset(np.arange(64))
    _, o = oracle_run(w)
    for precision, bar in (("mixed", MIXED_BAR), ("fp64", FP64_BAR)):
        g = gpu_run(w, precision=precision)
        assert g["stats"]["n_converged"] == w.n_systems, precision
        assert rel_err(g["rho"], o.rho) <= bar, precision
        assert rel_err(g["e"], o.e_node) <= bar, precision
        assert rel_err_per_node(g["rho"], o.rho) <= bar, precision
