"""GPU parity of the cluster kernel (SolverOptions(kernel="cluster")): each
(node, pole) system runs on one thread-block cluster whose CTAs hold z-slabs
of the Krylov vectors in shared memory and read their halo planes from the
neighbouring CTAs.  Against the FP64 oracle at the mixed bar (1e-5 relative
density error), and against the generic kernel for the fused adjoint and the
density-matrix rows.  Small regions are also run with forced cluster sizes,
so that slabs are thinner than the stencil half-width (halo planes held two
or more CTAs away) or empty (more CTAs than planes)."""
import numpy as np
import pytest

from synthetic import make_workload
from tests.gpu_helpers import gpu_run, oracle_run, rel_err, rel_err_per_node

pytestmark = pytest.mark.gpu

MIXED_BAR = 1e-5

CASES = [   # regions without whole-axis rings
    dict(shape=(9, 10, 11), fd_order=2, s=3),
    dict(shape=(9, 10, 11), fd_order=4, s=2, n_nodes=7),
    dict(shape=(8, 8, 8), fd_order=8, s=2, spacing=(0.5, 0.5, 0.5)),       # 5^3 regions, Q = 4
    dict(shape=(18, 18, 18), fd_order=8, s=3, nonlocal_proj=True, n_atoms=6, spacing=(0.5, 0.5, 0.5)),
    dict(shape=(14, 12, 16), fd_order=4, s=3, periodic=(False, True, False)),
]


def _inside_open_axes(w):
    if all(w.periodic):
        return w
    c = w.node_coords()
    ok = np.ones(len(w.nodes), bool)
    for d in range(3):
        if not w.periodic[d]:
            ok &= (c[:, d] - w.halfwidth >= 0) & (c[:, d] + w.halfwidth < w.shape[d])
    return w.subset(np.nonzero(ok)[0])


@pytest.mark.parametrize("csz", [1, 2, 3, 8])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_tiny_cases_forced_cluster_size(case, csz):
    w = _inside_open_axes(make_workload("tiny", **CASES[case]))
    assert len(w.nodes) > 0
    w.tol = 1e-11
    g = gpu_run(w, precision="mixed", kernel="cluster", ctas_per_sm=csz)
    _, o = oracle_run(w)
    assert g["stats"]["n_converged"] == w.n_systems
    assert rel_err(g["rho"], o.rho) <= MIXED_BAR
    assert rel_err(g["e"], o.e_node) <= MIXED_BAR
    assert rel_err_per_node(g["rho"], o.rho) <= MIXED_BAR


@pytest.mark.parametrize("csz", [0, 2, 4])
def test_ragged_region_sizes_in_one_launch(csz):
    w = make_workload("tiny", shape=(20, 20, 20), n_nodes=9, s=2, spacing=(0.5, 0.5, 0.5), n_atoms=6,
                      nonlocal_proj=True, fd_order=8)
    w.halfwidth = np.array([1, 2, 3, 4, 5, 6, 7, 8, 0], dtype=np.int32)
    w.tol = 1e-11
    g = gpu_run(w, precision="mixed", kernel="cluster", ctas_per_sm=csz)
    _, o = oracle_run(w)
    assert rel_err(g["rho"], o.rho) <= MIXED_BAR
    assert rel_err(g["e"], o.e_node) <= MIXED_BAR


def test_bulk_subset_vs_oracle():
    """1,024 atoms, 8th order, projectors, 33^3 regions, P = 16."""
    w = make_workload("bulk_mixed").subset(np.arange(3))
    g = gpu_run(w, precision="mixed", kernel="cluster")
    _, o = oracle_run(w)
    assert g["stats"]["n_converged"] == w.n_systems
    assert g["stats"]["reliable_updates"] > 0
    assert rel_err(g["rho"], o.rho) <= MIXED_BAR
    assert rel_err(g["e"], o.e_node) <= MIXED_BAR
    assert rel_err_per_node(g["rho"], o.rho) <= MIXED_BAR


def test_screw_sample_open_axes_vs_oracle():
    """Cylinder with open x, y axes; the largest and smallest regions."""
    w = make_workload("screw_batched")
    hw = w.halfwidth
    ws = w.subset(np.array([int(np.argmax(hw)), int(np.argmin(hw)), int(np.argsort(hw)[len(hw) // 2])]))
    g = gpu_run(ws, precision="mixed", kernel="cluster")
    _, o = oracle_run(ws)
    assert g["stats"]["n_converged"] == ws.n_systems
    assert rel_err(g["rho"], o.rho) <= MIXED_BAR


def test_matches_generic_kernel():
    """Same systems through the generic kernel and the cluster kernel."""
    w = make_workload("bulk_mixed").subset(np.arange(8))
    a = gpu_run(w, precision="mixed", kernel="cluster")
    b = gpu_run(w, precision="mixed", kernel="generic", block=512)
    assert rel_err(a["rho"], b["rho"]) <= MIXED_BAR
    assert rel_err(a["e"], b["e"]) <= MIXED_BAR


def test_fused_adjoint_matches_generic():
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density_fused_adjoint, make_poles
    w = make_workload("adjoint_fp64").subset(np.arange(6))
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    rng = np.random.default_rng(3)
    a = torch.tensor(rng.normal(size=6), dtype=torch.float64, device="cuda")
    b = torch.tensor(rng.normal(size=6), dtype=torch.float64, device="cuda")
    out = {}
    for kern, blk in (("cluster", 0), ("generic", 512)):
        opts = SolverOptions(tol=1e-10, precision="mixed", kernel=kern, block=blk)
        rho, e, g, F, st = density_fused_adjoint(ham, z, wt, w.nodes, w.halfwidth, a, b, opts, forces=True)
        assert st["n_converged"] == w.n_systems
        out[kern] = [t.cpu().numpy() for t in (rho, e, g, F)]
    for x, y in zip(out["cluster"], out["generic"]):
        assert rel_err(x, y) <= MIXED_BAR


def test_density_matrix_rows_match_oracle():
    from oracle import density as od
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density_matrix_rows, make_poles
    w = make_workload("bulk_mixed").subset(np.arange(2))
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    rho, _, rows, off = density_matrix_rows(ham, z, wt, w.nodes, w.halfwidth,
                                            SolverOptions(tol=1e-10, precision="mixed", kernel="cluster"))
    rows = rows.cpu().numpy()
    res = od.solve(w, od.build(w), tol=1e-12, keep_x=True)
    ro = od.density_matrix_rows(res)
    for j in range(len(w.nodes)):
        r = rows[off[j]:off[j + 1]]
        assert np.abs(r - ro[j]).max() <= MIXED_BAR * np.abs(ro[j]).max()


def test_deadline_and_maxit_end_the_launch():
    """The cluster-uniform stop paths: the kernel's own deadline (rank 0's
    clock, shared with the cluster) and the iteration cap."""
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density, make_poles
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_TIMEOUT
    w = make_workload("bulk_mixed").subset(np.arange(16))
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    with pytest.raises(MacroDFTError) as ei:
        density(ham, z, wt, w.nodes, w.halfwidth,
                SolverOptions(tol=1e-14, maxit=10 ** 6, timeout_s=1e-4, precision="mixed", kernel="cluster"))
    assert ei.value.status == MD_ERR_TIMEOUT
    torch.cuda.synchronize()
    rho, _, st = density(ham, z, wt, w.nodes[:2], w.halfwidth[:2],
                         SolverOptions(tol=1e-10, maxit=20, precision="mixed", kernel="cluster"), strict=False)
    assert st["status"] == "MD_ERR_NOCONV" and st["iters_max"] == 20
    assert np.isfinite(rho.cpu().numpy()).all()
