"""Density-matrix rows gamma_jk = sum_p Im(w_p x_jp(k)) over each region
(Eq. dm in the grid basis) against the oracle, their diagonal against rho,
and symmetry gamma_jk = gamma_kj where regions cover the whole cell."""
import numpy as np
import pytest

from synthetic import make_workload

pytestmark = pytest.mark.gpu


def _gpu(w, precision, tol):
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density_matrix_rows, make_poles
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    rho, e, rows, off = density_matrix_rows(ham, z, wt, w.nodes, w.halfwidth,
                                            SolverOptions(tol=tol, precision=precision))
    rows = rows.cpu().numpy()
    return rho.cpu().numpy(), [rows[off[j]:off[j + 1]] for j in range(len(w.nodes))]


@pytest.mark.parametrize("name,precision,bar", [("small_fp64", "fp64", 1e-6), ("small_fp64", "mixed", 1e-5),
                                                ("bulk_mixed", "mixed", 1e-5)])
def test_rows_match_oracle(name, precision, bar):
    from oracle import density as od
    w = make_workload(name).subset(np.arange(3))
    rho, rows = _gpu(w, precision, 1e-10)
    res = od.solve(w, od.build(w), tol=1e-12, keep_x=True)
    ro = od.density_matrix_rows(res)
    for j in range(len(w.nodes)):
        assert rows[j].shape == ro[j].shape
        assert np.abs(rows[j] - ro[j]).max() <= bar * np.abs(ro[j]).max()
        src = res.regions[j].src
        assert abs(2.0 / w.dV * rows[j][src] - rho[j]) <= 1e-12 * abs(rho[j]) + 1e-14


def test_rows_symmetric_on_whole_cell():
    w = make_workload("tiny", shape=(5, 6, 7), s=10, n_nodes=3)
    w.tol = 1e-12
    _, rows = _gpu(w, "fp64", 1e-12)
    g = [int(n) for n in w.nodes]
    for a in range(3):
        for b in range(3):
            assert abs(rows[a][g[b]] - rows[b][g[a]]) <= 1e-9 * np.abs(rows[a]).max()


def test_rows_refuse_shifted_and_accept_empty():
    """The rows need every pole's own solution vector, which shifted COCG
    does not keep; an empty node list returns empty outputs."""
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density_matrix_rows, make_poles
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_INVALID
    w = make_workload("tiny")
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    with pytest.raises(MacroDFTError) as ei:
        density_matrix_rows(ham, z, wt, w.nodes, w.halfwidth, SolverOptions(method="shifted"))
    assert ei.value.status == MD_ERR_INVALID
    rho, e, rows, off = density_matrix_rows(ham, z, wt, w.nodes[:0], w.halfwidth[:0])
    assert rho.numel() == 0 and rows.numel() == 0 and list(off) == [0]
