"""Locality of the nodal density (Section 2.1: the density at a node is
evaluated on a region around it; Section 4 studies how the fields converge
with the region size).  At finite temperature the entries of f(H) decay
exponentially with distance, and faster the larger kT, so the truncation
error |rho_j(s) - rho_j(whole cell)| of the region-restricted density falls
geometrically with the half-width s.  At kT = 1 Ha the decay is fast enough
to show on a 16^3 cell."""
import numpy as np

from oracle import density as od
from synthetic import make_workload


def _curve():
    w = make_workload("tiny", shape=(16, 16, 16), spacing=(0.5, 0.5, 0.5), fd_order=4, n_atoms=8, n_nodes=4, s=1)
    w.n_poles, w.kT, w.mu = 32, 1.0, 2.0
    H = od.build(w)
    rho = {}
    for s in range(1, 9):           # 2s + 1 >= 16 at s = 8: the whole periodic cell
        w.halfwidth = np.full(len(w.nodes), s, np.int32)
        rho[s] = od.solve(w, H, tol=1e-12).rho
    return rho


def test_truncation_error_decays_geometrically():
    rho = _curve()
    ref = rho[8]
    assert np.all(ref > 0.0)
    err = [np.abs(rho[s] - ref).max() / np.abs(ref).max() for s in range(1, 8)]
    # each step of s at least halves the error up to s = 6 (a region of
    # 13^3 in a 16^3 cell), and the 13^3 region is within 1e-3
    for s in range(5):
        assert err[s + 1] < 0.5 * err[s], (s + 1, err)
    assert err[5] < 1e-3, err
