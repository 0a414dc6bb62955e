"""The seeded workload generators: sizes, seeds and geometric invariants
(no GPU; the large configuration is checked at a reduced size)."""
import math

import numpy as np

from synthetic import make_workload
from synthetic.workloads import A_LAT, C_LAT, large_loop


def _regions_inside(w):
    c = w.node_coords()
    for d in range(3):
        if not w.periodic[d]:
            assert np.all(c[:, d] - w.halfwidth >= 0)
            assert np.all(c[:, d] + w.halfwidth < w.shape[d])


def test_periodic_cells():
    for name, n_atoms, shape, n_nodes in (("small_fp64", 16, (24, 24, 40), 32),
                                          ("bulk_mixed", 1024, (96, 96, 160), 4096),
                                          ("adjoint_fp64", 128, (48, 48, 80), 1024)):
        w = make_workload(name)
        assert len(w.atoms) == n_atoms and w.shape == shape and len(w.nodes) == n_nodes
        assert len(np.unique(w.nodes)) == n_nodes
        assert np.all((w.atoms >= 0) & (w.atoms < np.array(w.box)))
        assert np.all(np.abs(w.v_ext) <= 0.05)


def test_screw_cylinder():
    w = make_workload("screw_batched")
    assert len(w.atoms) == 4000 and w.n_systems == 20000
    assert w.halfwidth.min() == 8 and w.halfwidth.max() == 20
    _regions_inside(w)


def test_large_loop_reduced():
    """The large generator at 1/20 of the atoms: site count, the Al-like
    line, force atoms nearest the loop line, open-axis regions inside the
    grid, half-widths in [8, 20], displacement at most b/2 in z."""
    w = large_loop(n_atoms=5000, nz_cells=4, n_nodes=600)
    assert len(w.atoms) == 5000 and len(w.nodes) == 600
    assert w.periodic == (False, False, True) and w.fd_order == 8
    assert int(np.sum(w.depth == 1.3)) == 20
    assert w.halfwidth.min() >= 8 and w.halfwidth.max() <= 20
    _regions_inside(w)
    x0, y0, z0 = w.meta["loop_center"]
    R = w.meta["loop_radius"]
    d = np.hypot(np.hypot(w.atoms[:, 0] - x0, w.atoms[:, 1] - y0) - R, w.atoms[:, 2] - z0)
    fa = w.meta["force_atoms"]
    assert len(fa) == 2000 and d[fa].max() <= np.sort(d)[1999] + 1e-12
    assert abs(w.meta["burgers"] - 0.5 * C_LAT) < 1e-12
    assert math.isclose(w.spacing[0], 0.5) and abs(w.spacing[2] - 0.5) < 0.01
    assert w.box[2] == 4 * C_LAT and w.box[0] > 2 * w.meta["r_cyl"]
    ref = large_loop(n_atoms=5000, nz_cells=4, n_nodes=600)
    assert np.array_equal(ref.nodes, w.nodes) and np.array_equal(ref.atoms, w.atoms)
    assert A_LAT == 6.06
