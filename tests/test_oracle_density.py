"""Pins of the oracle's nodal density, band energy and adjoint (no GPU).

The oracle's COCG densities are checked against quantities that the
mathematics fixes independently of its code path:
* dense diagonalisation of H_R (numpy.linalg.eigh), rho_j = (2/dV)
  sum_i r(eps_i) |psi_i(j)|^2 (the spectral form of Eq. Electron_density:GQ);
* a direct complex solve of (H_R - z) x = e_j (numpy.linalg.solve);
* the free-electron closed form (plane waves, FD symbols);
* the trace invariant sum_j rho_j dV = 2 Tr r(H) = N_e (Eq. Fermi_level:GQ);
* reciprocity x_j(k) = x_k(j) and lattice translation symmetry;
* central finite differences for the adjoint and the forces.
"""
import numpy as np
import pytest

from oracle import density as od
from oracle import hamiltonian as ham
from oracle.poles import rational, rational_times_eps, fermi_poles
from synthetic import make_workload
from synthetic.workloads import Workload
from tests.oracle_pins_helpers import dense_region_hamiltonian, golden_fd_weights, fd_symbol


def _dense_for(w, H, reg):
    pl = ham.projectors_in_region(H.projs, reg, w.n_grid)
    return dense_region_hamiltonian(reg.dims, reg.ring, w.spacing, w.fd_order, H.V[reg.gidx], pl, w.dV)


@pytest.mark.parametrize("nonlocal_proj,order,s", [(False, 4, 2), (True, 8, 2), (False, 4, 10), (True, 4, 3)])
def test_density_vs_dense_eigh(nonlocal_proj, order, s):
    w = make_workload("tiny", nonlocal_proj=nonlocal_proj, fd_order=order, s=s, n_nodes=4)
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13)
    assert np.all(res.status == 0)
    for j, reg in enumerate(res.regions):
        Hd = _dense_for(w, H, reg)
        ev, U = np.linalg.eigh(Hd)
        wt = U[reg.src, :] ** 2
        rho = (2.0 / w.dV) * np.sum(rational(ev, res.z, res.wts) * wt)
        e = 2.0 * np.sum(rational_times_eps(ev, res.z, res.wts) * wt)
        assert abs(res.rho[j] - rho) <= 1e-10 * max(1.0, abs(rho))
        assert abs(res.e_node[j] - e) <= 1e-10 * max(1.0, abs(e))


def test_solution_vs_direct_solve():
    w = make_workload("tiny", shape=(9, 9, 9), s=4, nonlocal_proj=True, n_nodes=2, fd_order=8,
                      spacing=(0.5, 0.5, 0.5))
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13, keep_x=True)
    for j, reg in enumerate(res.regions):
        Hd = _dense_for(w, H, reg)
        b = np.zeros(Hd.shape[0]); b[reg.src] = 1.0
        for p, z in enumerate(res.z):
            x = np.linalg.solve(Hd - z * np.eye(len(b)), b)
            np.testing.assert_allclose(res.x_full[j][p], x, atol=1e-11 * np.abs(x).max())


def _free_electron(shape=(6, 6, 8), spacing=(0.55, 0.6, 0.5), order=4):
    n = int(np.prod(shape))
    return Workload(name="free", shape=shape, spacing=spacing, periodic=(True, True, True),
                    fd_order=order, atoms=np.zeros((0, 3)), depth=np.zeros(0), sigma=np.zeros(0),
                    v_ext=np.zeros(n), nodes=np.array([0, 17, 100, n - 1]),
                    halfwidth=np.full(4, 10, np.int32), n_poles=16, tol=1e-13)


def test_free_electron_closed_form():
    w = _free_electron()
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13)
    wts = golden_fd_weights()[w.fd_order]
    eps = np.zeros(w.shape[::-1])
    for d, (n, h) in enumerate(zip(w.shape, w.spacing)):
        k = 2 * np.pi * np.fft.fftfreq(n, d=h)
        lam = fd_symbol(k, h, wts)
        sh = [1, 1, 1]; sh[2 - d] = n
        eps = eps + lam.reshape(sh)
    N = w.n_grid
    rho_exact = (2.0 / (N * w.dV)) * np.sum(rational(eps.reshape(-1), res.z, res.wts))
    np.testing.assert_allclose(res.rho, rho_exact, rtol=1e-10)


def test_trace_invariant_full_grid():
    w = make_workload("tiny", shape=(5, 6, 6), s=10, nonlocal_proj=True)
    w = w.subset(np.arange(1))
    w.nodes = np.arange(w.n_grid)
    w.halfwidth = np.full(w.n_grid, 10, np.int32)
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13)
    ev = np.linalg.eigvalsh(_dense_for(w, H, res.regions[0]))
    Ne = 2.0 * np.sum(rational(ev, res.z, res.wts))
    assert abs(np.sum(res.rho) * w.dV - Ne) < 1e-9 * max(1.0, abs(Ne))


def test_reciprocity_full_region():
    w = make_workload("tiny", shape=(5, 6, 7), s=10, n_nodes=3)
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13, keep_x=True)
    g = [int(n) for n in w.nodes]
    for a in range(3):
        for b in range(3):
            ka = res.regions[b].gidx.tolist().index(g[a])
            kb = res.regions[a].gidx.tolist().index(g[b])
            np.testing.assert_allclose(res.x_full[b][:, ka], res.x_full[a][:, kb], atol=1e-11)


def test_translation_symmetry():
    """A potential periodic with half the box gives equal density at nodes
    one half-box apart (regions are windows, not whole axes)."""
    shape = (16, 8, 8)
    h = (0.5, 0.5, 0.5)
    n = int(np.prod(shape))
    atoms = np.array([[1.3, 1.1, 2.2], [1.3 + 4.0, 1.1, 2.2]])
    w = Workload(name="transl", shape=shape, spacing=h, periodic=(True, True, True), fd_order=4,
                 atoms=atoms, depth=np.ones(2), sigma=np.full(2, 0.7), v_ext=np.zeros(n),
                 nodes=np.array([3 + 16 * (2 + 8 * 5), 11 + 16 * (2 + 8 * 5)]),
                 halfwidth=np.full(2, 2, np.int32), n_poles=8, cutoff_sigmas=2.8)
    res = od.solve(w, tol=1e-13)
    assert abs(res.rho[0] - res.rho[1]) < 1e-11 * abs(res.rho[0])


def _loss_parts(w, tol=1e-13):
    H = od.build(w)
    res = od.solve(w, H, tol=tol, keep_x=True)
    return H, res


def test_adjoint_dV_vs_finite_difference():
    w = make_workload("tiny", shape=(6, 6, 6), s=2, n_nodes=3, spacing=(0.5, 0.5, 0.5))
    H, res = _loss_parts(w)
    a = np.array([0.7, -1.3, 0.4])
    b = np.array([0.2, 0.5, -0.9])
    g = od.dL_dV(w, res, a, b)
    rng = np.random.default_rng(3)
    touched = np.unique(np.concatenate([r.gidx for r in res.regions]))
    for k in rng.choice(touched, 5, replace=False):
        vals = []
        for sgn in (1, -1):
            w2 = make_workload("tiny", shape=(6, 6, 6), s=2, n_nodes=3, spacing=(0.5, 0.5, 0.5))
            w2.v_ext = w2.v_ext.copy(); w2.v_ext[k] += sgn * 1e-5
            H2 = od.build(w2)
            r2 = od.solve(w2, H2, z=res.z, wts=res.wts, tol=1e-13)
            vals.append(np.dot(a, r2.rho) + np.dot(b, r2.e_node))
        fd = (vals[0] - vals[1]) / 2e-5
        assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(g[k]))


def test_forces_vs_finite_difference():
    w = make_workload("tiny", shape=(8, 8, 8), s=3, n_nodes=3, spacing=(0.5, 0.5, 0.5), n_atoms=2)
    H, res = _loss_parts(w)
    a = np.array([1.0, -0.5, 0.3])
    b = np.ones(3)
    F = od.forces(w, od.dL_dV(w, res, a, b))
    step = 1e-4
    for atom in range(2):
        for d in range(3):
            vals = []
            for sgn in (1, -1):
                pos = w.atoms.copy(); pos[atom, d] += sgn * step
                w2 = w.with_atoms(pos)
                r2 = od.solve(w2, od.build(w2), z=res.z, wts=res.wts, tol=1e-13)
                vals.append(np.dot(a, r2.rho) + np.dot(b, r2.e_node))
            fd = -(vals[0] - vals[1]) / (2 * step)
            assert abs(fd - F[atom, d]) < 1e-6 * max(1.0, np.abs(F).max())


def test_density_matrix_rows_vs_dense():
    """gamma_jk = sum_p Im(w_p x_jp(k)) equals row j of r(H_R) from dense
    eigh, and its diagonal gives rho_j."""
    w = make_workload("tiny", nonlocal_proj=True, fd_order=4, s=2, n_nodes=3)
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13, keep_x=True)
    rows = od.density_matrix_rows(res)
    for j, reg in enumerate(res.regions):
        ev, U = np.linalg.eigh(_dense_for(w, H, reg))
        gamma = (U * rational(ev, res.z, res.wts)[None, :]) @ U[reg.src, :]
        np.testing.assert_allclose(rows[j], gamma, atol=1e-11 * np.abs(gamma).max())
        assert abs(2.0 / w.dV * rows[j][reg.src] - res.rho[j]) <= 1e-12 * abs(res.rho[j])
