"""Pins of the LSSGQ oracle (Section 2.1, Eq. 9): Gauss-rule moments against
dense matrix powers, exactness when the Krylov space closes, convergence to
the dense spectral sum for a smooth g, and the Fermi level of a free-electron
cell against its closed-form spectrum."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import density as od
from oracle import hamiltonian as ham
from oracle import lssgq
from synthetic import make_workload
from synthetic.workloads import Workload
from tests.oracle_pins_helpers import dense_region_hamiltonian, fd_symbol, golden_fd_weights


def _dense_for(w, H, reg):
    pl = ham.projectors_in_region(H.projs, reg, w.n_grid)
    return dense_region_hamiltonian(reg.dims, reg.ring, w.spacing, w.fd_order, H.V[reg.gidx], pl, w.dV)


@pytest.mark.parametrize("case", [dict(nonlocal_proj=False, fd_order=4, s=2),
                                  dict(nonlocal_proj=True, fd_order=8, s=2),
                                  dict(nonlocal_proj=True, fd_order=4, s=3, shape=(7, 12, 9)),
                                  dict(nonlocal_proj=False, fd_order=8, s=10, shape=(6, 5, 7))])
def test_gauss_rule_reproduces_moments(case):
    """sum_k w_k lambda_k^m = e_j^T H_R^m e_j for m < 2K (Gauss exactness)."""
    K = 6
    w = make_workload("tiny", n_nodes=3, **case)
    H = od.build(w)
    for node, s in zip(w.nodes, w.halfwidth):
        reg = ham.region_of(w, int(node), int(s))
        Hd = _dense_for(w, H, reg)
        nrm = np.linalg.norm(Hd, 2)
        a, b = lssgq.lanczos(lssgq.RegionOperator(w, H, reg), reg.src, K)
        assert len(a) == K
        lam, wt = lssgq.gauss_rule(a, b)
        v = np.zeros(Hd.shape[0])
        v[reg.src] = 1.0
        for m in range(2 * K):
            exact = v[reg.src]
            quad = float(np.sum(wt * lam ** m))
            assert abs(quad - exact) <= 1e-10 * nrm ** m, (m, quad, exact)
            v = Hd @ v


def _symmetric_window():
    shape = (9, 9, 9)
    n = int(np.prod(shape))
    return Workload(name="sym", shape=shape, spacing=(0.5, 0.5, 0.5), periodic=(True, True, True),
                    fd_order=4, atoms=np.zeros((0, 3)), depth=np.zeros(0), sigma=np.zeros(0),
                    v_ext=np.full(n, -0.3), nodes=np.array([4 + 9 * (4 + 9 * 4)]),
                    halfwidth=np.array([1], np.int32), n_poles=8)


def test_krylov_space_closes_and_rule_is_exact():
    """Constant potential on a 3^3 window: the Krylov space of the centre is
    {centre, faces, edges, corners}, so Lanczos stops at k = 4 and the rule
    equals the dense spectral sum."""
    w = _symmetric_window()
    H = od.build(w)
    lam, wts, k_used = lssgq.quadrature(w, H, w.nodes, w.halfwidth, K=20)
    assert k_used[0] == 4
    reg = ham.region_of(w, int(w.nodes[0]), 1)
    ev, U = np.linalg.eigh(_dense_for(w, H, reg))
    wt = U[reg.src, :] ** 2
    for mu, kT in ((0.2, 0.01), (5.0, 0.3), (-1.0, 1.0)):
        rho, e, s = lssgq.fields(lam, wts, mu, kT, w.dV)
        g = 0.5 * (1.0 - np.tanh(0.5 * (ev - mu) / kT))
        rho_d = 2.0 / w.dV * np.sum(wt * g)
        e_d = 2.0 * np.sum(wt * ev * g)
        with np.errstate(divide="ignore", invalid="ignore"):
            ent = np.where((g > 0) & (g < 1), g * np.log(g) + (1 - g) * np.log(1 - g), 0.0)
        s_d = -2.0 * kT * np.sum(wt * ent)
        assert abs(rho[0] - rho_d) <= 1e-12 * max(abs(rho_d), 1.0)
        assert abs(e[0] - e_d) <= 1e-12 * max(abs(e_d), 1.0)
        assert abs(s[0] - s_d) <= 1e-12 * max(abs(s_d), 1e-3)


def test_smooth_function_converges_to_dense():
    """g at kT = 2 Ha is analytic in a wide strip, so the K = 30 rule on a
    5^3 window with random wells matches the dense spectral sum."""
    w = make_workload("tiny", nonlocal_proj=True, fd_order=4, s=2, n_nodes=3)
    H = od.build(w)
    lam, wts, k_used = lssgq.quadrature(w, H, w.nodes, w.halfwidth, K=30)
    assert np.all(k_used == 30)
    rho, e, s = lssgq.fields(lam, wts, 0.5, 2.0, w.dV)
    for j, (node, sj) in enumerate(zip(w.nodes, w.halfwidth)):
        reg = ham.region_of(w, int(node), int(sj))
        ev, U = np.linalg.eigh(_dense_for(w, H, reg))
        g = 0.5 * (1.0 - np.tanh(0.5 * (ev - 0.5) / 2.0))
        wt = U[reg.src, :] ** 2
        assert abs(rho[j] - 2.0 / w.dV * np.sum(wt * g)) <= 1e-10 * rho[j]
        assert abs(e[j] - 2.0 * np.sum(wt * ev * g)) <= 1e-10 * max(1.0, abs(e[j]))


def test_entropy_density_stable_form():
    """The overflow-free entropy form equals g ln g + (1-g) ln(1-g) evaluated
    in 50-digit arithmetic, including the far tails where g or 1 - g is
    below double precision's resolution of 1."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    eps = np.linspace(-0.3, 0.7, 401)
    got = lssgq.entropy_density(eps, 0.2, 0.01)
    for e, v in zip(eps, got):
        x = (mp.mpf(float(e)) - mp.mpf("0.2")) / mp.mpf("0.01")
        g = 1 / (1 + mp.exp(x))
        ref = g * mp.log(g) + (1 - g) * mp.log(1 - g)
        assert abs(v - float(ref)) <= 1e-13 * abs(float(ref)) + 1e-300, (e, v, float(ref))
    assert abs(lssgq.entropy_density(0.2, 0.2, 0.01) + math.log(2.0)) < 1e-15
    far = lssgq.entropy_density(np.array([1e4, -1e4]), 0.0, 0.01)
    assert np.all(far == 0.0)


def test_fermi_level_free_electrons_closed_form():
    """V = 0 on a 6^3 periodic cell, one node whose region is the whole cell:
    the Krylov space has one vector per distinct FD eigenvalue (19 here), so
    a rule of K >= 19 nodes reproduces the spectral measure, and its Fermi
    level for N electrons matches the root of 2 sum_k g(eps_k; mu) = N over
    the closed-form spectrum.  (In floating point beta_19 is ~1e-9, not 0,
    and the process runs on; the extra nodes carry the measure unchanged.)"""
    shape, h = (6, 6, 6), 0.6
    n = int(np.prod(shape))
    w = Workload(name="free", shape=shape, spacing=(h, h, h), periodic=(True, True, True), fd_order=4,
                 atoms=np.zeros((0, 3)), depth=np.zeros(0), sigma=np.zeros(0), v_ext=np.zeros(n),
                 nodes=np.array([7]), halfwidth=np.array([10], np.int32), n_poles=8)
    H = od.build(w)
    lam, wts, k_used = lssgq.quadrature(w, H, w.nodes, w.halfwidth, K=24)
    fw = golden_fd_weights()[4]
    k = 2 * np.pi * np.fft.fftfreq(6, d=h)
    sym = fd_symbol(k, h, fw)
    eps = (sym[:, None, None] + sym[None, :, None] + sym[None, None, :]).reshape(-1)
    assert len(np.unique(np.round(eps, 10))) == 19
    kT = 0.05
    for N_e in (7.0, 40.0, 123.5):
        exact = brentq(lambda m: 2.0 * np.sum(0.5 * (1 - np.tanh(0.5 * (eps - m) / kT))) - N_e,
                       eps.min() - 5, eps.max() + 5, xtol=1e-14, rtol=1e-15)
        mu = lssgq.fermi_level(lam, wts, kT, N_e, nu=np.array([float(n)]))
        assert abs(mu - exact) < 1e-9, (N_e, mu, exact)
        assert abs(lssgq.electron_count(lam, wts, mu, kT, nu=[n]) - N_e) < 1e-8 * N_e


def test_trace_of_rules_is_electron_count():
    """Every grid point a node with its whole-cell region: sum_j rho_j dV
    from the rules equals N_e(mu) with unit node weights (Eq. Fermi:Rho)."""
    w = make_workload("tiny", shape=(5, 4, 6), s=10, nonlocal_proj=True)
    w = w.subset(np.arange(1))
    w.nodes = np.arange(w.n_grid)
    w.halfwidth = np.full(w.n_grid, 10, np.int32)
    H = od.build(w)
    lam, wts, _ = lssgq.quadrature(w, H, w.nodes, w.halfwidth, K=12)
    rho, _, _ = lssgq.fields(lam, wts, 0.2, 0.05, w.dV)
    assert abs(np.sum(rho) * w.dV - lssgq.electron_count(lam, wts, 0.2, 0.05)) < 1e-11 * np.sum(rho) * w.dV
    # and, with K = 120 = the cell size, close to 2 sum_i g(eps_i) of the dense H
    lam2, wts2, _ = lssgq.quadrature(w, H, w.nodes[:1], w.halfwidth[:1], K=120)
    ev = np.linalg.eigvalsh(_dense_for(w, H, ham.region_of(w, 0, 10)))
    g = 0.5 * (1.0 - np.tanh(0.5 * (ev - 0.2) / 0.05))
    assert np.isfinite(lam2).all() and abs(np.sum(wts2) - 1.0) < 1e-12
    assert abs(2.0 * np.sum(g) - lssgq.electron_count(lam, wts, 0.2, 0.05)) < 0.05 * 2.0 * np.sum(g)
