"""Pins of the oracle's free-energy terms and the pole-form Fermi level (no GPU).

* phi_S, the entropy function of Eq. (tot)'s last term, against its direct
  definition, its symmetry, its value ln 2 at mu, and the analyticity of the
  half-plane continuation (Cauchy-Riemann, and the two pieces agreeing on
  the imaginary axis between the Matsubara points);
* the entropy weights on the Fermi poles against the exact phi_S on 10^5
  points (bounds per P, the same geometric rate as the Fermi expansion);
* s_j from the COCG solves against dense diagonalisation, 2 kT sum_i
  phi_S^r(eps_i) |psi_i(j)|^2, and against the free-electron closed form;
* weighted totals: unit weights on a whole periodic cell reproduce the
  traces 2 Tr r(H), 2 Tr H r(H) and 2 kT Tr phi_S^r(H); integer node weights
  equal the sum over repeated nodes;
* cluster sampling (Eqs. free_cg, free_cg_sampling) against a brute-force
  minimum-image ball over every grid point, singletons for a radius below
  the spacing, and conservation sum_p nu_p = sum_q n_q;
* the pole-form Fermi level against a Brent root of the free-electron
  closed form N(mu) = 2 sum_k r_mu(eps_k).
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import density as od
from oracle import hamiltonian as ham
from oracle.poles import entropy_fn, entropy_weights, fermi, fermi_poles, rational, rational_times_eps
from synthetic import make_workload
from synthetic.workloads import Workload
from tests.oracle_pins_helpers import dense_region_hamiltonian, fd_symbol, golden_fd_weights

KT, MU = 0.01, 0.2
EMIN, EMAX = -3.04, 31.97


def test_entropy_fn_definition_and_symmetry():
    x = np.linspace(-0.25, 0.25, 2001)   # |y| <= 25: 1 - f still resolved in double
    f = fermi(x, KT)
    direct = -(f * np.log(f) + (1 - f) * np.log1p(-f))
    np.testing.assert_allclose(entropy_fn(x, KT), direct, rtol=0, atol=1e-14)
    np.testing.assert_allclose(entropy_fn(-x, KT), entropy_fn(x, KT), rtol=0, atol=1e-15)
    assert abs(entropy_fn(np.array([0.0]), KT)[0] - math.log(2.0)) < 1e-15
    # far tails: phi_S ~ e^-|y| (1 + |y|), positive, no cancellation to zero
    y = np.array([30.0, 60.0])
    np.testing.assert_allclose(entropy_fn(y * KT, KT), np.exp(-y) * (1 + y), rtol=1e-12)


def test_entropy_fn_is_analytic_off_the_matsubara_rays():
    # Cauchy-Riemann: d phi / d re = -i d phi / d im at complex points, in both half-planes
    for y0 in (0.7 + 0.4j, -1.3 + 2.5j, 5.0 - 7.0j, -0.2 + 0.1j):
        h = 1e-6
        x0 = y0 * KT
        d_re = (entropy_fn(np.array([x0 + h * KT]), KT) - entropy_fn(np.array([x0 - h * KT]), KT)) / (2 * h)
        d_im = (entropy_fn(np.array([x0 + 1j * h * KT]), KT) - entropy_fn(np.array([x0 - 1j * h * KT]), KT)) / (2 * h)
        assert abs(d_re[0] + 1j * d_im[0]) < 1e-7 * max(1.0, abs(d_re[0]))
    # the two half-plane pieces meet continuously on Re y = 0 for |Im y| < pi
    for b in (0.3, 1.5, 3.0):
        left = entropy_fn(np.array([(-1e-12 + 1j * b) * KT]), KT)[0]
        right = entropy_fn(np.array([(1e-12 + 1j * b) * KT]), KT)[0]
        assert abs(left - right) < 1e-9


@pytest.mark.parametrize("P,bound", [(8, 0.7), (16, 0.04), (32, 3e-4), (64, 2e-7)])
def test_entropy_weights_approximate_phi(P, bound):
    z, w = fermi_poles(KT, MU, EMIN, EMAX, P)
    ws = entropy_weights(KT, MU, EMIN, EMAX, P)
    e = np.linspace(EMIN, EMAX, 100001)
    err = np.max(np.abs(rational(e, z, ws) - entropy_fn(e - MU, KT)))
    assert err < bound


def test_entropy_weights_geometric_rate_matches_fermi():
    """Same singularities, same rate: over P = 16..96 the entropy error falls
    at the Fermi expansion's rate within 10% (step to step it is less even:
    the location of the largest error jumps)."""
    e = np.linspace(EMIN, EMAX, 100001)
    errs = {}
    for P in (16, 96):
        z, w = fermi_poles(KT, MU, EMIN, EMAX, P)
        ws = entropy_weights(KT, MU, EMIN, EMAX, P)
        errs[P] = (np.max(np.abs(rational(e, z, w) - fermi(e - MU, KT))),
                   np.max(np.abs(rational(e, z, ws) - entropy_fn(e - MU, KT))))
    slope_f = -(math.log(errs[96][0]) - math.log(errs[16][0])) / 80
    slope_s = -(math.log(errs[96][1]) - math.log(errs[16][1])) / 80
    assert abs(slope_s - slope_f) / slope_f < 0.1


def _dense_for(w, H, reg):
    pl = ham.projectors_in_region(H.projs, reg, w.n_grid)
    return dense_region_hamiltonian(reg.dims, reg.ring, w.spacing, w.fd_order, H.V[reg.gidx], pl, w.dV)


@pytest.mark.parametrize("nonlocal_proj,order,s", [(False, 4, 2), (True, 8, 2), (True, 4, 10)])
def test_entropy_node_vs_dense_eigh(nonlocal_proj, order, s):
    w = make_workload("tiny", nonlocal_proj=nonlocal_proj, fd_order=order, s=s, n_nodes=4)
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13)
    ws = entropy_weights(w.kT, w.mu, H.emin, H.emax, w.n_poles)
    s_node = od.entropy_node(res, ws, w.kT)
    for j, reg in enumerate(res.regions):
        ev, U = np.linalg.eigh(_dense_for(w, H, reg))
        s_ref = 2.0 * w.kT * np.sum(rational(ev, res.z, ws) * U[reg.src, :] ** 2)
        assert abs(s_node[j] - s_ref) <= 1e-10 * max(1e-3, abs(s_ref))


def _free_electron(shape=(6, 6, 8), spacing=(0.55, 0.6, 0.5), order=4, all_nodes=False):
    n = int(np.prod(shape))
    nodes = np.arange(n) if all_nodes else np.array([0, 17, 100, n - 1])
    return Workload(name="free", shape=shape, spacing=spacing, periodic=(True, True, True),
                    fd_order=order, atoms=np.zeros((0, 3)), depth=np.zeros(0), sigma=np.zeros(0),
                    v_ext=np.zeros(n), nodes=nodes, halfwidth=np.full(len(nodes), 10, np.int32),
                    n_poles=16, tol=1e-13)


def _fd_spectrum(w):
    wts = golden_fd_weights()[w.fd_order]
    eps = np.zeros(w.shape[::-1])
    for d, (n, h) in enumerate(zip(w.shape, w.spacing)):
        k = 2 * np.pi * np.fft.fftfreq(n, d=h)
        sh = [1, 1, 1]
        sh[2 - d] = n
        eps = eps + fd_symbol(k, h, wts).reshape(sh)
    return eps.reshape(-1)


def test_entropy_free_electron_closed_form():
    w = _free_electron()
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13)
    ws = entropy_weights(w.kT, w.mu, H.emin, H.emax, w.n_poles)
    eps = _fd_spectrum(w)
    s_exact = 2.0 * w.kT * np.sum(rational(eps, res.z, ws)) / w.n_grid
    np.testing.assert_allclose(od.entropy_node(res, ws, w.kT), s_exact, rtol=1e-9)


def test_unit_weights_on_whole_cell_give_traces():
    w = make_workload("tiny", shape=(4, 5, 6), s=10, n_atoms=3, fd_order=4)
    w.nodes = np.arange(w.n_grid)
    w.halfwidth = np.full(w.n_grid, 10, np.int32)
    H = od.build(w)
    res = od.solve(w, H, tol=1e-13)
    ws = entropy_weights(w.kT, w.mu, H.emin, H.emax, w.n_poles)
    t = od.free_energy_terms(w, res, ws)
    reg = res.regions[0]
    ev = np.linalg.eigvalsh(_dense_for(w, H, reg))
    assert abs(t["n_electrons"] - 2 * rational(ev, res.z, res.wts).sum()) < 1e-9
    assert abs(t["e_band"] - 2 * rational_times_eps(ev, res.z, res.wts).sum()) < 1e-9 * max(1, abs(t["e_band"]))
    assert abs(t["ts"] - 2 * w.kT * rational(ev, res.z, ws).sum()) < 1e-10
    assert abs(t["free_energy"] - (t["e_band"] - t["ts"])) == 0.0


def test_integer_weights_equal_repeated_nodes():
    w = make_workload("tiny", n_nodes=5, s=2, n_atoms=3)
    H = od.build(w)
    ws = entropy_weights(w.kT, w.mu, H.emin, H.emax, w.n_poles)
    mult = np.array([1, 3, 2, 1, 4])
    t = od.free_energy_terms(w, od.solve(w, H, tol=1e-13), ws, node_weight=mult)
    rep = w.subset(np.repeat(np.arange(5), mult))
    t2 = od.free_energy_terms(rep, od.solve(rep, H, tol=1e-13), ws)
    for k in ("n_electrons", "e_band", "ts", "free_energy"):
        assert abs(t[k] - t2[k]) <= 1e-12 * max(1.0, abs(t2[k]))


def _ball_bruteforce(w, g, radius):
    nx, ny, nz = w.shape
    c = np.array([g % nx, (g // nx) % ny, g // (nx * ny)])
    idx = np.arange(w.n_grid)
    p = np.stack([idx % nx, (idx // nx) % ny, idx // (nx * ny)], 1)
    d2 = np.zeros(w.n_grid)
    for d in range(3):
        o = p[:, d] - c[d]
        if w.periodic[d]:
            n = w.shape[d]
            o = np.minimum(np.abs(o), n - np.abs(o))
        d2 += (o * w.spacing[d]) ** 2
    return np.nonzero(d2 <= radius * radius)[0]


@pytest.mark.parametrize("periodic", [(True, True, True), (False, True, False)])
def test_cluster_sampling(periodic):
    w = make_workload("tiny", shape=(12, 10, 14), periodic=periodic, spacing=(0.5, 0.45, 0.55))
    esp = np.array([0, 5 + 12 * 4 + 120 * 7, 11 + 12 * 9 + 120 * 13, 6 + 12 * 5 + 120 * 6])
    n_q = np.array([1.0, 8.0, 27.0, 2.0])
    radius = 1.3
    nodes, nu = od.cluster_sampling(w, esp, n_q, radius)
    ref = {}
    for g, n in zip(esp, n_q):
        ball = _ball_bruteforce(w, int(g), radius)
        for p in ball:
            ref[int(p)] = ref.get(int(p), 0.0) + n / len(ball)
    assert list(nodes) == sorted(ref)
    np.testing.assert_allclose(nu, [ref[int(p)] for p in nodes], rtol=1e-15)
    assert abs(nu.sum() - n_q.sum()) < 1e-12
    n1, nu1 = od.cluster_sampling(w, esp, n_q, 0.4)    # below every spacing: the points alone
    assert list(n1) == sorted(esp.tolist()) and np.allclose(nu1, n_q[np.argsort(esp)])


def test_fermi_level_poles_free_electron():
    w = _free_electron(shape=(4, 4, 6), spacing=(0.6, 0.6, 0.5), all_nodes=True)
    w.n_poles = 16
    H = od.build(w)
    eps = _fd_spectrum(w)
    target = 20.0

    def count(mu):
        z, wt = fermi_poles(w.kT, mu, H.emin, H.emax, w.n_poles)
        return 2.0 * rational(eps, z, wt).sum() - target

    mu_ref = brentq(count, H.emin, H.emax, xtol=1e-13)
    mu, n, _ = od.fermi_level_poles(w, H, target, mu_tol=1e-10)
    assert abs(mu - mu_ref) < 1e-9
    assert abs(n - target) < 1e-6
