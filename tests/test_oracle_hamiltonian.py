"""Pins of the oracle's Hamiltonian pieces (no GPU)."""
import math

import numpy as np
import pytest

from oracle import hamiltonian as H
from synthetic import make_workload
from synthetic.workloads import Workload
from tests.oracle_pins_helpers import golden_fd_weights, dense_region_hamiltonian


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_fd_weights_match_fornberg_table(order):
    np.testing.assert_allclose(H.fd_second_derivative_weights(order),
                               golden_fd_weights()[order], rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_fd_exact_on_polynomials(order):
    """A central 2q-order stencil differentiates x^k exactly for k <= 2q+1."""
    w = H.fd_second_derivative_weights(order)
    q = order // 2
    x0 = 0.37
    for k in range(0, order + 2):
        f = lambda x: x ** k
        approx = w[0] * f(x0) + sum(w[o] * (f(x0 + o) + f(x0 - o)) for o in range(1, q + 1))
        exact = k * (k - 1) * x0 ** (k - 2) if k >= 2 else 0.0
        assert abs(approx - exact) < 1e-9 * max(1.0, abs(exact))


def _single_atom(shape=(40, 40, 40), h=0.5, R=(10.1, 9.7, 10.3), D=1.0, sig=1.2):
    n = int(np.prod(shape))
    return Workload(name="one_atom", shape=shape, spacing=(h, h, h), periodic=(True, True, True),
                    fd_order=4, atoms=np.array([R]), depth=np.array([D]), sigma=np.array([sig]),
                    v_ext=np.zeros(n), nodes=np.array([0]), halfwidth=np.array([2], np.int32))


def test_gaussian_well_integral():
    """sum_i V_i dV = -D (2 pi sigma^2)^(3/2) (Gaussian integral)."""
    w = _single_atom()
    V = H.local_potential(w)
    exact = -1.0 * (2 * math.pi * 1.2 ** 2) ** 1.5
    assert abs(V.sum() * w.dV - exact) < 1e-9 * abs(exact)
    assert abs(V.min() + 1.0) < 0.2


def test_potential_translation_covariance():
    w = _single_atom()
    V1 = H.local_potential(w).reshape(40, 40, 40)
    w2 = w.with_atoms(np.array([[10.1 + 0.5, 9.7, 10.3 + 3 * 0.5]]))
    V2 = H.local_potential(w2).reshape(40, 40, 40)
    np.testing.assert_allclose(np.roll(np.roll(V1, 1, axis=2), 3, axis=0), V2, atol=1e-15)
    w3 = w.with_atoms(np.array([[10.1 + 20.0, 9.7 - 20.0, 10.3]]))
    np.testing.assert_allclose(H.local_potential(w3), V1.reshape(-1), atol=1e-15)


def test_potential_gradient_matches_finite_difference():
    w = _single_atom(shape=(24, 24, 24), R=(5.3, 6.1, 4.7))
    a = 0
    gidx, dVdR = H.local_potential_gradient_terms(w, a)
    step = 1e-5
    for d in range(3):
        Rp = w.atoms.copy(); Rp[0, d] += step
        Rm = w.atoms.copy(); Rm[0, d] -= step
        fd = (H.local_potential(w.with_atoms(Rp)) - H.local_potential(w.with_atoms(Rm))) / (2 * step)
        np.testing.assert_allclose(fd[gidx], dVdR[:, d], atol=1e-8)


def test_projectors_normalised_and_parity():
    w = _single_atom(shape=(24, 24, 24), R=(6.0, 6.0, 6.0))
    w.nonlocal_proj = True
    projs = H.projectors(w)
    assert len(projs) == 4
    dense = []
    for p in projs:
        v = np.zeros(w.n_grid); v[p.idx] = p.val
        dense.append(v.reshape(24, 24, 24))
        assert abs(w.dV * np.sum(v * v) - 1.0) < 1e-13
    s, px, py, pz = dense
    # atom on the grid point (12,12,12): s even, p_alpha odd along alpha
    c = 12
    for d, pd in zip((2, 1, 0), (px, py, pz)):
        flip = np.flip(np.roll(pd, -c, axis=d), axis=d)
        np.testing.assert_allclose(np.roll(flip, c + 1, axis=d), -pd, atol=1e-14)
    assert abs(np.sum(s * px)) < 1e-12 and abs(np.sum(px * py)) < 1e-12


def test_gershgorin_contains_spectrum():
    w = make_workload("tiny", nonlocal_proj=True)
    V = H.local_potential(w)
    projs = H.projectors(w)
    lo, hi = H.gershgorin_bounds(w, V, projs)
    reg = H.region_of(w, int(w.nodes[0]), 10)       # whole periodic grid
    assert all(reg.ring)
    pl = H.projectors_in_region(projs, reg, w.n_grid)
    Hd = dense_region_hamiltonian(reg.dims, reg.ring, w.spacing, w.fd_order, V[reg.gidx], pl, w.dV)
    ev = np.linalg.eigvalsh(Hd)
    assert lo <= ev[0] and ev[-1] <= hi


def test_region_mapping():
    w = make_workload("tiny", shape=(10, 12, 14), s=3)
    node = 9 + 10 * (0 + 12 * 13)          # corner: wraps on x, y and z
    reg = H.region_of(w, node, 3)
    assert reg.dims == (7, 7, 7) and not any(reg.ring)
    assert reg.gidx[reg.src] == node
    g = reg.gidx.reshape(7, 7, 7)
    assert g[3, 3, 4] == 0 + 10 * (0 + 12 * 13)     # one step +x wraps to ix = 0
    with pytest.raises(ValueError):
        w2 = make_workload("tiny", shape=(10, 12, 14), s=3, periodic=(False, True, True))
        H.region_of(w2, node, 3)


def test_nonlocal_operator_spectrum():
    """For one atom on a grid point the four projectors are orthonormal in
    the dV inner product, so sum_l E_l dV |p_l><p_l| has eigenvalues
    exactly {E_s, E_p, E_p, E_p, 0, ...}."""
    w = _single_atom(shape=(16, 16, 16), h=0.6, R=(4.8, 4.8, 4.8))
    w.nonlocal_proj = True
    w.e_s, w.e_p = 0.5, 0.25
    projs = H.projectors(w)
    M = np.zeros((w.n_grid, w.n_grid))
    for p in projs:
        v = np.zeros(w.n_grid); v[p.idx] = p.val
        M += p.energy * w.dV * np.outer(v, v)
    ev = np.sort(np.linalg.eigvalsh(M))[::-1]
    np.testing.assert_allclose(ev[:4], [0.5, 0.25, 0.25, 0.25], atol=1e-12)
    assert np.abs(ev[4:]).max() < 1e-12


def test_potential_on_points_equals_full_grid():
    """The restricted potential (large grids) is the full-grid one at the
    same points: periodic cell, open-axis cylinder, and a restricted build
    with given bounds keeps V there."""
    from oracle import density as od
    rng = np.random.default_rng(3)
    for w in (make_workload("tiny", shape=(12, 10, 14), n_atoms=5),
              make_workload("tiny", shape=(14, 12, 16), periodic=(False, True, False), n_atoms=4)):
        V = H.local_potential(w)
        idx = rng.choice(w.n_grid, size=300, replace=False)
        np.testing.assert_allclose(H.local_potential_on(w, idx), V[idx], rtol=1e-13, atol=1e-15)
        c = w.node_coords()
        ok = np.ones(len(w.nodes), bool)
        for d in range(3):
            if not w.periodic[d]:
                ok &= (c[:, d] - w.halfwidth >= 0) & (c[:, d] + w.halfwidth < w.shape[d])
        ws = w.subset(np.nonzero(ok)[0][:2])
        pts = od.region_points(ws)
        Hr = od.build(ws, points=pts, bounds=(-3.0, 40.0))
        for p in pts:
            np.testing.assert_allclose(Hr.V[p], V[p], rtol=1e-13, atol=1e-15)
        assert (Hr.emin, Hr.emax) == (-3.0, 40.0)
