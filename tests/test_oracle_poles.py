"""Pins of the oracle's pole expansion (no GPU).

The expansion is pinned against the exact Fermi-Dirac function of the
paper's Eq. (dm) on 10^5 points, against its predicted geometric rate, and
the complex Jacobi functions against their identities.
"""
import math
import os

import numpy as np
import pytest
from scipy.special import ellipkm1, ellipk

from oracle.poles import fermi, fermi_poles, rational, rational_times_eps, _sn_cn_dn

KT, MU = 0.01, 0.2
EMIN, EMAX = -3.04, 31.97


def _max_err(P, emin=EMIN, emax=EMAX, kT=KT, mu=MU, n=100001):
    z, w = fermi_poles(kT, mu, emin, emax, P)
    e = np.linspace(emin, emax, n)
    return np.max(np.abs(rational(e, z, w) - fermi(e - mu, kT))), z, w


def test_fermi_exact_values():
    assert fermi(0.0, 0.01) == 0.5
    x = np.array([-50.0, -1.0, 1.0, 50.0])
    np.testing.assert_allclose(fermi(x, 1.0), 1.0 / (1.0 + np.exp(x)), rtol=1e-15)
    # complex argument: the function's own symmetry g(-x) = 1 - g(x)
    xc = np.array([0.3 + 0.2j, -2.0 + 0.05j, 40.0 + 3j])
    np.testing.assert_allclose(fermi(-xc, 0.1), 1.0 - fermi(xc, 0.1), atol=1e-15)


@pytest.mark.parametrize("P,bound", [(8, 0.35), (16, 0.04), (32, 4e-4), (64, 5e-8)])
def test_rational_approximates_fermi(P, bound):
    err, z, w = _max_err(P)
    assert err < bound
    assert np.all(z.imag > 0)


def test_geometric_rate_matches_theory():
    """Trapezoid-rule error ~ exp(-pi K' N / (4K)): the measured slope of
    log(err) vs N must match it within 10%."""
    dE = max(abs(EMIN - MU), abs(EMAX - MU))
    a = (math.pi * KT) ** 2
    M = dE * dE + a
    k = (math.sqrt(M) - math.sqrt(a)) / (math.sqrt(M) + math.sqrt(a))
    kp2 = (1 - k) * (1 + k)
    K, Kp = ellipkm1(kp2), ellipk(kp2)
    rate = math.pi * Kp / (4 * K)
    e32, _, _ = _max_err(32)
    e64, _, _ = _max_err(64)
    slope = -(math.log(e64) - math.log(e32)) / 32
    assert abs(slope - rate) / rate < 0.1


def test_pole_pairs_mirror_about_mu():
    z, w = fermi_poles(KT, MU, EMIN, EMAX, 16)
    np.testing.assert_allclose(z[1::2], 2 * MU - np.conj(z[0::2]), rtol=0, atol=1e-14)


def test_shift_covariance():
    """Moving mu and the interval together translates the poles only."""
    z1, w1 = fermi_poles(KT, MU, EMIN, EMAX, 16)
    z2, w2 = fermi_poles(KT, MU + 1.5, EMIN + 1.5, EMAX + 1.5, 16)
    np.testing.assert_allclose(z2 - 1.5, z1, atol=1e-12)
    np.testing.assert_allclose(w2, w1, atol=1e-13)


def test_band_energy_weight():
    z, w = fermi_poles(KT, MU, EMIN, EMAX, 64)
    e = np.linspace(EMIN, EMAX, 2001)
    np.testing.assert_allclose(rational_times_eps(e, z, w), e * rational(e, z, w), atol=1e-11)
    assert np.max(np.abs(rational_times_eps(e, z, w) - e * fermi(e - MU, KT))) < 2e-6


def test_jacobi_identities_complex():
    m = 0.93
    for t in [0.3 + 0.4j, -1.1 + 0.9j, 2.0 + 0.2j]:
        sn, cn, dn = _sn_cn_dn(t, m, 1 - m)
        assert abs(sn * sn + cn * cn - 1) < 1e-13
        assert abs(m * sn * sn + dn * dn - 1) < 1e-13
        # d sn / dt = cn dn (central difference along the real direction)
        hh = 1e-5
        sp, _, _ = _sn_cn_dn(t + hh, m, 1 - m)
        sm, _, _ = _sn_cn_dn(t - hh, m, 1 - m)
        assert abs((sp - sm) / (2 * hh) - cn * dn) < 1e-8


def test_elliptic_K_closed_forms():
    path = os.path.join(os.path.dirname(__file__), "golden", "elliptic_K_closed_forms.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for k, K in rows:
        k, K = float(k), float(K)
        assert abs(ellipkm1((1 - k) * (1 + k)) - K) < 1e-14


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        fermi_poles(KT, MU, EMIN, EMAX, 7)
    with pytest.raises(ValueError):
        fermi_poles(0.0, MU, EMIN, EMAX, 8)
    with pytest.raises(ValueError):
        fermi_poles(KT, MU, 1.0, -1.0, 8)
