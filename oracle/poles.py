"""Oracle: rational (pole) approximation of the Fermi-Dirac function.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's density matrix is g(H) with the Fermi-Dirac function of
Eq. (dm), g(eps) = 1 / (1 + exp((eps - mu)/kT)).  The paper evaluates
<e_p|g(H)|e_p> with Gauss quadrature (Eq. 9); the pole form used here writes

    g(eps) ~= r(eps) = sum_{p=1}^{P} Im( w_p / (eps - z_p) ),  Im z_p > 0,

so that [r(H)]_jj = sum_p Im(w_p [(H - z_p)^-1]_jj) needs one shifted solve
per pole.  The poles come from the contour-integral construction of Hale,
Higham & Trefethen (SIAM J. Numer. Anal. 46, 2008) with the square-root
substitution of Lin, Lu, Ying & E (Chin. Ann. Math. 30B, 2009), derived as
follows (x = eps - mu, a = (pi kT)^2, spectrum x in [-dE, dE]):

1. g(x) = (1/2 pi i) times the contour integral of g(xi)/(xi - x) dxi on a
   closed curve around
   [-dE, dE] that passes between the Matsubara poles +-i pi kT.
2. Substitute w = xi^2 + a.  The two half-curves Re xi > 0, Re xi < 0 both
   map onto one closed curve around [m, M] = [a, dE^2 + a], and the
   integrand becomes the even function of xi
       F(w) = (1/(2 xi)) [ g(xi)/(xi - x) + g(-xi)/(xi + x) ],
   analytic off (-inf, 0] U [m, M].
3. Map the period strip of sn(t | k), k = (sqrt M - sqrt m)/(sqrt M + sqrt m),
   conformally onto that doubly connected region:
       w(t) = sqrt(m M) (1/k + sn t)/(1/k - sn t),
   Im t = 0 -> [m, M], Im t = K' -> (-inf, 0].  On the middle line
   t = s + i K'/2 apply the N-point trapezoid rule in s (spacing 4K/N).
4. Conjugate symmetry halves the nodes: g(x) ~= -(h/pi) sum_{j<=N/2}
   Im(F(w_j) w'(t_j)) (the minus sign: increasing s runs clockwise).
5. Each node j gives two poles with Im > 0 (c_j = h w'(t_j) / (2 pi xi_j)):
       z = mu + xi_j,        w = c_j g(xi_j)
       z = mu - conj(xi_j),  w = conj(c_j g(-xi_j))
   so P = N shifted solves.  The error decays like exp(-pi K' N / (4K)).

Library primitives used as steps: scipy.special.ellipk / ellipkm1 (complete
elliptic integrals) and scipy.special.ellipj (Jacobi functions of a real
argument), extended to a complex argument by the addition formulas
(Abramowitz & Stegun 16.21.1-3).
"""
import math

import numpy as np
from scipy.special import ellipj, ellipk, ellipkm1


def fermi(x, kT: float):
    """1/(1+exp(x/kT)) for real or complex x, without overflow."""
    x = np.asarray(x)
    xc = x.astype(np.complex128)
    out = np.empty_like(xc)
    pos = xc.real > 0
    e = np.exp(-xc[pos] / kT)
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(xc[~pos] / kT))
    if not np.iscomplexobj(x):
        return out.real
    return out


def _sn_cn_dn(t: complex, m: float, m1: float):
    """Jacobi sn, cn, dn at complex t, parameter m = k^2 (m1 = 1 - m)."""
    s, c, d, _ = ellipj(t.real, m)
    s1, c1, d1, _ = ellipj(t.imag, m1)
    den = c1 * c1 + m * s * s * s1 * s1
    sn = (s * d1 + 1j * c * d * s1 * c1) / den
    cn = (c * c1 - 1j * s * d * s1 * d1) / den
    dn = (d * c1 * d1 - 1j * m * s * c * s1) / den
    return sn, cn, dn


def fermi_poles(kT: float, mu: float, emin: float, emax: float, P: int):
    """Poles z (complex128[P], Im > 0) and weights w (complex128[P])."""
    if P < 2 or P % 2:
        raise ValueError("P must be an even number >= 2")
    if not (kT > 0 and emax > emin):
        raise ValueError("need kT > 0 and emax > emin")
    dE = max(abs(emin - mu), abs(emax - mu))
    a = (math.pi * kT) ** 2
    m_lo, m_hi = a, dE * dE + a
    sq_m, sq_M = math.sqrt(m_lo), math.sqrt(m_hi)
    k = (sq_M - sq_m) / (sq_M + sq_m)
    kp2 = (1.0 - k) * (1.0 + k)           # k'^2, accurate for k near 1
    K = float(ellipkm1(kp2))              # K(k)
    Kp = float(ellipk(kp2))               # K(k') = K'
    h = 4.0 * K / P
    c0 = math.sqrt(m_lo * m_hi)
    z = np.empty(P, dtype=np.complex128)
    w = np.empty(P, dtype=np.complex128)
    for j in range(P // 2):
        t = complex(-K + (j + 0.5) * h, 0.5 * Kp)
        sn, cn, dn = _sn_cn_dn(t, k * k, kp2)
        wq = c0 * (1.0 / k + sn) / (1.0 / k - sn)
        dw = c0 * (2.0 / k) * cn * dn / (1.0 / k - sn) ** 2
        xi = np.sqrt(wq - a)                # principal root: first quadrant
        cj = h * dw / (2.0 * math.pi * xi)
        gp = fermi(np.array([xi]), kT)[0]
        gm = fermi(np.array([-xi]), kT)[0]
        z[2 * j] = mu + xi
        w[2 * j] = cj * gp
        z[2 * j + 1] = mu - np.conj(xi)
        w[2 * j + 1] = np.conj(cj * gm)
    return z, w


def rational(eps, z, w):
    """r(eps) = sum_p Im(w_p/(eps - z_p)) for real eps (vectorised)."""
    eps = np.asarray(eps, dtype=np.float64)
    return np.imag(w[None, :] / (eps.reshape(-1, 1) - z[None, :])).sum(axis=1).reshape(eps.shape)


def rational_times_eps(eps, z, w):
    """eps r(eps) = sum_p Im(w_p (1 + z_p/(eps - z_p))) (band-energy weight)."""
    eps = np.asarray(eps, dtype=np.float64)
    t = w[None, :] * (1.0 + z[None, :] / (eps.reshape(-1, 1) - z[None, :]))
    return np.imag(t).sum(axis=1).reshape(eps.shape)
