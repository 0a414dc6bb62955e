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
6. Nothing above uses more of g than its analyticity off the rays of the
   imaginary axis beyond +-i pi kT.  The entropy function of Eq. (tot)'s last
   term has its branch points at the same Matsubara points, so the same
   nodes with weights c_j phi_S(+-xi_j) approximate it (entropy_weights).

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


def _log1p_c(u):
    """log(1 + u) for complex u with |u| < 1, accurate also for tiny |u|
    (numpy's complex log1p forms 1 + u first): the alternating series
    sum_k (-1)^(k+1) u^k / k to k = 16 where |u| < 0.1 (truncation below
    0.1^17/17), log(1 + u) elsewhere."""
    u = np.asarray(u, dtype=np.complex128)
    out = np.log(1.0 + u)
    small = np.abs(u) < 0.1
    us = u[small]
    acc = np.zeros_like(us)
    for k in range(16, 0, -1):      # Horner form of the series
        acc = us * ((1.0 if k % 2 else -1.0) / k + acc)
    out[small] = acc
    return out


def entropy_fn(x, kT: float):
    """phi_S(x) = -[f ln f + (1 - f) ln(1 - f)], f = fermi(x, kT): the
    bracket of the last term of Eq. (tot) with its sign turned so that
    phi_S >= 0 on the real axis (phi_S(0) = ln 2), for real or complex x.

    With y = x/kT, ln f = -ln(1 + e^y) and ln(1 - f) = y - ln(1 + e^y), so
    phi_S = ln(1 + e^y) - (1 - f) y.  Written per half-plane so that nothing
    cancels and every logarithm has its argument in the disc |u - 1| < 1:
        Re y <= 0:  log1p(e^y)  - y e^y  / (1 + e^y)
        Re y >  0:  log1p(e^-y) + y e^-y / (1 + e^-y)
    The two pieces agree on Re y = 0 for |Im y| < pi, so together they are
    the analytic continuation of phi_S off the rays |Im y| >= pi of the
    imaginary axis, where its branch points (the Matsubara points) lie."""
    x = np.asarray(x)
    y = x.astype(np.complex128) / kT
    out = np.empty_like(y)
    pos = y.real > 0
    en = np.exp(-y[pos])
    out[pos] = _log1p_c(en) + y[pos] * en / (1.0 + en)
    ep = np.exp(y[~pos])
    out[~pos] = _log1p_c(ep) - y[~pos] * ep / (1.0 + ep)
    if not np.iscomplexobj(x):
        return out.real
    return out


def _contour_nodes(kT: float, mu: float, emin: float, emax: float, P: int):
    """Steps 2-4 of the construction: the P/2 trapezoid nodes xi_j (first
    quadrant) and their factors c_j = h w'(t_j) / (2 pi xi_j)."""
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
    xis = np.empty(P // 2, dtype=np.complex128)
    cs = np.empty(P // 2, dtype=np.complex128)
    for j in range(P // 2):
        t = complex(-K + (j + 0.5) * h, 0.5 * Kp)
        sn, cn, dn = _sn_cn_dn(t, k * k, kp2)
        wq = c0 * (1.0 / k + sn) / (1.0 / k - sn)
        dw = c0 * (2.0 / k) * cn * dn / (1.0 / k - sn) ** 2
        xis[j] = np.sqrt(wq - a)            # principal root: first quadrant
        cs[j] = h * dw / (2.0 * math.pi * xis[j])
    return xis, cs


def _poles_for_function(phi, kT: float, mu: float, emin: float, emax: float, P: int):
    """Step 5 for any phi(x) analytic off the Matsubara rays: node j gives
    z = mu + xi_j with weight c_j phi(xi_j) and z = mu - conj(xi_j) with
    weight conj(c_j phi(-xi_j))."""
    xis, cs = _contour_nodes(kT, mu, emin, emax, P)
    z = np.empty(P, dtype=np.complex128)
    w = np.empty(P, dtype=np.complex128)
    for j, (xi, cj) in enumerate(zip(xis, cs)):
        z[2 * j] = mu + xi
        w[2 * j] = cj * phi(np.array([xi]), kT)[0]
        z[2 * j + 1] = mu - np.conj(xi)
        w[2 * j + 1] = np.conj(cj * phi(np.array([-xi]), kT)[0])
    return z, w


def fermi_poles(kT: float, mu: float, emin: float, emax: float, P: int):
    """Poles z (complex128[P], Im > 0) and weights w (complex128[P])."""
    return _poles_for_function(fermi, kT, mu, emin, emax, P)


def entropy_weights(kT: float, mu: float, emin: float, emax: float, P: int):
    """Weights w^S (complex128[P]) on the poles of fermi_poles with the same
    arguments, such that sum_p Im(w^S_p / (eps - z_p)) ~= phi_S(eps - mu)
    (entropy_fn): step 1's contour integral taken of phi_S instead of g.
    phi_S has its singularities at the same Matsubara points as g, so the
    same quadrature nodes serve it and no further solves are needed: the
    entropy term per node is s_j = 2 kT sum_p Im(w^S_p x_jp(j))."""
    return _poles_for_function(entropy_fn, kT, mu, emin, emax, P)[1]


def rational(eps, z, w):
    """r(eps) = sum_p Im(w_p/(eps - z_p)) for real eps (vectorised)."""
    eps = np.asarray(eps, dtype=np.float64)
    return np.imag(w[None, :] / (eps.reshape(-1, 1) - z[None, :])).sum(axis=1).reshape(eps.shape)


def rational_times_eps(eps, z, w):
    """eps r(eps) = sum_p Im(w_p (1 + z_p/(eps - z_p))) (band-energy weight)."""
    eps = np.asarray(eps, dtype=np.float64)
    t = w[None, :] * (1.0 + z[None, :] / (eps.reshape(-1, 1) - z[None, :]))
    return np.imag(t).sum(axis=1).reshape(eps.shape)
