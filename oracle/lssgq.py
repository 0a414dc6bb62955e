"""Oracle: Lanczos spectral Gauss quadrature (LSSGQ), the paper's own way to
the nodal fields (Section 2.1, Eq. 9, Eqs. (Fermi:Rho), (Electron_density:GQ)
and (tot)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For node j the spectral measure of H_R(j) contracted with e_j is replaced by
a K-point Gauss rule.  K steps of the symmetric Lanczos process from
q_1 = e_j give the Jacobi matrix T_K (diagonal alpha_1..alpha_K, off-diagonal
beta_1..beta_{K-1}); its eigenvalues are the quadrature nodes lambda_k and the
squared first components of its unit eigenvectors are the weights w_k
(Golub & Welsch, Math. Comp. 23, 1969).  Then, with g the Fermi-Dirac
function of Eq. (dm) at Fermi level mu and temperature kT,

    rho_j = (2/dV) sum_k w_k g(lambda_k)                    Eq. (Electron_density:GQ)
    e_j   = 2 sum_k w_k lambda_k g(lambda_k)                first term of Eq. (tot)
    s_j   = -2 kT sum_k w_k [g ln g + (1-g) ln(1-g)]         last term of Eq. (tot)
    N_e(mu) = 2 sum_j nu_j sum_k w_k g(lambda_k; mu)          Eq. (Fermi:Rho)

where nu_j is the number of grid points node j stands for (1 when every grid
point is a node).  Because lambda_k and w_k do not depend on mu, the Fermi
level that makes N_e(mu) equal a given electron count is found afterwards by
bisection on the stored rules (N_e is increasing in mu).

The Lanczos process stops early at step k < K when beta_k falls to
breakdown_tol * (|alpha_1| + beta_1 + 1): the Krylov space is then invariant
and the k-point rule is exact.  No reorthogonalisation, as in the plain
process; the quadrature it produces still reproduces the moments
(e_j^T H_R^m e_j for m < 2K) to rounding.

Plain NumPy, FP64; the region operator is applied with whole-array shifts.
"""
import math

import numpy as np
from scipy.linalg import eigh_tridiagonal
from scipy.special import expit

from . import hamiltonian as ham_mod


class RegionOperator:
    """v -> H_R v on one region: the FD kinetic stencil restricted to the
    region (zero outside on window axes, wrapped on ring axes), the local
    potential on the diagonal, and sum_{a,l} E_l dV p_al (p_al . v)."""

    def __init__(self, w, H, region):
        self.dims = region.dims            # (mx, my, mz), x fastest
        self.ring = region.ring
        self.stencil = H.stencil
        self.V = H.V[region.gidx]
        self.dV = w.dV
        self.projs = ham_mod.projectors_in_region(H.projs, region, w.n_grid)

    def apply(self, v):
        """H_R v on the region (stencil with Dirichlet faces or ring wrap,
        local potential, projectors restricted to R)."""
        mx, my, mz = self.dims
        u = v.reshape(mz, my, mx)
        out = (self.stencil.diag + self.V.reshape(mz, my, mx)) * u
        # array axis of grid axis d: x -> 2, y -> 1, z -> 0
        for d, ax in ((0, 2), (1, 1), (2, 0)):
            m = u.shape[ax]
            for o in range(1, self.stencil.q + 1):
                c = self.stencil.coef[d, o - 1]
                if self.ring[d]:
                    out = out + c * (np.roll(u, o, axis=ax) + np.roll(u, -o, axis=ax))
                elif o < m:
                    up = np.zeros_like(u)
                    dn = np.zeros_like(u)
                    src_hi = [slice(None)] * 3
                    dst_lo = [slice(None)] * 3
                    src_hi[ax] = slice(o, m)
                    dst_lo[ax] = slice(0, m - o)
                    up[tuple(dst_lo)] = u[tuple(src_hi)]     # u(i + o)
                    dn[tuple(src_hi)] = u[tuple(dst_lo)]     # u(i - o)
                    out = out + c * (up + dn)
        out = out.reshape(-1)
        for li, val, e in self.projs:
            out[li] += e * self.dV * val * float(np.dot(val, v[li]))
        return out


def lanczos(op: RegionOperator, src: int, K: int, breakdown_tol: float = 1e-13):
    """Symmetric Lanczos from e_src: alpha (k,), beta (k-1,) with k <= K."""
    n = int(np.prod(op.dims))
    q_prev = np.zeros(n)
    q = np.zeros(n)
    q[src] = 1.0
    alpha, beta = [], []
    b_prev = 0.0
    scale = None
    for k in range(K):
        wv = op.apply(q) - b_prev * q_prev
        a = float(np.dot(q, wv))
        wv = wv - a * q
        b = math.sqrt(float(np.dot(wv, wv)))
        alpha.append(a)
        if scale is None:
            scale = abs(a) + b + 1.0
        if k == K - 1 or b <= breakdown_tol * scale:
            break
        beta.append(b)
        q_prev, q = q, wv / b
        b_prev = b
    return np.array(alpha), np.array(beta)


def gauss_rule(alpha, beta):
    """Nodes and weights of the Gauss rule of the Jacobi matrix (alpha, beta)."""
    if len(alpha) == 1:
        return np.array(alpha, dtype=float), np.ones(1)
    lam, U = eigh_tridiagonal(alpha, beta)
    return lam, U[0, :] ** 2


def fermi(eps, mu, kT):
    """g(eps; mu) = 1 / (1 + exp((eps - mu)/kT)) of Eq. (dm) (the logistic
    function of -(eps - mu)/kT, accurate also where g is tiny)."""
    x = (np.asarray(eps, dtype=float) - mu) / kT
    return expit(-x)


def entropy_density(eps, mu, kT):
    """g ln g + (1-g) ln(1-g) at eps, written to stay finite for |x| large:
    with x = (eps - mu)/kT, ln g = -ln(1 + e^x), ln(1-g) = -ln(1 + e^-x)."""
    x = (np.asarray(eps, dtype=float) - mu) / kT
    g = expit(-x)
    one_minus_g = expit(x)          # not 1 - g: keeps e^-|x| where g ~ 1
    l_pos = np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))     # ln(1 + e^x)
    l_neg = np.maximum(-x, 0.0) + np.log1p(np.exp(-np.abs(x)))    # ln(1 + e^-x)
    return -g * l_pos - one_minus_g * l_neg


def quadrature(w, H, nodes, halfwidth, K: int, breakdown_tol: float = 1e-13):
    """Gauss rules of every node: lam, wts (n_nodes, K), padded with weight
    0 beyond each node's k_used; k_used (n_nodes,)."""
    n = len(nodes)
    lam = np.zeros((n, K))
    wts = np.zeros((n, K))
    k_used = np.zeros(n, dtype=np.int32)
    for j, (node, s) in enumerate(zip(nodes, halfwidth)):
        region = ham_mod.region_of(w, int(node), int(s))
        op = RegionOperator(w, H, region)
        a, b = lanczos(op, region.src, K, breakdown_tol)
        l, g = gauss_rule(a, b)
        k = len(a)
        lam[j, :k] = l
        lam[j, k:] = l[-1]
        wts[j, :k] = g
        k_used[j] = k
    return lam, wts, k_used


def fields(lam, wts, mu, kT, dV):
    """rho_j, e_j, s_j of Eqs. (Electron_density:GQ) and (tot) per node."""
    g = fermi(lam, mu, kT)
    rho = (2.0 / dV) * np.sum(wts * g, axis=1)
    e = 2.0 * np.sum(wts * lam * g, axis=1)
    s = -2.0 * kT * np.sum(wts * entropy_density(lam, mu, kT), axis=1)
    return rho, e, s


def electron_count(lam, wts, mu, kT, nu=None):
    """N_e(mu) of Eq. (Fermi:Rho) with node weights nu (default 1)."""
    per_node = 2.0 * np.sum(wts * fermi(lam, mu, kT), axis=1)
    if nu is None:
        return float(np.sum(per_node))
    return float(np.sum(np.asarray(nu, dtype=float) * per_node))


def fermi_level(lam, wts, kT, n_electrons, nu=None, iters: int = 200):
    """mu with N_e(mu) = n_electrons, by bisection on [min lam - 40 kT,
    max lam + 40 kT] (N_e is increasing in mu); stops when the bracket no
    longer shrinks."""
    lo = float(np.min(lam)) - 40.0 * kT
    hi = float(np.max(lam)) + 40.0 * kT
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if electron_count(lam, wts, mid, kT, nu) < n_electrons:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
