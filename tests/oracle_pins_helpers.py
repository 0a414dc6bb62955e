"""Independent brute-force constructions used to pin the oracle.

Nothing here calls the oracle's Hamiltonian code: the FD weights come from
the textbook table in tests/golden, the operator is assembled as dense
Kronecker products, and spectra come from numpy.linalg.
"""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_fd_weights() -> dict:
    out = {}
    with open(os.path.join(GOLDEN, "fd_weights_fornberg1988.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            order, rest = line.split(":")
            out[int(order)] = np.array([float(Fraction(t)) for t in rest.split()])
    return out


def dense_1d(m: int, ring: bool, weights: np.ndarray, h: float) -> np.ndarray:
    """-1/2 d^2/dx^2 on m points: Dirichlet window or periodic ring."""
    q = len(weights) - 1
    T = np.zeros((m, m))
    for i in range(m):
        T[i, i] += -0.5 * weights[0] / h ** 2
        for o in range(1, q + 1):
            for t in (i + o, i - o):
                if ring:
                    T[i, t % m] += -0.5 * weights[o] / h ** 2
                elif 0 <= t < m:
                    T[i, t] += -0.5 * weights[o] / h ** 2
    return T


def dense_region_hamiltonian(dims, ring, spacing, order, V_region, projs=(), dV=None):
    """Dense H_R, local index x fastest: H = Tx(+)Ty(+)Tz + diag(V) + nonlocal."""
    w = golden_fd_weights()[order]
    mx, my, mz = dims
    Tx = dense_1d(mx, ring[0], w, spacing[0])
    Ty = dense_1d(my, ring[1], w, spacing[1])
    Tz = dense_1d(mz, ring[2], w, spacing[2])
    Ix, Iy, Iz = np.eye(mx), np.eye(my), np.eye(mz)
    H = (np.kron(Iz, np.kron(Iy, Tx)) + np.kron(Iz, np.kron(Ty, Ix))
         + np.kron(Tz, np.kron(Iy, Ix)))
    H = H + np.diag(V_region)
    for li, val, e in projs:
        p = np.zeros(H.shape[0])
        p[li] = val
        H = H + e * dV * np.outer(p, p)
    return H


def fd_symbol(k, h, weights):
    """Eigenvalue of -1/2 d^2/dx^2 (FD) on the plane wave exp(i k x)."""
    q = len(weights) - 1
    s = weights[0] + 2.0 * sum(weights[o] * np.cos(k * o * h) for o in range(1, q + 1))
    return -0.5 * s / h ** 2
