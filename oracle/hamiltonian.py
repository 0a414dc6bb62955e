"""Oracle: the discrete Kohn-Sham Hamiltonian on the real-space grid.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's Hamiltonian is H = -1/2 Laplacian + u + phi (Eq. Hamiltonian),
discretised by central finite differences on a uniform grid with an
orthonormal grid basis (Section 2.1, "sixth order finite difference").  Here
the effective potential u + phi is replaced by a synthetic local potential

    V(r_i) = sum_a -D_a exp(-|r_i - R_a|^2 / (2 sigma_a^2)) + v_ext(r_i)

(minimum-image distance on periodic axes, Gaussian cut off at 8 sigma), and
an optional separable nonlocal term sum_{a,l} E_l dV |p_al><p_al| with four
Gaussian projectors per atom (s, p_x, p_y, p_z), each normalised to
dV sum_i p^2 = 1 on the grid.  The FD order is 4 or 8 (13- or 25-point
stencil) as the workloads ask, instead of the paper's 6th order.

Everything here is plain NumPy in FP64, written for reading, not speed.
"""
import math
from dataclasses import dataclass

import numpy as np


def fd_second_derivative_weights(order: int) -> np.ndarray:
    """Central weights w_0..w_q of d^2/dx^2 of accuracy order 2q (h = 1).

    Closed form of the maximal-order central stencil:
        w_o = 2 (-1)^(o+1) (q!)^2 / (o^2 (q-o)! (q+o)!),  o = 1..q
        w_0 = -2 sum_{o=1}^{q} 1/o^2
    """
    if order % 2 or order < 2:
        raise ValueError("order must be even and >= 2")
    q = order // 2
    w = np.zeros(q + 1)
    fq = math.factorial(q)
    for o in range(1, q + 1):
        w[o] = 2.0 * (-1) ** (o + 1) * fq * fq / (o * o * math.factorial(q - o) * math.factorial(q + o))
    w[0] = -2.0 * sum(1.0 / (o * o) for o in range(1, q + 1))
    return w


@dataclass
class Stencil:
    """Kinetic part -1/2 Laplacian: off-diagonal weights per axis and the
    constant diagonal."""
    q: int
    coef: np.ndarray   # (3, q): weight of the +-o neighbour on axis d
    diag: float        # constant diagonal of -1/2 Laplacian


def kinetic_stencil(spacing, order: int) -> Stencil:
    """-1/2 of the FD Laplacian (Section 2.1's finite-difference
    discretisation) per axis: off-centre coefficients for offsets 1..q and
    the constant diagonal, from the central second-derivative weights."""
    w = fd_second_derivative_weights(order)
    q = order // 2
    coef = np.zeros((3, q))
    diag = 0.0
    for d in range(3):
        h2 = spacing[d] ** 2
        coef[d, :] = -0.5 * w[1:] / h2
        diag += -0.5 * w[0] / h2
    return Stencil(q=q, coef=coef, diag=diag)


def _axis_displacements(n: int, h: float, L: float, periodic: bool, X: float, rc: float):
    """Grid indices on one axis within rc of coordinate X and their
    (minimum-image, if periodic) displacements i*h - X."""
    i = np.arange(n)
    d = i * h - X
    if periodic:
        d = d - L * np.round(d / L)
    keep = np.abs(d) <= rc
    return i[keep], d[keep]


def _atom_box(w, R, rc):
    """Index sets and displacements of the grid points within the cube of
    half-side rc around R (minimum image on periodic axes)."""
    box = w.box
    parts = [_axis_displacements(w.shape[d], w.spacing[d], box[d], w.periodic[d], R[d], rc)
             for d in range(3)]
    return parts


def local_potential(w) -> np.ndarray:
    """V on the whole grid, flat (x fastest), FP64."""
    nx, ny, nz = w.shape
    V = np.zeros((nz, ny, nx))
    for a in range(len(w.atoms)):
        R = w.atoms[a]
        sig = float(w.sigma[a])
        rc = w.cutoff_sigmas * sig
        (ix, dx), (iy, dy), (iz, dz) = _atom_box(w, R, rc)
        if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
            continue
        r2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
        g = np.where(r2 <= rc * rc, -float(w.depth[a]) * np.exp(-r2 / (2.0 * sig * sig)), 0.0)
        V[np.ix_(iz, iy, ix)] += g
    return V.reshape(-1) + np.asarray(w.v_ext, dtype=np.float64)


def local_potential_on(w, gidx) -> np.ndarray:
    """V at the grid points gidx only (flat indices, x fastest): the same sum
    of wells as local_potential plus v_ext there, for grids too large to
    fill whole.  Atoms farther than the cutoff from the points' bounding box
    (minimum image on periodic axes) are skipped before the per-atom sum."""
    nx, ny, _ = w.shape
    gidx = np.asarray(gidx, dtype=np.int64)
    idx = (gidx % nx, (gidx // nx) % ny, gidx // (nx * ny))
    coords = [idx[d] * w.spacing[d] for d in range(3)]
    box = w.box
    lo = np.array([c.min() for c in coords])
    hi = np.array([c.max() for c in coords])
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    rc_all = w.cutoff_sigmas * np.asarray(w.sigma, dtype=np.float64)
    near = np.ones(len(w.atoms), dtype=bool)
    for d in range(3):
        dd = w.atoms[:, d] - mid[d]
        if w.periodic[d]:
            dd = dd - box[d] * np.round(dd / box[d])
        near &= np.abs(dd) <= half[d] + rc_all
    V = np.zeros(len(gidx))
    for a in np.nonzero(near)[0]:
        R = w.atoms[a]
        sig = float(w.sigma[a])
        rc = rc_all[a]
        r2 = np.zeros(len(gidx))
        for d in range(3):
            dd = coords[d] - R[d]
            if w.periodic[d]:
                dd = dd - box[d] * np.round(dd / box[d])
            r2 += dd * dd
        m = r2 <= rc * rc
        V[m] += -float(w.depth[a]) * np.exp(-r2[m] / (2.0 * sig * sig))
    return V + np.asarray(w.v_ext, dtype=np.float64)[gidx]


def local_potential_gradient_terms(w, a: int):
    """Grid points touched by atom a and dV_k/dR_a (3 columns) there."""
    R = w.atoms[a]
    sig = float(w.sigma[a])
    rc = w.cutoff_sigmas * sig
    (ix, dx), (iy, dy), (iz, dz) = _atom_box(w, R, rc)
    nx, ny, _ = w.shape
    Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
    DZ, DY, DX = np.meshgrid(dz, dy, dx, indexing="ij")
    r2 = DX ** 2 + DY ** 2 + DZ ** 2
    m = r2 <= rc * rc
    Va = -float(w.depth[a]) * np.exp(-r2[m] / (2.0 * sig * sig))
    gidx = (X[m] + nx * (Y[m] + ny * Z[m])).astype(np.int64)
    # d/dR of -D exp(-|r-R|^2/(2 s^2)) = V_a(r) (r - R)/s^2
    dV = np.stack([Va * DX[m], Va * DY[m], Va * DZ[m]], axis=1) / (sig * sig)
    return gidx, dV


@dataclass
class Projector:
    """One nonlocal projector p_al of atom a (an s or p Gaussian, zero
    beyond the cutoff radius): its grid support, its normalised values there
    and its energy E_l."""
    idx: np.ndarray    # grid indices of the support (r <= rc)
    val: np.ndarray    # normalised values there
    energy: float      # E_l
    atom: int
    kind: int          # 0 = s, 1..3 = p_x, p_y, p_z


def projectors(w) -> list:
    """The 4 normalised Gaussian projectors of every atom (empty if the
    workload has no nonlocal term)."""
    if not w.nonlocal_proj:
        return []
    nx, ny, _ = w.shape
    dV = w.dV
    out = []
    rc = w.proj_rc
    s2 = w.proj_sigma ** 2
    for a in range(len(w.atoms)):
        (ix, dx), (iy, dy), (iz, dz) = _atom_box(w, w.atoms[a], rc)
        Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
        DZ, DY, DX = np.meshgrid(dz, dy, dx, indexing="ij")
        r2 = DX ** 2 + DY ** 2 + DZ ** 2
        m = r2 <= rc * rc
        gidx = (X[m] + nx * (Y[m] + ny * Z[m])).astype(np.int64)
        g = np.exp(-r2[m] / (2.0 * s2))
        shapes = [g, DX[m] * g, DY[m] * g, DZ[m] * g]
        for kind, f in enumerate(shapes):
            nrm = math.sqrt(dV * float(np.sum(f * f)))
            e = w.e_s if kind == 0 else w.e_p
            out.append(Projector(idx=gidx, val=f / nrm, energy=e, atom=a, kind=kind))
    return out


def gershgorin_bounds(w, V: np.ndarray, projs: list) -> tuple:
    """[Emin, Emax] containing the spectrum of H (Gershgorin discs).

    Every H_R is a principal submatrix of H, so by Cauchy interlacing its
    spectrum lies in the same interval."""
    st = kinetic_stencil(w.spacing, w.fd_order)
    diag = st.diag + V.copy()
    radius = np.full(V.shape, 2.0 * np.abs(st.coef).sum())
    dV = w.dV
    for p in projs:
        s = np.abs(p.val).sum()
        diag[p.idx] += p.energy * dV * p.val * p.val
        radius[p.idx] += p.energy * dV * np.abs(p.val) * (s - np.abs(p.val))
    return float(np.min(diag - radius)), float(np.max(diag + radius))


@dataclass
class Region:
    """The cube R(j) around node j, mapped to global grid indices.

    Per axis: a window of 2s+1 points centred on the node (Dirichlet: H is
    restricted, so neighbours outside are absent), or, when 2s+1 >= n on a
    periodic axis, the whole axis as a ring (neighbours wrap)."""
    dims: tuple          # (mx, my, mz)
    ring: tuple          # per axis: whole periodic axis?
    gidx: np.ndarray     # (mz*my*mx,) global index of each local point, x fastest
    src: int             # local index of the node


def region_of(w, node: int, s: int) -> Region:
    """The truncation region R(j) of a node (Section 2.1's locality): the
    cube of side 2s+1 centred on it with H restricted to it (Dirichlet
    faces), wrapped on periodic axes, the whole axis as a ring where 2s+1
    reaches the axis length; raises if the cube leaves a non-periodic axis."""
    nx, ny, nz = w.shape
    c = (node % nx, (node // nx) % ny, node // (nx * ny))
    axes = []
    dims = []
    ring = []
    srcl = []
    for d, n in enumerate((nx, ny, nz)):
        m = 2 * s + 1
        if w.periodic[d] and m >= n:
            axes.append(np.arange(n))
            dims.append(n)
            ring.append(True)
            srcl.append(c[d])
        else:
            g = c[d] - s + np.arange(m)
            if w.periodic[d]:
                g = np.mod(g, n)
            elif g[0] < 0 or g[-1] >= n:
                raise ValueError("region leaves a non-periodic grid axis")
            axes.append(g)
            dims.append(m)
            ring.append(False)
            srcl.append(s)
    gz, gy, gx = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    gidx = (gx + nx * (gy + ny * gz)).reshape(-1).astype(np.int64)
    src = srcl[0] + dims[0] * (srcl[1] + dims[1] * srcl[2])
    return Region(dims=tuple(dims), ring=tuple(ring), gidx=gidx, src=int(src))


def projectors_in_region(projs: list, region: Region, n_grid: int):
    """Projectors restricted to a region: list of (local idx, values, E)."""
    if not projs:
        return []
    loc = np.full(n_grid, -1, dtype=np.int64)
    loc[region.gidx] = np.arange(len(region.gidx))
    out = []
    for p in projs:
        li = loc[p.idx]
        m = li >= 0
        if np.any(m):
            out.append((li[m], p.val[m], p.energy))
    return out
