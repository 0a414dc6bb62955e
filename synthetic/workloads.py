"""Synthetic Mg-like workloads for the nodal-density path.

Each workload is a seeded, fully deterministic set of plain arrays:

* a uniform real-space grid (nx, ny, nz) with spacing (hx, hy, hz), linear
  index ``g = ix + nx*(iy + ny*iz)`` (x fastest), periodic or not per axis;
* atoms of an hcp lattice (a = 6.06 bohr, c/a = 1.624), possibly displaced
  by a dislocation field, each carrying a Gaussian well depth D and width
  sigma;
* an additive seeded noise potential U[-0.05, 0.05] Ha on every grid point
  (SplitMix64 counter hash of the grid index);
* sampled electronic nodes (grid indices) with a cubic region half-width s
  per node (the region is the (2s+1)^3 cube centred on the node);
* the Fermi-Dirac parameters kT, mu, the pole count, and solver settings.

The paper's Mg systems (hcp magnesium with prismatic loops and screw
dislocations, Sections 4-5) are stood in for by these synthetic inputs: the
paper's pseudopotential and atomistic data are not used.  The recipes below
are the readings of the workload descriptions recorded in the design notes.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np

from .rng import uniform01

# Mg-like hcp lattice (bohr)
A_LAT = 6.06
C_OVER_A = 1.624
C_LAT = A_LAT * C_OVER_A

NOISE_AMPLITUDE = 0.05  # Ha, half-width of the uniform noise
NOISE_SEED = 1234


@dataclass
class Workload:
    name: str
    shape: tuple            # (nx, ny, nz)
    spacing: tuple          # (hx, hy, hz) bohr
    periodic: tuple         # (px, py, pz) bools
    fd_order: int           # 4 -> 13-point, 8 -> 25-point Laplacian
    atoms: np.ndarray       # (n_atoms, 3) float64, bohr, inside the box
    depth: np.ndarray       # (n_atoms,) Gaussian well depth D (Ha)
    sigma: np.ndarray       # (n_atoms,) Gaussian width (bohr)
    v_ext: np.ndarray       # (N,) float64 additive potential (seeded noise)
    nodes: np.ndarray       # (n_nodes,) int64 grid indices
    halfwidth: np.ndarray   # (n_nodes,) int32 region half-width s
    kT: float = 0.01
    mu: float = 0.2
    n_poles: int = 16
    precision: str = "fp64"  # "fp64" or "mixed"
    tol: float = 1e-10
    maxit: int = 20000
    cutoff_sigmas: float = 8.0
    nonlocal_proj: bool = False
    proj_sigma: float = 1.0
    proj_rc: float = 4.0
    e_s: float = 0.5
    e_p: float = 0.25
    meta: dict = field(default_factory=dict)

    @property
    def n_grid(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz

    @property
    def dV(self) -> float:
        return float(self.spacing[0] * self.spacing[1] * self.spacing[2])

    @property
    def box(self) -> tuple:
        return tuple(n * h for n, h in zip(self.shape, self.spacing))

    @property
    def n_systems(self) -> int:
        return int(len(self.nodes) * self.n_poles)

    def region_points(self) -> np.ndarray:
        """Number of points of each node's region (full periodic axes kept)."""
        out = np.ones(len(self.nodes), dtype=np.int64)
        for d in range(3):
            m = 2 * self.halfwidth.astype(np.int64) + 1
            n = self.shape[d]
            if self.periodic[d]:
                m = np.minimum(m, n)
            out *= m
        return out

    def node_coords(self) -> np.ndarray:
        nx, ny, _ = self.shape
        g = self.nodes.astype(np.int64)
        return np.stack([g % nx, (g // nx) % ny, g // (nx * ny)], axis=1)

    def subset(self, idx) -> "Workload":
        """Same Hamiltonian, only the selected nodes."""
        idx = np.asarray(idx)
        return replace(self, nodes=self.nodes[idx].copy(),
                       halfwidth=self.halfwidth[idx].copy(),
                       meta=dict(self.meta, subset_of=self.name))

    def with_atoms(self, atoms: np.ndarray) -> "Workload":
        return replace(self, atoms=np.ascontiguousarray(atoms, dtype=np.float64))


# ---------------------------------------------------------------------------
# geometry helpers (positions only)
# ---------------------------------------------------------------------------

def hcp_sites(n1: int, n2: int, n3: int) -> np.ndarray:
    """Sites i*a1 + j*a2 + k*a3 + basis of an hcp lattice (unwrapped).

    a1 = (a, 0, 0), a2 = (-a/2, a*sqrt(3)/2, 0), a3 = (0, 0, c); basis
    (0, 0, 0) and (1/3, 2/3, 1/2) in lattice coordinates.
    """
    a1 = np.array([A_LAT, 0.0, 0.0])
    a2 = np.array([-0.5 * A_LAT, 0.5 * math.sqrt(3.0) * A_LAT, 0.0])
    a3 = np.array([0.0, 0.0, C_LAT])
    basis = np.array([[0.0, 0.0, 0.0], [1.0 / 3.0, 2.0 / 3.0, 0.5]])
    i, j, k = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    lat = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    out = []
    for b in basis:
        f = lat + b
        out.append(f[:, :1] * a1 + f[:, 1:2] * a2 + f[:, 2:3] * a3)
    # interleave so atom order is cell-major, basis-minor
    pos = np.stack(out, axis=1).reshape(-1, 3)
    return pos


def periodic_hcp_cell(n: int) -> tuple:
    """n x n x n hexagonal cells (2 n^3 atoms) wrapped into the orthogonal
    box (n a, n a, n c)."""
    box = np.array([n * A_LAT, n * A_LAT, n * C_LAT])
    pos = np.mod(hcp_sites(n, n, n), box)
    return pos, box


def noise_potential(n_grid: int, seed: int = NOISE_SEED) -> np.ndarray:
    u = uniform01(seed, np.arange(n_grid, dtype=np.uint64))
    return NOISE_AMPLITUDE * (2.0 * u - 1.0)


def sample_uniform_nodes(n_grid: int, n_nodes: int, seed: int) -> np.ndarray:
    """n_nodes distinct grid points: the n_nodes smallest hash keys."""
    keys = uniform01(seed, np.arange(n_grid, dtype=np.uint64))
    sel = np.argpartition(keys, n_nodes - 1)[:n_nodes]
    sel = sel[np.argsort(keys[sel], kind="stable")]
    return sel.astype(np.int64)


def sample_weighted_nodes(candidates: np.ndarray, weights: np.ndarray,
                          n_nodes: int, seed: int) -> np.ndarray:
    """Weighted sampling without replacement (Efraimidis & Spirakis 2006):
    key_i = u_i^(1/w_i), keep the n_nodes largest keys."""
    u = uniform01(seed, candidates.astype(np.uint64))
    u = np.maximum(u, 1e-300)
    keys = np.log(u) / weights
    sel = np.argpartition(-keys, n_nodes - 1)[:n_nodes]
    sel = sel[np.argsort(-keys[sel], kind="stable")]
    return candidates[sel].astype(np.int64)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def _periodic_bulk(name, ncell, shape, fd_order, n_poles, n_nodes, node_seed,
                   s, precision, nonlocal_proj=False, tol=1e-10):
    pos, box = periodic_hcp_cell(ncell)
    spacing = tuple(float(L / n) for L, n in zip(box, shape))
    n_grid = int(np.prod(shape))
    na = len(pos)
    return Workload(
        name=name, shape=tuple(shape), spacing=spacing,
        periodic=(True, True, True), fd_order=fd_order,
        atoms=pos, depth=np.full(na, 1.0), sigma=np.full(na, 1.2),
        v_ext=noise_potential(n_grid),
        nodes=sample_uniform_nodes(n_grid, n_nodes, node_seed),
        halfwidth=np.full(n_nodes, s, dtype=np.int32),
        n_poles=n_poles, precision=precision, tol=tol,
        nonlocal_proj=nonlocal_proj,
        meta={"ncell": ncell, "box": tuple(float(b) for b in box)})


def small_fp64() -> Workload:
    """16 atoms (2x2x2 hcp), 24x24x40 grid, 4th order, P=8, 32 nodes, 21^3."""
    return _periodic_bulk("small_fp64", 2, (24, 24, 40), 4, 8, 32, 1, 10, "fp64")


def bulk_mixed() -> Workload:
    """1,024 atoms (8x8x8 hcp), 96x96x160 grid, 8th order, nonlocal
    projectors, P=16, 4,096 nodes, 33^3 regions, mixed precision."""
    return _periodic_bulk("bulk_mixed", 8, (96, 96, 160), 8, 16, 4096, 2, 16,
                          "mixed", nonlocal_proj=True)


def adjoint_fp64() -> Workload:
    """128 atoms (4x4x4 hcp), 48x48x80 grid, 8th order, P=16, 1,024 nodes,
    33^3 regions, FP64; target density from a seeded 2% jitter."""
    w = _periodic_bulk("adjoint_fp64", 4, (48, 48, 80), 8, 16, 1024, 4, 16, "fp64")
    w.meta["jitter_seed"] = 5
    w.meta["jitter_frac"] = 0.02
    w.meta["fd_step"] = 1e-4
    w.meta["fd_atoms"] = 6
    w.meta["fd_seed"] = 7
    return w


def jittered_atoms(w: Workload) -> np.ndarray:
    """Atom positions displaced by U[-f a, f a] per component (seeded)."""
    seed = int(w.meta.get("jitter_seed", 5))
    f = float(w.meta.get("jitter_frac", 0.02))
    n = len(w.atoms)
    u = uniform01(seed, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3)
    pos = w.atoms + f * A_LAT * (2.0 * u - 1.0)
    return np.mod(pos, np.array(w.box))


def fd_atom_choice(w: Workload) -> np.ndarray:
    """The seeded atoms whose forces are checked by finite differences."""
    n = int(w.meta.get("fd_atoms", 6))
    keys = uniform01(int(w.meta.get("fd_seed", 7)), np.arange(len(w.atoms), dtype=np.uint64))
    return np.argsort(keys, kind="stable")[:n].astype(np.int64)


def _cylinder_sites(n_atoms: int, nz_cells: int, center_xy) -> np.ndarray:
    """The n_atoms hcp sites nearest the cylinder axis (ties by index)."""
    rad_cells = int(math.ceil(math.sqrt(n_atoms / (2 * nz_cells) * 2 / math.sqrt(3)) / 1.0)) + 4
    nn = 2 * rad_cells + 1
    pos = hcp_sites(nn, nn, nz_cells)
    a1 = np.array([A_LAT, 0.0, 0.0])
    a2 = np.array([-0.5 * A_LAT, 0.5 * math.sqrt(3.0) * A_LAT, 0.0])
    pos = pos - rad_cells * (a1 + a2)            # lattice origin near xy = 0
    # put the axis at the centre of a triangle of sites (no atom on the line)
    shift = np.array([0.5 * A_LAT, 0.5 * A_LAT / math.sqrt(3.0), 0.0])
    pos = pos - shift
    r = np.hypot(pos[:, 0], pos[:, 1])
    order = np.lexsort((np.arange(len(pos)), np.round(r, 9)))
    pos = pos[order[:n_atoms]]
    pos[:, 0] += center_xy[0]
    pos[:, 1] += center_xy[1]
    return pos


def screw_batched() -> Workload:
    """4,000-atom hcp cylinder (axis along c, length 8c, periodic in z) with
    a straight screw dislocation u_z = b atan2(y-y0, x-x0)/(2 pi),
    b = 6.06 bohr, on a 256x256x160 grid (h = 0.5, 0.5, c/20 bohr), non
    periodic in x and y; 1,250 nodes sampled with density 1/(1+(d/d0)^2)
    around the core, region half-width s(d) = clamp(20 - floor(d/l), 8, 20),
    P=16, mixed precision.
    """
    nz_cells = 8
    shape = (256, 256, 160)
    h = 0.5
    Lz = nz_cells * C_LAT
    spacing = (h, h, Lz / shape[2])
    box = (shape[0] * h, shape[1] * h, Lz)
    x0, y0 = 0.5 * box[0], 0.5 * box[1]
    pos = _cylinder_sites(4000, nz_cells, (x0, y0))
    b = A_LAT
    theta = np.arctan2(pos[:, 1] - y0, pos[:, 0] - x0)
    pos[:, 2] = np.mod(pos[:, 2] + b * theta / (2.0 * math.pi), Lz)
    r_cyl = float(np.max(np.hypot(pos[:, 0] - x0, pos[:, 1] - y0)))
    n_grid = int(np.prod(shape))
    # candidate nodes: grid points inside the cylinder
    g = np.arange(n_grid, dtype=np.int64)
    ix = g % shape[0]
    iy = (g // shape[0]) % shape[1]
    d = np.hypot(ix * spacing[0] - x0, iy * spacing[1] - y0)
    inside = d <= r_cyl
    cand = g[inside]
    d0 = 8.0
    wts = 1.0 / (1.0 + (d[inside] / d0) ** 2)
    nodes = sample_weighted_nodes(cand, wts, 1250, 3)
    dn = np.hypot((nodes % shape[0]) * spacing[0] - x0,
                  ((nodes // shape[0]) % shape[1]) * spacing[1] - y0)
    ell = r_cyl / 13.0
    s = np.clip(20 - np.floor(dn / ell).astype(np.int64), 8, 20).astype(np.int32)
    na = len(pos)
    return Workload(
        name="screw_batched", shape=shape, spacing=spacing,
        periodic=(False, False, True), fd_order=8,
        atoms=pos, depth=np.full(na, 1.0), sigma=np.full(na, 1.2),
        v_ext=noise_potential(n_grid), nodes=nodes, halfwidth=s,
        n_poles=16, precision="mixed",
        meta={"core_xy": (x0, y0), "burgers": b, "r_cyl": r_cyl,
              "d0": d0, "ell": ell, "box": box})


def large_loop(n_atoms: int = 100_000, nz_cells: int = 24, n_nodes: int = 200_000,
               node_seed: int = 6, candidate_stride: int = 2) -> Workload:
    """hcp cylinder of n_atoms sites (axis along c, length nz_cells c,
    periodic in z) carrying a prismatic dislocation loop of radius R = 40
    bohr in the plane z0 = L_z/2 around the axis, with the synthetic
    displacement
        u_z = -(b/2) sgn(z - z0) exp(-|z - z0|/R) sigma((R - rho)/w),
    b = c/2, w = 2 bohr, sigma the logistic function, rho the distance to
    the axis; the 20 sites nearest the loop-plane diameter along x (within
    R + 10 bohr of the axis) are Al-like wells of depth 1.3 Ha.  Grid
    h = 0.5 bohr in x, y (open, 11 bohr vacuum margin) and ~0.5 bohr in z,
    8th order; n_nodes nodes sampled (on the sub-lattice of every
    candidate_stride-th grid point inside the cylinder) with density
    1/(1 + (d/8)^2), d the distance to the loop line, region half-width
    s(d) = clamp(20 - floor(d/l), 8, 20), l = r_cyl/13; P = 16, mixed.
    meta["force_atoms"]: the 2,000 sites nearest the loop line.
    """
    Lz = nz_cells * C_LAT
    per_area = 2.0 / (0.5 * math.sqrt(3.0) * A_LAT ** 2)        # sites per bohr^2 per cell layer
    r_est = math.sqrt(n_atoms / (nz_cells * per_area * math.pi))
    h = 0.5
    nxy = 2 * int(math.ceil((r_est + 4.0 + 11.0) / h))
    nz = 2 * int(round(Lz / h / 2.0))
    shape = (nxy, nxy, nz)
    spacing = (h, h, Lz / nz)
    box = (nxy * h, nxy * h, Lz)
    x0, y0 = 0.5 * box[0], 0.5 * box[1]
    z0 = 0.5 * Lz
    pos = _cylinder_sites(n_atoms, nz_cells, (x0, y0))
    R, b, wd = 40.0, 0.5 * C_LAT, 2.0
    rho = np.hypot(pos[:, 0] - x0, pos[:, 1] - y0)
    dz = pos[:, 2] - z0
    uz = -0.5 * b * np.sign(dz) * np.exp(-np.abs(dz) / R) / (1.0 + np.exp(-(R - rho) / wd))
    pos[:, 2] = np.mod(pos[:, 2] + uz, Lz)
    r_cyl = float(np.max(np.hypot(pos[:, 0] - x0, pos[:, 1] - y0)))
    na = len(pos)
    depth = np.full(na, 1.0)
    near_line = np.hypot(pos[:, 1] - y0, pos[:, 2] - z0)
    ok = np.abs(pos[:, 0] - x0) <= R + 10.0
    cand_al = np.nonzero(ok)[0]
    al = cand_al[np.lexsort((cand_al, np.round(near_line[cand_al], 9)))[:20]]
    depth[al] = 1.3
    d_atom = np.hypot(np.hypot(pos[:, 0] - x0, pos[:, 1] - y0) - R, pos[:, 2] - z0)
    force_atoms = np.lexsort((np.arange(na), np.round(d_atom, 9)))[:2000].astype(np.int64)
    n_grid = int(np.prod(shape))
    # candidate nodes: every candidate_stride-th grid point inside the cylinder
    st = candidate_stride
    ix, iy, iz = np.meshgrid(np.arange(0, shape[0], st), np.arange(0, shape[1], st),
                             np.arange(0, shape[2], st), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    rr = np.hypot(ix * spacing[0] - x0, iy * spacing[1] - y0)
    keep = rr <= r_cyl
    ix, iy, iz, rr = ix[keep], iy[keep], iz[keep], rr[keep]
    cand = (ix + shape[0] * (iy + shape[1] * iz)).astype(np.int64)
    d = np.hypot(rr - R, iz * spacing[2] - z0)
    nodes = sample_weighted_nodes(cand, 1.0 / (1.0 + (d / 8.0) ** 2), min(n_nodes, len(cand)), node_seed)
    dn = np.hypot(np.hypot((nodes % shape[0]) * spacing[0] - x0,
                           ((nodes // shape[0]) % shape[1]) * spacing[1] - y0) - R,
                  (nodes // (shape[0] * shape[1])) * spacing[2] - z0)
    ell = r_cyl / 13.0
    s = np.clip(20 - np.floor(dn / ell).astype(np.int64), 8, 20).astype(np.int32)
    return Workload(
        name="large_loop", shape=shape, spacing=spacing,
        periodic=(False, False, True), fd_order=8,
        atoms=pos, depth=depth, sigma=np.full(na, 1.2),
        v_ext=noise_potential(n_grid), nodes=nodes, halfwidth=s,
        n_poles=16, precision="mixed",
        meta={"loop_center": (x0, y0, z0), "loop_radius": R, "burgers": b, "r_cyl": r_cyl,
              "al_atoms": al.astype(np.int64), "force_atoms": force_atoms, "ell": ell, "box": box})


def tiny(shape=(6, 6, 8), n_atoms=3, fd_order=4, s=2, n_nodes=6, seed=11,
         nonlocal_proj=False, n_poles=8, spacing=(0.55, 0.6, 0.5),
         periodic=(True, True, True)) -> Workload:
    """A few atoms at seeded random positions on a tiny grid (pins/tests)."""
    box = np.array([n * h for n, h in zip(shape, spacing)])
    u = uniform01(seed, np.arange(3 * n_atoms, dtype=np.uint64)).reshape(n_atoms, 3)
    pos = u * box
    n_grid = int(np.prod(shape))
    du = uniform01(seed + 1, np.arange(2 * n_atoms, dtype=np.uint64)).reshape(n_atoms, 2)
    return Workload(
        name=f"tiny_{shape[0]}x{shape[1]}x{shape[2]}", shape=tuple(shape),
        spacing=tuple(spacing), periodic=tuple(periodic), fd_order=fd_order,
        atoms=pos, depth=0.5 + du[:, 0], sigma=0.8 + 0.6 * du[:, 1],
        v_ext=noise_potential(n_grid, seed + 2),
        nodes=sample_uniform_nodes(n_grid, n_nodes, seed + 3),
        halfwidth=np.full(n_nodes, s, dtype=np.int32),
        n_poles=n_poles, tol=1e-12, nonlocal_proj=nonlocal_proj,
        meta={"box": tuple(float(b) for b in box)})


WORKLOADS = {
    "small_fp64": small_fp64,
    "bulk_mixed": bulk_mixed,
    "screw_batched": screw_batched,
    "adjoint_fp64": adjoint_fp64,
    "large_loop": large_loop,
}


def make_workload(name: str, **kw) -> Workload:
    if name == "tiny":
        return tiny(**kw)
    return WORKLOADS[name](**kw)
