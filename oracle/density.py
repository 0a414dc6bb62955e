"""Oracle: nodal density, band energy, adjoint and forces.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For node j with region R(j) and poles (z_p, w_p):

* density (Eq. Electron_density:GQ with g -> r):
      rho_j = (2/dV) sum_p Im( w_p x_jp(j) ),  (H_R - z_p) x_jp = e_j
* band energy per node (first term of Eq. tot, 2 [H r(H)]_jj, using
  eps r(eps) = sum_p Im(w_p + w_p z_p/(eps - z_p))):
      e_j = 2 sum_p Im( w_p (1 + z_p x_jp(j)) )
* adjoint: with G = (H_R - z)^-1 complex symmetric, dG_jj/dV_k = -G_jk^2 =
  -x_jp(k)^2, so for L(rho, e) with a_j = dL/drho_j, b_j = dL/de_j:
      dL/dV_k = -sum_j sum_p Im( (2 a_j/dV + 2 b_j z_p) w_p x_jp(k)^2 )
* Hellmann-Feynman forces (Section 2.1, last paragraph) through the local
  potential only:  F_a = -sum_k dL/dV_k dV_k/dR_a.

The Python side gathers each region and its projectors; the C side
(``cocg.c``) runs COCG per system.
"""
import ctypes
from dataclasses import dataclass

import numpy as np

from . import hamiltonian as ham_mod
from . import poles as poles_mod
from ._native import load_cocg


@dataclass
class OracleHamiltonian:
    """The discrete Hamiltonian of Section 2.1 (Eq. Hamiltonian) as the
    oracle holds it: local potential on the grid (or on requested points),
    the nonlocal projectors, the FD kinetic stencil and the spectral
    interval [emin, emax] the poles are built on."""
    V: np.ndarray
    projs: list
    stencil: ham_mod.Stencil
    emin: float
    emax: float


def build(w, points=None, bounds=None) -> OracleHamiltonian:
    """The Hamiltonian of workload w.  With `points` (flat grid indices, or
    a list of such arrays, e.g. one per region to be solved) V is computed
    there only (zero elsewhere) and the spectral interval must be given as
    `bounds` = (emin, emax), since Gershgorin needs V on the whole grid."""
    projs = ham_mod.projectors(w)
    st = ham_mod.kinetic_stencil(w.spacing, w.fd_order)
    if points is None:
        V = ham_mod.local_potential(w)
        emin, emax = ham_mod.gershgorin_bounds(w, V, projs) if bounds is None else bounds
    else:
        if bounds is None:
            raise ValueError("a restricted build needs explicit spectral bounds")
        V = np.zeros(w.n_grid)
        chunks = points if isinstance(points, (list, tuple)) else [points]
        for c in chunks:   # one region at a time keeps each atom filter local
            pts = np.unique(np.asarray(c, dtype=np.int64))
            V[pts] = ham_mod.local_potential_on(w, pts)
        emin, emax = bounds
    return OracleHamiltonian(V=V, projs=projs, stencil=st, emin=float(emin), emax=float(emax))


def region_points(w) -> list:
    """The grid points of every node's region, one array per node."""
    return [ham_mod.region_of(w, int(n), int(s)).gidx for n, s in zip(w.nodes, w.halfwidth)]


def poles_for(w, H: OracleHamiltonian):
    """The P poles and weights of the rational Fermi expansion (contour
    quadrature, see oracle/poles.py) on the Hamiltonian's spectral interval,
    at the workload's kT and mu."""
    return poles_mod.fermi_poles(w.kT, w.mu, H.emin, H.emax, w.n_poles)


@dataclass
class OracleResult:
    """Per-node density and band energy (Eq. Electron_density:GQ with the
    pole expansion; first term of Eq. tot), with each (node, pole) solve's
    x_jp(j), iteration count, residual and status."""
    rho: np.ndarray        # (n_nodes,)
    e_node: np.ndarray     # (n_nodes,)
    x_src: np.ndarray      # (n_nodes, P) complex
    iters: np.ndarray      # (n_nodes, P)
    resid: np.ndarray      # (n_nodes, P)
    status: np.ndarray     # (n_nodes, P)
    z: np.ndarray
    wts: np.ndarray
    regions: list
    x_full: list           # per node: (P, n_region) complex, or None


def _pack(w, H, nodes, halfwidth):
    regions = [ham_mod.region_of(w, int(n), int(s)) for n, s in zip(nodes, halfwidth)]
    dims = np.array([r.dims for r in regions], dtype=np.int32).reshape(-1)
    ring = np.array([r.ring for r in regions], dtype=np.int32).reshape(-1)
    src = np.array([r.src for r in regions], dtype=np.int32)
    sizes = np.array([len(r.gidx) for r in regions], dtype=np.int64)
    voff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    Vp = np.concatenate([H.V[r.gidx] for r in regions]).astype(np.float64)
    pptr_reg = [0]
    p_ptr = [0]
    p_idx, p_val, p_E = [], [], []
    for r in regions:
        plist = ham_mod.projectors_in_region(H.projs, r, w.n_grid)
        for li, val, e in plist:
            p_idx.append(li.astype(np.int32))
            p_val.append(val.astype(np.float64))
            p_E.append(e)
            p_ptr.append(p_ptr[-1] + len(li))
        pptr_reg.append(pptr_reg[-1] + len(plist))
    p_idx = np.concatenate(p_idx) if p_idx else np.zeros(1, np.int32)
    p_val = np.concatenate(p_val) if p_val else np.zeros(1, np.float64)
    p_E = np.array(p_E if p_E else [0.0], dtype=np.float64)
    return (regions, dims, ring, src, voff, Vp, np.array(pptr_reg, np.int64),
            np.array(p_ptr, np.int64), p_idx, p_val, p_E, sizes)


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def solve(w, H: OracleHamiltonian = None, z=None, wts=None, tol: float = 1e-12,
          maxit: int = None, keep_x: bool = False) -> OracleResult:
    """Run every (node, pole) system of the workload."""
    if H is None:
        H = build(w)
    if z is None:
        z, wts = poles_for(w, H)
    maxit = int(maxit if maxit is not None else w.maxit)
    (regions, dims, ring, src, voff, Vp, pptr_reg, p_ptr, p_idx, p_val, p_E,
     sizes) = _pack(w, H, w.nodes, w.halfwidth)
    n_nodes, P = len(regions), len(z)
    n_sys = n_nodes * P
    sys_reg = np.repeat(np.arange(n_nodes, dtype=np.int32), P)
    sys_z = np.empty(2 * n_sys)
    zz = np.tile(z, n_nodes)
    sys_z[0::2], sys_z[1::2] = zz.real, zz.imag
    x_src = np.zeros(2 * n_sys)
    iters = np.zeros(n_sys, np.int32)
    resid = np.zeros(n_sys)
    status = np.zeros(n_sys, np.int32)
    if keep_x:
        sys_sizes = np.repeat(sizes, P)
        sys_xoff = np.concatenate([[0], np.cumsum(sys_sizes)[:-1]]).astype(np.int64)
        x_full = np.zeros(2 * int(sys_sizes.sum()))
        xf_ptr, xo_ptr = _ptr(x_full, ctypes.c_double), _ptr(sys_xoff, ctypes.c_longlong)
    else:
        x_full, sys_xoff = None, None
        xf_ptr, xo_ptr = None, None
    st = H.stencil
    coef = np.ascontiguousarray(st.coef.reshape(-1))
    lib = load_cocg()
    lib.oracle_cocg_batch(
        n_sys, _ptr(sys_reg, ctypes.c_int), _ptr(sys_z, ctypes.c_double),
        _ptr(dims, ctypes.c_int), _ptr(ring, ctypes.c_int), _ptr(src, ctypes.c_int),
        _ptr(voff, ctypes.c_longlong), _ptr(Vp, ctypes.c_double),
        _ptr(pptr_reg, ctypes.c_longlong), _ptr(p_ptr, ctypes.c_longlong),
        _ptr(p_idx, ctypes.c_int), _ptr(p_val, ctypes.c_double), _ptr(p_E, ctypes.c_double),
        st.q, _ptr(coef, ctypes.c_double), ctypes.c_double(st.diag), ctypes.c_double(w.dV),
        ctypes.c_double(tol), maxit,
        _ptr(x_src, ctypes.c_double), xf_ptr, xo_ptr,
        _ptr(iters, ctypes.c_int), _ptr(resid, ctypes.c_double), _ptr(status, ctypes.c_int))
    xs = (x_src[0::2] + 1j * x_src[1::2]).reshape(n_nodes, P)
    rho = (2.0 / w.dV) * np.imag(wts[None, :] * xs).sum(axis=1)
    e_node = 2.0 * np.imag(wts[None, :] * (1.0 + z[None, :] * xs)).sum(axis=1)
    xf = None
    if keep_x:
        xc = x_full[0::2] + 1j * x_full[1::2]
        xf = []
        off = 0
        for r in range(n_nodes):
            n = int(sizes[r])
            xf.append(xc[off:off + n * P].reshape(P, n))
            off += n * P
    return OracleResult(rho=rho, e_node=e_node, x_src=xs, iters=iters.reshape(n_nodes, P),
                        resid=resid.reshape(n_nodes, P), status=status.reshape(n_nodes, P),
                        z=z, wts=wts, regions=regions, x_full=xf)


def entropy_node(res: OracleResult, w_entropy, kT: float) -> np.ndarray:
    """Entropy term per node (the last term of Eq. tot taken at node j,
    g ln g + (1-g) ln(1-g) replaced by the rational form of -phi_S built on
    the solve's own poles, poles.entropy_weights):
        s_j = 2 kT sum_p Im( w^S_p x_jp(j) )  ~=  2 kT [phi_S(H_R)]_jj >= 0."""
    return 2.0 * kT * np.imag(np.asarray(w_entropy)[None, :] * res.x_src).sum(axis=1)


def free_energy_terms(w, res: OracleResult, w_entropy, node_weight=None) -> dict:
    """Node-weighted totals of the cluster-sampled energy (Section 3, Eqs.
    free_cg and free_cg_sampling: E ~= sum_q n_q (1/N_q) sum_{p in C_q} F_p),
    here sum_j nu_j F_j over the nodes with weights nu_j (1 if None):
        n_electrons = dV sum_j nu_j rho_j        (Eq. Fermi:Rho)
        e_band      = sum_j nu_j e_j             (first term of Eq. tot)
        ts          = sum_j nu_j s_j             (entropy term, >= 0)
        free_energy = e_band - ts                (Mermin: E - TS)."""
    nu = np.ones(len(res.rho)) if node_weight is None else np.asarray(node_weight, dtype=np.float64)
    s = entropy_node(res, w_entropy, w.kT)
    n_e = float(w.dV * np.sum(nu * res.rho))
    eb = float(np.sum(nu * res.e_node))
    ts = float(np.sum(nu * s))
    return {"n_electrons": n_e, "e_band": eb, "ts": ts, "free_energy": eb - ts, "s_node": s}


def cluster_sampling(w, esp_nodes, n_q, radius: float):
    """Nodes and weights of the cluster-sampled energy (Section 3, Eq.
    free_cg with Eq. free_cg_sampling): C_q is the set of fine-grid points
    within `radius` (bohr; minimum image on periodic axes) of the q-th
    sampling point, N_q = |C_q|, and every p in C_q carries n_q / N_q, so
    that sum_p nu_p F_p = sum_q n_q (1/N_q) sum_{p in C_q} F_p.  Points in
    several clusters appear once with their weights summed.  Returns
    (nodes ascending, nu)."""
    esp_nodes = np.asarray(esp_nodes, dtype=np.int64)
    n_q = np.asarray(n_q, dtype=np.float64)
    nx, ny, nz = w.shape
    h = np.asarray(w.spacing, dtype=np.float64)
    acc = {}
    for q, g in enumerate(esp_nodes):
        c = np.array([g % nx, (g // nx) % ny, g // (nx * ny)])
        reach = np.floor(radius / h).astype(int) + 1
        o = np.stack(np.meshgrid(*[np.arange(-r, r + 1) for r in reach], indexing="ij"), -1).reshape(-1, 3)
        o = o[np.sum((o * h) ** 2, axis=1) <= radius * radius]
        p = c[None, :] + o
        keep = np.ones(len(p), bool)
        for d in range(3):
            if w.periodic[d]:
                p[:, d] %= w.shape[d]      # every image in the ball: the minimum one is among them
            else:
                keep &= (p[:, d] >= 0) & (p[:, d] < w.shape[d])
        pts = np.unique(p[keep, 0] + nx * (p[keep, 1] + ny * p[keep, 2]))
        for pt in pts:
            acc[int(pt)] = acc.get(int(pt), 0.0) + n_q[q] / len(pts)
    nodes = np.array(sorted(acc), dtype=np.int64)
    return nodes, np.array([acc[int(p)] for p in nodes])


def electron_count_poles(w, H: OracleHamiltonian, mu: float, node_weight=None, tol: float = 1e-12) -> float:
    """N(mu) = dV sum_j nu_j rho_j(mu) (Eq. Fermi:Rho with g -> r), each
    rho_j(mu) from a fresh pole set built at mu on H's spectral interval
    (nu_j = 1 if node_weight is None: every grid point a node)."""
    z, wts = poles_mod.fermi_poles(w.kT, mu, H.emin, H.emax, w.n_poles)
    res = solve(w, H, z=z, wts=wts, tol=tol)
    nu = np.ones(len(res.rho)) if node_weight is None else np.asarray(node_weight, dtype=np.float64)
    return float(w.dV * np.sum(nu * res.rho))


def fermi_level_poles(w, H: OracleHamiltonian, n_electrons: float, node_weight=None, mu_tol: float = 1e-11,
                      tol: float = 1e-12):
    """Fermi level of the pole form: the mu with electron_count_poles(mu) =
    n_electrons, by bisection on [emin, emax] (N rises from ~0 to ~2 sum nu
    across the interval) until the bracket is narrower than mu_tol.  Returns
    (mu, N(mu), evaluations)."""
    lo, hi = H.emin, H.emax
    n_lo = electron_count_poles(w, H, lo, node_weight, tol) - n_electrons
    n_hi = electron_count_poles(w, H, hi, node_weight, tol) - n_electrons
    if n_lo > 0 or n_hi < 0:
        raise ValueError("n_electrons is outside the count range on the spectral interval")
    evals = 2
    while hi - lo > mu_tol:
        mid = 0.5 * (lo + hi)
        n_mid = electron_count_poles(w, H, mid, node_weight, tol) - n_electrons
        evals += 1
        if n_mid < 0:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    return mu, electron_count_poles(w, H, mu, node_weight, tol), evals + 1


def density_matrix_rows(res: OracleResult) -> list:
    """Row j of the density matrix over R(j) (Eq. dm in the grid basis, g
    replaced by r): gamma_jk = sum_p Im(w_p x_jp(k)); rho_j = (2/dV) gamma_jj."""
    if res.x_full is None:
        raise ValueError("solve with keep_x=True first")
    return [np.imag((res.wts[:, None] * xf).sum(axis=0)) for xf in res.x_full]


def dL_dV(w, res: OracleResult, a_node, b_node=None) -> np.ndarray:
    """Gradient of L with respect to the local potential on the grid."""
    if res.x_full is None:
        raise ValueError("solve with keep_x=True first")
    a_node = np.asarray(a_node, dtype=np.float64)
    b_node = np.zeros_like(a_node) if b_node is None else np.asarray(b_node, dtype=np.float64)
    g = np.zeros(w.n_grid)
    for j, reg in enumerate(res.regions):
        coefs = (2.0 * a_node[j] / w.dV + 2.0 * b_node[j] * res.z) * res.wts   # (P,)
        contrib = -np.imag((coefs[:, None] * res.x_full[j] ** 2).sum(axis=0))
        np.add.at(g, reg.gidx, contrib)
    return g


def forces(w, dLdV: np.ndarray, atoms=None) -> np.ndarray:
    """F_a = -sum_k dL/dV_k dV_k/dR_a (local Gaussian wells only), for every
    atom or for the listed ones (rows in that order)."""
    sel = np.arange(len(w.atoms)) if atoms is None else np.asarray(atoms, dtype=np.int64)
    F = np.zeros((len(sel), 3))
    for i, a in enumerate(sel):
        gidx, dVdR = ham_mod.local_potential_gradient_terms(w, int(a))
        F[i] = -(dLdV[gidx][:, None] * dVdR).sum(axis=0)
    return F
