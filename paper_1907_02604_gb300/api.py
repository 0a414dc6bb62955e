"""Python front end of the nodal-density library.

Thin marshalling over the C ABI (``_lib``): arguments become C structs and
raw pointers; PyTorch supplies device memory and the current CUDA stream.
Every computation runs in the library's CUDA kernels.

    ham = Hamiltonian.from_workload(w)                 # md_build_hamiltonian
    z, w = make_poles(kT, mu, *ham.spectral_bounds(), P)   # md_make_poles
    rho, e, stats = density(ham, z, w, nodes, halfwidth)    # md_density
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import check, load


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_lib.c_double_p)


def _stream_handle(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _cuda_f64(t: torch.Tensor, n: int, name: str) -> torch.Tensor:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"{name} must have {n} elements")
    return t.contiguous()


def fd_weights(order: int) -> np.ndarray:
    """Central second-derivative weights w_0..w_q (host code, no GPU)."""
    out = np.zeros(order // 2 + 1)
    check(load().md_fd_weights(order, _dptr(out)), "md_fd_weights")
    return out


def fma_rate(precision: str = "fp64", stream=None) -> float:
    """Measured FMA throughput of the device in TFLOP/s (md_fma_rate)."""
    prec = {"fp64": _lib.MD_PREC_FP64, "fp32": _lib.MD_PREC_MIXED}[precision]
    out = ctypes.c_double()
    check(load().md_fma_rate(prec, _stream_handle(stream), ctypes.byref(out)), "md_fma_rate")
    return out.value


def make_poles(kT: float, mu: float, emin: float, emax: float, P: int):
    """Poles and weights (complex128 arrays) of the rational Fermi
    approximation (host code, no GPU)."""
    z = np.zeros(2 * P)
    w = np.zeros(2 * P)
    check(load().md_make_poles(kT, mu, emin, emax, P, _dptr(z), _dptr(w)), "md_make_poles")
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


@dataclass
class SolverOptions:
    tol: float = 1e-10
    maxit: int = 20000
    precision: str = "fp64"        # "fp64" or "mixed"
    reliable_every: int = 0
    reliable_delta: float = 0.0
    timeout_s: float = 0.0
    block: int = 0
    ctas_per_sm: int = 0
    # "auto" (autotuned), "generic" or "zmarch" (both need block > 0), or
    # "cluster": Krylov vectors in shared memory, one thread-block cluster per
    # system (mixed precision); there ctas_per_sm is the CTAs per cluster
    # (0 = the fewest whose slabs fit) and block the threads per CTA (0 = auto)
    kernel: str = "auto"
    method: str = "cocg"           # "cocg" (one solve per pole) or "shifted" (one per node)

    def to_c(self) -> _lib.md_solver_opts:
        prec = {"fp64": _lib.MD_PREC_FP64, "mixed": _lib.MD_PREC_MIXED}[self.precision]
        kern = {"auto": 0, "generic": 1, "zmarch": 2, "cluster": 3}[self.kernel]
        meth = {"cocg": 0, "shifted": 1}[self.method]
        return _lib.md_solver_opts(self.tol, self.maxit, prec, self.reliable_every,
                                   self.reliable_delta, self.timeout_s, self.block, self.ctas_per_sm,
                                   kern, meth)


class Hamiltonian:
    """Device-resident discrete Hamiltonian (md_build_hamiltonian)."""

    def __init__(self, shape, spacing, periodic, fd_order, atoms, depth, sigma,
                 cutoff_sigmas=8.0, v_ext=None, nonlocal_proj=False, proj_sigma=1.0,
                 proj_rc=4.0, e_s=0.5, e_p=0.25, stream=None):
        lib = load()
        self.shape = tuple(int(n) for n in shape)
        self.spacing = tuple(float(h) for h in spacing)
        self.periodic = tuple(bool(p) for p in periodic)
        self.N = int(np.prod(self.shape))
        self.dV = float(np.prod(self.spacing))
        self._atoms = np.ascontiguousarray(np.asarray(atoms, dtype=np.float64).reshape(-1, 3))
        self._depth = np.ascontiguousarray(depth, dtype=np.float64)
        self._sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        self.n_atoms = len(self._atoms)
        g = _lib.md_grid((ctypes.c_int32 * 3)(*self.shape), (ctypes.c_double * 3)(*self.spacing),
                         (ctypes.c_int32 * 3)(*[int(bool(p)) for p in periodic]), int(fd_order))
        a = _lib.md_atoms(self.n_atoms, _dptr(self._atoms), _dptr(self._depth), _dptr(self._sigma))
        vext = None if v_ext is None else np.ascontiguousarray(v_ext, dtype=np.float64)
        if vext is not None and vext.size != self.N:
            raise ValueError("v_ext must have one value per grid point")
        pot = _lib.md_pot_params(float(cutoff_sigmas), None if vext is None else _dptr(vext),
                                 int(bool(nonlocal_proj)), float(proj_sigma), float(proj_rc),
                                 float(e_s), float(e_p))
        h = ctypes.c_void_p()
        check(lib.md_build_hamiltonian(ctypes.byref(g), ctypes.byref(a), ctypes.byref(pot),
                                       _stream_handle(stream), ctypes.byref(h)), "md_build_hamiltonian")
        self._h = h
        self.nonlocal_proj = bool(nonlocal_proj)

    @classmethod
    def from_workload(cls, w, atoms=None, stream=None) -> "Hamiltonian":
        return cls(w.shape, w.spacing, w.periodic, w.fd_order,
                   w.atoms if atoms is None else atoms, w.depth, w.sigma,
                   cutoff_sigmas=w.cutoff_sigmas, v_ext=w.v_ext, nonlocal_proj=w.nonlocal_proj,
                   proj_sigma=w.proj_sigma, proj_rc=w.proj_rc, e_s=w.e_s, e_p=w.e_p, stream=stream)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("Hamiltonian was closed")
        return self._h

    def potential(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.N, dtype=torch.float64, device="cuda")
        check(load().md_hamiltonian_potential(self.handle, ctypes.c_void_p(out.data_ptr()),
                                              _stream_handle(stream)), "md_hamiltonian_potential")
        return out

    def set_potential(self, V: torch.Tensor, stream=None):
        V = _cuda_f64(V, self.N, "V")
        check(load().md_hamiltonian_set_potential(self.handle, ctypes.c_void_p(V.data_ptr()),
                                                  _stream_handle(stream)), "md_hamiltonian_set_potential")

    def spectral_bounds(self, stream=None):
        lo, hi = ctypes.c_double(), ctypes.c_double()
        check(load().md_spectral_bounds(self.handle, _stream_handle(stream), ctypes.byref(lo),
                                        ctypes.byref(hi)), "md_spectral_bounds")
        return lo.value, hi.value

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().md_hamiltonian_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _PoleArgs:
    def __init__(self, z, w):
        z = np.asarray(z, dtype=np.complex128)
        w = np.asarray(w, dtype=np.complex128)
        self.zf = np.ascontiguousarray(np.stack([z.real, z.imag], axis=1).reshape(-1))
        self.wf = np.ascontiguousarray(np.stack([w.real, w.imag], axis=1).reshape(-1))
        self.c = _lib.md_poles(len(z), _dptr(self.zf), _dptr(self.wf))
        self.P = len(z)


class _NodeArgs:
    def __init__(self, nodes, halfwidth):
        self.node = np.ascontiguousarray(nodes, dtype=np.int64)
        self.hw = np.ascontiguousarray(halfwidth, dtype=np.int32)
        if self.node.shape != self.hw.shape:
            raise ValueError("nodes and halfwidth must have the same length")
        self.c = _lib.md_nodes(len(self.node), self.node.ctypes.data_as(_lib.c_int64_p),
                               self.hw.ctypes.data_as(_lib.c_int32_p))
        self.n = len(self.node)


class Workspace:
    """Checkpoint of every forward solution x_jp (md_workspace_create)."""

    def __init__(self, ham: Hamiltonian, nodes, halfwidth, n_poles: int):
        self._nodes = _NodeArgs(nodes, halfwidth)
        h = ctypes.c_void_p()
        check(load().md_workspace_create(ham.handle, ctypes.byref(self._nodes.c), int(n_poles),
                                         ctypes.byref(h)), "md_workspace_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().md_workspace_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_SOFT = (_lib.MD_ERR_NOCONV, _lib.MD_ERR_BREAKDOWN)


class Plan:
    """A prepared batched solve replayed as one CUDA graph (md_plan_*).

    The output tensors rho (and e) are owned by the plan object and
    rewritten by every launch."""

    def __init__(self, ham: Hamiltonian, z, w, nodes, halfwidth, opts: SolverOptions = None,
                 energy=True, checkpoint: Workspace = None, stream=None):
        opts = opts or SolverOptions()
        self._poles, self._nodes = _PoleArgs(z, w), _NodeArgs(nodes, halfwidth)
        self.rho = torch.empty(self._nodes.n, dtype=torch.float64, device="cuda")
        self.e = torch.empty(self._nodes.n, dtype=torch.float64, device="cuda") if energy else None
        self._opts = opts.to_c()
        self._ham = ham          # keep the Hamiltonian alive as long as the graph
        self._ckpt = checkpoint
        h = ctypes.c_void_p()
        check(load().md_plan_create(ham.handle, ctypes.byref(self._poles.c), ctypes.byref(self._nodes.c),
                                    ctypes.byref(self._opts), ctypes.c_void_p(self.rho.data_ptr()),
                                    ctypes.c_void_p(self.e.data_ptr()) if self.e is not None else None,
                                    checkpoint.handle if checkpoint is not None else None,
                                    _stream_handle(stream), ctypes.byref(h)), "md_plan_create")
        self._h = h
        self.n_systems = self._nodes.n * self._poles.P

    def launch(self, stream=None):
        check(load().md_plan_launch(self._h, _stream_handle(stream)), "md_plan_launch")

    def stats(self, stream=None, strict=True):
        st = _lib.md_stats()
        status = load().md_plan_stats(self._h, _stream_handle(stream), ctypes.byref(st))
        check(status, "md_plan_stats", allow=() if strict else _SOFT)
        d = st.as_dict()
        d["status"] = _lib.STATUS_NAMES[status]
        return d

    def system_info(self, stream=None):
        """Per-system (status, iterations, residual) of the last launch,
        indexed node * P + pole."""
        n = self.n_systems
        st = np.zeros(n, np.int32)
        it = np.zeros(n, np.int32)
        rs = np.zeros(n, np.float64)
        check(load().md_plan_system_info(self._h, _stream_handle(stream),
                                         st.ctypes.data_as(_lib.c_int32_p),
                                         it.ctypes.data_as(_lib.c_int32_p),
                                         rs.ctypes.data_as(_lib.c_double_p)), "md_plan_system_info")
        return st, it, rs

    def launch_shape(self):
        b, g = ctypes.c_int32(), ctypes.c_int32()
        check(load().md_plan_launch_shape(self._h, ctypes.byref(b), ctypes.byref(g)), "md_plan_launch_shape")
        return b.value, g.value

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().md_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def density(ham: Hamiltonian, z, w, nodes, halfwidth, opts: SolverOptions = None, energy=False,
            checkpoint: Workspace = None, out=None, stream=None, strict=True, sync=True):
    """rho_j (and e_j) for every node.  Returns (rho, e or None, stats dict).

    With strict=False a non-converged or broken-down system does not raise;
    its status is in the stats.  With sync=False the call only enqueues the
    work on `stream` (md_density without stats) and returns (rho, e, None):
    the tensors are valid once the stream has been synchronised, and no
    per-system status is reported."""
    opts = opts or SolverOptions()
    pa, na = _PoleArgs(z, w), _NodeArgs(nodes, halfwidth)
    rho = out if out is not None else torch.empty(na.n, dtype=torch.float64, device="cuda")
    e = torch.empty(na.n, dtype=torch.float64, device="cuda") if energy else None
    st = _lib.md_stats()
    copts = opts.to_c()
    status = load().md_density(ham.handle, ctypes.byref(pa.c), ctypes.byref(na.c), ctypes.byref(copts),
                               ctypes.c_void_p(rho.data_ptr()),
                               ctypes.c_void_p(e.data_ptr()) if e is not None else None,
                               checkpoint.handle if checkpoint is not None else None,
                               ctypes.byref(st) if sync else None, _stream_handle(stream))
    check(status, "md_density", allow=() if strict else _SOFT)
    if not sync:
        return rho, e, None
    d = st.as_dict()
    d["status"] = _lib.STATUS_NAMES[status]
    return rho, e, d


def energy(ham: Hamiltonian, z, w, nodes, halfwidth, opts: SolverOptions = None, node_weight=None,
           stream=None):
    """Band energy per node (device tensor) and its node-weighted sum (float;
    node_weight: float64 CUDA tensor of n_nodes, or None for weight 1)."""
    opts = opts or SolverOptions()
    pa, na = _PoleArgs(z, w), _NodeArgs(nodes, halfwidth)
    nu = None if node_weight is None else _cuda_f64(node_weight, na.n, "node_weight")
    e = torch.empty(na.n, dtype=torch.float64, device="cuda")
    eb = ctypes.c_double()
    st = _lib.md_stats()
    copts = opts.to_c()
    check(load().md_energy(ham.handle, ctypes.byref(pa.c), ctypes.byref(na.c),
                           None if nu is None else ctypes.c_void_p(nu.data_ptr()), ctypes.byref(copts),
                           ctypes.c_void_p(e.data_ptr()), ctypes.byref(eb), ctypes.byref(st),
                           _stream_handle(stream)), "md_energy")
    return e, eb.value, st.as_dict()


def make_entropy_weights(kT: float, mu: float, emin: float, emax: float, P: int):
    """Weights (complex128) of the entropy function on the poles make_poles
    returns for the same arguments (host code, no GPU)."""
    w = np.zeros(2 * P)
    check(load().md_make_entropy_weights(kT, mu, emin, emax, P, _dptr(w)), "md_make_entropy_weights")
    return w[0::2] + 1j * w[1::2]


def free_energy(ham: Hamiltonian, z, w, w_entropy, kT: float, nodes, halfwidth, opts: SolverOptions = None,
                node_weight=None, stream=None, strict=True):
    """rho_j, e_j and s_j (device tensors) and the node-weighted totals
    {n_electrons, e_band, ts, free_energy} (md_free_energy).  w_entropy from
    make_entropy_weights, or None (no entropy term: s is None, ts = 0)."""
    opts = opts or SolverOptions()
    pa, na = _PoleArgs(z, w), _NodeArgs(nodes, halfwidth)
    nu = None if node_weight is None else _cuda_f64(node_weight, na.n, "node_weight")
    ws = None
    if w_entropy is not None:
        w_entropy = np.asarray(w_entropy, dtype=np.complex128)
        if w_entropy.shape != (pa.P,):
            raise ValueError("w_entropy must have one weight per pole")
        ws = np.empty(2 * pa.P)
        ws[0::2], ws[1::2] = w_entropy.real, w_entropy.imag
    rho = torch.empty(na.n, dtype=torch.float64, device="cuda")
    e = torch.empty(na.n, dtype=torch.float64, device="cuda")
    s = torch.empty(na.n, dtype=torch.float64, device="cuda") if ws is not None else None
    terms = _lib.md_free_energy_terms()
    st = _lib.md_stats()
    copts = opts.to_c()
    vp = lambda t: None if t is None or t.numel() == 0 else ctypes.c_void_p(t.data_ptr())
    status = load().md_free_energy(ham.handle, ctypes.byref(pa.c), None if ws is None else _dptr(ws), float(kT),
                                   ctypes.byref(na.c), vp(nu), ctypes.byref(copts), vp(rho), vp(e), vp(s),
                                   ctypes.byref(terms), ctypes.byref(st), _stream_handle(stream))
    check(status, "md_free_energy", allow=() if strict else _SOFT)
    d = st.as_dict()
    d["status"] = _lib.STATUS_NAMES[status]
    return rho, e, s, terms.as_dict(), d


def cluster_sampling(shape, spacing, periodic, esp, n_q, radius: float):
    """Nodes (int64) and weights (float64) of the cluster-sampled energy of
    Section 3 (md_cluster_sampling; host code, no GPU)."""
    g = _lib.md_grid((ctypes.c_int32 * 3)(*[int(n) for n in shape]),
                     (ctypes.c_double * 3)(*[float(h) for h in spacing]),
                     (ctypes.c_int32 * 3)(*[1 if p else 0 for p in periodic]), 2)
    esp = np.ascontiguousarray(esp, dtype=np.int64)
    n_q = np.ascontiguousarray(n_q, dtype=np.float64)
    n = ctypes.c_int64(0)
    lib = load()
    check(lib.md_cluster_sampling(ctypes.byref(g), len(esp), esp.ctypes.data_as(_lib.c_int64_p), _dptr(n_q),
                                  float(radius), ctypes.byref(n), None, None), "md_cluster_sampling")
    nodes = np.zeros(n.value, np.int64)
    nu = np.zeros(n.value, np.float64)
    check(lib.md_cluster_sampling(ctypes.byref(g), len(esp), esp.ctypes.data_as(_lib.c_int64_p), _dptr(n_q),
                                  float(radius), ctypes.byref(n), nodes.ctypes.data_as(_lib.c_int64_p),
                                  _dptr(nu)), "md_cluster_sampling")
    return nodes, nu


def fermi_level_poles(ham: Hamiltonian, kT: float, P: int, nodes, halfwidth, n_electrons: float,
                      opts: SolverOptions = None, node_weight=None, mu_tol: float = 0.0, stream=None):
    """(mu, N(mu), counts made) with N(mu) = dV sum nu_j rho_j(mu) = n_electrons
    for the pole form (md_fermi_level_poles)."""
    opts = opts or SolverOptions()
    na = _NodeArgs(nodes, halfwidth)
    nu = None if node_weight is None else _cuda_f64(node_weight, na.n, "node_weight")
    mu, cnt, ev = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    copts = opts.to_c()
    check(load().md_fermi_level_poles(ham.handle, float(kT), int(P), ctypes.byref(na.c),
                                      None if nu is None else ctypes.c_void_p(nu.data_ptr()), ctypes.byref(copts),
                                      float(n_electrons), float(mu_tol), ctypes.byref(mu), ctypes.byref(cnt),
                                      ctypes.byref(ev), _stream_handle(stream)), "md_fermi_level_poles")
    return mu.value, cnt.value, ev.value


def density_fused_adjoint(ham: Hamiltonian, z, w, nodes, halfwidth, dL_drho: torch.Tensor = None,
                          dL_de: torch.Tensor = None, opts: SolverOptions = None, forces=False,
                          stream=None):
    """rho, e, dL/dV (and forces) in one pass without a checkpoint, for node
    sensitivities known before the solve (e.g. the band energy: dL_de = 1)."""
    opts = opts or SolverOptions()
    pa, na = _PoleArgs(z, w), _NodeArgs(nodes, halfwidth)
    a = None if dL_drho is None else _cuda_f64(dL_drho, na.n, "dL_drho")
    b = None if dL_de is None else _cuda_f64(dL_de, na.n, "dL_de")
    rho = torch.empty(na.n, dtype=torch.float64, device="cuda")
    e = torch.empty(na.n, dtype=torch.float64, device="cuda")
    g = torch.empty(ham.N, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * ham.n_atoms, dtype=torch.float64, device="cuda") if forces else None
    st = _lib.md_stats()
    copts = opts.to_c()
    vp = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    check(load().md_density_fused_adjoint(ham.handle, ctypes.byref(pa.c), ctypes.byref(na.c),
                                          ctypes.byref(copts), vp(a), vp(b), vp(rho), vp(e), vp(g), vp(F),
                                          ctypes.byref(st), _stream_handle(stream)),
          "md_density_fused_adjoint")
    return rho, e, g, (F.view(-1, 3) if F is not None else None), st.as_dict()


def density_matrix_rows(ham: Hamiltonian, z, w, nodes, halfwidth, opts: SolverOptions = None,
                        stream=None):
    """rho, e and the density-matrix rows gamma_jk (k over R(j)) of every
    node: returns (rho, e, rows, offsets) with row j = rows[offsets[j]:offsets[j+1]]
    in region-local order (x fastest)."""
    opts = opts or SolverOptions()
    pa, na = _PoleArgs(z, w), _NodeArgs(nodes, halfwidth)
    sizes = np.array([_region_size(ham, int(n), int(s)) for n, s in zip(na.node, na.hw)], dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rho = torch.empty(na.n, dtype=torch.float64, device="cuda")
    e = torch.empty(na.n, dtype=torch.float64, device="cuda")
    rows = torch.empty(int(offsets[-1]), dtype=torch.float64, device="cuda")
    st = _lib.md_stats()
    copts = opts.to_c()
    vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t.numel() else None
    check(load().md_density_matrix_rows(ham.handle, ctypes.byref(pa.c), ctypes.byref(na.c), ctypes.byref(copts),
                                        vp(rho), vp(e), vp(rows), ctypes.byref(st), _stream_handle(stream)),
          "md_density_matrix_rows")
    return rho, e, rows, offsets


def _region_size(ham: Hamiltonian, node: int, s: int) -> int:
    """Points of the region of a node (cube of side 2s+1; whole axis on a
    periodic axis it would cover), as the library lays it out."""
    n = 1
    for d in range(3):
        m = 2 * s + 1
        n *= ham.shape[d] if (ham.periodic[d] and m >= ham.shape[d]) else m
    return n


def density_adjoint(ham: Hamiltonian, z, w, nodes, halfwidth, dL_drho: torch.Tensor,
                    dL_de: torch.Tensor = None, opts: SolverOptions = None,
                    checkpoint: Workspace = None, forces=False, stream=None):
    """dL/dV on the grid and, optionally, the forces -dL/dR on the atoms."""
    opts = opts or SolverOptions()
    pa, na = _PoleArgs(z, w), _NodeArgs(nodes, halfwidth)
    a = _cuda_f64(dL_drho, na.n, "dL_drho")
    b = None if dL_de is None else _cuda_f64(dL_de, na.n, "dL_de")
    g = torch.empty(ham.N, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * ham.n_atoms, dtype=torch.float64, device="cuda") if forces else None
    st = _lib.md_stats()
    copts = opts.to_c()
    check(load().md_density_adjoint(ham.handle, ctypes.byref(pa.c), ctypes.byref(na.c),
                                    ctypes.byref(copts), ctypes.c_void_p(a.data_ptr()),
                                    None if b is None else ctypes.c_void_p(b.data_ptr()),
                                    checkpoint.handle if checkpoint is not None else None,
                                    ctypes.c_void_p(g.data_ptr()),
                                    None if F is None else ctypes.c_void_p(F.data_ptr()),
                                    ctypes.byref(st), _stream_handle(stream)), "md_density_adjoint")
    return g, (F.view(-1, 3) if F is not None else None)


class GaussRules:
    """Per-node Lanczos Gauss rules (md_lssgq_rules): lam, weight (device,
    n_nodes x K, float64), k_used (device, int32), dV of the grid."""

    def __init__(self, lam: torch.Tensor, weight: torch.Tensor, k_used: torch.Tensor, dV: float):
        self.lam, self.weight, self.k_used, self.dV = lam, weight, k_used, dV

    @property
    def n_nodes(self) -> int:
        return self.lam.shape[0]

    @property
    def K(self) -> int:
        return self.lam.shape[1]

    def fields(self, mu: float, kT: float, stream=None):
        """rho_j, e_j (band term) and s_j (entropy term) at (mu, kT)."""
        n = self.n_nodes
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
        e = torch.empty(n, dtype=torch.float64, device="cuda")
        s = torch.empty(n, dtype=torch.float64, device="cuda")
        vp = lambda t: ctypes.c_void_p(t.data_ptr())
        check(load().md_lssgq_fields(n, self.K, vp(self.lam), vp(self.weight), float(mu), float(kT),
                                     float(self.dV), vp(rho), vp(e), vp(s), _stream_handle(stream)),
              "md_lssgq_fields")
        return rho, e, s

    def fermi_level(self, kT: float, n_electrons: float, node_weight: torch.Tensor = None, stream=None):
        """(mu, N_e(mu)) with N_e(mu) = n_electrons (Eq. Fermi:Rho)."""
        nu = None if node_weight is None else _cuda_f64(node_weight, self.n_nodes, "node_weight")
        mu = ctypes.c_double(0.0)
        cnt = ctypes.c_double(0.0)
        check(load().md_fermi_level(self.n_nodes, self.K, ctypes.c_void_p(self.lam.data_ptr()),
                                    ctypes.c_void_p(self.weight.data_ptr()),
                                    None if nu is None else ctypes.c_void_p(nu.data_ptr()),
                                    float(kT), float(n_electrons), ctypes.byref(mu), ctypes.byref(cnt),
                                    _stream_handle(stream)), "md_fermi_level")
        return mu.value, cnt.value


def lssgq_rules(ham: Hamiltonian, nodes, halfwidth, K: int = 40, breakdown_tol: float = 0.0,
                timeout_s: float = 0.0, block: int = 0, precision: str = "fp64", stream=None) -> GaussRules:
    """K-point Lanczos Gauss rules of every node (Section 2.1, Eq. 9);
    precision "fp64" or "mixed" (FP32 vectors, FP64 scalars)."""
    na = _NodeArgs(nodes, halfwidth)
    lam = torch.empty((na.n, K), dtype=torch.float64, device="cuda")
    wt = torch.empty((na.n, K), dtype=torch.float64, device="cuda")
    ku = torch.empty(na.n, dtype=torch.int32, device="cuda")
    prec = {"fp64": _lib.MD_PREC_FP64, "mixed": _lib.MD_PREC_MIXED}[precision]
    o = _lib.md_lssgq_opts(int(K), float(breakdown_tol), float(timeout_s), int(block), prec)
    check(load().md_lssgq_rules(ham.handle, ctypes.byref(na.c), ctypes.byref(o), ctypes.c_void_p(lam.data_ptr()),
                                ctypes.c_void_p(wt.data_ptr()), ctypes.c_void_p(ku.data_ptr()),
                                _stream_handle(stream)), "md_lssgq_rules")
    return GaussRules(lam, wt, ku, ham.dV)
