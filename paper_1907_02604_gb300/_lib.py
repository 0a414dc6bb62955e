"""ctypes view of the C ABI in include/macrodft.h (argument marshalling only).

The shared library is the in-tree ``libmacrodft.so`` built by ``build.py``.
There is no fallback: if the library is missing or fails to load, every
entry point raises.
"""
import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmacrodft.so")

MD_OK, MD_ERR_INVALID, MD_ERR_NOCONV, MD_ERR_BREAKDOWN, MD_ERR_TIMEOUT, MD_ERR_OOM, MD_ERR_CUDA = range(7)
STATUS_NAMES = {0: "MD_OK", 1: "MD_ERR_INVALID", 2: "MD_ERR_NOCONV", 3: "MD_ERR_BREAKDOWN",
                4: "MD_ERR_TIMEOUT", 5: "MD_ERR_OOM", 6: "MD_ERR_CUDA"}
MD_PREC_FP64, MD_PREC_MIXED = 0, 1

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int64_p = ctypes.POINTER(ctypes.c_int64)
c_int32_p = ctypes.POINTER(ctypes.c_int32)


class md_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("h", ctypes.c_double * 3),
                ("periodic", ctypes.c_int32 * 3), ("fd_order", ctypes.c_int32)]


class md_atoms(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("xyz", c_double_p), ("depth", c_double_p),
                ("sigma", c_double_p)]


class md_pot_params(ctypes.Structure):
    _fields_ = [("cutoff_sigmas", ctypes.c_double), ("v_ext", c_double_p),
                ("nonlocal", ctypes.c_int32), ("proj_sigma", ctypes.c_double),
                ("proj_rc", ctypes.c_double), ("e_s", ctypes.c_double), ("e_p", ctypes.c_double)]


class md_poles(ctypes.Structure):
    _fields_ = [("n_poles", ctypes.c_int32), ("z", c_double_p), ("w", c_double_p)]


class md_nodes(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("node", c_int64_p), ("halfwidth", c_int32_p)]


class md_solver_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reliable_every", ctypes.c_int32), ("reliable_delta", ctypes.c_double),
                ("timeout_s", ctypes.c_double), ("block", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("method", ctypes.c_int32)]


class md_lssgq_opts(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("breakdown_tol", ctypes.c_double), ("timeout_s", ctypes.c_double),
                ("block", ctypes.c_int32), ("precision", ctypes.c_int32)]


class md_stats(ctypes.Structure):
    _fields_ = [("n_systems", ctypes.c_int64), ("n_converged", ctypes.c_int64),
                ("n_noconv", ctypes.c_int64), ("n_breakdown", ctypes.c_int64),
                ("n_timeout", ctypes.c_int64), ("iters_min", ctypes.c_int32),
                ("iters_max", ctypes.c_int32), ("iters_mean", ctypes.c_double),
                ("total_iters", ctypes.c_int64), ("total_point_iters", ctypes.c_int64),
                ("reliable_updates", ctypes.c_int64), ("max_resid", ctypes.c_double),
                ("kernel_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class md_free_energy_terms(ctypes.Structure):
    _fields_ = [("n_electrons", ctypes.c_double), ("e_band", ctypes.c_double), ("ts", ctypes.c_double),
                ("free_energy", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every symbol include/macrodft.h declares: (name, restype, argtypes)
_VP = ctypes.c_void_p
SIGNATURES = [
    ("md_build_hamiltonian", ctypes.c_int, [ctypes.POINTER(md_grid), ctypes.POINTER(md_atoms),
                                            ctypes.POINTER(md_pot_params), _VP, ctypes.POINTER(_VP)]),
    ("md_hamiltonian_destroy", ctypes.c_int, [_VP]),
    ("md_hamiltonian_potential", ctypes.c_int, [_VP, _VP, _VP]),
    ("md_hamiltonian_set_potential", ctypes.c_int, [_VP, _VP, _VP]),
    ("md_spectral_bounds", ctypes.c_int, [_VP, _VP, c_double_p, c_double_p]),
    ("md_make_poles", ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int32, c_double_p, c_double_p]),
    ("md_workspace_create", ctypes.c_int, [_VP, ctypes.POINTER(md_nodes), ctypes.c_int32,
                                           ctypes.POINTER(_VP)]),
    ("md_workspace_destroy", ctypes.c_int, [_VP]),
    ("md_density", ctypes.c_int, [_VP, ctypes.POINTER(md_poles), ctypes.POINTER(md_nodes),
                                  ctypes.POINTER(md_solver_opts), _VP, _VP, _VP,
                                  ctypes.POINTER(md_stats), _VP]),
    ("md_energy", ctypes.c_int, [_VP, ctypes.POINTER(md_poles), ctypes.POINTER(md_nodes), _VP,
                                 ctypes.POINTER(md_solver_opts), _VP, c_double_p,
                                 ctypes.POINTER(md_stats), _VP]),
    ("md_make_entropy_weights", ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int32, c_double_p]),
    ("md_free_energy", ctypes.c_int, [_VP, ctypes.POINTER(md_poles), c_double_p, ctypes.c_double,
                                      ctypes.POINTER(md_nodes), _VP, ctypes.POINTER(md_solver_opts),
                                      _VP, _VP, _VP, ctypes.POINTER(md_free_energy_terms),
                                      ctypes.POINTER(md_stats), _VP]),
    ("md_cluster_sampling", ctypes.c_int, [ctypes.POINTER(md_grid), ctypes.c_int64, c_int64_p, c_double_p,
                                           ctypes.c_double, c_int64_p, c_int64_p, c_double_p]),
    ("md_fermi_level_poles", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(md_nodes), _VP,
                                            ctypes.POINTER(md_solver_opts), ctypes.c_double, ctypes.c_double,
                                            c_double_p, c_double_p, c_int32_p, _VP]),
    ("md_density_adjoint", ctypes.c_int, [_VP, ctypes.POINTER(md_poles), ctypes.POINTER(md_nodes),
                                          ctypes.POINTER(md_solver_opts), _VP, _VP, _VP, _VP, _VP,
                                          ctypes.POINTER(md_stats), _VP]),
    ("md_density_fused_adjoint", ctypes.c_int, [_VP, ctypes.POINTER(md_poles), ctypes.POINTER(md_nodes),
                                                ctypes.POINTER(md_solver_opts), _VP, _VP, _VP, _VP, _VP,
                                                _VP, ctypes.POINTER(md_stats), _VP]),
    ("md_density_matrix_rows", ctypes.c_int, [_VP, ctypes.POINTER(md_poles), ctypes.POINTER(md_nodes),
                                              ctypes.POINTER(md_solver_opts), _VP, _VP, _VP,
                                              ctypes.POINTER(md_stats), _VP]),
    ("md_plan_create", ctypes.c_int, [_VP, ctypes.POINTER(md_poles), ctypes.POINTER(md_nodes),
                                      ctypes.POINTER(md_solver_opts), _VP, _VP, _VP, _VP,
                                      ctypes.POINTER(_VP)]),
    ("md_plan_launch", ctypes.c_int, [_VP, _VP]),
    ("md_plan_stats", ctypes.c_int, [_VP, _VP, ctypes.POINTER(md_stats)]),
    ("md_plan_launch_shape", ctypes.c_int, [_VP, c_int32_p, c_int32_p]),
    ("md_plan_system_info", ctypes.c_int, [_VP, _VP, c_int32_p, c_int32_p, c_double_p]),
    ("md_plan_destroy", ctypes.c_int, [_VP]),
    ("md_density_noalloc", ctypes.c_int, [_VP, ctypes.POINTER(md_poles), ctypes.POINTER(md_nodes),
                                          ctypes.POINTER(md_solver_opts), _VP, _VP,
                                          ctypes.POINTER(md_stats), _VP]),
    ("md_fd_weights", ctypes.c_int, [ctypes.c_int32, c_double_p]),
    ("md_lssgq_rules", ctypes.c_int, [_VP, ctypes.POINTER(md_nodes), ctypes.POINTER(md_lssgq_opts),
                                      _VP, _VP, _VP, _VP]),
    ("md_lssgq_fields", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, _VP, _VP, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP]),
    ("md_fermi_level", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_double,
                                      ctypes.c_double, c_double_p, c_double_p, _VP]),
    ("md_fma_rate", ctypes.c_int, [ctypes.c_int32, _VP, c_double_p]),
    ("md_last_error", ctypes.c_char_p, []),
    ("md_version", ctypes.c_char_p, []),
]

_lock = threading.Lock()
_lib = None


class MacroDFTError(RuntimeError):
    def __init__(self, status, where, message):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


def load(path: str = LIB_PATH):
    """Load (once) and return the CUDA library; raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with "
                                   "paper_1907_02604_gb300.build.build() (no CPU fallback exists)")
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int, where: str, allow=()):
    if status == MD_OK or status in allow:
        return status
    msg = load().md_last_error().decode(errors="replace")
    raise MacroDFTError(status, where, msg)
