"""GB300 nodal-density library (arXiv:1907.02604, MacroDFT hot path).

Electron density at sampled grid nodes, rho_j = (2/dV) sum_p Im(w_p
x_jp(j)) with (H_R(j) - z_p) x_jp = e_j solved by COCG in hand-written CUDA
kernels for sm_103a, behind the C ABI of include/macrodft.h.  This package
is the Python binding (``api``), the autograd wrapper (``torch_api``) and
the in-tree build (``build``).
"""
from .api import (GaussRules, Hamiltonian, Plan, SolverOptions, Workspace, cluster_sampling, density,
                  density_adjoint, density_fused_adjoint, density_matrix_rows, energy, fd_weights,
                  fermi_level_poles, fma_rate, free_energy, lssgq_rules, make_entropy_weights, make_poles)

__all__ = ["GaussRules", "Hamiltonian", "Plan", "SolverOptions", "Workspace", "cluster_sampling", "density",
           "density_adjoint", "density_fused_adjoint", "density_matrix_rows", "energy", "fd_weights",
           "fermi_level_poles", "fma_rate", "free_energy", "lssgq_rules", "make_entropy_weights", "make_poles"]
