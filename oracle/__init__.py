"""Oracle: a plain, slow, FP64 CPU statement of the nodal-density path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
runs this package; only the tests, the smoke check and the CPU-baseline leg
of the benchmark do.  It shares no code with the CUDA library: it builds the
Hamiltonian, the pole expansion and the solver from their definitions on its
own, and takes only the seeded synthetic inputs from ``synthetic``.

What it computes (the paper's Eq. (dm) density matrix g(H), read on the
diagonal as in Eq. (Electron_density:GQ), rho_p = 2 h^-3 <e_p|g(H)|e_p>, with
g replaced by a P-pole rational approximation r and H by its restriction to
a cube around each node, the locality of Section 2.1):

    rho_j = (2/dV) sum_p Im( w_p x_jp(j) ),   (H_R(j) - z_p) x_jp = e_j

solved by COCG.  Modules:

* ``poles``       rational approximation of the Fermi-Dirac function
* ``hamiltonian`` grid, FD Laplacian weights, local potential, projectors,
                  spectral bounds, restriction to a region
* ``cocg.c``      plain C FP64 COCG on one region (OpenMP over systems)
* ``density``     nodal density, band energy, adjoint and forces
* ``lssgq``       the paper's Lanczos spectral Gauss quadrature (Eq. 9):
                  per-node Gauss rules, rho / band energy / entropy per node,
                  electron count and Fermi level (Eq. Fermi:Rho)
"""
