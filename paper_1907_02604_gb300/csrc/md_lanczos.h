// Lanczos spectral Gauss quadrature (the paper's LSSGQ, Section 2.1, Eq. 9):
// per-node Gauss rules of the spectral measure of H_R(j) at e_j, the fields
// computed from them, and the Fermi level from the electron count.
#pragma once

#include <cuda_runtime.h>

#include "md_solver.h"

namespace md {

constexpr int kMaxLanczosK = 128;

struct LanczosParams {
    int K;                 // Lanczos steps = rule size
    double breakdown_tol;  // stop when beta_k <= tol * (|alpha_1| + beta_1 + 1)
    double* alpha;         // [n_nodes][K]
    double* beta;          // [n_nodes][K], entries 0..k_used-2
    int* k_used;           // [n_nodes]
    int* status;           // [n_nodes]: 0 ok, 1 too many projector atoms, 3 QR did not converge, 4 timeout
};

// Lanczos on every node of P.sys (pole fields unused); P.scratch holds one
// slot per CTA.
// precision: MD_PREC_FP64 (FP64 vectors) or MD_PREC_MIXED (FP32 vectors and
// stencil, FP64 scalars); slot = 2 n_max values of that width.
cudaError_t launch_lanczos(const SolveParams& P, const LanczosParams& L, int precision, int grid, int block,
                           cudaStream_t stream);
// Nodes and weights of each node's Gauss rule (ascending nodes; positions
// past k_used get the largest node and weight 0).
cudaError_t launch_gauss_rules(int n_nodes, const LanczosParams& L, double* lambda, double* weight,
                               cudaStream_t stream);
// rho_j, e_j (band term) and s_j (entropy term) at (mu, kT); e and s may be NULL.
cudaError_t launch_lssgq_fields(int n_nodes, int K, const double* lambda, const double* weight, double mu,
                                double kT, double dV, double* rho, double* e, double* s, cudaStream_t stream);
// out[0] = mu with 2 sum_j nu_j sum_k w_jk g(lambda_jk; mu) = n_electrons,
// out[1] = the count at out[0], out[2] = bisection steps taken.
cudaError_t launch_fermi_level(int n_nodes, int K, const double* lambda, const double* weight,
                               const double* nu, double kT, double n_electrons, double* out,
                               cudaStream_t stream);

}  // namespace md
