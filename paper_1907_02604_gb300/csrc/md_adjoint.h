// Parameters of the adjoint (dL/dV) and force kernels.
#pragma once

#include <cuda_runtime.h>

#include "md_solver.h"

namespace md {

struct AdjointParams {
    int n[3];
    long long n_nodes;
    int P;
    const NodeDesc* nodes;
    const long long* node_off;   // point offset of node j's block in ckpt (times P)
    const double2* ckpt;
    const double2* z;
    const double2* w;
    const double* dL_drho;
    const double* dL_de;         // may be NULL
    double dV;
    double* dLdV;                // zeroed by the caller
};

struct ForceParams {
    int n[3];
    double h[3];
    int periodic[3];
    long long n_atoms;
    const double* xyz;
    const double* depth;
    const double* sigma;
    double cutoff_sigmas;
    const double* dLdV;
    double* forces;
};

cudaError_t launch_adjoint_dV(const AdjointParams& A, cudaStream_t stream);
cudaError_t launch_forces(const ForceParams& F, cudaStream_t stream);

}  // namespace md
