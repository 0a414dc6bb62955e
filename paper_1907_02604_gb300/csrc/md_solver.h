// Parameters of the batched COCG kernel and its launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "md_internal.h"

namespace md {

struct SysDesc {   // one (node, pole) system in scheduling order
    int node;
    int pole;
};

struct NodeDesc {  // geometry of one node's region
    int dims[3];   // region points per axis
    int lo[3];     // unwrapped global coordinate of region-local 0 (ring: 0)
    int ring;      // bit d: axis d is a whole periodic ring
    int src;       // region-local linear index of the node
};

struct SolveParams {
    // grid and operator
    int n[3];
    int periodic[3];
    long long N;
    int q;
    double coef[3][kMaxQ];
    double diag;
    double dV;
    const double* V;
    const float* V32;
    // nonlocal projectors
    int nonlocal;
    long long n_atoms;
    const int* proj_i0;
    const int* proj_len;
    const double* proj_d;
    const double* proj_g;
    const float* proj_d32;
    const float* proj_g32;
    const double* proj_C;
    const float* proj_C32;
    const unsigned char* proj_rows;
    const int* pl_ptr;
    const int* pl_atom;
    const float4* pl_val32;
    const double2* pl_val64;
    double e_s, e_p;
    // systems
    int n_sys;
    int P;
    const SysDesc* sys;
    const NodeDesc* nodes;
    const double2* z;
    // solver settings
    double tol;
    int maxit;
    int reliable_every;
    double reliable_delta;
    unsigned long long timeout_ns;
    // workspace
    char* scratch;
    size_t slot_bytes;
    int n_max;                      // vector length per slot (rounded up)
    int zm_m0, zm_m1;               // z-march kernel: largest region extents in x, y
    int multishift;                 // 1: one shifted-COCG sequence per node (work items are nodes)
    // fused adjoint: when fused_dLdV != NULL every converged system adds
    // -Im((2 a_j/dV + 2 b_j z_p) w_p x(k)^2) to fused_dLdV[g(k)]
    double* fused_dLdV;
    const double* fused_a;          // dL/drho per node, or NULL (= 0)
    const double* fused_b;          // dL/de per node, or NULL (= 0)
    const double2* w;               // pole weights
    // density-matrix rows: when dm_rows != NULL every converged system adds
    // Im(w_p x(k)) to dm_rows[dm_off[node] + k] (k region-local)
    double* dm_rows;
    const long long* dm_off;
    double2* ckpt;                  // NULL or checkpoint base
    const long long* ckpt_sys_off;  // point offset of system (node*P + pole) in ckpt
    unsigned int* work_counter;
    // outputs, indexed node*P + pole
    double2* x_src;
    int* status;
    int* iters;
    double* resid;
    int* n_rel;
};

size_t slot_bytes_for(int precision, long long n_max);
// Shared-memory z-march variant (mixed precision, stencil half-width 2 or 4,
// regions without whole-axis rings); K columns per thread.
bool zm_supported(int precision, int q);
int zm_max_threads(int K);
size_t zm_smem_bytes(int q, int max_m0, int max_m1);
int zm_occupancy(int q, int K, int block, size_t smem);   // resident CTAs per SM
cudaError_t launch_cocg_zm(const SolveParams& P, int K, int grid, int block, size_t smem, cudaStream_t stream);
// per_sm >= 3 with block <= 512 (mixed precision) selects the instance
// compiled for three resident CTAs per SM (40 registers per thread).
cudaError_t launch_cocg(const SolveParams& P, int precision, int grid, int block, int per_sm,
                        cudaStream_t stream);
cudaError_t launch_accumulate(int n_nodes, int Pn, const double2* x_src, const double2* z,
                              const double2* w, double dV, double* rho, double* e, cudaStream_t stream);

}  // namespace md
