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
    int cl_slab;                    // cluster kernel: points of the thickest z-slab a CTA holds
    int cl_row_cap;                 // cluster kernel: nonlocal row records per CTA (upper bound)
    int cl_key_cap;                 // cluster kernel: region rows of the thickest slab
    int cl_wx;                      // cluster kernel: projector window length along x (tables)
    int cl_xcap;                    // cluster kernel: atoms whose x tables fit in shared memory
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
// Mixed-precision COCG with the Krylov vectors in shared memory, one thread
// block cluster of csz CTAs per system (regions without whole-axis rings,
// stencil half-width 1..4); grid = resident clusters * csz, block <=
// cl_max_threads(), smem = cl_smem_bytes(P.cl_slab, 2 P.cl_xcap P.cl_wx) dynamic bytes, and
// P.slot_bytes = cl_slot_bytes(n_max, csz, P.cl_slab, P.nonlocal, P.cl_row_cap, P.cl_key_cap)
// of scratch per cluster.
bool cl_supported(int precision, int q);
int cl_max_threads();
size_t cl_smem_bytes(int slab_pts, int xtab_floats);
size_t cl_static_smem_bytes();
int cl_max_clusters(int q, int csz, int block, size_t smem);   // resident clusters on the device
size_t cl_slot_bytes(long long n_max, int csz, int slab_pts, int nonlocal, int row_cap, int key_cap);
cudaError_t launch_cocg_cl(const SolveParams& P, int csz, int grid, int block, size_t smem, cudaStream_t stream);
// s_j = 2 kT sum_p Im(wS_p x_jp(j)) (entropy term per node).
cudaError_t launch_entropy(int n_nodes, int Pn, const double2* x_src, const double2* wS, double kT, double* s,
                           cudaStream_t stream);
// out[0..3] = dV sum nu rho, sum nu e, sum nu s, sum nu e - sum nu s (device,
// fixed summation order); any of rho, e, s may be NULL (its sum is 0), nu
// NULL means nu = 1.
cudaError_t launch_weighted_totals(long long n, const double* rho, const double* e, const double* s,
                                   const double* nu, double dV, double* out, cudaStream_t stream);
cudaError_t launch_accumulate(int n_nodes, int Pn, const double2* x_src, const double2* z,
                              const double2* w, double dV, double* rho, double* e, cudaStream_t stream);

}  // namespace md
