// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>
#include <vector_types.h>

#include "../../include/macrodft.h"

namespace md {

constexpr int kMaxQ = 8;               // fd_order <= 16
constexpr int kMaxProjWin = 40;        // projector window points per axis
constexpr int kMaxLocalProjAtoms = 256;

md_status set_error(md_status code, const std::string& msg);
void clear_error();

struct Ham;
md_status compute_bounds(Ham& H, void* stream);
md_status set_potential_device(Ham& H, const double* V_in, void* stream);
md_status make_poles(double kT, double mu, double emin, double emax, int P, double* z_out,
                     double* w_out);
md_status make_entropy_weights(double kT, double mu, double emin, double emax, int P, double* w_out);
md_status fma_rate_probe(int precision, cudaStream_t s, double* tflops);

// Device-resident Hamiltonian.
struct Ham {
    int n[3];
    double h[3];
    int periodic[3];
    int fd_order;
    int q;
    double coef[3][kMaxQ];   // -1/2 w_o / h_d^2, o = 1..q
    double diag;             // -1/2 sum_d w_0 / h_d^2
    long long N;
    double dV;
    int device;

    double* V = nullptr;     // [N] FP64
    float* V32 = nullptr;    // [N] FP32 copy (mixed precision)

    long long n_atoms = 0;
    double* atom_xyz = nullptr;   // [3 n_atoms]
    double* atom_depth = nullptr; // [n_atoms]
    double* atom_sigma = nullptr; // [n_atoms]
    double cutoff_sigmas = 8.0;

    // nonlocal projectors
    int nonlocal = 0;
    double proj_sigma = 1.0, proj_rc = 4.0, e_s = 0.5, e_p = 0.25;
    int win_max[3] = {0, 0, 0};       // table length per axis
    int* proj_i0 = nullptr;           // [n_atoms][3] unwrapped window start index
    int* proj_len = nullptr;          // [n_atoms][3] window length
    double* proj_d = nullptr;         // [n_atoms][3][kMaxProjWin] displacement i*h - X
    double* proj_g = nullptr;         // [n_atoms][3][kMaxProjWin] exp(-d^2/(2 s^2))
    float* proj_d32 = nullptr;
    float* proj_g32 = nullptr;
    double* proj_C = nullptr;         // [n_atoms][4] normalisation constants
    double* proj_absum = nullptr;     // [n_atoms][4] sum_i |p(i)| (Gershgorin radii)
    float* proj_C32 = nullptr;
    unsigned char* proj_rows = nullptr; // [n_atoms][W][W][2]: in-sphere u range of row (v, w)
    int* pl_ptr = nullptr;            // [N+1] per-point projector-atom lists
    int* pl_atom = nullptr;           // [nnz] atom ids, ascending per point
    float4* pl_val32 = nullptr;       // [nnz] (p_s, p_x, p_y, p_z) at the point, FP32
    double2* pl_val64 = nullptr;      // [nnz][2] the same in FP64
    long long pl_nnz = 0;

    bool bounds_valid = false;
    double emin = 0.0, emax = 0.0;

    // cached solver scratch (grow-only)
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // cached work lists and per-node Lanczos results of md_lssgq_rules (grow-only)
    void* lz_buf = nullptr;
    size_t lz_bytes = 0;
    // pinned staging of the uploads of asynchronous md_density calls, two in
    // turn; an event marks when a buffer's last uploads have been read
    struct Stage {
        void* buf = nullptr;
        size_t bytes = 0;
        cudaEvent_t ev = nullptr;
    } stage[2];
    int stage_next = 0;
    // recorded after each asynchronous md_density call: the scratch above is
    // in use until it completes
    cudaEvent_t scratch_ev = nullptr;
};

}  // namespace md

struct md_hamiltonian {
    md::Ham h;
};

struct md_workspace {
    int device;
    long long n_nodes;
    int n_poles;
    long long total_points;    // sum over nodes of region points
    long long* node_off;       // host [n_nodes]: point offset of node j's block
    double* x;                 // device complex128 [P * total_points]
    // layout: system (j, p) at x + 2 * (P * node_off[j] + p * |R(j)|)
};
