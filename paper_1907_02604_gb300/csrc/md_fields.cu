// Free-energy fields from the per-system node values x_jp(j) (md_free_energy,
// md_energy, md_fermi_level_poles):
//   s_j = 2 kT sum_p Im(w^S_p x_jp(j))   entropy term of Eq. (tot) at node j,
//         w^S the weights of the entropy function on the same poles;
// and the node-weighted totals of the cluster-sampled energy (Section 3,
// Eqs. free_cg, free_cg_sampling) and of the electron count (Eq. Fermi:Rho):
//   N = dV sum nu_j rho_j,  E = sum nu_j e_j,  TS = sum nu_j s_j,  F = E - TS.
#include <cuda_runtime.h>

#include "md_solver.h"

namespace md {

namespace {

__global__ void k_entropy(int n_nodes, int Pn, const double2* __restrict__ x_src, const double2* __restrict__ wS,
                          double kT, double* __restrict__ s) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_nodes) return;
    double acc = 0.0;
    for (int p = 0; p < Pn; ++p) {   // poles in a fixed order
        const double2 xv = x_src[(long long)j * Pn + p];
        const double2 ww = wS[p];
        acc += ww.x * xv.y + ww.y * xv.x;   // Im(w x)
    }
    s[j] = 2.0 * kT * acc;
}

constexpr int kTotThreads = 1024;

// One CTA: thread t sums nodes t, t + 1024, ... in order, then a fixed
// pairwise tree over the threads, so the totals do not depend on scheduling.
__global__ void __launch_bounds__(kTotThreads) k_weighted_totals(long long n, const double* __restrict__ rho,
                                                                 const double* __restrict__ e,
                                                                 const double* __restrict__ s,
                                                                 const double* __restrict__ nu, double dV,
                                                                 double* __restrict__ out) {
    __shared__ double sh[3][kTotThreads];
    double a = 0.0, b = 0.0, c = 0.0;
    for (long long j = threadIdx.x; j < n; j += kTotThreads) {
        const double w = nu ? nu[j] : 1.0;
        if (rho) a += w * rho[j];
        if (e) b += w * e[j];
        if (s) c += w * s[j];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int half = kTotThreads / 2; half > 0; half >>= 1) {
        if (threadIdx.x < half)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + half];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = dV * sh[0][0];
        out[1] = sh[1][0];
        out[2] = sh[2][0];
        out[3] = sh[1][0] - sh[2][0];
    }
}

}  // namespace

cudaError_t launch_entropy(int n_nodes, int Pn, const double2* x_src, const double2* wS, double kT, double* s,
                           cudaStream_t stream) {
    if (n_nodes <= 0) return cudaSuccess;
    k_entropy<<<(n_nodes + 127) / 128, 128, 0, stream>>>(n_nodes, Pn, x_src, wS, kT, s);
    return cudaGetLastError();
}

cudaError_t launch_weighted_totals(long long n, const double* rho, const double* e, const double* s,
                                   const double* nu, double dV, double* out, cudaStream_t stream) {
    k_weighted_totals<<<1, kTotThreads, 0, stream>>>(n, rho, e, s, nu, dV, out);
    return cudaGetLastError();
}

}  // namespace md
