// Adjoint of the nodal density and band energy (md_density_adjoint).
//
// G = (H_R - z)^-1 is complex symmetric, so the derivative of its diagonal
// entry with respect to the potential at region point k is
//   d G_jj / d V_k = -G_jk G_kj = -x_jp(k)^2,
// with x_jp the forward solution of (H_R - z_p) x = e_j: the adjoint systems
// are the forward systems and no second solve is needed.  For
// L(rho, e) with a_j = dL/drho_j, b_j = dL/de_j:
//   dL/dV_k = -sum_j sum_p Im( (2 a_j/dV + 2 b_j z_p) w_p x_jp(k)^2 ).
// Forces on the Gaussian centres follow by the chain rule through the local
// wells (Hellmann-Feynman, Section 2.1 of the paper):
//   F_a = -sum_k dL/dV_k dV_k/dR_a,  dV_k/dR_a = V_a(r_k) (r_k - R_a)/sigma_a^2.
#include <cuda_runtime.h>

#include "md_adjoint.h"
#include "md_device.cuh"

namespace md {

namespace {

__global__ void k_adjoint_dV(AdjointParams A) {
    extern __shared__ double2 coefs[];  // P complex coefficients of the node
    for (long long j = blockIdx.x; j < A.n_nodes; j += gridDim.x) {
        const NodeDesc nd = A.nodes[j];
        const int n = nd.dims[0] * nd.dims[1] * nd.dims[2];
        const double aj = A.dL_drho[j];
        const double bj = A.dL_de ? A.dL_de[j] : 0.0;
        __syncthreads();
        for (int p = threadIdx.x; p < A.P; p += blockDim.x) {
            // (2 a_j / dV + 2 b_j z_p) w_p
            const double2 z = A.z[p], w = A.w[p];
            const double cr = 2.0 * aj / A.dV + 2.0 * bj * z.x;
            const double ci = 2.0 * bj * z.y;
            coefs[p] = make_double2(cr * w.x - ci * w.y, cr * w.y + ci * w.x);
        }
        __syncthreads();
        const double2* xj = A.ckpt + A.P * A.node_off[j];
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double acc_im = 0.0;
            for (int p = 0; p < A.P; ++p) {
                const double2 x = xj[(long long)p * n + i];
                const double sq_re = x.x * x.x - x.y * x.y;
                const double sq_im = 2.0 * x.x * x.y;
                const double2 c = coefs[p];
                acc_im += c.x * sq_im + c.y * sq_re;
            }
            const int a = i % nd.dims[0];
            const int b = (i / nd.dims[0]) % nd.dims[1];
            const int c = i / (nd.dims[0] * nd.dims[1]);
            int gx = nd.lo[0] + a, gy = nd.lo[1] + b, gz = nd.lo[2] + c;
            gx = (gx % A.n[0] + A.n[0]) % A.n[0];
            gy = (gy % A.n[1] + A.n[1]) % A.n[1];
            gz = (gz % A.n[2] + A.n[2]) % A.n[2];
            const long long g = gx + (long long)A.n[0] * (gy + (long long)A.n[1] * gz);
            atomicAdd(&A.dLdV[g], -acc_im);
        }
    }
}

// Grid indices of the points within rc of X on one axis, enumerated by t.
struct AxisRange {
    int start;   // unwrapped first index (or 0 when the whole axis is used)
    int count;
    int full;    // whole axis, minimum-image displacement
};

__device__ __forceinline__ AxisRange axis_range(double X, double rc, double h, int n, int periodic) {
    AxisRange r;
    const int s = (int)ceil((X - rc) / h);
    const int e = (int)floor((X + rc) / h);
    if (periodic && e - s + 1 >= n) {
        r.start = 0;
        r.count = n;
        r.full = 1;
    } else if (periodic) {
        r.start = s;
        r.count = e - s + 1;
        r.full = 0;
    } else {
        const int s2 = s < 0 ? 0 : s;
        const int e2 = e > n - 1 ? n - 1 : e;
        r.start = s2;
        r.count = e2 >= s2 ? e2 - s2 + 1 : 0;
        r.full = 0;
    }
    return r;
}

__device__ __forceinline__ void axis_point(const AxisRange& r, int t, double X, double h, int n, int periodic,
                                           int& idx, double& d) {
    if (r.full) {
        idx = t;
        const double L = n * h;
        d = t * h - X;
        d -= L * rint(d / L);
    } else {
        const int u = r.start + t;
        d = u * h - X;
        idx = periodic ? ((u % n) + n) % n : u;
    }
}

__global__ void k_forces(ForceParams F) {
    __shared__ double red[32][3];
    for (long long at = blockIdx.x; at < F.n_atoms; at += gridDim.x) {
        const double X[3] = {F.xyz[3 * at], F.xyz[3 * at + 1], F.xyz[3 * at + 2]};
        const double sig = F.sigma[at], D = F.depth[at];
        const double rc = F.cutoff_sigmas * sig;
        AxisRange ax[3];
        for (int d = 0; d < 3; ++d) ax[d] = axis_range(X[d], rc, F.h[d], F.n[d], F.periodic[d]);
        const long long total = (long long)ax[0].count * ax[1].count * ax[2].count;
        double f[3] = {0, 0, 0};
        for (long long t = threadIdx.x; t < total; t += blockDim.x) {
            const int tx = (int)(t % ax[0].count);
            const int ty = (int)((t / ax[0].count) % ax[1].count);
            const int tz = (int)(t / ((long long)ax[0].count * ax[1].count));
            int ix, iy, iz;
            double dx, dy, dz;
            axis_point(ax[0], tx, X[0], F.h[0], F.n[0], F.periodic[0], ix, dx);
            axis_point(ax[1], ty, X[1], F.h[1], F.n[1], F.periodic[1], iy, dy);
            axis_point(ax[2], tz, X[2], F.h[2], F.n[2], F.periodic[2], iz, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > rc * rc) continue;
            const long long g = ix + (long long)F.n[0] * (iy + (long long)F.n[1] * iz);
            const double Va = -D * exp(-r2 / (2.0 * sig * sig));
            const double s = F.dLdV[g] * Va / (sig * sig);
            f[0] -= s * dx;
            f[1] -= s * dy;
            f[2] -= s * dz;
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int d = 0; d < 3; ++d) f[d] = warp_sum(f[d]);
        if (lane == 0)
            for (int d = 0; d < 3; ++d) red[warp][d] = f[d];
        __syncthreads();
        if (threadIdx.x < 3) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
            F.forces[3 * at + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_adjoint_dV(const AdjointParams& A, cudaStream_t stream) {
    const int grid = (int)(A.n_nodes < 152LL * 8 ? A.n_nodes : 152LL * 8);
    if (grid <= 0) return cudaSuccess;
    k_adjoint_dV<<<grid, 256, A.P * sizeof(double2), stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_forces(const ForceParams& F, cudaStream_t stream) {
    const int grid = (int)(F.n_atoms < 152LL * 8 ? F.n_atoms : 152LL * 8);
    if (grid <= 0) return cudaSuccess;
    k_forces<<<grid, 256, 0, stream>>>(F);
    return cudaGetLastError();
}

}  // namespace md
