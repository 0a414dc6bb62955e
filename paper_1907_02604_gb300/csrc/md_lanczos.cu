// Lanczos spectral Gauss quadrature (LSSGQ; Section 2.1, Eq. 9 and Eqs.
// (Fermi:Rho), (Electron_density:GQ), (tot)).
//
// k_lanczos: one CTA per node at a time (persistent, cost-sorted work list),
//   K steps of the symmetric Lanczos process on H_R(j) from q_1 = e_j in
//   real arithmetic (FP64, or FP32 vectors with FP64 scalars), no
//   reorthogonalisation.  Two region vectors per
//   CTA, each kept with a scale (q = sigma u) so that normalising the new
//   Lanczos vector costs no pass of its own.  Per step:
//     NL  c_al = sum_i p_al(i) u_c(i)                 (nonlocal coefficients)
//     A   w = sigma_c H u_c - beta_{k-1} sigma_p u_p  (stored over u_p)
//         alpha_k = sigma_c u_c . w
//     B   w -= alpha_k sigma_c u_c,  beta_k = ||w||  (stored over u_p)
//   then (u_c, u_p) <- (w, u_c) with sigma_c = 1/beta_k.  Stops after K
//   steps, or earlier when beta_k <= breakdown_tol (|alpha_1| + beta_1 + 1):
//   the Krylov space is invariant there and the shorter rule is exact.
//
// k_gauss_rules: one thread per node; the eigenvalues of the Jacobi matrix
//   T_k (diagonal alpha, off-diagonal beta) by implicit symmetric QR steps
//   with the Wilkinson shift (Golub & Van Loan, Matrix Computations,
//   Section 8.3), tracking only the first row of the accumulated rotations:
//   its squares are the Gauss weights (Golub & Welsch, Math. Comp. 23, 1969).
//
// k_lssgq_fields: per node rho_j = (2/dV) sum_k w_k g(l_k),
//   e_j = 2 sum_k w_k l_k g(l_k), s_j = -2 kT sum_k w_k [g ln g + (1-g) ln(1-g)].
//
// k_fermi_level: one CTA; bisection on mu for
//   N_e(mu) = 2 sum_j nu_j sum_k w_jk g(l_jk; mu) = n_electrons,
//   increasing in mu; the rules do not depend on mu, so no solve is repeated.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "md_lanczos.h"
#include "md_operator.cuh"

namespace md {

namespace {

// Block-wide sums of float-float partials, broadcast to every thread.
template <int K>
__device__ __forceinline__ void block_sum_ff(Shared& S, const float (&hi)[K], const float (&lo)[K],
                                             double (&v)[K]) {
    block_reduce_ff<K>(S, hi, lo, v);
    if (threadIdx.x == 0)
        for (int k = 0; k < K; ++k) S.bcast[k] = v[k];
    __syncthreads();
    for (int k = 0; k < K; ++k) v[k] = S.bcast[k];
}

// R = double: FP64 vectors and arithmetic.  R = float: FP32 vectors,
// stencil and projector terms, compensated FP32 partial sums reduced in
// float-float and FP64; alpha, beta and the vector scales stay FP64.
template <class R, int Q>
__global__ void __launch_bounds__(1024) k_lanczos(const __grid_constant__ SolveParams P,
                                                  const LanczosParams L) {
    __shared__ Shared S;
    constexpr bool kF32 = std::is_same<R, float>::value;
    const uint64_t t_start = global_time_ns();
    R* const u0 = reinterpret_cast<R*>(P.scratch + (size_t)blockIdx.x * P.slot_bytes);
    R* const u1 = u0 + P.n_max;
    for (int t = threadIdx.x; t < 3 * kMaxQ; t += blockDim.x) {
        (&S.coefD[0][0])[t] = (&P.coef[0][0])[t];
        (&S.coefF[0][0])[t] = (float)(&P.coef[0][0])[t];
    }
    if (P.nonlocal && P.n_atoms <= kMapMax)
        for (int t = threadIdx.x; t < P.n_atoms; t += blockDim.x) S.map[t] = -1;

    for (;;) {
        if (threadIdx.x == 0) {
            S.sys = (int)atomicAdd(P.work_counter, 1u);
            S.flag = 0;
        }
        __syncthreads();
        const int s = S.sys;
        if (s >= P.n_sys) break;
        const int node = P.sys[s].node;
        const NodeDesc nd = P.nodes[node];
        Geo G;
        G.any_ring = 0;
        for (int d = 0; d < 3; ++d) {
            G.m[d] = nd.dims[d];
            G.lo[d] = nd.lo[d];
            G.ring[d] = (nd.ring >> d) & 1;
            G.any_ring |= G.ring[d];
        }
        G.plane = G.m[0] * G.m[1];
        G.n = G.plane * G.m[2];
        G.src = nd.src;
        G.div_row = make_fastdiv((uint32_t)G.m[0]);
        G.div_plane = make_fastdiv((uint32_t)G.plane);
        const long long base = (long long)node * L.K;

        if (P.nonlocal) {
            collect_local_atoms(P, G, S);
            uint2* rec = reinterpret_cast<uint2*>(u1 + P.n_max);   // point records after the vectors
            build_nl_records(P, G, S, rec);
            G.nl_rec = rec;
        }
        R* uc = u0;
        R* up = u1;
        for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
            uc[i] = (i == G.src) ? (R)1 : (R)0;
            up[i] = (R)0;
        }
        double sc = 1.0, sp = 0.0, bprev = 0.0, scale = 0.0;
        int k_done = 0;
        bool timed_out = false;
        __syncthreads();
        for (int k = 0; k < L.K; ++k) {
            if (threadIdx.x == 0)
                S.action = (P.timeout_ns && (global_time_ns() - t_start) > P.timeout_ns) ? kStopTimeout : 0;
            __syncthreads();
            if (S.action == kStopTimeout) {
                timed_out = true;
                break;
            }
            if (P.nonlocal) nonlocal_coeffs<R, R>(P, G, S, uc);
            const double cb = bprev * sp;
            double a, b;
            if constexpr (kF32) {
                const float scf = (float)sc, cbf = (float)cb;
                KSum<float> acc;
                // each point's projector record is loaded one point ahead
                const bool pre = P.nonlocal && G.nl_rec;
                uint2 rc_next = make_uint2(0u, 0xFFFFFFFFu);
                if (pre && threadIdx.x < G.n) rc_next = G.nl_rec[threadIdx.x];
                for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                    const uint2 rc = rc_next;
                    if (pre && i + (int)blockDim.x < G.n) rc_next = G.nl_rec[i + blockDim.x];
                    const float y = matvec_point<float, float, Q, float>(P, G, S, uc, i, 0.f, 0.f, (float)P.diag,
                                                                         pre ? rc : make_uint2(0u, 0xFFFFFFFEu));
                    const float wv = scf * y - cbf * up[i];
                    up[i] = wv;
                    acc.add(uc[i] * wv);
                }
                double t1[1];
                const float h1[1] = {acc.hi()}, l1[1] = {acc.lo()};
                block_sum_ff<1>(S, h1, l1, t1);
                a = sc * t1[0];
                const float caf = (float)(a * sc);
                KSum<float> acc2;
                for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                    const float wv = up[i] - caf * uc[i];
                    up[i] = wv;
                    acc2.add(wv * wv);
                }
                double t2[1];
                const float h2[1] = {acc2.hi()}, l2[1] = {acc2.lo()};
                block_sum_ff<1>(S, h2, l2, t2);
                b = sqrt(t2[0]);
            } else {
                double acc[1] = {0.0};
                for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                    const double y = matvec_point<double, double, Q, double>(P, G, S, uc, i, 0.0, 0.0, P.diag);
                    const double wv = sc * y - cb * up[i];
                    up[i] = wv;
                    acc[0] += uc[i] * wv;
                }
                block_sum<1>(S, acc);
                a = sc * acc[0];
                const double ca = a * sc;
                double acc2[1] = {0.0};
                for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                    const double wv = up[i] - ca * uc[i];
                    up[i] = wv;
                    acc2[0] += wv * wv;
                }
                block_sum<1>(S, acc2);
                b = sqrt(acc2[0]);
            }
            if (k == 0) scale = fabs(a) + b + 1.0;
            if (threadIdx.x == 0) L.alpha[base + k] = a;
            k_done = k + 1;
            if (k == L.K - 1 || b <= L.breakdown_tol * scale) break;
            if (threadIdx.x == 0) L.beta[base + k] = b;
            R* t = uc;
            uc = up;
            up = t;
            sp = sc;
            sc = 1.0 / b;
            bprev = b;
        }
        if (threadIdx.x == 0) {
            L.k_used[node] = k_done;
            L.status[node] = timed_out ? 4 : (S.flag ? 1 : 0);
        }
        if (P.nonlocal) release_local_atoms(P, S);
        __syncthreads();
    }
}

// Eigenvalues and first-row eigenvector components of the n x n Jacobi
// matrix (d, e) in place; returns false if some eigenvalue did not converge
// within 30 n steps.
__device__ bool jacobi_eig_first_row(int n, double* d, double* e, double* z) {
    for (int i = 0; i < n; ++i) z[i] = (i == 0) ? 1.0 : 0.0;
    int hi = n - 1;
    int steps = 0;
    while (hi > 0) {
        if (fabs(e[hi - 1]) <= DBL_EPSILON * (fabs(d[hi - 1]) + fabs(d[hi]))) {
            e[hi - 1] = 0.0;   // d[hi] has converged
            --hi;
            continue;
        }
        int lo = hi - 1;       // unreduced block [lo, hi]
        while (lo > 0 && fabs(e[lo - 1]) > DBL_EPSILON * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
        if (lo > 0) e[lo - 1] = 0.0;
        if (++steps > 30 * n) return false;
        // Wilkinson shift: eigenvalue of the trailing 2x2 block nearer d[hi]
        const double delta = 0.5 * (d[hi - 1] - d[hi]);
        const double b2 = e[hi - 1] * e[hi - 1];
        const double mu = d[hi] - b2 / (delta + copysign(sqrt(delta * delta + b2), delta));
        // bulge chase: rotation k acts on rows / columns k, k+1; its first
        // one is fixed by the first column of T - mu I
        double x = d[lo] - mu, y = e[lo];
        for (int k = lo; k < hi; ++k) {
            const double r = hypot(x, y);
            double c = 1.0, s = 0.0;
            if (r > 0.0) {
                c = x / r;
                s = y / r;
            }
            if (k > lo) e[k - 1] = r;
            const double ak = d[k], ak1 = d[k + 1], bk = e[k];
            d[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
            d[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
            e[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
            if (k + 1 < hi) {
                const double bk1 = e[k + 1];
                y = s * bk1;          // bulge at (k+2, k)
                e[k + 1] = c * bk1;
                x = e[k];
            }
            const double zk = z[k], zk1 = z[k + 1];
            z[k] = c * zk + s * zk1;
            z[k + 1] = c * zk1 - s * zk;
        }
    }
    return true;
}

__global__ void k_gauss_rules(int n_nodes, const LanczosParams L, double* __restrict__ lambda,
                              double* __restrict__ weight) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_nodes) return;
    double d[kMaxLanczosK], e[kMaxLanczosK], z[kMaxLanczosK];
    const long long base = (long long)j * L.K;
    const int n = L.k_used[j];
    if (n <= 0) {
        for (int k = 0; k < L.K; ++k) {
            lambda[base + k] = 0.0;
            weight[base + k] = 0.0;
        }
        return;
    }
    for (int k = 0; k < n; ++k) d[k] = L.alpha[base + k];
    for (int k = 0; k + 1 < n; ++k) e[k] = L.beta[base + k];
    e[n - 1] = 0.0;
    const bool ok = jacobi_eig_first_row(n, d, e, z);
    if (!ok && L.status[j] == 0) L.status[j] = 3;
    // ascending nodes (insertion sort; n <= 128)
    for (int a = 1; a < n; ++a) {
        const double dv = d[a], zv = z[a];
        int b = a - 1;
        while (b >= 0 && d[b] > dv) {
            d[b + 1] = d[b];
            z[b + 1] = z[b];
            --b;
        }
        d[b + 1] = dv;
        z[b + 1] = zv;
    }
    for (int k = 0; k < L.K; ++k) {
        lambda[base + k] = d[k < n ? k : n - 1];
        weight[base + k] = k < n ? z[k] * z[k] : 0.0;
    }
}

// g(x) = 1/(1 + e^x) and 1 - g(x), each without cancellation.
__device__ __forceinline__ void fermi_pair(double x, double& g, double& h) {
    const double t = exp(-fabs(x));          // in (0, 1]
    const double inv = 1.0 / (1.0 + t);
    if (x > 0.0) {
        g = t * inv;
        h = inv;
    } else {
        g = inv;
        h = t * inv;
    }
}

__global__ void k_lssgq_fields(int n_nodes, int K, const double* __restrict__ lambda,
                               const double* __restrict__ weight, double mu, double kT, double dV,
                               double* __restrict__ rho, double* __restrict__ e, double* __restrict__ s) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_nodes) return;
    double sr = 0.0, se = 0.0, ss = 0.0;
    for (int k = 0; k < K; ++k) {
        const double l = lambda[(long long)j * K + k], wk = weight[(long long)j * K + k];
        const double x = (l - mu) / kT;
        double g, h;
        fermi_pair(x, g, h);
        // ln(1 + e^x) and ln(1 + e^-x)
        const double lp = fmax(x, 0.0) + log1p(exp(-fabs(x)));
        const double ln = fmax(-x, 0.0) + log1p(exp(-fabs(x)));
        sr += wk * g;
        se += wk * l * g;
        ss += wk * (-g * lp - h * ln);
    }
    rho[j] = 2.0 / dV * sr;
    if (e) e[j] = 2.0 * se;
    if (s) s[j] = -2.0 * kT * ss;
}

__device__ double block_total(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += red[k];   // same order in every thread
    return t;
}

__device__ double block_extreme(double v, double* red, bool want_max) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = want_max ? warp_max(v) : warp_min(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = red[0];
    for (int k = 1; k < nw; ++k) t = want_max ? fmax(t, red[k]) : fmin(t, red[k]);
    return t;
}

__global__ void __launch_bounds__(1024) k_fermi_level(int n_nodes, int K, const double* __restrict__ lambda,
                                                      const double* __restrict__ weight,
                                                      const double* __restrict__ nu, double kT,
                                                      double n_electrons, double* __restrict__ out) {
    __shared__ double red[32];
    const long long n = (long long)n_nodes * K;
    double lmin = DBL_MAX, lmax = -DBL_MAX;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) {
        lmin = fmin(lmin, lambda[t]);
        lmax = fmax(lmax, lambda[t]);
    }
    double lo = block_extreme(lmin, red, false) - 40.0 * kT;
    double hi = block_extreme(lmax, red, true) + 40.0 * kT;
    int steps = 0;
    double count = 0.0;
    for (; steps < 200; ++steps) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double part = 0.0;
        for (long long t = threadIdx.x; t < n; t += blockDim.x) {
            double g, h;
            fermi_pair((lambda[t] - mid) / kT, g, h);
            const double nj = nu ? nu[t / K] : 1.0;
            part += nj * weight[t] * g;
        }
        count = 2.0 * block_total(part, red);
        if (count < n_electrons) lo = mid;
        else hi = mid;
    }
    const double mu = 0.5 * (lo + hi);
    double part = 0.0;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) {
        double g, h;
        fermi_pair((lambda[t] - mu) / kT, g, h);
        part += (nu ? nu[t / K] : 1.0) * weight[t] * g;
    }
    count = 2.0 * block_total(part, red);
    if (threadIdx.x == 0) {
        out[0] = mu;
        out[1] = count;
        out[2] = (double)steps;
    }
}

template <class R>
cudaError_t launch_lanczos_r(const SolveParams& P, const LanczosParams& L, int grid, int block,
                             cudaStream_t stream) {
    switch (P.q) {
        case 1: k_lanczos<R, 1><<<grid, block, 0, stream>>>(P, L); break;
        case 2: k_lanczos<R, 2><<<grid, block, 0, stream>>>(P, L); break;
        case 3: k_lanczos<R, 3><<<grid, block, 0, stream>>>(P, L); break;
        case 4: k_lanczos<R, 4><<<grid, block, 0, stream>>>(P, L); break;
        case 5: k_lanczos<R, 5><<<grid, block, 0, stream>>>(P, L); break;
        case 6: k_lanczos<R, 6><<<grid, block, 0, stream>>>(P, L); break;
        case 7: k_lanczos<R, 7><<<grid, block, 0, stream>>>(P, L); break;
        case 8: k_lanczos<R, 8><<<grid, block, 0, stream>>>(P, L); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lanczos(const SolveParams& P, const LanczosParams& L, int precision, int grid, int block,
                           cudaStream_t stream) {
    if (precision == MD_PREC_MIXED) return launch_lanczos_r<float>(P, L, grid, block, stream);
    return launch_lanczos_r<double>(P, L, grid, block, stream);
}

cudaError_t launch_gauss_rules(int n_nodes, const LanczosParams& L, double* lambda, double* weight,
                               cudaStream_t stream) {
    if (n_nodes <= 0) return cudaSuccess;
    k_gauss_rules<<<(n_nodes + 63) / 64, 64, 0, stream>>>(n_nodes, L, lambda, weight);
    return cudaGetLastError();
}

cudaError_t launch_lssgq_fields(int n_nodes, int K, const double* lambda, const double* weight, double mu,
                                double kT, double dV, double* rho, double* e, double* s, cudaStream_t stream) {
    if (n_nodes <= 0) return cudaSuccess;
    k_lssgq_fields<<<(n_nodes + 127) / 128, 128, 0, stream>>>(n_nodes, K, lambda, weight, mu, kT, dV, rho, e, s);
    return cudaGetLastError();
}

cudaError_t launch_fermi_level(int n_nodes, int K, const double* lambda, const double* weight,
                               const double* nu, double kT, double n_electrons, double* out,
                               cudaStream_t stream) {
    k_fermi_level<<<1, 1024, 0, stream>>>(n_nodes, K, lambda, weight, nu, kT, n_electrons, out);
    return cudaGetLastError();
}

}  // namespace md
