// Batched COCG for the shifted systems (H_R(j) - z_p) x = e_j (md_density).
//
// One CTA owns one (node, pole) system at a time and takes the next one
// from a global work counter when it finishes (persistent scheduling over a
// cost-sorted list: largest regions and poles nearest the real axis
// first).  The Krylov vectors of the system live in a per-CTA slot of
// device scratch memory; the Hamiltonian (V, projector tables) is shared by
// all systems and stays in L2.
//
// Per COCG iteration (van der Vorst & Melissen 1990; bilinear u^T v, since
// H_R - z is complex symmetric):
//   P1  p = r + beta p
//   NL  c_al = sum_i p_al(i) p(i)          (nonlocal coefficients, warp per atom)
//   P2  Ap = (-1/2 L + V - z) p + sum_al E_l dV c_al p_al ;  p^T Ap
//   P3  x += alpha p ; r -= alpha Ap ;  r^T r, ||r||^2
// with alpha = r^T r / p^T Ap and beta = r_new^T r_new / r^T r.
//
// Precision modes:
//   FP64   every vector, scalar and product in double.
//   MIXED  p, r, Ap, the stencil, V and the projector values in float;
//          the solution is x_hi (double) + dx (float, reset at each
//          flush); each product/partial sum in a thread's run of points is
//          float, everything from the per-thread partial upward (warp and
//          block reductions, alpha, beta, norms) is double.  A reliable
//          update (van der Vorst & Ye 2000) recomputes the residual
//          r = e_j - (H_R - z) x_hi in double every `reliable_every`
//          iterations, whenever ||r|| fell by `reliable_delta` since the
//          last one, and before convergence is declared: the returned
//          solution always meets tol on its FP64 residual.
#include <cuda_runtime.h>

#include <cstdint>

#include "md_device.cuh"
#include "md_internal.h"
#include "md_solver.h"

namespace md {

namespace {

struct RegionGeo {
    int m[3];     // region points per axis
    int lo[3];    // unwrapped global coordinate of local 0 (ring axes: 0)
    int ring[3];  // axis is a whole periodic ring
    int n;        // total points
    int src;
};

template <class R>
struct Tables;

template <>
struct Tables<double> {
    __device__ static const double* d(const SolveParams& P) { return P.proj_d; }
    __device__ static const double* g(const SolveParams& P) { return P.proj_g; }
    __device__ static const double* C(const SolveParams& P) { return P.proj_C; }
    __device__ static double V(const SolveParams& P, long long gi) { return P.V[gi]; }
};
template <>
struct Tables<float> {
    __device__ static const float* d(const SolveParams& P) { return P.proj_d32; }
    __device__ static const float* g(const SolveParams& P) { return P.proj_g32; }
    __device__ static const float* C(const SolveParams& P) { return P.proj_C32; }
    __device__ static float V(const SolveParams& P, long long gi) { return P.V32[gi]; }
};

struct Shared {
    // nonlocal: local atom list (ascending id), window offsets in region coordinates
    int n_local;
    int la_id[kMaxLocalProjAtoms];
    short la_off[kMaxLocalProjAtoms][3];
    double2 c[kMaxLocalProjAtoms][4];     // projector coefficients of the current vector
    double red[32][4];
    double bcast[4];
    int sys;
    int flag;
};

__device__ __forceinline__ long long global_index(const SolveParams& P, const RegionGeo& G, int a, int b,
                                                  int c) {
    int gx = G.lo[0] + a, gy = G.lo[1] + b, gz = G.lo[2] + c;
    gx = (gx % P.n[0] + P.n[0]) % P.n[0];
    gy = (gy % P.n[1] + P.n[1]) % P.n[1];
    gz = (gz % P.n[2] + P.n[2]) % P.n[2];
    return gx + (long long)P.n[0] * (gy + (long long)P.n[1] * gz);
}

// Block-wide sum of K doubles (K <= 4); every thread gets the result.
template <int K>
__device__ __forceinline__ void block_sum(Shared& S, double (&v)[K]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) S.red[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nw ? S.red[lane][k] : 0.0;
            t = warp_sum(t);
            if (lane == 0) S.bcast[k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = S.bcast[k];
    __syncthreads();
}

// Region slot of window index u of an atom window starting at region offset off.
__device__ __forceinline__ int region_slot(int off, int u, int n, int m) {
    int a = off + u;
    if (a >= n) a -= n;
    return (a >= 0 && a < m) ? a : -1;
}

// Local atoms whose projector window meets the region; ascending atom id.
__device__ void collect_local_atoms(const SolveParams& P, const RegionGeo& G, Shared& S) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int count = 0;
        for (long long base = 0; base < P.n_atoms; base += 32) {
            const long long a = base + lane;
            bool hit = a < P.n_atoms;
            short off[3] = {0, 0, 0};
            if (hit) {
                for (int d = 0; d < 3; ++d) {
                    const int i0 = P.proj_i0[3 * a + d];
                    const int len = P.proj_len[3 * a + d];
                    int o = i0 - G.lo[d];
                    if (P.periodic[d]) {
                        o %= P.n[d];
                        if (o < 0) o += P.n[d];
                        // window covers region slots o..o+len-1 (mod n); meets [0, m)?
                        const bool meet = (o < G.m[d]) || (o + len - 1 >= P.n[d]);
                        hit = hit && meet;
                    } else {
                        hit = hit && (o < G.m[d]) && (o + len - 1 >= 0);
                    }
                    off[d] = (short)o;
                }
            }
            const unsigned mask = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int slot = count + __popc(mask & ((1u << lane) - 1u));
                if (slot < kMaxLocalProjAtoms) {
                    S.la_id[slot] = (int)a;
                    S.la_off[slot][0] = off[0];
                    S.la_off[slot][1] = off[1];
                    S.la_off[slot][2] = off[2];
                }
            }
            count += __popc(mask);
        }
        if (lane == 0) {
            S.n_local = count < kMaxLocalProjAtoms ? count : kMaxLocalProjAtoms;
            if (count > kMaxLocalProjAtoms) S.flag = 1;
        }
    }
    __syncthreads();
}

// c_al = sum_{i in region} p_al(i) v(i) for every local atom (warp per atom).
template <class R, class C>
__device__ void nonlocal_coeffs(const SolveParams& P, const RegionGeo& G, Shared& S, const C* __restrict__ v) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const R* dt = Tables<R>::d(P);
    const R* gt = Tables<R>::g(P);
    const R* Ct = Tables<R>::C(P);
    for (int k = warp; k < S.n_local; k += nw) {
        const int a = S.la_id[k];
        const int lx = P.proj_len[3 * a], ly = P.proj_len[3 * a + 1], lz = P.proj_len[3 * a + 2];
        const R* dx = dt + (3LL * a + 0) * kMaxProjWin;
        const R* dy = dt + (3LL * a + 1) * kMaxProjWin;
        const R* dz = dt + (3LL * a + 2) * kMaxProjWin;
        const R* gx = gt + (3LL * a + 0) * kMaxProjWin;
        const R* gy = gt + (3LL * a + 1) * kMaxProjWin;
        const R* gz = gt + (3LL * a + 2) * kMaxProjWin;
        R acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int row = lane; row < ly * lz; row += 32) {
            const int vv = row % ly, ww = row / ly;
            const int b = region_slot(S.la_off[k][1], vv, P.n[1], G.m[1]);
            const int c = region_slot(S.la_off[k][2], ww, P.n[2], G.m[2]);
            if (b < 0 || c < 0) continue;
            const unsigned char* rw = P.proj_rows + 2 * (((long long)a * kMaxProjWin + ww) * kMaxProjWin + vv);
            const int u0 = rw[0], u1 = rw[1];
            const R gyz = gy[vv] * gz[ww];
            for (int u = u0; u <= u1 && u < lx; ++u) {
                const int aa = region_slot(S.la_off[k][0], u, P.n[0], G.m[0]);
                if (aa < 0) continue;
                const C pv = v[aa + G.m[0] * (b + G.m[1] * c)];
                const R gg = gx[u] * gyz;
                const R f0 = gg, f1 = dx[u] * gg, f2 = dy[vv] * gg, f3 = dz[ww] * gg;
                acc[0] += f0 * pv.x; acc[1] += f0 * pv.y;
                acc[2] += f1 * pv.x; acc[3] += f1 * pv.y;
                acc[4] += f2 * pv.x; acc[5] += f2 * pv.y;
                acc[6] += f3 * pv.x; acc[7] += f3 * pv.y;
            }
        }
        double s[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) s[t] = warp_sum((double)acc[t]);
        if (lane == 0) {
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const double Cl = (double)Ct[4LL * a + l];
                const double E = (l == 0 ? P.e_s : P.e_p) * P.dV;
                // store E dV C c so the apply step only multiplies by the shape
                S.c[k][l] = make_double2(E * Cl * s[2 * l], E * Cl * s[2 * l + 1]);
            }
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int find_local(const Shared& S, int atom) {
    int lo = 0, hi = S.n_local - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = S.la_id[mid];
        if (v == atom) return mid;
        if (v < atom) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// y = (H_R - z) v at local point (a, b, c), linear index i, in real type R.
template <class R, class C, class CIn>
__device__ __forceinline__ C apply_point(const SolveParams& P, const RegionGeo& G, const Shared& S,
                                         const CIn* __restrict__ v, int i, int a, int b, int c, C z) {
    const long long gi = global_index(P, G, a, b, c);
    const CIn vi = v[i];
    const R dg = (R)P.diag + Tables<R>::V(P, gi);
    C y = cmake<C>((dg - z.x) * (R)vi.x + z.y * (R)vi.y, (dg - z.x) * (R)vi.y - z.y * (R)vi.x);
    const int pos[3] = {a, b, c};
    const int stride[3] = {1, G.m[0], G.m[0] * G.m[1]};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int md = G.m[d];
        for (int o = 1; o <= P.q; ++o) {
            const R w = (R)P.coef[d][o - 1];
            R sx = 0, sy = 0;
            int tp = pos[d] + o, tm = pos[d] - o;
            if (G.ring[d]) {
                tp %= md;
                tm = ((tm % md) + md) % md;
                const CIn up = v[i + (tp - pos[d]) * stride[d]];
                const CIn dn = v[i + (tm - pos[d]) * stride[d]];
                sx = (R)up.x + (R)dn.x;
                sy = (R)up.y + (R)dn.y;
            } else {
                if (tp < md) {
                    const CIn up = v[i + o * stride[d]];
                    sx += (R)up.x;
                    sy += (R)up.y;
                }
                if (tm >= 0) {
                    const CIn dn = v[i - o * stride[d]];
                    sx += (R)dn.x;
                    sy += (R)dn.y;
                }
            }
            y.x += w * sx;
            y.y += w * sy;
        }
    }
    if (P.nonlocal) {
        const R* dt = Tables<R>::d(P);
        const R* gt = Tables<R>::g(P);
        const R* Ct = Tables<R>::C(P);
        const int gx = (int)(gi % P.n[0]);
        const int gy = (int)((gi / P.n[0]) % P.n[1]);
        const int gz = (int)(gi / ((long long)P.n[0] * P.n[1]));
        for (long long e = P.pl_ptr[gi]; e < P.pl_ptr[gi + 1]; ++e) {
            const int at = P.pl_atom[e];
            const int k = find_local(S, at);
            if (k < 0) continue;
            int uu[3];
            const int gp[3] = {gx, gy, gz};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int u = gp[d] - P.proj_i0[3 * at + d];
                if (P.periodic[d]) {
                    u %= P.n[d];
                    if (u < 0) u += P.n[d];
                }
                uu[d] = u;
            }
            const R* ds = dt + 3LL * at * kMaxProjWin;
            const R* gs = gt + 3LL * at * kMaxProjWin;
            const R gg = gs[uu[0]] * gs[kMaxProjWin + uu[1]] * gs[2 * kMaxProjWin + uu[2]];
            const R f[4] = {gg, ds[uu[0]] * gg, ds[kMaxProjWin + uu[1]] * gg,
                            ds[2 * kMaxProjWin + uu[2]] * gg};
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const R sh = f[l] * Ct[4LL * at + l];
                y.x += sh * (R)S.c[k][l].x;
                y.y += sh * (R)S.c[k][l].y;
            }
        }
    }
    return y;
}

template <class Mode>
__global__ void __launch_bounds__(1024) k_cocg(const __grid_constant__ SolveParams P) {
    using R = typename Mode::real;
    using C = typename Mode::cplx;
    __shared__ Shared S;
    const uint64_t t_start = global_time_ns();
    char* slot = P.scratch + (size_t)blockIdx.x * P.slot_bytes;

    for (;;) {
        if (threadIdx.x == 0) {
            S.sys = (int)atomicAdd(P.work_counter, 1u);
            S.flag = 0;
        }
        __syncthreads();
        const int s = S.sys;
        if (s >= P.n_sys) break;
        const SysDesc sd = P.sys[s];
        const NodeDesc nd = P.nodes[sd.node];
        RegionGeo G;
        for (int d = 0; d < 3; ++d) {
            G.m[d] = nd.dims[d];
            G.lo[d] = nd.lo[d];
            G.ring[d] = (nd.ring >> d) & 1;
        }
        G.n = G.m[0] * G.m[1] * G.m[2];
        G.src = nd.src;
        const double2 zd = P.z[sd.pole];
        const C z = cmake<C>((R)zd.x, (R)zd.y);
        const long long out_idx = (long long)sd.node * P.P + sd.pole;

        // vectors
        C* r = (C*)slot;
        C* p = r + P.n_max;
        C* Ap = p + P.n_max;
        C* dx = Ap + P.n_max;                       // mixed only
        double2* x = (double2*)(dx + (Mode::kMixed ? P.n_max : 0));
        if (P.ckpt) x = P.ckpt + P.ckpt_sys_off[out_idx];

        if (P.nonlocal) collect_local_atoms(P, G, S);

        for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
            const R one = (i == G.src) ? (R)1 : (R)0;
            r[i] = cmake<C>(one, (R)0);
            p[i] = cmake<C>((R)0, (R)0);
            x[i] = make_double2(0.0, 0.0);
            if (Mode::kMixed) dx[i] = cmake<C>((R)0, (R)0);
        }
        __syncthreads();

        double rho_re = 1.0, rho_im = 0.0;   // r^T r
        double beta_re = 0.0, beta_im = 0.0;
        double rn = 1.0, rn_last_rel = 1.0;
        int it = 0, last_rel = 0, n_rel = 0;
        int status = 2;  // not converged
        bool timed_out = false;

        while (it < P.maxit) {
            if (P.timeout_ns && (global_time_ns() - t_start) > P.timeout_ns) {
                timed_out = true;
                break;
            }
            // P1: p = r + beta p
            {
                const R br = (R)beta_re, bi = (R)beta_im;
                for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                    const C ri = r[i], pi = p[i];
                    p[i] = cmake<C>(ri.x + br * pi.x - bi * pi.y, ri.y + br * pi.y + bi * pi.x);
                }
            }
            __syncthreads();
            if (P.nonlocal) nonlocal_coeffs<R, C>(P, G, S, p);
            // P2: Ap = (H_R - z) p ; p^T Ap
            double pap[2];
            {
                R acc_re = 0, acc_im = 0;
                for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                    const int a = i % G.m[0];
                    const int b = (i / G.m[0]) % G.m[1];
                    const int c = i / (G.m[0] * G.m[1]);
                    const C y = apply_point<R, C, C>(P, G, S, p, i, a, b, c, z);
                    Ap[i] = y;
                    const C pi = p[i];
                    acc_re += pi.x * y.x - pi.y * y.y;
                    acc_im += pi.x * y.y + pi.y * y.x;
                }
                pap[0] = (double)acc_re;
                pap[1] = (double)acc_im;
                block_sum<2>(S, pap);
            }
            ++it;
            const double den = pap[0] * pap[0] + pap[1] * pap[1];
            if (!(den > 0.0)) {
                status = 3;
                break;
            }
            const double al_re = (rho_re * pap[0] + rho_im * pap[1]) / den;
            const double al_im = (rho_im * pap[0] - rho_re * pap[1]) / den;
            // P3: x += alpha p ; r -= alpha Ap ; r^T r ; |r|^2
            double red3[3];
            {
                const R ar = (R)al_re, ai = (R)al_im;
                R s_re = 0, s_im = 0, s_n = 0;
                for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                    const C pi = p[i], api = Ap[i];
                    if (Mode::kMixed) {
                        C d = dx[i];
                        d.x += ar * pi.x - ai * pi.y;
                        d.y += ar * pi.y + ai * pi.x;
                        dx[i] = d;
                    } else {
                        double2 xv = x[i];
                        xv.x += al_re * (double)pi.x - al_im * (double)pi.y;
                        xv.y += al_re * (double)pi.y + al_im * (double)pi.x;
                        x[i] = xv;
                    }
                    C ri = r[i];
                    ri.x -= ar * api.x - ai * api.y;
                    ri.y -= ar * api.y + ai * api.x;
                    r[i] = ri;
                    s_re += ri.x * ri.x - ri.y * ri.y;
                    s_im += 2 * ri.x * ri.y;
                    s_n += ri.x * ri.x + ri.y * ri.y;
                }
                red3[0] = (double)s_re;
                red3[1] = (double)s_im;
                red3[2] = (double)s_n;
                block_sum<3>(S, red3);
            }
            rn = sqrt(red3[2]);
            if (Mode::kMixed) {
                const bool want = (rn <= P.tol) || (it - last_rel >= P.reliable_every) ||
                                  (rn < P.reliable_delta * rn_last_rel);
                if (want) {
                    // flush dx into x_hi, then r = e_j - (H_R - z) x_hi in FP64
                    for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                        const C d = dx[i];
                        double2 xv = x[i];
                        xv.x += (double)d.x;
                        xv.y += (double)d.y;
                        x[i] = xv;
                        dx[i] = cmake<C>((R)0, (R)0);
                    }
                    __syncthreads();
                    if (P.nonlocal) nonlocal_coeffs<double, double2>(P, G, S, x);
                    double t3[3] = {0, 0, 0};
                    const double2 z64 = zd;
                    for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                        const int a = i % G.m[0];
                        const int b = (i / G.m[0]) % G.m[1];
                        const int c = i / (G.m[0] * G.m[1]);
                        const double2 y = apply_point<double, double2, double2>(P, G, S, x, i, a, b, c, z64);
                        const double tre = (i == G.src ? 1.0 : 0.0) - y.x;
                        const double tim = -y.y;
                        r[i] = cmake<C>((R)tre, (R)tim);
                        const R rr = (R)tre, ri = (R)tim;
                        t3[0] += (double)(rr * rr - ri * ri);
                        t3[1] += (double)(2 * rr * ri);
                        t3[2] += tre * tre + tim * tim;
                    }
                    block_sum<3>(S, t3);
                    red3[0] = t3[0];
                    red3[1] = t3[1];
                    rn = sqrt(t3[2]);
                    rn_last_rel = rn;
                    last_rel = it;
                    ++n_rel;
                }
            }
            if (rn <= P.tol) {
                status = 0;
                break;
            }
            const double rr_abs = sqrt(red3[0] * red3[0] + red3[1] * red3[1]);
            if (!(rr_abs > 1e-300) || rr_abs < 1e-14 * rn * rn) {
                status = 3;
                break;
            }
            const double rd = rho_re * rho_re + rho_im * rho_im;
            beta_re = (red3[0] * rho_re + red3[1] * rho_im) / rd;
            beta_im = (red3[1] * rho_re - red3[0] * rho_im) / rd;
            rho_re = red3[0];
            rho_im = red3[1];
        }
        if (Mode::kMixed && status != 0) {
            // leave x_hi consistent with the iterate reached
            for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                const C d = dx[i];
                double2 xv = x[i];
                xv.x += (double)d.x;
                xv.y += (double)d.y;
                x[i] = xv;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            P.x_src[out_idx] = x[G.src];
            P.status[out_idx] = timed_out ? 4 : (S.flag ? 1 : status);
            P.iters[out_idx] = it;
            P.resid[out_idx] = rn;
            P.n_rel[out_idx] = n_rel;
        }
        __syncthreads();
    }
}

// rho_j and e_j from the per-system x_jp(j), poles summed in a fixed order.
__global__ void k_accumulate(int n_nodes, int Pn, const double2* __restrict__ x_src,
                             const double2* __restrict__ z, const double2* __restrict__ w, double dV,
                             double* __restrict__ rho, double* __restrict__ e) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_nodes) return;
    double sr = 0.0, se = 0.0;
    for (int p = 0; p < Pn; ++p) {
        const double2 xv = x_src[(long long)j * Pn + p];
        const double2 ww = w[p], zz = z[p];
        // Im(w x)
        sr += ww.x * xv.y + ww.y * xv.x;
        // Im(w (1 + z x))
        const double zx_re = zz.x * xv.x - zz.y * xv.y;
        const double zx_im = zz.x * xv.y + zz.y * xv.x;
        se += ww.y + ww.x * zx_im + ww.y * zx_re;
    }
    rho[j] = (2.0 / dV) * sr;
    if (e) e[j] = 2.0 * se;
}

struct FP64Mode {
    using real = double;
    using cplx = double2;
    static constexpr bool kMixed = false;
};
struct MixedMode {
    using real = float;
    using cplx = float2;
    static constexpr bool kMixed = true;
};

}  // namespace

size_t slot_bytes_for(int precision, long long n_max) {
    const size_t nm = (size_t)((n_max + 63) / 64 * 64);
    if (precision == MD_PREC_MIXED) return nm * (4 * sizeof(float2) + sizeof(double2));
    return nm * (3 * sizeof(double2) + sizeof(double2));
}

cudaError_t launch_cocg(const SolveParams& P, int precision, int grid, int block, cudaStream_t stream) {
    if (precision == MD_PREC_MIXED) {
        k_cocg<MixedMode><<<grid, block, 0, stream>>>(P);
    } else {
        k_cocg<FP64Mode><<<grid, block, 0, stream>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_accumulate(int n_nodes, int Pn, const double2* x_src, const double2* z,
                              const double2* w, double dV, double* rho, double* e, cudaStream_t stream) {
    k_accumulate<<<(n_nodes + 127) / 128, 128, 0, stream>>>(n_nodes, Pn, x_src, z, w, dV, rho, e);
    return cudaGetLastError();
}

}  // namespace md
