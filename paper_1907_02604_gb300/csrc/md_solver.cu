// Batched COCG for the shifted systems (H_R(j) - z_p) x = e_j (md_density).
//
// One CTA owns one (node, pole) system at a time and takes the next one
// from a global work counter when it finishes (persistent scheduling over a
// cost-sorted list: largest regions and poles nearest the real axis
// first).  The Krylov vectors of the system live in a per-CTA slot of
// device scratch memory; the Hamiltonian (V, projector tables and
// per-point projector values) is shared by all systems and stays in L2.
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
//          the solution is x_hi (double) + dx (float, flushed into x_hi at
//          each residual refresh).  Products and each thread's partial sum
//          over its own points (at most a few dozen terms) are float;
//          everything from the per-thread partial upward (warp and block
//          reductions, alpha, beta, norms) is double.  A reliable update
//          (van der Vorst & Ye, SIAM J. Sci. Comput. 22, 2000) recomputes
//          the residual r = e_j - (H_R - z) x_hi in double every
//          `reliable_every` iterations, whenever ||r|| fell by
//          `reliable_delta` since the last one, and before convergence is
//          declared, so the returned solution meets tol on its FP64
//          residual.
#include <cuda_runtime.h>

#include <cstdint>

#include "md_operator.cuh"


namespace md {

namespace {

// Mixed mode: flush dx into x_hi, then r = e_j - (H_R - z) x_hi in FP64
// (a reliable update).  Rare, so kept out of line to spare registers in the
// iteration.  On return thread 0 holds r^T r (re, im) and ||r||^2 in t3.
template <class Mode, int Q>
__device__ __noinline__ void refresh_residual(const SolveParams& P, const Geo& G, Shared& S,
                                              typename Mode::cplx* r, typename Mode::cplx* dx,
                                              double2* x, double2 zd, double (&t3)[3]) {
    using R = typename Mode::real;
    using C = typename Mode::cplx;
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
    KSum<R> q_re, q_im;
    double nrm = 0.0;
    for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
        const double2 y = matvec_point<double, double2, Q, double2>(P, G, S, x, i, zd.x, zd.y, P.diag);
        const double tre = (i == G.src ? 1.0 : 0.0) - y.x;
        const double tim = -y.y;
        const C rr = cmake<C>((R)tre, (R)tim);
        r[i] = rr;
        if (P.multishift && i == G.src) S.rj = make_double2((double)rr.x, (double)rr.y);
        q_re.add(rr.x * rr.x - rr.y * rr.y);
        q_im.add(2 * rr.x * rr.y);
        nrm += tre * tre + tim * tim;
    }
    t3[0] = q_re.get();
    t3[1] = q_im.get();
    t3[2] = nrm;
    block_reduce<3>(S, t3);
}

// Shifted COCG: one step of the P pole recurrences (warp 0; lane k updates
// poles k, k+32, ...).  With sigma_k = z_seed - z_k the shifted residuals are
// r / pi_k (Jegerlehner 1996; Takayama et al. 2006 for COCG):
//   pi_{n+1} = (1 + a_n sigma) pi_n + (a_n b_{n-1}/a_{n-1}) (pi_n - pi_{n-1})
//   a_k = a_n pi_n/pi_{n+1},  b_k = (pi_n/pi_{n+1})^2 b_n
//   x_k(j) += a_k p_k(j),  p_k(j) = r(j)/pi_{n+1} + b_k p_k(j)
// Only the node's entries are tracked: the density needs x_k(j) alone.  A
// pole counts as converged once ||r|| / |pi_k| <= tol and is then frozen.
__device__ __noinline__ void shifted_update(const SolveParams& P, Shared& S) {

                    const double2 an = make_double2(S.alpha[0], S.alpha[1]);
                    const double2 bn = (S.action == kStop) ? make_double2(0.0, 0.0) : make_double2(S.beta[0], S.beta[1]);
                    const double2 ap = make_double2(S.alpha_prev[0], S.alpha_prev[1]);
                    const double2 bp = make_double2(S.beta_prev[0], S.beta_prev[1]);
                    const double2 c3 = zdiv(zmul(an, bp), ap);
                    const double2 zs = P.z[P.sys[S.sys].pole];
                    const double2 rj = S.rj;
                    bool all = true;
                    for (int k = threadIdx.x; k < P.P; k += 32) {
                        if (!S.sh_conv[k]) {
                            const double2 zk = P.z[k];
                            const double2 sg = make_double2(zs.x - zk.x, zs.y - zk.y);
                            const double2 pc = S.sh_pi[k], pp = S.sh_pi_prev[k];
                            const double2 t1 = zmul(make_double2(1.0 + (an.x * sg.x - an.y * sg.y), an.x * sg.y + an.y * sg.x), pc);
                            const double2 t2 = zmul(c3, make_double2(pc.x - pp.x, pc.y - pp.y));
                            const double2 pn = make_double2(t1.x + t2.x, t1.y + t2.y);
                            const double2 ratio = zdiv(pc, pn);
                            const double2 ak = zmul(an, ratio);
                            const double2 bk = zmul(zmul(ratio, ratio), bn);
                            const double2 xk = S.sh_x[k], pk = S.sh_p[k];
                            const double2 axp = zmul(ak, pk);
                            S.sh_x[k] = make_double2(xk.x + axp.x, xk.y + axp.y);
                            const double2 rq = zdiv(rj, pn), bpk = zmul(bk, pk);
                            S.sh_p[k] = make_double2(rq.x + bpk.x, rq.y + bpk.y);
                            S.sh_pi_prev[k] = pc;
                            S.sh_pi[k] = pn;
                            const double apn = sqrt(pn.x * pn.x + pn.y * pn.y);
                            if (S.rn <= P.tol * apn) S.sh_conv[k] = S.it;
                        }
                        all = all && (S.sh_conv[k] != 0);
                    }
                    all = __all_sync(0xffffffffu, all);
                    if (threadIdx.x == 0) {
                        S.alpha_prev[0] = an.x;
                        S.alpha_prev[1] = an.y;
                        S.beta_prev[0] = bn.x;
                        S.beta_prev[1] = bn.y;
                        if (all && S.action != kStop) {
                            S.st = 0;
                            S.action = kStop;
                        }
                        if (S.action == kStop && S.st != 0 && all) S.st = 0;
                    }
                }

// kMinB = 1: up to 1,024 threads, 64 registers; kMinB = 3: 512 threads and
// 40 registers, so that three CTAs (three systems) share an SM; the loop is
// latency-bound and the extra resident warps hide more of it.
template <class Mode, int Q, int kMinB>
__global__ void __launch_bounds__(kMinB == 1 ? 1024 : 512, kMinB) k_cocg(const __grid_constant__ SolveParams P) {
    using R = typename Mode::real;
    using C = typename Mode::cplx;
    __shared__ Shared S;
    const uint64_t t_start = global_time_ns();
    char* slot = P.scratch + (size_t)blockIdx.x * P.slot_bytes;
    for (int t = threadIdx.x; t < 3 * kMaxQ; t += blockDim.x) {
        (&S.coefD[0][0])[t] = (&P.coef[0][0])[t];
        (&S.coefF[0][0])[t] = (float)(&P.coef[0][0])[t];
    }
    if (P.nonlocal && P.n_atoms <= kMapMax)
        for (int t = threadIdx.x; t < P.n_atoms; t += blockDim.x) S.map[t] = -1;
    const R diagR = (R)P.diag;

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
        const double2 zd = P.z[sd.pole];
        const R zr = (R)zd.x, zi = (R)zd.y;
        const long long out_idx = (long long)sd.node * P.P + sd.pole;

        C* r = (C*)slot;
        C* p = r + P.n_max;
        C* Ap = p + P.n_max;
        C* dx = Ap + P.n_max;                       // mixed only
        double2* x = (double2*)(dx + (Mode::kMixed ? P.n_max : 0));
        if (P.ckpt) x = P.ckpt + P.ckpt_sys_off[out_idx];

        if (P.nonlocal) collect_local_atoms(P, G, S);
        if (Mode::kMixed && P.nonlocal) {   // point records after the vectors
            uint2* rec = reinterpret_cast<uint2*>(reinterpret_cast<double2*>(dx + P.n_max) + P.n_max);
            build_nl_records(P, G, S, rec);
            G.nl_rec = rec;
        }
        if (P.multishift)
            for (int k = threadIdx.x; k < P.P; k += blockDim.x) {
                S.sh_pi_prev[k] = make_double2(1.0, 0.0);
                S.sh_pi[k] = make_double2(1.0, 0.0);
                S.sh_x[k] = make_double2(0.0, 0.0);
                S.sh_p[k] = make_double2(1.0, 0.0);   // p_0 = b, b(j) = 1
                S.sh_conv[k] = 0;
            }

        for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
            r[i] = cmake<C>((R)(i == G.src ? 1 : 0), (R)0);
            p[i] = cmake<C>((R)0, (R)0);
            x[i] = make_double2(0.0, 0.0);
            if (Mode::kMixed) dx[i] = cmake<C>((R)0, (R)0);
        }
        __syncthreads();

        // Scalar state lives in thread 0; the others see it through S.
        if (threadIdx.x == 0) {
            S.beta[0] = 0.0;
            S.beta[1] = 0.0;
            S.action = 0;
            S.rho[0] = 1.0;
            S.rho[1] = 0.0;
            S.rn = 1.0;
            S.rn_last = 1.0;
            S.it = 0;
            S.last_rel = 0;
            S.n_rel = 0;
            S.restart = 0;
            S.st = 2;   // not converged
            S.alpha_prev[0] = 1.0;
            S.alpha_prev[1] = 0.0;
            S.beta_prev[0] = 0.0;
            S.beta_prev[1] = 0.0;
            S.all_conv = 0;
        }
        __syncthreads();

        for (;;) {
            if (P.timeout_ns && threadIdx.x == 0 && (global_time_ns() - t_start) > P.timeout_ns)
                S.action = kStopTimeout;
            if (threadIdx.x == 0 && S.it >= P.maxit) S.action = kStop;
            __syncthreads();
            if (S.action == kStop || S.action == kStopTimeout) break;
            {   // P1: p = r + beta p
                const R br = (R)S.beta[0], bi = (R)S.beta[1];
                if constexpr (Mode::kMixed) {
                    // two complex64 per 16-byte access (slots are 512-byte aligned)
                    const float4* r4 = reinterpret_cast<const float4*>(r);
                    float4* p4 = reinterpret_cast<float4*>(p);
                    const int npair = G.n >> 1;
                    const uint64_t pol = l2_evict_first_policy();
                    for (int k = threadIdx.x; k < npair; k += blockDim.x) {
                        const float4 a = ld_stream(r4 + k, pol), b = ld_stream(p4 + k, pol);
                        // the new direction keeps the default priority: the next two passes re-read it
                        p4[k] = make_float4(a.x + br * b.x - bi * b.y, a.y + br * b.y + bi * b.x,
                                            a.z + br * b.z - bi * b.w, a.w + br * b.w + bi * b.z);
                    }
                    if ((G.n & 1) && threadIdx.x == 0) {
                        const int i = G.n - 1;
                        const C ri = r[i], pi = p[i];
                        p[i] = cmake<C>(ri.x + br * pi.x - bi * pi.y, ri.y + br * pi.y + bi * pi.x);
                    }
                } else {
                    for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                        const C ri = r[i], pi = p[i];
                        p[i] = cmake<C>(ri.x + br * pi.x - bi * pi.y, ri.y + br * pi.y + bi * pi.x);
                    }
                }
            }
            __syncthreads();
            if (P.nonlocal) nonlocal_coeffs<R, C>(P, G, S, p);
            {   // P2: Ap = (H_R - z) p ; p^T Ap
                KSum<R> acc_re, acc_im;
                // each point's projector record is loaded one point ahead
                const bool pre = Mode::kMixed && P.nonlocal && G.nl_rec;
                const uint64_t pol = l2_evict_first_policy();
                uint2 rc_next = make_uint2(0u, 0xFFFFFFFFu);
                if (pre && threadIdx.x < G.n) rc_next = ld_stream(G.nl_rec + threadIdx.x, pol);
                for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                    const uint2 rc = rc_next;
                    if (pre && i + (int)blockDim.x < G.n) rc_next = ld_stream(G.nl_rec + i + blockDim.x, pol);
                    const C y = matvec_point<R, C, Q, C>(P, G, S, p, i, zr, zi, diagR,
                                                         pre ? rc : make_uint2(0u, 0xFFFFFFFEu));
                    if constexpr (Mode::kMixed) st_stream(reinterpret_cast<float2*>(Ap + i), y, pol);
                    else Ap[i] = y;
                    const C pi = p[i];
                    acc_re.add(pi.x * y.x - pi.y * y.y);
                    acc_im.add(pi.x * y.y + pi.y * y.x);
                }
                double pap[2];
                if constexpr (Mode::kMixed) {
                    const float hi[2] = {acc_re.hi(), acc_im.hi()}, lo[2] = {acc_re.lo(), acc_im.lo()};
                    block_reduce_ff<2>(S, hi, lo, pap);
                } else {
                    pap[0] = acc_re.get();
                    pap[1] = acc_im.get();
                    block_reduce<2>(S, pap);
                }
                if (threadIdx.x == 0) {
                    ++S.it;
                    const double den = pap[0] * pap[0] + pap[1] * pap[1];
                    if (!(den > 0.0)) {
                        S.st = 3;
                        S.action = kStop;
                    } else {
                        S.alpha[0] = (S.rho[0] * pap[0] + S.rho[1] * pap[1]) / den;
                        S.alpha[1] = (S.rho[1] * pap[0] - S.rho[0] * pap[1]) / den;
                    }
                }
                __syncthreads();
                if (S.action == kStop) break;
            }
            double red3[3];
            {   // P3: x += alpha p ; r -= alpha Ap ; r^T r ; |r|^2
                const double al_re = S.alpha[0], al_im = S.alpha[1];
                const R ar = (R)al_re, ai = (R)al_im;
                KSum<R> s_re, s_im, s_n;
                if constexpr (Mode::kMixed) {
                    const float4* p4 = reinterpret_cast<const float4*>(p);
                    const float4* q4 = reinterpret_cast<const float4*>(Ap);
                    float4* d4 = reinterpret_cast<float4*>(dx);
                    float4* r4 = reinterpret_cast<float4*>(r);
                    const int npair = G.n >> 1;
                    const uint64_t pol = l2_evict_first_policy();
                    for (int k = threadIdx.x; k < npair; k += blockDim.x) {
                        const float4 pv = ld_stream(p4 + k, pol), qv = ld_stream(q4 + k, pol);
                        float4 d = ld_stream(d4 + k, pol), rv = ld_stream(r4 + k, pol);
                        d.x += ar * pv.x - ai * pv.y;
                        d.y += ar * pv.y + ai * pv.x;
                        d.z += ar * pv.z - ai * pv.w;
                        d.w += ar * pv.w + ai * pv.z;
                        rv.x -= ar * qv.x - ai * qv.y;
                        rv.y -= ar * qv.y + ai * qv.x;
                        rv.z -= ar * qv.z - ai * qv.w;
                        rv.w -= ar * qv.w + ai * qv.z;
                        st_stream(d4 + k, d, pol);
                        st_stream(r4 + k, rv, pol);
                        if (P.multishift && (G.src >> 1) == k)
                            S.rj = (G.src & 1) ? make_double2(rv.z, rv.w) : make_double2(rv.x, rv.y);
                        s_re.add(rv.x * rv.x - rv.y * rv.y + (rv.z * rv.z - rv.w * rv.w));
                        s_im.add(2.f * (rv.x * rv.y + rv.z * rv.w));
                        s_n.add(rv.x * rv.x + rv.y * rv.y + (rv.z * rv.z + rv.w * rv.w));
                    }
                    if ((G.n & 1) && threadIdx.x == 0) {
                        const int i = G.n - 1;
                        const C pi = p[i], api = Ap[i];
                        C d = dx[i], ri = r[i];
                        d.x += ar * pi.x - ai * pi.y;
                        d.y += ar * pi.y + ai * pi.x;
                        ri.x -= ar * api.x - ai * api.y;
                        ri.y -= ar * api.y + ai * api.x;
                        dx[i] = d;
                        r[i] = ri;
                        if (P.multishift && i == G.src) S.rj = make_double2(ri.x, ri.y);
                        s_re.add(ri.x * ri.x - ri.y * ri.y);
                        s_im.add(2.f * ri.x * ri.y);
                        s_n.add(ri.x * ri.x + ri.y * ri.y);
                    }
                } else {
                    for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                        const C pi = p[i], api = Ap[i];
                        double2 xv = x[i];
                        xv.x += al_re * (double)pi.x - al_im * (double)pi.y;
                        xv.y += al_re * (double)pi.y + al_im * (double)pi.x;
                        x[i] = xv;
                        C ri = r[i];
                        ri.x -= ar * api.x - ai * api.y;
                        ri.y -= ar * api.y + ai * api.x;
                        r[i] = ri;
                        if (P.multishift && i == G.src) S.rj = make_double2((double)ri.x, (double)ri.y);
                        s_re.add(ri.x * ri.x - ri.y * ri.y);
                        s_im.add(2 * ri.x * ri.y);
                        s_n.add(ri.x * ri.x + ri.y * ri.y);
                    }
                }
                if constexpr (Mode::kMixed) {
                    const float hi[3] = {s_re.hi(), s_im.hi(), s_n.hi()};
                    const float lo[3] = {s_re.lo(), s_im.lo(), s_n.lo()};
                    block_reduce_ff<3>(S, hi, lo, red3);
                } else {
                    red3[0] = s_re.get();
                    red3[1] = s_im.get();
                    red3[2] = s_n.get();
                    block_reduce<3>(S, red3);
                }
            }
            if (Mode::kMixed) {
                if (threadIdx.x == 0) {
                    const double rn = sqrt(red3[2]);
                    const bool want = (rn <= P.tol) || (S.it - S.last_rel >= P.reliable_every) ||
                                      (rn < P.reliable_delta * S.rn_last);
                    S.action = want ? kRefresh : 0;
                }
                __syncthreads();
                if (S.action == kRefresh) {
                    refresh_residual<Mode, Q>(P, G, S, r, dx, x, zd, red3);
                    if (threadIdx.x == 0) {
                        const double rt = sqrt(red3[2]);
                        // no progress since the previous refresh: restart (p = r next)
                        S.restart = (S.n_rel > 0 && rt >= S.rn_last) ? 1 : 0;
                        S.rn_last = rt;
                        S.last_rel = S.it;
                        ++S.n_rel;
                    }
                }
            }
            if (threadIdx.x == 0) {
                const double rn = sqrt(red3[2]);
                S.rn = rn;
                S.action = 0;
                const double rr_abs = sqrt(red3[0] * red3[0] + red3[1] * red3[1]);
                if (rn <= P.tol && !P.multishift) {
                    S.st = 0;
                    S.action = kStop;
                } else if (!(rr_abs > 1e-300) || rr_abs < 1e-14 * rn * rn) {
                    if (rn <= P.tol) {
                        S.st = 0;   // converged exactly: no further direction needed
                    } else {
                        S.st = 3;
                    }
                    S.action = kStop;
                } else {
                    const double rd = S.rho[0] * S.rho[0] + S.rho[1] * S.rho[1];
                    S.beta[0] = S.restart ? 0.0 : (red3[0] * S.rho[0] + red3[1] * S.rho[1]) / rd;
                    S.beta[1] = S.restart ? 0.0 : (red3[1] * S.rho[0] - red3[0] * S.rho[1]) / rd;
                    S.rho[0] = red3[0];
                    S.rho[1] = red3[1];
                }
                S.restart = 0;
            }
            __syncthreads();
            if (P.multishift) {   // shifted systems share the seed's Krylov space
                if (threadIdx.x < 32) shifted_update(P, S);
                __syncthreads();
            }
            if (S.action == kStop) break;
        }
        const bool timed_out = (S.action == kStopTimeout);
        __syncthreads();
        const int status = S.st;
        if (Mode::kMixed && status != 0) {
            for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                const C d = dx[i];
                double2 xv = x[i];
                xv.x += (double)d.x;
                xv.y += (double)d.y;
                x[i] = xv;
            }
        }
        __syncthreads();
        if (P.fused_dLdV) {
            // this system's share of dL/dV (the forward solution is the adjoint one)
            const double aj = P.fused_a ? P.fused_a[sd.node] : 0.0;
            const double bj = P.fused_b ? P.fused_b[sd.node] : 0.0;
            const double2 wp = P.w[sd.pole];
            const double cr = 2.0 * aj / P.dV + 2.0 * bj * zd.x, ci = 2.0 * bj * zd.y;
            const double c_re = cr * wp.x - ci * wp.y, c_im = cr * wp.y + ci * wp.x;
            for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                const int c = (int)fdiv((uint32_t)i, G.div_plane);
                const int rem = i - c * G.plane;
                const int b = (int)fdiv((uint32_t)rem, G.div_row);
                const int a = rem - b * G.m[0];
                const int gx = wrap_once(G.lo[0] + a, P.n[0]);
                const int gy = wrap_once(G.lo[1] + b, P.n[1]);
                const int gz = wrap_once(G.lo[2] + c, P.n[2]);
                const long long gi = gx + (long long)P.n[0] * (gy + (long long)P.n[1] * gz);
                const double2 xv = x[i];
                const double sq_re = xv.x * xv.x - xv.y * xv.y, sq_im = 2.0 * xv.x * xv.y;
                atomicAdd(P.fused_dLdV + gi, -(c_re * sq_im + c_im * sq_re));
            }
        }
        if (P.dm_rows) {
            // row j of the density matrix over the region: sum_p Im(w_p x_jp(k))
            const double2 wp = P.w[sd.pole];
            double* row = P.dm_rows + P.dm_off[sd.node];
            for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
                const double2 xv = x[i];
                atomicAdd(row + i, wp.x * xv.y + wp.y * xv.x);
            }
        }
        if (P.multishift) {
            for (int k = threadIdx.x; k < P.P; k += blockDim.x) {
                const long long o = (long long)sd.node * P.P + k;
                const double2 pk = S.sh_pi[k];
                P.x_src[o] = S.sh_x[k];
                P.status[o] = timed_out ? 4 : (S.flag ? 1 : (S.sh_conv[k] ? 0 : (status == 3 ? 3 : 2)));
                P.iters[o] = S.sh_conv[k] ? S.sh_conv[k] : S.it;
                P.resid[o] = S.rn / sqrt(pk.x * pk.x + pk.y * pk.y);
                P.n_rel[o] = (k == sd.pole) ? S.n_rel : 0;
            }
        } else if (threadIdx.x == 0) {
            P.x_src[out_idx] = x[G.src];
            P.status[out_idx] = timed_out ? 4 : (S.flag ? 1 : status);
            P.iters[out_idx] = S.it;
            P.resid[out_idx] = S.rn;
            P.n_rel[out_idx] = S.n_rel;
        }
        if (P.nonlocal) release_local_atoms(P, S);
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
        sr += ww.x * xv.y + ww.y * xv.x;                       // Im(w x)
        const double zx_re = zz.x * xv.x - zz.y * xv.y;
        const double zx_im = zz.x * xv.y + zz.y * xv.x;
        se += ww.y + ww.x * zx_im + ww.y * zx_re;              // Im(w (1 + z x))
    }
    rho[j] = (2.0 / dV) * sr;
    if (e) e[j] = 2.0 * se;
}


template <int K>
struct ZmThreads {
    static constexpr int value = K == 1 ? 1024 : (K == 2 ? 576 : (K == 3 ? 384 : 288));
};

constexpr int kStages = 4;               // staging slots: planes prefetched 3 ahead
constexpr uint32_t kWaitLimit = 1u << 22;

// Dynamic shared memory of the z-march kernel for launch-wide maximal
// region extents M0 x M1 (the same arithmetic on host and device).
struct ZmLayout {
    size_t cacc_off, plane_off, nl_off, stage_off, stage_bytes, total;
    __host__ __device__ ZmLayout(int q, int M0, int M1) {
        const size_t pb = (size_t)(M0 + 2 * q) * (size_t)(M1 + 2 * q);   // bordered plane
        const size_t pl = (size_t)M0 * (size_t)M1;
        cacc_off = 0;                                                       // float [kLocal][8]
        plane_off = (size_t)kLocal * 8 * sizeof(float);
        nl_off = plane_off + 2 * pb * sizeof(float2);
        stage_bytes = (pl * sizeof(float2) + 16 + 15) / 16 * 16;          // one staged plane
        stage_off = (nl_off + 2 * pl * sizeof(float2) + 127) / 128 * 128;
        total = stage_off + (size_t)kStages * 2 * stage_bytes;
    }
};

// Window index of region slot c for an atom window starting at region
// offset off (inverse of region_slot); -1 if the window misses it.
__device__ __forceinline__ int window_index(int off, int c, int n, int len, int periodic) {
    int w = c - off;
    if (periodic && w < 0) w += n;
    return (w >= 0 && w < len) ? w : -1;
}

// Issue the bulk copies of plane `cn` of r and p into staging slot cn % kStages.
__device__ __forceinline__ void zm_issue(const SolveParams& P, const Geo& G, unsigned char* stage,
                                         size_t stage_bytes, uint64_t* bars, const float2* r,
                                         const float2* p, int cn) {
    const int slot = cn % kStages;
    const uintptr_t sr = (uintptr_t)(r + (size_t)cn * G.plane);
    const uintptr_t sp = (uintptr_t)(p + (size_t)cn * G.plane);
    const uintptr_t ar = sr & ~(uintptr_t)15, ap = sp & ~(uintptr_t)15;
    const uint32_t br = (uint32_t)(((sr + (uintptr_t)G.plane * 8 + 15) & ~(uintptr_t)15) - ar);
    const uint32_t bp = (uint32_t)(((sp + (uintptr_t)G.plane * 8 + 15) & ~(uintptr_t)15) - ap);
    unsigned char* dst = stage + (size_t)slot * 2 * stage_bytes;
    fence_proxy_async();
    mbar_arrive_expect_tx(&bars[slot], br + bp);
    bulk_copy_g2s(dst, (const void*)ar, br, &bars[slot]);
    bulk_copy_g2s(dst + stage_bytes, (const void*)ap, bp, &bars[slot]);
}

// Projections of the published plane c (bordered buffer, row pitch `pitch`,
// border width q) onto the local projectors, added into cacc[k][8]: warp per
// local atom, lane per row of the disk where its sphere cuts the plane.
__device__ __noinline__ void zm_nl_dot_plane(const SolveParams& P, const Geo& G, Shared& S,
                                             const float2* __restrict__ buf, int pitch, int Q, int c,
                                             float* __restrict__ cacc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m0 = G.m[0], m1 = G.m[1];
            for (int kk = warp; kk < S.n_local; kk += nw) {
                const int at = S.la_id[kk];
                const int lz = __ldg(P.proj_len + 3 * at + 2);
                const int ww = window_index(S.la_off[kk][2], c, P.n[2], lz, P.periodic[2]);
                if (ww < 0) continue;
                const int lx = __ldg(P.proj_len + 3 * at), ly = __ldg(P.proj_len + 3 * at + 1);
                const float* dxt = P.proj_d32 + (3LL * at + 0) * kMaxProjWin;
                const float* gxt = P.proj_g32 + (3LL * at + 0) * kMaxProjWin;
                const Runs rx = axis_runs(S.la_off[kk][0], lx, P.n[0], m0, P.periodic[0]);
                const unsigned char* rows = P.proj_rows + 2 * (((long long)at * kMaxProjWin + ww) * kMaxProjWin);
                const float gz = __ldg(P.proj_g32 + (3LL * at + 2) * kMaxProjWin + ww);
                const float dz = __ldg(P.proj_d32 + (3LL * at + 2) * kMaxProjWin + ww);
                float acc8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                for (int vv2 = lane; vv2 < ly; vv2 += 32) {
                    const int b = region_slot(S.la_off[kk][1], vv2, P.n[1], m1, P.periodic[1]);
                    if (b < 0) continue;
                    const int u0 = rows[2 * vv2], u1 = rows[2 * vv2 + 1];
                    const float2* brow = buf + (b + Q) * pitch + Q;
                    float Ar = 0.f, Ai = 0.f, Br = 0.f, Bi = 0.f;
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const int lo = max(u0, rx.lo[t]), hi = min(u1, rx.hi[t]);
                        for (int u = lo; u <= hi; ++u) {
                            const float2 pv = brow[u + rx.shift[t]];
                            const float g1 = __ldg(gxt + u);
                            const float g2 = __ldg(dxt + u) * g1;
                            Ar += g1 * pv.x; Ai += g1 * pv.y;
                            Br += g2 * pv.x; Bi += g2 * pv.y;
                        }
                    }
                    const float gyz = __ldg(P.proj_g32 + (3LL * at + 1) * kMaxProjWin + vv2) * gz;
                    const float ey = __ldg(P.proj_d32 + (3LL * at + 1) * kMaxProjWin + vv2) * gyz;
                    const float ez = dz * gyz;
                    acc8[0] += gyz * Ar; acc8[1] += gyz * Ai;
                    acc8[2] += gyz * Br; acc8[3] += gyz * Bi;
                    acc8[4] += ey * Ar;  acc8[5] += ey * Ai;
                    acc8[6] += ez * Ar;  acc8[7] += ez * Ai;
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float v = warp_sum(acc8[t]);
                    if (lane == 0) atomicAdd(&cacc[kk * 8 + t], v);
                }
            }
        }

// Fused P1 + local P2 of the mixed iteration, staged through shared memory.
// Each thread owns K (x, y) columns of the region and walks z; the 2Q+1
// values of p_new along a column sit in registers (the z part of the
// stencil), and the current plane is published in a zero-bordered buffer
// for the x and y neighbours (two buffers alternate: one barrier per
// plane).  The r and p_old planes the window needs next arrive by bulk
// asynchronous copies three planes ahead (mbarrier completion), so HBM
// latency is off the critical path.  While a plane is published, warps
// also accumulate the nonlocal coefficients c_al over the disk where each
// local atom's projector sphere cuts that plane (separable Gaussian: per
// row A = sum g_x v, B = sum d_x g_x v).  Outputs: p (new), Ap_loc =
// (-1/2 L + V - z) p, cacc (raw projections), the thread's p^T Ap_loc.
template <int Q, int K>
__device__ __forceinline__ void zm_stencil_pass(const SolveParams& P, const Geo& G, Shared& S,
                                                unsigned char* dsm, const ZmLayout& L, uint32_t& ph,
                                                const float2* __restrict__ r, float2* __restrict__ p,
                                                float2* __restrict__ Ap, float br, float bi, float zr,
                                                float zi, float diag, KSum<float>& acc_re,
                                                KSum<float>& acc_im) {
    const int T = blockDim.x;
    const int m0 = G.m[0], m1 = G.m[1], m2 = G.m[2], plane = G.plane;
    const int pitch = m0 + 2 * Q;
    const int bufsz = pitch * (m1 + 2 * Q);
    const long long nxy = (long long)P.n[0] * P.n[1];
    const float* cf = coef_of<float>(S);
    float2* pbuf = reinterpret_cast<float2*>(dsm + L.plane_off);
    float* cacc = reinterpret_cast<float*>(dsm + L.cacc_off);
    unsigned char* stage = dsm + L.stage_off;
    // staging offset (elements) of the plane start inside a 16-byte aligned copy
    const int soff = (int)((((uintptr_t)r) & 15) / 8);   // r and p share the residue per plane parity
    int col[K], sidx[K];
    long long vbase[K];
    bool ok[K];
    float2 win[K][2 * Q + 1];
    if (P.nonlocal)
        for (int t = threadIdx.x; t < S.n_local * 8; t += T) cacc[t] = 0.f;
    if (threadIdx.x == 0)
        for (int cn = Q + 1; cn < m2 && cn <= Q + kStages - 1; ++cn) zm_issue(P, G, stage, L.stage_bytes, S.bar, r, p, cn);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        col[k] = threadIdx.x + k * T;
        ok[k] = col[k] < plane;
        const int cc = ok[k] ? col[k] : 0;
        const int b = (int)fdiv((uint32_t)cc, G.div_row);
        const int a = cc - b * m0;
        sidx[k] = (b + Q) * pitch + (a + Q);
        vbase[k] = wrap_once(G.lo[0] + a, P.n[0]) + (long long)P.n[0] * wrap_once(G.lo[1] + b, P.n[1]);
#pragma unroll
        for (int t = 0; t <= 2 * Q; ++t) {
            const int c = t - Q;
            float2 v = make_float2(0.f, 0.f);
            if (ok[k] && c >= 0 && c < m2) {
                const int idx = col[k] + c * plane;
                const float2 rv = r[idx], pv = p[idx];
                v = make_float2(rv.x + br * pv.x - bi * pv.y, rv.y + br * pv.y + bi * pv.x);
                p[idx] = v;
            }
            win[k][t] = v;
        }
    }
    for (int c = 0; c < m2; ++c) {
        float2* buf = pbuf + (c & 1) * bufsz;
        const int cn = c + Q + 1;
        const long long voff = nxy * wrap_once(G.lo[2] + c, P.n[2]);
        float2 nr[K], np[K];
        float vv[K];
        if (cn < m2) {
            const int slot = cn % kStages;
            if (!mbar_wait_bounded(&S.bar[slot], (ph >> slot) & 1u, kWaitLimit)) S.flag = 2;
            ph ^= 1u << slot;
        }
        const float2* sr = reinterpret_cast<const float2*>(stage + (size_t)(cn % kStages) * 2 * L.stage_bytes);
        const float2* sp = reinterpret_cast<const float2*>(stage + (size_t)(cn % kStages) * 2 * L.stage_bytes +
                                                           L.stage_bytes);
        const int so = (int)(((((uintptr_t)r) + (uintptr_t)cn * plane * 8) & 15) / 8);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            nr[k] = make_float2(0.f, 0.f);
            np[k] = make_float2(0.f, 0.f);
            vv[k] = 0.f;
            if (ok[k]) {
                vv[k] = __ldg(P.V32 + vbase[k] + voff);
                if (cn < m2) {
                    nr[k] = sr[so + col[k]];
                    np[k] = sp[so + col[k]];
                }
                buf[sidx[k]] = win[k][Q];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && cn + kStages - 1 < m2)
            zm_issue(P, G, stage, L.stage_bytes, S.bar, r, p, cn + kStages - 1);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (ok[k]) {
                const float2 ctr = win[k][Q];
                const float dg = diag + vv[k] - zr;
                float yx = dg * ctr.x + zi * ctr.y;
                float yy = dg * ctr.y - zi * ctr.x;
                const float2* bp = buf + sidx[k];
#pragma unroll
                for (int o = 1; o <= Q; ++o) {
                    const float wx = cf[0 * kMaxQ + o - 1], wy = cf[1 * kMaxQ + o - 1], wz = cf[2 * kMaxQ + o - 1];
                    const float2 xp = bp[o], xm = bp[-o];
                    const float2 yp = bp[o * pitch], ym = bp[-o * pitch];
                    const float2 zp = win[k][Q + o], zm = win[k][Q - o];
                    yx += wx * (xp.x + xm.x) + wy * (yp.x + ym.x) + wz * (zp.x + zm.x);
                    yy += wx * (xp.y + xm.y) + wy * (yp.y + ym.y) + wz * (zp.y + zm.y);
                }
                Ap[col[k] + c * plane] = make_float2(yx, yy);
                acc_re.add(ctr.x * yx - ctr.y * yy);
                acc_im.add(ctr.x * yy + ctr.y * yx);
            }
        }
        if (P.nonlocal) zm_nl_dot_plane(P, G, S, buf, pitch, Q, c, cacc);
#pragma unroll
        for (int k = 0; k < K; ++k) {
#pragma unroll
            for (int t = 0; t < 2 * Q; ++t) win[k][t] = win[k][t + 1];
            float2 v = make_float2(0.f, 0.f);
            if (ok[k] && cn < m2) {
                v = make_float2(nr[k].x + br * np[k].x - bi * np[k].y, nr[k].y + br * np[k].y + bi * np[k].x);
                p[col[k] + cn * plane] = v;
            }
            win[k][2 * Q] = v;
        }
    }
    (void)soff;
}

// Nonlocal contribution of plane c, accumulated atom by atom into the plane
// buffer nl (m0 x m1, shared memory) with shared-memory atomics:
//   nl(i) += sum_l C_l f_l(i) (E_l dV c_al),  f = (1, d_x, d_y, d_z) g_x g_y g_z.
__device__ __noinline__ void zm_nl_plane(const SolveParams& P, const Geo& G, const Shared& S,
                                            float2* nl, int c) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m0 = G.m[0], m1 = G.m[1];
    for (int kk = warp; kk < S.n_local; kk += nw) {
        const int at = S.la_id[kk];
        const int lz = __ldg(P.proj_len + 3 * at + 2);
        const int ww = window_index(S.la_off[kk][2], c, P.n[2], lz, P.periodic[2]);
        if (ww < 0) continue;
        const int lx = __ldg(P.proj_len + 3 * at), ly = __ldg(P.proj_len + 3 * at + 1);
        const float* dxt = P.proj_d32 + (3LL * at + 0) * kMaxProjWin;
        const float* gxt = P.proj_g32 + (3LL * at + 0) * kMaxProjWin;
        const Runs rx = axis_runs(S.la_off[kk][0], lx, P.n[0], m0, P.periodic[0]);
        const unsigned char* rows = P.proj_rows + 2 * (((long long)at * kMaxProjWin + ww) * kMaxProjWin);
        const float gz = __ldg(P.proj_g32 + (3LL * at + 2) * kMaxProjWin + ww);
        const float dz = __ldg(P.proj_d32 + (3LL * at + 2) * kMaxProjWin + ww);
        const float C0 = __ldg(P.proj_C32 + 4LL * at), C1 = __ldg(P.proj_C32 + 4LL * at + 1),
                    C2 = __ldg(P.proj_C32 + 4LL * at + 2), C3 = __ldg(P.proj_C32 + 4LL * at + 3);
        const float2 c0 = S.cf[kk][0], c1 = S.cf[kk][1], c2 = S.cf[kk][2], c3 = S.cf[kk][3];
        // per-atom constant parts: K1 = C_s c_s + d_y C_y c_y + d_z C_z c_z (row-wise), K2 = C_x c_x
        for (int vv2 = lane; vv2 < ly; vv2 += 32) {
            const int b = region_slot(S.la_off[kk][1], vv2, P.n[1], m1, P.periodic[1]);
            if (b < 0) continue;
            const int u0 = rows[2 * vv2], u1 = rows[2 * vv2 + 1];
            const float gyz = __ldg(P.proj_g32 + (3LL * at + 1) * kMaxProjWin + vv2) * gz;
            const float dy = __ldg(P.proj_d32 + (3LL * at + 1) * kMaxProjWin + vv2);
            const float k1r = gyz * (C0 * c0.x + dy * C2 * c2.x + dz * C3 * c3.x);
            const float k1i = gyz * (C0 * c0.y + dy * C2 * c2.y + dz * C3 * c3.y);
            const float k2r = gyz * C1 * c1.x, k2i = gyz * C1 * c1.y;
            float2* nrow = nl + b * m0;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int lo = max(u0, rx.lo[t]), hi = min(u1, rx.hi[t]);
                for (int u = lo; u <= hi; ++u) {
                    const float g1 = __ldg(gxt + u);
                    const float g2 = __ldg(dxt + u) * g1;
                    float2* dst = nrow + u + rx.shift[t];
                    atomicAdd(&dst->x, g1 * k1r + g2 * k2r);
                    atomicAdd(&dst->y, g1 * k1i + g2 * k2i);
                }
            }
        }
    }
}

// Mixed-precision persistent COCG with the shared-memory z-march stencil
// (regions without whole-axis rings; stencil half-width Q; K columns per
// thread, blockDim.x * K >= m0 * m1 for every region of the launch).
// The nonlocal term enters through the bilinear identity
//   p^T A p = p^T A_loc p + sum_al E_l dV c_al^2
// and is added to Ap plane by plane in P3 from a shared-memory buffer.
template <int Q, int K>
__global__ void __launch_bounds__(ZmThreads<K>::value) k_cocg_zm(const __grid_constant__ SolveParams P) {
    using Mode = MixedModeT;
    using C = float2;
    __shared__ Shared S;
    extern __shared__ __align__(128) unsigned char dsm[];
    const ZmLayout L(Q, P.zm_m0, P.zm_m1);
    const uint64_t t_start = global_time_ns();
    char* slot = P.scratch + (size_t)blockIdx.x * P.slot_bytes;
    for (int t = threadIdx.x; t < 3 * kMaxQ; t += blockDim.x) {
        (&S.coefD[0][0])[t] = (&P.coef[0][0])[t];
        (&S.coefF[0][0])[t] = (float)(&P.coef[0][0])[t];
    }
    if (P.nonlocal && P.n_atoms <= kMapMax)
        for (int t = threadIdx.x; t < P.n_atoms; t += blockDim.x) S.map[t] = -1;
    if (threadIdx.x < 32) S.pnl[threadIdx.x] = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        for (int k = 0; k < kStages; ++k) mbar_init(&S.bar[k], 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t ph = 0;   // parity of the next wait on each staging slot
    const float diagF = (float)P.diag;
    float2* nlbuf = reinterpret_cast<float2*>(dsm + L.nl_off);

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
        Geo G;
        G.any_ring = 0;
        for (int d = 0; d < 3; ++d) {
            G.m[d] = nd.dims[d];
            G.lo[d] = nd.lo[d];
            G.ring[d] = 0;
        }
        G.plane = G.m[0] * G.m[1];
        G.n = G.plane * G.m[2];
        G.src = nd.src;
        G.div_row = make_fastdiv((uint32_t)G.m[0]);
        G.div_plane = make_fastdiv((uint32_t)G.plane);
        const double2 zd = P.z[sd.pole];
        const float zr = (float)zd.x, zi = (float)zd.y;
        const long long out_idx = (long long)sd.node * P.P + sd.pole;

        C* r = (C*)slot;
        C* p = r + P.n_max;
        C* Ap = p + P.n_max;
        C* dx = Ap + P.n_max;
        double2* x = (double2*)(dx + P.n_max);
        if (P.ckpt) x = P.ckpt + P.ckpt_sys_off[out_idx];

        if (P.nonlocal) collect_local_atoms(P, G, S);
        {   // zero the bordered plane buffers (borders stay zero) and the nonlocal planes
            const int bufsz = (G.m[0] + 2 * Q) * (G.m[1] + 2 * Q);
            float2* pb = reinterpret_cast<float2*>(dsm + L.plane_off);
            for (int t = threadIdx.x; t < 2 * bufsz; t += blockDim.x) pb[t] = make_float2(0.f, 0.f);
            for (int t = threadIdx.x; t < 2 * G.plane; t += blockDim.x) nlbuf[t] = make_float2(0.f, 0.f);
        }
        for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
            r[i] = make_float2(i == G.src ? 1.f : 0.f, 0.f);
            p[i] = make_float2(0.f, 0.f);
            x[i] = make_double2(0.0, 0.0);
            dx[i] = make_float2(0.f, 0.f);
        }
        if (threadIdx.x == 0) {
            S.beta[0] = 0.0;
            S.beta[1] = 0.0;
            S.action = 0;
            S.rho[0] = 1.0;
            S.rho[1] = 0.0;
            S.rn = 1.0;
            S.rn_last = 1.0;
            S.it = 0;
            S.last_rel = 0;
            S.n_rel = 0;
            S.restart = 0;
            S.st = 2;
        }
        __syncthreads();

        for (;;) {
            if (P.timeout_ns && threadIdx.x == 0 && (global_time_ns() - t_start) > P.timeout_ns)
                S.action = kStopTimeout;
            if (threadIdx.x == 0 && S.it >= P.maxit) S.action = kStop;
            __syncthreads();
            if (S.action == kStop || S.action == kStopTimeout) break;
            KSum<float> acc_re, acc_im;
            zm_stencil_pass<Q, K>(P, G, S, dsm, L, ph, r, p, Ap, (float)S.beta[0], (float)S.beta[1], zr, zi,
                                  diagF, acc_re, acc_im);
            __syncthreads();
            float hi[2] = {acc_re.hi(), acc_im.hi()}, lo[2] = {acc_re.lo(), acc_im.lo()};
            if (P.nonlocal) {
                // coefficients E_l dV C_l s_l and the bilinear energy E_l dV (C_l s_l)^2
                const float* cacc = reinterpret_cast<const float*>(dsm + L.cacc_off);
                for (int t = threadIdx.x; t < S.n_local * 4; t += blockDim.x) {
                    const int kk = t >> 2, l = t & 3;
                    const double sr = cacc[kk * 8 + 2 * l], si = cacc[kk * 8 + 2 * l + 1];
                    const double Cl = __ldg(P.proj_C + 4LL * S.la_id[kk] + l);
                    const double E = (l == 0 ? P.e_s : P.e_p) * P.dV * Cl;
                    S.c[kk][l] = make_double2(E * sr, E * si);
                    S.cf[kk][l] = make_float2((float)(E * sr), (float)(E * si));
                    const double er = E * Cl * (sr * sr - si * si), ei = E * Cl * 2.0 * sr * si;
                    const float qr = (float)er, qi = (float)ei;
                    ff_add(hi[0], lo[0], qr, (float)(er - (double)qr));
                    ff_add(hi[1], lo[1], qi, (float)(ei - (double)qi));
                }
            }
            {
                double pap[2];
                block_reduce_ff<2>(S, hi, lo, pap);
                if (threadIdx.x == 0) {
                    ++S.it;
                    const double den = pap[0] * pap[0] + pap[1] * pap[1];
                    if (S.flag == 2 || !(den > 0.0)) {
                        S.st = 3;
                        S.action = kStop;
                    } else {
                        S.alpha[0] = (S.rho[0] * pap[0] + S.rho[1] * pap[1]) / den;
                        S.alpha[1] = (S.rho[1] * pap[0] - S.rho[0] * pap[1]) / den;
                    }
                }
                __syncthreads();
                if (S.action == kStop) break;
            }
            double red3[3];
            {   // P3, plane by plane: dx += alpha p ; r -= alpha (Ap_loc + Ap_nl) ; dots
                const float ar = (float)S.alpha[0], ai = (float)S.alpha[1];
                KSum<float> s_re, s_im, s_n;
                const int plane = G.plane, m2 = G.m[2];
                if (P.nonlocal) {
                    zm_nl_plane(P, G, S, nlbuf, 0);
                    __syncthreads();
                }
                for (int c = 0; c < m2; ++c) {
                    float2* nlc = nlbuf + (c & 1) * plane;
                    if (P.nonlocal && c + 1 < m2) zm_nl_plane(P, G, S, nlbuf + ((c + 1) & 1) * plane, c + 1);
                    for (int col = threadIdx.x; col < plane; col += blockDim.x) {
                        const int i = col + c * plane;
                        const float2 pv = p[i];
                        float2 qv = Ap[i];
                        if (P.nonlocal) {
                            const float2 nv = nlc[col];
                            qv.x += nv.x;
                            qv.y += nv.y;
                            nlc[col] = make_float2(0.f, 0.f);
                        }
                        float2 d = dx[i], rv = r[i];
                        d.x += ar * pv.x - ai * pv.y;
                        d.y += ar * pv.y + ai * pv.x;
                        rv.x -= ar * qv.x - ai * qv.y;
                        rv.y -= ar * qv.y + ai * qv.x;
                        dx[i] = d;
                        r[i] = rv;
                        s_re.add(rv.x * rv.x - rv.y * rv.y);
                        s_im.add(2.f * rv.x * rv.y);
                        s_n.add(rv.x * rv.x + rv.y * rv.y);
                    }
                    if (P.nonlocal) __syncthreads();
                }
                const float hi3[3] = {s_re.hi(), s_im.hi(), s_n.hi()};
                const float lo3[3] = {s_re.lo(), s_im.lo(), s_n.lo()};
                block_reduce_ff<3>(S, hi3, lo3, red3);
            }
            if (threadIdx.x == 0) {
                const double rn = sqrt(red3[2]);
                const bool want = (rn <= P.tol) || (S.it - S.last_rel >= P.reliable_every) ||
                                  (rn < P.reliable_delta * S.rn_last);
                S.action = want ? kRefresh : 0;
            }
            __syncthreads();
            if (S.action == kRefresh) {
                refresh_residual<Mode, Q>(P, G, S, r, dx, x, zd, red3);
                if (threadIdx.x == 0) {
                    const double rt = sqrt(red3[2]);
                    S.restart = (S.n_rel > 0 && rt >= S.rn_last) ? 1 : 0;
                    S.rn_last = rt;
                    S.last_rel = S.it;
                    ++S.n_rel;
                }
            }
            if (threadIdx.x == 0) {
                const double rn = sqrt(red3[2]);
                S.rn = rn;
                S.action = 0;
                const double rr_abs = sqrt(red3[0] * red3[0] + red3[1] * red3[1]);
                if (rn <= P.tol) {
                    S.st = 0;
                    S.action = kStop;
                } else if (!(rr_abs > 1e-300) || rr_abs < 1e-14 * rn * rn) {
                    S.st = 3;
                    S.action = kStop;
                } else {
                    const double rd = S.rho[0] * S.rho[0] + S.rho[1] * S.rho[1];
                    S.beta[0] = S.restart ? 0.0 : (red3[0] * S.rho[0] + red3[1] * S.rho[1]) / rd;
                    S.beta[1] = S.restart ? 0.0 : (red3[1] * S.rho[0] - red3[0] * S.rho[1]) / rd;
                    S.rho[0] = red3[0];
                    S.rho[1] = red3[1];
                }
                S.restart = 0;
            }
            __syncthreads();
            if (S.action == kStop) break;
        }
        const bool timed_out = (S.action == kStopTimeout);
        __syncthreads();
        const int status = S.st;
        if (status != 0) {
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
            P.status[out_idx] = timed_out ? 4 : (S.flag == 2 ? 5 : (S.flag ? 1 : status));
            P.iters[out_idx] = S.it;
            P.resid[out_idx] = S.rn;
            P.n_rel[out_idx] = S.n_rel;
        }
        if (P.nonlocal) release_local_atoms(P, S);
        __syncthreads();
    }
}

struct FP64Mode {
    using real = double;
    using cplx = double2;
    static constexpr bool kMixed = false;
};
using MixedMode = MixedModeT;

template <class Mode, int kMinB>
cudaError_t launch_q(const SolveParams& P, int grid, int block, cudaStream_t stream) {
    switch (P.q) {
        case 1: k_cocg<Mode, 1, kMinB><<<grid, block, 0, stream>>>(P); break;
        case 2: k_cocg<Mode, 2, kMinB><<<grid, block, 0, stream>>>(P); break;
        case 3: k_cocg<Mode, 3, kMinB><<<grid, block, 0, stream>>>(P); break;
        case 4: k_cocg<Mode, 4, kMinB><<<grid, block, 0, stream>>>(P); break;
        case 5: k_cocg<Mode, 5, kMinB><<<grid, block, 0, stream>>>(P); break;
        case 6: k_cocg<Mode, 6, kMinB><<<grid, block, 0, stream>>>(P); break;
        case 7: k_cocg<Mode, 7, kMinB><<<grid, block, 0, stream>>>(P); break;
        case 8: k_cocg<Mode, 8, kMinB><<<grid, block, 0, stream>>>(P); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int Q, int K>
cudaError_t launch_zm_k(const SolveParams& P, int grid, int block, size_t smem, cudaStream_t stream) {
    cudaError_t e = cudaFuncSetAttribute(k_cocg_zm<Q, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_cocg_zm<Q, K><<<grid, block, smem, stream>>>(P);
    return cudaGetLastError();
}

template <int Q>
cudaError_t launch_zm_q(const SolveParams& P, int K, int grid, int block, size_t smem, cudaStream_t stream) {
    switch (K) {
        case 1: return launch_zm_k<Q, 1>(P, grid, block, smem, stream);
        case 2: return launch_zm_k<Q, 2>(P, grid, block, smem, stream);
        case 3: return launch_zm_k<Q, 3>(P, grid, block, smem, stream);
        case 4: return launch_zm_k<Q, 4>(P, grid, block, smem, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int zm_max_threads(int K) {
    switch (K) {
        case 1: return ZmThreads<1>::value;
        case 2: return ZmThreads<2>::value;
        case 3: return ZmThreads<3>::value;
        case 4: return ZmThreads<4>::value;
        default: return 0;
    }
}

bool zm_supported(int precision, int q) { return precision == MD_PREC_MIXED && (q == 2 || q == 4); }

template <int Q, int K>
int zm_occ_k(int block, size_t smem) {
    if (cudaFuncSetAttribute(k_cocg_zm<Q, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cocg_zm<Q, K>, block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int zm_occupancy(int q, int K, int block, size_t smem) {
    if (q == 2) {
        switch (K) {
            case 1: return zm_occ_k<2, 1>(block, smem);
            case 2: return zm_occ_k<2, 2>(block, smem);
            case 3: return zm_occ_k<2, 3>(block, smem);
            case 4: return zm_occ_k<2, 4>(block, smem);
        }
    } else if (q == 4) {
        switch (K) {
            case 1: return zm_occ_k<4, 1>(block, smem);
            case 2: return zm_occ_k<4, 2>(block, smem);
            case 3: return zm_occ_k<4, 3>(block, smem);
            case 4: return zm_occ_k<4, 4>(block, smem);
        }
    }
    return 0;
}

size_t zm_smem_bytes(int q, int max_m0, int max_m1) { return ZmLayout(q, max_m0, max_m1).total; }

cudaError_t launch_cocg_zm(const SolveParams& P, int K, int grid, int block, size_t smem, cudaStream_t stream) {
    if (P.q == 2) return launch_zm_q<2>(P, K, grid, block, smem, stream);
    if (P.q == 4) return launch_zm_q<4>(P, K, grid, block, smem, stream);
    return cudaErrorInvalidValue;
}

size_t slot_bytes_for(int precision, long long n_max) {
    const size_t nm = (size_t)((n_max + 63) / 64 * 64);
    if (precision == MD_PREC_MIXED) return nm * (4 * sizeof(float2) + sizeof(double2) + sizeof(uint2));
    return nm * (3 * sizeof(double2) + sizeof(double2));
}

cudaError_t launch_cocg(const SolveParams& P, int precision, int grid, int block, int per_sm,
                        cudaStream_t stream) {
    if (precision == MD_PREC_MIXED) {
        if (per_sm >= 3 && block <= 512) return launch_q<MixedMode, 3>(P, grid, block, stream);
        return launch_q<MixedMode, 1>(P, grid, block, stream);
    }
    return launch_q<FP64Mode, 1>(P, grid, block, stream);
}

cudaError_t launch_accumulate(int n_nodes, int Pn, const double2* x_src, const double2* z,
                              const double2* w, double dV, double* rho, double* e, cudaStream_t stream) {
    k_accumulate<<<(n_nodes + 127) / 128, 128, 0, stream>>>(n_nodes, Pn, x_src, z, w, dV, rho, e);
    return cudaGetLastError();
}

}  // namespace md
