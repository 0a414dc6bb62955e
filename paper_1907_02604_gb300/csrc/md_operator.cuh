// Device side of the region operator H_R(j) shared by the solver kernels
// (COCG, shifted COCG, Lanczos): region geometry and index arithmetic, the
// per-CTA shared state, block reductions, the nonlocal projector
// coefficients and the pointwise matvec
//     (H_R - z) v = (-1/2 L_FD + V - z) v + sum_{a,l} E_l dV p_al (p_al^T v).
// Vectors are complex (float2 / double2) for the shifted solves or real
// (double) for Lanczos; re_of / im_of read either kind.
//
// Index arithmetic: each thread walks region points i = tid, tid + T, ...
// (coalesced); (a, b, c) come from i by multiply-shift division by the
// invariant row and plane sizes (Granlund & Montgomery, PLDI 1994).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "md_device.cuh"
#include "md_internal.h"
#include "md_solver.h"

namespace md {

namespace {


constexpr int kLocal = kMaxLocalProjAtoms;
constexpr int kMapMax = 2048;   // direct global->local atom map when n_atoms <= this
constexpr int kChunk = 8;       // points per FP32 partial sum before it joins the FP64 sum
constexpr int kStop = 1, kRefresh = 2, kStopTimeout = 3;
constexpr int kMaxShifts = 64;

// Per-thread partial sum: compensated (Kahan) in float, plain in double.
// The float partial is rounded to double once, where the block reduction
// (double) takes over.
template <class R>
struct KSum;
template <>
struct KSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
    __device__ __forceinline__ float hi() const { return s; }
    __device__ __forceinline__ float lo() const { return -c; }
};
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

struct MixedModeT {
    using real = float;
    using cplx = float2;
    static constexpr bool kMixed = true;
};

template <>
struct KSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double get() const { return s; }
};

// L2 eviction policy for data streamed once per pass (the Krylov vectors
// and point records): marked evict-first so that the lines the next pass
// re-reads (the direction p, the potential, the projector values) are the
// ones the L2 keeps.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ float4 ld_stream(const float4* a, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_stream(float4* a, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_stream(float2* a, float2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ uint2 ld_stream(const uint2* a, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(a), "l"(pol));
    return v;
}

struct FastDiv {
    uint32_t m;
    uint32_t l;
};

__device__ __forceinline__ FastDiv make_fastdiv(uint32_t d) {
    uint32_t l = 0;
    while ((1u << l) < d) ++l;
    const uint64_t m = ((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1;
    return FastDiv{(uint32_t)m, l};
}

// n / d for 0 <= n < 2^31
__device__ __forceinline__ uint32_t fdiv(uint32_t n, FastDiv f) { return (__umulhi(n, f.m) + n) >> f.l; }

// Real and imaginary parts of a vector element: complex (float2, double2)
// for the shifted solves, real (double) for Lanczos, whose imaginary part
// is the constant 0 (the compiler drops the arithmetic on it).
template <class R>
__device__ __forceinline__ R re_of(float2 v) { return (R)v.x; }
template <class R>
__device__ __forceinline__ R im_of(float2 v) { return (R)v.y; }
template <class R>
__device__ __forceinline__ R re_of(double2 v) { return (R)v.x; }
template <class R>
__device__ __forceinline__ R im_of(double2 v) { return (R)v.y; }
template <class R>
__device__ __forceinline__ R re_of(double v) { return (R)v; }
template <class R>
__device__ __forceinline__ R im_of(double) { return (R)0; }
template <class R>
__device__ __forceinline__ R re_of(float v) { return (R)v; }
template <class R>
__device__ __forceinline__ R im_of(float) { return (R)0; }
template <class C>
struct VMake {
    template <class R>
    __device__ static C make(R re, R im) { return cmake<C>(re, im); }
};
template <>
struct VMake<double> {
    template <class R>
    __device__ static double make(R re, R) { return (double)re; }
};
template <>
struct VMake<float> {
    template <class R>
    __device__ static float make(R re, R) { return (float)re; }
};

struct Geo {
    int m[3];
    int lo[3];
    int ring[3];
    int any_ring;
    int n;
    int plane;
    int src;
    FastDiv div_row, div_plane;
    // per region point: (local slots of its projector atoms, 8 bits each,
    // 0xFF ends the list; first CSR entry), or null for the CSR lists alone
    const uint2* nl_rec = nullptr;
};

template <class R>
struct Tab;
template <>
struct Tab<double> {
    __device__ static const double* d(const SolveParams& P) { return P.proj_d; }
    __device__ static const double* g(const SolveParams& P) { return P.proj_g; }
    __device__ static const double* C(const SolveParams& P) { return P.proj_C; }
    __device__ static double V(const SolveParams& P, long long gi) { return __ldg(P.V + gi); }
};
template <>
struct Tab<float> {
    __device__ static const float* d(const SolveParams& P) { return P.proj_d32; }
    __device__ static const float* g(const SolveParams& P) { return P.proj_g32; }
    __device__ static const float* C(const SolveParams& P) { return P.proj_C32; }
    __device__ static float V(const SolveParams& P, long long gi) { return __ldg(P.V32 + gi); }
};

struct Shared {
    double red[32][4];
    double bcast[4];
    double coefD[3][kMaxQ];
    float coefF[3][kMaxQ];
    double alpha[2];
    double beta[2];
    // COCG scalar state, owned by thread 0
    double rho[2];        // r^T r
    double rn, rn_last;   // ||r||, ||r|| at the last residual refresh
    int it, last_rel, n_rel, st;
    int restart;
    int action;
    int status;
    int sys;
    int flag;
    int n_local;
    int la_id[kLocal];
    short la_off[kLocal][3];
    double2 c[kLocal][4];   // E_l dV C_l sum_i f_l(i) v(i), double
    double2 pnl[32];        // per warp: sum over its atoms of E_l dV c_l^2 (v^T V_nl v)
    // shifted COCG (one Krylov sequence per node for all poles), per pole k:
    double2 sh_pi_prev[kMaxShifts], sh_pi[kMaxShifts];   // pi_{n-1}, pi_n
    double2 sh_x[kMaxShifts], sh_p[kMaxShifts];          // x_k(j), p_k(j)
    int sh_conv[kMaxShifts];                             // iteration at which pole k met tol, or 0
    double2 rj;                                          // seed residual at the node
    double alpha_prev[2], beta_prev[2];
    int all_conv;
    uint64_t bar[4];        // z-march: staging-slot mbarriers
    float2 cf[kLocal][4];   // the same rounded to float
    short map[kMapMax];     // global atom id -> local slot, -1 if absent
};

template <class R>
__device__ __forceinline__ const R* coef_of(const Shared& S);
template <>
__device__ __forceinline__ const double* coef_of<double>(const Shared& S) { return &S.coefD[0][0]; }
template <>
__device__ __forceinline__ const float* coef_of<float>(const Shared& S) { return &S.coefF[0][0]; }

// Error-free float-float addition (Knuth's TwoSum on the high parts, the
// low parts added in): keeps ~48 significant bits on the FP32 pipe.
__device__ __forceinline__ void ff_add(float& ah, float& al, float bh, float bl) {
    const float s = ah + bh;
    const float v = s - ah;
    const float e = (ah - (s - v)) + (bh - v) + (al + bl);
    ah = s + e;
    al = e - (ah - s);
}

// Block-wide sum of K per-thread float-float partials (hi, lo): the warp
// stage stays in float-float, the 32 warp totals are summed in double by
// warp 0.  Only thread 0 holds the totals afterwards (in v).
template <int K>
__device__ __forceinline__ void block_reduce_ff(Shared& S, const float (&hi)[K], const float (&lo)[K],
                                                double (&v)[K]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float h[K], l[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        h[k] = hi[k];
        l[k] = lo[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float bh = __shfl_xor_sync(0xffffffffu, h[k], o);
            const float bl = __shfl_xor_sync(0xffffffffu, l[k], o);
            ff_add(h[k], l[k], bh, bl);
        }
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) S.red[warp][k] = (double)h[k] + (double)l[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nw ? S.red[lane][k] : 0.0;
            v[k] = warp_sum(t);
        }
    }
}

// Block-wide sum of K doubles; only thread 0 holds the totals afterwards.
template <int K>
__device__ __forceinline__ void block_reduce(Shared& S, double (&v)[K]) {
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
            v[k] = warp_sum(t);
        }
    }
}

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
}

__device__ __forceinline__ int wrap_once(int g, int n) {
    g += (g < 0) ? n : 0;
    g -= (g >= n) ? n : 0;
    return g;
}

// Region slot of window index u for an atom window starting at region
// offset off (periodic axes: off in [0, n) and the window may wrap once).
__device__ __forceinline__ int region_slot(int off, int u, int n, int m, int periodic) {
    int a = off + u;
    if (periodic && a >= n) a -= n;
    return (a >= 0 && a < m) ? a : -1;
}

// The window indices u in [0, len) that land in the region on one axis form
// at most two runs; run k covers u in [lo_k, hi_k] with region slot u + shift_k.
struct Runs {
    int lo[2], hi[2], shift[2];
};

__device__ __forceinline__ Runs axis_runs(int off, int len, int n, int m, int periodic) {
    Runs r;
    r.lo[0] = max(0, -off);
    r.hi[0] = min(len - 1, m - 1 - off);
    if (periodic) r.hi[0] = min(r.hi[0], n - 1 - off);
    r.shift[0] = off;
    if (periodic) {
        r.lo[1] = max(0, n - off);
        r.hi[1] = min(len - 1, n - off + m - 1);
        r.shift[1] = off - n;
    } else {
        r.lo[1] = 1;
        r.hi[1] = 0;
        r.shift[1] = 0;
    }
    return r;
}

// Local atoms whose projector window meets the region; ascending atom id.
__device__ void collect_local_atoms(const SolveParams& P, const Geo& G, Shared& S) {
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
                        hit = hit && ((o < G.m[d]) || (o + len - 1 >= P.n[d]));
                    } else {
                        hit = hit && (o < G.m[d]) && (o + len - 1 >= 0);
                    }
                    off[d] = (short)o;
                }
            }
            const unsigned mask = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int slot = count + __popc(mask & ((1u << lane) - 1u));
                if (slot < kLocal) {
                    S.la_id[slot] = (int)a;
                    S.la_off[slot][0] = off[0];
                    S.la_off[slot][1] = off[1];
                    S.la_off[slot][2] = off[2];
                    if (P.n_atoms <= kMapMax) S.map[a] = (short)slot;
                }
            }
            count += __popc(mask);
        }
        if (lane == 0) {
            S.n_local = count < kLocal ? count : kLocal;
            if (count > kLocal) S.flag = 1;
        }
    }
    __syncthreads();
}

__device__ void release_local_atoms(const SolveParams& P, Shared& S) {
    if (P.n_atoms <= kMapMax)
        for (int k = threadIdx.x; k < S.n_local; k += blockDim.x) S.map[S.la_id[k]] = -1;
    __syncthreads();
}

__device__ __forceinline__ int local_slot(const SolveParams& P, const Shared& S, int atom) {
    if (P.n_atoms <= kMapMax) return S.map[atom];
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

// The nonlocal term's per-point record for the current region (collect_local_atoms
// first): the local slots of the point's projector atoms packed into .x and
// its first CSR entry in .y, so that an apply needs one coalesced load
// before the values instead of the point's CSR pointer, atom ids and slot
// lookups in turn.  Points with more than four atoms or an atom outside
// slots 0..254 get .y = 0xFFFFFFFF and keep the CSR path.
__device__ void build_nl_records(const SolveParams& P, const Geo& G, const Shared& S, uint2* __restrict__ rec) {
    for (int i = threadIdx.x; i < G.n; i += blockDim.x) {
        const int c = (int)fdiv((uint32_t)i, G.div_plane);
        const int rem = i - c * G.plane;
        const int b = (int)fdiv((uint32_t)rem, G.div_row);
        const int a = rem - b * G.m[0];
        const int gx = wrap_once(G.lo[0] + a, P.n[0]);
        const int gy = wrap_once(G.lo[1] + b, P.n[1]);
        const int gz = wrap_once(G.lo[2] + c, P.n[2]);
        const long long gi = gx + (long long)P.n[0] * (gy + (long long)P.n[1] * gz);
        const int e0 = __ldg(P.pl_ptr + gi), e1 = __ldg(P.pl_ptr + gi + 1);
        uint32_t sl = 0xFFFFFFFFu;
        bool ok = e1 - e0 <= 4;
        for (int e = e0; ok && e < e1; ++e) {
            const int k = local_slot(P, S, __ldg(P.pl_atom + e));
            ok = k >= 0 && k < 0xFF;
            const int sh = 8 * (e - e0);
            if (ok) sl = (sl & ~(0xFFu << sh)) | ((uint32_t)k << sh);
        }
        rec[i] = make_uint2(sl, ok ? (uint32_t)e0 : 0xFFFFFFFFu);
    }
}

// c_al = E_l dV sum_{i in region} p_al(i) v(i): warp per local atom, lane
// per window row (v, w).  The Gaussian is separable, so each row needs only
// A = sum_u g_x(u) v and B = sum_u d_x(u) g_x(u) v over its in-sphere run:
//   c_s += g_y g_z A, c_x += g_y g_z B, c_y += d_y g_y g_z A, c_z += d_z g_y g_z A.
template <class R, class C>
__device__ void nonlocal_coeffs(const SolveParams& P, const Geo& G, Shared& S, const C* __restrict__ v) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const R* dt = Tab<R>::d(P);
    const R* gt = Tab<R>::g(P);
    double pnl_re = 0.0, pnl_im = 0.0, t_re = 0.0, t_im = 0.0;
    for (int k = warp; k < S.n_local; k += nw) {
        const int a = S.la_id[k];
        const int lx = __ldg(P.proj_len + 3 * a), ly = __ldg(P.proj_len + 3 * a + 1),
                  lz = __ldg(P.proj_len + 3 * a + 2);
        const R* dx = dt + (3LL * a + 0) * kMaxProjWin;
        const R* dy = dt + (3LL * a + 1) * kMaxProjWin;
        const R* dz = dt + (3LL * a + 2) * kMaxProjWin;
        const R* gx = gt + (3LL * a + 0) * kMaxProjWin;
        const R* gy = gt + (3LL * a + 1) * kMaxProjWin;
        const R* gz = gt + (3LL * a + 2) * kMaxProjWin;
        const unsigned char* rows = P.proj_rows + 2LL * a * kMaxProjWin * kMaxProjWin;
        const Runs rx = axis_runs(S.la_off[k][0], lx, P.n[0], G.m[0], P.periodic[0]);
        R acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const int nrows = ly * lz;
        for (int row = lane; row < nrows; row += 32) {
            const int ww = row / ly, vv = row - ww * ly;
            const int b = region_slot(S.la_off[k][1], vv, P.n[1], G.m[1], P.periodic[1]);
            const int c = region_slot(S.la_off[k][2], ww, P.n[2], G.m[2], P.periodic[2]);
            if (b < 0 || c < 0) continue;
            const unsigned char* rw = rows + 2 * (ww * kMaxProjWin + vv);
            const int u0 = rw[0], u1 = rw[1];
            const C* vrow = v + G.m[0] * (b + G.m[1] * c);
            R Ar = 0, Ai = 0, Br = 0, Bi = 0;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int lo = max(u0, rx.lo[t]), hi = min(u1, rx.hi[t]);
                // unrolled so that a lane has several of its row's loads in flight
#pragma unroll 4
                for (int u = lo; u <= hi; ++u) {
                    const C pv = vrow[u + rx.shift[t]];
                    const R g1 = __ldg(gx + u);
                    const R g2 = __ldg(dx + u) * g1;
                    Ar += g1 * re_of<R>(pv); Ai += g1 * im_of<R>(pv);
                    Br += g2 * re_of<R>(pv); Bi += g2 * im_of<R>(pv);
                }
            }
            const R gyz = __ldg(gy + vv) * __ldg(gz + ww);
            const R ey = __ldg(dy + vv) * gyz, ez = __ldg(dz + ww) * gyz;
            acc[0] += gyz * Ar; acc[1] += gyz * Ai;
            acc[2] += gyz * Br; acc[3] += gyz * Bi;
            acc[4] += ey * Ar;  acc[5] += ey * Ai;
            acc[6] += ez * Ar;  acc[7] += ez * Ai;
        }
        double s[8];
        // warp sums in R (float in the mixed iteration: the FP64 pipe is
        // scarce), then one conversion of the warp total
#pragma unroll
        for (int t = 0; t < 8; ++t) s[t] = (double)warp_sum(acc[t]);
        if (lane < 4) {
            const double Cl = (double)__ldg(P.proj_C + 4LL * a + lane);
            const double E = (lane == 0 ? P.e_s : P.e_p) * P.dV * Cl;
            double sr = s[0], si = s[1];
            if (lane == 1) { sr = s[2]; si = s[3]; }
            if (lane == 2) { sr = s[4]; si = s[5]; }
            if (lane == 3) { sr = s[6]; si = s[7]; }
            S.c[k][lane] = make_double2(E * sr, E * si);
            S.cf[k][lane] = make_float2((float)(E * sr), (float)(E * si));
            // bilinear nonlocal energy of v: E_l dV (C_l s)^2
            t_re = E * Cl * (sr * sr - si * si);
            t_im = E * Cl * 2.0 * sr * si;
        }
        t_re += __shfl_xor_sync(0xffffffffu, t_re, 1);
        t_im += __shfl_xor_sync(0xffffffffu, t_im, 1);
        t_re += __shfl_xor_sync(0xffffffffu, t_re, 2);
        t_im += __shfl_xor_sync(0xffffffffu, t_im, 2);
        if (lane == 0) {
            pnl_re += t_re;
            pnl_im += t_im;
        }
        t_re = 0.0;
        t_im = 0.0;
    }
    if (lane == 0) S.pnl[warp] = make_double2(pnl_re, pnl_im);
    __syncthreads();
}

template <class R>
struct PVal;
template <>
struct PVal<float> {
    __device__ static void get(const SolveParams& P, int e, float (&f)[4]) {
        const float4 v = __ldg(P.pl_val32 + e);
        f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
    }
    __device__ static float2 c(const Shared& S, int k, int l) { return S.cf[k][l]; }
};
template <>
struct PVal<double> {
    __device__ static void get(const SolveParams& P, int e, double (&f)[4]) {
        const double2 a = __ldg(P.pl_val64 + 2 * e), b = __ldg(P.pl_val64 + 2 * e + 1);
        f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y;
    }
    __device__ static double2 c(const Shared& S, int k, int l) { return S.c[k][l]; }
};

// Nonlocal part of (H_R v)(i) from the coefficients in S.cf (mixed path):
// the point's projector list (global CSR) with its four stored values.
__device__ __forceinline__ float2 nl_apply(const SolveParams& P, const Geo& G, const Shared& S, int i) {
    const int c = (int)fdiv((uint32_t)i, G.div_plane);
    const int rem = i - c * G.plane;
    const int b = (int)fdiv((uint32_t)rem, G.div_row);
    const int a = rem - b * G.m[0];
    const int gx = wrap_once(G.lo[0] + a, P.n[0]);
    const int gy = wrap_once(G.lo[1] + b, P.n[1]);
    const int gz = wrap_once(G.lo[2] + c, P.n[2]);
    const long long gi = gx + (long long)P.n[0] * (gy + (long long)P.n[1] * gz);
    float yx = 0.f, yy = 0.f;
    const int e0 = __ldg(P.pl_ptr + gi), e1 = __ldg(P.pl_ptr + gi + 1);
    for (int e = e0; e < e1; ++e) {
        const int k = local_slot(P, S, __ldg(P.pl_atom + e));
        if (k < 0) continue;
        const float4 f = __ldg(P.pl_val32 + e);
        const float2 c0 = S.cf[k][0], c1 = S.cf[k][1], c2 = S.cf[k][2], c3 = S.cf[k][3];
        yx += f.x * c0.x + f.y * c1.x + f.z * c2.x + f.w * c3.x;
        yy += f.x * c0.y + f.y * c1.y + f.z * c2.y + f.w * c3.y;
    }
    return make_float2(yx, yy);
}

// y = (H_R - z) v at region point i (Q = stencil half-width), arithmetic in R;
// kNl = false leaves out the nonlocal term (added elsewhere).
template <class R, class C, int Q, class CIn, bool kNl = true>
__device__ __forceinline__ C matvec_point(const SolveParams& P, const Geo& G, const Shared& S,
                                          const CIn* __restrict__ v, int i, R zr, R zi, R diag,
                                          uint2 rc_pre = make_uint2(0u, 0xFFFFFFFEu)) {
    const int c = (int)fdiv((uint32_t)i, G.div_plane);
    const int rem = i - c * G.plane;
    const int b = (int)fdiv((uint32_t)rem, G.div_row);
    const int a = rem - b * G.m[0];
    const int gx = wrap_once(G.lo[0] + a, P.n[0]);
    const int gy = wrap_once(G.lo[1] + b, P.n[1]);
    const int gz = wrap_once(G.lo[2] + c, P.n[2]);
    const long long gi = gx + (long long)P.n[0] * (gy + (long long)P.n[1] * gz);
    // the point's projector record first: its load (from the system's slot
    // in device memory) then overlaps the stencil's
    uint2 rc = make_uint2(0u, 0xFFFFFFFFu);
    if (rc_pre.y != 0xFFFFFFFEu) rc = rc_pre;   // loaded ahead by the caller
    else if (kNl && P.nonlocal && G.nl_rec) rc = G.nl_rec[i];
    const CIn vi = v[i];
    const R dg = diag + Tab<R>::V(P, gi) - zr;
    R yx = dg * re_of<R>(vi) + zi * im_of<R>(vi);
    R yy = dg * im_of<R>(vi) - zi * re_of<R>(vi);
    const R* cf = coef_of<R>(S);
    const int pos[3] = {a, b, c};
    const int stride[3] = {1, G.m[0], G.plane};
    if (!G.any_ring) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int o = 1; o <= Q; ++o) {
                const R w = cf[d * kMaxQ + (o - 1)];
                R sx = 0, sy = 0;
                if (pos[d] + o < G.m[d]) {
                    const CIn t = v[i + o * stride[d]];
                    sx += re_of<R>(t);
                    sy += im_of<R>(t);
                }
                if (pos[d] - o >= 0) {
                    const CIn t = v[i - o * stride[d]];
                    sx += re_of<R>(t);
                    sy += im_of<R>(t);
                }
                yx += w * sx;
                yy += w * sy;
            }
        }
    } else {
        for (int d = 0; d < 3; ++d) {
            const int md = G.m[d];
            for (int o = 1; o <= Q; ++o) {
                const R w = cf[d * kMaxQ + (o - 1)];
                R sx = 0, sy = 0;
                if (G.ring[d]) {
                    const int tp = (pos[d] + o) % md;
                    const int tm = ((pos[d] - o) % md + md) % md;
                    const CIn up = v[i + (tp - pos[d]) * stride[d]];
                    const CIn dn = v[i + (tm - pos[d]) * stride[d]];
                    sx = re_of<R>(up) + re_of<R>(dn);
                    sy = im_of<R>(up) + im_of<R>(dn);
                } else {
                    if (pos[d] + o < md) {
                        const CIn t = v[i + o * stride[d]];
                        sx += re_of<R>(t);
                        sy += im_of<R>(t);
                    }
                    if (pos[d] - o >= 0) {
                        const CIn t = v[i - o * stride[d]];
                        sx += re_of<R>(t);
                        sy += im_of<R>(t);
                    }
                }
                yx += w * sx;
                yy += w * sy;
            }
        }
    }
    if (kNl && P.nonlocal && G.nl_rec) {
        if (rc.y != 0xFFFFFFFFu) {
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const uint32_t k = (rc.x >> (8 * l)) & 0xFFu;
                if (k == 0xFFu) break;
                R f[4];
                PVal<R>::get(P, (int)rc.y + l, f);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const auto cc = PVal<R>::c(S, (int)k, q);
                    yx += f[q] * (R)cc.x;
                    yy += f[q] * (R)cc.y;
                }
            }
            return VMake<C>::make(yx, yy);
        }
    }
    if (kNl && P.nonlocal) {
        const int e0 = __ldg(P.pl_ptr + gi), e1 = __ldg(P.pl_ptr + gi + 1);
        for (int e = e0; e < e1; ++e) {
            const int k = local_slot(P, S, __ldg(P.pl_atom + e));
            if (k < 0) continue;
            R f[4];
            PVal<R>::get(P, e, f);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const auto cc = PVal<R>::c(S, k, l);
                yx += f[l] * (R)cc.x;
                yy += f[l] * (R)cc.y;
            }
        }
    }
    return VMake<C>::make(yx, yy);
}

}  // namespace

}  // namespace md
