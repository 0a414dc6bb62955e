// Mixed-precision batched COCG with the Krylov vectors on chip: one
// thread-block cluster per (node, pole) system.
//
// The generic solver (md_solver.cu) keeps each system's vectors in device
// memory, so every COCG iteration streams them through HBM.  Here the region
// R(j) is cut into z-slabs, one per CTA of a cluster, and each CTA keeps its
// slab of p and r in shared memory for the whole solve.  Per iteration
// (same algebra as the generic kernel, van der Vorst & Melissen 1990):
//   P1  p = r + beta p                          own slab, shared memory
//   --  cluster barrier: p is visible to the neighbouring slabs
//   NL  partial c_al = sum_i f_al(i) p(i) over the own slab (warp per atom)
//   P2  Ap_loc = (-1/2 L + V - z) p, p^T Ap_loc; each thread marches its
//       (x, y) columns along z with the 2Q+1 stencil values in registers;
//       x and y neighbours come from the own slab, the Q planes above and
//       below the slab from the neighbouring CTAs' shared memory (DSMEM)
//   --  cluster barrier; every CTA sums the partials of all CTAs in rank
//       order, so every CTA holds bitwise the same alpha and coefficients
//   NL  r -= alpha sum_al E_l dV c_al p_al, scattered row by row from the
//       separable projector tables (shared-memory atomics)
//   P3  r -= alpha Ap_loc, dx += alpha p, r^T r, ||r||^2
//   --  cluster barrier; beta, convergence and refresh decisions, again
//       identical in every CTA, so the control flow stays uniform across
//       the cluster (every CTA meets every barrier)
// The nonlocal term enters p^T A p through the bilinear identity
//   p^T A p = p^T A_loc p + sum_al E_l dV c_al^2.
// Ap_loc and dx (FP32, slab-local per CTA) and x_hi (FP64, region-local)
// live in a per-cluster slot of device memory; Ap_loc and dx are touched by
// their own CTA only and stay in L2.
// Reliable updates (van der Vorst & Ye 2000) flush dx into x_hi and
// recompute r = e_j - (H_R - z) x_hi in FP64 from x_hi in device memory,
// with the FP64 operator of the generic kernel.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "md_operator.cuh"

namespace md {

namespace {

constexpr int kClMaxThreads = 576;

// ---- cluster primitives (PTX) ----------------------------------------------

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_nrank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
// All threads of all CTAs of the cluster; release/acquire at cluster scope
// (orders shared and global memory), and a CTA-wide barrier as well.
__device__ __forceinline__ void cl_sync() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::
            : "memory");
}
// Address in CTA `rank`'s shared memory of the local shared address `a`.
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 cl_ld_f2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ double cl_ld_f64(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
// Generic address, in CTA `rank`, of the location the generic shared-memory
// address p has in this CTA: plain loads through it reach the other CTA's
// shared memory (DSMEM) and the compiler can schedule them like any load.
__device__ __forceinline__ const float2* cl_map_ptr(const float2* p, uint32_t rank) {
    uint64_t r;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
    return reinterpret_cast<const float2*>(r);
}
__device__ __forceinline__ int cl_ld_s32(uint32_t a) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// Per-CTA values the other CTAs of the cluster read after a barrier.
struct ClRed {
    double pap[2];       // p^T A_loc p over the own slab
    double dots[3];      // r^T r (re, im), ||r||^2 over the own slab
    int sys;             // work item fetched by rank 0
    int timeout;         // rank 0: the deadline has passed
    int nrows;           // nonlocal row records of the own slab
    // halo planes of the stencil: z0-Q..z0-1 (t < Q) and z1..z1+Q-1 (t >= Q),
    // as generic addresses of the plane in the owning CTA's shared memory
    // (NULL: the plane lies outside the region and reads as zero)
    const float2* hptr[2 * kMaxQ];
};

// Dynamic shared memory: p and r slabs (slab_pts points each, float2), the
// per-atom partial projections (float2 [kLocal][4]) and ClRed.
struct ClLayout {
    size_t p_off, r_off, part_off, cnt_off, red_off, xt_off, total;
    __host__ __device__ ClLayout(int slab_pts, int xtab_floats) {
        const size_t sp = (size_t)((slab_pts + 1) & ~1);
        p_off = 0;
        r_off = p_off + sp * sizeof(float2);
        part_off = r_off + sp * sizeof(float2);
        cnt_off = part_off + (size_t)kLocal * 4 * sizeof(float2);              // int [2][kLocal + 1]
        red_off = cnt_off + ((size_t)2 * (kLocal + 1) * sizeof(int) + 15) / 16 * 16;
        xt_off = red_off + (sizeof(ClRed) + 15) / 16 * 16;                    // float [atoms][2][wx]
        total = xt_off + ((size_t)xtab_floats * sizeof(float) + 15) / 16 * 16;
    }
};

// A nonlocal row record: the row's constants c = (g_y g_z, d_y g_y g_z,
// d_z g_y g_z) in float (computed once per system), and its indices
//   idx.x: atom slot (bits 0-7) | x-run (bit 8) | slab plane (bits 9-16) | region row (bits 17-24)
//   idx.y: v (bits 0-7) | w (bits 8-15) | first and last window x index (bits 16-23, 24-31)
struct __align__(16) Row {
    float4 c;
    uint2 idx;
    uint2 pad;
};

// First plane of rank k's slab when m2 planes are cut into n slabs.
__device__ __forceinline__ int slab_start(int k, int m2, int n) { return (int)(((long long)k * m2) / n); }

// Owning rank of plane c (the largest k with slab_start(k) <= c).
__device__ __forceinline__ int slab_owner(int c, int m2, int n) {
    return (int)((((long long)c + 1) * n + m2 - 1) / m2) - 1;
}

// Window rows of an atom whose z-slot lies in [z0, z1): at most two runs
// [lo, hi] of window index w, region plane w + shift.
struct ZRows {
    int lo[2], hi[2], shift[2], n0, n;
};
__device__ __forceinline__ ZRows slab_rows(int off, int len, int n, int m, int periodic, int z0, int z1) {
    const Runs rz = axis_runs(off, len, n, m, periodic);
    ZRows r;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        r.lo[t] = max(rz.lo[t], z0 - rz.shift[t]);
        r.hi[t] = min(rz.hi[t], z1 - 1 - rz.shift[t]);
        r.shift[t] = rz.shift[t];
    }
    r.n0 = max(0, r.hi[0] - r.lo[0] + 1);
    r.n = r.n0 + max(0, r.hi[1] - r.lo[1] + 1);
    return r;
}

// Row records of the nonlocal term on the own slab, built once per system:
// one per (local atom, window row (v, w) in the slab, region x-run) whose
// in-sphere span meets the region.
//   .x: atom slot (bits 0-7) | x-run (bit 8) | slab plane (bits 9-16) | region row (bits 17-24)
//   .y: v (bits 0-7) | w (bits 8-15) | first and last window x index (bits 16-23, 24-31)
// Two orders of the same records: by atom (rows_a: the projection pass,
// whose warps then sum runs of one atom before a single atomic each), and
// by region row (rows_b with offsets off_b over the keys lc * m1 + b: the
// scatter pass, in which one thread owns a region row and updates it
// without atomics).
struct RowLists {
    Row* rows_a;
    Row* rows_b;
    int* off_b;     // [nkeys + 1]
    int* fill_b;    // [nkeys] scratch
    int cap;        // records per list
    int nkeys_cap;  // region rows per slab
};

// Visits every row record of the own slab: f(k, record) per record, warp
// per local atom, lanes over the atom's rows in a fixed order.
template <class F>
__device__ __forceinline__ void cl_for_rows(const SolveParams& P, const Geo& G, const Shared& S, int z0, int z1, F f) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < S.n_local; k += nw) {
        const int a = S.la_id[k];
        const int lx = __ldg(P.proj_len + 3 * a), ly = __ldg(P.proj_len + 3 * a + 1),
                  lz = __ldg(P.proj_len + 3 * a + 2);
        const unsigned char* tab = P.proj_rows + 2LL * a * kMaxProjWin * kMaxProjWin;
        const Runs rx = axis_runs(S.la_off[k][0], lx, P.n[0], G.m[0], P.periodic[0]);
        const ZRows rz = slab_rows(S.la_off[k][2], lz, P.n[2], G.m[2], P.periodic[2], z0, z1);
        const int nr = ly * rz.n;
        // warp-uniform trip count, so f may use warp collectives
        for (int base = 0; base < nr; base += 32) {
            const int row = base + lane;
            Row rec[2];
            bool ok[2] = {false, false};
            if (row < nr) {
                const int t = row / ly, vv = row - t * ly;
                const int ww = t < rz.n0 ? rz.lo[0] + t : rz.lo[1] + (t - rz.n0);
                const int c = ww + (t < rz.n0 ? rz.shift[0] : rz.shift[1]);
                const int b = region_slot(S.la_off[k][1], vv, P.n[1], G.m[1], P.periodic[1]);
                if (b >= 0) {
                    const unsigned char* rw = tab + 2 * (ww * kMaxProjWin + vv);
                    const int u0 = rw[0], u1 = rw[1];
                    const float gyz = __ldg(P.proj_g32 + (3LL * a + 1) * kMaxProjWin + vv) *
                                      __ldg(P.proj_g32 + (3LL * a + 2) * kMaxProjWin + ww);
                    const float4 cst = make_float4(gyz, __ldg(P.proj_d32 + (3LL * a + 1) * kMaxProjWin + vv) * gyz,
                                                   __ldg(P.proj_d32 + (3LL * a + 2) * kMaxProjWin + ww) * gyz, 0.f);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int lo = max(u0, rx.lo[q]), hi = min(u1, rx.hi[q]);
                        ok[q] = lo <= hi;
                        rec[q].c = cst;
                        rec[q].idx = make_uint2((uint32_t)k | ((uint32_t)q << 8) | ((uint32_t)(c - z0) << 9) |
                                                    ((uint32_t)b << 17),
                                                (uint32_t)vv | ((uint32_t)ww << 8) | ((uint32_t)lo << 16) |
                                                    ((uint32_t)hi << 24));
                        rec[q].pad = make_uint2(0u, 0u);
                    }
                }
            }
            f(k, rec, ok);
        }
    }
}

// Builds rows_a and rows_b/off_b for the own slab; returns the record count
// (in *n_out, shared) or cap + 1 if the lists would overflow.  cnt and off
// are shared int arrays of kLocal + 1 entries.
__device__ void cl_build_rows(const SolveParams& P, const Geo& G, Shared& S, int z0, int z1, const RowLists& L,
                              int* cnt, int* off, int* n_out) {
    const int lane = threadIdx.x & 31;
    const int nkeys = (z1 - z0) * G.m[1];
    if (nkeys > L.nkeys_cap) {   // cannot happen with the host's bounds; touch nothing
        if (threadIdx.x == 0) *n_out = L.cap + 1;
        __syncthreads();
        return;
    }
    for (int t = threadIdx.x; t <= kLocal; t += blockDim.x) cnt[t] = 0;
    for (int t = threadIdx.x; t < nkeys; t += blockDim.x) L.fill_b[t] = 0;
    __syncthreads();
    // counts per atom (warp-private) and per region row
    cl_for_rows(P, G, S, z0, z1, [&](int k, const Row (&rec)[2], const bool (&ok)[2]) {
        const int n = __popc(__ballot_sync(0xffffffffu, ok[0])) + __popc(__ballot_sync(0xffffffffu, ok[1]));
        if (lane == 0) cnt[k] += n;
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (ok[q])
                atomicAdd(&L.fill_b[(rec[q].idx.x >> 9 & 0xFFu) * G.m[1] + (rec[q].idx.x >> 17 & 0xFFu)], 1);
    });
    __syncthreads();
    if (threadIdx.x == 0) {   // exclusive scans (once per system)
        int acc = 0;
        for (int k = 0; k < S.n_local; ++k) {
            off[k] = acc;
            acc += cnt[k];
        }
        off[S.n_local] = acc;
        *n_out = acc;
        int accb = 0;
        for (int key = 0; key < nkeys; ++key) {
            L.off_b[key] = accb;
            accb += L.fill_b[key];
            L.fill_b[key] = 0;
        }
        L.off_b[nkeys] = accb;
    }
    __syncthreads();
    if (*n_out > L.cap) return;
    // fill: by atom in enumeration order, by region row in arrival order
    cl_for_rows(P, G, S, z0, z1, [&](int k, const Row (&rec)[2], const bool (&ok)[2]) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const unsigned m = __ballot_sync(0xffffffffu, ok[q]);
            const int before = __popc(m & ((1u << lane) - 1u));
            const int base_k = off[k];
            __syncwarp();   // every lane has read off[k] before lane 0 advances it
            if (ok[q]) {
                L.rows_a[base_k + before] = rec[q];
                const int key = (int)(rec[q].idx.x >> 9 & 0xFFu) * G.m[1] + (int)(rec[q].idx.x >> 17 & 0xFFu);
                L.rows_b[L.off_b[key] + atomicAdd(&L.fill_b[key], 1)] = rec[q];
            }
            if (lane == 0) off[k] = base_k + __popc(m);
            __syncwarp();
        }
    });
    __syncthreads();
}

struct RowRec {
    int k, q, lc, b, vv, ww, lo, hi;
};
__device__ __forceinline__ RowRec decode_row(uint2 r) {
    RowRec d;  // indices of Row::idx
    d.k = (int)(r.x & 0xFFu);
    d.q = (int)((r.x >> 8) & 1u);
    d.lc = (int)((r.x >> 9) & 0xFFu);
    d.b = (int)((r.x >> 17) & 0xFFu);
    d.vv = (int)(r.y & 0xFFu);
    d.ww = (int)((r.y >> 8) & 0xFFu);
    d.lo = (int)((r.y >> 16) & 0xFFu);
    d.hi = (int)(r.y >> 24);
    return d;
}

// Sum of v over the run of lanes holding the same key (runs are contiguous:
// the records are sorted by key); the run's first lane gets the total.
// Returns true on that lane.
template <class T, int N>
__device__ __forceinline__ bool run_sum(int key, T (&v)[N]) {
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int first = __ffs(peers) - 1, last = 31 - __clz(peers);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const T t = __shfl_down_sync(0xffffffffu, v[j], o);
            if (lane + o <= last) v[j] += t;
        }
    }
    return lane == first;
}

// Partial projections of the own slab of p onto each local atom's four
// projector shapes, f_al = (1, d_x, d_y, d_z) g_x g_y g_z (C_l applied after
// the cluster sum): records by atom, one per thread; per record A = sum g_x p
// and B = sum d_x g_x p, then c_s += g_y g_z A, c_x += g_y g_z B,
// c_y += d_y g_y g_z A, c_z += d_z g_y g_z A, summed over each run of one
// atom within the warp and added to acc[k][8] (shared, zeroed beforehand)
// by the run's first lane.
// x tables of local atom k: the shared copy (xt != NULL: g at xt + 2 wx k,
// d_x at xt + 2 wx k + wx), or the device tables.
__device__ __forceinline__ void x_tables(const SolveParams& P, const Shared& S, const float* xt, int wx, int k,
                                         const float*& g, const float*& d) {
    if (xt) {
        g = xt + 2 * wx * k;
        d = g + wx;
    } else {
        const long long a = S.la_id[k];
        g = P.proj_g32 + 3LL * a * kMaxProjWin;
        d = P.proj_d32 + 3LL * a * kMaxProjWin;
    }
}

__device__ __noinline__ void cl_nl_partials(const SolveParams& P, const Geo& G, const Shared& S,
                                            const float2* __restrict__ ps, const Row* __restrict__ rows,
                                            int nrows, float* __restrict__ acc, const float* xt, int wx) {
    const int plane = G.plane, m0 = G.m[0];
    for (int base = threadIdx.x & ~31; base < nrows; base += blockDim.x) {
        const int r = base + (threadIdx.x & 31);
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int key = -1;
        if (r < nrows) {
            const Row rr = rows[r];
            const RowRec d = decode_row(rr.idx);
            key = d.k;
            const float *gx, *dx;
            x_tables(P, S, xt, wx, d.k, gx, dx);
            const int shift = S.la_off[d.k][0] - (d.q ? P.n[0] : 0);
            const float2* vrow = ps + d.lc * plane + m0 * d.b + shift;
            float Ar = 0.f, Ai = 0.f, Br = 0.f, Bi = 0.f;
            for (int u = d.lo; u <= d.hi; u += 4) {   // four points' loads in flight at once
                float2 pv[4];
                float g1[4], g2[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool ok = u + j <= d.hi;
                    pv[j] = ok ? vrow[u + j] : make_float2(0.f, 0.f);
                    g1[j] = ok ? gx[u + j] : 0.f;
                    g2[j] = ok ? dx[u + j] : 0.f;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float gd = g2[j] * g1[j];
                    Ar += g1[j] * pv[j].x; Ai += g1[j] * pv[j].y;
                    Br += gd * pv[j].x;    Bi += gd * pv[j].y;
                }
            }
            v[0] = rr.c.x * Ar; v[1] = rr.c.x * Ai;
            v[2] = rr.c.x * Br; v[3] = rr.c.x * Bi;
            v[4] = rr.c.y * Ar; v[5] = rr.c.y * Ai;
            v[6] = rr.c.z * Ar; v[7] = rr.c.z * Ai;
        }
        if (run_sum(key, v) && key >= 0)
#pragma unroll
            for (int j = 0; j < 8; ++j) atomicAdd(acc + 8 * key + j, v[j]);
    }
}

// The same projections of x_hi (FP64, device memory, region-local) for the
// reliable update, added into acc[k][8] (device) with FP64 atomics.
__device__ __noinline__ void cl_nl_partials_x(const SolveParams& P, const Geo& G, const Shared& S,
                                              const double2* __restrict__ x, int z0, const Row* __restrict__ rows,
                                              int nrows, double* __restrict__ acc) {
    const int plane = G.plane, m0 = G.m[0];
    for (int base = threadIdx.x & ~31; base < nrows; base += blockDim.x) {
        const int r = base + (threadIdx.x & 31);
        double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int key = -1;
        if (r < nrows) {
            const RowRec d = decode_row(rows[r].idx);
            key = d.k;
            const int a = S.la_id[d.k];
            const double* gx = P.proj_g + (3LL * a + 0) * kMaxProjWin;
            const double* dx = P.proj_d + (3LL * a + 0) * kMaxProjWin;
            const int shift = S.la_off[d.k][0] - (d.q ? P.n[0] : 0);
            const double2* vrow = x + (size_t)(d.lc + z0) * plane + m0 * d.b + shift;
            double Ar = 0.0, Ai = 0.0, Br = 0.0, Bi = 0.0;
            for (int u = d.lo; u <= d.hi; ++u) {
                const double2 pv = vrow[u];
                const double g1 = __ldg(gx + u);
                const double g2 = __ldg(dx + u) * g1;
                Ar += g1 * pv.x; Ai += g1 * pv.y;
                Br += g2 * pv.x; Bi += g2 * pv.y;
            }
            const double gyz = __ldg(P.proj_g + (3LL * a + 1) * kMaxProjWin + d.vv) *
                               __ldg(P.proj_g + (3LL * a + 2) * kMaxProjWin + d.ww);
            const double ey = __ldg(P.proj_d + (3LL * a + 1) * kMaxProjWin + d.vv) * gyz;
            const double ez = __ldg(P.proj_d + (3LL * a + 2) * kMaxProjWin + d.ww) * gyz;
            v[0] = gyz * Ar; v[1] = gyz * Ai;
            v[2] = gyz * Br; v[3] = gyz * Bi;
            v[4] = ey * Ar;  v[5] = ey * Ai;
            v[6] = ez * Ar;  v[7] = ez * Ai;
        }
        if (run_sum(key, v) && key >= 0)
#pragma unroll
            for (int j = 0; j < 8; ++j) atomicAdd(acc + 8 * key + j, v[j]);
    }
}

// r(i) -= alpha sum_al E_l dV c_al p_al(i) over the own slab with
// cs[k][l] = alpha C_l E_l dV c_al (complex, float): one thread per region
// row (its records in rows_b from off_b), so each point is updated by one
// thread and needs no atomics.  Per record K1 = g_y g_z (cs_s + d_y cs_y +
// d_z cs_z), K2 = g_y g_z cs_x, and per point g_x (K1 + d_x K2).
// r(i) -= alpha sum_al E_l dV c_al p_al(i) over the own slab with
// cs[k][l] = alpha C_l E_l dV c_al (complex, float): one thread per region
// row (its records in rows_b from off[key]), so each point is updated by one
// thread and needs no atomics.  Per record K1 = g_y g_z (cs_s + d_y cs_y +
// d_z cs_z), K2 = g_y g_z cs_x, and per point g_x (K1 + d_x K2).
__device__ __noinline__ void cl_nl_scatter(const SolveParams& P, const Geo& G, const Shared& S,
                                           float2* __restrict__ rs, const Row* __restrict__ rows,
                                           const int* __restrict__ off, int nkeys, const float2 (*cs)[4],
                                           const float* xt, int wx) {
    const int plane = G.plane, m0 = G.m[0];
    for (int key = threadIdx.x; key < nkeys; key += blockDim.x) {
        const int e1 = off[key + 1];
        Row nxt = off[key] < e1 ? rows[off[key]] : Row{};
        for (int e = off[key]; e < e1; ++e) {
            const Row rr = nxt;
            if (e + 1 < e1) nxt = rows[e + 1];   // the next record is in flight while this one computes
            const RowRec d = decode_row(rr.idx);
            const float *gx, *dx;
            x_tables(P, S, xt, wx, d.k, gx, dx);
            const float2 c0 = cs[d.k][0], c1 = cs[d.k][1], c2 = cs[d.k][2], c3 = cs[d.k][3];
            const float k1r = rr.c.x * c0.x + rr.c.y * c2.x + rr.c.z * c3.x;
            const float k1i = rr.c.x * c0.y + rr.c.y * c2.y + rr.c.z * c3.y;
            const float k2r = rr.c.x * c1.x, k2i = rr.c.x * c1.y;
            const int shift = S.la_off[d.k][0] - (d.q ? P.n[0] : 0);
            float2* rrow = rs + d.lc * plane + m0 * d.b + shift;
            // four points at a time, their loads issued before any store (the
            // tables and the r slab never alias, but the compiler cannot know)
            for (int u = d.lo; u <= d.hi; u += 4) {
                float g1[4], g2[4];
                float2 v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool ok = u + j <= d.hi;
                    g1[j] = ok ? gx[u + j] : 0.f;
                    g2[j] = ok ? dx[u + j] : 0.f;
                    v[j] = ok ? rrow[u + j] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float gd = g2[j] * g1[j];
                    v[j].x -= g1[j] * k1r + gd * k2r;
                    v[j].y -= g1[j] * k1i + gd * k2i;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (u + j <= d.hi) rrow[u + j] = v[j];
            }
        }
    }
}

// p at plane c (region index) of column col: own slab from shared memory,
// the halo planes from the owning CTA's shared memory, zero outside.
__device__ __forceinline__ float2 cl_fetch(const float2* __restrict__ ps, const ClRed& H, int c, int z0, int z1,
                                           int plane, int col, int Q) {
    if (c >= z0 && c < z1) return ps[(c - z0) * plane + col];
    const float2* hp = H.hptr[c < z0 ? c - (z0 - Q) : Q + (c - z1)];
    return hp ? hp[col] : make_float2(0.f, 0.f);
}

// P2: Ap_loc = (-1/2 L + V - z) p on the own slab (Ap in device memory,
// slab-local index), accumulating p^T Ap_loc in compensated float.
template <int Q>
__device__ __forceinline__ void cl_stencil(const SolveParams& P, const Geo& G, const Shared& S,
                                           const float2* __restrict__ ps, const ClRed& H, int z0, int z1,
                                           float2* __restrict__ Ap, float zr, float zi, float diag,
                                           KSum<float>& acc_re, KSum<float>& acc_im) {
    if (z1 <= z0) return;
    const int m0 = G.m[0], m1 = G.m[1], plane = G.plane;
    float wx[Q], wy[Q], wz[Q];
#pragma unroll
    for (int o = 0; o < Q; ++o) {
        wx[o] = S.coefF[0][o];
        wy[o] = S.coefF[1][o];
        wz[o] = S.coefF[2][o];
    }
    const long long nxy = (long long)P.n[0] * P.n[1];
    const float dgb = diag - zr;
    for (int col = threadIdx.x; col < plane; col += blockDim.x) {
        const int b = (int)fdiv((uint32_t)col, G.div_row);
        const int a = col - b * m0;
        const long long vcol = wrap_once(G.lo[0] + a, P.n[0]) + (long long)P.n[0] * wrap_once(G.lo[1] + b, P.n[1]);
        float2 win[2 * Q + 1];
#pragma unroll
        for (int t = 0; t <= 2 * Q; ++t) win[t] = cl_fetch(ps, H, z0 - Q + t, z0, z1, plane, col, Q);
        // the potential three planes ahead is in flight while a plane computes
        float vq[3];
#pragma unroll
        for (int t = 0; t < 3; ++t)
            vq[t] = (z0 + t < z1) ? __ldg(P.V32 + vcol + nxy * wrap_once(G.lo[2] + z0 + t, P.n[2])) : 0.f;
        for (int z = z0; z < z1; ++z) {
            const float2* pl = ps + (z - z0) * plane + col;
            const float v = vq[0];
            vq[0] = vq[1];
            vq[1] = vq[2];
            if (z + 3 < z1) vq[2] = __ldg(P.V32 + vcol + nxy * wrap_once(G.lo[2] + z + 3, P.n[2]));
            const float2 c = win[Q];
            const float dg = dgb + v;
            float yx = dg * c.x + zi * c.y;
            float yy = dg * c.y - zi * c.x;
#pragma unroll
            for (int o = 1; o <= Q; ++o) {
                float sx = win[Q + o].x + win[Q - o].x;
                float sy = win[Q + o].y + win[Q - o].y;
                yx += wz[o - 1] * sx;
                yy += wz[o - 1] * sy;
                sx = 0.f;
                sy = 0.f;
                if (a + o < m0) {
                    const float2 t = pl[o];
                    sx += t.x;
                    sy += t.y;
                }
                if (a - o >= 0) {
                    const float2 t = pl[-o];
                    sx += t.x;
                    sy += t.y;
                }
                yx += wx[o - 1] * sx;
                yy += wx[o - 1] * sy;
                sx = 0.f;
                sy = 0.f;
                if (b + o < m1) {
                    const float2 t = pl[o * m0];
                    sx += t.x;
                    sy += t.y;
                }
                if (b - o >= 0) {
                    const float2 t = pl[-o * m0];
                    sx += t.x;
                    sy += t.y;
                }
                yx += wy[o - 1] * sx;
                yy += wy[o - 1] * sy;
            }
            Ap[(z - z0) * plane + col] = make_float2(yx, yy);
            acc_re.add(c.x * yx - c.y * yy);
            acc_im.add(c.x * yy + c.y * yx);
            if (z + 1 < z1) {
#pragma unroll
                for (int t = 0; t < 2 * Q; ++t) win[t] = win[t + 1];
                win[2 * Q] = cl_fetch(ps, H, z + Q + 1, z0, z1, plane, col, Q);
            }
        }
    }
}

// Reliable update: x_hi += dx over the own slab; after a cluster barrier
// every CTA reads x_hi across the whole region to recompute r = e_j -
// (H_R - z) x_hi in FP64 on its slab (rounded to float into the shared
// slab).  The projections of x_hi are summed slab by slab in FP64 (device
// memory, one area per CTA) and then over the cluster in rank order.  On
// return thread 0 holds the cluster totals of r^T r and ||r||^2.
template <int Q>
__device__ __noinline__ void cl_refresh(const SolveParams& P, const Geo& G, Shared& S, float2* rs,
                                        float2* dx, double2* x, double2 zd, int z0, int z1, ClRed* red,
                                        uint32_t a_red, uint32_t rank, uint32_t nrank, const Row* rows_a,
                                        double* nlp, double (&t3)[3]) {
    const int plane = G.plane, nown = (z1 - z0) * plane;
    for (int t = threadIdx.x; t < nown; t += blockDim.x) {
        const int i = z0 * plane + t;
        const float2 d = dx[t];
        double2 xv = x[i];
        xv.x += (double)d.x;
        xv.y += (double)d.y;
        x[i] = xv;
        dx[t] = make_float2(0.f, 0.f);
    }
    double* own = nlp + (size_t)rank * kLocal * 8;
    if (P.nonlocal)
        for (int t = threadIdx.x; t < 8 * S.n_local; t += blockDim.x) own[t] = 0.0;
    cl_sync();   // x_hi complete; the own projection area zeroed
    if (P.nonlocal) {
        cl_nl_partials_x(P, G, S, x, z0, rows_a, red->nrows, own);
        cl_sync();
        for (int t = threadIdx.x; t < 4 * S.n_local; t += blockDim.x) {
            const int k = t >> 2, l = t & 3;
            double sr = 0.0, si = 0.0;
            for (uint32_t q = 0; q < nrank; ++q) {
                sr += nlp[(size_t)q * kLocal * 8 + 8 * k + 2 * l];
                si += nlp[(size_t)q * kLocal * 8 + 8 * k + 2 * l + 1];
            }
            const double Cl = __ldg(P.proj_C + 4LL * S.la_id[k] + l);
            const double E = (l == 0 ? P.e_s : P.e_p) * P.dV * Cl;
            S.c[k][l] = make_double2(E * sr, E * si);
            S.cf[k][l] = make_float2((float)(E * sr), (float)(E * si));
        }
        __syncthreads();
    }
    KSum<float> q_re, q_im;
    double nrm = 0.0;
    for (int t = threadIdx.x; t < nown; t += blockDim.x) {
        const int i = z0 * plane + t;
        const double2 y = matvec_point<double, double2, Q, double2>(P, G, S, x, i, zd.x, zd.y, P.diag);
        const double tre = (i == G.src ? 1.0 : 0.0) - y.x;
        const double tim = -y.y;
        const float2 rr = make_float2((float)tre, (float)tim);
        rs[t] = rr;
        q_re.add(rr.x * rr.x - rr.y * rr.y);
        q_im.add(2.f * rr.x * rr.y);
        nrm += tre * tre + tim * tim;
    }
    t3[0] = q_re.get();
    t3[1] = q_im.get();
    t3[2] = nrm;
    block_reduce<3>(S, t3);
    if (threadIdx.x == 0) {
        red->dots[0] = t3[0];
        red->dots[1] = t3[1];
        red->dots[2] = t3[2];
    }
    cl_sync();
    if (threadIdx.x == 0) {
        double sm[3] = {0.0, 0.0, 0.0};
        for (uint32_t k = 0; k < nrank; ++k) {
            const uint32_t ra = cl_map(a_red + (uint32_t)offsetof(ClRed, dots), k);
#pragma unroll
            for (int q = 0; q < 3; ++q) sm[q] += cl_ld_f64(ra + 8u * q);
        }
        t3[0] = sm[0];
        t3[1] = sm[1];
        t3[2] = sm[2];
    }
}

template <int Q>
__global__ void __launch_bounds__(kClMaxThreads, 1) k_cocg_cl(const __grid_constant__ SolveParams P) {
    __shared__ Shared S;
    extern __shared__ __align__(16) unsigned char dsm[];
    const int tid = threadIdx.x, T = blockDim.x;
    const uint32_t rank = cl_rank(), nrank = cl_nrank();
    const ClLayout L(P.cl_slab, P.cl_xcap * 2 * P.cl_wx);
    float2* ps = reinterpret_cast<float2*>(dsm + L.p_off);
    float2* rs = reinterpret_cast<float2*>(dsm + L.r_off);
    float2* part = reinterpret_cast<float2*>(dsm + L.part_off);
    ClRed* red = reinterpret_cast<ClRed*>(dsm + L.red_off);
    float* xt_s = reinterpret_cast<float*>(dsm + L.xt_off);
    const uint32_t a_ps = smem_addr(ps), a_part = smem_addr(part), a_red = smem_addr(red);
    const uint64_t t_start = global_time_ns();
    char* slot = P.scratch + (size_t)cl_id() * P.slot_bytes;
    for (int t = tid; t < 3 * kMaxQ; t += T) {
        (&S.coefD[0][0])[t] = (&P.coef[0][0])[t];
        (&S.coefF[0][0])[t] = (float)(&P.coef[0][0])[t];
    }
    if (P.nonlocal && P.n_atoms <= kMapMax)
        for (int t = tid; t < P.n_atoms; t += T) S.map[t] = -1;
    if (tid == 0) S.n_local = 0;   // no projector atoms unless collect_local_atoms finds some
    const float diagF = (float)P.diag;
    const float eS = (float)(P.e_s * P.dV), eP = (float)(P.e_p * P.dV);

    for (;;) {
        if (rank == 0 && tid == 0) red->sys = (int)atomicAdd(P.work_counter, 1u);
        cl_sync();
        if (tid == 0) S.sys = cl_ld_s32(cl_map(a_red + (uint32_t)offsetof(ClRed, sys), 0));
        cl_sync();   // every CTA has read rank 0's slot (and may leave)
        const int s = S.sys;
        if (s >= P.n_sys) break;
        if (tid == 0) S.flag = 0;
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
        const int m2 = G.m[2], plane = G.plane;
        const int z0 = slab_start((int)rank, m2, (int)nrank), z1 = slab_start((int)rank + 1, m2, (int)nrank);
        const int nown = (z1 - z0) * plane;
        const double2 zd = P.z[sd.pole];
        const float zr = (float)zd.x, zi = (float)zd.y;
        const long long out_idx = (long long)sd.node * P.P + sd.pole;

        // slot: Ap_loc and dx of every CTA (slab-local, 16-byte aligned), x_hi,
        // then (with projectors) the FP64 projection areas and row records
        const size_t slab_even = (size_t)((P.cl_slab + 1) & ~1);
        float2* Ap = reinterpret_cast<float2*>(slot) + rank * slab_even;
        float2* dx = reinterpret_cast<float2*>(slot) + (nrank + rank) * slab_even;
        double2* x = reinterpret_cast<double2*>(reinterpret_cast<float2*>(slot) + 2 * nrank * slab_even);
        double* nlp = reinterpret_cast<double*>(x + P.n_max);
        RowLists RL;
        {
            const size_t per_cta = ((size_t)2 * P.cl_row_cap * sizeof(Row) +
                                    ((size_t)2 * P.cl_key_cap + 1) * sizeof(int) + 15) / 16 * 16;
            char* area = reinterpret_cast<char*>(nlp + (size_t)nrank * kLocal * 8) + (size_t)rank * per_cta;
            RL.rows_a = reinterpret_cast<Row*>(area);
            RL.rows_b = RL.rows_a + P.cl_row_cap;
            RL.off_b = reinterpret_cast<int*>(RL.rows_b + P.cl_row_cap);
            RL.fill_b = RL.off_b + P.cl_key_cap + 1;
            RL.cap = P.cl_row_cap;
            RL.nkeys_cap = P.cl_key_cap;
        }
        if (P.ckpt) x = P.ckpt + P.ckpt_sys_off[out_idx];

        if (tid < 2 * P.q) {   // halo planes of this slab
            const int t = tid;
            const int c = t < P.q ? z0 - P.q + t : z1 + (t - P.q);
            const float2* hp = nullptr;
            if (c >= 0 && c < m2) {
                const int k = slab_owner(c, m2, (int)nrank);
                hp = cl_map_ptr(ps + (size_t)(c - slab_start(k, m2, (int)nrank)) * plane, (uint32_t)k);
            }
            red->hptr[t] = hp;
        }
        if (tid == 0) red->nrows = 0;
        if (P.nonlocal) {
            collect_local_atoms(P, G, S);
            int* cnt = reinterpret_cast<int*>(dsm + L.cnt_off);
            cl_build_rows(P, G, S, z0, z1, RL, cnt, cnt + kLocal + 1, &red->nrows);
            __syncthreads();
            if (tid == 0 && red->nrows > P.cl_row_cap) {   // cannot happen with the host's bounds; stay in bounds
                red->nrows = 0;
                S.flag = 1;
            }
            // the local atoms' x tables (g_x, d_x g_x's d_x) in shared memory when they fit
            if (S.n_local <= P.cl_xcap)
                for (int t = tid; t < S.n_local * P.cl_wx; t += T) {
                    const int k = t / P.cl_wx, u = t - k * P.cl_wx;
                    const long long a = S.la_id[k];
                    xt_s[2 * P.cl_wx * k + u] = __ldg(P.proj_g32 + 3LL * a * kMaxProjWin + u);
                    xt_s[2 * P.cl_wx * k + P.cl_wx + u] = __ldg(P.proj_d32 + 3LL * a * kMaxProjWin + u);
                }
            __syncthreads();
        }
        for (int t = tid; t < nown; t += T) {
            const int i = z0 * plane + t;
            rs[t] = make_float2(i == G.src ? 1.f : 0.f, 0.f);
            ps[t] = make_float2(0.f, 0.f);
            x[i] = make_double2(0.0, 0.0);
            dx[t] = make_float2(0.f, 0.f);
        }
        if (tid == 0) {
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
            if (tid == 0 && S.it >= P.maxit) S.action = kStop;
            __syncthreads();
            if (S.action == kStop || S.action == kStopTimeout) break;
            {   // P1: p = r + beta p (two complex64 per 16-byte access)
                const float br = (float)S.beta[0], bi = (float)S.beta[1];
                const float4* r4 = reinterpret_cast<const float4*>(rs);
                float4* p4 = reinterpret_cast<float4*>(ps);
                for (int k = tid; k < (nown >> 1); k += T) {
                    const float4 a = r4[k], b = p4[k];
                    p4[k] = make_float4(a.x + br * b.x - bi * b.y, a.y + br * b.y + bi * b.x,
                                        a.z + br * b.z - bi * b.w, a.w + br * b.w + bi * b.z);
                }
                if ((nown & 1) && tid == 0) {
                    const float2 ri = rs[nown - 1], pi = ps[nown - 1];
                    ps[nown - 1] = make_float2(ri.x + br * pi.x - bi * pi.y, ri.y + br * pi.y + bi * pi.x);
                }
                if (P.nonlocal) {
                    float* acc8 = reinterpret_cast<float*>(part);
                    for (int t = tid; t < 8 * S.n_local; t += T) acc8[t] = 0.f;
                }
            }
            cl_sync();
            if (P.nonlocal)
                cl_nl_partials(P, G, S, ps, RL.rows_a, red->nrows, reinterpret_cast<float*>(part),
                               S.n_local <= P.cl_xcap ? xt_s : nullptr, P.cl_wx);
            double pap[2];
            {
                KSum<float> acc_re, acc_im;
                cl_stencil<Q>(P, G, S, ps, *red, z0, z1, Ap, zr, zi, diagF, acc_re, acc_im);
                const float hi[2] = {acc_re.hi(), acc_im.hi()}, lo[2] = {acc_re.lo(), acc_im.lo()};
                block_reduce_ff<2>(S, hi, lo, pap);
            }
            if (tid == 0) {
                red->pap[0] = pap[0];
                red->pap[1] = pap[1];
                red->timeout = (rank == 0 && P.timeout_ns && (global_time_ns() - t_start) > P.timeout_ns) ? 1 : 0;
            }
            cl_sync();
            // every CTA sums the partials of every rank in rank order
            if (tid == 0) {
                double s0 = 0.0, s1 = 0.0;
                for (uint32_t k = 0; k < nrank; ++k) {
                    const uint32_t ra = cl_map(a_red + (uint32_t)offsetof(ClRed, pap), k);
                    s0 += cl_ld_f64(ra);
                    s1 += cl_ld_f64(ra + 8u);
                }
                S.bcast[0] = s0;
                S.bcast[1] = s1;
                S.bcast[2] = (double)cl_ld_s32(cl_map(a_red + (uint32_t)offsetof(ClRed, timeout), 0));
            }
            double pn[2] = {0.0, 0.0};
            if (P.nonlocal) {
                // FP32 products and compensated partial sums, as in the local
                // part of p^T A p; FP64 from the per-thread partial upward
                KSum<float> pn_re, pn_im;
                for (int t = tid; t < 4 * S.n_local; t += T) {
                    const int k = t >> 2, l = t & 3;
                    float sr = 0.f, si = 0.f;
                    for (uint32_t q = 0; q < nrank; ++q) {
                        const float2 v = cl_ld_f2(cl_map(a_part + 8u * (uint32_t)t, q));
                        sr += v.x;
                        si += v.y;
                    }
                    // c_al = C_l sum f_al p; S.cf = E_l dV c_al, the bilinear
                    // energy E_l dV c_al^2
                    const float Cl = __ldg(P.proj_C32 + 4LL * S.la_id[k] + l);
                    const float E = (l == 0 ? eS : eP) * Cl;
                    S.cf[k][l] = make_float2(E * sr, E * si);
                    pn_re.add(E * Cl * (sr * sr - si * si));
                    pn_im.add(E * Cl * 2.f * sr * si);
                }
                const float hi[2] = {pn_re.hi(), pn_im.hi()}, lo[2] = {pn_re.lo(), pn_im.lo()};
                block_reduce_ff<2>(S, hi, lo, pn);
            }
            if (tid == 0) {
                ++S.it;
                const double pr = S.bcast[0] + pn[0], pim = S.bcast[1] + pn[1];
                const double den = pr * pr + pim * pim;
                if (S.bcast[2] != 0.0) {
                    S.action = kStopTimeout;
                } else if (!(den > 0.0)) {
                    S.st = 3;
                    S.action = kStop;
                } else {
                    S.alpha[0] = (S.rho[0] * pr + S.rho[1] * pim) / den;
                    S.alpha[1] = (S.rho[1] * pr - S.rho[0] * pim) / den;
                }
            }
            __syncthreads();
            if (S.action == kStop || S.action == kStopTimeout) break;
            const double al_re = S.alpha[0], al_im = S.alpha[1];
            if (P.nonlocal) {
                // alpha C_l E_l dV c_al per (atom, shape), in place of S.cf
                const float ar = (float)al_re, ai = (float)al_im;
                for (int t = tid; t < 4 * S.n_local; t += T) {
                    const int k = t >> 2, l = t & 3;
                    const float Cl = __ldg(P.proj_C32 + 4LL * S.la_id[k] + l);
                    const float2 c = S.cf[k][l];
                    S.cf[k][l] = make_float2(Cl * (ar * c.x - ai * c.y), Cl * (ar * c.y + ai * c.x));
                }
                __syncthreads();
                cl_nl_scatter(P, G, S, rs, RL.rows_b, RL.off_b, red->nrows ? (z1 - z0) * G.m[1] : 0, S.cf,
                              S.n_local <= P.cl_xcap ? xt_s : nullptr, P.cl_wx);
                __syncthreads();
            }
            double red3[3];
            {   // P3: dx += alpha p ; r -= alpha Ap_loc ; r^T r ; |r|^2 (two points per 16-byte access)
                const float ar = (float)al_re, ai = (float)al_im;
                KSum<float> s_re, s_im, s_n;
                const float4* p4 = reinterpret_cast<const float4*>(ps);
                const float4* q4 = reinterpret_cast<const float4*>(Ap);
                float4* d4 = reinterpret_cast<float4*>(dx);
                float4* r4 = reinterpret_cast<float4*>(rs);
                const int npair = nown >> 1;
                // two pairs per trip, all loads (two of them from device
                // memory) issued before the arithmetic
                for (int k = tid; k < npair; k += 2 * T) {
                    const int kk[2] = {k, k + T};
                    float4 pv[2], qv[2], d[2], rv[2];
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const bool ok = kk[j] < npair;
                        const int kj = ok ? kk[j] : k;
                        pv[j] = p4[kj];
                        qv[j] = q4[kj];
                        d[j] = d4[kj];
                        rv[j] = r4[kj];
                    }
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        if (kk[j] >= npair) break;
                        d[j].x += ar * pv[j].x - ai * pv[j].y;
                        d[j].y += ar * pv[j].y + ai * pv[j].x;
                        d[j].z += ar * pv[j].z - ai * pv[j].w;
                        d[j].w += ar * pv[j].w + ai * pv[j].z;
                        rv[j].x -= ar * qv[j].x - ai * qv[j].y;
                        rv[j].y -= ar * qv[j].y + ai * qv[j].x;
                        rv[j].z -= ar * qv[j].z - ai * qv[j].w;
                        rv[j].w -= ar * qv[j].w + ai * qv[j].z;
                        d4[kk[j]] = d[j];
                        r4[kk[j]] = rv[j];
                        s_re.add(rv[j].x * rv[j].x - rv[j].y * rv[j].y + (rv[j].z * rv[j].z - rv[j].w * rv[j].w));
                        s_im.add(2.f * (rv[j].x * rv[j].y + rv[j].z * rv[j].w));
                        s_n.add(rv[j].x * rv[j].x + rv[j].y * rv[j].y + (rv[j].z * rv[j].z + rv[j].w * rv[j].w));
                    }
                }
                if ((nown & 1) && tid == 0) {
                    const int t = nown - 1;
                    const float2 pv = ps[t], qv = Ap[t];
                    float2 d = dx[t], rv = rs[t];
                    d.x += ar * pv.x - ai * pv.y;
                    d.y += ar * pv.y + ai * pv.x;
                    rv.x -= ar * qv.x - ai * qv.y;
                    rv.y -= ar * qv.y + ai * qv.x;
                    dx[t] = d;
                    rs[t] = rv;
                    s_re.add(rv.x * rv.x - rv.y * rv.y);
                    s_im.add(2.f * rv.x * rv.y);
                    s_n.add(rv.x * rv.x + rv.y * rv.y);
                }
                const float hi3[3] = {s_re.hi(), s_im.hi(), s_n.hi()};
                const float lo3[3] = {s_re.lo(), s_im.lo(), s_n.lo()};
                block_reduce_ff<3>(S, hi3, lo3, red3);
            }
            if (tid == 0) {
                red->dots[0] = red3[0];
                red->dots[1] = red3[1];
                red->dots[2] = red3[2];
            }
            cl_sync();
            if (tid == 0) {
                double sm[3] = {0.0, 0.0, 0.0};
                for (uint32_t k = 0; k < nrank; ++k) {
                    const uint32_t ra = cl_map(a_red + (uint32_t)offsetof(ClRed, dots), k);
#pragma unroll
                    for (int q = 0; q < 3; ++q) sm[q] += cl_ld_f64(ra + 8u * q);
                }
                red3[0] = sm[0];
                red3[1] = sm[1];
                red3[2] = sm[2];
                const double rn = sqrt(red3[2]);
                const bool want = (rn <= P.tol) || (S.it - S.last_rel >= P.reliable_every) ||
                                  (rn < P.reliable_delta * S.rn_last);
                S.action = want ? kRefresh : 0;
            }
            __syncthreads();
            if (S.action == kRefresh) {
                cl_refresh<Q>(P, G, S, rs, dx, x, zd, z0, z1, red, a_red, rank, nrank, RL.rows_a, nlp, red3);
                if (tid == 0) {
                    const double rt = sqrt(red3[2]);
                    S.restart = (S.n_rel > 0 && rt >= S.rn_last) ? 1 : 0;
                    S.rn_last = rt;
                    S.last_rel = S.it;
                    ++S.n_rel;
                }
            }
            if (tid == 0) {
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
            for (int t = tid; t < nown; t += T) {
                const int i = z0 * plane + t;
                const float2 d = dx[t];
                double2 xv = x[i];
                xv.x += (double)d.x;
                xv.y += (double)d.y;
                x[i] = xv;
            }
        }
        cl_sync();   // x_hi complete across the cluster
        if (P.fused_dLdV) {
            const double aj = P.fused_a ? P.fused_a[sd.node] : 0.0;
            const double bj = P.fused_b ? P.fused_b[sd.node] : 0.0;
            const double2 wp = P.w[sd.pole];
            const double cr = 2.0 * aj / P.dV + 2.0 * bj * zd.x, ci = 2.0 * bj * zd.y;
            const double c_re = cr * wp.x - ci * wp.y, c_im = cr * wp.y + ci * wp.x;
            for (int t = tid; t < nown; t += T) {
                const int i = z0 * plane + t;
                const int c = (int)fdiv((uint32_t)i, G.div_plane);
                const int rem = i - c * plane;
                const int b = (int)fdiv((uint32_t)rem, G.div_row);
                const int a = rem - b * G.m[0];
                const long long gi = wrap_once(G.lo[0] + a, P.n[0]) +
                                     (long long)P.n[0] * (wrap_once(G.lo[1] + b, P.n[1]) +
                                                          (long long)P.n[1] * wrap_once(G.lo[2] + c, P.n[2]));
                const double2 xv = x[i];
                const double sq_re = xv.x * xv.x - xv.y * xv.y, sq_im = 2.0 * xv.x * xv.y;
                atomicAdd(P.fused_dLdV + gi, -(c_re * sq_im + c_im * sq_re));
            }
        }
        if (P.dm_rows) {
            const double2 wp = P.w[sd.pole];
            double* row = P.dm_rows + P.dm_off[sd.node];
            for (int t = tid; t < nown; t += T) {
                const int i = z0 * plane + t;
                const double2 xv = x[i];
                atomicAdd(row + i, wp.x * xv.y + wp.y * xv.x);
            }
        }
        if (rank == 0 && tid == 0) {
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

template <int Q>
cudaError_t launch_cl_q(const SolveParams& P, int csz, int grid, int block, size_t smem, cudaStream_t s) {
    // the attribute is set outside stream capture (cl_max_clusters sets it
    // when the plan is made)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusNone) {
        e = cudaFuncSetAttribute(k_cocg_cl<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csz;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_cocg_cl<Q>, P);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int Q>
int cl_clusters_q(int csz, int block, size_t smem) {
    if (cudaFuncSetAttribute(k_cocg_cl<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)csz);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csz;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_cocg_cl<Q>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace

bool cl_supported(int precision, int q) { return precision == MD_PREC_MIXED && q >= 1 && q <= 4; }

int cl_max_threads() { return kClMaxThreads; }

size_t cl_smem_bytes(int slab_pts, int xtab_floats) { return ClLayout(slab_pts, xtab_floats).total; }

size_t cl_static_smem_bytes() { return sizeof(Shared); }

int cl_max_clusters(int q, int csz, int block, size_t smem) {
    switch (q) {
        case 1: return cl_clusters_q<1>(csz, block, smem);
        case 2: return cl_clusters_q<2>(csz, block, smem);
        case 3: return cl_clusters_q<3>(csz, block, smem);
        case 4: return cl_clusters_q<4>(csz, block, smem);
        default: return 0;
    }
}

cudaError_t launch_cocg_cl(const SolveParams& P, int csz, int grid, int block, size_t smem, cudaStream_t s) {
    switch (P.q) {
        case 1: return launch_cl_q<1>(P, csz, grid, block, smem, s);
        case 2: return launch_cl_q<2>(P, csz, grid, block, smem, s);
        case 3: return launch_cl_q<3>(P, csz, grid, block, smem, s);
        case 4: return launch_cl_q<4>(P, csz, grid, block, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

size_t cl_slot_bytes(long long n_max, int csz, int slab_pts, int nonlocal, int row_cap, int key_cap) {
    const size_t nm = (size_t)((n_max + 63) / 64 * 64);
    const size_t se = (size_t)((slab_pts + 1) & ~1);
    size_t b = 2 * (size_t)csz * se * sizeof(float2) + nm * sizeof(double2);
    if (nonlocal) {
        const size_t per_cta =
            ((size_t)2 * row_cap * sizeof(Row) + ((size_t)2 * key_cap + 1) * sizeof(int) + 15) / 16 * 16;
        b += (size_t)csz * kLocal * 8 * sizeof(double) + (size_t)csz * per_cta;
    }
    return (b + 255) / 256 * 256;
}

}  // namespace md
