// Hamiltonian build on the device (md_build_hamiltonian, md_spectral_bounds).
//
// H = -1/2 L_FD + diag(V) + sum_{a,l} E_l dV |p_al><p_al|   (the paper's
// Eq. (Hamiltonian) on the finite-difference grid of Section 2.1, with a
// synthetic local potential and separable Gaussian projectors).
//
//   V(r_i)   = v_ext(r_i) + sum_a -D_a exp(-|r_i - R_a|^2 / (2 sigma_a^2))
//              (minimum image on periodic axes, cut at cutoff_sigmas*sigma)
//   p_s      = C_s g,  p_alpha = C_alpha (r_alpha - R_alpha) g,
//   g        = exp(-|r - R|^2/(2 proj_sigma^2)), zero beyond proj_rc,
//   C        = 1/sqrt(dV sum_i f_i^2) for each of the four shapes f.
//
// Atoms are binned in a host-built cell list (cells no smaller than the
// largest cutoff) so each grid point visits only neighbouring cells.  The
// Gaussian is separable, so each atom's projector window is stored as 1-D
// tables of displacements d and factors exp(-d^2/(2 s^2)) per axis; the
// solver rebuilds p_l(r) = C_l * (d_x or 1) * g_x g_y g_z from them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "md_device.cuh"
#include "md_internal.h"

namespace md {

namespace {

struct CellList {
    int nc[3];
    double cell[3];
    int* start = nullptr;  // [ncell + 1]
    int* atoms = nullptr;  // [n_atoms] atom ids grouped by cell
};

struct GridGeo {
    int n[3];
    double h[3];
    double L[3];
    int periodic[3];
};

__device__ __forceinline__ double min_image(double d, double L, int periodic) {
    return periodic ? d - L * rint(d / L) : d;
}

// Visit every atom in the cells around grid point (ix, iy, iz).
template <class F>
__device__ __forceinline__ void for_each_near_atom(const GridGeo& g, const int* nc, const double* cell,
                                                   const int* cstart, const int* catoms, int ix,
                                                   int iy, int iz, F&& f) {
    const int pc[3] = {min(max((int)floor(ix * g.h[0] / cell[0]), 0), nc[0] - 1),
                       min(max((int)floor(iy * g.h[1] / cell[1]), 0), nc[1] - 1),
                       min(max((int)floor(iz * g.h[2] / cell[2]), 0), nc[2] - 1)};
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        if (g.periodic[d] && nc[d] < 3) {
            lo[d] = 0;
            hi[d] = nc[d] - 1;
        } else {
            lo[d] = pc[d] - 1;
            hi[d] = pc[d] + 1;
        }
    }
    for (int cz = lo[2]; cz <= hi[2]; ++cz) {
        int wz = cz;
        if (g.periodic[2] && nc[2] >= 3) wz = (cz + nc[2]) % nc[2];
        else if (wz < 0 || wz >= nc[2]) continue;
        for (int cy = lo[1]; cy <= hi[1]; ++cy) {
            int wy = cy;
            if (g.periodic[1] && nc[1] >= 3) wy = (cy + nc[1]) % nc[1];
            else if (wy < 0 || wy >= nc[1]) continue;
            for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                int wx = cx;
                if (g.periodic[0] && nc[0] >= 3) wx = (cx + nc[0]) % nc[0];
                else if (wx < 0 || wx >= nc[0]) continue;
                const int c = wx + nc[0] * (wy + nc[1] * wz);
                for (int e = cstart[c]; e < cstart[c + 1]; ++e) f(catoms[e]);
            }
        }
    }
}

struct CellArgs {
    int nc[3];
    double cell[3];
    const int* start;
    const int* atoms;
};

__global__ void k_local_potential(GridGeo g, CellArgs cl, const double* __restrict__ xyz,
                                  const double* __restrict__ depth, const double* __restrict__ sigma,
                                  double cutoff_sigmas, const double* __restrict__ v_ext,
                                  double* __restrict__ V, float* __restrict__ V32, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % g.n[0]);
        const int iy = (int)((i / g.n[0]) % g.n[1]);
        const int iz = (int)(i / ((long long)g.n[0] * g.n[1]));
        const double px = ix * g.h[0], py = iy * g.h[1], pz = iz * g.h[2];
        double v = v_ext ? v_ext[i] : 0.0;
        for_each_near_atom(g, cl.nc, cl.cell, cl.start, cl.atoms, ix, iy, iz, [&](int a) {
            const double dx = min_image(px - xyz[3 * a + 0], g.L[0], g.periodic[0]);
            const double dy = min_image(py - xyz[3 * a + 1], g.L[1], g.periodic[1]);
            const double dz = min_image(pz - xyz[3 * a + 2], g.L[2], g.periodic[2]);
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double s = sigma[a];
            const double rc = cutoff_sigmas * s;
            if (r2 <= rc * rc) v -= depth[a] * exp(-r2 / (2.0 * s * s));
        });
        V[i] = v;
        V32[i] = (float)v;
    }
}

// One thread per (atom, axis, window slot): displacement and Gaussian factor.
__global__ void k_proj_tables(GridGeo g, const double* __restrict__ xyz, long long n_atoms,
                              double rc, double psig, int* i0, int* len, double* dtab, double* gtab,
                              float* dtab32, float* gtab32) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n_atoms * 3 * kMaxProjWin) return;
    const int u = (int)(t % kMaxProjWin);
    const int d = (int)((t / kMaxProjWin) % 3);
    const long long a = t / (3 * kMaxProjWin);
    const double X = xyz[3 * a + d];
    const int start = (int)ceil((X - rc) / g.h[d]);
    const int stop = (int)floor((X + rc) / g.h[d]);
    if (u == 0) {
        i0[3 * a + d] = start;
        len[3 * a + d] = stop - start + 1;
    }
    const double dd = (start + u) * g.h[d] - X;
    const double gg = (start + u <= stop) ? exp(-dd * dd / (2.0 * psig * psig)) : 0.0;
    dtab[t] = dd;
    gtab[t] = gg;
    dtab32[t] = (float)dd;
    gtab32[t] = (float)gg;
}

// One thread per (atom, v, w): the window slots u of row (v, w) inside the
// sphere form one interval [lo, hi] (d_u^2 is convex in u); hi < lo if empty.
// This FP64 test is the single definition of projector support used by the
// normalisation, the per-point lists and the solver.
__global__ void k_proj_rows(const int* __restrict__ len, const double* __restrict__ dtab,
                            long long n_atoms, double rc, unsigned char* rows) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n_atoms * kMaxProjWin * kMaxProjWin) return;
    const int v = (int)(t % kMaxProjWin);
    const int w = (int)((t / kMaxProjWin) % kMaxProjWin);
    const long long a = t / ((long long)kMaxProjWin * kMaxProjWin);
    const int lx = len[3 * a], ly = len[3 * a + 1], lz = len[3 * a + 2];
    int lo = 1, hi = 0;
    if (v < ly && w < lz) {
        const double* dx = dtab + (3 * a + 0) * kMaxProjWin;
        const double dy = dtab[(3 * a + 1) * kMaxProjWin + v];
        const double dz = dtab[(3 * a + 2) * kMaxProjWin + w];
        int first = -1, last = -2;
        for (int u = 0; u < lx; ++u) {
            if (dx[u] * dx[u] + dy * dy + dz * dz <= rc * rc) {
                if (first < 0) first = u;
                last = u;
            }
        }
        if (first >= 0) {
            lo = first;
            hi = last;
        }
    }
    rows[2 * t + 0] = (unsigned char)lo;
    rows[2 * t + 1] = (unsigned char)hi;
}

// One block per atom: sums of f^2 and |f| over the sphere for the 4 shapes.
__global__ void k_proj_norms(const int* __restrict__ len, const double* __restrict__ dtab,
                             const double* __restrict__ gtab, const unsigned char* __restrict__ rows,
                             double dV, double* C, float* C32, double* absum) {
    const long long a = blockIdx.x;
    const int lx = len[3 * a], ly = len[3 * a + 1], lz = len[3 * a + 2];
    const double* dx = dtab + (3 * a + 0) * kMaxProjWin;
    const double* dy = dtab + (3 * a + 1) * kMaxProjWin;
    const double* dz = dtab + (3 * a + 2) * kMaxProjWin;
    const double* gx = gtab + (3 * a + 0) * kMaxProjWin;
    const double* gy = gtab + (3 * a + 1) * kMaxProjWin;
    const double* gz = gtab + (3 * a + 2) * kMaxProjWin;
    double s2[4] = {0, 0, 0, 0}, s1[4] = {0, 0, 0, 0};
    const int n = lx * ly * lz;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int u = i % lx, v = (i / lx) % ly, w = i / (lx * ly);
        const unsigned char* rw = rows + 2 * ((a * kMaxProjWin + w) * kMaxProjWin + v);
        if (u < rw[0] || u > rw[1]) continue;
        const double gg = gx[u] * gy[v] * gz[w];
        const double f[4] = {gg, dx[u] * gg, dy[v] * gg, dz[w] * gg};
        for (int k = 0; k < 4; ++k) {
            s2[k] += f[k] * f[k];
            s1[k] += fabs(f[k]);
        }
    }
    __shared__ double red[8][32];
    for (int k = 0; k < 4; ++k) {
        s2[k] = warp_sum(s2[k]);
        s1[k] = warp_sum(s1[k]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) {
            red[k][warp] = s2[k];
            red[4 + k][warp] = s1[k];
        }
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        red[threadIdx.x][0] = s;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const double c = 1.0 / sqrt(dV * red[threadIdx.x][0]);
        C[4 * a + threadIdx.x] = c;
        C32[4 * a + threadIdx.x] = (float)c;
        absum[4 * a + threadIdx.x] = c * red[4 + threadIdx.x][0];
    }
}

// Window slot of grid coordinate i for a window starting at (unwrapped) i0
// of length len on an axis of n points; -1 when outside the window.
__device__ __forceinline__ int window_slot(int i, int i0, int len, int n, int periodic) {
    int u = i - i0;
    if (periodic) {
        u %= n;
        if (u < 0) u += n;
    }
    return (u >= 0 && u < len) ? u : -1;
}

// Per grid point: atoms whose projector support contains the point (the
// row-interval test above), ascending atom id.  The fill pass also stores
// the four normalised projector values at the point (FP64 and FP32).
template <bool kFill>
__global__ void k_proj_lists(GridGeo g, CellArgs cl, const int* __restrict__ i0,
                             const int* __restrict__ len, const unsigned char* __restrict__ rows,
                             const double* __restrict__ dtab, const double* __restrict__ gtab,
                             const double* __restrict__ C, long long N, int* __restrict__ count_or_ptr,
                             int* __restrict__ out_atoms, double2* __restrict__ val64,
                             float4* __restrict__ val32, int* __restrict__ overflow) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % g.n[0]);
        const int iy = (int)((i / g.n[0]) % g.n[1]);
        const int iz = (int)(i / ((long long)g.n[0] * g.n[1]));
        int ids[16];
        int cnt = 0;
        for_each_near_atom(g, cl.nc, cl.cell, cl.start, cl.atoms, ix, iy, iz, [&](int a) {
            const int u = window_slot(ix, i0[3 * a + 0], len[3 * a + 0], g.n[0], g.periodic[0]);
            const int v = window_slot(iy, i0[3 * a + 1], len[3 * a + 1], g.n[1], g.periodic[1]);
            const int w = window_slot(iz, i0[3 * a + 2], len[3 * a + 2], g.n[2], g.periodic[2]);
            if (u < 0 || v < 0 || w < 0) return;
            const unsigned char* rw = rows + 2 * (((long long)a * kMaxProjWin + w) * kMaxProjWin + v);
            if (u < rw[0] || u > rw[1]) return;
            if (cnt < 16) ids[cnt] = a;
            ++cnt;
        });
        if (!kFill) {
            count_or_ptr[i] = cnt;
            if (cnt > 16) atomicExch(overflow, 1);
        } else {
            const int m = cnt < 16 ? cnt : 16;
            for (int x = 1; x < m; ++x) {  // insertion sort, ascending atom id
                const int v = ids[x];
                int y = x - 1;
                while (y >= 0 && ids[y] > v) {
                    ids[y + 1] = ids[y];
                    --y;
                }
                ids[y + 1] = v;
            }
            const long long base = count_or_ptr[i];
            const int pi[3] = {ix, iy, iz};
            for (int x = 0; x < m; ++x) {
                const int a = ids[x];
                out_atoms[base + x] = a;
                int uu[3];
                for (int d = 0; d < 3; ++d)
                    uu[d] = window_slot(pi[d], i0[3 * a + d], len[3 * a + d], g.n[d], g.periodic[d]);
                const double* dt = dtab + 3 * (long long)a * kMaxProjWin;
                const double* gt = gtab + 3 * (long long)a * kMaxProjWin;
                const double gg = gt[uu[0]] * gt[kMaxProjWin + uu[1]] * gt[2 * kMaxProjWin + uu[2]];
                const double p0 = C[4 * a + 0] * gg;
                const double p1 = C[4 * a + 1] * dt[uu[0]] * gg;
                const double p2 = C[4 * a + 2] * dt[kMaxProjWin + uu[1]] * gg;
                const double p3 = C[4 * a + 3] * dt[2 * kMaxProjWin + uu[2]] * gg;
                val64[2 * (base + x) + 0] = make_double2(p0, p1);
                val64[2 * (base + x) + 1] = make_double2(p2, p3);
                val32[base + x] = make_float4((float)p0, (float)p1, (float)p2, (float)p3);
            }
        }
    }
}

// Per grid point Gershgorin disc; per block min of (diag - radius) and
// max of (diag + radius).
__global__ void k_gershgorin(GridGeo g, const double* __restrict__ V, double diag0, double rad0,
                             long long N, int nonlocal, const int* __restrict__ pl_ptr,
                             const int* __restrict__ pl_atom, const int* __restrict__ i0,
                             const int* __restrict__ len, const double* __restrict__ dtab,
                             const double* __restrict__ gtab, const double* __restrict__ C,
                             const double* __restrict__ absum, double rc, double Es, double Ep,
                             double dV, double* blk_lo, double* blk_hi) {
    double lo = 1e300, hi = -1e300;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        double dg = diag0 + V[i];
        double rad = rad0;
        if (nonlocal) {
            const int ix = (int)(i % g.n[0]);
            const int iy = (int)((i / g.n[0]) % g.n[1]);
            const int iz = (int)(i / ((long long)g.n[0] * g.n[1]));
            const int pi[3] = {ix, iy, iz};
            for (int e = pl_ptr[i]; e < pl_ptr[i + 1]; ++e) {
                const int a = pl_atom[e];
                int uu[3];
                for (int d = 0; d < 3; ++d)
                    uu[d] = window_slot(pi[d], i0[3 * a + d], len[3 * a + d], g.n[d], g.periodic[d]);
                const double* dt = dtab + 3 * (long long)a * kMaxProjWin;
                const double* gt = gtab + 3 * (long long)a * kMaxProjWin;
                const double gg = gt[uu[0]] * gt[kMaxProjWin + uu[1]] * gt[2 * kMaxProjWin + uu[2]];
                const double f[4] = {gg, dt[uu[0]] * gg, dt[kMaxProjWin + uu[1]] * gg,
                                     dt[2 * kMaxProjWin + uu[2]] * gg};
                for (int k = 0; k < 4; ++k) {
                    const double E = k == 0 ? Es : Ep;
                    const double p = C[4 * a + k] * f[k];
                    dg += E * dV * p * p;
                    rad += fabs(E) * dV * fabs(p) * (absum[4 * a + k] - fabs(p));
                }
            }
        }
        lo = fmin(lo, dg - rad);
        hi = fmax(hi, dg + rad);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    __shared__ double slo[32], shi[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        slo[warp] = lo;
        shi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = fmin(lo, slo[w]);
            hi = fmax(hi, shi[w]);
        }
        blk_lo[blockIdx.x] = lo;
        blk_hi[blockIdx.x] = hi;
    }
}

GridGeo geo_of(const Ham& H) {
    GridGeo g;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = H.n[d];
        g.h[d] = H.h[d];
        g.L[d] = H.n[d] * H.h[d];
        g.periodic[d] = H.periodic[d];
    }
    return g;
}

// Host cell list.  Cell size >= rcut so neighbours lie in the 27 cells around.
md_status build_cells(const Ham& H, const std::vector<double>& xyz, double rcut,
                      std::vector<int>& start, std::vector<int>& ids, int nc[3], double cell[3]) {
    for (int d = 0; d < 3; ++d) {
        const double L = H.n[d] * H.h[d];
        int c = (int)std::floor(L / rcut);
        c = std::max(1, std::min(c, 512));
        nc[d] = c;
        cell[d] = L / c;
    }
    const long long ncell = (long long)nc[0] * nc[1] * nc[2];
    const long long na = H.n_atoms;
    std::vector<long long> cid(na);
    std::vector<int> cnt(ncell + 1, 0);
    for (long long a = 0; a < na; ++a) {
        long long c = 0, mul = 1;
        for (int d = 0; d < 3; ++d) {
            const double L = H.n[d] * H.h[d];
            double x = xyz[3 * a + d];
            if (H.periodic[d]) x = x - L * std::floor(x / L);
            int k = (int)std::floor(x / cell[d]);
            k = std::max(0, std::min(k, nc[d] - 1));
            c += k * mul;
            mul *= nc[d];
        }
        cid[a] = c;
        cnt[c + 1]++;
    }
    start.assign(ncell + 1, 0);
    for (long long c = 0; c < ncell; ++c) start[c + 1] = start[c] + cnt[c + 1];
    ids.assign(na > 0 ? na : 1, 0);
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (long long a = 0; a < na; ++a) ids[fill[cid[a]]++] = (int)a;
    return MD_OK;
}

}  // namespace

#define MD_CUDA_TRY(expr)                                                                 \
    do {                                                                                  \
        cudaError_t _e = (expr);                                                          \
        if (_e != cudaSuccess) {                                                          \
            st = (_e == cudaErrorMemoryAllocation) ? MD_ERR_OOM : MD_ERR_CUDA;            \
            set_error(st, std::string("CUDA: ") + cudaGetErrorString(_e) + " at " #expr); \
            goto fail;                                                                    \
        }                                                                                 \
    } while (0)

__global__ void k_set_potential(const double* __restrict__ Vin, double* __restrict__ V,
                                float* __restrict__ V32, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = Vin[i];
        V[i] = v;
        V32[i] = (float)v;
    }
}

md_status set_potential_device(Ham& H, const double* V_in, void* stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    const int blocks = (int)std::min<long long>((H.N + 255) / 256, 152LL * 32);
    k_set_potential<<<blocks, 256, 0, stream>>>(V_in, H.V, H.V32, H.N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    H.bounds_valid = false;
    return compute_bounds(H, stream_);
}

md_status compute_bounds(Ham& H, void* stream_) {
    md_status st = MD_OK;
    cudaStream_t stream = (cudaStream_t)stream_;
    const long long N = H.N;
    GridGeo g = geo_of(H);
    const int threads = 256;
    double rad0 = 0.0;
    for (int d = 0; d < 3; ++d)
        for (int o = 0; o < H.q; ++o) rad0 += 2.0 * std::fabs(H.coef[d][o]);
    const int gb = (int)std::min<long long>((N + threads - 1) / threads, 152LL * 16);
    double* d_lo = nullptr;
    double* d_hi = nullptr;
    std::vector<double> lo(gb), hi(gb);
    double a = 1e300, b = -1e300;
    MD_CUDA_TRY(cudaMalloc(&d_lo, gb * sizeof(double)));
    MD_CUDA_TRY(cudaMalloc(&d_hi, gb * sizeof(double)));
    k_gershgorin<<<gb, threads, 0, stream>>>(g, H.V, H.diag, rad0, N, H.nonlocal && H.n_atoms > 0,
                                             H.pl_ptr, H.pl_atom, H.proj_i0, H.proj_len, H.proj_d,
                                             H.proj_g, H.proj_C, H.proj_absum, H.proj_rc, H.e_s,
                                             H.e_p, H.dV, d_lo, d_hi);
    MD_CUDA_TRY(cudaGetLastError());
    MD_CUDA_TRY(cudaMemcpyAsync(lo.data(), d_lo, gb * sizeof(double), cudaMemcpyDeviceToHost, stream));
    MD_CUDA_TRY(cudaMemcpyAsync(hi.data(), d_hi, gb * sizeof(double), cudaMemcpyDeviceToHost, stream));
    MD_CUDA_TRY(cudaStreamSynchronize(stream));
    for (int i = 0; i < gb; ++i) {
        a = std::min(a, lo[i]);
        b = std::max(b, hi[i]);
    }
    H.emin = a;
    H.emax = b;
    H.bounds_valid = true;
fail:
    cudaFree(d_lo);
    cudaFree(d_hi);
    return st;
}

md_status build_hamiltonian_device(Ham& H, const md_atoms* atoms, const md_pot_params* pot,
                                   cudaStream_t stream) {
    md_status st = MD_OK;
    const long long N = H.N;
    std::vector<double> xyz(3 * H.n_atoms), depth(H.n_atoms), sigma(H.n_atoms);
    std::vector<int> cstart, cids, cstart_p, cids_p;
    int nc[3], ncp[3];
    double cell[3], cellp[3];
    int* d_cstart = nullptr;
    int* d_cids = nullptr;
    double* d_vext = nullptr;
    int* d_overflow = nullptr;
    int* d_count = nullptr;
    double max_sigma = 0.0;
    GridGeo g = geo_of(H);
    const int threads = 256;
    int blocks = (int)std::min<long long>((N + threads - 1) / threads, 152LL * 64);
    CellArgs ca;

    for (long long a = 0; a < H.n_atoms; ++a) {
        for (int d = 0; d < 3; ++d) xyz[3 * a + d] = atoms->xyz[3 * a + d];
        depth[a] = atoms->depth[a];
        sigma[a] = atoms->sigma[a];
        max_sigma = std::max(max_sigma, sigma[a]);
    }
    MD_CUDA_TRY(cudaMalloc(&H.V, N * sizeof(double)));
    MD_CUDA_TRY(cudaMalloc(&H.V32, N * sizeof(float)));
    if (H.n_atoms > 0) {
        MD_CUDA_TRY(cudaMalloc(&H.atom_xyz, 3 * H.n_atoms * sizeof(double)));
        MD_CUDA_TRY(cudaMalloc(&H.atom_depth, H.n_atoms * sizeof(double)));
        MD_CUDA_TRY(cudaMalloc(&H.atom_sigma, H.n_atoms * sizeof(double)));
        MD_CUDA_TRY(cudaMemcpy(H.atom_xyz, xyz.data(), 3 * H.n_atoms * sizeof(double), cudaMemcpyHostToDevice));
        MD_CUDA_TRY(cudaMemcpy(H.atom_depth, depth.data(), H.n_atoms * sizeof(double), cudaMemcpyHostToDevice));
        MD_CUDA_TRY(cudaMemcpy(H.atom_sigma, sigma.data(), H.n_atoms * sizeof(double), cudaMemcpyHostToDevice));
    }
    build_cells(H, xyz, std::max(1e-3, H.cutoff_sigmas * max_sigma), cstart, cids, nc, cell);
    MD_CUDA_TRY(cudaMalloc(&d_cstart, cstart.size() * sizeof(int)));
    MD_CUDA_TRY(cudaMalloc(&d_cids, cids.size() * sizeof(int)));
    MD_CUDA_TRY(cudaMemcpy(d_cstart, cstart.data(), cstart.size() * sizeof(int), cudaMemcpyHostToDevice));
    MD_CUDA_TRY(cudaMemcpy(d_cids, cids.data(), cids.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (pot->v_ext) {
        MD_CUDA_TRY(cudaMalloc(&d_vext, N * sizeof(double)));
        MD_CUDA_TRY(cudaMemcpy(d_vext, pot->v_ext, N * sizeof(double), cudaMemcpyHostToDevice));
    }
    for (int d = 0; d < 3; ++d) {
        ca.nc[d] = nc[d];
        ca.cell[d] = cell[d];
    }
    ca.start = d_cstart;
    ca.atoms = d_cids;
    k_local_potential<<<blocks, threads, 0, stream>>>(g, ca, H.atom_xyz, H.atom_depth, H.atom_sigma,
                                                     H.cutoff_sigmas, d_vext, H.V, H.V32, N);
    MD_CUDA_TRY(cudaGetLastError());

    if (H.nonlocal && H.n_atoms > 0) {
        const long long na = H.n_atoms;
        const size_t tab = (size_t)na * 3 * kMaxProjWin;
        MD_CUDA_TRY(cudaMalloc(&H.proj_i0, 3 * na * sizeof(int)));
        MD_CUDA_TRY(cudaMalloc(&H.proj_len, 3 * na * sizeof(int)));
        MD_CUDA_TRY(cudaMalloc(&H.proj_d, tab * sizeof(double)));
        MD_CUDA_TRY(cudaMalloc(&H.proj_g, tab * sizeof(double)));
        MD_CUDA_TRY(cudaMalloc(&H.proj_d32, tab * sizeof(float)));
        MD_CUDA_TRY(cudaMalloc(&H.proj_g32, tab * sizeof(float)));
        MD_CUDA_TRY(cudaMalloc(&H.proj_C, 4 * na * sizeof(double)));
        MD_CUDA_TRY(cudaMalloc(&H.proj_C32, 4 * na * sizeof(float)));
        MD_CUDA_TRY(cudaMalloc(&H.proj_absum, 4 * na * sizeof(double)));
        MD_CUDA_TRY(cudaMalloc(&H.proj_rows, (size_t)na * kMaxProjWin * kMaxProjWin * 2));
        {
            const long long nt = (long long)tab;
            k_proj_tables<<<(unsigned)((nt + 255) / 256), 256, 0, stream>>>(
                g, H.atom_xyz, na, H.proj_rc, H.proj_sigma, H.proj_i0, H.proj_len, H.proj_d,
                H.proj_g, H.proj_d32, H.proj_g32);
            MD_CUDA_TRY(cudaGetLastError());
            const long long nr = na * kMaxProjWin * kMaxProjWin;
            k_proj_rows<<<(unsigned)((nr + 255) / 256), 256, 0, stream>>>(H.proj_len, H.proj_d, na,
                                                                         H.proj_rc, H.proj_rows);
            MD_CUDA_TRY(cudaGetLastError());
            k_proj_norms<<<(unsigned)na, 256, 0, stream>>>(H.proj_len, H.proj_d, H.proj_g, H.proj_rows,
                                                            H.dV, H.proj_C, H.proj_C32, H.proj_absum);
            MD_CUDA_TRY(cudaGetLastError());
        }
        // per-point lists: count, host scan, fill
        build_cells(H, xyz, H.proj_rc, cstart_p, cids_p, ncp, cellp);
        MD_CUDA_TRY(cudaFree(d_cstart));
        d_cstart = nullptr;
        MD_CUDA_TRY(cudaMalloc(&d_cstart, cstart_p.size() * sizeof(int)));
        MD_CUDA_TRY(cudaMemcpy(d_cstart, cstart_p.data(), cstart_p.size() * sizeof(int), cudaMemcpyHostToDevice));
        MD_CUDA_TRY(cudaMemcpy(d_cids, cids_p.data(), cids_p.size() * sizeof(int), cudaMemcpyHostToDevice));
        for (int d = 0; d < 3; ++d) {
            ca.nc[d] = ncp[d];
            ca.cell[d] = cellp[d];
        }
        ca.start = d_cstart;
        MD_CUDA_TRY(cudaMalloc(&d_count, (N + 1) * sizeof(int)));
        MD_CUDA_TRY(cudaMalloc(&d_overflow, sizeof(int)));
        MD_CUDA_TRY(cudaMemsetAsync(d_overflow, 0, sizeof(int), stream));
        k_proj_lists<false><<<blocks, threads, 0, stream>>>(g, ca, H.proj_i0, H.proj_len, H.proj_rows,
                                                            H.proj_d, H.proj_g, H.proj_C, N, d_count,
                                                            nullptr, nullptr, nullptr, d_overflow);
        MD_CUDA_TRY(cudaGetLastError());
        {
            std::vector<int> cnt(N + 1, 0);
            int ovf = 0;
            MD_CUDA_TRY(cudaMemcpyAsync(cnt.data(), d_count, N * sizeof(int), cudaMemcpyDeviceToHost, stream));
            MD_CUDA_TRY(cudaMemcpyAsync(&ovf, d_overflow, sizeof(int), cudaMemcpyDeviceToHost, stream));
            MD_CUDA_TRY(cudaStreamSynchronize(stream));
            if (ovf) {
                st = set_error(MD_ERR_INVALID, "md_build_hamiltonian: more than 16 projector atoms at one grid point");
                goto fail;
            }
            long long run = 0;
            for (long long i = 0; i < N; ++i) {
                const long long c = cnt[i];
                if (run > 2147483647LL - 16) {
                    st = set_error(MD_ERR_INVALID, "md_build_hamiltonian: too many projector entries (2^31)");
                    goto fail;
                }
                cnt[i] = (int)run;
                run += c;
            }
            cnt[N] = (int)run;
            H.pl_nnz = run;
            MD_CUDA_TRY(cudaMalloc(&H.pl_ptr, (N + 1) * sizeof(int)));
            MD_CUDA_TRY(cudaMalloc(&H.pl_atom, std::max<long long>(run, 1) * sizeof(int)));
            MD_CUDA_TRY(cudaMalloc(&H.pl_val32, std::max<long long>(run, 1) * sizeof(float4)));
            MD_CUDA_TRY(cudaMalloc(&H.pl_val64, std::max<long long>(run, 1) * 2 * sizeof(double2)));
            MD_CUDA_TRY(cudaMemcpy(H.pl_ptr, cnt.data(), (N + 1) * sizeof(int), cudaMemcpyHostToDevice));
        }
        k_proj_lists<true><<<blocks, threads, 0, stream>>>(g, ca, H.proj_i0, H.proj_len, H.proj_rows,
                                                           H.proj_d, H.proj_g, H.proj_C, N, H.pl_ptr,
                                                           H.pl_atom, H.pl_val64, H.pl_val32, d_overflow);
        MD_CUDA_TRY(cudaGetLastError());
    }
    {
        const md_status sb = compute_bounds(H, stream);
        if (sb != MD_OK) {
            st = sb;
            goto fail;
        }
    }
    MD_CUDA_TRY(cudaStreamSynchronize(stream));
fail:
    cudaFree(d_cstart);
    cudaFree(d_cids);
    cudaFree(d_vext);
    cudaFree(d_overflow);
    cudaFree(d_count);
    return st;
}

}  // namespace md
