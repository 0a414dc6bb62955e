// C ABI of the library: argument checks, region descriptors, scheduling
// order, workspace management and kernel launches.  See include/macrodft.h
// for the contract of each entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "md_adjoint.h"
#include "md_internal.h"
#include "md_lanczos.h"
#include "md_solver.h"

namespace md {

namespace {
thread_local std::string g_last_error;
}

md_status set_error(md_status code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
void clear_error() { g_last_error.clear(); }

md_status build_hamiltonian_device(Ham& H, const md_atoms* atoms, const md_pot_params* pot,
                                   cudaStream_t stream);

// FD weights of d^2/dx^2 with accuracy order 2q by Fornberg's recursion
// (B. Fornberg, Math. Comp. 51 (1988) 699-706) on the nodes 0, +-1, ..., +-q
// (h = 1); returns w_0..w_q of the symmetric stencil.
static void fornberg_second_derivative(int q, double* w_out) {
    const int np = 2 * q + 1;
    std::vector<double> x(np);
    x[0] = 0.0;
    for (int o = 1; o <= q; ++o) {
        x[2 * o - 1] = o;
        x[2 * o] = -o;
    }
    const int M = 2;
    // delta[m][n][nu]
    std::vector<double> delta((M + 1) * np * np, 0.0);
    auto D = [&](int m, int n, int nu) -> double& { return delta[(m * np + n) * np + nu]; };
    D(0, 0, 0) = 1.0;
    double c1 = 1.0;
    for (int n = 1; n < np; ++n) {
        double c2 = 1.0;
        for (int nu = 0; nu < n; ++nu) {
            const double c3 = x[n] - x[nu];
            c2 *= c3;
            for (int m = 0; m <= std::min(n, M); ++m) {
                const double prev = D(m, n - 1, nu);
                const double prevm = m > 0 ? D(m - 1, n - 1, nu) : 0.0;
                D(m, n, nu) = (x[n] * prev - m * prevm) / c3;
            }
        }
        for (int m = 0; m <= std::min(n, M); ++m) {
            const double a = m > 0 ? D(m - 1, n - 1, n - 1) : 0.0;
            const double b = D(m, n - 1, n - 1);
            D(m, n, n) = (c1 / c2) * (m * a - x[n - 1] * b);
        }
        c1 = c2;
    }
    w_out[0] = D(2, np - 1, 0);
    for (int o = 1; o <= q; ++o) w_out[o] = D(2, np - 1, 2 * o - 1);
}

namespace {

#define MD_TRY_CUDA(expr)                                                                 \
    do {                                                                                  \
        cudaError_t _e = (expr);                                                          \
        if (_e != cudaSuccess) {                                                          \
            st = (_e == cudaErrorMemoryAllocation) ? MD_ERR_OOM : MD_ERR_CUDA;            \
            set_error(st, std::string("CUDA: ") + cudaGetErrorString(_e) + " (" #expr ")"); \
            goto done;                                                                    \
        }                                                                                 \
    } while (0)

md_status check_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0)
        return set_error(MD_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    if (prop.major * 10 + prop.minor < 100)
        return set_error(MD_ERR_CUDA, "this library is built for sm_103a (Blackwell Ultra)");
    return MD_OK;
}

void free_ham(Ham& H) {
    // an asynchronous md_density may still be reading the operator, the
    // scratch or a staging buffer: wait for it first
    if (H.scratch_ev) {
        cudaEventSynchronize(H.scratch_ev);
        cudaEventDestroy(H.scratch_ev);
        H.scratch_ev = nullptr;
    }
    for (Ham::Stage& sg : H.stage) {
        if (sg.ev) {
            cudaEventSynchronize(sg.ev);
            cudaEventDestroy(sg.ev);
            sg.ev = nullptr;
        }
        if (sg.buf) cudaFreeHost(sg.buf);
        sg.buf = nullptr;
    }
    void* ptrs[] = {H.V, H.V32, H.atom_xyz, H.atom_depth, H.atom_sigma, H.proj_i0, H.proj_len,
                    H.proj_d, H.proj_g, H.proj_d32, H.proj_g32, H.proj_C, H.proj_absum,
                    H.proj_C32, H.proj_rows, H.pl_ptr, H.pl_atom, H.pl_val32, H.pl_val64,
                    H.scratch, H.lz_buf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// Host wait until the last asynchronous md_density call on the handle has
// finished with its scratch (at once when there was none).
cudaError_t scratch_idle(Ham& H) { return H.scratch_ev ? cudaEventSynchronize(H.scratch_ev) : cudaSuccess; }

struct Regions {
    std::vector<NodeDesc> desc;
    std::vector<long long> points;
    long long total = 0;
    long long n_max = 0;
    int max_dim[3] = {0, 0, 0};
    bool any_ring = false;
};

// Region of node g with half-width s (the cube of side 2s+1 around it,
// wrapped on periodic axes, the whole axis as a ring where 2s+1 >= n):
// descriptor and point count; MD_ERR_INVALID for a bad node or region.
md_status build_node_desc(const Ham& H, long long g, int s, NodeDesc& d, long long& pts) {
    if (g < 0 || g >= H.N) return set_error(MD_ERR_INVALID, "node index out of range");
    if (s < 0) return set_error(MD_ERR_INVALID, "negative region half-width");
    const int c[3] = {(int)(g % H.n[0]), (int)((g / H.n[0]) % H.n[1]), (int)(g / ((long long)H.n[0] * H.n[1]))};
    d.ring = 0;
    int srcc[3];
    pts = 1;
    for (int ax = 0; ax < 3; ++ax) {
        const long long m = 2LL * s + 1;
        if (H.periodic[ax] && m >= H.n[ax]) {
            d.dims[ax] = H.n[ax];
            d.lo[ax] = 0;
            d.ring |= 1 << ax;
            srcc[ax] = c[ax];
        } else {
            if (!H.periodic[ax] && (c[ax] - s < 0 || c[ax] + s >= H.n[ax]))
                return set_error(MD_ERR_INVALID, "region leaves a non-periodic grid axis");
            d.dims[ax] = (int)m;
            d.lo[ax] = c[ax] - s;
            srcc[ax] = s;
        }
        pts *= d.dims[ax];
    }
    if (pts > (1LL << 30)) return set_error(MD_ERR_INVALID, "region too large");
    d.src = srcc[0] + d.dims[0] * (srcc[1] + d.dims[1] * srcc[2]);
    return MD_OK;
}

md_status make_regions(const Ham& H, const md_nodes* nodes, Regions& R) {
    if (!nodes || nodes->n_nodes < 0 || (nodes->n_nodes > 0 && (!nodes->node || !nodes->halfwidth)))
        return set_error(MD_ERR_INVALID, "nodes: null arrays or negative count");
    const long long nn = nodes->n_nodes;
    R.desc.resize(nn);
    R.points.resize(nn);
    R.total = 0;
    R.n_max = 0;
    for (long long j = 0; j < nn; ++j) {
        NodeDesc& d = R.desc[j];
        long long pts = 0;
        const md_status st = build_node_desc(H, nodes->node[j], nodes->halfwidth[j], d, pts);
        if (st != MD_OK) return st;
        for (int ax = 0; ax < 3; ++ax) R.max_dim[ax] = std::max(R.max_dim[ax], d.dims[ax]);
        if (d.ring) R.any_ring = true;
        R.points[j] = pts;
        R.total += pts;
        R.n_max = std::max(R.n_max, pts);
    }
    return MD_OK;
}

md_status check_poles(const md_poles* poles) {
    if (!poles || poles->n_poles < 1 || !poles->z || !poles->w)
        return set_error(MD_ERR_INVALID, "poles: need n_poles >= 1 and z, w");
    for (int p = 0; p < poles->n_poles; ++p) {
        if (!std::isfinite(poles->z[2 * p]) || !std::isfinite(poles->z[2 * p + 1]) ||
            !std::isfinite(poles->w[2 * p]) || !std::isfinite(poles->w[2 * p + 1]))
            return set_error(MD_ERR_INVALID, "poles: non-finite value");
        if (!(poles->z[2 * p + 1] > 0.0)) return set_error(MD_ERR_INVALID, "poles: need Im z > 0");
    }
    return MD_OK;
}

md_solver_opts normalise_opts(const md_solver_opts* o) {
    md_solver_opts r;
    std::memset(&r, 0, sizeof(r));
    if (o) r = *o;
    if (r.reliable_every <= 0) r.reliable_every = 300;
    if (!(r.reliable_delta > 0.0)) r.reliable_delta = 3e-3;
    return r;
}

md_status check_opts(const md_solver_opts* o) {
    if (!o) return set_error(MD_ERR_INVALID, "opts is NULL");
    if (!(o->tol > 0.0) || o->maxit <= 0)
        return set_error(MD_ERR_INVALID, "opts: need tol > 0 and maxit > 0");
    if (o->precision != MD_PREC_FP64 && o->precision != MD_PREC_MIXED)
        return set_error(MD_ERR_INVALID, "opts: unknown precision");
    if (o->block != 0 && (o->block < 64 || o->block > 1024 || o->block % 32))
        return set_error(MD_ERR_INVALID, "opts: block must be a multiple of 32 in [64, 1024]");
    if (o->kernel < 0 || o->kernel > 3) return set_error(MD_ERR_INVALID, "opts: kernel must be 0, 1, 2 or 3");
    if (o->method < 0 || o->method > 1) return set_error(MD_ERR_INVALID, "opts: method must be 0 or 1");
    return MD_OK;
}

md_status upload_poles(const md_poles* poles, double2** d_z, double2** d_w, cudaStream_t stream) {
    const int Pn = poles->n_poles;
    cudaError_t e = cudaMallocAsync((void**)d_z, Pn * sizeof(double2), stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)d_w, Pn * sizeof(double2), stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(*d_z, poles->z, Pn * sizeof(double2), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(*d_w, poles->w, Pn * sizeof(double2), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    return MD_OK;
}

}  // namespace
}  // namespace md

// ---------------------------------------------------------------------------
// Plans: one prepared batched solve, replayed as a CUDA graph.
// ---------------------------------------------------------------------------
struct md_plan {
    md::Ham* H = nullptr;
    int precision = 0;
    int Pn = 0;
    long long nn = 0;
    long long n_sys = 0;
    int grid = 0, block = 0, per_sm = 1;
    int variant = 0;                   // 0 generic kernel, K > 0: z-march kernel with K columns per thread
    int cluster = 0;                   // > 0: cluster kernel with this many CTAs per system
    size_t cl_smem = 0;                // dynamic shared memory of the cluster kernel
    int cl_block = 0;                  // its threads per CTA
    bool multishift = false;           // one shifted-COCG work item per node
    size_t smem = 0;                   // dynamic shared memory of the z-march kernel
    std::vector<long long> points;     // region points per node
    md::SolveParams P;
    // device buffers owned by the plan
    void* scratch = nullptr;
    bool own_scratch = true;
    md::SysDesc* d_sys = nullptr;
    md::NodeDesc* d_nodes = nullptr;
    long long* d_ckoff = nullptr;
    int* d_status = nullptr;
    int* d_iters = nullptr;
    int* d_nrel = nullptr;
    double* d_resid = nullptr;
    double2* d_xsrc = nullptr;
    double2* d_z = nullptr;
    double2* d_w = nullptr;
    unsigned int* d_counter = nullptr;
    double* rho_out = nullptr;
    double* e_out = nullptr;
    cudaStream_t cap = nullptr;
    bool direct = false;               // launched at creation on `dstream`, temporaries freed stream-ordered
    cudaStream_t dstream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool launched = false;
};

namespace md {
namespace {

#define PLAN_TRY(expr)                                                                    \
    do {                                                                                  \
        cudaError_t _e = (expr);                                                          \
        if (_e != cudaSuccess) {                                                          \
            return set_error((_e == cudaErrorMemoryAllocation) ? MD_ERR_OOM : MD_ERR_CUDA, \
                             std::string("CUDA: ") + cudaGetErrorString(_e) + " (" #expr ")"); \
        }                                                                                 \
    } while (0)

void plan_free(md_plan* pl) {
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->cap) cudaStreamDestroy(pl->cap);
    if (pl->ev0) cudaEventDestroy(pl->ev0);
    if (pl->ev1) cudaEventDestroy(pl->ev1);
    void* ptrs[] = {pl->d_sys, pl->d_nodes, pl->d_ckoff, pl->d_status, pl->d_iters, pl->d_nrel,
                    pl->d_resid, pl->d_xsrc, pl->d_z, pl->d_w, pl->d_counter};
    for (void* p : ptrs)
        if (p) {
            if (pl->direct) cudaFreeAsync(p, pl->dstream);
            else cudaFree(p);
        }
    if (pl->own_scratch && pl->scratch) cudaFree(pl->scratch);
    delete pl;
}

// A launch shape.  Generic and z-march kernels: per_sm CTAs per SM.  Cluster
// kernel (cluster > 0): per_sm = resident clusters on the device.
struct Shape {
    int variant, block, per_sm;
    int cluster = 0;
};

int grid_of(const Shape& sh, int n_sm, long long n_work) {
    if (sh.cluster > 0) return (int)std::min<long long>(sh.per_sm, n_work) * sh.cluster;
    return (int)std::min<long long>((long long)n_sm * sh.per_sm, n_work);
}

// Scratch the shape needs: one Krylov slot per CTA, or per cluster.
size_t scratch_of(const SolveParams& P, const Shape& sh, int grid) {
    if (sh.cluster > 0)
        return cl_slot_bytes(P.n_max, sh.cluster, P.cl_slab, P.nonlocal, P.cl_row_cap, P.cl_key_cap) * (size_t)(grid / sh.cluster);
    return P.slot_bytes * (size_t)grid;
}

cudaError_t launch_shape(const md_plan* pl, const SolveParams& P, const Shape& sh, int grid, cudaStream_t s) {
    if (sh.cluster > 0) {
        SolveParams C = P;
        C.slot_bytes = cl_slot_bytes(P.n_max, sh.cluster, P.cl_slab, P.nonlocal, P.cl_row_cap, P.cl_key_cap);
        return launch_cocg_cl(C, sh.cluster, grid, sh.block, pl->cl_smem, s);
    }
    if (sh.variant > 0) return launch_cocg_zm(P, sh.variant, grid, sh.block, pl->smem, s);
    return launch_cocg(P, pl->precision, grid, sh.block, sh.per_sm, s);
}

// Cluster-kernel geometry for regions of at most m2 planes of at most
// `plane` points: among the cluster sizes (<= 8 CTAs, or the given size
// `force` > 0) whose thickest slab of p and r fits in shared memory, the one
// that keeps the most SMs busy; the CTA size (a multiple of 32 up to the
// kernel's limit) with the most threads that wastes at most 6 % more thread
// slots on one plane's columns than the best; and, with projector windows
// wx points long (0: no projectors), how many atoms' x tables the leftover
// shared memory holds (xcap).  Returns false if no cluster size fits.
bool cl_geometry(int q, int m2, int plane, int dev, int force, int wx, int& csz, int& slab, size_t& smem,
                 int& block, int& xcap) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t budget = (size_t)optin > cl_static_smem_bytes() ? (size_t)optin - cl_static_smem_bytes() : 0;
    // CTA size: the most threads whose column assignment wastes at most 6 %
    // more thread slots than the best one (more warps hide more latency)
    double best = 0.0;
    for (int t = 64; t <= cl_max_threads(); t += 32)
        best = std::max(best, (double)plane / (double)(((plane + t - 1) / t) * t));
    block = 64;
    for (int t = 64; t <= cl_max_threads(); t += 32)
        if ((double)plane / (double)(((plane + t - 1) / t) * t) >= best - 0.06) block = t;
    // among the sizes whose slabs fit, the one that keeps the most SMs busy
    // (clusters are placed within a GPC, so larger clusters strand SMs);
    // ties go to the smaller cluster (fewer halo planes)
    csz = 0;
    long long best_cover = 0;
    for (int c = force > 0 ? force : 1; c <= (force > 0 ? force : 8); ++c) {
        const long long sp = (long long)((m2 + c - 1) / c) * plane;
        if (sp >= (1LL << 30) || cl_smem_bytes((int)sp, 0) > budget) continue;
        if ((m2 + c - 1) / c > 255) continue;   // the nonlocal row records hold the slab plane in 8 bits
        const long long cover = (long long)cl_max_clusters(q, c, block, cl_smem_bytes((int)sp, 0)) * c;
        if (cover > best_cover) {
            best_cover = cover;
            csz = c;
            slab = (int)sp;
        }
    }
    if (csz == 0) return false;
    const size_t base = cl_smem_bytes(slab, 0);
    xcap = wx > 0 ? (int)std::min<size_t>(kMaxLocalProjAtoms, (budget - base) / (8 * (size_t)wx)) : 0;
    smem = cl_smem_bytes(slab, 2 * xcap * wx);
    return true;
}

// Candidate launch shapes: the generic kernel at 1024x1 and 512x2 (and, in
// mixed precision, 512x3 from its 40-register instance), and, when the
// z-march kernel applies, K = 1..4 columns per thread with the smallest
// warp-multiple block covering the largest plane, at every CTAs-per-SM
// count the occupancy calculator allows.
std::vector<Shape> candidate_shapes(const md_plan* pl, bool zm_ok, int max_plane) {
    std::vector<Shape> c = {{0, 1024, 1}, {0, 512, 2}};
    if (pl->precision == MD_PREC_MIXED) c.push_back({0, 512, 3});
    if (pl->cluster > 0) {
        const int n_cl = cl_max_clusters(pl->P.q, pl->cluster, pl->cl_block, pl->cl_smem);
        if (n_cl > 0) c.push_back({0, pl->cl_block, n_cl, pl->cluster});
    }
    if (!zm_ok) return c;
    for (int K = 1; K <= 4; ++K) {
        const int need = (max_plane + K - 1) / K;
        const int block = (need + 31) / 32 * 32;
        if (block > zm_max_threads(K) || block < 64) continue;
        const int occ = zm_occupancy(pl->P.q, K, block, pl->smem);
        for (int per = 1; per <= std::min(occ, 2); ++per) c.push_back({K, block, per});
    }
    return c;
}

// Launch-shape autotuner: times each candidate on the same evenly spread
// sample of systems with a short iteration cap and keeps the one with the
// most region-point iterations per second.  Results are cached per
// (precision, stencil width, region-size bucket, nonlocal, z-march
// eligibility, device) for the life of the process; plans may be created
// from several host threads, so the cache is guarded (two threads tuning the
// same key at once both run their trials and store the same kind of answer).
struct TuneKey {
    int precision, q, bucket, nonlocal, zm, device;
    bool operator==(const TuneKey& o) const {
        return precision == o.precision && q == o.q && bucket == o.bucket && nonlocal == o.nonlocal &&
               zm == o.zm && device == o.device;
    }
};
struct TuneEntry {
    TuneKey key;
    Shape shape;
};
std::vector<TuneEntry> g_tune_cache;
std::mutex g_tune_mutex;

md_status autotune(md_plan* pl, int n_sm, const std::vector<Shape>& cands, size_t scratch_bytes,
                   Shape& out, cudaStream_t wait_first = nullptr) {
    int dev = 0;
    cudaGetDevice(&dev);
    const TuneKey key{pl->precision, pl->P.q, (int)((pl->P.n_max + 4095) / 4096), pl->P.nonlocal,
                      (cands.size() > 2 ? 1 : 0) + 2 * pl->P.multishift + 4 * (pl->cluster > 0 ? 1 : 0), dev};
    {
        std::lock_guard<std::mutex> guard(g_tune_mutex);
        for (const auto& e : g_tune_cache)
            if (e.key == key) {
                out = e.shape;
                return MD_OK;
            }
    }
    // a miss runs trials on the plan's stream: the caller's stream must have
    // finished the uploads they read
    if (pl->direct) PLAN_TRY(cudaStreamSynchronize(wait_first));
    const long long nw = pl->P.n_sys;   // work items (systems, or nodes with shifted COCG)
    // systems in flight at once per candidate: one per CTA, or one per cluster
    long long max_flight = 1;
    for (const auto& c : cands)
        max_flight = std::max<long long>(max_flight, c.cluster > 0 ? c.per_sm : (long long)n_sm * c.per_sm);
    // enough systems that every candidate's CTAs each take four in turn, so
    // that the trial's tail (CTAs idle at its end) weighs little, as in a
    // full batch
    const long long ns = std::min<long long>(nw, 4LL * max_flight);
    std::vector<SysDesc> all(nw), sample;
    PLAN_TRY(cudaMemcpy(all.data(), pl->d_sys, nw * sizeof(SysDesc), cudaMemcpyDeviceToHost));
    for (long long k = 0; k < ns; ++k) sample.push_back(all[(k * nw) / ns]);
    SysDesc* d_sample = nullptr;
    PLAN_TRY(cudaMalloc(&d_sample, ns * sizeof(SysDesc)));
    cudaMemcpy(d_sample, sample.data(), ns * sizeof(SysDesc), cudaMemcpyHostToDevice);
    // iterations per trial system (MD_AUTOTUNE_ITERS overrides, 16..4096)
    int trial_iters = 64;
    if (const char* ev = std::getenv("MD_AUTOTUNE_ITERS")) trial_iters = std::max(16, std::min(4096, std::atoi(ev)));
    double best = -1.0;
    Shape bs = cands[0];
    std::vector<int> h_it(pl->n_sys);
    bool zm_hopeless = false;
    for (const auto& c : cands) {
        // the z-march candidates come last; once one runs at under half the
        // best rate so far the others are not tried
        if (c.variant > 0 && zm_hopeless) continue;
        SolveParams T = pl->P;
        T.sys = d_sample;
        T.n_sys = (int)ns;
        T.maxit = std::min(pl->P.maxit, trial_iters);
        T.ckpt = nullptr;         // trials never touch the checkpoint
        T.fused_dLdV = nullptr;   // nor the gradient
        T.dm_rows = nullptr;
        const int grid = grid_of(c, n_sm, ns);
        if (scratch_of(pl->P, c, grid) > scratch_bytes) continue;
        // best of two runs (one for a z-march shape already far behind); the
        // counter reset is ordered on the trial stream
        float ms = 0.f;
        bool failed = false;
        long long pit = 0;
        for (int rep = 0; rep < 2 && !failed; ++rep) {
            cudaMemsetAsync(T.work_counter, 0, sizeof(unsigned int), pl->cap);
            cudaEventRecord(pl->ev0, pl->cap);
            cudaError_t e = launch_shape(pl, T, c, grid, pl->cap);
            cudaEventRecord(pl->ev1, pl->cap);
            if (e != cudaSuccess) {
                cudaGetLastError();
                failed = true;
                break;
            }
            if (cudaStreamSynchronize(pl->cap) != cudaSuccess) {
                cudaFree(d_sample);
                return set_error(MD_ERR_CUDA, "autotune trial failed");
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, pl->ev0, pl->ev1);
            if (rep == 0 || t < ms) ms = t;
            if (rep == 0) {   // iteration counts are the same in every repetition
                cudaMemcpy(h_it.data(), T.iters, pl->n_sys * sizeof(int), cudaMemcpyDeviceToHost);
                for (const auto& sd : sample) {
                    int it = h_it[(long long)sd.node * pl->Pn + sd.pole];
                    if (pl->multishift)
                        for (int p = 0; p < pl->Pn; ++p) it = std::max(it, h_it[(long long)sd.node * pl->Pn + p]);
                    pit += (long long)it * pl->points[sd.node];
                }
                if (c.variant > 0 && ms > 0 && (double)pit / ms < 0.5 * best) break;
            }
        }
        if (failed) continue;
        const double rate = ms > 0 ? (double)pit / ms : 0.0;
        if (std::getenv("MD_AUTOTUNE_LOG"))
            std::fprintf(stderr,
                         "md autotune: variant %d cluster %d block %d ctas/SM or clusters %d: %.3f ms, %.3g "
                         "point-iterations/s\n",
                         c.variant, c.cluster, c.block, c.per_sm, ms, rate * 1e3);
        if (c.variant > 0 && rate < 0.5 * best) zm_hopeless = true;
        if (rate > best) {
            best = rate;
            bs = c;
        }
    }
    cudaFree(d_sample);
    {
        std::lock_guard<std::mutex> guard(g_tune_mutex);
        g_tune_cache.push_back(TuneEntry{key, bs});
    }
    out = bs;
    return MD_OK;
}

// Grid, stencil, potential and projector fields of the solver parameters.
void fill_operator(SolveParams& P, const Ham& H) {
    for (int d = 0; d < 3; ++d) {
        P.n[d] = H.n[d];
        P.periodic[d] = H.periodic[d];
        for (int o = 0; o < kMaxQ; ++o) P.coef[d][o] = H.coef[d][o];
    }
    P.N = H.N;
    P.q = H.q;
    P.diag = H.diag;
    P.dV = H.dV;
    P.V = H.V;
    P.V32 = H.V32;
    P.nonlocal = H.nonlocal && H.n_atoms > 0;
    P.n_atoms = H.n_atoms;
    P.proj_i0 = H.proj_i0;
    P.proj_len = H.proj_len;
    P.proj_d = H.proj_d;
    P.proj_g = H.proj_g;
    P.proj_d32 = H.proj_d32;
    P.proj_g32 = H.proj_g32;
    P.proj_C = H.proj_C;
    P.proj_C32 = H.proj_C32;
    P.proj_rows = H.proj_rows;
    P.pl_ptr = H.pl_ptr;
    P.pl_atom = H.pl_atom;
    P.pl_val32 = H.pl_val32;
    P.pl_val64 = H.pl_val64;
    P.e_s = H.e_s;
    P.e_p = H.e_p;
}

struct FusedArgs {
    double* dLdV;           // fused adjoint (may be NULL)
    const double* a;
    const double* b;
    double* dm_rows;        // density-matrix rows (may be NULL)
    const long long* dm_off;
};

// direct: launch at once on `stream` without a graph and without
// synchronising it (device temporaries allocated and freed stream-ordered,
// uploads staged through the handle's pinned buffers); the caller frees the
// plan right after.  Otherwise the batch is captured as a graph for replay.
md_status plan_create(const md_hamiltonian* ham, const md_poles* poles, const md_nodes* nodes,
                      const md_solver_opts* opts_in, double* rho_out, double* e_out, md_workspace* ckpt,
                      bool borrow_scratch, cudaStream_t stream, md_plan** out,
                      const FusedArgs* fused = nullptr, bool direct = false) {
    *out = nullptr;
    md_status st = check_device();
    if (st != MD_OK) return st;
    if (!ham) return set_error(MD_ERR_INVALID, "ham is NULL");
    if ((st = check_poles(poles)) != MD_OK) return st;
    if ((st = check_opts(opts_in)) != MD_OK) return st;
    Ham& H = const_cast<md_hamiltonian*>(ham)->h;
    Regions R;
    if ((st = make_regions(H, nodes, R)) != MD_OK) return st;
    const long long nn = (long long)R.desc.size();
    if (!rho_out && nn > 0) return set_error(MD_ERR_INVALID, "rho_out is NULL");
    if (ckpt && (ckpt->n_nodes != nn || ckpt->n_poles != poles->n_poles || ckpt->total_points != R.total))
        return set_error(MD_ERR_INVALID, "checkpoint workspace was made for other nodes or poles");
    const md_solver_opts opts = normalise_opts(opts_in);
    const int Pn = poles->n_poles;
    const long long n_sys = nn * Pn;
    if (n_sys > (1LL << 31) - 1) return set_error(MD_ERR_INVALID, "too many systems");
    const bool ms = opts.method == 1;
    if (ms && ckpt) return set_error(MD_ERR_INVALID, "method 1 (shifted COCG) keeps no checkpoint");
    if (ms && Pn > 64) return set_error(MD_ERR_INVALID, "method 1 (shifted COCG) handles at most 64 poles");
    if (ms && opts.kernel >= 2) return set_error(MD_ERR_INVALID, "method 1 runs on the generic kernel");
    if (fused && ms) return set_error(MD_ERR_INVALID, "the fused adjoint needs method 0");

    md_plan* pl = new md_plan();
    pl->H = &H;
    pl->precision = opts.precision;
    pl->Pn = Pn;
    pl->nn = nn;
    pl->n_sys = n_sys;
    pl->points = R.points;
    pl->rho_out = rho_out;
    pl->e_out = e_out;
    pl->own_scratch = !borrow_scratch;
    pl->multishift = ms;
    pl->direct = direct;
    pl->dstream = stream;
    std::memset(&pl->P, 0, sizeof(pl->P));
    auto fail = [&](md_status s) {
        plan_free(pl);
        return s;
    };
#define PTRY(expr)                                                                          \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess)                                                              \
            return fail(set_error((_e == cudaErrorMemoryAllocation) ? MD_ERR_OOM : MD_ERR_CUDA, \
                                  std::string("CUDA: ") + cudaGetErrorString(_e) + " (" #expr ")")); \
    } while (0)
    PTRY(cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking));
    PTRY(cudaEventCreate(&pl->ev0));
    PTRY(cudaEventCreate(&pl->ev1));
    if (n_sys == 0) {
        *out = pl;
        return MD_OK;
    }
    int dev = 0, n_sm = 0;
    PTRY(cudaGetDevice(&dev));
    PTRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));

    // cost-sorted work list: big regions first, then poles nearest the real axis;
    // with shifted COCG one item per node, seeded by the pole nearest the axis
    std::vector<SysDesc> sys;
    if (ms) {
        int seed = 0;
        for (int p = 1; p < Pn; ++p)
            if (poles->z[2 * p + 1] < poles->z[2 * seed + 1]) seed = p;
        for (long long j = 0; j < nn; ++j) sys.push_back(SysDesc{(int)j, seed});
    } else {
        sys.resize(n_sys);
        for (long long j = 0; j < nn; ++j)
            for (int p = 0; p < Pn; ++p) sys[j * Pn + p] = SysDesc{(int)j, p};
    }
    std::stable_sort(sys.begin(), sys.end(), [&](const SysDesc& a, const SysDesc& b) {
        const double ca = (double)R.points[a.node] / std::sqrt(poles->z[2 * a.pole + 1]);
        const double cb = (double)R.points[b.node] / std::sqrt(poles->z[2 * b.pole + 1]);
        return ca > cb;
    });
    const long long n_work = (long long)sys.size();
    auto dmalloc = [&](auto** p, size_t b) {
        return direct ? cudaMallocAsync((void**)p, b, stream) : cudaMalloc((void**)p, b);
    };
    PTRY(dmalloc(&pl->d_sys, n_work * sizeof(SysDesc)));
    PTRY(dmalloc(&pl->d_nodes, nn * sizeof(NodeDesc)));
    PTRY(dmalloc(&pl->d_status, n_sys * sizeof(int)));
    PTRY(dmalloc(&pl->d_iters, n_sys * sizeof(int)));
    PTRY(dmalloc(&pl->d_nrel, n_sys * sizeof(int)));
    PTRY(dmalloc(&pl->d_resid, n_sys * sizeof(double)));
    PTRY(dmalloc(&pl->d_xsrc, n_sys * sizeof(double2)));
    PTRY(dmalloc(&pl->d_z, Pn * sizeof(double2)));
    PTRY(dmalloc(&pl->d_w, Pn * sizeof(double2)));
    PTRY(dmalloc(&pl->d_counter, sizeof(unsigned int)));
    std::vector<long long> ckoff;
    if (ckpt) {
        ckoff.resize(n_sys);
        for (long long j = 0; j < nn; ++j)
            for (int p = 0; p < Pn; ++p) ckoff[j * Pn + p] = Pn * ckpt->node_off[j] + p * R.points[j];
        PTRY(dmalloc(&pl->d_ckoff, n_sys * sizeof(long long)));
    }
    if (direct) {
        // uploads from the handle's pinned staging buffer (a pageable source
        // would make the copy wait for the stream's earlier work); two
        // buffers in turn, each reused once its previous uploads are done
        Ham::Stage& sg = H.stage[H.stage_next];
        H.stage_next ^= 1;
        auto up = [](size_t b) { return (b + 255) / 256 * 256; };
        const size_t o_nodes = up(n_work * sizeof(SysDesc)), o_z = o_nodes + up(nn * sizeof(NodeDesc));
        const size_t o_w = o_z + up(Pn * sizeof(double2)), o_ck = o_w + up(Pn * sizeof(double2));
        const size_t need_h = o_ck + (ckpt ? n_sys * sizeof(long long) : 0);
        if (sg.ev) PTRY(cudaEventSynchronize(sg.ev));
        else PTRY(cudaEventCreateWithFlags(&sg.ev, cudaEventDisableTiming));
        if (need_h > sg.bytes) {
            if (sg.buf) cudaFreeHost(sg.buf);
            sg.buf = nullptr;
            sg.bytes = 0;
            PTRY(cudaMallocHost(&sg.buf, need_h));
            sg.bytes = need_h;
        }
        char* hb = (char*)sg.buf;
        std::memcpy(hb, sys.data(), n_work * sizeof(SysDesc));
        std::memcpy(hb + o_nodes, R.desc.data(), nn * sizeof(NodeDesc));
        std::memcpy(hb + o_z, poles->z, Pn * sizeof(double2));
        std::memcpy(hb + o_w, poles->w, Pn * sizeof(double2));
        if (ckpt) std::memcpy(hb + o_ck, ckoff.data(), n_sys * sizeof(long long));
        PTRY(cudaMemcpyAsync(pl->d_sys, hb, n_work * sizeof(SysDesc), cudaMemcpyHostToDevice, stream));
        PTRY(cudaMemcpyAsync(pl->d_nodes, hb + o_nodes, nn * sizeof(NodeDesc), cudaMemcpyHostToDevice, stream));
        PTRY(cudaMemcpyAsync(pl->d_z, hb + o_z, Pn * sizeof(double2), cudaMemcpyHostToDevice, stream));
        PTRY(cudaMemcpyAsync(pl->d_w, hb + o_w, Pn * sizeof(double2), cudaMemcpyHostToDevice, stream));
        if (ckpt)
            PTRY(cudaMemcpyAsync(pl->d_ckoff, hb + o_ck, n_sys * sizeof(long long), cudaMemcpyHostToDevice, stream));
        PTRY(cudaEventRecord(sg.ev, stream));
        PTRY(cudaMemsetAsync(pl->d_iters, 0, n_sys * sizeof(int), stream));
    } else {
        PTRY(cudaMemcpy(pl->d_sys, sys.data(), n_work * sizeof(SysDesc), cudaMemcpyHostToDevice));
        PTRY(cudaMemcpy(pl->d_nodes, R.desc.data(), nn * sizeof(NodeDesc), cudaMemcpyHostToDevice));
        PTRY(cudaMemcpy(pl->d_z, poles->z, Pn * sizeof(double2), cudaMemcpyHostToDevice));
        PTRY(cudaMemcpy(pl->d_w, poles->w, Pn * sizeof(double2), cudaMemcpyHostToDevice));
        PTRY(cudaMemsetAsync(pl->d_iters, 0, n_sys * sizeof(int), pl->cap));
        if (ckpt) PTRY(cudaMemcpy(pl->d_ckoff, ckoff.data(), n_sys * sizeof(long long), cudaMemcpyHostToDevice));
        // the copies above run on the legacy stream; the trials and the capture
        // below run on the plan's own (non-blocking) stream
        PTRY(cudaStreamSynchronize(cudaStreamLegacy));
    }

    SolveParams& P = pl->P;
    fill_operator(P, H);
    P.n_sys = (int)n_work;
    P.multishift = ms ? 1 : 0;
    P.w = pl->d_w;
    if (fused) {
        P.fused_dLdV = fused->dLdV;
        P.fused_a = fused->a;
        P.fused_b = fused->b;
        P.dm_rows = fused->dm_rows;
        P.dm_off = fused->dm_off;
    }
    P.P = Pn;
    P.sys = pl->d_sys;
    P.nodes = pl->d_nodes;
    P.z = pl->d_z;
    P.tol = opts.tol;
    P.maxit = opts.maxit;
    P.reliable_every = opts.reliable_every;
    P.reliable_delta = opts.reliable_delta;
    P.timeout_ns = opts.timeout_s > 0 ? (unsigned long long)(opts.timeout_s * 1e9) : 0ULL;
    P.slot_bytes = slot_bytes_for(opts.precision, R.n_max);
    P.n_max = (int)((R.n_max + 63) / 64 * 64);
    P.ckpt = ckpt ? (double2*)ckpt->x : nullptr;
    P.ckpt_sys_off = pl->d_ckoff;
    P.work_counter = pl->d_counter;
    P.x_src = pl->d_xsrc;
    P.status = pl->d_status;
    P.iters = pl->d_iters;
    P.resid = pl->d_resid;
    P.n_rel = pl->d_nrel;

    const int max_plane = R.max_dim[0] * R.max_dim[1];
    const bool zm_ok = zm_supported(opts.precision, H.q) && !R.any_ring && !ms && !fused;
    P.zm_m0 = R.max_dim[0];
    P.zm_m1 = R.max_dim[1];
    if (zm_ok) pl->smem = zm_smem_bytes(H.q, R.max_dim[0], R.max_dim[1]);
    // the cluster kernel: mixed precision, no whole-axis rings, per-pole COCG
    // (regions with at most 255 points along y: the row records hold the row in 8 bits)
    P.cl_wx = P.nonlocal ? std::min(2 * (int)std::floor(H.proj_rc / H.h[0]) + 2, kMaxProjWin) : 0;
    const bool cl_ok = cl_supported(opts.precision, H.q) && !R.any_ring && !ms && R.max_dim[1] <= 255 &&
                       cl_geometry(H.q, R.max_dim[2], max_plane, dev,
                                   opts.kernel == 3 && opts.ctas_per_sm > 0 ? std::min(opts.ctas_per_sm, 8) : 0,
                                   P.cl_wx, pl->cluster, P.cl_slab, pl->cl_smem, pl->cl_block, P.cl_xcap);
    if (!cl_ok) pl->cluster = 0;
    if (cl_ok && P.nonlocal) {
        // row records per CTA: every local atom (at most kMaxLocalProjAtoms) x
        // its window rows on y x the slab's planes x two x-runs
        const int win_y = 2 * (int)std::floor(H.proj_rc / H.h[1]) + 2;
        const int depth = (R.max_dim[2] + pl->cluster - 1) / pl->cluster;
        P.cl_row_cap = kMaxLocalProjAtoms * std::min(win_y, kMaxProjWin) * depth * 2;
        P.cl_key_cap = depth * R.max_dim[1];
    }
    // scratch sized for the widest candidate (3 CTAs per SM, or one slot per SM for clusters)
    const int max_ctas = (int)std::min<long long>((long long)n_sm * 3, n_work);
    const size_t need = std::max(P.slot_bytes * (size_t)max_ctas,
                                 cl_ok ? cl_slot_bytes(P.n_max, pl->cluster, P.cl_slab, P.nonlocal, P.cl_row_cap, P.cl_key_cap) *
                                             (size_t)std::min<long long>(n_sm, n_work)
                                       : 0);
    if (borrow_scratch) {
        // an asynchronous call may still use the scratch: a direct plan
        // orders its stream after it, any other waits on the host (its
        // trials and its graph run on other streams)
        if (direct && H.scratch_ev) PTRY(cudaStreamWaitEvent(stream, H.scratch_ev, 0));
        if (!direct || need > H.scratch_bytes) PTRY(scratch_idle(H));
        if (need > H.scratch_bytes) {
            if (H.scratch) cudaFree(H.scratch);
            H.scratch = nullptr;
            H.scratch_bytes = 0;
            PTRY(cudaMalloc(&H.scratch, need));
            H.scratch_bytes = need;
        }
        pl->scratch = H.scratch;
    } else {
        PTRY(cudaMalloc(&pl->scratch, need));
    }
    P.scratch = (char*)pl->scratch;

    Shape shape{0, opts.block > 0 ? opts.block : 512, opts.ctas_per_sm > 0 ? opts.ctas_per_sm : 0};
    if (opts.kernel == 3) {   // the cluster kernel, forced
        if (!cl_ok)
            return fail(set_error(MD_ERR_INVALID,
                                  "opts: the cluster kernel needs mixed precision, stencil order <= 8, no "
                                  "whole-axis rings, method 0 and regions whose slabs fit in shared memory"));
        const int blk = opts.block > 0 ? opts.block : pl->cl_block;
        if (blk > cl_max_threads())
            return fail(set_error(MD_ERR_INVALID, "opts: block exceeds the cluster kernel's thread limit"));
        const int n_cl = cl_max_clusters(H.q, pl->cluster, blk, pl->cl_smem);
        if (n_cl <= 0) return fail(set_error(MD_ERR_CUDA, "the cluster kernel cannot be made resident"));
        shape = Shape{0, blk, n_cl, pl->cluster};
    } else if (opts.block > 0 && opts.kernel == 2) {
        const int K = (max_plane + opts.block - 1) / opts.block;
        if (!zm_ok || K < 1 || K > 4 || opts.block > zm_max_threads(K))
            return fail(set_error(MD_ERR_INVALID,
                                  "opts: the z-march kernel needs mixed precision, 4th or 8th order, no "
                                  "whole-axis rings and block >= m0*m1/4 within its thread limit"));
        shape.variant = K;
        if (shape.per_sm <= 0) shape.per_sm = 1;
    }
    if (opts.block <= 0 && opts.kernel != 3) {
        const std::vector<Shape> cands = candidate_shapes(pl, zm_ok, max_plane);
        md_status ts = autotune(pl, n_sm, cands, need, shape, stream);
        if (ts != MD_OK) return fail(ts);
    }
    if (shape.cluster == 0) {
        if (shape.per_sm <= 0) shape.per_sm = std::max(1, 1024 / shape.block);
        shape.per_sm = std::min(shape.per_sm, opts.precision == MD_PREC_MIXED && shape.variant == 0 ? 3 : 2);
    }
    pl->variant = shape.variant;
    pl->block = shape.block;
    pl->per_sm = shape.per_sm;
    pl->cluster = shape.cluster;
    pl->grid = grid_of(shape, n_sm, n_work);

    if (direct) {   // [reset counter, solver, accumulation] on the caller's stream, now
        PTRY(cudaMemsetAsync(pl->d_counter, 0, sizeof(unsigned int), stream));
        PTRY(launch_shape(pl, P, Shape{pl->variant, pl->block, pl->per_sm, pl->cluster}, pl->grid, stream));
        PTRY(launch_accumulate((int)nn, Pn, pl->d_xsrc, pl->d_z, pl->d_w, H.dV, rho_out, e_out, stream));
        if (!H.scratch_ev) PTRY(cudaEventCreateWithFlags(&H.scratch_ev, cudaEventDisableTiming));
        PTRY(cudaEventRecord(H.scratch_ev, stream));
        pl->launched = true;
        *out = pl;
        return MD_OK;
    }
    // capture [reset counter, solver, accumulation] once; launches replay it
    PTRY(cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal));
    {
        cudaError_t e1 = cudaMemsetAsync(pl->d_counter, 0, sizeof(unsigned int), pl->cap);
        cudaError_t e2 = launch_shape(pl, P, Shape{pl->variant, pl->block, pl->per_sm, pl->cluster}, pl->grid, pl->cap);
        cudaError_t e3 = launch_accumulate((int)nn, Pn, pl->d_xsrc, pl->d_z, pl->d_w, H.dV, rho_out, e_out, pl->cap);
        cudaError_t e4 = cudaStreamEndCapture(pl->cap, &pl->graph);
        PTRY(e1);
        PTRY(e2);
        PTRY(e3);
        PTRY(e4);
    }
    PTRY(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
#undef PTRY
    *out = pl;
    return MD_OK;
}

md_status plan_launch(md_plan* pl, cudaStream_t stream) {
    if (!pl) return set_error(MD_ERR_INVALID, "plan is NULL");
    if (pl->n_sys == 0) return MD_OK;
    PLAN_TRY(cudaEventRecord(pl->ev0, stream));
    PLAN_TRY(cudaGraphLaunch(pl->exec, stream));
    PLAN_TRY(cudaEventRecord(pl->ev1, stream));
    pl->launched = true;
    return MD_OK;
}

md_status plan_stats(md_plan* pl, cudaStream_t stream, md_stats* stats) {
    if (!pl) return set_error(MD_ERR_INVALID, "plan is NULL");
    md_stats sst;
    std::memset(&sst, 0, sizeof(sst));
    if (pl->n_sys == 0 || !pl->launched) {
        if (stats) *stats = sst;
        return MD_OK;
    }
    const long long n_sys = pl->n_sys;
    std::vector<int> h_status(n_sys), h_iters(n_sys), h_nrel(n_sys);
    std::vector<double> h_resid(n_sys);
    PLAN_TRY(cudaMemcpyAsync(h_status.data(), pl->d_status, n_sys * sizeof(int), cudaMemcpyDeviceToHost, stream));
    PLAN_TRY(cudaMemcpyAsync(h_iters.data(), pl->d_iters, n_sys * sizeof(int), cudaMemcpyDeviceToHost, stream));
    PLAN_TRY(cudaMemcpyAsync(h_nrel.data(), pl->d_nrel, n_sys * sizeof(int), cudaMemcpyDeviceToHost, stream));
    PLAN_TRY(cudaMemcpyAsync(h_resid.data(), pl->d_resid, n_sys * sizeof(double), cudaMemcpyDeviceToHost, stream));
    PLAN_TRY(cudaStreamSynchronize(stream));
    float ms = 0.f;
    PLAN_TRY(cudaEventElapsedTime(&ms, pl->ev0, pl->ev1));
    sst.n_systems = n_sys;
    sst.iters_min = 1 << 30;
    bool invalid = false, staging_failed = false;
    for (long long k = 0; k < n_sys; ++k) {
        const int s = h_status[k];
        if (s == 0) sst.n_converged++;
        else if (s == 2) sst.n_noconv++;
        else if (s == 3) sst.n_breakdown++;
        else if (s == 4) sst.n_timeout++;
        else if (s == 1) invalid = true;
        else if (s == 5) staging_failed = true;
        sst.iters_min = std::min(sst.iters_min, h_iters[k]);
        sst.iters_max = std::max(sst.iters_max, h_iters[k]);
        sst.total_iters += h_iters[k];
        if (!pl->multishift) sst.total_point_iters += (long long)h_iters[k] * pl->points[k / pl->Pn];
        sst.reliable_updates += h_nrel[k];
        sst.max_resid = std::max(sst.max_resid, h_resid[k]);
    }
    if (pl->multishift)   // one matvec sequence per node: as long as its slowest pole
        for (long long j = 0; j < pl->nn; ++j) {
            int mx = 0;
            for (int p = 0; p < pl->Pn; ++p) mx = std::max(mx, h_iters[j * pl->Pn + p]);
            sst.total_point_iters += (long long)mx * pl->points[j];
        }
    sst.iters_mean = (double)sst.total_iters / (double)n_sys;
    sst.kernel_ms = ms;
    if (stats) *stats = sst;
    if (staging_failed)
        return set_error(MD_ERR_CUDA, "a shared-memory staging copy did not complete in time");
    if (invalid)
        return set_error(MD_ERR_INVALID, "a region meets more projector atoms than the solver holds (256)");
    if (sst.n_timeout) return set_error(MD_ERR_TIMEOUT, "device time budget exhausted; outputs incomplete");
    if (sst.n_breakdown) return set_error(MD_ERR_BREAKDOWN, "COCG breakdown (r^T r ~ 0) in some systems");
    if (sst.n_noconv) return set_error(MD_ERR_NOCONV, "some systems reached maxit");
    return MD_OK;
}

md_status density_impl(const md_hamiltonian* ham, const md_poles* poles, const md_nodes* nodes,
                       const md_solver_opts* opts, double* rho_out, double* e_out, md_workspace* ckpt,
                       md_stats* stats, cudaStream_t stream) {
    md_plan* pl = nullptr;
    if (!stats) {   // asynchronous: launch, free the temporaries stream-ordered, report the launch
        md_status st = plan_create(ham, poles, nodes, opts, rho_out, e_out, ckpt, true, stream, &pl, nullptr, true);
        if (pl) plan_free(pl);
        return st;
    }
    md_status st = plan_create(ham, poles, nodes, opts, rho_out, e_out, ckpt, true, stream, &pl);
    if (st != MD_OK) return st;
    if (pl->n_sys == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        plan_free(pl);
        return MD_OK;
    }
    st = plan_launch(pl, stream);
    if (st == MD_OK) st = plan_stats(pl, stream, stats);
    plan_free(pl);
    return st;
}

// Fatal statuses end a composite call; NOCONV and BREAKDOWN leave outputs
// written and are passed on.
bool fatal(md_status st) { return st != MD_OK && st != MD_ERR_NOCONV && st != MD_ERR_BREAKDOWN; }

// Per-pole solves, then s_j from the entropy weights (when given) and the
// node-weighted totals (Section 3, Eqs. free_cg and free_cg_sampling; Eq.
// Fermi:Rho for the count).  Synchronises `stream`.
md_status free_energy_impl(const md_hamiltonian* ham, const md_poles* poles, const double* w_entropy, double kT,
                           const md_nodes* nodes, const double* node_weight, const md_solver_opts* opts,
                           double* rho_out, double* e_out, double* s_out, md_free_energy_terms* terms,
                           md_stats* stats, cudaStream_t s) {
    if (!ham || !nodes || !terms) return set_error(MD_ERR_INVALID, "ham, nodes and terms are required");
    if (s_out && !w_entropy) return set_error(MD_ERR_INVALID, "s_out needs the entropy weights");
    if (w_entropy && !(kT > 0.0)) return set_error(MD_ERR_INVALID, "the entropy term needs kT > 0");
    md_status st = check_poles(poles);
    if (st != MD_OK) return st;
    if (w_entropy)
        for (int p = 0; p < 2 * poles->n_poles; ++p)
            if (!std::isfinite(w_entropy[p])) return set_error(MD_ERR_INVALID, "entropy weights: non-finite value");
    std::memset(terms, 0, sizeof(*terms));
    const long long nn = nodes->n_nodes;
    if (nn < 0) return set_error(MD_ERR_INVALID, "nodes: negative count");
    if (nn == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return MD_OK;
    }
    const Ham& H = ham->h;
    const int Pn = poles->n_poles;
    double *d_rho = rho_out, *d_e = e_out, *d_s = s_out, *d_tot = nullptr;
    double2* d_ws = nullptr;
    md_plan* pl = nullptr;
    double h_tot[4] = {0.0, 0.0, 0.0, 0.0};
    st = MD_OK;
    MD_TRY_CUDA(cudaMallocAsync((void**)&d_tot, 4 * sizeof(double), s));
    if (!d_rho) MD_TRY_CUDA(cudaMallocAsync((void**)&d_rho, nn * sizeof(double), s));
    if (!d_e) MD_TRY_CUDA(cudaMallocAsync((void**)&d_e, nn * sizeof(double), s));
    if (w_entropy && !d_s) MD_TRY_CUDA(cudaMallocAsync((void**)&d_s, nn * sizeof(double), s));
    if (w_entropy) {
        MD_TRY_CUDA(cudaMallocAsync((void**)&d_ws, Pn * sizeof(double2), s));
        MD_TRY_CUDA(cudaMemcpyAsync(d_ws, w_entropy, Pn * sizeof(double2), cudaMemcpyHostToDevice, s));
    }
    st = plan_create(ham, poles, nodes, opts, d_rho, d_e, nullptr, true, s, &pl);
    if (st != MD_OK) goto done;
    if ((st = plan_launch(pl, s)) != MD_OK) goto done;
    st = plan_stats(pl, s, stats);
    if (fatal(st)) goto done;
    if (w_entropy) MD_TRY_CUDA(launch_entropy((int)nn, Pn, pl->d_xsrc, d_ws, kT, d_s, s));
    MD_TRY_CUDA(launch_weighted_totals(nn, d_rho, d_e, w_entropy ? d_s : nullptr, node_weight, H.dV, d_tot, s));
    MD_TRY_CUDA(cudaMemcpyAsync(h_tot, d_tot, sizeof(h_tot), cudaMemcpyDeviceToHost, s));
    MD_TRY_CUDA(cudaStreamSynchronize(s));
    terms->n_electrons = h_tot[0];
    terms->e_band = h_tot[1];
    terms->ts = h_tot[2];
    terms->free_energy = h_tot[3];
done:
    if (pl) plan_free(pl);
    if (!rho_out && d_rho) cudaFreeAsync(d_rho, s);
    if (!e_out && d_e) cudaFreeAsync(d_e, s);
    if (!s_out && d_s) cudaFreeAsync(d_s, s);
    if (d_ws) cudaFreeAsync(d_ws, s);
    if (d_tot) cudaFreeAsync(d_tot, s);
    return st;
}

// Cluster sampling of Section 3 (Eqs. free_cg, free_cg_sampling): C_q = the
// grid points within `radius` of ESP q (minimum image on periodic axes;
// inside the grid on open ones), N_q = |C_q|; every p in C_q carries
// n_q / N_q, weights of a point in several clusters summed; points ascending.
md_status cluster_sampling(const md_grid* g, int64_t n_esp, const int64_t* esp, const double* n_q, double radius,
                           int64_t* n_out, int64_t* node_out, double* weight_out) {
    if (!g || !n_out) return set_error(MD_ERR_INVALID, "grid and n_out are required");
    if (n_esp < 0 || (n_esp > 0 && (!esp || !n_q))) return set_error(MD_ERR_INVALID, "esp and n_q are required");
    if (!(radius >= 0.0) || !std::isfinite(radius)) return set_error(MD_ERR_INVALID, "radius must be finite, >= 0");
    long long N = 1;
    for (int d = 0; d < 3; ++d) {
        if (g->n[d] < 1 || !(g->h[d] > 0.0)) return set_error(MD_ERR_INVALID, "grid: need n >= 1 and h > 0");
        N *= g->n[d];
    }
    std::vector<std::pair<long long, double>> acc;
    std::vector<long long> pts;
    for (long long q = 0; q < n_esp; ++q) {
        if (esp[q] < 0 || esp[q] >= N) return set_error(MD_ERR_INVALID, "ESP index out of range");
        if (!std::isfinite(n_q[q])) return set_error(MD_ERR_INVALID, "n_q: non-finite value");
        const long long c[3] = {esp[q] % g->n[0], (esp[q] / g->n[0]) % g->n[1], esp[q] / ((long long)g->n[0] * g->n[1])};
        int reach[3];
        for (int d = 0; d < 3; ++d) reach[d] = (int)std::floor(radius / g->h[d]) + 1;
        pts.clear();
        for (int oz = -reach[2]; oz <= reach[2]; ++oz)
            for (int oy = -reach[1]; oy <= reach[1]; ++oy)
                for (int ox = -reach[0]; ox <= reach[0]; ++ox) {
                    const int o[3] = {ox, oy, oz};
                    double r2 = 0.0;
                    for (int d = 0; d < 3; ++d) r2 += (o[d] * g->h[d]) * (o[d] * g->h[d]);
                    if (r2 > radius * radius) continue;
                    long long p[3];
                    bool ok = true;
                    for (int d = 0; d < 3; ++d) {
                        p[d] = c[d] + o[d];
                        if (g->periodic[d]) {
                            p[d] %= g->n[d];
                            if (p[d] < 0) p[d] += g->n[d];
                        } else if (p[d] < 0 || p[d] >= g->n[d]) {
                            ok = false;
                        }
                    }
                    if (ok) pts.push_back(p[0] + (long long)g->n[0] * (p[1] + (long long)g->n[1] * p[2]));
                }
        std::sort(pts.begin(), pts.end());
        pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
        for (long long p : pts) acc.emplace_back(p, n_q[q] / (double)pts.size());
    }
    std::stable_sort(acc.begin(), acc.end(),
                     [](const std::pair<long long, double>& a, const std::pair<long long, double>& b) {
                         return a.first < b.first;
                     });
    std::vector<std::pair<long long, double>> merged;
    for (const auto& e : acc) {
        if (!merged.empty() && merged.back().first == e.first) merged.back().second += e.second;
        else merged.push_back(e);
    }
    const long long cap = *n_out;
    *n_out = (int64_t)merged.size();
    if (!node_out && !weight_out) return MD_OK;
    if (cap < (long long)merged.size())
        return set_error(MD_ERR_INVALID, "md_cluster_sampling: output capacity below the point count");
    for (size_t k = 0; k < merged.size(); ++k) {
        if (node_out) node_out[k] = merged[k].first;
        if (weight_out) weight_out[k] = merged[k].second;
    }
    return MD_OK;
}

// Fermi level of the pole form: mu with N(mu) = dV sum_j nu_j rho_j(mu) =
// n_electrons (Eq. Fermi:Rho with g -> r), each N(mu) from the same plan
// relaunched with the poles rebuilt at mu on the spectral interval
// (Illinois variant of regula falsi, Dowell & Jarratt, BIT 11 (1971)).
md_status fermi_level_poles(const md_hamiltonian* ham, double kT, int P, const md_nodes* nodes,
                            const double* node_weight, const md_solver_opts* opts, double n_electrons,
                            double mu_tol, double* mu_out, double* count_out, int32_t* evals_out, cudaStream_t s) {
    if (!ham || !nodes || !mu_out) return set_error(MD_ERR_INVALID, "ham, nodes and mu_out are required");
    if (!(kT > 0.0) || P < 2 || P % 2) return set_error(MD_ERR_INVALID, "need kT > 0 and an even P >= 2");
    if (!(n_electrons >= 0.0) || !std::isfinite(n_electrons))
        return set_error(MD_ERR_INVALID, "n_electrons must be finite and >= 0");
    if (!(mu_tol >= 0.0)) return set_error(MD_ERR_INVALID, "mu_tol must be >= 0");
    if (mu_tol == 0.0) mu_tol = 1e-10;
    const long long nn = nodes->n_nodes;
    if (nn < 1) return set_error(MD_ERR_INVALID, "need at least one node");
    Ham& H = const_cast<md_hamiltonian*>(ham)->h;
    md_status st = MD_OK;
    if (!H.bounds_valid && (st = compute_bounds(H, s)) != MD_OK) return st;
    const double emin = H.emin, emax = H.emax;
    std::vector<double> z(2 * P), w(2 * P);
    if ((st = make_poles(kT, 0.5 * (emin + emax), emin, emax, P, z.data(), w.data())) != MD_OK) return st;
    md_poles pz{P, z.data(), w.data()};
    double *d_rho = nullptr, *d_tot = nullptr;
    md_plan* pl = nullptr;
    int evals = 0;
    double a = emin, b = emax, fa = 0.0, fb = 0.0, mu = 0.0, fm = 0.0;
    int side = 0;
    auto count = [&](double m, double& f) -> md_status {
        md_status cs = make_poles(kT, m, emin, emax, P, z.data(), w.data());
        if (cs != MD_OK) return cs;
        cudaError_t e = cudaMemcpyAsync(pl->d_z, z.data(), P * sizeof(double2), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pl->d_w, w.data(), P * sizeof(double2), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
        if ((cs = plan_launch(pl, s)) != MD_OK) return cs;
        cs = plan_stats(pl, s, nullptr);
        if (fatal(cs)) return cs;
        double tot[4];
        e = launch_weighted_totals(nn, d_rho, nullptr, nullptr, node_weight, H.dV, d_tot, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tot, d_tot, sizeof(tot), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
        ++evals;
        f = tot[0] - n_electrons;
        return MD_OK;
    };
    MD_TRY_CUDA(cudaMallocAsync((void**)&d_rho, nn * sizeof(double), s));
    MD_TRY_CUDA(cudaMallocAsync((void**)&d_tot, 4 * sizeof(double), s));
    if ((st = plan_create(ham, &pz, nodes, opts, d_rho, nullptr, nullptr, true, s, &pl)) != MD_OK) goto done;
    if ((st = count(a, fa)) != MD_OK) goto done;
    if ((st = count(b, fb)) != MD_OK) goto done;
    if (fa > 0.0 || fb < 0.0) {
        st = set_error(MD_ERR_INVALID, "n_electrons lies outside the counts at the ends of the spectral interval");
        goto done;
    }
    mu = fa == 0.0 ? a : b;
    fm = fa == 0.0 ? fa : fb;
    while (b - a > mu_tol && evals < 200 && fm != 0.0) {
        double c = (a * fb - b * fa) / (fb - fa);
        if (!(c > a && c < b)) c = 0.5 * (a + b);
        double fc = 0.0;
        if ((st = count(c, fc)) != MD_OK) goto done;
        mu = c;
        fm = fc;
        if (fc < 0.0) {
            a = c;
            fa = fc;
            if (side == -1) fb *= 0.5;   // the same end moved twice: halve the other's value
            side = -1;
        } else {
            b = c;
            fb = fc;
            if (side == +1) fa *= 0.5;
            side = +1;
        }
    }
    *mu_out = mu;
    if (count_out) *count_out = fm + n_electrons;
    if (evals_out) *evals_out = evals;
done:
    if (pl) plan_free(pl);
    if (d_rho) cudaFreeAsync(d_rho, s);
    if (d_tot) cudaFreeAsync(d_tot, s);
    cudaStreamSynchronize(s);
    return st;
}

}  // namespace
}  // namespace md

// ---------------------------------------------------------------------------
// Density without device allocation (md_density_noalloc).
//
// For callers that cannot allocate device memory while they solve: a
// process whose GPU memory is owned by another allocator with a fixed
// budget (a framework's caching allocator, a serving engine that reserves
// its memory at start-up), or code running where an allocation would
// synchronise or be refused.  All device storage of the call (Krylov slots,
// work list, region descriptors, poles, per-system results, the work
// counter) lives in the file-scope array below, so the call itself allocates
// nothing on the device and nothing on the host heap on its success path.
// The Hamiltonian must have been built beforehand.
// ---------------------------------------------------------------------------
namespace md {
namespace {

constexpr size_t kNaScratchBytes = (size_t)MD_NOALLOC_SCRATCH_BYTES;
constexpr long long kNaMaxSystems = MD_NOALLOC_MAX_SYSTEMS;
constexpr long long kNaMaxNodes = MD_NOALLOC_MAX_NODES;
constexpr int kNaMaxPoles = MD_NOALLOC_MAX_POLES;

// layout of the static array: [descriptors and results | Krylov slots]
constexpr size_t kNaOffSys = 0;
constexpr size_t kNaOffNodes = kNaOffSys + sizeof(SysDesc) * kNaMaxSystems;
constexpr size_t kNaOffZ = kNaOffNodes + sizeof(NodeDesc) * kNaMaxNodes;
constexpr size_t kNaOffW = kNaOffZ + sizeof(double2) * kNaMaxPoles;
constexpr size_t kNaOffXsrc = kNaOffW + sizeof(double2) * kNaMaxPoles;
constexpr size_t kNaOffStatus = kNaOffXsrc + sizeof(double2) * kNaMaxSystems;
constexpr size_t kNaOffIters = kNaOffStatus + sizeof(int) * kNaMaxSystems;
constexpr size_t kNaOffNrel = kNaOffIters + sizeof(int) * kNaMaxSystems;
constexpr size_t kNaOffResid = kNaOffNrel + sizeof(int) * kNaMaxSystems;
constexpr size_t kNaOffCounter = kNaOffResid + sizeof(double) * kNaMaxSystems;
constexpr size_t kNaOffSlots = (kNaOffCounter + sizeof(unsigned int) + 255) / 256 * 256;
constexpr size_t kNaTotalBytes = kNaOffSlots + kNaScratchBytes;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_area[kNaTotalBytes];

std::mutex g_na_mutex;                       // host buffers below are shared
SysDesc g_na_sys[kNaMaxSystems];
NodeDesc g_na_nodes[kNaMaxNodes];
long long g_na_points[kNaMaxNodes];
int g_na_status[kNaMaxSystems];
int g_na_iters[kNaMaxSystems];
int g_na_nrel[kNaMaxSystems];
double g_na_resid[kNaMaxSystems];

}  // namespace
}  // namespace md

extern "C" md_status md_density_noalloc(const md_hamiltonian* ham, const md_poles* poles,
                                        const md_nodes* nodes, const md_solver_opts* opts,
                                        double* rho_out, double* e_out, md_stats* stats,
                                        void* stream_) {
    using namespace md;
    clear_error();
    std::lock_guard<std::mutex> guard(g_na_mutex);
    cudaStream_t stream = (cudaStream_t)stream_;
    {   // a captured call would replay without the host lock and race on the array
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return set_error(MD_ERR_INVALID, "md_density_noalloc cannot be captured in a CUDA graph");
        }
    }
    md_status st = check_device();
    if (st != MD_OK) return st;
    if (!ham) return set_error(MD_ERR_INVALID, "ham is NULL");
    if ((st = check_poles(poles)) != MD_OK) return st;
    if ((st = check_opts(opts)) != MD_OK) return st;
    if (!nodes || nodes->n_nodes < 0 || (nodes->n_nodes > 0 && (!nodes->node || !nodes->halfwidth)))
        return set_error(MD_ERR_INVALID, "nodes: null arrays or negative count");
    const Ham& H = ham->h;
    const long long nn = nodes->n_nodes;
    const int Pn = poles->n_poles;
    if (nn == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return MD_OK;
    }
    if (!rho_out) return set_error(MD_ERR_INVALID, "rho_out is NULL");
    if (nn > kNaMaxNodes || Pn > kNaMaxPoles || nn * Pn > kNaMaxSystems)
        return set_error(MD_ERR_INVALID,
                         "md_density_noalloc: more than MD_NOALLOC_MAX_NODES nodes, "
                         "MD_NOALLOC_MAX_POLES poles or MD_NOALLOC_MAX_SYSTEMS systems");
    // region descriptors, built as md_density builds them, into the static host buffers
    long long n_max = 0;
    for (long long j = 0; j < nn; ++j) {
        long long pts = 0;
        if ((st = build_node_desc(H, nodes->node[j], nodes->halfwidth[j], g_na_nodes[j], pts)) != MD_OK) return st;
        g_na_points[j] = pts;
        n_max = std::max(n_max, pts);
    }
    const md_solver_opts o = normalise_opts(opts);
    const size_t slot = slot_bytes_for(o.precision, n_max);
    if (slot > kNaScratchBytes)
        return set_error(MD_ERR_INVALID,
                         "md_density_noalloc: one region's Krylov vectors exceed MD_NOALLOC_SCRATCH_BYTES");
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    // the device address of the static array in the current device's context
    // (its host-side name is only a stand-in), looked up on every call so
    // that a reset context never leaves a stale address behind
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_area);
    if (e != cudaSuccess || !ptr)
        return set_error(MD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    char* base = (char*)ptr;
    const long long n_sys = nn * Pn;
    for (long long j = 0; j < nn; ++j)
        for (int p = 0; p < Pn; ++p) g_na_sys[j * Pn + p] = SysDesc{(int)j, p};
    std::sort(g_na_sys, g_na_sys + n_sys, [&](const SysDesc& a, const SysDesc& b) {
        const double ca = (double)g_na_points[a.node] / std::sqrt(poles->z[2 * a.pole + 1]);
        const double cb = (double)g_na_points[b.node] / std::sqrt(poles->z[2 * b.pole + 1]);
        if (ca != cb) return ca > cb;
        return a.node != b.node ? a.node < b.node : a.pole < b.pole;
    });
    SysDesc* d_sys = (SysDesc*)(base + kNaOffSys);
    NodeDesc* d_nodes = (NodeDesc*)(base + kNaOffNodes);
    double2* d_z = (double2*)(base + kNaOffZ);
    double2* d_w = (double2*)(base + kNaOffW);
    double2* d_xsrc = (double2*)(base + kNaOffXsrc);
    int* d_status = (int*)(base + kNaOffStatus);
    int* d_iters = (int*)(base + kNaOffIters);
    int* d_nrel = (int*)(base + kNaOffNrel);
    double* d_resid = (double*)(base + kNaOffResid);
    unsigned int* d_counter = (unsigned int*)(base + kNaOffCounter);
    char* slots = base + kNaOffSlots;
    e = cudaMemcpyAsync(d_sys, g_na_sys, n_sys * sizeof(SysDesc), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_nodes, g_na_nodes, nn * sizeof(NodeDesc), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_z, poles->z, Pn * sizeof(double2), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_w, poles->w, Pn * sizeof(double2), cudaMemcpyHostToDevice, stream);
    // the array keeps the previous call's contents: the work counter must start at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned int), stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(stream);   // copies already queued finish before the lock is released
        cudaGetLastError();
        return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    }

    SolveParams P;
    std::memset(&P, 0, sizeof(P));
    for (int d = 0; d < 3; ++d) {
        P.n[d] = H.n[d];
        P.periodic[d] = H.periodic[d];
        for (int q = 0; q < kMaxQ; ++q) P.coef[d][q] = H.coef[d][q];
    }
    P.N = H.N;
    P.q = H.q;
    P.diag = H.diag;
    P.dV = H.dV;
    P.V = H.V;
    P.V32 = H.V32;
    P.nonlocal = H.nonlocal && H.n_atoms > 0;
    P.n_atoms = H.n_atoms;
    P.proj_i0 = H.proj_i0;
    P.proj_len = H.proj_len;
    P.proj_d = H.proj_d;
    P.proj_g = H.proj_g;
    P.proj_d32 = H.proj_d32;
    P.proj_g32 = H.proj_g32;
    P.proj_C = H.proj_C;
    P.proj_C32 = H.proj_C32;
    P.proj_rows = H.proj_rows;
    P.pl_ptr = H.pl_ptr;
    P.pl_atom = H.pl_atom;
    P.pl_val32 = H.pl_val32;
    P.pl_val64 = H.pl_val64;
    P.e_s = H.e_s;
    P.e_p = H.e_p;
    P.n_sys = (int)n_sys;
    P.P = Pn;
    P.sys = d_sys;
    P.nodes = d_nodes;
    P.z = d_z;
    P.tol = o.tol;
    P.maxit = o.maxit;
    P.reliable_every = o.reliable_every;
    P.reliable_delta = o.reliable_delta;
    P.timeout_ns = o.timeout_s > 0 ? (unsigned long long)(o.timeout_s * 1e9) : 0ULL;
    P.scratch = slots;
    P.slot_bytes = slot;
    P.n_max = (int)((n_max + 63) / 64 * 64);
    P.ckpt = nullptr;
    P.ckpt_sys_off = nullptr;
    P.work_counter = d_counter;
    P.x_src = d_xsrc;
    P.status = d_status;
    P.iters = d_iters;
    P.resid = d_resid;
    P.n_rel = d_nrel;
    // one CTA of 1024 threads per SM, as many as the slots in the array allow
    const long long max_slots = (long long)(kNaScratchBytes / slot);
    const int grid = (int)std::min<long long>(std::min<long long>(n_sm, max_slots), n_sys);
    e = launch_cocg(P, o.precision, grid, 1024, 1, stream);
    if (e == cudaSuccess) e = launch_accumulate((int)nn, Pn, d_xsrc, d_z, d_w, H.dV, rho_out, e_out, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_na_status, d_status, n_sys * sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_na_iters, d_iters, n_sys * sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_na_nrel, d_nrel, n_sys * sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_na_resid, d_resid, n_sys * sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        // whatever was queued must finish before the lock is released: the
        // next call may run on another stream and would overlap on the array
        cudaStreamSynchronize(stream);
        cudaGetLastError();
        return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    }
    md_stats sst;
    std::memset(&sst, 0, sizeof(sst));
    sst.n_systems = n_sys;
    sst.iters_min = 1 << 30;
    bool invalid = false;
    for (long long k = 0; k < n_sys; ++k) {
        const int s = g_na_status[k];
        if (s == 0) sst.n_converged++;
        else if (s == 2) sst.n_noconv++;
        else if (s == 3) sst.n_breakdown++;
        else if (s == 4) sst.n_timeout++;
        else if (s == 1) invalid = true;
        sst.iters_min = std::min(sst.iters_min, g_na_iters[k]);
        sst.iters_max = std::max(sst.iters_max, g_na_iters[k]);
        sst.total_iters += g_na_iters[k];
        sst.total_point_iters += (long long)g_na_iters[k] * g_na_points[k / Pn];
        sst.reliable_updates += g_na_nrel[k];
        sst.max_resid = std::max(sst.max_resid, g_na_resid[k]);
    }
    sst.iters_mean = (double)sst.total_iters / (double)n_sys;
    if (stats) *stats = sst;
    if (invalid)
        return set_error(MD_ERR_INVALID, "a region meets more projector atoms than the solver holds (256)");
    if (sst.n_timeout) return set_error(MD_ERR_TIMEOUT, "device time budget exhausted; outputs incomplete");
    if (sst.n_breakdown) return set_error(MD_ERR_BREAKDOWN, "COCG breakdown (r^T r ~ 0) in some systems");
    if (sst.n_noconv) return set_error(MD_ERR_NOCONV, "some systems reached maxit");
    return MD_OK;
}

using namespace md;

extern "C" {

// ---- Lanczos spectral Gauss quadrature ------------------------------------

extern "C" md_status md_lssgq_rules(const md_hamiltonian* ham, const md_nodes* nodes,
                                    const md_lssgq_opts* opts, double* lambda_out, double* weight_out,
                                    int32_t* k_used_out, void* stream) {
    using namespace md;
    clear_error();
    md_status st = check_device();
    if (st != MD_OK) return st;
    if (!ham || !opts) return set_error(MD_ERR_INVALID, "ham and opts are required");
    const int K = opts->K;
    if (K < 1 || K > kMaxLanczosK) return set_error(MD_ERR_INVALID, "opts.K must be in 1..MD_LSSGQ_MAX_K");
    if (!(opts->breakdown_tol >= 0.0) || !(opts->timeout_s >= 0.0))
        return set_error(MD_ERR_INVALID, "opts: breakdown_tol and timeout_s must be >= 0");
    if (opts->block != 0 && (opts->block < 64 || opts->block > 1024 || opts->block % 32))
        return set_error(MD_ERR_INVALID, "opts.block must be 0 or a multiple of 32 in 64..1024");
    if (opts->precision != MD_PREC_FP64 && opts->precision != MD_PREC_MIXED)
        return set_error(MD_ERR_INVALID, "opts.precision must be MD_PREC_FP64 or MD_PREC_MIXED");
    Ham& H = const_cast<md_hamiltonian*>(ham)->h;
    Regions R;
    if ((st = make_regions(H, nodes, R)) != MD_OK) return st;
    const long long nn = (long long)R.desc.size();
    if (nn == 0) return MD_OK;
    if (!lambda_out || !weight_out) return set_error(MD_ERR_INVALID, "lambda_out and weight_out are required");
    if (nn > (1LL << 31) - 1) return set_error(MD_ERR_INVALID, "too many nodes");
    cudaStream_t s = (cudaStream_t)stream;

    std::vector<SysDesc> sys(nn);
    for (long long j = 0; j < nn; ++j) sys[j] = SysDesc{(int)j, 0};
    std::stable_sort(sys.begin(), sys.end(),
                     [&](const SysDesc& a, const SysDesc& b) { return R.points[a.node] > R.points[b.node]; });
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // 1,024 threads: one node per SM with every warp on its region (faster
    // than two 512-thread nodes per SM on the bulk cell, +7 % to +11 % in FP32)
    const int block = opts->block > 0 ? opts->block : 1024;
    const int per_sm = std::max(1, std::min(2, 1024 / block));
    const int grid = (int)std::min<long long>((long long)n_sm * per_sm, nn);

    SolveParams P;
    std::memset(&P, 0, sizeof(P));
    fill_operator(P, H);
    P.n_sys = (int)nn;
    P.timeout_ns = opts->timeout_s > 0 ? (unsigned long long)(opts->timeout_s * 1e9) : 0ULL;
    P.n_max = (int)((R.n_max + 63) / 64 * 64);
    const size_t elem = opts->precision == MD_PREC_MIXED ? sizeof(float) : sizeof(double);
    P.slot_bytes = ((size_t)2 * P.n_max * elem + (size_t)P.n_max * sizeof(uint2) + 511) / 512 * 512;

#define LTRY(expr)                                                                                   \
    do {                                                                                             \
        cudaError_t _e = (expr);                                                                     \
        if (_e != cudaSuccess)                                                                       \
            return set_error((_e == cudaErrorMemoryAllocation) ? MD_ERR_OOM : MD_ERR_CUDA,           \
                             std::string("CUDA: ") + cudaGetErrorString(_e) + " (" #expr ")");       \
    } while (0)
    // every call but an asynchronous md_density ends synchronised with its
    // stream; wait for the last of those before using the scratch
    LTRY(scratch_idle(H));
    const size_t need = P.slot_bytes * (size_t)grid;
    if (need > H.scratch_bytes) {
        LTRY(cudaStreamSynchronize(s));
        if (H.scratch) cudaFree(H.scratch);
        H.scratch = nullptr;
        H.scratch_bytes = 0;
        LTRY(cudaMalloc(&H.scratch, need));
        H.scratch_bytes = need;
    }
    P.scratch = (char*)H.scratch;
    auto up256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t o_nodes = up256(nn * sizeof(SysDesc));
    const size_t o_alpha = o_nodes + up256(nn * sizeof(NodeDesc));
    const size_t o_beta = o_alpha + up256((size_t)nn * K * sizeof(double));
    const size_t o_kused = o_beta + up256((size_t)nn * K * sizeof(double));
    const size_t o_status = o_kused + up256(nn * sizeof(int));
    const size_t o_counter = o_status + up256(nn * sizeof(int));
    const size_t lz_need = o_counter + 256;
    if (lz_need > H.lz_bytes) {
        LTRY(cudaStreamSynchronize(s));
        if (H.lz_buf) cudaFree(H.lz_buf);
        H.lz_buf = nullptr;
        H.lz_bytes = 0;
        LTRY(cudaMalloc(&H.lz_buf, lz_need));
        H.lz_bytes = lz_need;
    }
    char* lz = (char*)H.lz_buf;
    SysDesc* d_sys = (SysDesc*)lz;
    NodeDesc* d_nodes = (NodeDesc*)(lz + o_nodes);
    double* d_alpha = (double*)(lz + o_alpha);
    double* d_beta = (double*)(lz + o_beta);
    int* d_kused = (int*)(lz + o_kused);
    int* d_status = (int*)(lz + o_status);
    unsigned int* d_counter = (unsigned int*)(lz + o_counter);
    LTRY(cudaMemcpyAsync(d_sys, sys.data(), nn * sizeof(SysDesc), cudaMemcpyHostToDevice, s));
    LTRY(cudaMemcpyAsync(d_nodes, R.desc.data(), nn * sizeof(NodeDesc), cudaMemcpyHostToDevice, s));
    LTRY(cudaMemsetAsync(d_counter, 0, sizeof(unsigned int), s));
    LTRY(cudaMemsetAsync(d_kused, 0, nn * sizeof(int), s));
    P.sys = d_sys;
    P.nodes = d_nodes;
    P.work_counter = d_counter;
    LanczosParams L;
    L.K = K;
    L.breakdown_tol = opts->breakdown_tol > 0 ? opts->breakdown_tol : 1e-13;
    L.alpha = d_alpha;
    L.beta = d_beta;
    L.k_used = d_kused;
    L.status = d_status;
    LTRY(launch_lanczos(P, L, opts->precision, grid, block, s));
    LTRY(launch_gauss_rules((int)nn, L, lambda_out, weight_out, s));
    if (k_used_out)
        LTRY(cudaMemcpyAsync(k_used_out, d_kused, nn * sizeof(int), cudaMemcpyDeviceToDevice, s));
    std::vector<int> h_status(nn);
    LTRY(cudaMemcpyAsync(h_status.data(), d_status, nn * sizeof(int), cudaMemcpyDeviceToHost, s));
    LTRY(cudaStreamSynchronize(s));
#undef LTRY
    int worst = 0;
    for (int v : h_status) worst = (v == 4 || worst == 4) ? 4 : std::max(worst, v);
    if (worst == 4) return set_error(MD_ERR_TIMEOUT, "device time budget exhausted; rules incomplete");
    if (worst == 1)
        return set_error(MD_ERR_INVALID, "a region meets more projector atoms than the solver holds (256)");
    if (worst == 3) return set_error(MD_ERR_BREAKDOWN, "the tridiagonal QR did not converge for some node");
    return MD_OK;
}

extern "C" md_status md_lssgq_fields(int64_t n_nodes, int32_t K, const double* lambda, const double* weight,
                                     double mu, double kT, double dV, double* rho_out, double* e_out,
                                     double* s_out, void* stream) {
    using namespace md;
    clear_error();
    md_status st = check_device();
    if (st != MD_OK) return st;
    if (n_nodes < 0 || n_nodes > (1LL << 31) - 1 || K < 1 || K > kMaxLanczosK)
        return set_error(MD_ERR_INVALID, "n_nodes or K out of range");
    if (!(kT > 0.0) || !(dV > 0.0) || !std::isfinite(mu))
        return set_error(MD_ERR_INVALID, "kT and dV must be > 0 and mu finite");
    if (n_nodes == 0) return MD_OK;
    if (!lambda || !weight || !rho_out) return set_error(MD_ERR_INVALID, "lambda, weight and rho_out are required");
    cudaError_t e = launch_lssgq_fields((int)n_nodes, K, lambda, weight, mu, kT, dV, rho_out, e_out, s_out,
                                        (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    return MD_OK;
}

extern "C" md_status md_fermi_level(int64_t n_nodes, int32_t K, const double* lambda, const double* weight,
                                    const double* node_weight, double kT, double n_electrons, double* mu_out,
                                    double* count_out, void* stream) {
    using namespace md;
    clear_error();
    md_status st = check_device();
    if (st != MD_OK) return st;
    if (n_nodes < 1 || n_nodes > (1LL << 31) - 1 || K < 1 || K > kMaxLanczosK)
        return set_error(MD_ERR_INVALID, "n_nodes or K out of range");
    if (!(kT > 0.0) || !(n_electrons >= 0.0) || !std::isfinite(n_electrons))
        return set_error(MD_ERR_INVALID, "kT must be > 0 and n_electrons finite and >= 0");
    if (!lambda || !weight || !mu_out) return set_error(MD_ERR_INVALID, "lambda, weight and mu_out are required");
    cudaStream_t s = (cudaStream_t)stream;
    double* d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_out, 3 * sizeof(double));
    if (e == cudaSuccess) e = launch_fermi_level((int)n_nodes, K, lambda, weight, node_weight, kT, n_electrons,
                                                 d_out, s);
    double h[3] = {0.0, 0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_out);
    if (e != cudaSuccess)
        return set_error(e == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA,
                         std::string("CUDA: ") + cudaGetErrorString(e));
    *mu_out = h[0];
    if (count_out) *count_out = h[1];
    return MD_OK;
}


md_status md_fma_rate(int32_t precision, void* stream, double* tflops_out) {
    clear_error();
    if (!tflops_out || (precision != MD_PREC_FP64 && precision != MD_PREC_MIXED))
        return set_error(MD_ERR_INVALID, "md_fma_rate: need tflops_out and MD_PREC_FP64 or MD_PREC_MIXED");
    md_status st = check_device();
    if (st != MD_OK) return st;
    return fma_rate_probe(precision, (cudaStream_t)stream, tflops_out);
}

const char* md_last_error(void) { return md::g_last_error.c_str(); }

const char* md_version(void) { return "macrodft-gb300 0.1 (sm_103a)"; }

md_status md_make_poles(double kT, double mu, double emin, double emax, int32_t P, double* z_out,
                        double* w_out) {
    clear_error();
    return make_poles(kT, mu, emin, emax, P, z_out, w_out);
}

md_status md_build_hamiltonian(const md_grid* grid, const md_atoms* atoms, const md_pot_params* pot,
                               void* stream, md_hamiltonian** out) {
    clear_error();
    if (!out) return set_error(MD_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!grid || !atoms || !pot) return set_error(MD_ERR_INVALID, "grid, atoms and pot are required");
    for (int d = 0; d < 3; ++d) {
        if (grid->n[d] < 1) return set_error(MD_ERR_INVALID, "grid: need n >= 1 on every axis");
        if (!(grid->h[d] > 0.0) || !std::isfinite(grid->h[d]))
            return set_error(MD_ERR_INVALID, "grid: spacing must be positive");
    }
    if (grid->fd_order < 2 || grid->fd_order > 2 * kMaxQ || grid->fd_order % 2)
        return set_error(MD_ERR_INVALID, "grid: fd_order must be even, 2..16");
    if (atoms->n < 0 || (atoms->n > 0 && (!atoms->xyz || !atoms->depth || !atoms->sigma)))
        return set_error(MD_ERR_INVALID, "atoms: null arrays");
    for (long long a = 0; a < atoms->n; ++a) {
        if (!(atoms->sigma[a] > 0.0) || !std::isfinite(atoms->depth[a]) ||
            !std::isfinite(atoms->xyz[3 * a]) || !std::isfinite(atoms->xyz[3 * a + 1]) ||
            !std::isfinite(atoms->xyz[3 * a + 2]))
            return set_error(MD_ERR_INVALID, "atoms: need finite positions/depths and sigma > 0");
    }
    if (!(pot->cutoff_sigmas > 0.0)) return set_error(MD_ERR_INVALID, "pot: cutoff_sigmas must be > 0");
    const long long N = (long long)grid->n[0] * grid->n[1] * grid->n[2];
    if (pot->v_ext)
        for (long long i = 0; i < N; ++i)
            if (!std::isfinite(pot->v_ext[i])) return set_error(MD_ERR_INVALID, "pot: non-finite v_ext");
    if (pot->nonlocal) {
        if (!(pot->proj_sigma > 0.0) || !(pot->proj_rc > 0.0))
            return set_error(MD_ERR_INVALID, "pot: projector sigma and cutoff must be > 0");
        for (int d = 0; d < 3; ++d) {
            if (grid->periodic[d] && !(grid->n[d] * grid->h[d] > 2.0 * pot->proj_rc))
                return set_error(MD_ERR_INVALID, "pot: nonlocal needs every periodic box length > 2 proj_rc");
            if (2.0 * std::floor(pot->proj_rc / grid->h[d]) + 2 > kMaxProjWin)
                return set_error(MD_ERR_INVALID, "pot: proj_rc / h too large for the projector window");
        }
    }
    md_status st = check_device();
    if (st != MD_OK) return st;
    md_hamiltonian* hp = new md_hamiltonian();
    Ham& H = hp->h;
    for (int d = 0; d < 3; ++d) {
        H.n[d] = grid->n[d];
        H.h[d] = grid->h[d];
        H.periodic[d] = grid->periodic[d] ? 1 : 0;
    }
    H.fd_order = grid->fd_order;
    H.q = grid->fd_order / 2;
    H.N = N;
    H.dV = H.h[0] * H.h[1] * H.h[2];
    cudaGetDevice(&H.device);
    {
        double w[kMaxQ + 1];
        fornberg_second_derivative(H.q, w);
        H.diag = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double h2 = H.h[d] * H.h[d];
            for (int o = 0; o < kMaxQ; ++o) H.coef[d][o] = o < H.q ? -0.5 * w[o + 1] / h2 : 0.0;
            H.diag += -0.5 * w[0] / h2;
        }
    }
    H.n_atoms = atoms->n;
    H.cutoff_sigmas = pot->cutoff_sigmas;
    H.nonlocal = pot->nonlocal ? 1 : 0;
    H.proj_sigma = pot->proj_sigma;
    H.proj_rc = pot->proj_rc;
    H.e_s = pot->e_s;
    H.e_p = pot->e_p;
    st = build_hamiltonian_device(H, atoms, pot, (cudaStream_t)stream);
    if (st != MD_OK) {
        free_ham(H);
        delete hp;
        return st;
    }
    *out = hp;
    return MD_OK;
}

md_status md_hamiltonian_destroy(md_hamiltonian* ham) {
    clear_error();
    if (!ham) return MD_OK;
    free_ham(ham->h);
    delete ham;
    return MD_OK;
}

md_status md_hamiltonian_potential(const md_hamiltonian* ham, double* V_out, void* stream) {
    clear_error();
    if (!ham || !V_out) return set_error(MD_ERR_INVALID, "ham and V_out are required");
    cudaError_t e = cudaMemcpyAsync(V_out, ham->h.V, ham->h.N * sizeof(double), cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(MD_ERR_CUDA, cudaGetErrorString(e));
    return MD_OK;
}

md_status md_spectral_bounds(const md_hamiltonian* ham, void* stream, double* emin, double* emax) {
    clear_error();
    if (!ham || !emin || !emax) return set_error(MD_ERR_INVALID, "ham, emin and emax are required");
    Ham& H = const_cast<md_hamiltonian*>(ham)->h;
    if (!H.bounds_valid) {
        md_status st = compute_bounds(H, stream);
        if (st != MD_OK) return st;
    }
    *emin = H.emin;
    *emax = H.emax;
    return MD_OK;
}

md_status md_workspace_create(const md_hamiltonian* ham, const md_nodes* nodes, int32_t n_poles,
                              md_workspace** out) {
    clear_error();
    if (!out) return set_error(MD_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!ham || n_poles < 1) return set_error(MD_ERR_INVALID, "ham and n_poles >= 1 are required");
    Regions R;
    md_status st = make_regions(ham->h, nodes, R);
    if (st != MD_OK) return st;
    md_workspace* ws = new md_workspace();
    ws->device = ham->h.device;
    ws->n_nodes = (long long)R.desc.size();
    ws->n_poles = n_poles;
    ws->total_points = R.total;
    ws->node_off = new long long[std::max<long long>(ws->n_nodes, 1)];
    long long off = 0;
    for (long long j = 0; j < ws->n_nodes; ++j) {
        ws->node_off[j] = off;
        off += R.points[j];
    }
    ws->x = nullptr;
    const size_t bytes = (size_t)n_poles * (size_t)std::max<long long>(R.total, 1) * 16;
    cudaError_t e = cudaMalloc((void**)&ws->x, bytes);
    if (e != cudaSuccess) {
        delete[] ws->node_off;
        delete ws;
        return set_error(e == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA,
                         std::string("workspace: ") + cudaGetErrorString(e));
    }
    *out = ws;
    return MD_OK;
}

md_status md_workspace_destroy(md_workspace* ws) {
    clear_error();
    if (!ws) return MD_OK;
    cudaFree(ws->x);
    delete[] ws->node_off;
    delete ws;
    return MD_OK;
}

md_status md_density(const md_hamiltonian* ham, const md_poles* poles, const md_nodes* nodes,
                     const md_solver_opts* opts, double* rho_out, double* e_out, md_workspace* ckpt,
                     md_stats* stats, void* stream) {
    clear_error();
    return density_impl(ham, poles, nodes, opts, rho_out, e_out, ckpt, stats, (cudaStream_t)stream);
}

md_status md_energy(const md_hamiltonian* ham, const md_poles* poles, const md_nodes* nodes,
                    const double* node_weight, const md_solver_opts* opts, double* e_out, double* e_band,
                    md_stats* stats, void* stream) {
    clear_error();
    if (!e_band) return set_error(MD_ERR_INVALID, "e_band is NULL");
    md_free_energy_terms t;
    md_status st = free_energy_impl(ham, poles, nullptr, 0.0, nodes, node_weight, opts, nullptr, e_out, nullptr,
                                    &t, stats, (cudaStream_t)stream);
    if (st == MD_OK || st == MD_ERR_NOCONV || st == MD_ERR_BREAKDOWN) *e_band = t.e_band;
    return st;
}

md_status md_free_energy(const md_hamiltonian* ham, const md_poles* poles, const double* w_entropy, double kT,
                         const md_nodes* nodes, const double* node_weight, const md_solver_opts* opts,
                         double* rho_out, double* e_out, double* s_out, md_free_energy_terms* terms,
                         md_stats* stats, void* stream) {
    clear_error();
    return free_energy_impl(ham, poles, w_entropy, kT, nodes, node_weight, opts, rho_out, e_out, s_out, terms,
                            stats, (cudaStream_t)stream);
}

md_status md_make_entropy_weights(double kT, double mu, double emin, double emax, int32_t P, double* w_out) {
    clear_error();
    return make_entropy_weights(kT, mu, emin, emax, P, w_out);
}

md_status md_cluster_sampling(const md_grid* grid, int64_t n_esp, const int64_t* esp, const double* n_q,
                              double radius, int64_t* n_out, int64_t* node_out, double* weight_out) {
    clear_error();
    return cluster_sampling(grid, n_esp, esp, n_q, radius, n_out, node_out, weight_out);
}

md_status md_fermi_level_poles(const md_hamiltonian* ham, double kT, int32_t P, const md_nodes* nodes,
                               const double* node_weight, const md_solver_opts* opts, double n_electrons,
                               double mu_tol, double* mu_out, double* count_out, int32_t* evals_out,
                               void* stream) {
    clear_error();
    return fermi_level_poles(ham, kT, P, nodes, node_weight, opts, n_electrons, mu_tol, mu_out, count_out,
                             evals_out, (cudaStream_t)stream);
}

md_status md_density_adjoint(const md_hamiltonian* ham, const md_poles* poles, const md_nodes* nodes,
                             const md_solver_opts* opts, const double* dL_drho, const double* dL_de,
                             md_workspace* ckpt, double* dL_dV_out, double* forces_out, md_stats* stats,
                             void* stream) {
    clear_error();
    md_status st = check_device();
    if (st != MD_OK) return st;
    if (!ham || !dL_dV_out) return set_error(MD_ERR_INVALID, "ham and dL_dV_out are required");
    if ((st = check_poles(poles)) != MD_OK) return st;
    Ham& H = const_cast<md_hamiltonian*>(ham)->h;
    cudaStream_t s = (cudaStream_t)stream;
    Regions R;
    if ((st = make_regions(H, nodes, R)) != MD_OK) return st;
    if (!dL_drho && R.desc.size() > 0) return set_error(MD_ERR_INVALID, "dL_drho is NULL");
    if (forces_out && H.nonlocal && H.n_atoms > 0)
        return set_error(MD_ERR_INVALID, "forces need a Hamiltonian without the nonlocal term");
    if (forces_out && H.n_atoms == 0) return set_error(MD_ERR_INVALID, "forces need atoms");
    md_workspace* own = nullptr;
    NodeDesc* d_nodes = nullptr;
    long long* d_off = nullptr;
    double2* d_z = nullptr;
    double2* d_w = nullptr;
    const long long nn = (long long)R.desc.size();
    md_status solve_st = MD_OK;
    AdjointParams A;
    std::memset(&A, 0, sizeof(A));
    if (!ckpt) {
        if ((st = check_opts(opts)) != MD_OK) return st;
        if ((st = md_workspace_create(ham, nodes, poles->n_poles, &own)) != MD_OK) return st;
        ckpt = own;
        std::vector<double> dummy;
        double* d_rho = nullptr;
        cudaMallocAsync((void**)&d_rho, std::max<long long>(nn, 1) * sizeof(double), s);
        solve_st = density_impl(ham, poles, nodes, opts, d_rho, nullptr, ckpt, stats, s);
        cudaFreeAsync(d_rho, s);
        if (solve_st == MD_ERR_INVALID || solve_st == MD_ERR_CUDA || solve_st == MD_ERR_OOM ||
            solve_st == MD_ERR_TIMEOUT) {
            st = solve_st;
            goto done;
        }
    } else if (ckpt->n_nodes != nn || ckpt->n_poles != poles->n_poles || ckpt->total_points != R.total) {
        return set_error(MD_ERR_INVALID, "checkpoint workspace was made for other nodes or poles");
    }
    MD_TRY_CUDA(cudaMemsetAsync(dL_dV_out, 0, H.N * sizeof(double), s));
    if (nn > 0) {
        if ((st = upload_poles(poles, &d_z, &d_w, s)) != MD_OK) goto done;
        MD_TRY_CUDA(cudaMallocAsync((void**)&d_nodes, nn * sizeof(NodeDesc), s));
        MD_TRY_CUDA(cudaMallocAsync((void**)&d_off, nn * sizeof(long long), s));
        MD_TRY_CUDA(cudaMemcpyAsync(d_nodes, R.desc.data(), nn * sizeof(NodeDesc), cudaMemcpyHostToDevice, s));
        MD_TRY_CUDA(cudaMemcpyAsync(d_off, ckpt->node_off, nn * sizeof(long long), cudaMemcpyHostToDevice, s));
        for (int d = 0; d < 3; ++d) A.n[d] = H.n[d];
        A.n_nodes = nn;
        A.P = poles->n_poles;
        A.nodes = d_nodes;
        A.node_off = d_off;
        A.ckpt = (const double2*)ckpt->x;
        A.z = d_z;
        A.w = d_w;
        A.dL_drho = dL_drho;
        A.dL_de = dL_de;
        A.dV = H.dV;
        A.dLdV = dL_dV_out;
        MD_TRY_CUDA(launch_adjoint_dV(A, s));
    }
    if (forces_out) {
        ForceParams F;
        for (int d = 0; d < 3; ++d) {
            F.n[d] = H.n[d];
            F.h[d] = H.h[d];
            F.periodic[d] = H.periodic[d];
        }
        F.n_atoms = H.n_atoms;
        F.xyz = H.atom_xyz;
        F.depth = H.atom_depth;
        F.sigma = H.atom_sigma;
        F.cutoff_sigmas = H.cutoff_sigmas;
        F.dLdV = dL_dV_out;
        F.forces = forces_out;
        MD_TRY_CUDA(launch_forces(F, s));
    }
    MD_TRY_CUDA(cudaStreamSynchronize(s));
    st = solve_st;
done:
    cudaFreeAsync(d_nodes, s);
    cudaFreeAsync(d_off, s);
    cudaFreeAsync(d_z, s);
    cudaFreeAsync(d_w, s);
    if (own) {
        cudaStreamSynchronize(s);
        md_workspace_destroy(own);
    }
    return st;
}

md_status md_density_fused_adjoint(const md_hamiltonian* ham, const md_poles* poles,
                                   const md_nodes* nodes, const md_solver_opts* opts,
                                   const double* dL_drho, const double* dL_de, double* rho_out,
                                   double* e_out, double* dL_dV_out, double* forces_out, md_stats* stats,
                                   void* stream) {
    clear_error();
    md_status st = check_device();
    if (st != MD_OK) return st;
    if (!ham || !dL_dV_out) return set_error(MD_ERR_INVALID, "ham and dL_dV_out are required");
    const Ham& H = ham->h;
    if (forces_out && H.nonlocal && H.n_atoms > 0)
        return set_error(MD_ERR_INVALID, "forces need a Hamiltonian without the nonlocal term");
    if (forces_out && H.n_atoms == 0) return set_error(MD_ERR_INVALID, "forces need atoms");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(dL_dV_out, 0, H.N * sizeof(double), s);
    if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    FusedArgs fa{dL_dV_out, dL_drho, dL_de, nullptr, nullptr};
    md_plan* pl = nullptr;
    st = plan_create(ham, poles, nodes, opts, rho_out, e_out, nullptr, true, s, &pl, &fa);
    if (st != MD_OK) return st;
    if (pl->n_sys == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        plan_free(pl);
        return MD_OK;
    }
    st = plan_launch(pl, s);
    md_status st2 = MD_OK;
    if (st == MD_OK) st2 = plan_stats(pl, s, stats);
    plan_free(pl);
    if (st != MD_OK) return st;
    if (st2 == MD_ERR_CUDA || st2 == MD_ERR_INVALID || st2 == MD_ERR_TIMEOUT) return st2;
    if (forces_out) {
        ForceParams F;
        for (int d = 0; d < 3; ++d) {
            F.n[d] = H.n[d];
            F.h[d] = H.h[d];
            F.periodic[d] = H.periodic[d];
        }
        F.n_atoms = H.n_atoms;
        F.xyz = H.atom_xyz;
        F.depth = H.atom_depth;
        F.sigma = H.atom_sigma;
        F.cutoff_sigmas = H.cutoff_sigmas;
        F.dLdV = dL_dV_out;
        F.forces = forces_out;
        e = launch_forces(F, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    }
    return st2;
}

md_status md_density_matrix_rows(const md_hamiltonian* ham, const md_poles* poles, const md_nodes* nodes,
                                 const md_solver_opts* opts, double* rho_out, double* e_out,
                                 double* rows_out, md_stats* stats, void* stream) {
    clear_error();
    md_status st = check_device();
    if (st != MD_OK) return st;
    if (!ham || !nodes) return set_error(MD_ERR_INVALID, "ham and nodes are required");
    if (opts && opts->method == 1) return set_error(MD_ERR_INVALID, "density-matrix rows need method 0");
    Regions R;
    if ((st = make_regions(ham->h, nodes, R)) != MD_OK) return st;
    const long long nn = (long long)R.desc.size();
    if (nn > 0 && !rows_out) return set_error(MD_ERR_INVALID, "rows_out is NULL");
    std::vector<long long> off(nn + 1, 0);
    for (long long j = 0; j < nn; ++j) off[j + 1] = off[j] + R.points[j];
    cudaStream_t s = (cudaStream_t)stream;
    long long* d_off = nullptr;
    auto cu = [&](cudaError_t e) -> md_status {
        if (e == cudaSuccess) return MD_OK;
        cudaFree(d_off);
        return set_error(e == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA,
                         std::string("CUDA: ") + cudaGetErrorString(e));
    };
    if (nn > 0) {
        if ((st = cu(cudaMalloc(&d_off, (nn + 1) * sizeof(long long)))) != MD_OK) return st;
        if ((st = cu(cudaMemcpyAsync(d_off, off.data(), (nn + 1) * sizeof(long long), cudaMemcpyHostToDevice, s))) !=
            MD_OK)
            return st;
        if ((st = cu(cudaMemsetAsync(rows_out, 0, off[nn] * sizeof(double), s))) != MD_OK) return st;
    }
    md_solver_opts o = opts ? *opts : md_solver_opts{};
    if (!opts) {
        o.tol = 1e-10;
        o.maxit = 20000;
        o.precision = MD_PREC_MIXED;
    }
    if (o.kernel == 2) o.kernel = 1;   // the row epilogue lives in the generic kernel
    FusedArgs fa{nullptr, nullptr, nullptr, rows_out, d_off};
    md_plan* pl = nullptr;
    st = plan_create(ham, poles, nodes, &o, rho_out, e_out, nullptr, true, s, &pl, &fa);
    if (st != MD_OK) {
        cudaFree(d_off);
        return st;
    }
    md_status st2 = MD_OK;
    if (pl->n_sys > 0) {
        st = plan_launch(pl, s);
        if (st == MD_OK) st2 = plan_stats(pl, s, stats);
    } else if (stats) {
        std::memset(stats, 0, sizeof(*stats));
    }
    plan_free(pl);
    cudaStreamSynchronize(s);
    cudaFree(d_off);
    return st != MD_OK ? st : st2;
}

md_status md_plan_create(const md_hamiltonian* ham, const md_poles* poles, const md_nodes* nodes,
                         const md_solver_opts* opts, double* rho_out, double* e_out, md_workspace* ckpt,
                         void* stream, md_plan** out) {
    clear_error();
    if (!out) return set_error(MD_ERR_INVALID, "out is NULL");
    return plan_create(ham, poles, nodes, opts, rho_out, e_out, ckpt, false, (cudaStream_t)stream, out);
}

md_status md_plan_launch(md_plan* plan, void* stream) {
    clear_error();
    return plan_launch(plan, (cudaStream_t)stream);
}

md_status md_plan_stats(md_plan* plan, void* stream, md_stats* stats) {
    clear_error();
    return plan_stats(plan, (cudaStream_t)stream, stats);
}

md_status md_plan_launch_shape(const md_plan* plan, int32_t* block, int32_t* grid) {
    clear_error();
    if (!plan || !block || !grid) return set_error(MD_ERR_INVALID, "plan, block and grid are required");
    *block = plan->block;
    *grid = plan->grid;
    return MD_OK;
}

md_status md_plan_system_info(md_plan* plan, void* stream, int32_t* status, int32_t* iters,
                              double* resid) {
    clear_error();
    if (!plan || !status || !iters || !resid) return set_error(MD_ERR_INVALID, "plan and outputs are required");
    if (plan->n_sys == 0) return MD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(status, plan->d_status, plan->n_sys * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(iters, plan->d_iters, plan->n_sys * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(resid, plan->d_resid, plan->n_sys * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    return MD_OK;
}

md_status md_plan_destroy(md_plan* plan) {
    clear_error();
    plan_free(plan);
    return MD_OK;
}

md_status md_hamiltonian_set_potential(md_hamiltonian* ham, const double* V_in, void* stream) {
    clear_error();
    if (!ham || !V_in) return set_error(MD_ERR_INVALID, "ham and V_in are required");
    // after any asynchronous md_density still reading the old potential
    if (ham->h.scratch_ev) {
        const cudaError_t e = cudaStreamWaitEvent((cudaStream_t)stream, ham->h.scratch_ev, 0);
        if (e != cudaSuccess) return set_error(MD_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    }
    return set_potential_device(ham->h, V_in, stream);
}

md_status md_fd_weights(int32_t order, double* w_out) {
    clear_error();
    if (order < 2 || order > 2 * kMaxQ || order % 2 || !w_out)
        return set_error(MD_ERR_INVALID, "md_fd_weights: order must be even, 2..16");
    fornberg_second_derivative(order / 2, w_out);
    return MD_OK;
}

}  // extern "C"
