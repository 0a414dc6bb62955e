/*
 * macrodft.h -- C ABI of the GB300 nodal-density library.
 *
 * The library computes the electron density at sampled grid nodes as the
 * diagonal of the finite-temperature density matrix, rho_p = 2 h^-3
 * <e_p| g(H) |e_p> (arXiv:1907.02604, Section 2.1, Eqs. (dm) and
 * (Electron_density:GQ)), with the Fermi-Dirac function g replaced by a
 * P-pole rational approximation r(eps) = sum_p Im(w_p / (eps - z_p)) and
 * H replaced by its restriction H_R to a cube around each node (the
 * locality argument of Section 2.1).  Every (node j, pole z_p) pair is one
 * complex-symmetric solve (H_R - z_p I) x = e_j done with COCG on the GPU:
 *
 *     rho_j = (2/dV) sum_p Im( w_p x_jp(j) )
 *     e_j   = 2 sum_p Im( w_p (1 + z_p x_jp(j)) )        (band energy)
 *
 * Conventions (all entry points):
 *   - Grid arrays are flat, x fastest: g = ix + nx*(iy + ny*iz).
 *   - Pointers documented "device" are CUDA device pointers owned by the
 *     caller; "host" pointers are read during the call only.  The library
 *     owns only the opaque handles it returns, each with a destroy call.
 *   - Calls are asynchronous on the given stream (cudaStream_t passed as
 *     void*, NULL = legacy default stream) unless documented otherwise.
 *   - On error the call returns a non-zero md_status, launches nothing
 *     (validation errors) and md_last_error() describes the problem.
 *   - Complex numbers are interleaved doubles (re, im).
 *   - Requires an sm_103a GPU; every compute entry point returns
 *     MD_ERR_CUDA when no such device is present.
 *   - Threads: calls on different Hamiltonian handles may run from
 *     different host threads at once.  Calls on one handle that solve
 *     (md_density, md_energy, md_density_adjoint, md_density_fused_adjoint,
 *     md_density_matrix_rows, md_lssgq_rules) share scratch the handle
 *     caches, so issue them from one thread at a time.  Each of them but
 *     the asynchronous form of md_density ends synchronised with its
 *     stream; the handle orders every solving call after the last
 *     asynchronous md_density on it (the stream waits on an event, or the
 *     host does), so consecutive calls never overlap on the GPU, whatever
 *     streams they use.  A plan (md_plan_create) owns its own scratch.
 */
#ifndef MACRODFT_H
#define MACRODFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MD_OK = 0,
    MD_ERR_INVALID = 1,    /* bad argument; nothing launched */
    MD_ERR_NOCONV = 2,     /* outputs written, some systems hit maxit */
    MD_ERR_BREAKDOWN = 3,  /* outputs written, some systems broke down (r^T r ~ 0) */
    MD_ERR_TIMEOUT = 4,    /* device deadline passed; outputs incomplete */
    MD_ERR_OOM = 5,        /* device allocation failed */
    MD_ERR_CUDA = 6        /* CUDA runtime error or no usable device */
} md_status;

typedef enum { MD_PREC_FP64 = 0, MD_PREC_MIXED = 1 } md_precision;

/* Uniform real-space grid (Section 2.1: uniform spacing h, finite
 * differences of order fd_order).  Spacing may differ per axis; dV =
 * h[0]*h[1]*h[2] plays the role of the paper's h^3. */
typedef struct {
    int32_t n[3];          /* points per axis (x, y, z), each >= 1 */
    double h[3];           /* spacing, bohr, > 0 */
    int32_t periodic[3];   /* 1 = periodic axis, 0 = open (Dirichlet) */
    int32_t fd_order;      /* even, 2..16: 2q-order central Laplacian */
} md_grid;

/* Atoms carrying Gaussian wells V_a(r) = -depth exp(-|r-R|^2/(2 sigma^2)).
 * Host arrays, read during md_build_hamiltonian only. */
typedef struct {
    int64_t n;
    const double* xyz;     /* host, 3n, bohr, (x, y, z) per atom */
    const double* depth;   /* host, n, Ha */
    const double* sigma;   /* host, n, bohr, > 0 */
} md_atoms;

/* Potential model: local wells (minimum-image distance on periodic axes,
 * cut at cutoff_sigmas*sigma), an optional additive grid potential, and an
 * optional separable nonlocal term sum_{a,l} E_l dV |p_al><p_al| with four
 * Gaussian projectors per atom (s, p_x, p_y, p_z; g = exp(-r^2/(2
 * proj_sigma^2)), p_s = C g, p_alpha = C (r_alpha - R_alpha) g, zero beyond
 * proj_rc, each normalised to dV sum p^2 = 1 on the grid).  The nonlocal
 * term needs every periodic box length > 2*proj_rc. */
typedef struct {
    double cutoff_sigmas;  /* > 0 (8.0 in the shipped workloads) */
    const double* v_ext;   /* host, N = nx*ny*nz additive potential (Ha) or NULL */
    int32_t nonlocal;      /* 0 or 1 */
    double proj_sigma;     /* bohr */
    double proj_rc;        /* bohr */
    double e_s;            /* Ha, energy of the s projector */
    double e_p;            /* Ha, energy of the three p projectors */
} md_pot_params;

typedef struct md_hamiltonian md_hamiltonian;   /* opaque, device resident */
typedef struct md_workspace md_workspace;       /* opaque checkpoint of x_jp */

/* Pole set of the rational Fermi approximation (host arrays). */
typedef struct {
    int32_t n_poles;       /* P >= 1 */
    const double* z;       /* host, 2P: poles, Im z > 0 */
    const double* w;       /* host, 2P: weights */
} md_poles;

/* Sampled nodes (the paper's electronic sampling points, Section 2.2) and
 * the half-width s of each node's cubic region: the region is the
 * (2s+1)^3 cube centred on the node, wrapped on periodic axes; where
 * 2s+1 >= n on a periodic axis the region spans the whole axis as a ring.
 * On an open axis the cube must stay inside the grid. */
typedef struct {
    int64_t n_nodes;
    const int64_t* node;       /* host, n_nodes grid indices */
    const int32_t* halfwidth;  /* host, n_nodes, s >= 0 */
} md_nodes;

typedef struct {
    double tol;            /* stop when ||r||_2 <= tol (||e_j|| = 1); > 0 */
    int32_t maxit;         /* iteration cap per system, > 0 */
    int32_t precision;     /* md_precision */
    int32_t reliable_every;/* mixed: max iterations between FP64 residual
                              recomputations (0 = 300) */
    double reliable_delta; /* mixed: also recompute when ||r|| fell by this
                              factor since the last one (0 = 3e-3); a refresh
                              that finds the residual larger than at the
                              previous one restarts the Krylov recurrence */
    double timeout_s;      /* device wall-clock budget for the call, 0 = none */
    int32_t block;         /* threads per CTA; 0 = library choice (autotuned) */
    int32_t ctas_per_sm;   /* resident CTAs per SM; 0 = library choice.  With
                              kernel 3: CTAs per cluster (1..8; 0 = the fewest
                              whose slabs fit in shared memory) */
    int32_t kernel;        /* with block > 0: 0 or 1 = generic kernel, 2 = shared-memory
                              z-march kernel (mixed precision, 4th/8th order, no
                              whole-axis rings; ceil(m0*m1/block) <= 4).
                              3 = cluster kernel (block may be 0): mixed precision,
                              fd_order <= 8, no whole-axis rings, method 0; each
                              (node, pole) system runs on one thread-block cluster
                              whose CTAs hold z-slabs of the Krylov vectors p and r
                              in shared memory (halo planes read from the
                              neighbouring CTAs), so the vectors do not stream
                              through HBM.  With kernel 0 and block 0 the
                              autotuner includes it among its candidates. */
    int32_t method;        /* 0 = one COCG per (node, pole) system.
                              1 = shifted COCG: per node one Krylov sequence, seeded
                              with the pole nearest the real axis, serves all P poles
                              (residuals r/pi_k; Jegerlehner 1996, Takayama et al.
                              2006); only x_k(j) is tracked, so it gives rho and e but
                              no checkpoint (md_density_adjoint needs method 0);
                              P <= 64.  Matvecs per node drop from sum_k iters_k to
                              max_k iters_k. */
} md_solver_opts;

/* Per-call statistics, filled (after a stream synchronisation) when the
 * pointer passed to a compute call is non-NULL. */
typedef struct {
    int64_t n_systems;
    int64_t n_converged;
    int64_t n_noconv;
    int64_t n_breakdown;
    int64_t n_timeout;
    int32_t iters_min;
    int32_t iters_max;
    double iters_mean;
    int64_t total_iters;       /* sum over systems */
    int64_t total_point_iters; /* sum over systems of iters * region points */
    int64_t reliable_updates;  /* mixed: FP64 residual recomputations */
    double max_resid;          /* max final relative residual */
    double kernel_ms;          /* device time of the solver launch */
} md_stats;

/* ---- Hamiltonian (Eq. Hamiltonian, discretised as in Section 2.1) ----- */

/* Builds V on the grid on the device (sum of wells + v_ext), the per-atom
 * projector normalisations and the per-point projector lists.  *out is
 * owned by the library; free it with md_hamiltonian_destroy.  Synchronous
 * with respect to the host for its own allocations; the kernels run on
 * `stream`.  Errors: MD_ERR_INVALID (bad sizes, non-positive spacing or
 * sigma, odd fd_order, nonlocal with a periodic box <= 2 proj_rc),
 * MD_ERR_OOM, MD_ERR_CUDA. */
md_status md_build_hamiltonian(const md_grid* grid, const md_atoms* atoms,
                               const md_pot_params* pot, void* stream,
                               md_hamiltonian** out);
md_status md_hamiltonian_destroy(md_hamiltonian* ham);

/* Copies V (N doubles) to device memory V_out, stream-ordered. */
md_status md_hamiltonian_potential(const md_hamiltonian* ham, double* V_out, void* stream);

/* Replaces V by the device array V_in (N doubles), stream-ordered (and
 * ordered after the last asynchronous md_density on the handle); used to
 * differentiate with respect to the local potential directly. */
md_status md_hamiltonian_set_potential(md_hamiltonian* ham, const double* V_in, void* stream);

/* Gershgorin interval [emin, emax] containing the spectrum of H and hence
 * of every H_R (Cauchy interlacing).  Synchronises `stream`. */
md_status md_spectral_bounds(const md_hamiltonian* ham, void* stream,
                             double* emin, double* emax);

/* ---- Poles (host) -------------------------------------------------------
 * P-pole approximation of g(eps) = 1/(1+exp((eps-mu)/kT)) (Eq. dm) on
 * [emin, emax]: contour quadrature of Hale, Higham & Trefethen (2008) with
 * the square-root substitution of Lin, Lu, Ying & E (2009); P must be even.
 * z_out, w_out: host, 2P doubles each (interleaved complex).  Pure host
 * code: needs no GPU. */
md_status md_make_poles(double kT, double mu, double emin, double emax, int32_t P,
                        double* z_out, double* w_out);

/* ---- Density, band energy, adjoint -------------------------------------- */

/* Checkpoint of all forward solutions x_jp (complex128, one region-sized
 * vector per system) for md_density_adjoint.  Allocates
 * 16 * P * sum_j |R(j)| bytes of device memory. */
md_status md_workspace_create(const md_hamiltonian* ham, const md_nodes* nodes,
                              int32_t n_poles, md_workspace** out);
md_status md_workspace_destroy(md_workspace* ws);

/* Nodal density (Eq. Electron_density:GQ with g -> r):
 *   rho_out: device, n_nodes doubles, rho_j = (2/dV) sum_p Im(w_p x_jp(j)).
 *   e_out:   device, n_nodes doubles or NULL, e_j = 2 sum_p Im(w_p(1+z_p x_jp(j))).
 *   ckpt:    NULL, or a workspace made for the same nodes and pole count;
 *            receives every x_jp.
 *   stats:   NULL, or host; receives the solver statistics.
 * With stats != NULL the call synchronises `stream` and returns MD_OK, or
 * MD_ERR_NOCONV / MD_ERR_BREAKDOWN / MD_ERR_TIMEOUT with the outputs still
 * written.  With stats == NULL it is asynchronous: it enqueues the uploads
 * (from a pinned staging buffer of the handle, two used in turn), the solver
 * and the accumulation on `stream`, frees its temporaries stream-ordered
 * (cudaFreeAsync) and returns MD_OK once they are enqueued; the outputs are
 * valid after `stream` has been synchronised and per-system failures are not
 * reported.  The host still waits (a) for the uploads of the call before the
 * previous one, before it reuses their staging buffer, (b) for the stream,
 * the first time a node set of its shape is tuned (opts.block == 0), and
 * (c) for earlier asynchronous calls on the handle, when the handle's
 * scratch has to grow. */
md_status md_density(const md_hamiltonian* ham, const md_poles* poles,
                     const md_nodes* nodes, const md_solver_opts* opts,
                     double* rho_out, double* e_out, md_workspace* ckpt,
                     md_stats* stats, void* stream);

/* Band energy (first term of Eq. tot): e_out per node (device, may be
 * NULL) and the node-weighted sum *e_band = sum_j nu_j e_j (host), with
 * node_weight (device, n_nodes doubles, or NULL for nu = 1) the weights of
 * the cluster-sampled energy (Section 3, Eq. free_cg; see
 * md_cluster_sampling).  Same solves as md_density; synchronises `stream`;
 * the sum is formed on the device in a fixed order. */
md_status md_energy(const md_hamiltonian* ham, const md_poles* poles,
                    const md_nodes* nodes, const double* node_weight,
                    const md_solver_opts* opts, double* e_out, double* e_band,
                    md_stats* stats, void* stream);

/* ---- Free-energy terms (Section 3; Eq. tot) ------------------------------
 * The entropy term of Eq. (tot) needs no further solves: the contour
 * quadrature behind md_make_poles uses no more of the Fermi-Dirac function
 * than its analyticity off the imaginary rays through the Matsubara points,
 * and the entropy function phi_S(x) = -[g ln g + (1-g) ln(1-g)] has its
 * singularities at the same points.  md_make_entropy_weights returns the
 * weights w^S on the poles md_make_poles returns for the same arguments,
 * with sum_p Im(w^S_p / (eps - z_p)) ~= phi_S(eps - mu) on [emin, emax]
 * (the error falls at the Fermi expansion's rate in P).  Per node,
 *     s_j = 2 kT sum_p Im(w^S_p x_jp(j))  ~= 2 kT [phi_S(H_R)]_jj >= 0,
 * the last term of Eq. (tot) at node j (its printed sign makes it +TS; the
 * free energy below takes Mermin's E - TS).  w_out: host, 2P doubles.  Pure
 * host code: needs no GPU. */
md_status md_make_entropy_weights(double kT, double mu, double emin, double emax, int32_t P,
                                  double* w_out);

typedef struct {
    double n_electrons;   /* dV sum_j nu_j rho_j                    (Eq. Fermi:Rho) */
    double e_band;        /* sum_j nu_j e_j                    (first term, Eq. tot) */
    double ts;            /* sum_j nu_j s_j       (entropy term, Eq. tot; 0 without w^S) */
    double free_energy;   /* e_band - ts */
} md_free_energy_terms;

/* Density, band energy and entropy per node from one set of per-pole solves,
 * and their node-weighted totals: the cluster-sampled energy of Section 3,
 * E ~= sum_q n_q (1/N_q) sum_{p in C_q} F_p (Eqs. free_cg, free_cg_sampling),
 * is sum_j nu_j F_j over the nodes and weights md_cluster_sampling returns.
 *   w_entropy: host, 2P doubles from md_make_entropy_weights (same poles), or
 *              NULL (no entropy term: ts = 0, s_out must be NULL).
 *   kT:        temperature of the weights (> 0 when w_entropy is given).
 *   node_weight: device, n_nodes doubles, or NULL (nu = 1).
 *   rho_out, e_out, s_out: device, n_nodes doubles each, or NULL.
 *   terms:     host, the totals (formed on the device in a fixed order).
 * Synchronises `stream`.  Status as md_density. */
md_status md_free_energy(const md_hamiltonian* ham, const md_poles* poles,
                         const double* w_entropy, double kT, const md_nodes* nodes,
                         const double* node_weight, const md_solver_opts* opts,
                         double* rho_out, double* e_out, double* s_out,
                         md_free_energy_terms* terms, md_stats* stats, void* stream);

/* Nodes and weights of the cluster-sampled energy (Section 3, Eqs. free_cg
 * and free_cg_sampling): C_q = the grid points within `radius` (bohr) of
 * electronic sampling point q (grid index esp[q]), by minimum image on
 * periodic axes and inside the grid on open ones; N_q = |C_q|; every p in
 * C_q carries n_q / N_q, the weights of a point in several clusters summed.
 * Points are returned ascending, each once.  Two calls: with node_out and
 * weight_out NULL, *n_out receives the count; then with arrays of *n_out
 * entries (host).  Errors: MD_ERR_INVALID (bad grid, index, radius or
 * n_q, capacity below the count; *n_out then holds the count).  Pure host
 * code: needs no GPU. */
md_status md_cluster_sampling(const md_grid* grid, int64_t n_esp, const int64_t* esp,
                              const double* n_q, double radius, int64_t* n_out,
                              int64_t* node_out, double* weight_out);

/* Fermi level of the pole form (Eq. Fermi:Rho with g -> r, the step before
 * the density in Algorithm 1): the mu at which
 *     N(mu) = dV sum_j nu_j rho_j(mu) = n_electrons,
 * each N(mu) from per-pole solves with the P poles rebuilt at mu on the
 * Hamiltonian's spectral interval (one prepared batch relaunched), by the
 * Illinois variant of regula falsi on [emin, emax] until the bracket is
 * narrower than mu_tol (0 = 1e-10 Ha) or 200 counts.  node_weight: device,
 * n_nodes, or NULL (nu = 1: every grid point a node).  opts as md_density
 * (method 1, shifted COCG, makes each count cheaper).  *mu_out, *count_out
 * (N at *mu_out; may be NULL), *evals_out (counts made; may be NULL): host.
 * Errors: MD_ERR_INVALID when n_electrons lies outside [N(emin), N(emax)];
 * solver statuses as md_density.  Synchronises `stream`. */
md_status md_fermi_level_poles(const md_hamiltonian* ham, double kT, int32_t P,
                               const md_nodes* nodes, const double* node_weight,
                               const md_solver_opts* opts, double n_electrons, double mu_tol,
                               double* mu_out, double* count_out, int32_t* evals_out,
                               void* stream);

/* Density, band energy and the adjoint in one pass, without a checkpoint,
 * for losses whose node sensitivities a_j = dL/drho_j and b_j = dL/de_j are
 * known before the solve (for example the band energy, L = E_band: a = 0,
 * b = 1; the Hellmann-Feynman forces of Section 2.1 follow).  Each system,
 * once converged, adds its share
 *     -Im((2 a_j/dV + 2 b_j z_p) w_p x_jp(k)^2)
 * to dL_dV_out (device, N doubles, zeroed first) while its solution is still
 * in the solver's scratch, so memory stays one region per resident CTA
 * instead of the 16 P sum_j |R(j)| bytes of md_workspace_create.
 *   dL_drho, dL_de: device, n_nodes each, or NULL (= 0).
 *   rho_out (device, n_nodes), e_out (device or NULL), forces_out (device,
 *   3 n_atoms, or NULL; needs atoms and no nonlocal term).
 * Per-pole COCG only (method 0).  Synchronises `stream`.  Status as for
 * md_density; dL_dV accumulates with FP64 atomics. */
md_status md_density_fused_adjoint(const md_hamiltonian* ham, const md_poles* poles,
                                   const md_nodes* nodes, const md_solver_opts* opts,
                                   const double* dL_drho, const double* dL_de, double* rho_out,
                                   double* e_out, double* dL_dV_out, double* forces_out,
                                   md_stats* stats, void* stream);

/* Rows of the density matrix within each region (Eq. dm in the orthonormal
 * grid basis, g replaced by r): for node j and every region point k,
 *     gamma_jk = sum_p Im(w_p x_jp(k)),   so that rho_j = (2/dV) gamma_jj,
 * from the same per-pole COCG solves as md_density.  rows_out: device,
 * sum_j |R(j)| doubles; row j starts at sum_{i<j} |R(i)| and is laid out
 * region-local (x fastest, as the region of md_density).  Every converged
 * system adds its pole's share with FP64 atomics (last-bit
 * nondeterministic).  rho_out (device, n_nodes; required when n_nodes > 0)
 * and e_out (device or NULL) as in md_energy.  opts may be NULL (mixed,
 * tol 1e-10); method 1 is refused.  Synchronises `stream`.  Status as in
 * md_density. */
md_status md_density_matrix_rows(const md_hamiltonian* ham, const md_poles* poles,
                                 const md_nodes* nodes, const md_solver_opts* opts,
                                 double* rho_out, double* e_out, double* rows_out,
                                 md_stats* stats, void* stream);

/* ---- Plans: a prepared batched solve replayed as a CUDA graph ----------
 * md_plan_create validates the inputs once, uploads the cost-sorted
 * (node, pole) work list and region descriptors, allocates the plan's own
 * Krylov scratch and per-system outputs, picks the launch shape (threads
 * per CTA and CTAs per SM; timed by the library's autotuner on a sample of
 * the systems when opts->block == 0, cached per precision, stencil width,
 * region size and nonlocal term) and captures [reset the work counter,
 * the persistent solver kernel, the pole accumulation into rho_out/e_out]
 * as one CUDA graph.  The pointers given here (rho_out, e_out, ckpt, the
 * Hamiltonian's arrays) are baked into the graph: they must stay valid
 * until md_plan_destroy; md_hamiltonian_set_potential between launches is
 * seen by the next launch.  Creation synchronises `stream` (autotuning);
 * md_plan_launch is asynchronous (one cudaGraphLaunch); md_plan_stats
 * synchronises `stream` and returns the status of the last launch
 * (MD_ERR_NOCONV / MD_ERR_BREAKDOWN / MD_ERR_TIMEOUT as for md_density).
 * A plan may not be launched concurrently with itself. */
typedef struct md_plan md_plan;
md_status md_plan_create(const md_hamiltonian* ham, const md_poles* poles,
                         const md_nodes* nodes, const md_solver_opts* opts,
                         double* rho_out, double* e_out, md_workspace* ckpt,
                         void* stream, md_plan** out);
md_status md_plan_launch(md_plan* plan, void* stream);
md_status md_plan_stats(md_plan* plan, void* stream, md_stats* stats);
/* Launch shape chosen for the plan (threads per CTA, CTAs in the grid). */
md_status md_plan_launch_shape(const md_plan* plan, int32_t* block, int32_t* grid);
/* Per-system outcome of the last launch, indexed node * P + pole: status
 * (0 converged, 1 too many projector atoms, 2 maxit, 3 breakdown,
 * 4 deadline), iterations and final residual norm.  Host arrays of
 * n_nodes * P entries; synchronises `stream`. */
md_status md_plan_system_info(md_plan* plan, void* stream, int32_t* status, int32_t* iters,
                              double* resid);
md_status md_plan_destroy(md_plan* plan);

/* Adjoint of (rho, e) -> L.  With a_j = dL/drho_j and b_j = dL/de_j:
 *   dL/dV_k = -sum_j sum_p Im((2 a_j/dV + 2 b_j z_p) w_p x_jp(k)^2)
 * (G = (H_R - z)^-1 is complex symmetric, so dG_jj/dV_k = -x_jp(k)^2 and
 * the adjoint systems are the forward ones), and, when forces_out is
 * non-NULL, the Hellmann-Feynman forces through the local wells
 * (Section 2.1, last paragraph):
 *   F_a = -sum_k dL/dV_k dV_k/dR_a.
 *   dL_drho: device, n_nodes.  dL_de: device, n_nodes, or NULL (= 0).
 *   ckpt: workspace filled by md_density with the same inputs, or NULL to
 *         re-solve the systems here.
 *   dL_dV_out: device, N doubles (overwritten).
 *   forces_out: device, 3*n_atoms doubles (overwritten) or NULL; needs a
 *         Hamiltonian built from atoms without the nonlocal term.
 * Regions of different nodes overlap, so dL_dV is accumulated with FP64
 * atomics and its last bits depend on scheduling. */
md_status md_density_adjoint(const md_hamiltonian* ham, const md_poles* poles,
                             const md_nodes* nodes, const md_solver_opts* opts,
                             const double* dL_drho, const double* dL_de,
                             md_workspace* ckpt, double* dL_dV_out,
                             double* forces_out, md_stats* stats, void* stream);

/* ---- Density without device allocation ---------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they solve -- a process whose GPU
 * memory is owned by another allocator with a fixed budget (a framework's
 * caching allocator, a serving engine that reserves its memory at start-up)
 * or code running where an allocation would synchronise or be refused.  It
 * computes what md_density computes (rho_out and, if non-NULL, e_out:
 * device, n_nodes doubles; stats as in md_density) but keeps every
 * temporary (Krylov vectors, work list, descriptors, per-system results)
 * in one static device array of MD_NOALLOC_SCRATCH_BYTES of Krylov space
 * plus room for MD_NOALLOC_MAX_SYSTEMS systems, which every GPU that loads
 * the library holds until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine, and nothing on the host heap on
 * success (error messages excepted).  The Hamiltonian must be built
 * beforehand (md_build_hamiltonian allocates).  It always solves one COCG
 * per (node, pole) system on the generic kernel (opts->method, ->kernel and
 * ->block are ignored).
 *   - Limits: n_nodes <= MD_NOALLOC_MAX_NODES, P <= MD_NOALLOC_MAX_POLES,
 *     n_nodes * P <= MD_NOALLOC_MAX_SYSTEMS, and one region's Krylov slot
 *     (56 B per point mixed, 64 B per point FP64) within
 *     MD_NOALLOC_SCRATCH_BYTES; beyond them it returns MD_ERR_INVALID with
 *     nothing launched.  Concurrency is one CTA per SM, capped by the number
 *     of slots that fit, so large regions run on fewer SMs.
 *   - Every call looks up the array's device address in the current
 *     device's context (cudaGetSymbolAddress), so a reset context leaves no
 *     stale address behind.
 *   - The call cannot be captured into a CUDA graph: it copies from pageable
 *     host memory, waits for its stream, and relies on a host lock that a
 *     replayed graph would bypass.  On a capturing stream it returns
 *     MD_ERR_INVALID with nothing enqueued.
 *   - Every call shares the array, which keeps the last call's contents;
 *     the call zeroes what must start at zero.  Calls that overlap on the
 *     GPU race on the array and corrupt each other's results.  Calls made
 *     through this entry point in one process take a host lock and each
 *     synchronises its stream before returning, error returns included, so
 *     they do not overlap. */
#define MD_NOALLOC_SCRATCH_BYTES (64u << 20)
#define MD_NOALLOC_MAX_SYSTEMS 16384
#define MD_NOALLOC_MAX_NODES 4096
#define MD_NOALLOC_MAX_POLES 64
md_status md_density_noalloc(const md_hamiltonian* ham, const md_poles* poles,
                             const md_nodes* nodes, const md_solver_opts* opts,
                             double* rho_out, double* e_out, md_stats* stats, void* stream);

/* ---- Lanczos spectral Gauss quadrature (LSSGQ) -------------------------
 * The paper's own route to the nodal fields (Section 2.1, Eq. 9): for node j
 * the spectral measure of H_R(j) contracted with e_j is replaced by a
 * K-point Gauss rule from K steps of the symmetric Lanczos process started
 * at e_j (FP64, no reorthogonalisation); the rule's nodes lambda_jk are the
 * eigenvalues of the Lanczos tridiagonal matrix and its weights w_jk the
 * squared first components of its unit eigenvectors.  The rules do not
 * depend on the Fermi level, so the fields at any (mu, kT) and the Fermi
 * level itself (Eq. Fermi:Rho) follow without another pass over H. */
#define MD_LSSGQ_MAX_K 128
typedef struct {
    int32_t K;             /* rule size = Lanczos steps, 1..MD_LSSGQ_MAX_K (paper: 40) */
    double breakdown_tol;  /* stop early when beta_k <= tol (|alpha_1| + beta_1 + 1),
                              the Krylov space being invariant (0 = 1e-13) */
    double timeout_s;      /* device wall-clock budget, 0 = none */
    int32_t block;         /* threads per CTA, 0 = 1024; multiple of 32 in 64..1024 */
    int32_t precision;     /* MD_PREC_FP64: FP64 Lanczos vectors and arithmetic;
                              MD_PREC_MIXED: FP32 vectors, stencil and projector
                              terms with compensated FP32 partial sums, FP64
                              reductions, alpha, beta and vector scales */
} md_lssgq_opts;

/* Gauss rules of every node: lambda_out, weight_out (device, n_nodes x K
 * doubles, row j = node j, nodes ascending; entries past k_used_j repeat
 * the largest node with weight 0); k_used_out (device, n_nodes int32, or
 * NULL) = Lanczos steps taken (< K after a breakdown).  Regions as in
 * md_density.  Synchronises `stream`.  Errors: MD_ERR_INVALID (bad options,
 * nodes or regions, a region meeting more than 256 projector atoms),
 * MD_ERR_TIMEOUT, MD_ERR_BREAKDOWN (the tridiagonal eigensolver did not
 * converge for a node), MD_ERR_OOM, MD_ERR_CUDA. */
md_status md_lssgq_rules(const md_hamiltonian* ham, const md_nodes* nodes,
                         const md_lssgq_opts* opts, double* lambda_out,
                         double* weight_out, int32_t* k_used_out, void* stream);

/* Fields from the rules at Fermi level mu and temperature kT (Eqs.
 * Electron_density:GQ and tot, per node):
 *   rho_j = (2/dV) sum_k w_jk g(lambda_jk)
 *   e_j   = 2 sum_k w_jk lambda_jk g(lambda_jk)                (band term)
 *   s_j   = -2 kT sum_k w_jk [g ln g + (1-g) ln(1-g)]         (entropy term)
 * with g the Fermi-Dirac function of Eq. (dm).  lambda, weight: device,
 * n_nodes x K; rho_out (device, n_nodes), e_out and s_out (device or NULL).
 * Stream-ordered, no synchronisation. */
md_status md_lssgq_fields(int64_t n_nodes, int32_t K, const double* lambda,
                          const double* weight, double mu, double kT, double dV,
                          double* rho_out, double* e_out, double* s_out, void* stream);

/* Fermi level (Eq. Fermi:Rho): the mu at which
 *   N_e(mu) = 2 sum_j nu_j sum_k w_jk g(lambda_jk; mu)
 * equals n_electrons, by bisection on the device between the smallest node
 * - 40 kT and the largest + 40 kT, run until the bracket stops shrinking.
 * node_weight: device, n_nodes (nu_j = grid points node j stands for), or
 * NULL for 1 (every grid point a node).  *mu_out and *count_out (N_e at
 * *mu_out; may be NULL) are host doubles.  Synchronises `stream`. */
md_status md_fermi_level(int64_t n_nodes, int32_t K, const double* lambda,
                         const double* weight, const double* node_weight, double kT,
                         double n_electrons, double* mu_out, double* count_out,
                         void* stream);

/* Central weights w_0..w_q (q = order/2) of d^2/dx^2 on a unit grid with
 * accuracy order `order` (even, 2..16), by Fornberg's recursion (Math.
 * Comp. 51 (1988)); the library's Laplacian is -1/2 sum_d w / h_d^2 (the
 * paper's Section 2.1 uses order 6).  w_out: host, q+1 doubles.  Pure host
 * code: needs no GPU. */
md_status md_fd_weights(int32_t order, double* w_out);

/* Measured fused multiply-add rate of this GPU (the paper has no
 * counterpart: it is the peak the FP64 solver form's roofline is reported
 * against).  precision MD_PREC_FP64 times FP64 FMAs, MD_PREC_MIXED FP32
 * FMAs: 8 independent chains per thread on every SM, a fixed chain length
 * (a bounded run of some milliseconds), timed with CUDA events on
 * `stream`.  *tflops_out (host) = 2 x FMAs / s / 1e12.  Allocates a few
 * bytes of device memory; synchronises `stream`. */
md_status md_fma_rate(int32_t precision, void* stream, double* tflops_out);

/* Description of the last error on the calling host thread ("" if none). */
const char* md_last_error(void);

/* Library version string. */
const char* md_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MACRODFT_H */
