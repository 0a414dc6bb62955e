/*
 * Oracle: plain FP64 COCG on one truncated region per system.
 *
 * TEST INFRASTRUCTURE ONLY: built and called by the oracle package for the
 * tests and the CPU baseline; the product library never links it.
 *
 * Each system solves (H_R - z I) x = e_src, with H_R the Hamiltonian of the
 * region (the cube around a node; locality of Section 2.1 of the paper):
 *   (H_R v)(i) = diag v(i) + V(i) v(i)
 *              + sum_axes sum_{o=1..q} coef[d][o-1] (v(i + o e_d) + v(i - o e_d))
 *              + sum_pi E_pi dV p_pi(i) sum_k p_pi(k) v(k)
 * where neighbours outside a window axis are absent (Dirichlet restriction)
 * and neighbours on a ring axis wrap around.
 *
 * COCG (conjugate orthogonal conjugate gradient; van der Vorst & Melissen,
 * IEEE Trans. Magn. 26, 1990) is CG with the bilinear form u^T v (no complex
 * conjugate), valid because H_R - z I is complex symmetric:
 *   x = 0, r = p = b, rho = r^T r
 *   repeat: q = A p; alpha = rho / p^T q; x += alpha p; r -= alpha q;
 *           stop when ||r||_2 <= tol ||b||_2 (Hermitian norm);
 *           rho' = r^T r; beta = rho'/rho; p = r + beta p
 * Everything is scalar loops over doubles; systems run in parallel with
 * OpenMP, each with its own buffers.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int dims[3];
    int ring[3];
    const double* V;        /* region potential, x fastest */
    int n_proj;
    const long long* pptr;  /* n_proj + 1 offsets into pidx/pval */
    const int* pidx;        /* local indices */
    const double* pval;
    const double* pE;
} region_t;

static void apply_shifted(const region_t* R, int q, const double* coef, double diag,
                          double dV, cplx z, const cplx* v, cplx* out, cplx* work_c)
{
    const int mx = R->dims[0], my = R->dims[1], mz = R->dims[2];
    const int m[3] = {mx, my, mz};
    for (int c = 0; c < mz; ++c)
        for (int b = 0; b < my; ++b)
            for (int a = 0; a < mx; ++a) {
                const long long i = a + (long long)mx * (b + (long long)my * c);
                cplx acc = (diag + R->V[i] - z) * v[i];
                const int pos[3] = {a, b, c};
                for (int d = 0; d < 3; ++d) {
                    for (int o = 1; o <= q; ++o) {
                        for (int sgn = -1; sgn <= 1; sgn += 2) {
                            int t = pos[d] + sgn * o;
                            if (R->ring[d]) {
                                t %= m[d];
                                if (t < 0) t += m[d];
                            } else if (t < 0 || t >= m[d]) {
                                continue;
                            }
                            int nb[3] = {a, b, c};
                            nb[d] = t;
                            const long long k = nb[0] + (long long)mx * (nb[1] + (long long)my * nb[2]);
                            acc += coef[d * q + (o - 1)] * v[k];
                        }
                    }
                }
                out[i] = acc;
            }
    /* separable nonlocal part: c_pi = p_pi^T v, then out += E dV c_pi p_pi */
    for (int p = 0; p < R->n_proj; ++p) {
        cplx cp = 0.0;
        for (long long e = R->pptr[p]; e < R->pptr[p + 1]; ++e)
            cp += R->pval[e] * v[R->pidx[e]];
        work_c[p] = cp;
    }
    for (int p = 0; p < R->n_proj; ++p) {
        const cplx f = R->pE[p] * dV * work_c[p];
        for (long long e = R->pptr[p]; e < R->pptr[p + 1]; ++e)
            out[R->pidx[e]] += f * R->pval[e];
    }
}

static cplx dotu(const cplx* a, const cplx* b, long long n)
{
    cplx s = 0.0;
    for (long long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double norm2(const cplx* a, long long n)
{
    double s = 0.0;
    for (long long i = 0; i < n; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return sqrt(s);
}

/* status: 0 converged, 2 not converged within maxit, 3 breakdown */
static int cocg_one(const region_t* R, int q, const double* coef, double diag, double dV,
                    cplx z, int src, double tol, int maxit, cplx* x,
                    int* iters, double* resid)
{
    const long long n = (long long)R->dims[0] * R->dims[1] * R->dims[2];
    cplx* r = (cplx*)calloc((size_t)n, sizeof(cplx));
    cplx* p = (cplx*)calloc((size_t)n, sizeof(cplx));
    cplx* Ap = (cplx*)calloc((size_t)n, sizeof(cplx));
    cplx* wc = (cplx*)calloc((size_t)(R->n_proj > 0 ? R->n_proj : 1), sizeof(cplx));
    int status = 2;
    memset(x, 0, (size_t)n * sizeof(cplx));
    r[src] = 1.0;
    p[src] = 1.0;
    cplx rho = dotu(r, r, n);
    const double bnorm = 1.0;
    double rn = 1.0;
    int it = 0;
    while (it < maxit) {
        apply_shifted(R, q, coef, diag, dV, z, p, Ap, wc);
        const cplx pAp = dotu(p, Ap, n);
        ++it;
        if (cabs(pAp) == 0.0) { status = 3; break; }
        const cplx alpha = rho / pAp;
        for (long long i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
        }
        rn = norm2(r, n);
        if (rn <= tol * bnorm) { status = 0; break; }
        const cplx rho_new = dotu(r, r, n);
        if (cabs(rho_new) <= 1e-300 || cabs(rho_new) < 1e-14 * rn * rn) { status = 3; break; }
        const cplx beta = rho_new / rho;
        rho = rho_new;
        for (long long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    }
    *iters = it;
    *resid = rn;
    free(r); free(p); free(Ap); free(wc);
    return status;
}

/*
 * Batched entry point.  Regions are packed:
 *   reg_dims[3r..3r+2], reg_ring[3r..], reg_src[r], V packed at reg_voff[r],
 *   projectors of region r are entries reg_pptr[r] .. reg_pptr[r+1]-1 of the
 *   projector table (proj_ptr / proj_idx / proj_val / proj_E).
 * System s uses region sys_reg[s] and shift (sys_z[2s], sys_z[2s+1]).
 * Outputs: x_src (2 per system); optionally the full solution at
 * x_full + 2*sys_xoff[s] (pass NULL to skip).
 */
int oracle_cocg_batch(int n_sys, const int* sys_reg, const double* sys_z,
                      const int* reg_dims, const int* reg_ring, const int* reg_src,
                      const long long* reg_voff, const double* V,
                      const long long* reg_pptr, const long long* proj_ptr,
                      const int* proj_idx, const double* proj_val, const double* proj_E,
                      int q, const double* coef, double diag, double dV,
                      double tol, int maxit,
                      double* x_src, double* x_full, const long long* sys_xoff,
                      int* iters, double* resid, int* status)
{
    int n_bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_bad)
    for (int s = 0; s < n_sys; ++s) {
        const int rg = sys_reg[s];
        region_t R;
        for (int d = 0; d < 3; ++d) {
            R.dims[d] = reg_dims[3 * rg + d];
            R.ring[d] = reg_ring[3 * rg + d];
        }
        R.V = V + reg_voff[rg];
        R.n_proj = (int)(reg_pptr[rg + 1] - reg_pptr[rg]);
        R.pptr = proj_ptr + reg_pptr[rg];
        R.pidx = proj_idx;
        R.pval = proj_val;
        R.pE = proj_E + reg_pptr[rg];
        const long long n = (long long)R.dims[0] * R.dims[1] * R.dims[2];
        cplx* x = (cplx*)malloc((size_t)n * sizeof(cplx));
        const cplx z = sys_z[2 * s] + I * sys_z[2 * s + 1];
        status[s] = cocg_one(&R, q, coef, diag, dV, z, reg_src[rg], tol, maxit, x,
                             &iters[s], &resid[s]);
        if (status[s] != 0) n_bad += 1;
        x_src[2 * s] = creal(x[reg_src[rg]]);
        x_src[2 * s + 1] = cimag(x[reg_src[rg]]);
        if (x_full) {
            double* dst = x_full + 2 * sys_xoff[s];
            for (long long i = 0; i < n; ++i) {
                dst[2 * i] = creal(x[i]);
                dst[2 * i + 1] = cimag(x[i]);
            }
        }
        free(x);
    }
    return n_bad;
}
