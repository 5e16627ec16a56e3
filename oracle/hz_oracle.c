/*
 * hz_oracle.c -- CPU oracle for the complex Helmholtz Krylov path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * path never does.  It shares no code, header, table or helper with the CUDA
 * sources.
 *
 * Arithmetic is IEEE binary64 (binary32 for the inner solve of the mixed
 * precision refinement), summed in the order the definitions are written.
 * Build with -ffp-contract=off so no multiply-add is fused behind our back.
 *
 * Complex numbers are two contiguous doubles (real, imaginary), the layout
 * of the paper's Section 4 (listing "Complex number in memory").  Matrices
 * are CSR as in Section 3.2 (AA values, JA column indices, IA row pointers),
 * 0-based.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Built plainly (the tests, the smoke check and the single-thread baseline)
 * every loop below runs sequentially and OR_PAR_FOR is empty.  Built with
 * -fopenmp (only for the benchmark's all-cores CPU baseline), the SpMV rows
 * and the BiCGStab vector updates are spread over threads, and the reductions
 * (or_zdotc, or_dznrm2) sum fixed chunks of OR_CHUNK elements with the same
 * compensated sum and then add the chunk totals in chunk order, so that the
 * result does not depend on the number of threads. */
#ifdef _OPENMP
#include <omp.h>
#define OR_PAR_FOR _Pragma("omp parallel for schedule(static)")
#define OR_CHUNK 8192
void or_set_threads(int32_t k) { omp_set_num_threads(k); }
#else
#define OR_PAR_FOR
#endif

typedef struct { double re, im; } oz;   /* complex double */
typedef struct { float re, im; } oc;    /* complex float  */

enum { OR_OK = 0, OR_NOT_CONVERGED = 4, OR_BREAKDOWN = 5, OR_NAN = 6 };

static oz z_mul(oz a, oz b) { oz r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static oz z_add(oz a, oz b) { oz r = {a.re + b.re, a.im + b.im}; return r; }
static oz z_sub(oz a, oz b) { oz r = {a.re - b.re, a.im - b.im}; return r; }
static oz z_conj(oz a) { oz r = {a.re, -a.im}; return r; }
static oz z_div(oz a, oz b) {
    /* textbook quotient a * conj(b) / |b|^2 */
    double d = b.re * b.re + b.im * b.im;
    oz r = {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
    return r;
}
static int z_isfinite(oz a) { return isfinite(a.re) && isfinite(a.im); }

static oc c_mul(oc a, oc b) { oc r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static oc c_add(oc a, oc b) { oc r = {a.re + b.re, a.im + b.im}; return r; }
static oc c_sub(oc a, oc b) { oc r = {a.re - b.re, a.im - b.im}; return r; }
static oc c_conj(oc a) { oc r = {a.re, -a.im}; return r; }
static oc c_div(oc a, oc b) {
    float d = b.re * b.re + b.im * b.im;
    oc r = {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
    return r;
}

/* ---------------------------------------------------------------------- */
/* Neumaier-compensated summation, used by every reduction so that the    */
/* oracle is more accurate than any blocked GPU reduction it is compared   */
/* against.                                                                */
typedef struct { double s, c; } ksum;
static void ks_add(ksum *k, double v) {
    double t = k->s + v;
    if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
    else k->c += (v - t) + k->s;
    k->s = t;
}
static double ks_val(const ksum *k) { return k->s + k->c; }

/* ---------------------------------------------------------------------- */
/* Section 6: y = A x with A in CSR, y_i = sum_{k=IA(i)}^{IA(i+1)-1} AA(k) x(JA(k)),
 * summed in storage order. */
void or_zspmv(int32_t n, const int32_t *rowptr, const int32_t *col, const oz *val,
              const oz *x, oz *y)
{
    OR_PAR_FOR
    for (int32_t i = 0; i < n; ++i) {
        oz acc = {0.0, 0.0};
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            acc = z_add(acc, z_mul(val[k], x[col[k]]));
        y[i] = acc;
    }
}

/* complex64 SpMV for the inner solve of the mixed-precision refinement */
void or_cspmv(int32_t n, const int32_t *rowptr, const int32_t *col, const oc *val,
              const oc *x, oc *y)
{
    for (int32_t i = 0; i < n; ++i) {
        oc acc = {0.0f, 0.0f};
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            acc = c_add(acc, c_mul(val[k], x[col[k]]));
        y[i] = acc;
    }
}

/* Section 5, dot product: sum_i conj(x_i) y_i (conjugated) */
#ifndef _OPENMP
void or_zdotc(int64_t n, const oz *x, const oz *y, oz *out)
{
    ksum re = {0, 0}, im = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        oz p = z_mul(z_conj(x[i]), y[i]);
        ks_add(&re, p.re);
        ks_add(&im, p.im);
    }
    out->re = ks_val(&re);
    out->im = ks_val(&im);
}
#else
void or_zdotc(int64_t n, const oz *x, const oz *y, oz *out)
{
    int64_t nc = (n + OR_CHUNK - 1) / OR_CHUNK;
    oz *part = malloc((size_t)(nc > 0 ? nc : 1) * sizeof(oz));
    ksum re = {0, 0}, im = {0, 0};
    OR_PAR_FOR
    for (int64_t c = 0; c < nc; ++c) {
        ksum cr = {0, 0}, ci = {0, 0};
        int64_t e = (c + 1) * OR_CHUNK < n ? (c + 1) * OR_CHUNK : n;
        for (int64_t i = c * OR_CHUNK; i < e; ++i) {
            oz p = z_mul(z_conj(x[i]), y[i]);
            ks_add(&cr, p.re);
            ks_add(&ci, p.im);
        }
        part[c].re = ks_val(&cr);
        part[c].im = ks_val(&ci);
    }
    for (int64_t c = 0; c < nc; ++c) { ks_add(&re, part[c].re); ks_add(&im, part[c].im); }
    free(part);
    out->re = ks_val(&re);
    out->im = ks_val(&im);
}
#endif

/* Section 5, dot product without conjugation: sum_i x_i y_i */
void or_zdotu(int64_t n, const oz *x, const oz *y, oz *out)
{
    ksum re = {0, 0}, im = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        oz p = z_mul(x[i], y[i]);
        ks_add(&re, p.re);
        ks_add(&im, p.im);
    }
    out->re = ks_val(&re);
    out->im = ks_val(&im);
}

/* Section 5, L2 norm: sqrt(sum_i |x_i|^2) */
#ifndef _OPENMP
double or_dznrm2(int64_t n, const oz *x)
{
    ksum s = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        ks_add(&s, x[i].re * x[i].re);
        ks_add(&s, x[i].im * x[i].im);
    }
    return sqrt(ks_val(&s));
}
#else
double or_dznrm2(int64_t n, const oz *x)
{
    int64_t nc = (n + OR_CHUNK - 1) / OR_CHUNK;
    double *part = malloc((size_t)(nc > 0 ? nc : 1) * sizeof(double));
    ksum s = {0, 0};
    OR_PAR_FOR
    for (int64_t c = 0; c < nc; ++c) {
        ksum cs = {0, 0};
        int64_t e = (c + 1) * OR_CHUNK < n ? (c + 1) * OR_CHUNK : n;
        for (int64_t i = c * OR_CHUNK; i < e; ++i) {
            ks_add(&cs, x[i].re * x[i].re);
            ks_add(&cs, x[i].im * x[i].im);
        }
        part[c] = ks_val(&cs);
    }
    for (int64_t c = 0; c < nc; ++c) ks_add(&s, part[c]);
    free(part);
    return sqrt(ks_val(&s));
}
#endif

/* Section 5, Zaxpy: y_i = alpha x_i + y_i */
void or_zaxpy(int64_t n, const oz *alpha, const oz *x, oz *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = z_add(z_mul(*alpha, x[i]), y[i]);
}

/* Section 5, scale: x_i = alpha x_i */
void or_zscal(int64_t n, const oz *alpha, oz *x)
{
    for (int64_t i = 0; i < n; ++i) x[i] = z_mul(*alpha, x[i]);
}

/* Section 5, assign: y_i = x_i */
void or_zcopy(int64_t n, const oz *x, oz *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = x[i];
}

/* ---------------------------------------------------------------------- */
/* Section 7: BiCGStab (van der Vorst's method as given in Saad's "Iterative
 * Methods for Sparse Linear Systems", which the paper cites), without a
 * preconditioner, with the Hermitian inner product <u,w> = sum conj(u_i) w_i.
 *
 *   r = b - A x;  rh = r;  rho_old = alpha = omega = 1;  v = p = 0
 *   loop:  rho = <rh, r>;  beta = (rho/rho_old)(alpha/omega)
 *          p = r + beta (p - omega v);  v = A p;  alpha = rho / <rh, v>
 *          s = r - alpha v;   stop with x += alpha p if ||s|| <= tol ||b||
 *          t = A s;  omega = <t, s> / <t, t>
 *          x += alpha p + omega s;  r = s - omega t;  rho_old = rho
 *          stop if ||r|| <= tol ||b||
 *
 * Stopping test: relative 2-norm residual against ||b||.  Breakdown: rho == 0
 * or omega == 0 or <rh, v> == 0 (exact zeros).  After the loop the true
 * residual ||b - A x|| / ||b|| is formed; if it exceeds tol while the
 * recursive one did not, the iteration restarts once from the current x.
 *
 * hist (optional, length maxit+1): hist[0] = ||r0||/||b||, hist[j] = the
 * recursive residual ratio after iteration j (||s|| for a half-step exit).
 */
typedef struct {
    int32_t iters;
    int32_t status;
    int32_t restarts;
    double relres_rec;
    double relres_true;
} or_info;

static double z_norm(int64_t n, const oz *x) { return or_dznrm2(n, x); }

/* z_i = x_i y_i: the element-wise product of Section 5 */
void or_zmul_elementwise(int64_t n, const oz *x, const oz *y, oz *z)
{
    for (int64_t i = 0; i < n; ++i) z[i] = z_mul(x[i], y[i]);
}

/* Jacobi (diagonal) preconditioner of Section 7's "P-" solvers, stored as
 * its inverse: dinv_i = 1 / a_ii, where a_ii is the sum of the stored
 * entries of row i in column i; a row whose diagonal is absent or zero gets
 * dinv_i = 1 (it is left unscaled). */
void or_jacobi_dinv(int32_t n, const int32_t *rowptr, const int32_t *col, const oz *val, oz *dinv)
{
    for (int32_t i = 0; i < n; ++i) {
        oz d = {0.0, 0.0};
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (col[k] == i) d = z_add(d, val[k]);
        if (d.re == 0.0 && d.im == 0.0) { dinv[i].re = 1.0; dinv[i].im = 0.0; }
        else { oz one = {1.0, 0.0}; dinv[i] = z_div(one, d); }
    }
}

/* BiCGStab right-preconditioned by M^{-1} = diag(dinv) (dinv = NULL: no
 * preconditioner, and then every step below is the unpreconditioned
 * algorithm unchanged).  The textbook right-preconditioned form: the search
 * directions are mapped through M^{-1} before each product with A,
 *   p^ = M^{-1} p,  v = A p^,  s^ = M^{-1} s,  t = A s^,  x += alpha p^ + omega s^,
 * so the residuals r, s are those of the original system A x = b and the
 * stopping test is unchanged. */
int or_bicgstab_pc(int32_t n, const int32_t *rowptr, const int32_t *col, const oz *val,
                   const oz *dinv, const oz *b, oz *x, double tol, int32_t maxit, double *hist,
                   or_info *info)
{
    oz *r = calloc((size_t)n, sizeof(oz)), *rh = calloc((size_t)n, sizeof(oz));
    oz *p = calloc((size_t)n, sizeof(oz)), *v = calloc((size_t)n, sizeof(oz));
    oz *s = calloc((size_t)n, sizeof(oz)), *t = calloc((size_t)n, sizeof(oz));
    oz *ph = dinv ? calloc((size_t)n, sizeof(oz)) : p;   /* M^{-1} p (p itself without M) */
    oz *sh = dinv ? calloc((size_t)n, sizeof(oz)) : s;   /* M^{-1} s */
    double nb = z_norm(n, b);
    int32_t it = 0, status = OR_NOT_CONVERGED, restarts = 0;
    double rel = 0.0;

    if (nb == 0.0) {                     /* b = 0: the solution is x = 0 */
        memset(x, 0, (size_t)n * sizeof(oz));
        info->iters = 0; info->status = OR_OK; info->restarts = 0;
        info->relres_rec = 0.0; info->relres_true = 0.0;
        if (hist) hist[0] = 0.0;
        if (dinv) { free(ph); free(sh); }
        free(r); free(rh); free(p); free(v); free(s); free(t);
        return OR_OK;
    }

    for (;;) {                           /* at most one restart */
        oz rho_old = {1, 0}, alpha = {1, 0}, omega = {1, 0};
        or_zspmv(n, rowptr, col, val, x, r);
        OR_PAR_FOR
        for (int32_t i = 0; i < n; ++i) { r[i] = z_sub(b[i], r[i]); rh[i] = r[i]; }
        memset(p, 0, (size_t)n * sizeof(oz));
        memset(v, 0, (size_t)n * sizeof(oz));
        rel = z_norm(n, r) / nb;
        if (hist && it == 0) hist[0] = rel;
        if (!isfinite(rel)) { status = OR_NAN; break; }
        if (rel <= tol) { status = OR_OK; }
        else {
            status = OR_NOT_CONVERGED;
            while (it < maxit) {
                oz rho, sig, ts, tt, beta;
                ++it;
                or_zdotc(n, rh, r, &rho);
                if (rho.re == 0.0 && rho.im == 0.0) { status = OR_BREAKDOWN; break; }
                beta = z_mul(z_div(rho, rho_old), z_div(alpha, omega));
                OR_PAR_FOR
                for (int32_t i = 0; i < n; ++i)
                    p[i] = z_add(r[i], z_mul(beta, z_sub(p[i], z_mul(omega, v[i]))));
                if (dinv) or_zmul_elementwise(n, dinv, p, ph);
                or_zspmv(n, rowptr, col, val, ph, v);
                or_zdotc(n, rh, v, &sig);
                if (sig.re == 0.0 && sig.im == 0.0) { status = OR_BREAKDOWN; break; }
                alpha = z_div(rho, sig);
                OR_PAR_FOR
                for (int32_t i = 0; i < n; ++i) s[i] = z_sub(r[i], z_mul(alpha, v[i]));
                rel = z_norm(n, s) / nb;
                if (!isfinite(rel)) { status = OR_NAN; break; }
                if (rel <= tol) {        /* half-step exit */
                    for (int32_t i = 0; i < n; ++i) x[i] = z_add(x[i], z_mul(alpha, ph[i]));
                    if (hist) hist[it] = rel;
                    status = OR_OK;
                    break;
                }
                if (dinv) or_zmul_elementwise(n, dinv, s, sh);
                or_zspmv(n, rowptr, col, val, sh, t);
                or_zdotc(n, t, s, &ts);
                or_zdotc(n, t, t, &tt);
                if (tt.re == 0.0 && tt.im == 0.0) { status = OR_BREAKDOWN; break; }
                omega = z_div(ts, tt);
                OR_PAR_FOR
                for (int32_t i = 0; i < n; ++i) {
                    x[i] = z_add(x[i], z_add(z_mul(alpha, ph[i]), z_mul(omega, sh[i])));
                    r[i] = z_sub(s[i], z_mul(omega, t[i]));
                }
                rho_old = rho;
                rel = z_norm(n, r) / nb;
                if (hist) hist[it] = rel;
                if (!isfinite(rel)) { status = OR_NAN; break; }
                if (rel <= tol) { status = OR_OK; break; }
                if (omega.re == 0.0 && omega.im == 0.0) { status = OR_BREAKDOWN; break; }
            }
        }
        /* true residual */
        or_zspmv(n, rowptr, col, val, x, t);
        for (int32_t i = 0; i < n; ++i) t[i] = z_sub(b[i], t[i]);
        info->relres_true = z_norm(n, t) / nb;
        info->relres_rec = rel;
        if (status == OR_OK && info->relres_true > tol && restarts == 0 && it < maxit) {
            ++restarts;
            continue;
        }
        if (status == OR_OK && info->relres_true > tol) status = OR_NOT_CONVERGED;
        break;
    }
    info->iters = it;
    info->status = status;
    info->restarts = restarts;
    if (dinv) { free(ph); free(sh); }
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return status;
}

int or_bicgstab(int32_t n, const int32_t *rowptr, const int32_t *col, const oz *val,
                const oz *b, oz *x, double tol, int32_t maxit, double *hist, or_info *info)
{
    return or_bicgstab_pc(n, rowptr, col, val, NULL, b, x, tol, maxit, hist, info);
}

/* ---------------------------------------------------------------------- */
/* BiCGStab(l) of Sleijpen and Fokkema (Section 7 lists P-BiCGSTAB(l) among
 * the paper's solvers; no preconditioner here, as for BiCGStab).  Each outer
 * iteration takes l BiCG steps that build r_0..r_l and u_0..u_l with
 * r_{i+1} = A r_i and u_{i+1} = A u_i, then a minimal-residual step: r_0 is
 * replaced by the residual of the least-squares fit of r_0 by r_1..r_l,
 * computed by modified Gram-Schmidt on r_1..r_l.  Hermitian inner products
 * throughout.  The loop stops when ||r_0|| <= tol ||b||, tested after every
 * BiCG step and after the minimal-residual step; maxit counts BiCG steps and
 * is checked before each outer iteration.  hist[k] holds ||r_0|| / ||b||
 * after the k-th BiCG step.  Breakdown: rho_0 = 0, <r^, u_{j+1}> = 0, a
 * zero Gram-Schmidt norm, or omega = 0.  As for BiCGStab, the true residual
 * is recomputed at exit and the iteration restarts once if it misses tol. */
int or_bicgstabl(int32_t n, const int32_t *rowptr, const int32_t *col, const oz *val, int32_t ell,
                 const oz *b, oz *x, double tol, int32_t maxit, double *hist, or_info *info)
{
    const size_t nn = (size_t)n;
    oz *R = calloc((size_t)(ell + 1) * nn, sizeof(oz)), *U = calloc((size_t)(ell + 1) * nn, sizeof(oz));
    oz *rh = calloc(nn, sizeof(oz)), *tmp = calloc(nn, sizeof(oz));
    oz tau[9][9], gp[9], g[9], gpp[9];
    double sigma[9];
    double nb = z_norm(n, b), rel = 0.0;
    int32_t it = 0, status = OR_NOT_CONVERGED, restarts = 0;
#define RV(i) (R + (size_t)(i) * nn)
#define UV(i) (U + (size_t)(i) * nn)
    if (ell < 1 || ell > 8) {
        free(R); free(U); free(rh); free(tmp);
        return -1;
    }
    if (nb == 0.0) {
        memset(x, 0, nn * sizeof(oz));
        info->iters = 0; info->status = OR_OK; info->restarts = 0;
        info->relres_rec = 0.0; info->relres_true = 0.0;
        if (hist) hist[0] = 0.0;
        free(R); free(U); free(rh); free(tmp);
        return OR_OK;
    }
    for (;;) {
        oz rho0 = {1, 0}, alpha = {0, 0}, omega = {1, 0};
        or_zspmv(n, rowptr, col, val, x, RV(0));
        for (int32_t i = 0; i < n; ++i) { RV(0)[i] = z_sub(b[i], RV(0)[i]); rh[i] = RV(0)[i]; }
        memset(UV(0), 0, nn * sizeof(oz));
        rel = z_norm(n, RV(0)) / nb;
        if (hist && it == 0) hist[0] = rel;
        if (!isfinite(rel)) status = OR_NAN;
        else if (rel <= tol) status = OR_OK;
        else status = OR_NOT_CONVERGED;
        while (status == OR_NOT_CONVERGED && it < maxit) {
            int done = 0;
            rho0 = z_mul((oz){-omega.re, -omega.im}, rho0);
            /* BiCG part */
            for (int32_t j = 0; j < ell && !done; ++j) {
                oz rho1, gam, beta;
                if (rho0.re == 0.0 && rho0.im == 0.0) { status = OR_BREAKDOWN; done = 1; break; }
                or_zdotc(n, rh, RV(j), &rho1);
                beta = z_mul(alpha, z_div(rho1, rho0));
                rho0 = rho1;
                for (int32_t i = 0; i <= j; ++i)
                    for (int32_t e = 0; e < n; ++e) UV(i)[e] = z_sub(RV(i)[e], z_mul(beta, UV(i)[e]));
                or_zspmv(n, rowptr, col, val, UV(j), UV(j + 1));
                or_zdotc(n, rh, UV(j + 1), &gam);
                if (gam.re == 0.0 && gam.im == 0.0) { status = OR_BREAKDOWN; done = 1; break; }
                alpha = z_div(rho0, gam);
                for (int32_t i = 0; i <= j; ++i)
                    for (int32_t e = 0; e < n; ++e) RV(i)[e] = z_sub(RV(i)[e], z_mul(alpha, UV(i + 1)[e]));
                for (int32_t e = 0; e < n; ++e) x[e] = z_add(x[e], z_mul(alpha, UV(0)[e]));
                ++it;
                rel = z_norm(n, RV(0)) / nb;
                if (hist) hist[it] = rel;
                if (!isfinite(rel)) { status = OR_NAN; done = 1; break; }
                if (rel <= tol) { status = OR_OK; done = 1; break; }
                or_zspmv(n, rowptr, col, val, RV(j), RV(j + 1));
            }
            if (done) break;
            /* minimal-residual part: modified Gram-Schmidt on r_1..r_l */
            for (int32_t j = 1; j <= ell; ++j) {
                for (int32_t i = 1; i < j; ++i) {
                    oz d;
                    or_zdotc(n, RV(i), RV(j), &d);
                    tau[i][j].re = d.re / sigma[i]; tau[i][j].im = d.im / sigma[i];
                    for (int32_t e = 0; e < n; ++e) RV(j)[e] = z_sub(RV(j)[e], z_mul(tau[i][j], RV(i)[e]));
                }
                sigma[j] = z_norm(n, RV(j));
                sigma[j] *= sigma[j];
                if (sigma[j] == 0.0) { status = OR_BREAKDOWN; done = 1; break; }
                {
                    oz d;
                    or_zdotc(n, RV(j), RV(0), &d);
                    gp[j].re = d.re / sigma[j]; gp[j].im = d.im / sigma[j];
                }
            }
            if (done) break;
            /* back substitution: g solves the triangular system of the fit */
            g[ell] = gp[ell];
            omega = g[ell];
            for (int32_t j = ell - 1; j >= 1; --j) {
                oz acc = gp[j];
                for (int32_t i = j + 1; i <= ell; ++i) acc = z_sub(acc, z_mul(tau[j][i], g[i]));
                g[j] = acc;
            }
            for (int32_t j = 1; j < ell; ++j) {
                oz acc = g[j + 1];
                for (int32_t i = j + 1; i < ell; ++i) acc = z_add(acc, z_mul(tau[j][i], g[i + 1]));
                gpp[j] = acc;
            }
            /* updates (the orthogonalised r_1..r_l are what the coefficients refer to) */
            for (int32_t e = 0; e < n; ++e) {
                x[e] = z_add(x[e], z_mul(g[1], RV(0)[e]));
                RV(0)[e] = z_sub(RV(0)[e], z_mul(gp[ell], RV(ell)[e]));
                UV(0)[e] = z_sub(UV(0)[e], z_mul(g[ell], UV(ell)[e]));
            }
            for (int32_t j = 1; j < ell; ++j)
                for (int32_t e = 0; e < n; ++e) {
                    UV(0)[e] = z_sub(UV(0)[e], z_mul(g[j], UV(j)[e]));
                    x[e] = z_add(x[e], z_mul(gpp[j], RV(j)[e]));
                    RV(0)[e] = z_sub(RV(0)[e], z_mul(gp[j], RV(j)[e]));
                }
            rel = z_norm(n, RV(0)) / nb;
            if (hist) hist[it] = rel;   /* the step's entry now reflects the minimal-residual update */
            if (!isfinite(rel)) { status = OR_NAN; break; }
            if (rel <= tol) { status = OR_OK; break; }
            if (omega.re == 0.0 && omega.im == 0.0) { status = OR_BREAKDOWN; break; }
        }
        or_zspmv(n, rowptr, col, val, x, tmp);
        for (int32_t i = 0; i < n; ++i) tmp[i] = z_sub(b[i], tmp[i]);
        info->relres_true = z_norm(n, tmp) / nb;
        info->relres_rec = rel;
        if (status == OR_OK && info->relres_true > tol && restarts == 0 && it < maxit) {
            ++restarts;
            continue;
        }
        if (status == OR_OK && info->relres_true > tol) status = OR_NOT_CONVERGED;
        break;
    }
#undef RV
#undef UV
    info->iters = it;
    info->status = status;
    info->restarts = restarts;
    free(R); free(U); free(rh); free(tmp);
    return status;
}

/* ---------------------------------------------------------------------- */
/* TFQMR, Freund's transpose-free QMR (Section 7 lists P-TFQMR among the
 * paper's solvers; no preconditioner here).  Iteration j (two products with
 * A) runs the half steps m = 2j+1 and m = 2j+2:
 *   alpha = rho / <r^, v>,  u_{2j+2} = u_{2j+1} - alpha v
 *   per half step m:  w <- w - alpha A u_m  (A u_{2j+1} kept from when
 *                     u_{2j+1} was formed; A u_{2j+2} is the second product),
 *     theta_m = ||w|| / tau_{m-1},  c_m = 1/sqrt(1 + theta_m^2),
 *     tau_m = tau_{m-1} theta_m c_m,  eta_m = c_m^2 alpha,
 *     d <- u_m + (theta_{m-1}^2 eta_{m-1} / alpha) d,  x <- x + eta_m d
 *   rho' = <r^, w>,  beta = rho'/rho,  u_{2j+3} = w + beta u_{2j+2},
 *   v <- A u_{2j+3} + beta (A u_{2j+2} + beta v)   (v is not A u: it is the
 *   product with the CGS search direction).
 * The stopping test uses the quasi-residual bound ||r_m|| <= sqrt(m+1) tau_m:
 * after the second half step of each iteration, stop when
 * sqrt(m+1) tau_m <= tol ||b||.  hist[j] holds sqrt(m+1) tau_m / ||b|| of
 * iteration j.  A zero tau_{m-1} (the previous half step reached the exact
 * solution) gives theta_m = 0.  Breakdown: rho = 0 or <r^, v> = 0.  The true
 * residual is recomputed at exit; one restart as for BiCGStab. */
int or_tfqmr(int32_t n, const int32_t *rowptr, const int32_t *col, const oz *val,
             const oz *b, oz *x, double tol, int32_t maxit, double *hist, or_info *info)
{
    const size_t nn = (size_t)n;
    oz *w = calloc(nn, sizeof(oz)), *u1 = calloc(nn, sizeof(oz)), *u2 = calloc(nn, sizeof(oz));
    oz *v = calloc(nn, sizeof(oz)), *d = calloc(nn, sizeof(oz)), *au = calloc(nn, sizeof(oz));
    oz *rh = calloc(nn, sizeof(oz)), *tmp = calloc(nn, sizeof(oz)), *au1 = calloc(nn, sizeof(oz));
    double nb = z_norm(n, b), rel = 0.0;
    int32_t it = 0, status = OR_NOT_CONVERGED, restarts = 0;
    if (nb == 0.0) {
        memset(x, 0, nn * sizeof(oz));
        info->iters = 0; info->status = OR_OK; info->restarts = 0;
        info->relres_rec = 0.0; info->relres_true = 0.0;
        if (hist) hist[0] = 0.0;
        free(w); free(u1); free(u2); free(v); free(d); free(au); free(rh); free(tmp); free(au1);
        return OR_OK;
    }
    for (;;) {
        double tau, theta = 0.0;
        oz eta = {0, 0}, rho;
        int32_t m = 0;
        or_zspmv(n, rowptr, col, val, x, w);
        for (int32_t i = 0; i < n; ++i) {
            w[i] = z_sub(b[i], w[i]);
            u1[i] = w[i];
            rh[i] = w[i];
            d[i].re = d[i].im = 0.0;
        }
        tau = z_norm(n, w);
        or_zdotc(n, rh, w, &rho);
        or_zspmv(n, rowptr, col, val, u1, au1);     /* A u_1 */
        memcpy(v, au1, nn * sizeof(oz));             /* v_0 = A u_1 */
        rel = tau / nb;
        if (hist && it == 0) hist[0] = rel;
        if (!isfinite(rel)) status = OR_NAN;
        else if (rel <= tol) status = OR_OK;
        else status = OR_NOT_CONVERGED;
        while (status == OR_NOT_CONVERGED && it < maxit) {
            oz sig, alpha, rho1, beta;
            if (rho.re == 0.0 && rho.im == 0.0) { status = OR_BREAKDOWN; break; }
            or_zdotc(n, rh, v, &sig);
            if (sig.re == 0.0 && sig.im == 0.0) { status = OR_BREAKDOWN; break; }
            alpha = z_div(rho, sig);
            for (int32_t i = 0; i < n; ++i) u2[i] = z_sub(u1[i], z_mul(alpha, v[i]));
            for (int32_t half = 0; half < 2; ++half) {
                const oz *um = half == 0 ? u1 : u2;
                oz coef;
                double th_prev = theta, wn, c;
                if (half == 0) memcpy(au, au1, nn * sizeof(oz));        /* A u_{2j+1} */
                else or_zspmv(n, rowptr, col, val, u2, au);            /* A u_{2j+2} */
                for (int32_t i = 0; i < n; ++i) w[i] = z_sub(w[i], z_mul(alpha, au[i]));
                ++m;
                wn = z_norm(n, w);
                theta = tau == 0.0 ? 0.0 : wn / tau;
                c = 1.0 / sqrt(1.0 + theta * theta);
                tau = tau * theta * c;
                coef = z_div(z_mul((oz){th_prev * th_prev, 0.0}, eta), alpha);
                eta.re = c * c * alpha.re; eta.im = c * c * alpha.im;
                for (int32_t i = 0; i < n; ++i) {
                    d[i] = z_add(um[i], z_mul(coef, d[i]));
                    x[i] = z_add(x[i], z_mul(eta, d[i]));
                }
            }
            ++it;
            rel = sqrt((double)m + 1.0) * tau / nb;
            if (hist) hist[it] = rel;
            if (!isfinite(rel)) { status = OR_NAN; break; }
            if (rel <= tol) { status = OR_OK; break; }
            or_zdotc(n, rh, w, &rho1);
            beta = z_div(rho1, rho);
            rho = rho1;
            /* au holds A u_{2j+2} */
            for (int32_t i = 0; i < n; ++i) {
                u1[i] = z_add(w[i], z_mul(beta, u2[i]));
                tmp[i] = z_add(au[i], z_mul(beta, v[i]));
            }
            or_zspmv(n, rowptr, col, val, u1, au1);
            for (int32_t i = 0; i < n; ++i) v[i] = z_add(au1[i], z_mul(beta, tmp[i]));
        }
        or_zspmv(n, rowptr, col, val, x, tmp);
        for (int32_t i = 0; i < n; ++i) tmp[i] = z_sub(b[i], tmp[i]);
        info->relres_true = z_norm(n, tmp) / nb;
        info->relres_rec = rel;
        if (status == OR_OK && info->relres_true > tol && restarts == 0 && it < maxit) {
            ++restarts;
            continue;
        }
        if (status == OR_OK && info->relres_true > tol) status = OR_NOT_CONVERGED;
        break;
    }
    info->iters = it;
    info->status = status;
    info->restarts = restarts;
    free(w); free(u1); free(u2); free(v); free(d); free(au); free(rh); free(tmp); free(au1);
    return status;
}

/* ---------------------------------------------------------------------- */
/* Same iteration in complex64 with binary32 sums: the inner solver of the
 * mixed-precision refinement.  x0 = 0, stopping on ||r|| <= tol ||b||.
 * Returns the iteration count; *status gets the exit reason.  hist
 * (optional, maxit+1 entries) receives ||r_j|| / ||b|| as or_bicgstab's does:
 * hist[0] = 1 (r0 = b), hist[j] after iteration j (||s|| / ||b|| for a
 * half-step exit). */
static float c_norm(int32_t n, const oc *x)
{
    float s = 0.0f;
    for (int32_t i = 0; i < n; ++i) s += x[i].re * x[i].re + x[i].im * x[i].im;
    return sqrtf(s);
}
static oc c_dotc(int32_t n, const oc *x, const oc *y)
{
    oc s = {0.0f, 0.0f};
    for (int32_t i = 0; i < n; ++i) s = c_add(s, c_mul(c_conj(x[i]), y[i]));
    return s;
}

int32_t or_cbicgstab(int32_t n, const int32_t *rowptr, const int32_t *col, const oc *val,
                     const oc *b, oc *x, float tol, int32_t maxit, int32_t *status, double *hist)
{
    oc *r = calloc((size_t)n, sizeof(oc)), *rh = calloc((size_t)n, sizeof(oc));
    oc *p = calloc((size_t)n, sizeof(oc)), *v = calloc((size_t)n, sizeof(oc));
    oc *s = calloc((size_t)n, sizeof(oc)), *t = calloc((size_t)n, sizeof(oc));
    oc rho_old = {1, 0}, alpha = {1, 0}, omega = {1, 0};
    float nb = c_norm(n, b);
    int32_t it = 0;
    *status = OR_NOT_CONVERGED;
    memset(x, 0, (size_t)n * sizeof(oc));
    if (nb == 0.0f) { *status = OR_OK; if (hist) hist[0] = 0.0; goto done; }
    if (hist) hist[0] = 1.0;
    for (int32_t i = 0; i < n; ++i) { r[i] = b[i]; rh[i] = b[i]; }
    while (it < maxit) {
        oc rho, sig, ts, tt, beta;
        float rel;
        ++it;
        rho = c_dotc(n, rh, r);
        if (rho.re == 0.0f && rho.im == 0.0f) { *status = OR_BREAKDOWN; break; }
        beta = c_mul(c_div(rho, rho_old), c_div(alpha, omega));
        for (int32_t i = 0; i < n; ++i)
            p[i] = c_add(r[i], c_mul(beta, c_sub(p[i], c_mul(omega, v[i]))));
        or_cspmv(n, rowptr, col, val, p, v);
        sig = c_dotc(n, rh, v);
        if (sig.re == 0.0f && sig.im == 0.0f) { *status = OR_BREAKDOWN; break; }
        alpha = c_div(rho, sig);
        for (int32_t i = 0; i < n; ++i) s[i] = c_sub(r[i], c_mul(alpha, v[i]));
        rel = c_norm(n, s) / nb;
        if (!isfinite(rel)) { *status = OR_NAN; break; }
        if (rel <= tol) {
            for (int32_t i = 0; i < n; ++i) x[i] = c_add(x[i], c_mul(alpha, p[i]));
            if (hist) hist[it] = (double)rel;
            *status = OR_OK;
            break;
        }
        or_cspmv(n, rowptr, col, val, s, t);
        ts = c_dotc(n, t, s);
        tt = c_dotc(n, t, t);
        if (tt.re == 0.0f && tt.im == 0.0f) { *status = OR_BREAKDOWN; break; }
        omega = c_div(ts, tt);
        for (int32_t i = 0; i < n; ++i) {
            x[i] = c_add(x[i], c_add(c_mul(alpha, p[i]), c_mul(omega, s[i])));
            r[i] = c_sub(s[i], c_mul(omega, t[i]));
        }
        rho_old = rho;
        rel = c_norm(n, r) / nb;
        if (hist) hist[it] = (double)rel;
        if (!isfinite(rel)) { *status = OR_NAN; break; }
        if (rel <= tol) { *status = OR_OK; break; }
        if (omega.re == 0.0f && omega.im == 0.0f) { *status = OR_BREAKDOWN; break; }
    }
done:
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return it;
}

/* Mixed-precision iterative refinement (classical, Wilkinson/Moler):
 *   repeat: r = b - A x (binary64);  stop if ||r|| <= tol ||b||
 *           solve A d = r approximately in complex64 (inner BiCGStab, tol_in)
 *           x = x + d (binary64)
 * The complex64 operator is the rounded copy val32 of val.  The refinement
 * keeps the iterate with the smallest outer residual: when a step fails to
 * reduce ||r|| (or the residual is not finite), it stops and returns that
 * best iterate with its residual instead of the last one. */
int or_refine_mixed(int32_t n, const int32_t *rowptr, const int32_t *col, const oz *val,
                    const oc *val32, const oz *b, oz *x, double tol, float tol_in,
                    int32_t maxit_in, int32_t max_outer, int32_t *outer_out,
                    int32_t *inner_total, double *relres_out)
{
    oz *r = calloc((size_t)n, sizeof(oz)), *xbest = calloc((size_t)n, sizeof(oz));
    oc *r32 = calloc((size_t)n, sizeof(oc)), *d32 = calloc((size_t)n, sizeof(oc));
    double nb = z_norm(n, b), rel = 0.0, best = INFINITY;
    int32_t outer = 0, inner = 0, status = OR_NOT_CONVERGED, use_best = 0;
    if (nb == 0.0) {
        memset(x, 0, (size_t)n * sizeof(oz));
        status = OR_OK;
    } else {
        for (;;) {
            int32_t st, k;
            or_zspmv(n, rowptr, col, val, x, r);
            for (int32_t i = 0; i < n; ++i) r[i] = z_sub(b[i], r[i]);
            rel = z_norm(n, r) / nb;
            if (!isfinite(rel)) { status = OR_NAN; use_best = outer > 0; break; }
            if (rel <= tol) { status = OR_OK; break; }
            if (rel >= best) { use_best = 1; break; }
            if (outer >= max_outer) break;
            best = rel;
            memcpy(xbest, x, (size_t)n * sizeof(oz));
            ++outer;
            for (int32_t i = 0; i < n; ++i) { r32[i].re = (float)r[i].re; r32[i].im = (float)r[i].im; }
            k = or_cbicgstab(n, rowptr, col, val32, r32, d32, tol_in, maxit_in, &st, NULL);
            inner += k;
            for (int32_t i = 0; i < n; ++i) {
                x[i].re += (double)d32[i].re;
                x[i].im += (double)d32[i].im;
            }
        }
    }
    if (use_best) {
        memcpy(x, xbest, (size_t)n * sizeof(oz));
        rel = best;
    }
    *outer_out = outer;
    *inner_total = inner;
    *relres_out = rel;
    free(r); free(xbest); free(r32); free(d32);
    return status;
}

/* ---------------------------------------------------------------------- */
/* Adjoint of x = A^{-1} b for a complex-symmetric A (A = A^T): with mu the
 * solution of A^T mu = conj(g), where g is the conjugate-Wirtinger gradient
 * of a real loss with respect to x, the gradient with respect to the stored
 * entry A_ij is -conj(mu_i x_j).  This routine forms that product on A's
 * sparsity pattern. */
void or_outer_on_pattern(int32_t n, const int32_t *rowptr, const int32_t *col,
                         const oz *mu, const oz *x, oz *grad)
{
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            oz m = z_mul(mu[i], x[col[k]]);
            grad[k].re = -m.re;
            grad[k].im = m.im;
        }
}
