/*
 * hz.h -- C ABI of the GB300 complex Helmholtz Krylov library (libhz.so).
 *
 * The library computes the hot path of Cheik Ahamed & Magoules, "Accelerated
 * solution of Helmholtz equation with Iterative Krylov Methods on GPU":
 * complex-double sparse matrix-vector products on CSR matrices (Section 6),
 * the complex BLAS-1 operations assign / scale / axpy / dot / norm
 * (Section 5), and the BiCGStab Krylov solver built from them (Section 7),
 * for complex-symmetric Helmholtz systems (Section 2: -lap(u) - k^2 u = g).
 *
 * Conventions shared by every entry point:
 *  - Complex numbers are two contiguous IEEE doubles (real, imaginary), the
 *    layout of Section 4 (listing "Complex number in memory"); hz_z is
 *    layout-identical to cuDoubleComplex, std::complex<double> and one
 *    element of a torch.complex128 tensor.  hz_c is the complex64 analogue.
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device,
 *    allocated and owned by the caller; the library never frees them.
 *    Pointers named h_* are host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call is asynchronous on that stream unless its comment
 *    says it synchronises.
 *  - Every call returns an hz_status; nothing throws across the ABI.  On an
 *    error, hz_last_error() returns a message for the calling thread.
 *  - Scalars (alpha, dot results) live in device memory so that no call
 *    needs a host round trip.
 *  - Reductions use a small scratch area (block partial sums and a
 *    completion counter) that the library allocates once per (device,
 *    stream) pair on first use and keeps until process exit, so calls on
 *    different streams never share scratch.  The first reduction issued on
 *    a new stream therefore allocates: issue it before any stream capture.
 */
#ifndef HZ_H
#define HZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HZ_API __attribute__((visibility("default")))
#else
#define HZ_API
#endif

typedef struct { double re, im; } hz_z;   /* complex128 element (Section 4) */
typedef struct { float re, im; } hz_c;    /* complex64 element */

typedef struct hz_mat hz_mat;             /* opaque matrix handle */

typedef enum {
    HZ_OK = 0,
    HZ_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad CSR) */
    HZ_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    HZ_ERR_ALLOC = 3,        /* device or host allocation failed */
    HZ_NOT_CONVERGED = 4,    /* solver stopped at maxit above tolerance */
    HZ_BREAKDOWN = 5,        /* BiCGStab breakdown: rho, <rh,v> or omega became 0 */
    HZ_ERR_NAN = 6,          /* a residual became NaN or Inf */
    HZ_ERR_TIMEOUT = 7       /* a bounded device-side wait gave up */
} hz_status;

/* matrix creation flags */
enum {
    HZ_FLAG_VALIDATE = 1u,   /* check rowptr monotone, rowptr[n]==nnz, cols in range (host copy) */
    HZ_FLAG_SELL = 2u,       /* also build a SELL-C-sigma copy and use it for SpMV */
    HZ_FLAG_C64 = 4u,        /* also build the complex64 copy used by the mixed solver */
    HZ_FLAG_AUTOTUNE = 8u,   /* time the SpMV variants once on this matrix and keep the fastest;
                                `group` becomes the fastest binary64 CSR-vector group (the row
                                tile of this matrix in hz_zsolve_batched's complex64 and
                                double-float products) whichever kind wins */
    HZ_FLAG_FF = 16u         /* also build the double-float split of the values and use the
                                double-float SpMV: every binary64 value is carried as hi + lo
                                binary32 parts (48 significant bits, NOT binary64) on the
                                binary32 pipes.  The split keeps its 48 bits only for values
                                of magnitude in [2^-100, 2^101): if any stored value lies
                                outside, the handle keeps the binary64 kind HZ_SPMV_FLAT64P
                                (hz_mat_query reports it).  hz_zspmv on a double-float kind
                                needs x in the same range; the BiCGStab solve scales b and the
                                operator by powers of two (exact) so that its vectors stay
                                there whatever the size of b */
};

/* solver modes */
enum {
    HZ_MODE_FP64 = 0u,       /* complex128 BiCGStab */
    HZ_MODE_MIXED = 1u       /* complex64 inner BiCGStab + complex128 iterative refinement */
};

/* Krylov methods of Section 7 */
enum {
    HZ_METHOD_BICGSTAB = 0u,   /* BiCGStab (van der Vorst) */
    HZ_METHOD_BICGSTABL = 1u,  /* BiCGStab(l) (Sleijpen and Fokkema), 1 <= l <= 8; iterations are
                                  counted in BiCG steps (two products with A each) */
    HZ_METHOD_TFQMR = 2u       /* TFQMR (Freund); stops on the quasi-residual bound
                                  sqrt(m+1) tau_m <= tol ||b||, which bounds ||b - A x|| */
};

/* preconditioners (Section 7 names its solvers P-BiCGSTAB etc. without
 * saying which preconditioner; none is the default reading) */
enum {
    HZ_PRECOND_NONE = 0u,
    HZ_PRECOND_JACOBI = 1u   /* right preconditioning by the inverse diagonal: 1 / a_ii, or 1 where
                                row i has no (or a zero) diagonal; the stopping test stays on the
                                residual of A x = b */
};

/* SpMV kernel variants reported by hz_mat_query */
enum {
    HZ_SPMV_CSR_VECTOR = 0,  /* a group of `group` lanes per row */
    HZ_SPMV_SELL = 1,        /* SELL-C-sigma, one lane per row, C = 32 */
    HZ_SPMV_FF = 2,          /* CSR-vector in double-float arithmetic: every binary64 value is
                                split into hi + lo binary32 parts (48 significant bits) and each
                                product and sum uses error-free transformations; per-entry error
                                <= about (4 + row length / group) * 2^-48 * sum_j |a_ij| |x_j| */
    HZ_SPMV_SELL_FF = 3,     /* SELL-C-sigma layout in double-float arithmetic (one lane per row;
                                error bound as HZ_SPMV_FF with group 1) */
    HZ_SPMV_FF_FLAT = 4,     /* double-float, row blocks streamed flat: each entry's product is
                                formed with coalesced loads and all lanes busy, then whole rows
                                are summed from shared memory (the default with HZ_FLAG_FF) */
    HZ_SPMV_FF_TMA = 5,      /* HZ_SPMV_FF_FLAT with the values and columns moved into shared
                                memory by bulk asynchronous copies, one row block ahead of the
                                arithmetic */
    HZ_SPMV_FLAT64 = 6,      /* binary64 (IEEE double FMAs), row blocks of complete rows with every
                                lane summing one contiguous run of entries, rows that cross a
                                run boundary finished from the runs' partial sums (the default
                                without HZ_FLAG_FF where the packed copy below cannot be built:
                                more than 2^31 slots); groups of real values take two FMAs per
                                entry (the skipped terms are exact zeros; 0 * inf still gives
                                NaN); per-entry error within the binary64 bound of a row sum,
                                (2 m + 1) 2^-53 sum_j |a_ij| |x_j| for a row of m entries */
    HZ_SPMV_FLAT64P = 7      /* HZ_SPMV_FLAT64 on a packed copy of the row blocks that the handle
                                owns (built by hz_csr_create, rebuilt by hz_mat_refresh_values):
                                step u of the 32 lane runs stored as 32 consecutive slots (column,
                                real part), so every load is coalesced, and the imaginary parts
                                stored only for groups of steps that have a nonzero one (a group
                                without is known to be real before its loads; the same sums as
                                HZ_SPMV_FLAT64).  Device memory: 20 bytes per slot, about nnz
                                slots.  The default without HZ_FLAG_FF */
};

typedef struct {
    int32_t n, nnz;
    int32_t max_row, min_row;
    double mean_row;
    int32_t spmv_kind;       /* HZ_SPMV_* */
    int32_t group;           /* lanes per row for HZ_SPMV_CSR_VECTOR */
    int64_t sell_slots;      /* padded slots of the SELL copy (0 if none) */
    int32_t sell_sigma;      /* sorting window of the SELL copy */
    int32_t has_c64;
} hz_mat_props;

/*
 * Create a matrix handle from a CSR matrix already on the device.
 *
 * Section 3.2 defines CSR by three arrays: values AA (nnz), column indices
 * JA (nnz) and row pointers IA (n+1), with row i stored in positions
 * IA(i) .. IA(i+1)-1.  Here d_val = AA, d_col = JA, d_rowptr = IA,
 * int32 indices with base index_base (0, or 1 as in the paper, where
 * IA(n+1) = nnz+1).  Within a row, columns may come in any order.
 *
 * The handle BORROWS d_rowptr, d_col and d_val when index_base == 0 (the
 * caller keeps them alive and unchanged until hz_mat_destroy, except through
 * hz_mat_set_diag); with index_base == 1 it keeps 0-based copies it owns.
 * SELL-C-sigma and complex64 copies (flags) are owned by the handle.
 * Synchronises `stream` once (row statistics are computed on the host).
 * d_val must be 16-byte aligned (any complex128 allocation is), d_col and
 * d_rowptr 4-byte aligned.
 * Errors: HZ_ERR_ARG for n < 0, nnz < 0, n or nnz above 2^31 - 4097 (the
 * kernels' int32 index arithmetic runs up to 4096 past them), null pointers
 * with nonzero sizes, misaligned arrays, index_base not 0/1, or (with
 * HZ_FLAG_VALIDATE) a malformed CSR; all but the last are detected before
 * any array is read.
 */
HZ_API hz_status hz_csr_create(hz_mat **A, int32_t n, int32_t nnz, const int32_t *d_rowptr,
                               const int32_t *d_col, const hz_z *d_val, int32_t index_base,
                               uint32_t flags, void *stream);

/* Release a handle and everything it owns (synchronises the device). */
HZ_API hz_status hz_mat_destroy(hz_mat *A);

/* Row statistics and the SpMV variant chosen for this matrix. */
HZ_API hz_status hz_mat_query(const hz_mat *A, hz_mat_props *props);

/*
 * Health of the asynchronous work on a handle (no counterpart in the paper).
 * The HZ_SPMV_FF_TMA kernel waits on its bulk copies with a wall-time limit
 * (1 s); if a wait ever expires, the kernel stops early, its output is
 * incomplete, and it sets a sticky fault word in the handle.  This call
 * synchronises `stream` and returns HZ_ERR_TIMEOUT if that word is set,
 * HZ_OK otherwise.  A solve on the handle reports the same condition in its
 * own status.
 */
HZ_API hz_status hz_mat_check(const hz_mat *A, void *stream);

/*
 * Force the SpMV variant of a handle: kind HZ_SPMV_CSR_VECTOR or HZ_SPMV_FF
 * with group in {2, 4, 8, 16, 32} lanes per row (HZ_SPMV_FF needs a handle
 * created with HZ_FLAG_FF), or HZ_SPMV_SELL (the handle must have been
 * created with HZ_FLAG_SELL), or HZ_SPMV_SELL_FF (both flags), or
 * HZ_SPMV_FF_FLAT / HZ_SPMV_FF_TMA (HZ_FLAG_FF); group is ignored for all
 * but the CSR-vector kinds.  Overrides the histogram choice and the
 * autotuner; solver graphs built for the old variant are rebuilt on the
 * next solve.  Errors: HZ_ERR_ARG for an unknown variant.
 */
HZ_API hz_status hz_mat_set_spmv(hz_mat *A, int32_t kind, int32_t group);

/*
 * Re-derive the handle's SELL and complex64 copies after the caller changed
 * the values in d_val (the pattern must be unchanged).
 */
HZ_API hz_status hz_mat_refresh_values(hz_mat *A, void *stream);

/*
 * y = A x (Section 6, CSR matrix-vector product), complex128.
 * d_x and d_y have n entries, are 16-byte aligned and must not overlap.  On the double-float
 * variants (HZ_SPMV_FF, HZ_SPMV_SELL_FF, HZ_SPMV_FF_FLAT, HZ_SPMV_FF_TMA)
 * the handle's own x scratch holds
 * the split of d_x, so calls on one handle must not overlap in time
 * (different handles may).
 */
HZ_API hz_status hz_zspmv(const hz_mat *A, const hz_z *d_x, hz_z *d_y, void *stream);

/* y = A32 x in complex64 with binary32 sums, using the handle's complex64
 * copy of the values (created on demand; synchronises on first use). */
HZ_API hz_status hz_cspmv(hz_mat *A, const hz_c *d_x, hz_c *d_y, void *stream);

/* *d_result = sum_i conj(x_i) y_i (Section 5, dot product; conjugated form). */
HZ_API hz_status hz_zdotc(int64_t n, const hz_z *d_x, const hz_z *d_y, hz_z *d_result,
                          void *stream);

/* *d_result = sum_i x_i y_i (Section 5, dot product; unconjugated form). */
HZ_API hz_status hz_zdotu(int64_t n, const hz_z *d_x, const hz_z *d_y, hz_z *d_result,
                          void *stream);

/*
 * hz_zdotc without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory,
 * for example code that runs inside a fixed memory budget already handed to
 * its own pool allocator, or code on a latency-critical path where the
 * implicit device synchronisation of cudaMalloc is not acceptable.
 * hz_zdotc allocates its reduction scratch on the first call on each stream;
 * this variant instead keeps its scratch (1 MiB of tile partial sums and a
 * completion counter) in a fixed array compiled into the library, present on
 * every GPU that loads the library until the process exits.
 *
 * Result, arguments and errors as hz_zdotc, except:
 *  - n must be at most 2^28 (268,435,456); larger n returns HZ_ERR_ARG.
 *  - The first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *  - Every call shares the one array (the counter is cleared on the caller's
 *    stream at each call; the partial sums keep the last call's contents),
 *    so calls whose kernels overlap on the GPU -- on different streams or
 *    from different threads -- race and give wrong results.  Serialise them.
 *  - The sum is folded over fixed tiles of 4096 elements, so the result is
 *    bitwise reproducible across GPUs; it may differ from hz_zdotc's in the
 *    last bits.
 */
HZ_API hz_status hz_zdotc_noalloc(int64_t n, const hz_z *d_x, const hz_z *d_y, hz_z *d_result,
                                  void *stream);

/* *d_result = sqrt(sum_i |x_i|^2) (Section 5, L2 norm). */
HZ_API hz_status hz_dznrm2(int64_t n, const hz_z *d_x, double *d_result, void *stream);

/* y_i = alpha x_i + y_i (Section 5, Zaxpy); *d_alpha is read on the device. */
HZ_API hz_status hz_zaxpy(int64_t n, const hz_z *d_alpha, const hz_z *d_x, hz_z *d_y,
                          void *stream);

/* x_i = alpha x_i (Section 5, scale); *d_alpha is read on the device. */
HZ_API hz_status hz_zscal(int64_t n, const hz_z *d_alpha, hz_z *d_x, void *stream);

/* y_i = x_i (Section 5, assign). */
HZ_API hz_status hz_zcopy(int64_t n, const hz_z *d_x, hz_z *d_y, void *stream);

/*
 * z_i = x_i * y_i (Section 5, element-wise product; with y = D^-1 it is the
 * Jacobi preconditioner step z = D^-1 r).  Vectors of n complex128 entries;
 * z may equal x or y.
 */
HZ_API hz_status hz_zmul_elementwise(int64_t n, const hz_z *d_x, const hz_z *d_y, hz_z *d_z, void *stream);

/* y_i = conj(x_i); y may equal x. */
HZ_API hz_status hz_zconj(int64_t n, const hz_z *d_x, hz_z *d_y, void *stream);

typedef struct {
    int32_t iters;           /* BiCGStab iterations (inner iterations summed in mixed mode) */
    int32_t status;          /* hz_status of the solve */
    int32_t restarts;        /* restarts taken after a recursive/true residual mismatch */
    int32_t outer;           /* refinement steps (mixed mode), else 0 */
    double relres_rec;       /* last recursive residual ||r|| / ||b|| */
    double relres_true;      /* ||b - A x|| / ||b|| recomputed at exit */
} hz_info;

typedef struct {
    double tol;              /* relative residual tolerance ||b - A x|| <= tol ||b|| */
    int32_t maxit;           /* iteration cap (inner iterations summed in mixed mode) */
    uint32_t mode;           /* HZ_MODE_FP64 or HZ_MODE_MIXED */
    float inner_tol;         /* mixed: inner complex64 relative tolerance (default 1e-5) */
    int32_t inner_maxit;     /* mixed: inner iteration cap per refinement step */
    int32_t max_outer;       /* mixed: refinement step cap */
    int32_t x0_is_zero;      /* 1: ignore d_x on entry and start from x0 = 0 */
    double *d_hist;          /* optional device array of maxit+1 doubles: residual history */
    uint32_t precond;        /* HZ_PRECOND_NONE or HZ_PRECOND_JACOBI */
    uint32_t method;         /* HZ_METHOD_BICGSTAB (default 0), HZ_METHOD_BICGSTABL or HZ_METHOD_TFQMR */
    int32_t ell;             /* BiCGStab(l): l in 1..8 */
} hz_solve_opts;

/*
 * Solve A x = b with preconditioner-free BiCGStab (Section 7; van der
 * Vorst's algorithm as stated in Saad's book, which the paper cites).
 * Inner products are Hermitian (<u,w> = sum conj(u_i) w_i); the stopping
 * test is ||r|| <= tol ||b|| on the recursive residual, with a half-step
 * exit on ||s||; on exit the true residual is recomputed and, if it misses
 * tol while the recursive one met it, the iteration restarts once from the
 * current x.  b = 0 gives x = 0.
 *
 * d_x holds x0 on entry (unless x0_is_zero) and the solution on exit (also
 * on HZ_NOT_CONVERGED / HZ_BREAKDOWN: the last iterate).  The whole
 * iteration runs on the device inside one CUDA graph with a device-side
 * loop; the call synchronises `stream` once per (re)start and fills *h_info.
 * The handle keeps the solver workspace (7 vectors of n complex numbers,
 * plus the complex64 copies in mixed mode) and the graph between calls.
 * Calls on the same handle must not overlap.
 * Returns the solve status (HZ_OK, HZ_NOT_CONVERGED, HZ_BREAKDOWN,
 * HZ_ERR_NAN) or an error code.
 */
HZ_API hz_status hz_zsolve(hz_mat *A, const hz_z *d_b, hz_z *d_x, double tol, int32_t maxit,
                           uint32_t mode, hz_info *h_info, void *stream);

/*
 * hz_zsolve with every option explicit (opts must not be NULL).
 * With precond = HZ_PRECOND_JACOBI the handle builds, on first use, the
 * column-scaled operator A D^-1 (D = diag(A), a second set of values the
 * handle owns, with the same SpMV copies as A) and solves A D^-1 y = b from
 * y0 = D x0, returning x = D^-1 y; the residuals and the stopping test are
 * those of A x = b.  The scaled copy is rebuilt after hz_mat_refresh_values
 * or hz_mat_set_diag.
 */
HZ_API hz_status hz_zsolve_opts(hz_mat *A, const hz_z *d_b, hz_z *d_x,
                                const hz_solve_opts *opts, hz_info *h_info, void *stream);

/*
 * Solve nsys independent systems A[s] x[s] = b[s] (a frequency sweep) in one
 * persistent cooperative launch: every system keeps its own BiCGStab state
 * on the device; all systems advance together through the phases of the
 * iteration and leave the batch as they converge.  Same algorithm,
 * stopping rule and status semantics as hz_zsolve (no restart), per system.
 * mode HZ_MODE_FP64: the batch runs in double-float arithmetic when every
 * handle (with n > 0) was created with HZ_FLAG_FF and its SpMV kind is a
 * double-float one, in binary64 otherwise.  mode HZ_MODE_MIXED: every system
 * runs the mixed-precision refinement of hz_zsolve (binary64 outer residual
 * and update, complex64 inner BiCGStab to 1e-5 with at most 1000 iterations,
 * at most 50 refinement steps, maxit capping the inner iterations in total,
 * the best iterate kept), each system at its own stage; the handles' complex64
 * copies are made on demand (synchronising).  Binary64 products run on each
 * handle's row blocks (the block-flat core of HZ_SPMV_FLAT64), complex64 and
 * double-float ones with `group` lanes per row.  d_x[s] holds x0 on entry and
 * the solution on exit.  h_info has nsys entries.  Synchronises `stream`.
 * Errors: HZ_ERR_ARG (nsys outside 0..1024, unknown mode, null pointers),
 * HZ_ERR_ALLOC, HZ_ERR_TIMEOUT (a grid-barrier wait expired).
 */
HZ_API hz_status hz_zsolve_batched(int32_t nsys, hz_mat *const *A, const hz_z *const *d_b,
                                   hz_z *const *d_x, double tol, int32_t maxit, uint32_t mode,
                                   hz_info *h_info, void *stream);

/*
 * Adjoint product on the sparsity pattern: for every stored entry k = (i, j)
 * of A, d_gradval[k] = -conj(mu_i x_j).  With x = A^{-1} b, g the
 * conjugate-Wirtinger gradient of a real loss with respect to x, and mu the
 * solution of A^T mu = conj(g), this is the gradient of the loss with
 * respect to the stored values of A (A complex symmetric, so A^T = A).
 */
HZ_API hz_status hz_outer_on_pattern(const hz_mat *A, const hz_z *d_mu, const hz_z *d_x,
                                     hz_z *d_gradval, void *stream);

/*
 * Parametrised diagonal: A_ii = base_i + scale * theta_i, written into the
 * caller's value array (every row must store its diagonal entry), then the
 * handle's copies are refreshed.
 */
HZ_API hz_status hz_mat_set_diag(hz_mat *A, const hz_z *d_base, hz_z scale, const hz_z *d_theta,
                                 void *stream);

/*
 * Gradient with respect to theta of the parametrised diagonal above:
 * d_grad_theta_i = conj(scale) * (-conj(mu_i x_i)).
 */
HZ_API hz_status hz_diag_grad(const hz_mat *A, const hz_z *d_mu, const hz_z *d_x, hz_z scale,
                              hz_z *d_grad_theta, void *stream);

/* Thread-local message describing the last error (never NULL). */
HZ_API const char *hz_last_error(void);

/* Library ABI version (major * 100 + minor). */
HZ_API int32_t hz_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HZ_H */
