// precond.cu -- Jacobi (diagonal) right preconditioning for the solvers and
// the element-wise product of Section 5.
//
// Section 7 runs "P-" Krylov solvers without naming the preconditioner; the
// Jacobi form z = D^-1 r is the paper's element-wise product kernel applied
// with the inverse diagonal.  Right preconditioning solves A D^-1 y = b and
// returns x = D^-1 y, so the residual the solver tracks is that of A x = b.
// Rather than one more vector pass per SpMV, the scaling is folded into the
// operator once: the handle keeps a second hz_mat over the same rowptr/col
// with values a_ij / d_j (and whatever SELL / double-float / complex64 copies
// the original has), and the solver graph built on it is the unpreconditioned
// one; only the start (y0 = D x0) and the copy-out (x = D^-1 y) change.
#include <algorithm>

#include "spmv.cuh"

namespace hz {

// d_i = sum of row i's stored entries in column i (1 if that is 0 or there
// is none); dinv_i = 1 / d_i.  One row per thread (rows are short; the pass
// runs once per handle).
__global__ void k_jacobi_diag(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                              const double2 *__restrict__ val, double2 *__restrict__ d,
                              double2 *__restrict__ dinv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (col[k] == i) s = cadd(s, val[k]);
        if (s.x == 0.0 && s.y == 0.0) s = make_double2(1.0, 0.0);
        d[i] = s;
        dinv[i] = cdiv(make_double2(1.0, 0.0), s);
    }
}

// out_k = val_k * dinv[col_k]: the columns of A scaled by D^-1
__global__ void k_scale_cols(int64_t nnz, const int *__restrict__ col, const double2 *__restrict__ val,
                             const double2 *__restrict__ dinv, double2 *__restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = cmul(val[k], dinv[col[k]]);
}

__global__ void k_zmul_ew(int64_t n, const double2 *__restrict__ x, const double2 *__restrict__ y,
                          double2 *__restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = cmul(x[i], y[i]);
}

void free_jacobi(hz_mat *A) {
    if (A->jac) hz_mat_destroy(A->jac);
    cudaFree(A->jac_val);
    cudaFree(A->jac_d);
    cudaFree(A->jac_dinv);
    A->jac = nullptr;
    A->jac_val = A->jac_d = A->jac_dinv = nullptr;
}

hz_status ensure_jacobi(hz_mat *A, cudaStream_t s) {
    if (A->jac) return HZ_OK;
    DevInfo d;
    HZ_TRY(dev_info(&d));
    const int n = A->n, nnz = A->nnz;
    if (cudaMalloc(&A->jac_d, sizeof(double2) * std::max(n, 1)) != cudaSuccess ||
        cudaMalloc(&A->jac_dinv, sizeof(double2) * std::max(n, 1)) != cudaSuccess ||
        cudaMalloc(&A->jac_val, sizeof(double2) * std::max(nnz, 1)) != cudaSuccess) {
        free_jacobi(A);
        set_error("Jacobi preconditioner: allocation failed");
        return HZ_ERR_ALLOC;
    }
    if (n) k_jacobi_diag<<<stream_grid(d, n, 256, 8), 256, 0, s>>>(n, A->rowptr, A->col, A->val, A->jac_d, A->jac_dinv);
    if (nnz) k_scale_cols<<<stream_grid(d, nnz, 256, 8), 256, 0, s>>>(nnz, A->col, A->val, A->jac_dinv, A->jac_val);
    if (cudaGetLastError() != cudaSuccess) {
        free_jacobi(A);
        set_error("Jacobi preconditioner: launch failed");
        return HZ_ERR_CUDA;
    }
    const uint32_t flags = (A->sell_val ? HZ_FLAG_SELL : 0u) | (A->val_ff ? HZ_FLAG_FF : 0u) |
                           (A->val32 ? HZ_FLAG_C64 : 0u);
    hz_mat *J = nullptr;
    const hz_status st = hz_csr_create(&J, n, nnz, A->rowptr, A->col, (const hz_z *)A->jac_val, 0, flags, s);
    if (st != HZ_OK) {
        free_jacobi(A);
        return st;
    }
    J->spmv_kind = A->spmv_kind;
    J->group = A->group;
    A->jac = J;
    return HZ_OK;
}

}  // namespace hz

using namespace hz;

extern "C" HZ_API hz_status hz_zmul_elementwise(int64_t n, const hz_z *d_x, const hz_z *d_y, hz_z *d_z,
                                                void *stream) {
    HZ_CHECK(n >= 0, "hz_zmul_elementwise: negative n");
    if (n == 0) return HZ_OK;
    HZ_CHECK(d_x && d_y && d_z, "hz_zmul_elementwise: null vector");
    DevInfo d;
    HZ_TRY(dev_info(&d));
    k_zmul_ew<<<stream_grid(d, n, 256, 8), 256, 0, (cudaStream_t)stream>>>(n, (const double2 *)d_x,
                                                                         (const double2 *)d_y, (double2 *)d_z);
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}
