// adjoint.cu -- kernels of the adjoint (reverse-mode) solve x = A^{-1} b.
//
// For a real loss L with conjugate-Wirtinger gradient g = 2 dL/d(conj x),
// and mu the solution of A^T mu = conj(g) (A complex symmetric, so the same
// operator as the forward solve), the gradients are
//     dL/dA_ij (stored entries)  = -conj(mu_i x_j)
//     dL/db                      =  conj(mu)
// and for a diagonal parametrised as A_ii = base_i + c * theta_i,
//     dL/dtheta_i                =  conj(c) * (-conj(mu_i x_i)).
#include <algorithm>
#include <vector>

#include "hz_internal.cuh"
#include "spmv.cuh"   // kFlatCap: the entries of a row block with more than one row

namespace hz {

// -conj(a b) = (Im a Im b - Re a Re b, Re a Im b + Im a Re b), with the sign
// on the FMA operands: four binary64 operations (negating the finished
// product would take a fifth on the binary64 pipe)
__device__ __forceinline__ double2 neg_conj_mul(double2 a, double2 b) {
    return make_double2(fma(a.y, b.y, -a.x * b.x), fma(a.x, b.y, a.y * b.x));
}

// W lanes per row (W near the mean row length, so short rows do not leave
// most of a warp idle): every stored entry (i, j) gets -conj(mu_i x_j); the
// row's entries are read and written contiguously by its W lanes
template <int W>
__global__ void __launch_bounds__(256) k_outer_pattern(int n, const int *__restrict__ rowptr,
                                                       const int *__restrict__ col, const double2 *__restrict__ mu,
                                                       const double2 *__restrict__ x, double2 *__restrict__ g) {
    const int lane = threadIdx.x & (W - 1);
    const int groups = (gridDim.x * blockDim.x) / W;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / W; i < n; i += groups) {
        const double2 m = __ldg(mu + i);
        const int beg = __ldg(rowptr + i), end = __ldg(rowptr + i + 1);
        for (int k = beg + lane; k < end; k += W) {
            g[k] = neg_conj_mul(m, __ldg(x + __ldg(col + k)));
        }
    }
}

// The same product on the row blocks of the block-flat SpMV kernels (<= 32
// complete rows and <= 512 entries, or one longer row): one warp per block,
// lane l takes entries kb + l, kb + l + 32, ... so that every lane of every
// binary64 instruction is busy (the binary64 pipe is the limit here: four
// multiply-adds per entry) and the writes of g are coalesced.  The row of
// each entry comes from a per-warp table in shared memory (one byte per
// entry, filled by the lane that owns the row), so an entry costs one table
// read instead of a walk over the row pointers; a block with one row (the
// only kind longer than kFlatCap entries) needs no table.
constexpr int kOpThreads = 128;
constexpr int kOpGroup = 8;
__global__ void __launch_bounds__(kOpThreads) k_outer_flat(int nfblk, const int *__restrict__ fblk,
                                                           const int *__restrict__ fblk_k,
                                                           const int *__restrict__ rowptr,
                                                           const int *__restrict__ col,
                                                           const double2 *__restrict__ mu,
                                                           const double2 *__restrict__ x, double2 *__restrict__ g) {
    __shared__ int rps[kOpThreads / 32][33];
    __shared__ unsigned char rows_s[kOpThreads / 32][kFlatCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *rp = rps[w];
    unsigned char *rowof = rows_s[w];
    const int step = gridDim.x * (kOpThreads / 32);
    for (int b = blockIdx.x * (kOpThreads / 32) + w; b < nfblk; b += step) {
        const int r0 = __ldg(fblk + b), r1 = __ldg(fblk + b + 1);
        const int kb = __ldg(fblk_k + b), ke = __ldg(fblk_k + b + 1);
        const int nr = r1 - r0;
        if (lane < nr) rp[lane] = __ldg(rowptr + r0 + lane);
        if (lane == 0) rp[nr] = ke;
        __syncwarp();
        if (nr > 1) {   // (then ke - kb <= kFlatCap)
            if (lane < nr)
                for (int k = rp[lane]; k < rp[lane + 1]; ++k) rowof[k - kb] = (unsigned char)lane;
            __syncwarp();
        }
        // kOpGroup entries per lane at a time: their column loads, x gathers
        // and mu loads are all issued before the first product
        for (int k0 = kb + lane; k0 < ke; k0 += 32 * kOpGroup) {
            int c[kOpGroup];
            double2 xv[kOpGroup], m[kOpGroup];
#pragma unroll
            for (int u = 0; u < kOpGroup; ++u) {
                const int k = k0 + 32 * u;
                c[u] = k < ke ? __ldg(col + k) : -1;
            }
#pragma unroll
            for (int u = 0; u < kOpGroup; ++u) {   // mu by row: needs no column
                const int k = k0 + 32 * u;
                const int j = (nr > 1 && k < ke) ? rowof[k - kb] : 0;
                m[u] = k < ke ? __ldg(mu + r0 + j) : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < kOpGroup; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : make_double2(0.0, 0.0);
#pragma unroll
            for (int u = 0; u < kOpGroup; ++u) {
                if (c[u] < 0) continue;
                g[k0 + 32 * u] = neg_conj_mul(m[u], xv[u]);
            }
        }
        __syncwarp();
    }
}

// position of the diagonal entry of every row (-1 if absent)
__global__ void k_find_diag(int n, const int *__restrict__ rowptr, const int *__restrict__ col, int *__restrict__ pos) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int f = -1;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (col[k] == i) { f = k; break; }
        pos[i] = f;
    }
}

__global__ void k_set_diag(int n, const int *__restrict__ pos, const double2 *__restrict__ base, double2 c,
                           const double2 *__restrict__ theta, double2 *__restrict__ val) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double2 v = base[i];
        cmac(v, c, theta[i]);
        val[pos[i]] = v;
    }
}

__global__ void k_diag_grad(int n, const double2 *__restrict__ mu, const double2 *__restrict__ x, double2 c,
                            double2 *__restrict__ gt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // conj(c) (-conj(mu_i x_i)) = -conj(c mu_i x_i)
        gt[i] = neg_conj_mul(c, cmul(mu[i], x[i]));
    }
}

static hz_status ensure_diag(hz_mat *A, cudaStream_t s) {
    if (A->diag_pos) return HZ_OK;
    HZ_CUDA(cudaMalloc(&A->diag_pos, sizeof(int) * std::max(A->n, 1)));
    k_find_diag<<<std::max(1, std::min(4096, (A->n + 255) / 256)), 256, 0, s>>>(A->n, A->rowptr, A->col, A->diag_pos);
    HZ_CUDA(cudaGetLastError());
    std::vector<int> pos(A->n);
    HZ_CUDA(cudaMemcpyAsync(pos.data(), A->diag_pos, sizeof(int) * A->n, cudaMemcpyDeviceToHost, s));
    HZ_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < A->n; ++i)
        if (pos[i] < 0) {
            cudaFree(A->diag_pos);
            A->diag_pos = nullptr;
            set_error("hz_mat_set_diag: row " + std::to_string(i) + " stores no diagonal entry");
            return HZ_ERR_ARG;
        }
    return HZ_OK;
}

static int grid_for(int64_t n) {
    DevInfo d;
    if (dev_info(&d) != HZ_OK) return 1;
    return stream_grid(d, n, 256, 8);
}

}  // namespace hz

using namespace hz;

extern "C" HZ_API hz_status hz_outer_on_pattern(const hz_mat *A, const hz_z *d_mu, const hz_z *d_x,
                                                hz_z *d_gradval, void *stream) {
    HZ_CHECK(A, "hz_outer_on_pattern: null handle");
    if (A->n == 0 || A->nnz == 0) return HZ_OK;
    HZ_CHECK(d_mu && d_x && d_gradval, "hz_outer_on_pattern: null vector");
    if (A->fblk) {   // every handle has its row blocks; the row-group kernel stays for the rest
        DevInfo d;
        HZ_TRY(dev_info(&d));
        const int grid = (int)std::max<int64_t>(
            1, std::min<int64_t>((A->nfblk + kOpThreads / 32 - 1) / (kOpThreads / 32), (int64_t)d.num_sms * 16));
        k_outer_flat<<<grid, kOpThreads, 0, (cudaStream_t)stream>>>(A->nfblk, A->fblk, A->fblk_k, A->rowptr, A->col,
                                                                     (const double2 *)d_mu, (const double2 *)d_x,
                                                                     (double2 *)d_gradval);
        HZ_CUDA(cudaGetLastError());
        return HZ_OK;
    }
    int w = 2;
    while (w < 32 && w < A->mean_row) w *= 2;
    const int grid = grid_for((int64_t)A->n * w);
    auto launch = [&](auto kern) {
        kern<<<grid, 256, 0, (cudaStream_t)stream>>>(A->n, A->rowptr, A->col, (const double2 *)d_mu,
                                                      (const double2 *)d_x, (double2 *)d_gradval);
    };
    switch (w) {
        case 2: launch(k_outer_pattern<2>); break;
        case 4: launch(k_outer_pattern<4>); break;
        case 8: launch(k_outer_pattern<8>); break;
        case 16: launch(k_outer_pattern<16>); break;
        default: launch(k_outer_pattern<32>); break;
    }
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_mat_set_diag(hz_mat *A, const hz_z *d_base, hz_z scale, const hz_z *d_theta,
                                            void *stream) {
    HZ_CHECK(A, "hz_mat_set_diag: null handle");
    if (A->n == 0) return HZ_OK;
    HZ_CHECK(d_base && d_theta, "hz_mat_set_diag: null vector");
    cudaStream_t s = (cudaStream_t)stream;
    HZ_TRY(ensure_diag(A, s));
    k_set_diag<<<grid_for(A->n), 256, 0, s>>>(A->n, A->diag_pos, (const double2 *)d_base,
                                               make_double2(scale.re, scale.im), (const double2 *)d_theta, A->val);
    HZ_CUDA(cudaGetLastError());
    return hz_mat_refresh_values(A, stream);
}

extern "C" HZ_API hz_status hz_diag_grad(const hz_mat *A, const hz_z *d_mu, const hz_z *d_x, hz_z scale,
                                         hz_z *d_grad_theta, void *stream) {
    HZ_CHECK(A, "hz_diag_grad: null handle");
    if (A->n == 0) return HZ_OK;
    HZ_CHECK(d_mu && d_x && d_grad_theta, "hz_diag_grad: null vector");
    k_diag_grad<<<grid_for(A->n), 256, 0, (cudaStream_t)stream>>>(
        A->n, (const double2 *)d_mu, (const double2 *)d_x, make_double2(scale.re, scale.im), (double2 *)d_grad_theta);
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}
