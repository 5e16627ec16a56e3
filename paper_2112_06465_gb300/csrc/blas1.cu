// blas1.cu -- complex128 BLAS-1 operations of the paper's Section 5:
// assign, scale, Zaxpy, dot product (conjugated and not) and L2 norm.
//
// Streaming kernels: each block walks tiles of kUnroll * blockDim elements
// (16-byte loads per element), grid-stride over a whole number of waves.
// Reductions are single pass: block partial sums plus a last-block fold in a
// fixed order, so results are bitwise reproducible for a given launch shape.
// Scalars (alpha, results) are device pointers: no host round trip.
#include "hz_internal.cuh"

namespace hz {

constexpr int kBlasBlock = 256;
constexpr int kUnroll = 4;

template <class F>
__device__ __forceinline__ void for_tiles(int64_t n, F f) {
    const int64_t tile = (int64_t)kUnroll * blockDim.x;
    for (int64_t base = blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t i = base + u * blockDim.x + threadIdx.x;
            if (i < n) f(i);
        }
    }
}

__global__ void __launch_bounds__(kBlasBlock) k_zaxpy(int64_t n, const double2 *__restrict__ alpha,
                                                      const double2 *__restrict__ x, double2 *__restrict__ y) {
    const double2 a = *alpha;
    for_tiles(n, [&](int64_t i) {
        double2 yi = y[i];
        cmac(yi, a, x[i]);
        y[i] = yi;
    });
}

__global__ void __launch_bounds__(kBlasBlock) k_zscal(int64_t n, const double2 *__restrict__ alpha,
                                                      double2 *__restrict__ x) {
    const double2 a = *alpha;
    for_tiles(n, [&](int64_t i) { x[i] = cmul(a, x[i]); });
}

__global__ void __launch_bounds__(kBlasBlock) k_zcopy(int64_t n, const double2 *__restrict__ x,
                                                      double2 *__restrict__ y) {
    for_tiles(n, [&](int64_t i) { y[i] = x[i]; });
}

__global__ void __launch_bounds__(kBlasBlock) k_zconj(int64_t n, const double2 *x, double2 *y) {
    for_tiles(n, [&](int64_t i) { y[i] = cconj(x[i]); });
}

template <bool CONJ>
__global__ void __launch_bounds__(kBlasBlock) k_zdot(int64_t n, const double2 *__restrict__ x,
                                                     const double2 *__restrict__ y, double2 *__restrict__ out,
                                                     RedScratch red) {
    double2 acc = make_double2(0.0, 0.0);
    for_tiles(n, [&](int64_t i) {
        if (CONJ) cmac_conj(acc, x[i], y[i]);
        else cmac(acc, x[i], y[i]);
    });
    double v[2] = {acc.x, acc.y}, tot[2];
    if (grid_reduce_last<double, 2>(v, red, tot) && threadIdx.x == 0) *out = make_double2(tot[0], tot[1]);
}

__global__ void __launch_bounds__(kBlasBlock) k_dznrm2(int64_t n, const double2 *__restrict__ x,
                                                       double *__restrict__ out, RedScratch red) {
    double acc = 0.0;
    for_tiles(n, [&](int64_t i) {
        const double2 a = x[i];
        acc = fma(a.x, a.x, acc);
        acc = fma(a.y, a.y, acc);
    });
    double v[1] = {acc}, tot[1];
    if (grid_reduce_last<double, 1>(v, red, tot) && threadIdx.x == 0) *out = sqrt(tot[0]);
}

static int blas_grid(int64_t n) {
    DevInfo d;
    if (dev_info(&d) != HZ_OK) return 1;
    return stream_grid(d, (n + kUnroll - 1) / kUnroll, kBlasBlock, 8);
}

}  // namespace hz

using namespace hz;

#define HZ_VEC_ARGS(n, p) HZ_CHECK((n) >= 0, "negative length"); HZ_CHECK((n) == 0 || (p), "null vector")

extern "C" HZ_API hz_status hz_zaxpy(int64_t n, const hz_z *d_alpha, const hz_z *d_x, hz_z *d_y, void *stream) {
    HZ_VEC_ARGS(n, d_x && d_y && d_alpha);
    if (n == 0) return HZ_OK;
    k_zaxpy<<<blas_grid(n), kBlasBlock, 0, (cudaStream_t)stream>>>(n, (const double2 *)d_alpha,
                                                                  (const double2 *)d_x, (double2 *)d_y);
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_zscal(int64_t n, const hz_z *d_alpha, hz_z *d_x, void *stream) {
    HZ_VEC_ARGS(n, d_x && d_alpha);
    if (n == 0) return HZ_OK;
    k_zscal<<<blas_grid(n), kBlasBlock, 0, (cudaStream_t)stream>>>(n, (const double2 *)d_alpha, (double2 *)d_x);
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_zcopy(int64_t n, const hz_z *d_x, hz_z *d_y, void *stream) {
    HZ_VEC_ARGS(n, d_x && d_y);
    if (n == 0) return HZ_OK;
    k_zcopy<<<blas_grid(n), kBlasBlock, 0, (cudaStream_t)stream>>>(n, (const double2 *)d_x, (double2 *)d_y);
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_zconj(int64_t n, const hz_z *d_x, hz_z *d_y, void *stream) {
    HZ_VEC_ARGS(n, d_x && d_y);
    if (n == 0) return HZ_OK;
    k_zconj<<<blas_grid(n), kBlasBlock, 0, (cudaStream_t)stream>>>(n, (const double2 *)d_x, (double2 *)d_y);
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}

template <bool CONJ>
static hz_status zdot(int64_t n, const hz_z *d_x, const hz_z *d_y, hz_z *d_result, void *stream) {
    HZ_CHECK(n >= 0, "negative length");
    HZ_CHECK(d_result, "null result");
    HZ_CHECK(n == 0 || (d_x && d_y), "null vector");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        HZ_CUDA(cudaMemsetAsync(d_result, 0, sizeof(hz_z), s));
        return HZ_OK;
    }
    RedScratch red;
    HZ_TRY(get_scratch(s, &red));
    k_zdot<CONJ><<<blas_grid(n), kBlasBlock, 0, s>>>(n, (const double2 *)d_x, (const double2 *)d_y,
                                                     (double2 *)d_result, red);
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_zdotc(int64_t n, const hz_z *d_x, const hz_z *d_y, hz_z *d_result, void *stream) {
    return zdot<true>(n, d_x, d_y, d_result, stream);
}

extern "C" HZ_API hz_status hz_zdotu(int64_t n, const hz_z *d_x, const hz_z *d_y, hz_z *d_result, void *stream) {
    return zdot<false>(n, d_x, d_y, d_result, stream);
}

extern "C" HZ_API hz_status hz_dznrm2(int64_t n, const hz_z *d_x, double *d_result, void *stream) {
    HZ_CHECK(n >= 0, "negative length");
    HZ_CHECK(d_result, "null result");
    HZ_CHECK(n == 0 || d_x, "null vector");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        HZ_CUDA(cudaMemsetAsync(d_result, 0, sizeof(double), s));
        return HZ_OK;
    }
    RedScratch red;
    HZ_TRY(get_scratch(s, &red));
    k_dznrm2<<<blas_grid(n), kBlasBlock, 0, s>>>(n, (const double2 *)d_x, d_result, red);
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}
