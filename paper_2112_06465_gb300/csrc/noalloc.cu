// noalloc.cu -- hz_zdotc_noalloc: the conjugated dot product of hz_zdotc
// with its reduction scratch held in a fixed device array instead of memory
// the library allocates, for callers that must not see any device
// allocation (see include/hz.h for who they are and the limits).
//
// Scheme: the vector is cut into fixed tiles of kNaTile elements, one block
// per tile; each block writes its tile's partial sum into the array and
// bumps a completion counter, and the block that finishes last folds the
// partials in tile order.  Because the tiling does not depend on the GPU's
// SM count, the result is bitwise reproducible on any device.
#include <mutex>

#include "hz_internal.cuh"

namespace hz {
namespace {

constexpr int kNaBlock = 256;
constexpr int kNaTile = 4096;                                    // elements per tile
constexpr int kNaMaxTiles = 65536;                               // capacity of the array
constexpr int64_t kNaMaxN = (int64_t)kNaTile * kNaMaxTiles;      // 2^28 elements

struct NaScratch {
    double partials[2 * kNaMaxTiles];   // (re, im) of every tile: 1 MiB
    unsigned int counter;               // tiles finished; must be 0 at launch
};

// One copy per device that loads this library, alive until process exit.
static __device__ __align__(256) NaScratch g_na_scratch;

// Host side: the device address of g_na_scratch, looked up once per device
// (host code cannot use the symbol's name as an address).
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
NaScratch *g_na_addr[kNaMaxDevices] = {};

__global__ void __launch_bounds__(kNaBlock) k_zdotc_na(int64_t n, const double2 *__restrict__ x,
                                                       const double2 *__restrict__ y, double2 *__restrict__ out,
                                                       NaScratch *sc) {
    __shared__ double sh[32][2];
    __shared__ int am_last;
    const int64_t base = (int64_t)blockIdx.x * kNaTile;
    double v[2] = {0.0, 0.0};
    for (int j = threadIdx.x; j < kNaTile; j += kNaBlock) {
        const int64_t i = base + j;
        if (i < n) {
            const double2 a = x[i], b = y[i];
            v[0] = fma(a.x, b.x, v[0]); v[0] = fma(a.y, b.y, v[0]);
            v[1] = fma(a.x, b.y, v[1]); v[1] = fma(-a.y, b.x, v[1]);
        }
    }
    block_sum<double, 2>(v, sh);
    if (threadIdx.x == 0) {
        sc->partials[2 * blockIdx.x] = v[0];
        sc->partials[2 * blockIdx.x + 1] = v[1];
        __threadfence();
        am_last = atomicAdd(&sc->counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double t[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kNaBlock) {
        t[0] += __ldcg(&sc->partials[2 * b]);
        t[1] += __ldcg(&sc->partials[2 * b + 1]);
    }
    block_sum<double, 2>(t, sh);
    if (threadIdx.x == 0) {
        *out = make_double2(t[0], t[1]);
        sc->counter = 0u;
    }
}

// The array's device address on the current device; the first call on a
// device does the lookup (with that device current).
hz_status na_scratch(NaScratch **out) {
    int dev = 0;
    HZ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("hz_zdotc_noalloc: device ordinal out of range");
        return HZ_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        NaScratch *p = nullptr;
        HZ_CUDA(cudaGetSymbolAddress((void **)&p, g_na_scratch));
        g_na_addr[dev] = p;
    }
    *out = g_na_addr[dev];
    return HZ_OK;
}

}  // namespace
}  // namespace hz

using namespace hz;

extern "C" HZ_API hz_status hz_zdotc_noalloc(int64_t n, const hz_z *d_x, const hz_z *d_y, hz_z *d_result,
                                             void *stream) {
    HZ_CHECK(n >= 0, "hz_zdotc_noalloc: negative length");
    HZ_CHECK(n <= kNaMaxN, "hz_zdotc_noalloc: n exceeds the fixed scratch capacity of 2^28 elements");
    HZ_CHECK(d_result, "hz_zdotc_noalloc: null result");
    HZ_CHECK(n == 0 || (d_x && d_y), "hz_zdotc_noalloc: null vector");
    cudaStream_t s = (cudaStream_t)stream;
    NaScratch *sc = nullptr;
    HZ_TRY(na_scratch(&sc));
    if (n == 0) {
        HZ_CUDA(cudaMemsetAsync(d_result, 0, sizeof(hz_z), s));
        return HZ_OK;
    }
    // the completion counter must start at zero: clear it on this stream
    HZ_CUDA(cudaMemsetAsync(&sc->counter, 0, sizeof(unsigned int), s));
    const int tiles = (int)((n + kNaTile - 1) / kNaTile);
    k_zdotc_na<<<tiles, kNaBlock, 0, s>>>(n, (const double2 *)d_x, (const double2 *)d_y, (double2 *)d_result, sc);
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}
