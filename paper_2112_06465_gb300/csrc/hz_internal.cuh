// hz_internal.cuh -- shared device helpers and internal structures of libhz.
//
// Complex values are double2 / float2 (real in .x, imaginary in .y), the
// two-contiguous-reals layout of the paper's Section 4.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/hz.h"

namespace hz {

// ---------------------------------------------------------------------------
// error plumbing
void set_error(const std::string &msg);
hz_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define HZ_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t _e = (call);                                                   \
        if (_e != cudaSuccess) return ::hz::cuda_fail(_e, #call, __FILE__, __LINE__); \
    } while (0)

#define HZ_CHECK(cond, msg)                                                        \
    do {                                                                           \
        if (!(cond)) { ::hz::set_error(msg); return HZ_ERR_ARG; }                   \
    } while (0)

#define HZ_TRY(call)                                                               \
    do {                                                                           \
        hz_status _s = (call);                                                     \
        if (_s != HZ_OK) return _s;                                                \
    } while (0)

// ---------------------------------------------------------------------------
// device properties (cached per device)
struct DevInfo {
    int device = -1;
    int num_sms = 0;
    int max_threads_per_sm = 0;
};
hz_status dev_info(DevInfo *out);

// ---------------------------------------------------------------------------
// complex arithmetic (4 fused multiply-adds per complex multiply-accumulate)
template <class T> struct Cplx;
template <> struct Cplx<double2> { using R = double; };
template <> struct Cplx<float2> { using R = float; };

__device__ __forceinline__ double2 cmk(double r, double i) { return make_double2(r, i); }
__device__ __forceinline__ float2 cmk(float r, float i) { return make_float2(r, i); }

template <class T> __device__ __forceinline__ T czero() { T z; z.x = 0; z.y = 0; return z; }

template <class T> __device__ __forceinline__ T cadd(T a, T b) { T r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <class T> __device__ __forceinline__ T csub(T a, T b) { T r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <class T> __device__ __forceinline__ T cconj(T a) { T r; r.x = a.x; r.y = -a.y; return r; }
template <class T> __device__ __forceinline__ T cmul(T a, T b) {
    T r;
    r.x = fma(a.x, b.x, -a.y * b.y);
    r.y = fma(a.x, b.y, a.y * b.x);
    return r;
}
// acc += a * b
template <class T> __device__ __forceinline__ void cmac(T &acc, T a, T b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <class T> __device__ __forceinline__ void cmac_conj(T &acc, T a, T b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
// a / b as a * conj(b) / |b|^2 (operands here are O(1) Krylov scalars)
template <class T> __device__ __forceinline__ T cdiv(T a, T b) {
    auto d = b.x * b.x + b.y * b.y;
    T r;
    r.x = (a.x * b.x + a.y * b.y) / d;
    r.y = (a.y * b.x - a.x * b.y) / d;
    return r;
}
template <class T> __device__ __forceinline__ bool cis_zero(T a) { return a.x == 0 && a.y == 0; }

__device__ __forceinline__ float2 to_c64(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_c128(float2 a) { return make_double2((double)a.x, (double)a.y); }

// ---------------------------------------------------------------------------
// global loads with cache hints (PTX ISA: createpolicy + ld ... L2::cache_hint).
// The matrix is read once per product, so it is streamed with an L2
// evict-first policy and kept out of L1; the gathered vector uses the default
// cached path.  The asm statements are not volatile: they read data that no
// kernel writes while it runs, so the compiler may schedule them freely.
__device__ __forceinline__ uint64_t pol_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ double2 ld_stream(const double2 *ptr) {
    double2 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
        : "=d"(v.x), "=d"(v.y) : "l"(ptr), "l"(pol_evict_first()));
    return v;
}
__device__ __forceinline__ float2 ld_stream(const float2 *ptr) {
    float2 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
        : "=f"(v.x), "=f"(v.y) : "l"(ptr), "l"(pol_evict_first()));
    return v;
}
__device__ __forceinline__ int ld_stream(const int *ptr) {
    int v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
        : "=r"(v) : "l"(ptr), "l"(pol_evict_first()));
    return v;
}
__device__ __forceinline__ float4 ld_stream(const float4 *ptr) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(ptr), "l"(pol_evict_first()));
    return v;
}
// the same loads with a policy created once by the caller
__device__ __forceinline__ float4 ld_stream(const float4 *ptr, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ int ld_stream(const int *ptr, uint64_t pol) {
    int v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}

// ---------------------------------------------------------------------------
// double-float ("ff") arithmetic on the binary32 pipes.
//
// GB300 executes binary64 FMAs at 1/58 of the binary32 rate (about 2 per SM
// per clock), which caps a binary64 complex SpMV near 45% of HBM bandwidth.
// The ff path represents a binary64 value d as hi + lo with
// hi = fl32(d), lo = fl32(d - hi) (48 significant bits; relative
// representation error <= 2^-48 for |d| in [2^-100, 2^100]) and forms
// products and sums with the classical error-free transformations:
//   TwoProd (Dekker, via FMA): p = fl(a*b), e = fma(a, b, -p), a*b = p + e
//   TwoSum (Knuth):            s = fl(a+b), e = (a - (s - z)) + (b - z), z = s - a
// The explicit __f*_rn intrinsics keep the compiler from contracting or
// reassociating these sequences.
//
// Conversions between binary64 and binary32 run on GB300's slow conversion
// path (about 276 G conversions/s for the whole GPU, measured), so the split
// and the widening below work on the bit patterns with integer operations
// and fall back to the conversion instructions only outside the range where
// the bit formula holds.  Both give the same bits as the conversions.
//
// split: hi = RN_32(d), lo = RN_32(d - hi).  With d = (-1)^s * m * 2^(E-52),
// m a 53-bit integer, hi takes the top 24 bits of m rounded to nearest even
// and lo is the signed 29-bit remainder times 2^(E-52); for -74 <= E <= 126
// both are normal binary32 numbers (or lo = 0) and the power-of-two scaling
// is exact.
__device__ __forceinline__ void split_d(double d, float &hi, float &lo) {
    const unsigned hw = (unsigned)__double2hiint(d), lw = (unsigned)__double2loint(d);
    const int E = (int)((hw >> 20) & 0x7ffu) - 1023;
    if (((hw & 0x7fffffffu) | lw) == 0u) {   // signed zero
        hi = __uint_as_float(hw & 0x80000000u);
        lo = 0.f;
        return;
    }
    if (E >= -74 && E <= 126) {
        unsigned top = (((hw & 0xfffffu) | 0x100000u) << 3) | (lw >> 29);   // 24 bits
        int low = (int)(lw & 0x1fffffffu);                                 // 29 bits
        constexpr int kHalf = 1 << 28;
        if (low > kHalf || (low == kHalf && (top & 1u))) {
            top += 1u;   // a carry into bit 24 moves hi to the next binade below
            low -= 1 << 29;
        }
        hi = __uint_as_float((hw & 0x80000000u) | (((unsigned)(E + 127) << 23) + (top - 0x800000u)));
        if (hw & 0x80000000u) low = -low;
        lo = __fmul_rn(__int2float_rn(low), __uint_as_float((unsigned)(E - 52 + 127) << 23));
        return;
    }
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
}

// exact binary32 -> binary64 widening (normal numbers by bits, others by conversion)
__device__ __forceinline__ double widen_d(float f) {
    const unsigned u = __float_as_uint(f), ex = (u >> 23) & 0xffu;
    if (ex - 1u < 254u)
        return __hiloint2double((int)((u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7fffffu) >> 3)),
                                (int)(u << 29));
    return (double)f;
}

// binary exponents of the values for which split_d keeps all 48 bits
// (both parts normal binary32 numbers, no overflow of the products with an
// O(1) vector)
constexpr int kFFMinExp = -100;
constexpr int kFFMaxExp = 100;

// largest n and nnz of a handle: the kernels form int32 indices up to a few
// thousand past a row or entry count (a group, a row block, a lane step)
constexpr int32_t kMaxCsrSize = 0x7fffffff - 4096;

__device__ __forceinline__ float4 split_ff(double2 d) {
    float4 r;
    split_d(d.x, r.x, r.y);
    split_d(d.y, r.z, r.w);
    return r;
}

// ff pair (hi, lo) rounded once to binary64
__device__ __forceinline__ double join_d(float hi, float lo) { return widen_d(hi) + widen_d(lo); }

// (s, c) += p, with the rounding error of s + p carried into c
__device__ __forceinline__ void ff_acc(float &s, float &c, float p) {
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, e);
}

// (s, c) += (ah + al) * (xh + xl); the al*xl term (2^-48 relative) is dropped
__device__ __forceinline__ void ff_mac(float &s, float &c, float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);
    e = __fmaf_rn(ah, xl, e);
    e = __fmaf_rn(al, xh, e);
    ff_acc(s, c, p);
    c = __fadd_rn(c, e);
}

// (s, c) = (ah + al) * (xh + xl): ff_mac into a zero accumulator with the
// exact steps 0 + p = p and 0 + e = e left out (the same values; only the
// sign of a zero can differ)
__device__ __forceinline__ void ff_mul(float &s, float &c, float ah, float al, float xh, float xl) {
    s = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -s);
    e = __fmaf_rn(ah, xl, e);
    c = __fmaf_rn(al, xh, e);
}

// ---------------------------------------------------------------------------
// packed binary32 pairs (PTX .f32x2 on sm_100 and later): one instruction
// applies the same IEEE round-to-nearest operation to two lanes, so the
// error-free transformations above stay exact lane by lane while the real
// and imaginary halves of a complex double-float sum share instructions.
// GB300 retires these at the scalar lane rate with half the issue slots.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// TwoSum on both lanes: s + p = t + e exactly
__device__ __forceinline__ void two_sum2(f32x2 s, f32x2 p, f32x2 &t, f32x2 &e) {
    t = add2(s, p);
    const f32x2 z = sub2(t, s);
    e = add2(sub2(s, sub2(t, z)), sub2(p, z));
}

// complex double-float product a * x for a, x in the (re_hi, re_lo, im_hi,
// im_lo) layout.  The four real products are formed by ff_mul; the pairs
// (re, im) are then summed with one packed TwoSum.  Returned as
// (re_hi, im_hi, re_lo, im_lo): the hi pair and the pair of their error
// sums (not renormalised).  The dropped lo*lo terms are 2^-48 relative.
__device__ __forceinline__ float4 ff_cprod(float4 a, float4 x) {
    float prr, err, pii, eii, pri, eri, pir, eir;
    ff_mul(prr, err, a.x, a.y, x.x, x.y);
    ff_mul(pii, eii, -a.z, -a.w, x.z, x.w);
    ff_mul(pri, eri, a.x, a.y, x.z, x.w);
    ff_mul(pir, eir, a.z, a.w, x.x, x.y);
    f32x2 t, e;
    two_sum2(pk2(prr, pri), pk2(pii, pir), t, e);
    const f32x2 c = add2(add2(pk2(err, eri), pk2(eii, eir)), e);
    float4 r;
    upk2(t, r.x, r.y);
    upk2(c, r.z, r.w);
    return r;
}

// (S, C) += q for a product q in the layout ff_cprod returns
__device__ __forceinline__ void ff_cacc(f32x2 &S, f32x2 &C, float4 q) {
    f32x2 t, e;
    two_sum2(S, pk2(q.x, q.y), t, e);
    S = t;
    C = add2(C, add2(e, pk2(q.z, q.w)));
}

// ---------------------------------------------------------------------------
// programmatic dependent launch (PTX griddepcontrol).  A kernel launched with
// the programmatic-serialization attribute may start while its predecessor
// is still draining; pdl_wait() blocks until the predecessor grid has
// completed and its memory is visible, so every kernel calls it before its
// first read of data another kernel produced.  pdl_release() lets the next
// kernel in the stream begin launching.  Both are no-ops without the
// attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// host: launch `k` with the programmatic-serialization attribute set (the
// launch may overlap the tail of the previous kernel on the stream)
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, ((KArgs)args)...);
}

// ---------------------------------------------------------------------------
// bulk asynchronous copies (the TMA unit's untiled cp.async.bulk) into
// shared memory, completed on an mbarrier by transaction count.  Source and
// destination must be 16-byte aligned and the size a multiple of 16 bytes.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make initialised barriers visible to the async proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// arrive once and add `bytes` to the transactions the current phase waits for
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for phase `parity` of the barrier to complete, giving up after
// about `limit_ns` of wall time; returns false on expiry
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}
// order this thread's earlier shared-memory accesses before later
// async-proxy (bulk copy) writes to the same locations
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// deterministic single-pass grid reduction.
//
// Every block reduces its NV per-thread values (warp shuffles, then shared
// memory), writes them to partials[blockIdx.x * NV + j], and increments a
// completion counter.  The block that arrives last sums the partials in a
// fixed order (thread t takes blocks t, t + blockDim, ...) and returns true
// with the totals in tot[] (valid in thread 0).  For a fixed grid the result
// is bitwise reproducible.  The counter is reset by the last block.
struct RedScratch {
    void *partials;            // >= max_blocks * NV * sizeof(R)
    unsigned int *counter;     // one counter, zero between kernels
};

// Warp sums of NV values per lane.  For 2..4 values the first one or two
// butterfly levels split the values between the two halves of each exchange
// (each lane keeps the half it adds and sends the other), so a warp does 5
// (NV = 2) or 6 (NV = 3, 4) additions per lane instead of 5 NV; the total of
// value q ends in lane q * (32 / P), P = NV rounded up to a power of two.
// (On GB300 a binary64 addition occupies the binary64 pipe for a whole warp
// instruction, so the solver's three-value reductions save nine of fifteen.)
template <class R, int NV>
__device__ __forceinline__ void warp_sum_split(R (&v)[NV], R &out) {
    const int lane = threadIdx.x & 31;
    if constexpr (NV == 1) {
        out = v[0];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) out += __shfl_xor_sync(0xffffffffu, out, off);
    } else if constexpr (NV == 2) {
        const bool hi = lane & 16;
        R t = (hi ? v[1] : v[0]) + __shfl_xor_sync(0xffffffffu, hi ? v[0] : v[1], 16);
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        out = t;
    } else {
        static_assert(NV <= 4, "warp_sum_split takes at most four values");
        R w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = q < NV ? v[q] : R(0);
        const bool h16 = lane & 16, h8 = lane & 8;
        // level 16: keep values {0,1} (low half) or {2,3} (high half)
        const R k0 = (h16 ? w[2] : w[0]) + __shfl_xor_sync(0xffffffffu, h16 ? w[0] : w[2], 16);
        const R k1 = (h16 ? w[3] : w[1]) + __shfl_xor_sync(0xffffffffu, h16 ? w[1] : w[3], 16);
        // level 8: keep the first or the second of the two
        R t = (h8 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        out = t;
    }
}

template <class R, int NV>
__device__ __forceinline__ void block_sum(R (&v)[NV], R (*sh)[NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    if constexpr (NV <= 4) {
        R t;
        warp_sum_split<R, NV>(v, t);
        constexpr int P = NV == 1 ? 1 : NV == 2 ? 2 : 4;
        const int q = lane / (32 / P);
        if (q < NV && lane % (32 / P) == 0) sh[warp][q] = t;
    } else {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
        }
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < NV; ++j) sh[warp][j] = v[j];
        }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            R t = lane < nwarps ? sh[lane][j] : R(0);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            v[j] = t;
        }
    }
    __syncthreads();
}

template <class R, int NV>
__device__ __forceinline__ bool grid_reduce_last(R (&v)[NV], RedScratch red, R (&tot)[NV]) {
    __shared__ R sh[32][NV];
    __shared__ int am_last;
    R *partials = reinterpret_cast<R *>(red.partials);
    block_sum<R, NV>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) partials[blockIdx.x * NV + j] = v[j];
        __threadfence();
        unsigned int t = atomicAdd(red.counter, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    R acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = R(0);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] += __ldcg(&partials[b * NV + j]);
    }
    block_sum<R, NV>(acc, sh);
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = acc[j];
    if (threadIdx.x == 0) *red.counter = 0u;
    return true;
}

// ---------------------------------------------------------------------------
// per-(device, stream) reduction scratch
constexpr int kMaxRedBlocks = 4096;
constexpr int kMaxRedValues = 8;
hz_status get_scratch(cudaStream_t s, RedScratch *out);

// grid size for streaming kernels: a whole number of waves over the SMs
int stream_grid(const DevInfo &d, int64_t work_items, int block, int blocks_per_sm);

}  // namespace hz

// ---------------------------------------------------------------------------
// SpMV kinds that run in double-float arithmetic on the split x
inline bool is_ff_kind(int k) {
    return k == HZ_SPMV_FF || k == HZ_SPMV_SELL_FF || k == HZ_SPMV_FF_FLAT || k == HZ_SPMV_FF_TMA;
}

// matrix handle
struct hz_mat {
    int device = -1;
    int32_t n = 0, nnz = 0;
    const int32_t *rowptr = nullptr;   // 0-based, device
    const int32_t *col = nullptr;
    double2 *val = nullptr;            // caller's values (writable through set_diag)
    int32_t *own_rowptr = nullptr;     // owned 0-based copies (index_base 1)
    int32_t *own_col = nullptr;
    // row statistics
    int32_t max_row = 0, min_row = 0;
    double mean_row = 0;
    // SpMV selection
    int spmv_kind = HZ_SPMV_CSR_VECTOR;
    int group = 4;
    // SELL-C-sigma copy (C = 32)
    int32_t sell_nchunks = 0;
    int32_t sell_sigma = 0;
    int64_t sell_slots = 0;
    int32_t *sell_chunk_off = nullptr;   // [nchunks+1] slot offsets
    int32_t *sell_chunk_w = nullptr;     // [nchunks] chunk widths
    int32_t *sell_perm = nullptr;        // [nchunks*32] original row of each lane (-1 pad)
    int32_t *sell_col = nullptr;         // [slots] column (-1 = padding)
    int32_t *sell_src = nullptr;         // [slots] CSR position of the slot (-1 = padding)
    double2 *sell_val = nullptr;         // [slots]
    float2 *sell_val32 = nullptr;        // [slots] complex64 copy, if c64
    float4 *sell_vff = nullptr;          // [slots] double-float split, if SELL and FF
    // complex64 copy
    float2 *val32 = nullptr;
    // double-float split of the values (hi_re, lo_re, hi_im, lo_im) and the
    // handle's x scratch for hz_zspmv on that path
    float4 *val_ff = nullptr;
    float4 *x_ff = nullptr;
    bool ff_range_ok = false;   // every value lies where the split keeps 48 bits
    // row blocks of the block-flat double-float kernel (complete rows)
    int32_t nfblk = 0;
    int32_t *fblk = nullptr;
    int32_t *fblk_k = nullptr;   // rowptr[fblk[b]] for b = 0 .. nfblk
    // packed binary64 stream of the same row blocks (HZ_SPMV_FLAT64P): block
    // b owns slots [pk_base[b], pk_base[b+1]), 32 per lane step u, slot
    // pk_base[b] + 32 u + l holding entry u of lane l's run (padding past
    // the run's end); groups of kD64Group steps, group pk_gbase[b] + g of
    // block b keeping its imaginary parts at pk_im + pk_gim[..] (same slot
    // order) or, with pk_gim < 0, none (every imaginary part is zero)
    int64_t pk_slots = 0;
    int32_t pk_groups = 0;
    int32_t *pk_base = nullptr;    // [nfblk + 1]
    int32_t *pk_gbase = nullptr;   // [nfblk + 1]
    int32_t *pk_gim = nullptr;     // [pk_groups]
    int32_t *pk_col = nullptr;     // [pk_slots]
    double *pk_re = nullptr;       // [pk_slots]
    double *pk_im = nullptr;       // [pk_slots] (complex groups only use it)
    int32_t nfblk_t = 0;       // the same for the bulk-copy kernel's smaller chunks
    int32_t *fblk_t = nullptr;
    // owned copy of col, 16-byte aligned and padded by 8 entries, that the
    // bulk-copy kernel reads in 16-byte units; and its device fault word
    // (nonzero once a bounded wait on a bulk copy expired)
    int32_t *col_pad = nullptr;
    int *fault = nullptr;
    // diagonal positions (for set_diag), built on demand
    int32_t *diag_pos = nullptr;
    // solver state (one per mode, and the BiCGStab(l) solver), created on first solve
    void *solver[2] = {nullptr, nullptr};
    void *solver_bl = nullptr;
    void *solver_tq = nullptr;
    // Jacobi right preconditioning: the column-scaled operator A D^-1 as a
    // handle of its own (borrowing rowptr/col), its values, and D, D^-1
    hz_mat *jac = nullptr;
    double2 *jac_val = nullptr;
    double2 *jac_d = nullptr;
    double2 *jac_dinv = nullptr;
};

namespace hz {
hz_status ensure_jacobi(hz_mat *A, cudaStream_t s);   // build A->jac on first use
void free_jacobi(hz_mat *A);                          // drop it (values changed, destroy)
}  // namespace hz
