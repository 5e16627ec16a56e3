// arith.cuh -- element arithmetic of the Krylov vector kernels, for three
// vector formats:
//   double2  complex128, binary64 FMAs (the reference arithmetic)
//   float2   complex64 with binary32 sums (inner solve of the mixed method)
//   float4   complex128 held as double-float (re_hi, re_lo, im_hi, im_lo),
//            every operation an error-free-transformation sequence on the
//            binary32 pipes (the GB300 fast path: binary64 FMAs run at
//            1/58 of the binary32 rate on this part)
//
// Ar<V> gives, for vector element type V:
//   St   type of the Krylov scalars kept in device state (alpha, omega, ...)
//   S    the scalar as the vector kernels use it
//   R    type of the grid reductions (block partials, totals)
//   Acc  per-thread accumulator of one real sum
// and the operations the BiCGStab kernels need.
#pragma once

#include <type_traits>

#include "hz_internal.cuh"

namespace hz {

template <class V> struct Ar;

// ------------------------------------------------------------------ binary64
template <> struct Ar<double2> {
    using V = double2; using St = double2; using S = double2; using R = double; using Acc = double;
    static constexpr bool kFF = false;
    __device__ static S scal(St a) { return a; }
    __device__ static V zero() { return make_double2(0.0, 0.0); }
    __device__ static V from_c128(double2 a) { return a; }
    __device__ static double2 to_c128(V a) { return a; }
    // a * s for a power of two s (exact)
    __device__ static V pow2(V a, double s) { return make_double2(a.x * s, a.y * s); }
    // y + a x
    __device__ static V axpy(V y, S a, V x) { cmac(y, a, x); return y; }
    // y - a x
    __device__ static V axmy(V y, S a, V x) {
        y.x = fma(-a.x, x.x, y.x); y.x = fma(a.y, x.y, y.x);
        y.y = fma(-a.x, x.y, y.y); y.y = fma(-a.y, x.x, y.y);
        return y;
    }
    __device__ static V sub(V a, V b) { return make_double2(a.x - b.x, a.y - b.y); }
    __device__ static V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
    __device__ static void acc_zero(Acc &a) { a = 0.0; }
    // (re, im) += conj(a) b
    __device__ static void dotc(Acc &re, Acc &im, V a, V b) {
        re = fma(a.x, b.x, re); re = fma(a.y, b.y, re);
        im = fma(a.x, b.y, im); im = fma(-a.y, b.x, im);
    }
    __device__ static void nrm2(Acc &s, V a) { s = fma(a.x, a.x, s); s = fma(a.y, a.y, s); }
    __device__ static R total(Acc a) { return a; }
};

// ------------------------------------------------------------------ binary32
template <> struct Ar<float2> {
    using V = float2; using St = float2; using S = float2; using R = float; using Acc = float;
    static constexpr bool kFF = false;
    __device__ static S scal(St a) { return a; }
    __device__ static V zero() { return make_float2(0.f, 0.f); }
    __device__ static V axpy(V y, S a, V x) { cmac(y, a, x); return y; }
    __device__ static V axmy(V y, S a, V x) {
        y.x = fmaf(-a.x, x.x, y.x); y.x = fmaf(a.y, x.y, y.x);
        y.y = fmaf(-a.x, x.y, y.y); y.y = fmaf(-a.y, x.x, y.y);
        return y;
    }
    __device__ static V sub(V a, V b) { return make_float2(a.x - b.x, a.y - b.y); }
    __device__ static V add(V a, V b) { return make_float2(a.x + b.x, a.y + b.y); }
    __device__ static void acc_zero(Acc &a) { a = 0.f; }
    __device__ static void dotc(Acc &re, Acc &im, V a, V b) {
        re = fmaf(a.x, b.x, re); re = fmaf(a.y, b.y, re);
        im = fmaf(a.x, b.y, im); im = fmaf(-a.y, b.x, im);
    }
    __device__ static void nrm2(Acc &s, V a) { s = fmaf(a.x, a.x, s); s = fmaf(a.y, a.y, s); }
    __device__ static R total(Acc a) { return a; }
};

// ------------------------------------------------------------------ double-float
// (s, c) -> normalized (hi, lo) with hi = fl(s + c) and lo its exact
// rounding error (TwoSum: no ordering assumption, since cancellation can
// leave |c| > |s|)
__device__ __forceinline__ float2 ff_norm(float s, float c) {
    const float h = __fadd_rn(s, c);
    const float z = __fsub_rn(h, s);
    return make_float2(h, __fadd_rn(__fsub_rn(s, __fsub_rn(h, z)), __fsub_rn(c, z)));
}

struct FFAcc { float s, c; };

template <> struct Ar<float4> {
    using V = float4; using St = double2; using S = float4; using R = double; using Acc = FFAcc;
    static constexpr bool kFF = true;
    __device__ static S scal(St a) { return split_ff(a); }
    __device__ static V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static V from_c128(double2 a) { return split_ff(a); }
    __device__ static double2 to_c128(V a) {
        return make_double2(join_d(a.x, a.y), join_d(a.z, a.w));
    }
    // a * s for a power of two s (exact while the parts stay in binary32 range)
    __device__ static V pow2(V a, double s) {
        const float f = (float)s;
        return make_float4(a.x * f, a.y * f, a.z * f, a.w * f);
    }
    // y + a x, each component accumulated exactly from y then rounded once
    __device__ static V axpy(V y, S a, V x) {
        float sr = y.x, cr = y.y, si = y.z, ci = y.w;
        ff_mac(sr, cr, a.x, a.y, x.x, x.y);
        ff_mac(sr, cr, -a.z, -a.w, x.z, x.w);
        ff_mac(si, ci, a.x, a.y, x.z, x.w);
        ff_mac(si, ci, a.z, a.w, x.x, x.y);
        const float2 r = ff_norm(sr, cr), i = ff_norm(si, ci);
        return make_float4(r.x, r.y, i.x, i.y);
    }
    __device__ static V axmy(V y, S a, V x) { return axpy(y, make_float4(-a.x, -a.y, -a.z, -a.w), x); }
    __device__ static V sub(V a, V b) {
        float sr = a.x, cr = a.y, si = a.z, ci = a.w;
        ff_acc(sr, cr, -b.x); cr = __fsub_rn(cr, b.y);
        ff_acc(si, ci, -b.z); ci = __fsub_rn(ci, b.w);
        const float2 r = ff_norm(sr, cr), i = ff_norm(si, ci);
        return make_float4(r.x, r.y, i.x, i.y);
    }
    __device__ static V add(V a, V b) {
        float sr = a.x, cr = a.y, si = a.z, ci = a.w;
        ff_acc(sr, cr, b.x); cr = __fadd_rn(cr, b.y);
        ff_acc(si, ci, b.z); ci = __fadd_rn(ci, b.w);
        const float2 r = ff_norm(sr, cr), i = ff_norm(si, ci);
        return make_float4(r.x, r.y, i.x, i.y);
    }
    __device__ static void acc_zero(Acc &a) { a.s = 0.f; a.c = 0.f; }
    __device__ static void dotc(Acc &re, Acc &im, V a, V b) {
        ff_mac(re.s, re.c, a.x, a.y, b.x, b.y);
        ff_mac(re.s, re.c, a.z, a.w, b.z, b.w);
        ff_mac(im.s, im.c, a.x, a.y, b.z, b.w);
        ff_mac(im.s, im.c, -a.z, -a.w, b.x, b.y);
    }
    __device__ static void nrm2(Acc &s, V a) {
        ff_mac(s.s, s.c, a.x, a.y, a.x, a.y);
        ff_mac(s.s, s.c, a.z, a.w, a.z, a.w);
    }
    __device__ static R total(Acc a) { return (double)a.s + (double)a.c; }
};

// ------------------------------------------------------------------ reductions
// Grid reduction of double-float accumulators.  The block and grid sums stay
// in (s, c) pairs added with binary32 TwoSums and are widened to binary64
// once, by thread 0 of the last block: on this GPU the binary64 pipe runs at
// about 1/60 of the binary32 rate, so a binary64 block sum (and the two
// conversions per thread before it) cost microseconds per reduction.  The
// order of the additions is fixed, so the result is bitwise reproducible for
// a fixed grid.  Partials are float2 pairs in red.partials.
__device__ __forceinline__ void ff_pair_add(float &s, float &c, float bs, float bc) {
    ff_acc(s, c, bs);
    c = __fadd_rn(c, bc);
}

template <int NV>
__device__ __forceinline__ void block_sum_ff(float (&s)[NV], float (&c)[NV], float2 (*sh)[NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, s[j], off);
            const float oc = __shfl_xor_sync(0xffffffffu, c[j], off);
            ff_pair_add(s[j], c[j], os, oc);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) sh[warp][j] = make_float2(s[j], c[j]);
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const float2 t = lane < nwarps ? sh[lane][j] : make_float2(0.f, 0.f);
            float ts = t.x, tc = t.y;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float os = __shfl_xor_sync(0xffffffffu, ts, off);
                const float oc = __shfl_xor_sync(0xffffffffu, tc, off);
                ff_pair_add(ts, tc, os, oc);
            }
            s[j] = ts;
            c[j] = tc;
        }
    }
    __syncthreads();
}

// as grid_reduce_last; tot[] is valid in thread 0 of the last block only
template <int NV>
__device__ __forceinline__ bool grid_reduce_last_ff(const FFAcc (&v)[NV], RedScratch red, double (&tot)[NV]) {
    __shared__ float2 sh[32][NV];
    __shared__ int am_last;
    float2 *partials = reinterpret_cast<float2 *>(red.partials);
    float s[NV], c[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        s[j] = v[j].s;
        c[j] = v[j].c;
    }
    block_sum_ff<NV>(s, c, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) partials[blockIdx.x * NV + j] = make_float2(s[j], c[j]);
        __threadfence();
        const unsigned int t = atomicAdd(red.counter, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
#pragma unroll
    for (int j = 0; j < NV; ++j) s[j] = c[j] = 0.f;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const float2 p = __ldcg(&partials[b * NV + j]);
            ff_pair_add(s[j], c[j], p.x, p.y);
        }
    }
    block_sum_ff<NV>(s, c, sh);
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = threadIdx.x == 0 ? (double)s[j] + (double)c[j] : 0.0;
    if (threadIdx.x == 0) *red.counter = 0u;
    return true;
}

// grid reduction of per-thread accumulators of any element type: pairs for
// double-float, otherwise the accumulator's own type through grid_reduce_last
template <class Acc, class R, int NV, class Total>
__device__ __forceinline__ bool grid_reduce_acc(const Acc (&acc)[NV], RedScratch red, R (&tot)[NV], Total total) {
    if constexpr (std::is_same<Acc, FFAcc>::value) {
        static_assert(std::is_same<R, double>::value, "double-float totals are binary64");
        return grid_reduce_last_ff<NV>(acc, red, tot);
    } else {
        R v[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = total(acc[j]);
        return grid_reduce_last<R, NV>(v, red, tot);
    }
}

}  // namespace hz
