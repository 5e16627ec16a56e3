// batched.cu -- a sweep of independent BiCGStab solves (one per frequency or
// geometry) in ONE persistent cooperative launch.
//
// Every system keeps its own BiCGStab state on the device (the Section 7
// algorithm, as in bicgstab.cu).  All systems advance together through the
// phases of an iteration; a phase is a list of work items (row blocks for
// the SpMV phases, element tiles for the vector phases) over the systems
// still running, shared out over every CTA of the grid, so a few large
// systems left at the end still use the whole GPU.  Per-system reductions
// are deterministic: each item writes its block partial sum, and the CTA
// that completes a system's last item folds that system's partials in item
// order and does its scalar update.  Phases are separated by a grid barrier
// whose wait is bounded in time (it reports HZ_ERR_TIMEOUT instead of
// hanging if a CTA never arrives).
//
// In binary64 an SpMV item is kBBlock / 32 row blocks of the handle's
// block-flat layout, one per warp, each summed in contiguous lane runs (the
// core of the single-system HZ_SPMV_FLAT64 kernel, groups of kBFlatG steps);
// the double-float and complex64 products keep W lanes per row (the handle's
// autotuned CSR-vector group) over runs of rows.
//
// The kernel is written once over the vector format V: complex128 in
// binary64 (double2), or complex128 in double-float on the binary32 pipes
// (float4, when every handle of the batch was created with HZ_FLAG_FF): the
// products then read the handles' split values, the iterate lives in a
// double-float workspace loaded from and stored to the caller's x, and the
// per-item reductions are folded in binary64 as before.
//
// Mixed precision (HZ_MODE_MIXED, k_batched_mixed): every system runs the
// refinement of the single-system mixed solve -- outer residual r = b - A x
// in binary64 (phase P_OUT), an inner BiCGStab on the complex64 copy of A
// with complex64 vectors and binary32 sums (phases F1..F5 in float2), then
// x += d in binary64 (P_UPD) -- each system at its own stage: in one round
// the systems whose inner solve is running take an inner iteration, those
// whose inner solve just ended are updated and take their next outer
// residual.  The refinement keeps each system's best iterate and stops a
// system when a step fails to reduce its outer residual.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "arith.cuh"
#include "spmv.cuh"

namespace hz {

constexpr int kBBlock = 256;
#ifndef HZ_BATCHED_MIN_BLOCKS
#define HZ_BATCHED_MIN_BLOCKS 3
#endif
// resident CTAs per SM asked of the register allocator (the cooperative grid
// is as many CTAs as fit, up to four per SM): the binary64 kernel with its
// block-flat products, the double-float one, the mixed one
constexpr int kBMinBlocks = HZ_BATCHED_MIN_BLOCKS;
template <class V> struct BMin { static constexpr int value = std::is_same<V, double2>::value ? kBMinBlocks : 3; };
#ifndef HZ_BATCHED_MIXED_MIN_BLOCKS
#define HZ_BATCHED_MIXED_MIN_BLOCKS 4
#endif
constexpr int kBMinBlocksMixed = HZ_BATCHED_MIXED_MIN_BLOCKS;
#ifndef HZ_BATCHED_FLAT_G
#define HZ_BATCHED_FLAT_G 2
#endif
// binary64 batches: products on the block-flat core with groups of kBFlatG
// steps (unpacked; few registers, so the cooperative grid keeps two CTAs per
// SM), 0 = the W-lane CSR-vector rows
constexpr int kBFlatG = HZ_BATCHED_FLAT_G;
constexpr int kBVecItem = kBBlock * 4;     // elements per vector item
constexpr int kBMaxSys = 1024;             // systems per launch (shared-memory tables)

struct BSys {
    int n, W, rows_per_item;
    int sp_item0, sp_items;      // SpMV items [sp_item0, sp_item0 + sp_items) (W lanes per row)
    int fl_item0, fl_items;      // binary64 SpMV items: kBBlock / 32 row blocks each, one per warp
    int vc_item0, vc_items;      // vector items
    int nfblk;                   // the handle's row blocks and packed binary64 stream
    const int *fblk, *fblk_k, *pk_base, *pk_gbase, *pk_gim, *pk_col;
    const double *pk_re, *pk_im;
    const int *rowptr;
    const int *col;
    const double2 *val;
    const float4 *vff;           // double-float split of val (double-float batches)
    const double2 *b;
    double2 *x;                  // the caller's x0 / solution
    void *xw;                    // the iterate (double-float batches; else x itself)
    void *r, *rh, *p, *v, *s, *t;
    // mixed batches: complex64 values and inner vectors (d = the inner
    // iterate), and the refinement's best iterate
    const float2 *val32;
    float2 *r32, *rh32, *p32, *v32, *s32, *t32, *d32;
    double2 *xbest;
};

// the system's vectors in format V
template <class V> struct BVecs {
    V *x, *r, *rh, *p, *v, *s, *t;
};
template <class V>
__device__ __forceinline__ BVecs<V> bvecs(const BSys &sy) {
    BVecs<V> o;
    if constexpr (std::is_same<V, float2>::value) {   // the inner solve of a mixed batch
        o.x = sy.d32; o.r = sy.r32; o.rh = sy.rh32; o.p = sy.p32; o.v = sy.v32; o.s = sy.s32; o.t = sy.t32;
    } else {
        o.x = std::is_same<V, double2>::value ? (V *)sy.x : (V *)sy.xw;
        o.r = (V *)sy.r; o.rh = (V *)sy.rh; o.p = (V *)sy.p; o.v = (V *)sy.v; o.s = (V *)sy.s; o.t = (V *)sy.t;
    }
    return o;
}

// a device-state scalar (binary64 complex) in the arithmetic of format V
template <class V>
__device__ __forceinline__ typename Ar<V>::S bscal(double2 a) {
    if constexpr (std::is_same<V, float2>::value) return to_c64(a);
    else return Ar<V>::scal(a);
}

struct BState {
    double2 rho, rho_old, alpha, omega, beta;   // BiCGStab scalars (the inner solve in a mixed batch)
    double nb, rel, relres_true;
    int iter, done, half, status;
    unsigned int cnt;            // items finished in the current phase
    // mixed batches: the refinement
    int stage;                   // S_OUTER, S_INNER, S_UPDATE or S_FINISHED
    int outer, total_inner, out_status, use_best, save, zero_x;
    double nb_out, rel_out, rel_best;
};
enum Stage { S_OUTER = 0, S_INNER = 1, S_UPDATE = 2, S_FINISHED = 3 };

struct BCtl {
    double tol;
    int maxit;
    int nsys;
    unsigned int bar_count;
    volatile unsigned int bar_gen;
    int err;
    // mixed batches
    int mixed;
    double in_tol;
    int in_maxit, max_outer;
};

enum Phase { P_INIT = 0, P_F1, P_F2, P_F3, P_F4, P_F5, P_TRUE, P_LOAD, P_STORE, P_OUT, P_UPD, P_BEST };

// bounded grid barrier: gives up after ~1 s and flags the error
__device__ bool bgrid_sync(BCtl *c) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int gen = c->bar_gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            c->bar_count = 0u;
            __threadfence();
            atomicAdd((unsigned int *)&c->bar_gen, 1u);
        } else {
            uint64_t t0, t1;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            while (c->bar_gen == gen) {
                __nanosleep(64);
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
                if (t1 - t0 > 1000000000ull) { atomicExch(&c->err, 1); break; }
                if (*(volatile int *)&c->err) break;
            }
        }
        __threadfence();
        ok = (*(volatile int *)&c->err) == 0;
    }
    __syncthreads();
    return ok != 0;
}

template <int NV>
__device__ __forceinline__ void bsum(double (&v)[NV]) {
    __shared__ double sh[kBBlock / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) sh[warp][j] = v[j];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double t = lane < kBBlock / 32 ? sh[lane][j] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            v[j] = t;
        }
    }
    __syncthreads();
}

// per-system scalar work after a phase's reduction (thread 0)
__device__ void finalize_phase(int phase, const BCtl *c, BState *S, const double *tot);

__device__ void finalize(int phase, const BCtl *c, BState *S, const double *tot) {
    finalize_phase(phase, c, S, tot);
    if (c->mixed && phase >= P_F1 && phase <= P_F5) {
        if (phase == P_F5) {   // one more inner iteration, held to the total cap
            S->total_inner += 1;
            if (!S->done && S->total_inner >= c->maxit) { S->status = HZ_NOT_CONVERGED; S->done = 1; }
        }
        if (S->done && S->stage == S_INNER) S->stage = S_UPDATE;
    }
}

// the outer step of a mixed batch: the refinement's decision after r = b - A x
// (tot = ||r||^2, ||b||^2, ||r32||^2) and the start of the next inner solve
__device__ void finalize_outer(const BCtl *c, BState *S, const double *tot) {
    const double2 one = make_double2(1.0, 0.0);
    const double nb = sqrt(tot[1]);
    S->nb_out = nb;
    S->save = 0;
    S->stage = S_FINISHED;
    if (nb == 0.0) { S->rel_out = 0.0; S->out_status = HZ_OK; S->zero_x = 1; return; }
    const double rel = sqrt(tot[0]) / nb;
    S->rel_out = rel;
    if (!isfinite(rel)) { S->out_status = HZ_ERR_NAN; S->use_best = S->outer > 0; return; }
    if (rel <= c->tol) { S->out_status = HZ_OK; return; }
    if (rel >= S->rel_best) { S->out_status = HZ_NOT_CONVERGED; S->use_best = 1; return; }
    if (S->outer >= c->max_outer || S->total_inner >= c->maxit) { S->out_status = HZ_NOT_CONVERGED; return; }
    S->rel_best = rel;
    S->save = 1;   // this x is the best so far: P_UPD keeps a copy before x += d
    S->outer += 1;
    const double nb32 = sqrt(tot[2]);
    S->rho = make_double2(tot[2], 0.0);
    S->rho_old = one; S->alpha = one; S->omega = one; S->beta = make_double2(0.0, 0.0);
    S->nb = nb32; S->rel = 1.0; S->half = 0; S->iter = 1;
    S->status = HZ_NOT_CONVERGED;
    S->done = nb32 == 0.0;
    S->stage = S->done ? S_UPDATE : S_INNER;
}

__device__ void finalize_phase(int phase, const BCtl *c, BState *S, const double *tot) {
    const double2 one = make_double2(1.0, 0.0);
    const double tol = c->mixed ? c->in_tol : c->tol;
    const int maxit = c->mixed ? c->in_maxit : c->maxit;
    switch (phase) {
        case P_INIT: {
            const double nb = sqrt(tot[1]);
            S->nb = nb; S->half = 0; S->iter = 0;
            S->rho = make_double2(tot[0], 0.0);
            S->rho_old = one; S->alpha = one; S->omega = one; S->beta = make_double2(0.0, 0.0);
            S->done = 1;
            if (nb == 0.0) { S->rel = 0.0; S->status = HZ_OK; break; }
            const double rel = sqrt(tot[0]) / nb;
            S->rel = rel;
            if (!isfinite(rel)) S->status = HZ_ERR_NAN;
            else if (rel <= c->tol) S->status = HZ_OK;
            else if (c->maxit <= 0) S->status = HZ_NOT_CONVERGED;
            else { S->status = HZ_NOT_CONVERGED; S->done = 0; S->iter = 1; }
            break;
        }
        case P_F2: {
            const double2 sig = make_double2(tot[0], tot[1]);
            if (cis_zero(sig)) { S->status = HZ_BREAKDOWN; S->done = 1; break; }
            S->alpha = cdiv(S->rho, sig);
            break;
        }
        case P_F3: {
            const double rel = sqrt(tot[0]) / S->nb;
            if (!isfinite(rel)) { S->status = HZ_ERR_NAN; S->done = 1; S->rel = rel; break; }
            if (rel <= tol) { S->half = 1; S->rel = rel; }
            break;
        }
        case P_F4: {
            if (tot[2] == 0.0) { S->status = HZ_BREAKDOWN; S->done = 1; break; }
            S->omega = make_double2(tot[0] / tot[2], tot[1] / tot[2]);
            break;
        }
        case P_F5: {
            if (S->half) { S->status = HZ_OK; S->done = 1; break; }
            const double rel = sqrt(tot[2]) / S->nb;
            S->rel = rel;
            if (!isfinite(rel)) { S->status = HZ_ERR_NAN; S->done = 1; }
            else if (rel <= tol) { S->status = HZ_OK; S->done = 1; }
            else if (cis_zero(S->omega)) { S->status = HZ_BREAKDOWN; S->done = 1; }
            else if (S->iter >= maxit) { S->status = HZ_NOT_CONVERGED; S->done = 1; }
            else {
                const double2 rn = make_double2(tot[0], tot[1]);
                S->beta = cmul(cdiv(rn, S->rho), cdiv(S->alpha, S->omega));
                S->rho_old = S->rho;
                S->rho = rn;
                S->iter += 1;                                  // next iteration starts
                if (cis_zero(rn)) { S->status = HZ_BREAKDOWN; S->done = 1; }
            }
            break;
        }
        case P_TRUE: {
            const double nb = c->mixed ? S->nb_out : S->nb;
            S->relres_true = nb == 0.0 ? 0.0 : sqrt(tot[0]) / nb;
            break;
        }
        case P_OUT:
            finalize_outer(c, S, tot);
            break;
        default: break;
    }
}

template <int NV>
__device__ void item_done(int phase, const BCtl *c, const BSys &sy, BState *S, double *partials, int item_global,
                          int item0, int nitems, double (&acc)[NV]) {
    __shared__ int last;
    bsum<NV>(acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) partials[(size_t)item_global * 4 + j] = acc[j];
        __threadfence();
        const unsigned int k = atomicAdd(&S->cnt, 1u);
        last = (k == (unsigned int)nitems - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double tot[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = 0.0;
    for (int it = threadIdx.x; it < nitems; it += kBBlock)
#pragma unroll
        for (int j = 0; j < NV; ++j) tot[j] += __ldcg(&partials[(size_t)(item0 + it) * 4 + j]);
    bsum<NV>(tot);
    if (threadIdx.x == 0) {
        S->cnt = 0u;
        finalize(phase, c, S, tot);
        __threadfence();
    }
    __syncthreads();
}

// the phase epilogue of one finished row y (lane 0 of the row's group)
// item_done for double-float accumulators: the block sum and the fold over
// a system's items stay in binary32 (s, c) pairs (float2 in the partials
// slots) and are widened once for finalize; the binary64 pipe is far slower
// than the binary32 one on this GPU
template <int NV>
__device__ void item_done_ff(int phase, const BCtl *c, const BSys &sy, BState *S, double *partials,
                             int item_global, int item0, int nitems, const FFAcc *acc) {
    __shared__ float2 sh[32][NV];
    __shared__ int last;
    float2 *pp = reinterpret_cast<float2 *>(partials);
    float hs[NV], lc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        hs[j] = acc[j].s;
        lc[j] = acc[j].c;
    }
    block_sum_ff<NV>(hs, lc, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) pp[(size_t)item_global * 4 + j] = make_float2(hs[j], lc[j]);
        __threadfence();
        const unsigned int k = atomicAdd(&S->cnt, 1u);
        last = (k == (unsigned int)nitems - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int j = 0; j < NV; ++j) hs[j] = lc[j] = 0.f;
    for (int it = threadIdx.x; it < nitems; it += kBBlock)
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const float2 q = __ldcg(&pp[(size_t)(item0 + it) * 4 + j]);
            ff_pair_add(hs[j], lc[j], q.x, q.y);
        }
    block_sum_ff<NV>(hs, lc, sh);
    if (threadIdx.x == 0) {
        double tot[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) tot[j] = (double)hs[j] + (double)lc[j];
        S->cnt = 0u;
        finalize(phase, c, S, tot);
        __threadfence();
    }
    __syncthreads();
}

template <class V, class Acc>
__device__ __forceinline__ void row_epilogue(int phase, const BSys &sy, int row, V y, Acc (&acc)[3]) {
    using A = Ar<V>;
    constexpr bool kC64 = std::is_same<V, float2>::value;   // inner solve of a mixed batch
    const BVecs<V> w = bvecs<V>(sy);
    if (phase == P_INIT) {
        if constexpr (!kC64) {
            const V bi = A::from_c128(sy.b[row]);
            const V ri = A::sub(bi, y);
            w.r[row] = ri; w.rh[row] = ri;
            w.p[row] = A::zero(); w.v[row] = A::zero();
            A::nrm2(acc[0], ri);
            A::nrm2(acc[1], bi);
        }
    } else if (phase == P_F2) {
        w.v[row] = y;
        A::dotc(acc[0], acc[1], w.rh[row], y);
    } else if (phase == P_F4) {
        w.t[row] = y;
        A::dotc(acc[0], acc[1], y, w.s[row]);
        A::nrm2(acc[2], y);
    } else if (phase == P_OUT) {   // mixed: outer residual in binary64, inner start in complex64
        if constexpr (std::is_same<V, double2>::value) {
            const double2 ri = csub(sy.b[row], y);
            const float2 r32 = to_c64(ri);
            sy.r32[row] = r32; sy.rh32[row] = r32;
            sy.p32[row] = make_float2(0.f, 0.f); sy.v32[row] = make_float2(0.f, 0.f);
            sy.d32[row] = make_float2(0.f, 0.f);
            A::nrm2(acc[0], ri);
            A::nrm2(acc[1], sy.b[row]);
            A::nrm2(acc[2], to_c128(r32));
        }
    } else if constexpr (!kC64) {   // P_TRUE
        A::nrm2(acc[0], A::sub(A::from_c128(sy.b[row]), y));
    }
}

// SpMV rows [r0, r1) of one system with W lanes per row and the phase epilogue
template <int W, class V>
__device__ void spmv_item(int phase, const BSys &sy, int r0, int r1, typename Ar<V>::Acc (&acc)[3]) {
    const int lane = threadIdx.x & (W - 1);
    const unsigned gmask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << ((threadIdx.x & 31) & ~(W - 1)));
    const BVecs<V> w = bvecs<V>(sy);
    const V *x = phase == P_F2 ? w.p : phase == P_F4 ? w.s : w.x;
    for (int row = r0 + (int)threadIdx.x / W; row < r1; row += kBBlock / W) {
        const int beg = __ldg(sy.rowptr + row), end = __ldg(sy.rowptr + row + 1);
        V y;
        if constexpr (std::is_same<V, double2>::value) {
            y = make_double2(0.0, 0.0);
            for (int k = beg + lane; k < end; k += W) cmac(y, ld_stream(sy.val + k), __ldg(x + ld_stream(sy.col + k)));
#pragma unroll
            for (int off = W / 2; off > 0; off >>= 1) {
                y.x += __shfl_xor_sync(gmask, y.x, off, W);
                y.y += __shfl_xor_sync(gmask, y.y, off, W);
            }
        } else if constexpr (std::is_same<V, float2>::value) {   // complex64 inner operator
            y = make_float2(0.f, 0.f);
            for (int k = beg + lane; k < end; k += W) cmac(y, ld_stream(sy.val32 + k), __ldg(x + ld_stream(sy.col + k)));
#pragma unroll
            for (int off = W / 2; off > 0; off >>= 1) {
                y.x += __shfl_xor_sync(gmask, y.x, off, W);
                y.y += __shfl_xor_sync(gmask, y.y, off, W);
            }
        } else {
            // packed double-float sums (re, im) per lane, folded over the group
            f32x2 S = 0ull, C = 0ull;
            for (int k = beg + lane; k < end; k += W) ff_cacc(S, C, ff_cprod(ld_stream(sy.vff + k), __ldg(x + ld_stream(sy.col + k))));
#pragma unroll
            for (int off = W / 2; off > 0; off >>= 1) {
                const f32x2 S2 = __shfl_xor_sync(gmask, S, off, W), C2 = __shfl_xor_sync(gmask, C, off, W);
                f32x2 t, e;
                two_sum2(S, S2, t, e);
                S = t;
                C = add2(C, add2(C2, e));
            }
            f32x2 h, l;
            two_sum2(S, C, h, l);
            float hr, hi, lr, li;
            upk2(h, hr, hi);
            upk2(l, lr, li);
            y = make_float4(hr, lr, hi, li);
        }
        if (lane != 0) continue;
        row_epilogue<V>(phase, sy, row, y, acc);
    }
}

// the phase epilogue as a block-flat SpMV epilogue
struct BEpi {
    using Acc = double;
    int phase;
    const BSys *sy;
    __device__ void row(int i, double2 y, Acc (&acc)[3]) const { row_epilogue<double2>(phase, *sy, i, y, acc); }
};

// binary64 SpMV item `local` of one system: warp w takes row block
// kBBlock / 32 * local + w with the block-flat core (the caller's CSR arrays,
// groups of kBFlatG steps), rows finished with the phase epilogue
__device__ void spmv_item_flat(int phase, const BSys &sy, int local, double (&acc)[3]) {
    __shared__ D64Seg seg[kBBlock / 32];
    const BVecs<double2> w = bvecs<double2>(sy);
    const double2 *x = phase == P_F2 ? w.p : phase == P_F4 ? w.s : w.x;
    MatView<double2> A{};
    A.n = sy.n; A.rowptr = sy.rowptr; A.col = sy.col; A.val = sy.val;
    A.nfblk = sy.nfblk; A.fblk = sy.fblk; A.fblk_k = sy.fblk_k;
    A.pk_base = sy.pk_base; A.pk_gbase = sy.pk_gbase; A.pk_gim = sy.pk_gim; A.pk_col = sy.pk_col;
    A.pk_re = sy.pk_re; A.pk_im = sy.pk_im;
    const BEpi epi{phase, &sy};
    constexpr int wpi = kBBlock / 32;
    const int b0 = local * wpi + (int)(threadIdx.x >> 5), bend = min(sy.nfblk, (local + 1) * wpi);
    flat_rows_d64<BEpi, 3, false, (kBFlatG > 0 ? kBFlatG : 1)>(A, x, epi, acc, &seg[threadIdx.x >> 5], b0, wpi,
                                                               bend);
}

template <class V>
__device__ void vec_item(int phase, const BSys &sy, const BState *S, int e0, int e1, typename Ar<V>::Acc (&acc)[3]) {
    using A = Ar<V>;
    const BVecs<V> w = bvecs<V>(sy);
    const typename A::S alpha = bscal<V>(S->alpha), omega = bscal<V>(S->omega), beta = bscal<V>(S->beta);
    const bool half = S->half;
    if constexpr (std::is_same<V, double2>::value) {
        if (phase == P_UPD) {   // mixed: keep the best iterate, then x += d
            const bool save = S->save != 0;
            for (int i = e0 + threadIdx.x; i < e1; i += kBBlock) {
                const double2 xi = sy.x[i];
                if (save) sy.xbest[i] = xi;
                sy.x[i] = cadd(xi, to_c128(sy.d32[i]));
            }
            return;
        }
        if (phase == P_BEST) {   // mixed: the answer is the kept best iterate (or 0 for b = 0)
            const bool zero = S->zero_x != 0;
            for (int i = e0 + threadIdx.x; i < e1; i += kBBlock)
                sy.x[i] = zero ? make_double2(0.0, 0.0) : sy.xbest[i];
            return;
        }
    }
    // the BiCGStab passes: each thread loads the operands of all its
    // elements of the item before the first store (the stores may alias
    // nothing here, but the compiler cannot know, and would otherwise wait
    // out one memory round trip per element); loads are clamped into the item
    // (complex64: all four elements at once; 16-byte formats two at a time)
    constexpr int U = std::is_same<V, float2>::value ? kBVecItem / kBBlock : 2;
    static_assert((kBVecItem / kBBlock) % U == 0, "whole stages per item");
    if (phase == P_F1 || phase == P_F3 || (phase == P_F5 && !half)) {
        for (int i0 = e0 + (int)threadIdx.x; i0 < e0 + kBVecItem; i0 += U * kBBlock) {
        auto at = [&](int u) { return min(i0 + u * kBBlock, e1 - 1); };
        auto in = [&](int u) { return i0 + u * kBBlock < e1; };
        if (phase == P_F1) {
            V a[U], b[U], q[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                a[u] = w.r[at(u)];
                b[u] = w.p[at(u)];
                q[u] = w.v[at(u)];
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (in(u)) w.p[at(u)] = A::axpy(a[u], beta, A::axmy(b[u], omega, q[u]));
            continue;
        }
        if (phase == P_F3) {
            V a[U], q[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                a[u] = w.r[at(u)];
                q[u] = w.v[at(u)];
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (in(u)) {
                    const V o = A::axmy(a[u], alpha, q[u]);
                    w.s[at(u)] = o;
                    A::nrm2(acc[0], o);
                }
            continue;
        }
        if (phase == P_F5 && !half) {
            V xs[U], ps[U], ss[U], ts[U], hs[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                xs[u] = w.x[at(u)];
                ps[u] = w.p[at(u)];
                ss[u] = w.s[at(u)];
                ts[u] = w.t[at(u)];
                hs[u] = w.rh[at(u)];
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (in(u)) {
                    w.x[at(u)] = A::axpy(A::axpy(xs[u], alpha, ps[u]), omega, ss[u]);
                    const V ri = A::axmy(ss[u], omega, ts[u]);
                    w.r[at(u)] = ri;
                    A::dotc(acc[0], acc[1], hs[u], ri);
                    A::nrm2(acc[2], ri);
                }
            continue;
        }
        }
        return;
    }
    for (int i = e0 + threadIdx.x; i < e1; i += kBBlock) {
        if (phase == P_F5) {   // the half step: x += alpha p
            w.x[i] = A::axpy(w.x[i], alpha, w.p[i]);
        } else if constexpr (!std::is_same<V, float2>::value) {
            if (phase == P_LOAD) w.x[i] = A::from_c128(sy.x[i]);
            else if (phase == P_STORE) sy.x[i] = A::to_c128(w.x[i]);
        }
    }
}

// one phase over the systems in the block's active table (Flat: binary64
// products on the block-flat core, item lists I_FLAT)
template <class V, bool Flat = false>
__device__ void run_phase(int phase, const BCtl *c, const BSys *sys, BState *st, double *partials, const int *act,
                          const int *pref, int nact) {
    const bool spmv = phase == P_INIT || phase == P_F2 || phase == P_F4 || phase == P_TRUE || phase == P_OUT;
    // phases over a list the stage already filters (mixed) or over every system
    const bool listed = phase == P_INIT || phase == P_TRUE || phase == P_LOAD || phase == P_STORE ||
                        phase == P_OUT || phase == P_UPD || phase == P_BEST;
    const int total = pref[nact];
    for (int j = blockIdx.x; j < total; j += gridDim.x) {
        int lo = 0, hi = nact - 1;          // system owning item j
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pref[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const int s = act[lo];
        const BSys &sy = sys[s];
        BState *S = &st[s];
        const int local = j - pref[lo];
        __shared__ int skip;
        if (threadIdx.x == 0) {
            const int done = *(volatile int *)&S->done, half = *(volatile int *)&S->half;
            skip = (!listed && done) || (phase == P_F4 && half);
        }
        __syncthreads();
        if (skip) continue;
        typename Ar<V>::Acc va[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) Ar<V>::acc_zero(va[q]);
        double acc[3];
        if (spmv) {
            constexpr bool kFlat = Flat && std::is_same<V, double2>::value;
            if constexpr (kFlat) {
                spmv_item_flat(phase, sy, local, va);
            } else {
                const int r0 = local * sy.rows_per_item, r1 = min(sy.n, r0 + sy.rows_per_item);
                switch (sy.W) {
                    case 2: spmv_item<2, V>(phase, sy, r0, r1, va); break;
                    case 4: spmv_item<4, V>(phase, sy, r0, r1, va); break;
                    case 8: spmv_item<8, V>(phase, sy, r0, r1, va); break;
                    case 16: spmv_item<16, V>(phase, sy, r0, r1, va); break;
                    default: spmv_item<32, V>(phase, sy, r0, r1, va); break;
                }
            }
            const int nit = kFlat ? sy.fl_items : sy.sp_items;
            const int g = (kFlat ? sy.fl_item0 : sy.sp_item0) + local;
            if constexpr (Ar<V>::kFF) {
                if (phase == P_F4) item_done_ff<3>(phase, c, sy, S, partials, g, sy.sp_item0, nit, va);
                else if (phase == P_TRUE) item_done_ff<1>(phase, c, sy, S, partials, g, sy.sp_item0, nit, va);
                else item_done_ff<2>(phase, c, sy, S, partials, g, sy.sp_item0, nit, va);
            } else {
#pragma unroll
                for (int q = 0; q < 3; ++q) acc[q] = (double)Ar<V>::total(va[q]);
                const int i0 = kFlat ? sy.fl_item0 : sy.sp_item0;
                if (phase == P_F4 || phase == P_OUT) item_done<3>(phase, c, sy, S, partials, g, i0, nit, acc);
                else if (phase == P_TRUE) {
                    double a1[1] = {acc[0]};
                    item_done<1>(phase, c, sy, S, partials, g, i0, nit, a1);
                } else {
                    double a2[2] = {acc[0], acc[1]};
                    item_done<2>(phase, c, sy, S, partials, g, i0, nit, a2);
                }
            }
        } else {
            const int e0 = local * kBVecItem, e1 = min(sy.n, e0 + kBVecItem);
            vec_item<V>(phase, sy, S, e0, e1, va);
            const int nit = sy.vc_items;
            const int g = sy.vc_item0 + local;
            if constexpr (Ar<V>::kFF) {
                if (phase == P_F3) item_done_ff<1>(phase, c, sy, S, partials, g, sy.vc_item0, nit, va);
                else if (phase == P_F5) item_done_ff<3>(phase, c, sy, S, partials, g, sy.vc_item0, nit, va);
            } else {
#pragma unroll
                for (int q = 0; q < 3; ++q) acc[q] = (double)Ar<V>::total(va[q]);
                if (phase == P_F3) {
                    double a1[1] = {acc[0]};
                    item_done<1>(phase, c, sy, S, partials, g, sy.vc_item0, nit, a1);
                } else if (phase == P_F5) {
                    item_done<3>(phase, c, sy, S, partials, g, sy.vc_item0, nit, acc);
                }
            }
        }
        __syncthreads();   // `skip` is rewritten by the next item
    }
}

// table of systems still running and their item prefix sums: the flags and
// item counts are loaded by all threads at once, the prefix is taken in
// shared memory by one thread
enum { A_ALL = 0, A_RUNNING = 1, A_INNER = 2, A_UPDATE = 3, A_BEST = 4, A_UNFINISHED = 5 };

__device__ __forceinline__ bool bactive(int which, const BState &S) {
    switch (which) {
        case A_ALL: return true;
        case A_RUNNING: return !*(volatile const int *)&S.done;
        case A_INNER: return *(volatile const int *)&S.stage == S_INNER && !*(volatile const int *)&S.done;
        case A_UPDATE: return *(volatile const int *)&S.stage == S_UPDATE;
        case A_BEST:
            return *(volatile const int *)&S.stage == S_FINISHED &&
                   (*(volatile const int *)&S.use_best || *(volatile const int *)&S.zero_x);
        default: return *(volatile const int *)&S.stage != S_FINISHED;
    }
}

enum { I_VEC = 0, I_SPMV = 1, I_FLAT = 2 };   // item lists: vector tiles, W-lane SpMV rows, binary64 row blocks

__device__ int build_active(int items, const BCtl *c, const BSys *sys, const BState *st, int *act,
                            int *pref, int which) {
    __shared__ int nact;
    __shared__ int cnt[kBMaxSys];
    const int nsys = c->nsys;
    for (int s = threadIdx.x; s < nsys; s += kBBlock) {
        const bool run = bactive(which, st[s]);
        cnt[s] = run ? (items == I_FLAT ? sys[s].fl_items : items == I_SPMV ? sys[s].sp_items : sys[s].vc_items) : -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int k = 0;
        pref[0] = 0;
        for (int s = 0; s < nsys; ++s) {
            if (cnt[s] < 0) continue;
            act[k] = s;
            pref[k + 1] = pref[k] + cnt[s];
            ++k;
        }
        nact = k;
    }
    __syncthreads();
    return nact;
}

template <class V>
__global__ void __launch_bounds__(kBBlock, BMin<V>::value) k_batched(BCtl *c, const BSys *sys, BState *st, double *partials) {
    __shared__ int act[kBMaxSys];
    __shared__ int pref_sp[kBMaxSys + 1];
    __shared__ int pref_vc[kBMaxSys + 1];
    constexpr bool kFF = !std::is_same<V, double2>::value;
    constexpr bool kFl = !kFF && kBFlatG > 0;   // binary64 products on the block-flat core
    constexpr int kSp = kFl ? I_FLAT : I_SPMV;
    int nact;
    if constexpr (kFF) {   // the iterate into the double-float workspace
        nact = build_active(I_VEC, c, sys, st, act, pref_vc, A_ALL);
        run_phase<V, kFl>(P_LOAD, c, sys, st, partials, act, pref_vc, nact);
        if (!bgrid_sync(c)) return;
    }
    nact = build_active(kSp, c, sys, st, act, pref_sp, A_ALL);
    run_phase<V, kFl>(P_INIT, c, sys, st, partials, act, pref_sp, nact);
    if (!bgrid_sync(c)) return;
    for (int guard = 0; guard <= c->maxit + 1; ++guard) {
        nact = build_active(kSp, c, sys, st, act, pref_sp, A_RUNNING);
        if (nact == 0) break;
        build_active(I_VEC, c, sys, st, act, pref_vc, A_RUNNING);
        run_phase<V, kFl>(P_F1, c, sys, st, partials, act, pref_vc, nact);
        if (!bgrid_sync(c)) return;
        run_phase<V, kFl>(P_F2, c, sys, st, partials, act, pref_sp, nact);
        if (!bgrid_sync(c)) return;
        run_phase<V, kFl>(P_F3, c, sys, st, partials, act, pref_vc, nact);
        if (!bgrid_sync(c)) return;
        run_phase<V, kFl>(P_F4, c, sys, st, partials, act, pref_sp, nact);
        if (!bgrid_sync(c)) return;
        run_phase<V, kFl>(P_F5, c, sys, st, partials, act, pref_vc, nact);
        if (!bgrid_sync(c)) return;
    }
    nact = build_active(kSp, c, sys, st, act, pref_sp, A_ALL);
    run_phase<V, kFl>(P_TRUE, c, sys, st, partials, act, pref_sp, nact);
    if constexpr (kFF) {   // the solution back to the caller's x
        if (!bgrid_sync(c)) return;
        nact = build_active(I_VEC, c, sys, st, act, pref_vc, A_ALL);
        run_phase<V, kFl>(P_STORE, c, sys, st, partials, act, pref_vc, nact);
    }
}

// mixed-precision sweep: every system refines in binary64 around complex64
// inner BiCGStab solves, each at its own stage (see the file comment)
__global__ void __launch_bounds__(kBBlock, kBMinBlocksMixed) k_batched_mixed(BCtl *c, const BSys *sys, BState *st, double *partials) {
    __shared__ int act[kBMaxSys];
    __shared__ int pref_sp[kBMaxSys + 1];
    __shared__ int pref_vc[kBMaxSys + 1];
    int nact = build_active(I_SPMV, c, sys, st, act, pref_sp, A_UNFINISHED);
    run_phase<double2>(P_OUT, c, sys, st, partials, act, pref_sp, nact);
    if (!bgrid_sync(c)) return;
    // every round advances each system by one inner iteration or one
    // refinement step, so a system leaves within maxit + max_outer + 1 rounds
    const int cap = c->maxit + c->max_outer + 2;
    for (int round = 0; round <= cap; ++round) {
        const int nin = build_active(I_SPMV, c, sys, st, act, pref_sp, A_INNER);
        if (nin > 0) {
            build_active(I_VEC, c, sys, st, act, pref_vc, A_INNER);
            run_phase<float2>(P_F1, c, sys, st, partials, act, pref_vc, nin);
            if (!bgrid_sync(c)) return;
            run_phase<float2>(P_F2, c, sys, st, partials, act, pref_sp, nin);
            if (!bgrid_sync(c)) return;
            run_phase<float2>(P_F3, c, sys, st, partials, act, pref_vc, nin);
            if (!bgrid_sync(c)) return;
            run_phase<float2>(P_F4, c, sys, st, partials, act, pref_sp, nin);
            if (!bgrid_sync(c)) return;
            run_phase<float2>(P_F5, c, sys, st, partials, act, pref_vc, nin);
            if (!bgrid_sync(c)) return;
        }
        const int nup = build_active(I_VEC, c, sys, st, act, pref_vc, A_UPDATE);
        if (nin == 0 && nup == 0) break;
        if (nup > 0) {
            run_phase<double2>(P_UPD, c, sys, st, partials, act, pref_vc, nup);
            if (!bgrid_sync(c)) return;
            build_active(I_SPMV, c, sys, st, act, pref_sp, A_UPDATE);
            run_phase<double2>(P_OUT, c, sys, st, partials, act, pref_sp, nup);
            if (!bgrid_sync(c)) return;
        }
    }
    nact = build_active(I_VEC, c, sys, st, act, pref_vc, A_BEST);
    run_phase<double2>(P_BEST, c, sys, st, partials, act, pref_vc, nact);
    if (!bgrid_sync(c)) return;
    nact = build_active(I_SPMV, c, sys, st, act, pref_sp, A_ALL);
    run_phase<double2>(P_TRUE, c, sys, st, partials, act, pref_sp, nact);
}

hz_status ensure_c64(hz_mat *A, cudaStream_t s);

}  // namespace hz

using namespace hz;

extern "C" HZ_API hz_status hz_zsolve_batched(int32_t nsys, hz_mat *const *A, const hz_z *const *d_b,
                                              hz_z *const *d_x, double tol, int32_t maxit, uint32_t mode,
                                              hz_info *h_info, void *stream) {
    HZ_CHECK(nsys >= 0 && nsys <= kBMaxSys, "hz_zsolve_batched: nsys out of range (0..1024)");
    HZ_CHECK(mode == HZ_MODE_FP64 || mode == HZ_MODE_MIXED, "hz_zsolve_batched: unknown mode");
    const bool mixed = mode == HZ_MODE_MIXED;
    HZ_CHECK(maxit >= 0 && tol >= 0.0, "hz_zsolve_batched: bad tol/maxit");
    if (nsys == 0) return HZ_OK;
    HZ_CHECK(A && d_b && d_x && h_info, "hz_zsolve_batched: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<BSys> hs(nsys);
    int64_t sp = 0, fl = 0, vc = 0, vec_elems = 0;
    // double-float when every handle carries the split values and runs a
    // double-float SpMV kind; binary64 otherwise
    // (a mixed batch refines in binary64 around complex64 inner solves)
    bool ff = !mixed;
    for (int k = 0; k < nsys; ++k) {
        HZ_CHECK(A[k], "hz_zsolve_batched: null matrix handle");
        if (A[k]->n > 0 && !(A[k]->val_ff && is_ff_kind(A[k]->spmv_kind))) ff = false;
        if (mixed && A[k]->n > 0) HZ_TRY(ensure_c64(A[k], s));
    }
    // per system: 16-byte vectors (6 binary64 or 7 double-float; mixed: the
    // best iterate) and, in a mixed batch, 7 complex64 inner vectors
    const int nvec = mixed ? 1 : ff ? 7 : 6;
    const int nvec32 = mixed ? 7 : 0;
    for (int k = 0; k < nsys; ++k) {
        HZ_CHECK(A[k]->n == 0 || (d_b[k] && d_x[k]), "hz_zsolve_batched: null vector");
        BSys &y = hs[k];
        y.n = A[k]->n;
        y.W = A[k]->group;
        y.rows_per_item = (kBBlock / y.W) * 4;
        y.sp_item0 = (int)sp;
        y.sp_items = (y.n + y.rows_per_item - 1) / y.rows_per_item;
        y.fl_item0 = (int)fl;
        y.fl_items = (A[k]->nfblk + kBBlock / 32 - 1) / (kBBlock / 32);
        y.nfblk = A[k]->nfblk; y.fblk = A[k]->fblk; y.fblk_k = A[k]->fblk_k;
        y.pk_base = A[k]->pk_base; y.pk_gbase = A[k]->pk_gbase; y.pk_gim = A[k]->pk_gim;
        y.pk_col = A[k]->pk_col; y.pk_re = A[k]->pk_re; y.pk_im = A[k]->pk_im;
        y.vc_item0 = (int)vc;
        y.vc_items = (y.n + kBVecItem - 1) / kBVecItem;
        y.rowptr = A[k]->rowptr; y.col = A[k]->col; y.val = A[k]->val; y.vff = A[k]->val_ff;
        y.val32 = A[k]->val32;
        y.b = (const double2 *)d_b[k]; y.x = (double2 *)d_x[k]; y.xw = nullptr;
        sp += y.sp_items;
        fl += y.fl_items;
        vc += y.vc_items;
        vec_elems += y.n;
    }
    HZ_CHECK(sp < INT32_MAX / 4 && fl < INT32_MAX / 4 && vc < INT32_MAX / 4, "hz_zsolve_batched: batch too large");
    // workspace: 6 vectors per system, item partials, states, controls
    double2 *work = nullptr;
    float2 *work32 = nullptr;
    double *partials = nullptr;
    BState *st = nullptr;
    BSys *dsys = nullptr;
    BCtl *ctl = nullptr;
    auto cleanup = [&]() {
        cudaFree(work); cudaFree(work32); cudaFree(partials); cudaFree(st); cudaFree(dsys); cudaFree(ctl);
    };
    if (cudaMalloc(&work, sizeof(double2) * std::max<int64_t>(nvec * vec_elems, 1)) != cudaSuccess ||
        cudaMalloc(&work32, sizeof(float2) * std::max<int64_t>(nvec32 * vec_elems, 1)) != cudaSuccess ||
        cudaMalloc(&partials, sizeof(double) * 4 * std::max<int64_t>(std::max(std::max(sp, fl), vc), 1)) != cudaSuccess ||
        cudaMalloc(&st, sizeof(BState) * nsys) != cudaSuccess || cudaMalloc(&dsys, sizeof(BSys) * nsys) != cudaSuccess ||
        cudaMalloc(&ctl, sizeof(BCtl)) != cudaSuccess) {
        cleanup();
        set_error("hz_zsolve_batched: workspace allocation failed");
        return HZ_ERR_ALLOC;
    }
    int64_t off = 0, off32 = 0;
    for (auto &y : hs) {   // 16-byte elements in either format
        if (mixed) {
            y.xbest = work + off;
            off += y.n;
            float2 **v32[7] = {&y.r32, &y.rh32, &y.p32, &y.v32, &y.s32, &y.t32, &y.d32};
            for (int q = 0; q < nvec32; ++q) { *v32[q] = work32 + off32; off32 += y.n; }
            continue;
        }
        void **vecs[7] = {&y.r, &y.rh, &y.p, &y.v, &y.s, &y.t, &y.xw};
        for (int q = 0; q < nvec; ++q) { *vecs[q] = work + off; off += y.n; }
    }
    BCtl hc{};
    hc.tol = tol; hc.maxit = maxit; hc.nsys = nsys;
    // the refinement's controls: the defaults of the single-system mixed solve
    hc.mixed = mixed ? 1 : 0;
    hc.in_tol = 1e-5;
    hc.in_maxit = 1000;
    hc.max_outer = 50;
    cudaError_t e = cudaMemcpyAsync(dsys, hs.data(), sizeof(BSys) * nsys, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, &hc, sizeof(BCtl), cudaMemcpyHostToDevice, s);
    std::vector<BState> hst(nsys);
    for (int k = 0; k < nsys; ++k) {
        hst[k] = BState{};
        hst[k].stage = S_OUTER;
        hst[k].rel_best = INFINITY;
        if (hs[k].n == 0) {   // nothing to solve
            hst[k].done = 1; hst[k].status = HZ_OK;
            hst[k].stage = S_FINISHED; hst[k].out_status = HZ_OK;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(st, hst.data(), sizeof(BState) * nsys, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    DevInfo d;
    int occ = 0;
    void *kern = mixed ? (void *)k_batched_mixed : ff ? (void *)k_batched<float4> : (void *)k_batched<double2>;
    if (e == cudaSuccess && dev_info(&d) == HZ_OK)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBBlock, 0);
    if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) {
        dim3 grid(d.num_sms * std::min(occ, 4)), block(kBBlock);
        void *args[] = {&ctl, &dsys, &st, &partials};
        e = cudaLaunchCooperativeKernel(kern, grid, block, args, 0, s);
    }
    BCtl hc2{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), st, sizeof(BState) * nsys, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc2, ctl, sizeof(BCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "hz_zsolve_batched", __FILE__, __LINE__);
    if (hc2.err) {
        set_error("hz_zsolve_batched: a grid barrier wait timed out");
        return HZ_ERR_TIMEOUT;
    }
    hz_status worst = HZ_OK;
    for (int k = 0; k < nsys; ++k) {
        hz_info &o = h_info[k];
        o = hz_info{};
        if (mixed) {
            o.iters = hst[k].total_inner;
            o.status = hst[k].out_status;
            o.outer = hst[k].outer;
            o.relres_rec = hst[k].use_best ? hst[k].rel_best : hst[k].rel_out;
        } else {
            o.iters = hst[k].iter;
            o.status = hst[k].status;
            o.relres_rec = hst[k].rel;
        }
        o.relres_true = hst[k].relres_true;
        if (A[k]->n == 0) { o.status = HZ_OK; o.iters = 0; }
        if (o.status == HZ_OK && o.relres_true > tol) o.status = HZ_NOT_CONVERGED;
        if (o.status != HZ_OK && worst == HZ_OK) worst = (hz_status)o.status;
    }
    return worst;
}
