// bicgstab.cu -- preconditioner-free BiCGStab (Section 7 of the paper, the
// algorithm of van der Vorst as stated in Saad's book, which it cites),
// fused into five kernels per iteration and run entirely on the device:
//
//   F1  p = r + beta (p - omega v)                       (stream)
//   F2  v = A p,           sigma = <rh, v>               (SpMV + dot epilogue)
//   F3  s = r - alpha v,   ||s||^2                       (stream + reduction)
//   F4  t = A s,           <t, s>, <t, t>                (SpMV + dot epilogue)
//   F5  x += alpha p + omega s,  r = s - omega t,
//                          rho' = <rh, r>, ||r||^2       (stream + reduction)
//
// Each reduction's last block also does the scalar work (alpha, omega, beta,
// stopping and breakdown tests), so the scalars never leave the device.  The
// iteration is one CUDA graph: init -> WHILE(conditional node){F1..F5} ->
// true residual -> copy-out -> info readback; the loop guard after F5 sets
// the loop condition (no kernel of the body but the guard touches it).
//
// The kernels are written once over the vector element type (arith.cuh):
// complex128 in binary64 (HZ_SPMV_CSR_VECTOR / HZ_SPMV_SELL handles),
// complex128 in double-float on the binary32 pipes (HZ_SPMV_FF handles), and
// complex64 for the inner solve of the mixed-precision refinement: an outer
// loop in complex128 (residual b - A x, its norm, x += d) around the same
// five-kernel iteration on a rounded complex64 copy of A (nested WHILE nodes).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "krylov.cuh"

namespace hz {

hz_status ensure_c64(hz_mat *A, cudaStream_t s);

// ---------------------------------------------------------------------------
// F1: p = r + beta (p - omega v)
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_bicg_p(int n, StateOf<V> *st, V *__restrict__ p,
                                                      const V *__restrict__ r, const V *__restrict__ v,
                                                      int *total_iters) {
    using A = Ar<V>;
    pdl_wait();
    pdl_release();
    if (*(volatile int *)&st->done) return;
    const typename A::S beta = A::scal(st->beta), omega = A::scal(st->omega);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->iter += 1;
        if (total_iters) *total_iters += 1;
        if (cis_zero(st->rho)) { st->status = HZ_BREAKDOWN; st->done = 1; }
    }
    vec_tiles_staged(
        n, [&](int i) { return In3<V>{r[i], p[i], v[i]}; },
        [&](int i, const In3<V> &q) { p[i] = A::axpy(q.a, beta, A::axmy(q.b, omega, q.c)); });
}

// F2 epilogue: v = A p, sigma = <rh, v>, alpha = rho / sigma
template <class V>
struct EpiSigma : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 2;
    StateOf<V> *st;
    V *v;
    const V *rh;
    __device__ bool skip() const { return st->done; }
    using Pre = V;   // rh[i], fetched ahead by the block-flat kernel
    __device__ V pre(int i) const { return rh[i]; }
    double s;   // operator scale (double-float path; 1 in binary64)
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N], const V &rhi) const {
        if constexpr (Ar<V>::kFF) y = Ar<V>::pow2(y, s);
        v[i] = y;
        Ar<V>::dotc(acc[0], acc[1], rhi, y);
    }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const { row(i, y, acc, rh[i]); }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        const auto sig = cmk(tot[0], tot[1]);
        if (cis_zero(sig)) { st->status = HZ_BREAKDOWN; st->done = 1; return; }
        st->alpha = cdiv(st->rho, sig);
    }
};

// F3: s = r - alpha v and ||s||; half-step exit test
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_bicg_s(int n, StateOf<V> *st, const Ctl *ctl, V *__restrict__ s,
                                                      const V *__restrict__ r, const V *__restrict__ v,
                                                      RedScratch red, int outer_level) {
    using A = Ar<V>;
    pdl_wait();
    pdl_release();
    if (st->done) return;
    const typename A::S alpha = A::scal(st->alpha);
    typename A::Acc acc[1];
    A::acc_zero(acc[0]);
    vec_tiles_staged(
        n, [&](int i) { return In2<V>{r[i], v[i]}; },
        [&](int i, const In2<V> &q) {
            const V o = A::axmy(q.a, alpha, q.b);
            s[i] = o;
            A::nrm2(acc[0], o);
        });
    typename A::R tot[1];
    if (vec_reduce<V, 1>(acc, red, tot) && threadIdx.x == 0) {
        const double ss = (double)tot[0];
        const double rel = sqrt(ss) / st->nb;
        st->ss = ss;
        if (!finite_d(rel)) { st->status = HZ_ERR_NAN; st->done = 1; st->rel = rel; return; }
        if (outer_level ? rel <= ctl->tol : (float)rel <= st->tol32) {
            st->half = 1;
            st->rel = rel;
        }
    }
}

// F4 epilogue: t = A s, <t, s>, <t, t>, omega = <t, s> / <t, t>
template <class V>
struct EpiOmega : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 3;
    StateOf<V> *st;
    V *t;
    const V *s;
    __device__ bool skip() const { return st->done || st->half; }
    using Pre = V;   // s[i], fetched ahead by the block-flat kernel
    __device__ V pre(int i) const { return s[i]; }
    double sc;   // operator scale (double-float path; 1 in binary64)
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N], const V &si) const {
        if constexpr (Ar<V>::kFF) y = Ar<V>::pow2(y, sc);
        t[i] = y;
        Ar<V>::dotc(acc[0], acc[1], y, si);
        Ar<V>::nrm2(acc[2], y);
    }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const { row(i, y, acc, s[i]); }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        if (tot[2] == R(0)) { st->status = HZ_BREAKDOWN; st->done = 1; return; }
        st->omega = cmk(tot[0] / tot[2], tot[1] / tot[2]);
    }
};

// F5: x += alpha p + omega s, r = s - omega t, rho' = <rh, r>, ||r||; loop test.
// It reads five vectors: four elements per thread in flight (not eight) and
// two resident blocks per SM keep its registers at 128, so the whole grid is
// resident at once (eight elements took 208 registers, one block per SM and
// two waves: 143.4 vs 138.8 us per C2 iteration)
constexpr int kXrUnroll = 4;
template <class V>
__global__ void __launch_bounds__(kVecBlock, 2) k_bicg_xr(int n, StateOf<V> *st, const Ctl *ctl, V *__restrict__ x,
                                                       V *__restrict__ r, const V *__restrict__ rh,
                                                       const V *__restrict__ p, const V *__restrict__ s,
                                                       const V *__restrict__ t, const int *total_iters,
                                                       RedScratch red, int outer_level) {
    using A = Ar<V>;
    pdl_wait();
    pdl_release();
    if (st->done) return;
    const typename A::S alpha = A::scal(st->alpha);
    if (st->half) {   // half-step exit: x += alpha p, r = s
        vec_tiles(n, [&](int i) {
            x[i] = A::axpy(x[i], alpha, p[i]);
            r[i] = s[i];
        });
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->status = HZ_OK;
            st->done = 1;
            if (outer_level && ctl->hist) ctl->hist[st->iter] = st->rel;
        }
        return;
    }
    const auto omega_st = st->omega;
    const typename A::S omega = A::scal(omega_st);
    typename A::Acc acc[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) A::acc_zero(acc[j]);
    vec_tiles_staged<kXrUnroll>(
        n, [&](int i) { return In5<V>{s[i], x[i], p[i], t[i], rh[i]}; },
        [&](int i, const In5<V> &q) {
            x[i] = A::axpy(A::axpy(q.b, alpha, q.c), omega, q.a);
            const V ri = A::axmy(q.a, omega, q.d);
            r[i] = ri;
            A::dotc(acc[0], acc[1], q.e, ri);
            A::nrm2(acc[2], ri);
        });
    typename A::R tot[3];
    if (vec_reduce<V, 3>(acc, red, tot) && threadIdx.x == 0) {
        const double rel = sqrt((double)tot[2]) / st->nb;
        const int it = st->iter;
        st->rel = rel;
        if (outer_level && ctl->hist) ctl->hist[it] = rel;
        const int maxit = outer_level ? ctl->maxit : st->maxit;
        const bool conv = outer_level ? rel <= ctl->tol : (float)rel <= st->tol32;
        if (!finite_d(rel)) { st->status = HZ_ERR_NAN; st->done = 1; }
        else if (conv) { st->status = HZ_OK; st->done = 1; }
        else if (cis_zero(omega_st)) { st->status = HZ_BREAKDOWN; st->done = 1; }
        else if (it >= maxit || (!outer_level && total_iters && *total_iters >= ctl->maxit)) {
            st->status = HZ_NOT_CONVERGED; st->done = 1;
        } else {
            const auto rn = cmk(tot[0], tot[1]);
            st->beta = cmul(cdiv(rn, st->rho), cdiv(st->alpha, omega_st));
            st->rho_old = st->rho;
            st->rho = rn;
        }
    }
}

// init epilogue: r = b - A x, rh = r, p = v = 0, ||r||^2, ||b||^2
template <class V>
struct EpiInit : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 2;
    StateOf<V> *st;
    Info *info;
    const Ctl *ctl;
    V *r, *rh, *p, *v;
    cudaGraphConditionalHandle h;
    __device__ bool skip() const { return false; }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const {
        const V bi = Ar<V>::from_c128(zscale(ctl->b[i], rhs_scale(ctl)));
        const V ri = Ar<V>::sub(bi, Ar<V>::pow2(y, ctl->op_scale));
        r[i] = ri;
        rh[i] = ri;
        p[i] = Ar<V>::zero();
        v[i] = Ar<V>::zero();
        Ar<V>::nrm2(acc[0], ri);
        Ar<V>::nrm2(acc[1], bi);
    }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        const bool restart = ctl->restart != 0;
        const double nb = sqrt((double)tot[1]);
        st->nb = nb;
        st->half = 0;
        if (!restart) { st->iter = 0; info->zero_x = 0; }
        const double2 one = make_double2(1.0, 0.0);
        st->rho = make_double2((double)tot[0], 0.0);
        st->rho_old = one; st->alpha = one; st->omega = one;
        st->beta = make_double2(0.0, 0.0);
        if (nb == 0.0) {
            st->rel = 0.0; st->status = HZ_OK; st->done = 1; info->zero_x = 1;
            if (ctl->hist && !restart) ctl->hist[0] = 0.0;
        } else {
            const double rel = sqrt((double)tot[0]) / nb;
            st->rel = rel;
            if (ctl->hist && !restart) ctl->hist[0] = rel;
            st->done = 1;
            if (!finite_d(rel)) st->status = HZ_ERR_NAN;
            else if (rel <= ctl->tol) st->status = HZ_OK;
            else if (st->iter >= ctl->maxit) st->status = HZ_NOT_CONVERGED;
            else { st->status = HZ_NOT_CONVERGED; st->done = 0; }
        }
        set_cond(h, st->done ? 0 : 1);
    }
};

// ---------------------------------------------------------------------------
// mixed precision: outer residual in complex128 (binary64 or double-float),
// written as the complex64 right-hand side of the inner solve (d = 0)
template <class V>
struct EpiOuter : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 3;
    OuterState *ost;
    BiState<float2> *in;
    Info *info;
    const Ctl *ctl;
    float2 *r, *rh, *p, *v, *d;
    const int *total_inner;
    cudaGraphConditionalHandle h_outer, h_inner;
    __device__ bool skip() const { return false; }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const {
        const V bi = Ar<V>::from_c128(ctl->b[i]);
        const V ri = Ar<V>::sub(bi, y);
        const float2 r32 = to_c64(Ar<V>::to_c128(ri));
        r[i] = r32;
        rh[i] = r32;
        p[i] = make_float2(0.f, 0.f);
        v[i] = make_float2(0.f, 0.f);
        d[i] = make_float2(0.f, 0.f);
        Ar<V>::nrm2(acc[0], ri);
        Ar<V>::nrm2(acc[1], bi);
        Ar<V>::nrm2(acc[2], Ar<V>::from_c128(to_c128(r32)));
    }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        const double nb = sqrt((double)tot[1]);
        ost->nb = nb;
        bool done = true;
        if (nb == 0.0) {
            ost->rel = 0.0; ost->status = HZ_OK; ost->zero_x = 1;
            if (ctl->hist) ctl->hist[ost->outer] = 0.0;
        } else {
            // the refinement keeps the iterate with the smallest outer
            // residual and stops as soon as a step fails to reduce it: the
            // answer is then that best iterate, not the last one
            const double rel = sqrt((double)tot[0]) / nb;
            const double best = ost->rel_best;
            ost->rel = rel;
            if (ctl->hist) ctl->hist[ost->outer] = rel;
            ost->save = 0;
            if (!finite_d(rel)) { ost->status = HZ_ERR_NAN; ost->use_best = ost->outer > 0; }
            else if (rel <= ctl->tol) ost->status = HZ_OK;
            else if (rel >= best) { ost->status = HZ_NOT_CONVERGED; ost->use_best = 1; }
            else if (ost->outer >= ctl->max_outer || *total_inner >= ctl->maxit) ost->status = HZ_NOT_CONVERGED;
            else {
                done = false;
                ost->rel_best = rel;
                ost->save = 1;   // x is the best so far: k_mixed_update keeps a copy
            }
        }
        ost->done = done ? 1 : 0;
        if (!done) {
            ost->outer += 1;
            const float2 one = make_float2(1.f, 0.f);
            in->rho = make_float2((float)tot[2], 0.f);
            in->rho_old = one; in->alpha = one; in->omega = one;
            in->beta = make_float2(0.f, 0.f);
            in->nb = (double)sqrtf((float)tot[2]);
            in->rel = 1.0;
            in->tol32 = ctl->inner_tol;
            in->maxit = ctl->inner_maxit;
            in->iter = 0; in->half = 0; in->status = HZ_NOT_CONVERGED;
            in->done = (in->nb == 0.0) ? 1 : 0;
        } else {
            in->done = 1;
        }
        set_cond(h_inner, (!done && !in->done) ? 1 : 0);
        set_cond(h_outer, done ? 0 : 1);
    }
};

// last node of the refinement loop body: the outer loop goes on only while
// the refinement state is not done and the body has run at most
// max_outer + 1 times (the cap that EpiOuter itself enforces)
__global__ void k_outer_guard(OuterState *ost, const Ctl *ctl, cudaGraphConditionalHandle h) {
    const int runs = ost->guard + 1;
    const bool go = !ost->done && runs <= ctl->max_outer + 1;
    if (!go && !ost->done) {
        ost->status = HZ_NOT_CONVERGED;
        ost->done = 1;
    }
    ost->guard = go ? runs : 0;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

template <class V>
__global__ void __launch_bounds__(kVecBlock) k_mixed_start(int n, const Ctl *ctl, OuterState *ost, int *total_inner,
                                                           V *__restrict__ xw) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ost->outer = 0; ost->done = 0; ost->status = HZ_NOT_CONVERGED; ost->zero_x = 0;
        ost->rel_best = INFINITY; ost->save = 0; ost->use_best = 0; ost->guard = 0;
        *total_inner = 0;
    }
    const double2 *x0 = ctl->x, *pd = ctl->pre_d;
    const bool zero = ctl->x0_zero != 0;
    vec_tiles(n, [&](int i) { xw[i] = zero ? Ar<V>::zero() : Ar<V>::from_c128(pd ? cmul(x0[i], pd[i]) : x0[i]); });
}

// x += d (d from the complex64 inner solve); when the refinement marked the
// current x as its best iterate so far, x is first copied to xb
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_mixed_update(int n, const OuterState *ost, V *__restrict__ xw,
                                                            V *__restrict__ xb, const float2 *__restrict__ d) {
    if (ost->done) return;
    const bool save = ost->save != 0;
    vec_tiles(n, [&](int i) {
        const V xi = xw[i];
        if (save) xb[i] = xi;
        xw[i] = Ar<V>::sub(xi, Ar<V>::from_c128(to_c128(make_float2(-d[i].x, -d[i].y))));
    });
}

// copy-out of the refinement: the answer is the current x, or the kept best
// iterate when the last step did not reduce the outer residual; the info
// block is written from the refinement state
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_mixed_copy_out(int n, const Ctl *ctl, const OuterState *ost,
                                                              const int *total_inner, Info *info,
                                                              const V *__restrict__ xw, const V *__restrict__ xb,
                                                              const int *fault) {
    const bool best = ost->use_best != 0, zero = ost->zero_x != 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        info->iters = *total_inner;
        info->status = ost->status;
        info->outer = ost->outer;
        info->relres_rec = info->relres_true = best ? ost->rel_best : ost->rel;
        info->zero_x = ost->zero_x;
        // an expired bounded wait in an SpMV of this solve voids the result
        if (fault && *(volatile const int *)fault) info->status = HZ_ERR_TIMEOUT;
    }
    double2 *x = ctl->x;
    const double2 *pdi = ctl->pre_dinv;
    const V *src = best ? xb : xw;
    vec_tiles(n, [&](int i) {
        const double2 y = Ar<V>::to_c128(src[i]);
        x[i] = zero ? make_double2(0.0, 0.0) : (pdi ? cmul(y, pdi[i]) : y);
    });
}

// ---------------------------------------------------------------------------
struct Solver {
    int mode = 0;
    int n = 0;
    int kind = 0, group = 4;
    int grid_spmv = 1, grid_vec = 1;
    int grid_spmv_cv = 1;   // grid of the binary64/complex64 CSR or SELL kernels
    int grid_c64 = 1;       // grid of the block-flat complex64 kernel
    double op_scale = 1.0;  // double-float BiCGStab: the iteration runs on op_scale * A
    bool pdl = false;       // programmatic dependent launches inside the iteration
    void *x = nullptr, *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr;
    void *xbest = nullptr;  // mixed: the refinement's best iterate
    float2 *r32 = nullptr, *rh32 = nullptr, *p32 = nullptr, *v32 = nullptr, *s32 = nullptr, *t32 = nullptr,
           *d32 = nullptr;
    BiState<double2> *st = nullptr;
    BiState<float2> *st32 = nullptr;
    OuterState *ost = nullptr;
    Info *dinfo = nullptr;
    Ctl *dctl = nullptr;
    int *total = nullptr;
    Ctl *hctl = nullptr;    // pinned
    Info *hinfo = nullptr;  // pinned
    RedScratch red{};
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void solver_free(Solver *S) {
    if (!S) return;
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->cap) cudaStreamDestroy(S->cap);
    void *dev[] = {S->x, S->xbest, S->r, S->rh, S->p, S->v, S->s, S->t, S->r32, S->rh32, S->p32, S->v32, S->s32, S->t32,
                   S->d32, S->st, S->st32, S->ost, S->dinfo, S->dctl, S->total, S->red.partials, S->red.counter};
    for (void *q : dev) cudaFree(q);
    cudaFreeHost(S->hctl);
    cudaFreeHost(S->hinfo);
    delete S;
}

void free_solvers(hz_mat *A) {
    for (int m = 0; m < 2; ++m) {
        solver_free((Solver *)A->solver[m]);
        A->solver[m] = nullptr;
    }
    bl_solver_free(A->solver_bl);
    A->solver_bl = nullptr;
    tq_solver_free(A->solver_tq);
    A->solver_tq = nullptr;
}

#define HZ_ALLOC(ptr, bytes) HZ_CUDA(cudaMalloc((void **)&(ptr), std::max<size_t>((bytes), 16)))

static hz_status solver_alloc(Solver *S) {
    const size_t n = (size_t)S->n;
    const size_t vb = 16;   // complex128 and double-float elements are both 16 bytes
    HZ_ALLOC(S->x, n * vb);
    if (S->mode == HZ_MODE_FP64) {
        HZ_ALLOC(S->r, n * vb);
        HZ_ALLOC(S->rh, n * vb);
        HZ_ALLOC(S->p, n * vb);
        HZ_ALLOC(S->v, n * vb);
        HZ_ALLOC(S->s, n * vb);
        HZ_ALLOC(S->t, n * vb);
    } else {
        HZ_ALLOC(S->xbest, n * vb);
        HZ_ALLOC(S->r32, n * sizeof(float2));
        HZ_ALLOC(S->rh32, n * sizeof(float2));
        HZ_ALLOC(S->p32, n * sizeof(float2));
        HZ_ALLOC(S->v32, n * sizeof(float2));
        HZ_ALLOC(S->s32, n * sizeof(float2));
        HZ_ALLOC(S->t32, n * sizeof(float2));
        HZ_ALLOC(S->d32, n * sizeof(float2));
    }
    HZ_ALLOC(S->st, sizeof(BiState<double2>));
    HZ_ALLOC(S->st32, sizeof(BiState<float2>));
    HZ_ALLOC(S->ost, sizeof(OuterState));
    HZ_ALLOC(S->dinfo, sizeof(Info));
    HZ_ALLOC(S->dctl, sizeof(Ctl));
    HZ_ALLOC(S->total, sizeof(int));
    HZ_ALLOC(S->red.partials, sizeof(double) * kMaxRedBlocks * kMaxRedValues);
    HZ_ALLOC(S->red.counter, 256);
    HZ_CUDA(cudaMemset(S->red.counter, 0, 256));
    HZ_CUDA(cudaMemset(S->st, 0, sizeof(BiState<double2>)));
    HZ_CUDA(cudaMemset(S->st32, 0, sizeof(BiState<float2>)));
    HZ_CUDA(cudaMemset(S->dinfo, 0, sizeof(Info)));
    HZ_CUDA(cudaMallocHost((void **)&S->hctl, sizeof(Ctl)));
    HZ_CUDA(cudaMallocHost((void **)&S->hinfo, sizeof(Info)));
    memset(S->hctl, 0, sizeof(Ctl));
    memset(S->hinfo, 0, sizeof(Info));
    HZ_CUDA(cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking));
    HZ_CUDA(cudaDeviceSynchronize());
    return HZ_OK;
}

// one SpMV with epilogue, on the kernel family of the vector element type
template <class V, class Epi>
static void spmv_on(const Solver *S, const hz_mat *A, const V *x, const Epi &e, cudaStream_t cs,
                    bool pdl = false) {
    if constexpr (std::is_same<V, float4>::value) {
        launch_spmv_ff(S->kind, S->group, mat_view<double2>(A), x, e, S->red, S->grid_spmv, cs, pdl);
    } else if constexpr (std::is_same<V, float2>::value) {
        // complex64 inner operator: block-flat when the handle runs a block-flat kind
        if (A->fblk && is_flat64(d64_kind(A, S->kind)))
            launch_k(pdl, k_spmv_c64b<Epi>, S->grid_c64, kFlatThreads, cs, mat_view<float2>(A), x, e, S->red);
        else
            launch_spmv<V>(d64_kind(A, S->kind),
                           S->group, mat_view<V>(A), x, e, S->red, S->grid_spmv_cv, cs, pdl);
    } else {
        launch_spmv<V>(d64_kind(A, S->kind), S->group, mat_view<V>(A), x, e, S->red,
                       S->grid_spmv_cv, cs, pdl);
    }
}

template <class V>
static void launch_iteration(const Solver *S, const hz_mat *A, StateOf<V> *st, V *x, V *r, V *rh, V *p, V *v, V *s,
                             V *t, int *total, int outer_level, cudaStream_t cs) {
    // with S->pdl, F2..F5 are launched as programmatic dependents of their
    // predecessor: each kernel's CTAs may be scheduled while the previous one
    // drains and wait in pdl_wait() for its results
    const int n = S->n;
    const bool pdl = S->pdl;
    launch_k(false, k_bicg_p<V>, S->grid_vec, kVecBlock, cs, n, st, p, r, v, total);
    EpiSigma<V> e2;
    e2.st = st; e2.v = v; e2.rh = rh; e2.s = S->op_scale;
    spmv_on<V>(S, A, p, e2, cs, pdl);
    launch_k(pdl, k_bicg_s<V>, S->grid_vec, kVecBlock, cs, n, st, (const Ctl *)S->dctl, s, r, v, S->red,
             outer_level);
    EpiOmega<V> e4;
    e4.st = st; e4.t = t; e4.s = s; e4.sc = S->op_scale;
    spmv_on<V>(S, A, s, e4, cs, pdl);
    launch_k(pdl, k_bicg_xr<V>, S->grid_vec, kVecBlock, cs, n, st, (const Ctl *)S->dctl, x, r, rh, p, s, t,
             (const int *)total, S->red, outer_level);
}

// FP64-mode graph: start -> WHILE{F1..F5} -> true residual, copy-out, info
template <class V>
static hz_status build_fp64_graph(Solver *S, const hz_mat *A, cudaGraph_t g) {
    cudaStream_t cs = S->cap;
    const auto mode = cudaStreamCaptureModeThreadLocal;
    const int n = S->n;
    std::vector<cudaGraphNode_t> leaves;
    V *x = (V *)S->x, *r = (V *)S->r, *rh = (V *)S->rh, *p = (V *)S->p, *v = (V *)S->v, *s = (V *)S->s,
      *t = (V *)S->t;
    StateOf<V> *st = (StateOf<V> *)S->st;
    // HZ_PROFILE_UNROLL=k: k straight-line copies of the iteration (krylov.cuh)
    const int unroll = profile_unroll();
    cudaGraphConditionalHandle h = 0;
    if (unroll <= 0) HZ_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, mode));
    cudaMemcpyAsync(S->dctl, S->hctl, sizeof(Ctl), cudaMemcpyHostToDevice, cs);
    // double-float: scale the right-hand side to O(1) (binary32 exponent range)
    if constexpr (Ar<V>::kFF) k_bmax<<<S->grid_vec, 256, 0, cs>>>(n, S->dctl);
    k_init_x<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->dctl, x);
    EpiInit<V> ei;
    ei.st = st; ei.info = S->dinfo; ei.ctl = S->dctl; ei.r = r; ei.rh = rh; ei.p = p; ei.v = v; ei.h = h;
    spmv_on<V>(S, A, x, ei, cs);
    if (unroll > 0) {
        for (int k = 0; k < unroll; ++k) launch_iteration<V>(S, A, st, x, r, rh, p, v, s, t, nullptr, 1, cs);
    } else {
        HZ_TRY(capture_leaves(cs, &leaves));
        HZ_CUDA(cudaStreamEndCapture(cs, &g));
        cudaGraphNode_t wn;
        cudaGraph_t body;
        HZ_TRY(add_while(g, leaves, h, &wn, &body));
        HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, mode));
        launch_iteration<V>(S, A, st, x, r, rh, p, v, s, t, nullptr, 1, cs);
        k_loop_guard<typename Ar<V>::St><<<1, 1, 0, cs>>>(st, S->dctl, 1, h);
        HZ_CUDA(cudaStreamEndCapture(cs, &body));
        HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, g, &wn, nullptr, 1, mode));
    }
    EpiTrue<V> et;
    et.st = st; et.info = S->dinfo; et.ctl = S->dctl;
    spmv_on<V>(S, A, x, et, cs);
    k_copy_out<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->dctl, S->dinfo, x, A->fault);
    cudaMemcpyAsync(S->hinfo, S->dinfo, sizeof(Info), cudaMemcpyDeviceToHost, cs);
    HZ_CUDA(cudaStreamEndCapture(cs, &g));
    return HZ_OK;
}

// mixed-mode graph: start -> WHILE_outer{ residual -> WHILE_inner{F1..F5} -> x += d } -> copy-out, info
template <class V>
static hz_status build_mixed_graph(Solver *S, const hz_mat *A, cudaGraph_t g) {
    cudaStream_t cs = S->cap;
    const auto mode = cudaStreamCaptureModeThreadLocal;
    const int n = S->n;
    std::vector<cudaGraphNode_t> leaves;
    V *x = (V *)S->x;
    const int unroll = profile_unroll();
    cudaGraphConditionalHandle ho = 0, hi = 0;
    if (unroll <= 0) HZ_CUDA(cudaGraphConditionalHandleCreate(&ho, g, 1, cudaGraphCondAssignDefault));
    HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, mode));
    cudaMemcpyAsync(S->dctl, S->hctl, sizeof(Ctl), cudaMemcpyHostToDevice, cs);
    k_mixed_start<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->dctl, S->ost, S->total, x);
    if (unroll > 0) {   // one refinement step with `unroll` inner iterations, straight-line
        EpiOuter<V> eo;
        eo.ost = S->ost; eo.in = S->st32; eo.info = S->dinfo; eo.ctl = S->dctl; eo.r = S->r32; eo.rh = S->rh32;
        eo.p = S->p32; eo.v = S->v32; eo.d = S->d32; eo.total_inner = S->total; eo.h_outer = 0; eo.h_inner = 0;
        spmv_on<V>(S, A, x, eo, cs);
        for (int k = 0; k < unroll; ++k)
            launch_iteration<float2>(S, A, S->st32, S->d32, S->r32, S->rh32, S->p32, S->v32, S->s32, S->t32,
                                     S->total, 0, cs);
        k_mixed_update<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->ost, x, (V *)S->xbest, S->d32);
        k_mixed_copy_out<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->dctl, S->ost, S->total, S->dinfo, x,
                                                              (const V *)S->xbest, A->fault);
        cudaMemcpyAsync(S->hinfo, S->dinfo, sizeof(Info), cudaMemcpyDeviceToHost, cs);
        HZ_CUDA(cudaStreamEndCapture(cs, &g));
        return HZ_OK;
    }
    HZ_TRY(capture_leaves(cs, &leaves));
    HZ_CUDA(cudaStreamEndCapture(cs, &g));
    cudaGraphNode_t wo;
    cudaGraph_t obody;
    HZ_TRY(add_while(g, leaves, ho, &wo, &obody));
    HZ_CUDA(cudaGraphConditionalHandleCreate(&hi, obody, 0, 0));
    HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, obody, nullptr, nullptr, 0, mode));
    EpiOuter<V> eo;
    eo.ost = S->ost; eo.in = S->st32; eo.info = S->dinfo; eo.ctl = S->dctl; eo.r = S->r32; eo.rh = S->rh32;
    eo.p = S->p32; eo.v = S->v32; eo.d = S->d32; eo.total_inner = S->total; eo.h_outer = ho; eo.h_inner = hi;
    spmv_on<V>(S, A, x, eo, cs);
    HZ_TRY(capture_leaves(cs, &leaves));
    HZ_CUDA(cudaStreamEndCapture(cs, &obody));
    cudaGraphNode_t wi;
    cudaGraph_t ibody;
    HZ_TRY(add_while(obody, leaves, hi, &wi, &ibody));
    HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, ibody, nullptr, nullptr, 0, mode));
    launch_iteration<float2>(S, A, S->st32, S->d32, S->r32, S->rh32, S->p32, S->v32, S->s32, S->t32, S->total, 0,
                             cs);
    k_loop_guard<float2><<<1, 1, 0, cs>>>(S->st32, S->dctl, 0, hi);
    HZ_CUDA(cudaStreamEndCapture(cs, &ibody));
    HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, obody, &wi, nullptr, 1, mode));
    k_mixed_update<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->ost, x, (V *)S->xbest, S->d32);
    k_outer_guard<<<1, 1, 0, cs>>>(S->ost, S->dctl, ho);
    HZ_CUDA(cudaStreamEndCapture(cs, &obody));
    HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, g, &wo, nullptr, 1, mode));
    k_mixed_copy_out<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->dctl, S->ost, S->total, S->dinfo, x,
                                                          (const V *)S->xbest, A->fault);
    cudaMemcpyAsync(S->hinfo, S->dinfo, sizeof(Info), cudaMemcpyDeviceToHost, cs);
    HZ_CUDA(cudaStreamEndCapture(cs, &g));
    return HZ_OK;
}

static hz_status build_graph(Solver *S, const hz_mat *A) {
    cudaGraph_t g;
    HZ_CUDA(cudaGraphCreate(&g, 0));
    S->graph = g;
    const bool ff = is_ff_kind(S->kind);
    if (S->mode == HZ_MODE_FP64)
        HZ_TRY(ff ? build_fp64_graph<float4>(S, A, g) : build_fp64_graph<double2>(S, A, g));
    else
        HZ_TRY(ff ? build_mixed_graph<float4>(S, A, g) : build_mixed_graph<double2>(S, A, g));
    HZ_CUDA(cudaGraphInstantiate(&S->exec, g, 0));
    return HZ_OK;
}

static hz_status get_solver(hz_mat *A, uint32_t mode, cudaStream_t s, Solver **out) {
    Solver *S = (Solver *)A->solver[mode];
    if (S && (S->kind != A->spmv_kind || S->group != A->group)) {   // variant changed: rebuild
        solver_free(S);
        A->solver[mode] = S = nullptr;
    }
    if (!S) {
        if (mode == HZ_MODE_MIXED) HZ_TRY(ensure_c64(A, s));
        DevInfo d;
        HZ_TRY(dev_info(&d));
        S = new Solver();
        S->mode = (int)mode;
        S->n = A->n;
        S->kind = A->spmv_kind;
        S->group = A->group;
        S->grid_spmv = spmv_grid(A, S->kind, S->group);
        S->grid_spmv_cv = spmv_grid(A, d64_kind(A, S->kind), S->group);
        if (A->fblk) {
            // the CTAs of both complex64 products of the iteration that fit
            // at once: a grid sized for another epilogue's instantiation
            // would run a partial second wave if these held more registers
            int o1 = 0, o2 = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_spmv_c64b<EpiSigma<float2>>, kFlatThreads, 0) !=
                    cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_spmv_c64b<EpiOmega<float2>>, kFlatThreads, 0) !=
                    cudaSuccess)
                o1 = o2 = 1;
            const int64_t g = std::min<int64_t>(A->nfblk, (int64_t)d.num_sms * std::max(1, std::min(o1, o2)));
            S->grid_c64 = (int)std::max<int64_t>(1, std::min<int64_t>(g, kMaxRedBlocks));
        }
        // HZ_PDL=1 (environment) captures F2..F5 as programmatic dependent
        // launches; measured no faster on a 24^3 box (41.5 vs 41.9 us per
        // iteration) and slower on a 64^3 box (99 vs 93 us) and on C2
        // (191 vs 187 us), so plain launches are the default
        const char *pdl_env = getenv("HZ_PDL");
        S->pdl = pdl_env && atoi(pdl_env) != 0;
        S->grid_vec = vec_grid(d, A->n);
        hz_status st = HZ_OK;
        // the double-float iteration runs on A scaled to unit size, so that
        // A p and A s stay inside the binary32 exponent range
        if (mode == HZ_MODE_FP64 && is_ff_kind(S->kind)) st = operator_scale(A, &S->op_scale);
        if (st == HZ_OK) st = solver_alloc(S);
        if (st == HZ_OK) st = build_graph(S, A);
        if (st != HZ_OK) { solver_free(S); return st; }
        A->solver[mode] = S;
    }
    *out = S;
    return HZ_OK;
}

}  // namespace hz

using namespace hz;

extern "C" HZ_API hz_status hz_zsolve_opts(hz_mat *A, const hz_z *d_b, hz_z *d_x, const hz_solve_opts *o,
                                           hz_info *h_info, void *stream) {
    HZ_CHECK(A && o && h_info, "hz_zsolve: null argument");
    HZ_CHECK(o->mode == HZ_MODE_FP64 || o->mode == HZ_MODE_MIXED, "hz_zsolve: unknown mode");
    HZ_CHECK(o->maxit >= 0, "hz_zsolve: negative maxit");
    HZ_CHECK(o->tol >= 0.0, "hz_zsolve: negative tol");
    HZ_CHECK(o->precond == HZ_PRECOND_NONE || o->precond == HZ_PRECOND_JACOBI, "hz_zsolve: unknown preconditioner");
    HZ_CHECK(o->method == HZ_METHOD_BICGSTAB || o->method == HZ_METHOD_BICGSTABL || o->method == HZ_METHOD_TFQMR,
             "hz_zsolve: unknown method");
    HZ_CHECK(o->method != HZ_METHOD_BICGSTABL || (o->ell >= 1 && o->ell <= 8), "hz_zsolve: ell must be in 1..8");
    HZ_CHECK(o->method == HZ_METHOD_BICGSTAB || o->mode == HZ_MODE_FP64,
             "hz_zsolve: the mixed mode runs BiCGStab only");
    *h_info = hz_info{};
    if (A->n == 0) { h_info->status = HZ_OK; return HZ_OK; }
    HZ_CHECK(d_b && d_x, "hz_zsolve: null vector");
    cudaStream_t s = (cudaStream_t)stream;
    hz_mat *op = A;   // the operator the iteration runs on
    if (o->precond == HZ_PRECOND_JACOBI) {
        HZ_TRY(ensure_jacobi(A, s));
        op = A->jac;
        op->spmv_kind = A->spmv_kind;   // follow the caller's choice of SpMV variant
        op->group = A->group;
    }
    Ctl c{};
    c.tol = o->tol;
    c.b = (const double2 *)d_b;
    c.x = (double2 *)d_x;
    c.hist = o->d_hist;
    c.maxit = o->maxit;
    c.restart = 0;
    c.x0_zero = o->x0_is_zero ? 1 : 0;
    c.max_outer = o->max_outer > 0 ? o->max_outer : 50;
    c.inner_tol = o->inner_tol > 0.f ? o->inner_tol : 1e-5f;
    c.inner_maxit = o->inner_maxit > 0 ? o->inner_maxit : 1000;
    c.pre_d = op != A ? A->jac_d : nullptr;
    c.pre_dinv = op != A ? A->jac_dinv : nullptr;
    c.op_scale = 1.0;
    if (o->method == HZ_METHOD_BICGSTABL || o->method == HZ_METHOD_TFQMR) {
        Info inf{};
        int restarts = 0;
        if (o->method == HZ_METHOD_BICGSTABL) HZ_TRY(bl_solve(op, o->ell, c, &inf, &restarts, s));
        else HZ_TRY(tq_solve(op, c, &inf, &restarts, s));
        if (inf.status == HZ_OK && inf.relres_true > o->tol) inf.status = HZ_NOT_CONVERGED;
        h_info->iters = inf.iters;
        h_info->status = inf.status;
        h_info->restarts = restarts;
        h_info->outer = 0;
        h_info->relres_rec = inf.relres_rec;
        h_info->relres_true = inf.relres_true;
        return (hz_status)inf.status;
    }
    Solver *S = nullptr;
    HZ_TRY(get_solver(op, o->mode, s, &S));
    *S->hctl = c;
    S->hctl->op_scale = S->op_scale;
    HZ_CUDA(cudaGraphLaunch(S->exec, s));
    HZ_CUDA(cudaStreamSynchronize(s));
    Info inf = *S->hinfo;
    int restarts = 0;
    if (o->mode == HZ_MODE_FP64 && inf.status == HZ_OK && inf.relres_true > o->tol && inf.iters < o->maxit) {
        S->hctl->restart = 1;
        restarts = 1;
        HZ_CUDA(cudaGraphLaunch(S->exec, s));
        HZ_CUDA(cudaStreamSynchronize(s));
        inf = *S->hinfo;
    }
    if (inf.status == HZ_OK && inf.relres_true > o->tol) inf.status = HZ_NOT_CONVERGED;
    h_info->iters = inf.iters;
    h_info->status = inf.status;
    h_info->restarts = restarts;
    h_info->outer = inf.outer;
    h_info->relres_rec = inf.relres_rec;
    h_info->relres_true = inf.relres_true;
    return (hz_status)inf.status;
}

extern "C" HZ_API hz_status hz_zsolve(hz_mat *A, const hz_z *d_b, hz_z *d_x, double tol, int32_t maxit,
                                      uint32_t mode, hz_info *h_info, void *stream) {
    hz_solve_opts o{};
    o.tol = tol;
    o.maxit = maxit;
    o.mode = mode;
    return hz_zsolve_opts(A, d_b, d_x, &o, h_info, stream);
}
