// krylov.cuh -- pieces shared by the device-resident Krylov solvers
// (BiCGStab, BiCGStab(l), TFQMR): the host control block uploaded by each
// solve graph, per-system state and info blocks, the vector-kernel tile
// walkers, the fused-reduction plumbing, the start / true-residual /
// copy-out steps and the CUDA-graph capture helpers.
#pragma once

#include <cstdlib>
#include <vector>

#include "spmv.cuh"

namespace hz {

constexpr int kVecBlock = 256;
#ifndef HZ_VEC_UNROLL
#define HZ_VEC_UNROLL 8
#endif
constexpr int kVecUnroll = HZ_VEC_UNROLL;   // elements per thread per tile of the vector kernels

// host-written controls of one solve (uploaded by the graph itself)
struct Ctl {
    double tol;
    const double2 *b;
    double2 *x;
    double *hist;
    int maxit;
    int restart;
    int x0_zero;
    int max_outer;
    float inner_tol;
    int inner_maxit;
    const double2 *pre_d;      // Jacobi: y0 = D x0 (null without a preconditioner)
    const double2 *pre_dinv;   // Jacobi: x = D^-1 y
    double op_scale;           // s = 2^-k: the iteration runs on s A (x0 -> x0 / s, x -> s y); 1 = unscaled
    // largest |Re b_i|, |Im b_i| as the bits of a non-negative double, written
    // on the device by k_bmax (0: no scaling).  With it the iteration solves
    // (s A) y = c b for c = 2^-e, 2^(e-1) <= max |b| < 2^e, so that the
    // right-hand side and the residuals are O(1) whatever the size of b.
    unsigned long long bmax_bits;
};

// c of the right-hand-side scaling above (a power of two: exact in binary64)
__device__ __forceinline__ double rhs_scale(const Ctl *c) {
    const double m = __longlong_as_double((long long)c->bmax_bits);
    if (!(m > 0.0) || !isfinite(m)) return 1.0;
    int e;
    frexp(m, &e);
    return ldexp(1.0, -e);
}

__device__ __forceinline__ double2 zscale(double2 a, double c) { return make_double2(a.x * c, a.y * c); }

// the largest |Re b_i|, |Im b_i| into ctl->bmax_bits (zero on entry);
// non-negative doubles order like their bit patterns read as unsigned
static __global__ void __launch_bounds__(256) k_bmax(int n, Ctl *ctl) {
    double m = 0.0;
    const double2 *b = ctl->b;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double2 v = b[i];
        m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(&ctl->bmax_bits, (unsigned long long)__double_as_longlong(m));
}

template <class St>
struct BiState {
    St rho, rho_old, alpha, omega, beta;
    double nb;       // ||b|| of this (inner) system
    double rel;      // last recursive residual ratio
    double ss;       // ||s||^2
    float tol32;     // inner tolerance (mixed)
    int maxit;       // inner iteration cap (mixed)
    int iter, done, half, status;
    int guard;       // loop-body runs since the loop began (k_loop_guard; 0 between loops)
};

template <class V> using StateOf = BiState<typename Ar<V>::St>;

struct OuterState {   // mixed-precision refinement state
    double nb, rel;
    double rel_best;  // smallest outer residual ratio so far (its iterate is in the best-x vector)
    int outer, done, status, zero_x;
    int save;         // 1: the current x is the best so far; keep a copy before x += d
    int use_best;     // 1: the answer is the kept copy, not the current x
    int guard;        // outer-loop body runs (k_outer_guard; 0 between solves)
    int pad;
};

struct Info {
    int iters, status, restarts, outer;
    double relres_rec, relres_true;
    int zero_x, pad;
};

// Element walkers of the vector kernels.  Thread t of the T = gridDim.x *
// blockDim.x threads takes elements t, t + T, t + 2T, ..., kVecUnroll (or U)
// of them per pass, so consecutive threads touch consecutive elements and a
// grid larger than n / kVecUnroll threads spreads a short vector over more
// SMs (vec_grid below) instead of leaving its blocks idle.
template <class F>
__device__ __forceinline__ void vec_tiles(int n, F f) {
    const int T = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x + threadIdx.x; base < n; base += kVecUnroll * T) {
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int i = base + u * T;
            if (i < n) f(i);
        }
    }
}

// The same walk issuing every load of a pass before the first compute:
// load(i) returns the element's inputs (indices are clamped to n-1, so the
// loads need no branch), comp(i, in) computes and stores for i < n.
template <int U = kVecUnroll, class Ld, class Cp>
__device__ __forceinline__ void vec_tiles_staged(int n, Ld load, Cp comp) {
    using In = decltype(load(0));
    const int T = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x + threadIdx.x; base < n; base += U * T) {
        In in[U];
#pragma unroll
        for (int u = 0; u < U; ++u) in[u] = load(min(base + u * T, n - 1));
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * T;
            if (i < n) comp(i, in[u]);
        }
    }
}

// grid of the vector kernels over n elements: kVecUnroll elements per
// thread for long vectors; a short vector gets at least two blocks per SM
// (down to one element per thread), since its binary64 work would otherwise
// sit on a few SMs
inline int vec_grid(const DevInfo &d, int n) {
    const int64_t per_unroll = ((int64_t)n + (int64_t)kVecUnroll * kVecBlock - 1) / ((int64_t)kVecUnroll * kVecBlock);
    const int64_t spread = std::min<int64_t>(((int64_t)n + kVecBlock - 1) / kVecBlock, 2 * (int64_t)d.num_sms);
    return stream_grid(d, std::max(per_unroll, spread) * kVecBlock, kVecBlock, 8);
}

template <class V> struct In2 { V a, b; };
template <class V> struct In3 { V a, b, c; };
template <class V> struct In5 { V a, b, c, d, e; };

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// loop condition of the enclosing WHILE node; handle 0 = the graph has no
// conditional node (the unrolled profiling graph), nothing to set
__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, unsigned v) {
    if (h) cudaGraphSetConditional(h, v);
}

// Last node of every solver loop body.  The WHILE condition a kernel of the
// body set is replaced by one that also holds the loop to its caps: the loop
// goes on only while the state is not done, the iteration count is below its
// cap and the body has run at most cap times since the loop began (a body
// that stopped advancing the count still ends).  A loop the guard ends is
// marked done and NOT_CONVERGED.  cap = ctl->maxit for a solver's own loop
// (outer_level), the inner iteration cap for the mixed method's inner loop.
template <class St>
__global__ void k_loop_guard(BiState<St> *st, const Ctl *ctl, int outer_level, cudaGraphConditionalHandle h) {
    const int cap = outer_level ? ctl->maxit : st->maxit;
    const int runs = st->guard + 1;
    const bool go = !st->done && st->iter < cap && runs <= cap;
    if (!go && !st->done) {
        st->status = HZ_NOT_CONVERGED;
        st->done = 1;
    }
    st->guard = go ? runs : 0;
    set_cond(h, go ? 1u : 0u);
}

template <class V, int NV>
__device__ __forceinline__ bool vec_reduce(typename Ar<V>::Acc (&acc)[NV], RedScratch red,
                                           typename Ar<V>::R (&tot)[NV]) {
    return grid_reduce_acc(acc, red, tot, [](const typename Ar<V>::Acc &a) { return Ar<V>::total(a); });
}

// base of the solver epilogues: accumulator plumbing for element type V
template <class V>
struct EpiBase {
    using Acc = typename Ar<V>::Acc;
    using R = typename Ar<V>::R;
    static constexpr bool kFFRow = Ar<V>::kFF;
    __device__ static void zero(Acc &a) { Ar<V>::acc_zero(a); }
    __device__ static R total(const Acc &a) { return Ar<V>::total(a); }
    __device__ void on_skip() const {}
};

// ---------------------------------------------------------------------------
// start: x_w from the caller's x0 (or 0); on a restart x_w is kept
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_init_x(int n, const Ctl *ctl, V *__restrict__ xw) {
    if (ctl->restart) return;
    const double2 *x0 = ctl->x, *pd = ctl->pre_d;
    const bool zero = ctl->x0_zero != 0;
    const double inv_s = rhs_scale(ctl) / ctl->op_scale;   // powers of two: exact
    vec_tiles(n, [&](int i) {
        const double2 v = pd ? cmul(x0[i], pd[i]) : x0[i];
        xw[i] = zero ? Ar<V>::zero() : Ar<V>::from_c128(make_double2(v.x * inv_s, v.y * inv_s));
    });
}

// exit: true residual ||b - A x|| / ||b|| and the info block
template <class V>
struct EpiTrue : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 1;
    StateOf<V> *st;
    Info *info;
    const Ctl *ctl;
    __device__ bool skip() const { return false; }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const {
        const V bi = Ar<V>::from_c128(zscale(ctl->b[i], rhs_scale(ctl)));
        Ar<V>::nrm2(acc[0], Ar<V>::sub(bi, Ar<V>::pow2(y, ctl->op_scale)));
    }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        info->iters = st->iter;
        info->status = st->status;
        info->outer = 0;
        info->relres_rec = st->rel;
        info->relres_true = info->zero_x ? 0.0 : sqrt((double)tot[0]) / st->nb;
    }
};

template <class V>
__global__ void __launch_bounds__(kVecBlock) k_copy_out(int n, const Ctl *ctl, Info *info,
                                                        const V *__restrict__ xw, const int *fault) {
    double2 *x = ctl->x;
    const double2 *pdi = ctl->pre_dinv;
    const bool zero = info->zero_x != 0;
    // an expired bounded wait in an SpMV of this solve voids the result
    if (fault && blockIdx.x == 0 && threadIdx.x == 0 && *(volatile const int *)fault) info->status = HZ_ERR_TIMEOUT;
    const double s = ctl->op_scale / rhs_scale(ctl);   // powers of two: exact
    vec_tiles(n, [&](int i) {
        const double2 y0 = Ar<V>::to_c128(xw[i]);
        const double2 y = make_double2(y0.x * s, y0.y * s);
        x[i] = zero ? make_double2(0.0, 0.0) : (pdi ? cmul(y, pdi[i]) : y);
    });
}

// capture helpers -------------------------------------------------------------
static inline hz_status capture_leaves(cudaStream_t s, std::vector<cudaGraphNode_t> *leaves) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    HZ_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd));
    leaves->assign(deps, deps + nd);
    return HZ_OK;
}

// HZ_PROFILE_UNROLL=k (environment, read when a solver graph is built): the
// graph holds k straight-line copies of its loop body instead of a WHILE
// node, for profilers that do not descend into conditional bodies.  The
// kernels are the same; condition handles are 0, so nothing sets a
// condition, and once a solve is done the remaining copies exit at once.
static inline int profile_unroll() {
    const char *e = getenv("HZ_PROFILE_UNROLL");
    return e ? atoi(e) : 0;
}

static inline hz_status add_while(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                           cudaGraphNode_t *node, cudaGraph_t *body) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    HZ_CUDA(cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &cp));
    *body = cp.conditional.phGraph_out[0];
    return HZ_OK;
}

// 2^-k with 2^(k-1) <= ||A||_inf < 2^k (1 for a zero matrix): the power of
// two that brings an operator to unit scale for the double-float path
// (bicgstabl.cu; synchronises the device)
hz_status operator_scale(const hz_mat *A, double *out);

// BiCGStab(l) (bicgstabl.cu): one solve on `op` with controls c, 1 <= l <= 8
hz_status bl_solve(hz_mat *op, int ell, const Ctl &c, Info *out, int *restarts, cudaStream_t s);
void bl_solver_free(void *solver);
// TFQMR (tfqmr.cu): one solve on `op` with controls c
hz_status tq_solve(hz_mat *op, const Ctl &c, Info *out, int *restarts, cudaStream_t s);
void tq_solver_free(void *solver);

}  // namespace hz
