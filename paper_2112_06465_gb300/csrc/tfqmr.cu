// tfqmr.cu -- TFQMR, Freund's transpose-free QMR (Section 7 of the paper lists
// P-TFQMR among its solvers), run on the device like BiCGStab: one CUDA graph
// per handle, a conditional WHILE node over iterations, scalars in device
// memory.
//
// Iteration j (half steps m = 2j+1, 2j+2; two products with A):
//   Q1  u2 = u1 - alpha v,  w -= alpha A u1,  ||w||  -> half-step scalars
//   Q2  au = A u2;  epilogue: d = u1 + coef1 d, x += eta1 d (half step 1),
//       w -= alpha au, ||w||, <r^, w>  -> half-step scalars, the stopping
//       test on the quasi-residual bound sqrt(m+1) tau_m, rho', beta
//   Q3  d = u2 + coef2 d, x += eta2 d (half step 2); then u1 = w + beta u2,
//       v = beta (au + beta v)
//   Q4  au1 = A u1;  epilogue: v += au1, <r^, v>  -> alpha = rho / <r^, v>
// per half step: theta = ||w|| / tau, c = 1/sqrt(1 + theta^2), tau *= theta c,
// coef = theta_prev^2 eta_prev / alpha, eta = c^2 alpha.  The d/x update of
// a half step needs that step's reduction, so it rides on the next kernel.
//
// Range guard.  In a stagnating or erratic run u, v and w (squared-BiCG
// vectors) can grow without bound while x stays sensible; on the
// double-float path their squares leave the binary32 exponent range long
// before binary64 would notice.  The iteration is invariant under scaling
// u, v, w, d, A u and rho, tau by the same factor if x is updated with
// eta / G (G the accumulated factor) and the bound uses tau / G.  When
// ||v||^2 or tau^2 passes 2^120 the next iteration first scales those
// vectors by 2^-64 (exact) and the scalars with them (inside Q1).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "krylov.cuh"

namespace hz {

struct TqExtra {
    double2 eta;       // eta of the last half step
    double2 coef1, eta1, coef2, eta2;   // d/x coefficients of the two half steps of this iteration
    double tau, theta;
    double xs;         // 1 / G: x moves by eta * xs * d (vectors held scaled by G <= 1)
    double2 eta1x, eta2x;   // eta1 * xs, eta2 * xs
    int m;             // half steps since the (re)start
    int stop;          // the stopping test fired: finish the pending x update, then stop
    int pend;          // rescale by 2^-64 at the start of the next iteration
};

constexpr double kTqBig = 1.329227995784916e36;     // 2^120: rescale threshold for squared norms
constexpr double kTqShrink = 5.421010862427522e-20;  // 2^-64

// one half step's scalars from ||w||^2 (single thread)
__device__ __forceinline__ void tq_half_step(StateOf<double2> *st, TqExtra *q, double ww, double2 &coef,
                                             double2 &eta_h) {
    q->m += 1;
    const double th_prev = q->theta;
    const double theta = q->tau == 0.0 ? 0.0 : sqrt(ww) / q->tau;
    const double c = 1.0 / sqrt(1.0 + theta * theta);
    q->tau = q->tau * theta * c;
    coef = cdiv(make_double2(th_prev * th_prev * q->eta.x, th_prev * th_prev * q->eta.y), st->alpha);
    eta_h = make_double2(c * c * st->alpha.x, c * c * st->alpha.y);
    q->eta = eta_h;
    q->theta = theta;
}

// start epilogue: w = u1 = r^ = b - A x, d = v = 0, ||r||^2, ||b||^2
template <class V>
struct EpiTqInit : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 2;
    StateOf<V> *st;
    TqExtra *q;
    Info *info;
    const Ctl *ctl;
    V *w, *u1, *rh, *d, *v;
    cudaGraphConditionalHandle h;
    __device__ bool skip() const { return false; }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const {
        const V bi = Ar<V>::from_c128(ctl->b[i]);
        const V ri = Ar<V>::sub(bi, y);
        w[i] = ri;
        u1[i] = ri;
        rh[i] = ri;
        d[i] = Ar<V>::zero();
        v[i] = Ar<V>::zero();
        Ar<V>::nrm2(acc[0], ri);
        Ar<V>::nrm2(acc[1], bi);
    }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        const bool restart = ctl->restart != 0;
        const double nb = sqrt((double)tot[1]), rr = (double)tot[0];
        st->nb = nb;
        if (!restart) { st->iter = 0; info->zero_x = 0; }
        q->tau = sqrt(rr);
        q->theta = 0.0;
        q->eta = make_double2(0.0, 0.0);
        q->m = 0;
        q->stop = 0;
        q->pend = 0;
        q->xs = 1.0;
        st->rho = make_double2(rr, 0.0);
        if (nb == 0.0) {
            st->rel = 0.0; st->status = HZ_OK; st->done = 1; info->zero_x = 1;
            if (ctl->hist && !restart) ctl->hist[0] = 0.0;
        } else {
            const double rel = sqrt(rr) / nb;
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

// Q4 (and the start): au1 = A u1, v += au1, <r^, v>, alpha = rho / <r^, v>;
// sets the loop condition
template <class V>
struct EpiTqV : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 3;
    StateOf<V> *st;
    TqExtra *q;
    const Ctl *ctl;
    V *au1, *v;
    const V *rh;
    cudaGraphConditionalHandle h;
    __device__ bool skip() const { return st->done; }
    // a finished solve must leave the loop even when this product is skipped
    __device__ void on_skip() const { set_cond(h, 0); }
    struct Pre {   // v[i] and rh[i], fetched ahead by the block-flat kernel
        V v, rh;
    };
    __device__ Pre pre(int i) const { return Pre{v[i], rh[i]}; }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N], const Pre &pf) const {
        au1[i] = y;
        const V vi = Ar<V>::add(y, pf.v);
        v[i] = vi;
        Ar<V>::dotc(acc[0], acc[1], pf.rh, vi);
        Ar<V>::nrm2(acc[2], vi);
    }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const { row(i, y, acc, pre(i)); }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        const double2 sig = make_double2((double)tot[0], (double)tot[1]);
        if (!((double)tot[2] < kTqBig) || !(q->tau * q->tau < kTqBig)) q->pend = 1;
        if (cis_zero(st->rho) || cis_zero(sig)) { st->status = HZ_BREAKDOWN; st->done = 1; }
        else if (st->iter >= ctl->maxit) { st->status = HZ_NOT_CONVERGED; st->done = 1; }
        else st->alpha = cdiv(st->rho, sig);
        set_cond(h, st->done ? 0 : 1);
    }
};

// Q1: u2 = u1 - alpha v, w -= alpha A u1, ||w||^2 -> half step 2j+1.
// With the range guard's flag set, u1, v, w, d and A u1 are first scaled by
// 2^-64 (exact) element by element, in place (the same thread reads and
// writes each element, so no other kernel is needed)
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_tq_half1(int n, StateOf<V> *st, TqExtra *q, V *__restrict__ u2,
                                                        V *__restrict__ u1, V *__restrict__ v, V *__restrict__ w,
                                                        V *__restrict__ d, V *__restrict__ au1, RedScratch red) {
    using A = Ar<V>;
    if (st->done) return;
    const typename A::S alpha = A::scal(st->alpha);
    const bool pend = q->pend != 0;   // read by every block before the last one resets it
    typename A::Acc acc[1];
    A::acc_zero(acc[0]);
    vec_tiles(n, [&](int i) {
        V u1i = u1[i], vi = v[i], wi = w[i], ai = au1[i];
        if (pend) {
            u1i = A::pow2(u1i, kTqShrink);
            vi = A::pow2(vi, kTqShrink);
            wi = A::pow2(wi, kTqShrink);
            ai = A::pow2(ai, kTqShrink);
            u1[i] = u1i;
            v[i] = vi;
            au1[i] = ai;
            d[i] = A::pow2(d[i], kTqShrink);
        }
        u2[i] = A::axmy(u1i, alpha, vi);
        wi = A::axmy(wi, alpha, ai);
        w[i] = wi;
        A::nrm2(acc[0], wi);
    });
    typename A::R tot[1];
    if (vec_reduce<V, 1>(acc, red, tot) && threadIdx.x == 0) {
        if (q->pend) {   // the vectors were scaled above
            q->pend = 0;
            q->tau *= kTqShrink;
            st->rho = make_double2(st->rho.x * kTqShrink, st->rho.y * kTqShrink);
            q->xs /= kTqShrink;
        }
        tq_half_step(st, q, (double)tot[0], q->coef1, q->eta1);
        q->eta1x = make_double2(q->eta1.x * q->xs, q->eta1.y * q->xs);
    }
}

// Q2 epilogue: au = A u2; d/x update of half step 2j+1; w -= alpha au;
// ||w||^2, <r^, w> -> half step 2j+2, stopping test, rho', beta
template <class V>
struct EpiTqW : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 3;
    StateOf<V> *st;
    TqExtra *q;
    const Ctl *ctl;
    V *au, *d, *x, *w;
    const V *u1, *rh;
    __device__ bool skip() const { return st->done; }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const {
        using A = Ar<V>;
        au[i] = y;
        const V di = A::axpy(u1[i], A::scal(q->coef1), d[i]);
        d[i] = di;
        x[i] = A::axpy(x[i], A::scal(q->eta1x), di);
        const V wi = A::axmy(w[i], A::scal(st->alpha), y);
        w[i] = wi;
        A::nrm2(acc[0], wi);
        A::dotc(acc[1], acc[2], rh[i], wi);
    }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        tq_half_step(st, q, (double)tot[0], q->coef2, q->eta2);
        q->eta2x = make_double2(q->eta2.x * q->xs, q->eta2.y * q->xs);
        const int it = st->iter + 1;
        st->iter = it;
        const double rel = sqrt((double)q->m + 1.0) * q->tau * q->xs / st->nb;
        st->rel = rel;
        if (ctl->hist) ctl->hist[it] = rel;
        if (!finite_d(rel)) { st->status = HZ_ERR_NAN; q->stop = 1; }
        else if (rel <= ctl->tol) { st->status = HZ_OK; q->stop = 1; }
        else {
            const double2 rho1 = make_double2((double)tot[1], (double)tot[2]);
            st->beta = cdiv(rho1, st->rho);
            st->rho = rho1;
        }
    }
};

// Q3: d/x update of half step 2j+2; then (unless stopping) u1 = w + beta u2
// and v = beta (au + beta v)
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_tq_update(int n, StateOf<V> *st, const TqExtra *q, V *__restrict__ d,
                                                         V *__restrict__ x, const V *__restrict__ u2,
                                                         V *__restrict__ u1, const V *__restrict__ w,
                                                         const V *__restrict__ au, V *__restrict__ v) {
    using A = Ar<V>;
    if (st->done) return;
    const typename A::S coef = A::scal(q->coef2), eta = A::scal(q->eta2x), beta = A::scal(st->beta);
    const bool stop = q->stop != 0;
    vec_tiles(n, [&](int i) {
        const V di = A::axpy(u2[i], coef, d[i]);
        d[i] = di;
        x[i] = A::axpy(x[i], eta, di);
        if (!stop) {
            u1[i] = A::axpy(w[i], beta, u2[i]);
            v[i] = A::axpy(A::zero(), beta, A::axpy(au[i], beta, v[i]));
        }
    });
    if (stop && blockIdx.x == 0 && threadIdx.x == 0) st->done = 1;
}

// ---------------------------------------------------------------------------
struct TqSolver {
    int n = 0, kind = 0, group = 4;
    int grid_spmv = 1, grid_spmv_cv = 1, grid_vec = 1;
    void *x = nullptr, *w = nullptr, *u1 = nullptr, *u2 = nullptr, *v = nullptr, *d = nullptr, *au1 = nullptr,
         *au = nullptr, *rh = nullptr;
    BiState<double2> *st = nullptr;
    TqExtra *q = nullptr;
    Info *dinfo = nullptr;
    Ctl *dctl = nullptr;
    Ctl *hctl = nullptr;
    Info *hinfo = nullptr;
    RedScratch red{};
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

void tq_solver_free(void *p) {
    TqSolver *S = (TqSolver *)p;
    if (!S) return;
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->cap) cudaStreamDestroy(S->cap);
    void *dev[] = {S->x, S->w, S->u1, S->u2, S->v, S->d, S->au1, S->au, S->rh,
                   S->st, S->q, S->dinfo, S->dctl, S->red.partials, S->red.counter};
    for (void *p2 : dev) cudaFree(p2);
    cudaFreeHost(S->hctl);
    cudaFreeHost(S->hinfo);
    delete S;
}

template <class V, class Epi>
static void tq_spmv(const TqSolver *S, const hz_mat *A, const V *x, const Epi &e, cudaStream_t cs) {
    if constexpr (std::is_same<V, float4>::value) {
        launch_spmv_ff(S->kind, S->group, mat_view<double2>(A), x, e, S->red, S->grid_spmv, cs);
    } else {
        launch_spmv<V>(d64_kind(A, S->kind), S->group, mat_view<V>(A), x, e, S->red,
                       S->grid_spmv_cv, cs);
    }
}

template <class V>
static hz_status tq_build_graph(TqSolver *S, const hz_mat *A, cudaGraph_t g) {
    cudaStream_t cs = S->cap;
    const auto mode = cudaStreamCaptureModeThreadLocal;
    const int n = S->n;
    V *x = (V *)S->x, *w = (V *)S->w, *u1 = (V *)S->u1, *u2 = (V *)S->u2, *v = (V *)S->v, *d = (V *)S->d,
      *au1 = (V *)S->au1, *au = (V *)S->au, *rh = (V *)S->rh;
    StateOf<V> *st = (StateOf<V> *)S->st;
    const int unroll = profile_unroll();
    cudaGraphConditionalHandle h = 0;
    std::vector<cudaGraphNode_t> leaves;
    if (unroll <= 0) HZ_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, mode));
    cudaMemcpyAsync(S->dctl, S->hctl, sizeof(Ctl), cudaMemcpyHostToDevice, cs);
    k_init_x<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->dctl, x);
    EpiTqInit<V> ei;
    ei.st = st; ei.q = S->q; ei.info = S->dinfo; ei.ctl = S->dctl; ei.w = w; ei.u1 = u1; ei.rh = rh; ei.d = d;
    ei.v = v; ei.h = h;
    tq_spmv<V>(S, A, x, ei, cs);
    EpiTqV<V> ev;
    ev.st = st; ev.q = S->q; ev.ctl = S->dctl; ev.au1 = au1; ev.v = v; ev.rh = rh; ev.h = h;
    tq_spmv<V>(S, A, u1, ev, cs);   // v_0 = A u_1, alpha; sets the loop condition
    EpiTqW<V> ew;
    ew.st = st; ew.q = S->q; ew.ctl = S->dctl; ew.au = au; ew.d = d; ew.x = x; ew.w = w; ew.u1 = u1; ew.rh = rh;
    auto iteration = [&]() {
        k_tq_half1<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, st, S->q, u2, u1, v, w, d, au1, S->red);
        tq_spmv<V>(S, A, u2, ew, cs);
        k_tq_update<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, st, S->q, d, x, u2, u1, w, au, v);
        tq_spmv<V>(S, A, u1, ev, cs);
    };
    if (unroll > 0) {
        for (int k = 0; k < unroll; ++k) iteration();
    } else {
        HZ_TRY(capture_leaves(cs, &leaves));
        HZ_CUDA(cudaStreamEndCapture(cs, &g));
        cudaGraphNode_t wn;
        cudaGraph_t body;
        HZ_TRY(add_while(g, leaves, h, &wn, &body));
        HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, mode));
        iteration();
        k_loop_guard<typename Ar<V>::St><<<1, 1, 0, cs>>>(st, S->dctl, 1, h);
        HZ_CUDA(cudaStreamEndCapture(cs, &body));
        HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, g, &wn, nullptr, 1, mode));
    }
    EpiTrue<V> et;
    et.st = st; et.info = S->dinfo; et.ctl = S->dctl;
    tq_spmv<V>(S, A, x, et, cs);
    k_copy_out<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->dctl, S->dinfo, x, A->fault);
    cudaMemcpyAsync(S->hinfo, S->dinfo, sizeof(Info), cudaMemcpyDeviceToHost, cs);
    HZ_CUDA(cudaStreamEndCapture(cs, &g));
    return HZ_OK;
}

#define HZ_TQ_ALLOC(ptr, bytes) HZ_CUDA(cudaMalloc((void **)&(ptr), std::max<size_t>((bytes), 16)))

static hz_status tq_get_solver(hz_mat *A, TqSolver **out) {
    TqSolver *S = (TqSolver *)A->solver_tq;
    if (S && (S->kind != A->spmv_kind || S->group != A->group)) {
        tq_solver_free(S);
        A->solver_tq = S = nullptr;
    }
    if (S) { *out = S; return HZ_OK; }
    DevInfo dv;
    HZ_TRY(dev_info(&dv));
    S = new TqSolver();
    A->solver_tq = S;   // freed with the handle even if the build below fails
    S->n = A->n;
    S->kind = A->spmv_kind;
    S->group = A->group;
    S->grid_spmv = spmv_grid(A, S->kind, S->group);
    S->grid_spmv_cv = spmv_grid(A, d64_kind(A, S->kind), S->group);
    S->grid_vec = vec_grid(dv, A->n);
    const size_t nb = (size_t)A->n * 16;
    void **vecs[] = {&S->x, &S->w, &S->u1, &S->u2, &S->v, &S->d, &S->au1, &S->au, &S->rh};
    for (void **p : vecs) HZ_TQ_ALLOC(*p, nb);
    HZ_TQ_ALLOC(S->st, sizeof(BiState<double2>));
    HZ_TQ_ALLOC(S->q, sizeof(TqExtra));
    HZ_TQ_ALLOC(S->dinfo, sizeof(Info));
    HZ_TQ_ALLOC(S->dctl, sizeof(Ctl));
    HZ_TQ_ALLOC(S->red.partials, sizeof(double) * kMaxRedBlocks * kMaxRedValues);
    HZ_TQ_ALLOC(S->red.counter, 256);
    HZ_CUDA(cudaMemset(S->red.counter, 0, 256));
    HZ_CUDA(cudaMemset(S->st, 0, sizeof(BiState<double2>)));
    HZ_CUDA(cudaMemset(S->q, 0, sizeof(TqExtra)));
    HZ_CUDA(cudaMemset(S->dinfo, 0, sizeof(Info)));
    HZ_CUDA(cudaMallocHost((void **)&S->hctl, sizeof(Ctl)));
    HZ_CUDA(cudaMallocHost((void **)&S->hinfo, sizeof(Info)));
    memset(S->hctl, 0, sizeof(Ctl));
    memset(S->hinfo, 0, sizeof(Info));
    HZ_CUDA(cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking));
    HZ_CUDA(cudaDeviceSynchronize());
    cudaGraph_t g;
    HZ_CUDA(cudaGraphCreate(&g, 0));
    S->graph = g;
    HZ_TRY(is_ff_kind(S->kind) ? tq_build_graph<float4>(S, A, g) : tq_build_graph<double2>(S, A, g));
    HZ_CUDA(cudaGraphInstantiate(&S->exec, g, 0));
    *out = S;
    return HZ_OK;
}

hz_status tq_solve(hz_mat *op, const Ctl &c, Info *out, int *restarts, cudaStream_t s) {
    TqSolver *S = nullptr;
    HZ_TRY(tq_get_solver(op, &S));
    *S->hctl = c;
    HZ_CUDA(cudaGraphLaunch(S->exec, s));
    HZ_CUDA(cudaStreamSynchronize(s));
    *out = *S->hinfo;
    *restarts = 0;
    if (out->status == HZ_OK && out->relres_true > c.tol && out->iters < c.maxit) {
        S->hctl->restart = 1;
        HZ_CUDA(cudaGraphLaunch(S->exec, s));
        HZ_CUDA(cudaStreamSynchronize(s));
        *out = *S->hinfo;
        *restarts = 1;
    }
    return HZ_OK;
}

}  // namespace hz
