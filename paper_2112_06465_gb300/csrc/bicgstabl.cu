// bicgstabl.cu -- BiCGStab(l) (Sleijpen and Fokkema; Section 7 of the paper
// lists P-BiCGSTAB(l) among its solvers), run on the device like BiCGStab:
// one CUDA graph per handle and l, a conditional WHILE node over outer
// iterations, scalars in device memory, no host round trip per step.
//
// One outer iteration = l BiCG steps j = 0..l-1, each
//   K2  u_i = r_i - beta u_i  (i <= j)                    vector pass
//   K3  u_{j+1} = A u_j,  gamma = <r^, u_{j+1}>           SpMV + dot epilogue
//   K4  r_i -= alpha u_{i+1} (i <= j), x += alpha u_0,
//       ||r_0||  (convergence test after every step)      vector pass + reduction
//   K5  r_{j+1} = A r_j,  rho_1 = <r^, r_{j+1}>           SpMV + dot epilogue
// then the minimal-residual step
//   M1  Gram matrix G_ik = <r_i, r_k> (1 <= i <= k <= l) and c_i = <r_i, r_0>
//       in one pass over r_0..r_l; the last block solves G g = c (Cholesky)
//   M2  x += sum_j g_j r_{j-1},  r_0 -= sum_j g_j r_j,  u_0 -= sum_j g_j u_j,
//       <r^, r_0>, ||r_0||, the stopping test and the next outer iteration's
//       scalars (rho_0 = -omega rho_0, beta = alpha rho_1 / rho_0).
// The least-squares coefficients come from the normal equations of the
// Gram matrix instead of modified Gram-Schmidt (one reduction pass instead
// of l(l+1)/2 dependent ones); the same minimiser in exact arithmetic, and
// x and r_0 stay consistent whatever its rounding, since r_j = A r_{j-1}.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "krylov.cuh"

namespace hz {

constexpr int kMaxEll = 8;
constexpr int kGramTile = 32;   // elements per tile of the Gram pass
constexpr int kMaxPairs = kMaxEll + kMaxEll * (kMaxEll + 1) / 2;

struct BlExtra {
    double2 g[kMaxEll + 1];   // minimal-residual coefficients g_1..g_l
};

// element e of vector i in a block of vectors stored one after another
template <class V>
__device__ __forceinline__ V &vat(V *base, int i, int n, int e) {
    return base[(size_t)i * (size_t)n + (size_t)e];
}

// start epilogue: r_0 = b - A x, r^ = r_0, u_0 = 0, ||r_0||^2, ||b||^2
template <class V>
struct EpiBlInit : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 2;
    StateOf<V> *st;
    Info *info;
    const Ctl *ctl;
    V *r0, *rh, *u0;
    cudaGraphConditionalHandle h;
    __device__ bool skip() const { return false; }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const {
        const V bi = Ar<V>::from_c128(ctl->b[i]);
        const V ri = Ar<V>::sub(bi, Ar<V>::pow2(y, ctl->op_scale));
        r0[i] = ri;
        rh[i] = ri;
        u0[i] = Ar<V>::zero();
        Ar<V>::nrm2(acc[0], ri);
        Ar<V>::nrm2(acc[1], bi);
    }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        const bool restart = ctl->restart != 0;
        const double nb = sqrt((double)tot[1]);
        st->nb = nb;
        if (!restart) { st->iter = 0; info->zero_x = 0; }
        // alpha = 0, omega = 1, rho_0 = 1; the first outer iteration's
        // rho_0 = -omega rho_0 = -1 and beta = alpha rho_1 / rho_0 = 0
        st->alpha = make_double2(0.0, 0.0);
        st->omega = make_double2(1.0, 0.0);
        st->beta = make_double2(0.0, 0.0);
        st->rho = make_double2((double)tot[0], 0.0);   // rho_1 = <r^, r_0> = ||r_0||^2
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

// K2: u_i = r_i - beta u_i for i = 0..j
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_bl_u(int n, int j, const StateOf<V> *st, V *__restrict__ U,
                                                    const V *__restrict__ R) {
    if (st->done) return;
    const typename Ar<V>::S beta = Ar<V>::scal(st->beta);
    vec_tiles(n, [&](int e) {
        for (int i = 0; i <= j; ++i) vat(U, i, n, e) = Ar<V>::axmy(vat(R, i, n, e), beta, vat(U, i, n, e));
    });
}

// K3 epilogue: u_{j+1} = A u_j, gamma = <r^, u_{j+1}>, alpha = rho_0 / gamma
template <class V>
struct EpiBlU : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 2;
    StateOf<V> *st;
    V *u_next;
    const V *rh;
    double s;   // operator scale
    __device__ bool skip() const { return st->done; }
    using Pre = V;   // rh[i], fetched ahead by the block-flat kernel
    __device__ V pre(int i) const { return rh[i]; }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N], const V &rhi) const {
        y = Ar<V>::pow2(y, s);
        u_next[i] = y;
        Ar<V>::dotc(acc[0], acc[1], rhi, y);
    }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const { row(i, y, acc, rh[i]); }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        const double2 g = make_double2((double)tot[0], (double)tot[1]);
        if (cis_zero(g)) { st->status = HZ_BREAKDOWN; st->done = 1; return; }
        st->alpha = cdiv(st->rho, g);
    }
};

// K4: r_i -= alpha u_{i+1} (i = 0..j), x += alpha u_0, ||r_0||: one BiCG step done
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_bl_r(int n, int j, StateOf<V> *st, const Ctl *ctl, V *__restrict__ R,
                                                    const V *__restrict__ U, V *__restrict__ X, RedScratch red) {
    using A = Ar<V>;
    if (st->done) return;
    const typename A::S alpha = A::scal(st->alpha);
    typename A::Acc acc[1];
    A::acc_zero(acc[0]);
    vec_tiles(n, [&](int e) {
        for (int i = 0; i <= j; ++i) vat(R, i, n, e) = A::axmy(vat(R, i, n, e), alpha, vat(U, i + 1, n, e));
        X[e] = A::axpy(X[e], alpha, U[e]);
        A::nrm2(acc[0], R[e]);
    });
    typename A::R tot[1];
    if (vec_reduce<V, 1>(acc, red, tot) && threadIdx.x == 0) {
        const int it = st->iter + 1;
        st->iter = it;
        const double rel = sqrt((double)tot[0]) / st->nb;
        st->rel = rel;
        if (ctl->hist) ctl->hist[it] = rel;
        if (!finite_d(rel)) { st->status = HZ_ERR_NAN; st->done = 1; }
        else if (rel <= ctl->tol) { st->status = HZ_OK; st->done = 1; }
    }
}

// K5 epilogue: r_{j+1} = A r_j; for j + 1 < l also rho_1 = <r^, r_{j+1}>,
// beta = alpha rho_1 / rho_0, rho_0 = rho_1 for the next BiCG step
template <class V>
struct EpiBlR : EpiBase<V> {
    using typename EpiBase<V>::Acc;
    using typename EpiBase<V>::R;
    static constexpr int NV = 2;
    StateOf<V> *st;
    V *r_next;
    const V *rh;
    int want_rho;
    double s;   // operator scale
    __device__ bool skip() const { return st->done; }
    template <int N> __device__ void row(int i, V y, Acc (&acc)[N]) const {
        y = Ar<V>::pow2(y, s);
        r_next[i] = y;
        if (want_rho) Ar<V>::dotc(acc[0], acc[1], rh[i], y);
    }
    template <int N> __device__ void finish(R (&tot)[N]) const {
        if (!want_rho) return;
        if (cis_zero(st->rho)) { st->status = HZ_BREAKDOWN; st->done = 1; return; }
        const double2 rho1 = make_double2((double)tot[0], (double)tot[1]);
        st->beta = cmul(st->alpha, cdiv(rho1, st->rho));
        st->rho = rho1;
    }
};

// the p-th (i, k) of the Gram pass: p < l gives (i, 0) = c_i, then the
// upper triangle 1 <= i <= k <= l row by row
__device__ __forceinline__ void gram_pair(int ell, int p, int &i, int &k) {
    if (p < ell) { i = p + 1; k = 0; return; }
    int q = p - ell;
    for (i = 1; q >= ell - i + 1; ++i) q -= ell - i + 1;
    k = i + q;
}

// G g = c for the Hermitian positive semidefinite Gram matrix G (l x l,
// 1-based, upper triangle given).  G is first equilibrated to unit diagonal
// (the r_j grow like powers of A, so their norms spread over many orders of
// magnitude); Cholesky of the equilibrated matrix then treats a pivot below
// kPivotFloor as a numerically dependent direction and floors it there,
// which regularises the least-squares fit instead of failing: the fitted
// coefficients still give a consistent update (r_j = A r_{j-1}), only a
// slightly less than minimal residual.  For l = 8 the Gram matrix of the
// Krylov-like basis can be that ill-conditioned, notably with double-float
// dot products.  False only for a zero or non-finite diagonal (some r_j = 0).
constexpr double kPivotFloor = 1e-13;

__device__ bool chol_solve(int ell, const double2 (*G)[kMaxEll + 1], const double2 *c, double2 *g) {
    double2 L[kMaxEll + 1][kMaxEll + 1];
    double2 z[kMaxEll + 1];
    double sc[kMaxEll + 1];
    for (int k = 1; k <= ell; ++k) {
        const double d = G[k][k].x;
        if (!(d > 0.0) || !isfinite(d)) return false;
        sc[k] = 1.0 / sqrt(d);
    }
    for (int k = 1; k <= ell; ++k) {
        double d = 1.0;   // equilibrated diagonal
        for (int m = 1; m < k; ++m) d -= L[k][m].x * L[k][m].x + L[k][m].y * L[k][m].y;
        if (!isfinite(d)) return false;
        const double lkk = sqrt(d > kPivotFloor ? d : kPivotFloor);
        L[k][k] = make_double2(lkk, 0.0);
        for (int i = k + 1; i <= ell; ++i) {
            // equilibrated G[i][k] = conj(G[k][i]) sc_i sc_k
            const double2 gki = G[k][i];
            double2 a = make_double2(gki.x * sc[i] * sc[k], -gki.y * sc[i] * sc[k]);
            for (int m = 1; m < k; ++m) a = csub(a, cmul(L[i][m], cconj(L[k][m])));
            L[i][k] = make_double2(a.x / lkk, a.y / lkk);
        }
    }
    for (int i = 1; i <= ell; ++i) {
        double2 a = make_double2(c[i].x * sc[i], c[i].y * sc[i]);
        for (int m = 1; m < i; ++m) a = csub(a, cmul(L[i][m], z[m]));
        z[i] = make_double2(a.x / L[i][i].x, a.y / L[i][i].x);
    }
    for (int i = ell; i >= 1; --i) {
        double2 a = z[i];
        for (int m = i + 1; m <= ell; ++m) a = csub(a, cmul(cconj(L[m][i]), g[m]));
        g[i] = make_double2(a.x / L[i][i].x, a.y / L[i][i].x);
    }
    for (int i = 1; i <= ell; ++i) g[i] = make_double2(g[i].x * sc[i], g[i].y * sc[i]);
    return true;
}

// accumulator pairs of the Gram reduction: binary64 sums on the binary64
// path, (s, c) pairs with binary32 TwoSums on the double-float path (the
// binary64 pipe is far slower than the binary32 one on this GPU)
__device__ __forceinline__ void pacc(double &a, double b) { a += b; }
__device__ __forceinline__ void pacc(FFAcc &a, FFAcc b) { ff_pair_add(a.s, a.c, b.s, b.c); }
__device__ __forceinline__ double pshfl(double a, int off) { return __shfl_xor_sync(0xffffffffu, a, off); }
__device__ __forceinline__ FFAcc pshfl(FFAcc a, int off) {
    return FFAcc{__shfl_xor_sync(0xffffffffu, a.s, off), __shfl_xor_sync(0xffffffffu, a.c, off)};
}
__device__ __forceinline__ double pld(const double *p) { return __ldcg(p); }
__device__ __forceinline__ FFAcc pld(const FFAcc *p) {   // 8-byte slots of the scratch buffer
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return FFAcc{v.x, v.y};
}
__device__ __forceinline__ double pwiden(double a) { return a; }
__device__ __forceinline__ double pwiden(FFAcc a) { return (double)a.s + (double)a.c; }

// M1: Gram matrix of r_1..r_l and their products with r_0, reduced
// deterministically (fixed-order sums within and across blocks); the last
// block solves the normal equations for the minimal-residual coefficients
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_bl_gram(int n, int ell, StateOf<V> *st, const V *__restrict__ R,
                                                       RedScratch red, BlExtra *ex) {
    using A = Ar<V>;
    if (st->done) return;
    __shared__ V tile[kMaxEll + 1][kGramTile];
    __shared__ typename Ar<V>::Acc part[kVecBlock][2];
    __shared__ double tot[kMaxPairs][2];
    __shared__ int am_last;
    const int np = ell + ell * (ell + 1) / 2;
    const int tpp = blockDim.x / np;   // threads per pair (>= 5 for l <= 8)
    const int p = threadIdx.x / tpp, sub = threadIdx.x % tpp;
    int pi = 0, pk = 0;
    if (p < np) gram_pair(ell, p, pi, pk);
    typename A::Acc ar, ai;
    A::acc_zero(ar);
    A::acc_zero(ai);
    for (int base = blockIdx.x * kGramTile; base < n; base += gridDim.x * kGramTile) {
        for (int idx = threadIdx.x; idx < (ell + 1) * kGramTile; idx += blockDim.x) {
            const int vi = idx / kGramTile, e = idx % kGramTile;
            tile[vi][e] = base + e < n ? vat(R, vi, n, base + e) : A::zero();
        }
        __syncthreads();
        if (p < np)
            for (int e = sub; e < kGramTile; e += tpp) A::dotc(ar, ai, tile[pi][e], tile[pk][e]);
        __syncthreads();
    }
    // block partial of each pair: its tpp threads folded in order
    using P = typename A::Acc;
    part[threadIdx.x][0] = ar;
    part[threadIdx.x][1] = ai;
    __syncthreads();
    P *partials = reinterpret_cast<P *>(red.partials);
    if (threadIdx.x < np) {
        P sr = part[threadIdx.x * tpp][0], si = part[threadIdx.x * tpp][1];
        for (int t = 1; t < tpp; ++t) {
            pacc(sr, part[threadIdx.x * tpp + t][0]);
            pacc(si, part[threadIdx.x * tpp + t][1]);
        }
        partials[((size_t)blockIdx.x * np + threadIdx.x) * 2] = sr;
        partials[((size_t)blockIdx.x * np + threadIdx.x) * 2 + 1] = si;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = atomicAdd(red.counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // last block: one warp per pair, lane l folds blocks l, l + 32, ... and
    // the lanes are combined by a fixed shuffle tree
    const int lane = threadIdx.x & 31;
    for (int q = threadIdx.x >> 5; q < np; q += blockDim.x >> 5) {
        P sr, si;
        A::acc_zero(sr);
        A::acc_zero(si);
        for (int b = lane; b < (int)gridDim.x; b += 32) {
            pacc(sr, pld(&partials[((size_t)b * np + q) * 2]));
            pacc(si, pld(&partials[((size_t)b * np + q) * 2 + 1]));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            pacc(sr, pshfl(sr, off));
            pacc(si, pshfl(si, off));
        }
        if (lane == 0) {
            tot[q][0] = pwiden(sr);
            tot[q][1] = pwiden(si);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *red.counter = 0u;
        double2 G[kMaxEll + 1][kMaxEll + 1], c[kMaxEll + 1], g[kMaxEll + 1];
        for (int q = 0; q < np; ++q) {
            int i, k;
            gram_pair(ell, q, i, k);
            const double2 v = make_double2(tot[q][0], tot[q][1]);
            if (k == 0) c[i] = v;
            else G[i][k] = v;
        }
        if (!chol_solve(ell, G, c, g)) {
            st->status = HZ_BREAKDOWN;
            st->done = 1;
            return;
        }
        for (int j = 1; j <= ell; ++j) ex->g[j] = g[j];
        st->omega = g[ell];
    }
}

// M2: the minimal-residual update, <r^, r_0>, ||r_0||, stopping test and
// the scalars of the next outer iteration; sets the loop condition
template <class V>
__global__ void __launch_bounds__(kVecBlock) k_bl_update(int n, int ell, StateOf<V> *st, const Ctl *ctl,
                                                         V *__restrict__ X, V *__restrict__ R, V *__restrict__ U,
                                                         const V *__restrict__ rh, const BlExtra *ex, RedScratch red) {
    using A = Ar<V>;
    if (st->done) return;
    typename A::S g[kMaxEll + 1];
    for (int j = 1; j <= ell; ++j) g[j] = A::scal(ex->g[j]);
    typename A::Acc acc[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) A::acc_zero(acc[q]);
    vec_tiles(n, [&](int e) {
        const V r0 = R[e];
        V x = X[e], r = r0, u = U[e];
        for (int j = 1; j <= ell; ++j) {
            x = A::axpy(x, g[j], j == 1 ? r0 : vat(R, j - 1, n, e));
            r = A::axmy(r, g[j], vat(R, j, n, e));
            u = A::axmy(u, g[j], vat(U, j, n, e));
        }
        X[e] = x;
        R[e] = r;
        U[e] = u;
        A::dotc(acc[0], acc[1], rh[e], r);
        A::nrm2(acc[2], r);
    });
    typename A::R tot[3];
    if (vec_reduce<V, 3>(acc, red, tot) && threadIdx.x == 0) {
        const double rel = sqrt((double)tot[2]) / st->nb;
        st->rel = rel;
        if (ctl->hist) ctl->hist[st->iter] = rel;
        if (!finite_d(rel)) { st->status = HZ_ERR_NAN; st->done = 1; }
        else if (rel <= ctl->tol) { st->status = HZ_OK; st->done = 1; }
        else if (cis_zero(st->omega)) { st->status = HZ_BREAKDOWN; st->done = 1; }
        else if (st->iter >= ctl->maxit) { st->status = HZ_NOT_CONVERGED; st->done = 1; }
        else {
            const double2 rho0 = cmul(make_double2(-st->omega.x, -st->omega.y), st->rho);
            if (cis_zero(rho0)) { st->status = HZ_BREAKDOWN; st->done = 1; }
            else {
                const double2 rho1 = make_double2((double)tot[0], (double)tot[1]);
                st->beta = cmul(st->alpha, cdiv(rho1, rho0));
                st->rho = rho1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
struct BlSolver {
    int ell = 0, n = 0, kind = 0, group = 4;
    double op_scale = 1.0;   // 2^-k with 2^(k-1) <= ||A||_inf < 2^k
    int grid_spmv = 1, grid_spmv_cv = 1, grid_vec = 1, grid_gram = 1;
    void *x = nullptr, *R = nullptr, *U = nullptr, *rh = nullptr;
    BiState<double2> *st = nullptr;
    BlExtra *ex = nullptr;
    Info *dinfo = nullptr;
    Ctl *dctl = nullptr;
    Ctl *hctl = nullptr;
    Info *hinfo = nullptr;
    RedScratch red{};
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

void bl_solver_free(void *p) {
    BlSolver *S = (BlSolver *)p;
    if (!S) return;
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->cap) cudaStreamDestroy(S->cap);
    void *dev[] = {S->x, S->R, S->U, S->rh, S->st, S->ex, S->dinfo, S->dctl, S->red.partials, S->red.counter};
    for (void *q : dev) cudaFree(q);
    cudaFreeHost(S->hctl);
    cudaFreeHost(S->hinfo);
    delete S;
}

template <class V, class Epi>
static void bl_spmv(const BlSolver *S, const hz_mat *A, const V *x, const Epi &e, cudaStream_t cs) {
    if constexpr (std::is_same<V, float4>::value) {
        launch_spmv_ff(S->kind, S->group, mat_view<double2>(A), x, e, S->red, S->grid_spmv, cs);
    } else {
        launch_spmv<V>(d64_kind(A, S->kind), S->group, mat_view<V>(A), x, e, S->red,
                       S->grid_spmv_cv, cs);
    }
}

template <class V>
static hz_status bl_build_graph(BlSolver *S, const hz_mat *A, cudaGraph_t g) {
    cudaStream_t cs = S->cap;
    const auto mode = cudaStreamCaptureModeThreadLocal;
    const int n = S->n, ell = S->ell;
    V *x = (V *)S->x, *R = (V *)S->R, *U = (V *)S->U, *rh = (V *)S->rh;
    auto Rv = [&](int i) { return R + (size_t)i * n; };
    auto Uv = [&](int i) { return U + (size_t)i * n; };
    StateOf<V> *st = (StateOf<V> *)S->st;
    const int unroll = profile_unroll();
    cudaGraphConditionalHandle h = 0;
    std::vector<cudaGraphNode_t> leaves;
    if (unroll <= 0) HZ_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    HZ_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, mode));
    cudaMemcpyAsync(S->dctl, S->hctl, sizeof(Ctl), cudaMemcpyHostToDevice, cs);
    k_init_x<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->dctl, x);
    EpiBlInit<V> ei;
    ei.st = st; ei.info = S->dinfo; ei.ctl = S->dctl; ei.r0 = Rv(0); ei.rh = rh; ei.u0 = Uv(0); ei.h = h;
    bl_spmv<V>(S, A, x, ei, cs);
    auto iteration = [&]() {
        for (int j = 0; j < ell; ++j) {
            k_bl_u<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, j, st, U, R);
            EpiBlU<V> eu;
            eu.st = st; eu.u_next = Uv(j + 1); eu.rh = rh; eu.s = S->op_scale;
            bl_spmv<V>(S, A, Uv(j), eu, cs);
            k_bl_r<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, j, st, S->dctl, R, U, x, S->red);
            EpiBlR<V> er;
            er.st = st; er.r_next = Rv(j + 1); er.rh = rh; er.want_rho = j + 1 < ell; er.s = S->op_scale;
            bl_spmv<V>(S, A, Rv(j), er, cs);
        }
        k_bl_gram<V><<<S->grid_gram, kVecBlock, 0, cs>>>(n, ell, st, R, S->red, S->ex);
        k_bl_update<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, ell, st, S->dctl, x, R, U, rh, S->ex, S->red);
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
    bl_spmv<V>(S, A, x, et, cs);
    k_copy_out<V><<<S->grid_vec, kVecBlock, 0, cs>>>(n, S->dctl, S->dinfo, x, A->fault);
    cudaMemcpyAsync(S->hinfo, S->dinfo, sizeof(Info), cudaMemcpyDeviceToHost, cs);
    HZ_CUDA(cudaStreamEndCapture(cs, &g));
    return HZ_OK;
}

// max_i sum_j |a_ij| (the infinity norm) into *out as the bits of a
// non-negative double (which order like unsigned integers); *out starts at 0
__global__ void k_row_abs_max(int n, const int *__restrict__ rowptr, const double2 *__restrict__ val,
                              unsigned long long *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) sum += sqrt(val[k].x * val[k].x + val[k].y * val[k].y);
        if (isfinite(sum)) atomicMax(out, (unsigned long long)__double_as_longlong(sum));
    }
}

// 2^-k with 2^(k-1) <= ||A||_inf < 2^k (1 for a zero matrix): the power of
// two that brings the operator to unit scale, so that the vectors r_j = A^j r_0
// of an outer iteration and their Gram products stay inside the exponent
// range of binary32 on the double-float path
hz_status operator_scale(const hz_mat *A, double *out) {
    DevInfo d;
    HZ_TRY(dev_info(&d));
    unsigned long long *dm = nullptr, hm = 0;
    HZ_CUDA(cudaMalloc(&dm, sizeof(unsigned long long)));
    HZ_CUDA(cudaMemset(dm, 0, sizeof(unsigned long long)));
    if (A->n) k_row_abs_max<<<stream_grid(d, A->n, 256, 8), 256>>>(A->n, A->rowptr, A->val, dm);
    const cudaError_t e = cudaMemcpy(&hm, dm, sizeof(hm), cudaMemcpyDeviceToHost);
    cudaFree(dm);
    HZ_CUDA(e);
    double m;
    memcpy(&m, &hm, sizeof(m));
    int k = 0;
    if (m > 0.0 && std::isfinite(m)) std::frexp(m, &k);   // m = f 2^k, f in [0.5, 1)
    *out = std::ldexp(1.0, -k);
    return HZ_OK;
}

#define HZ_BL_ALLOC(ptr, bytes) HZ_CUDA(cudaMalloc((void **)&(ptr), std::max<size_t>((bytes), 16)))

static hz_status bl_get_solver(hz_mat *A, int ell, BlSolver **out) {
    BlSolver *S = (BlSolver *)A->solver_bl;
    if (S && (S->kind != A->spmv_kind || S->group != A->group || S->ell != ell)) {
        bl_solver_free(S);
        A->solver_bl = S = nullptr;
    }
    if (S) { *out = S; return HZ_OK; }
    DevInfo d;
    HZ_TRY(dev_info(&d));
    S = new BlSolver();
    A->solver_bl = S;   // freed with the handle even if the build below fails
    S->ell = ell;
    S->n = A->n;
    S->kind = A->spmv_kind;
    S->group = A->group;
    S->grid_spmv = spmv_grid(A, S->kind, S->group);
    S->grid_spmv_cv = spmv_grid(A, d64_kind(A, S->kind), S->group);
    S->grid_vec = vec_grid(d, A->n);
    const int np = ell + ell * (ell + 1) / 2;
    S->grid_gram = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)2 * d.num_sms,
                                                                  (int64_t)kMaxRedBlocks * kMaxRedValues / (2 * np),
                                                                  ((int64_t)A->n + kGramTile - 1) / kGramTile}));
    HZ_TRY(operator_scale(A, &S->op_scale));
    const size_t n = (size_t)A->n, vb = 16;
    HZ_BL_ALLOC(S->x, n * vb);
    HZ_BL_ALLOC(S->rh, n * vb);
    HZ_BL_ALLOC(S->R, (size_t)(ell + 1) * n * vb);
    HZ_BL_ALLOC(S->U, (size_t)(ell + 1) * n * vb);
    HZ_BL_ALLOC(S->st, sizeof(BiState<double2>));
    HZ_BL_ALLOC(S->ex, sizeof(BlExtra));
    HZ_BL_ALLOC(S->dinfo, sizeof(Info));
    HZ_BL_ALLOC(S->dctl, sizeof(Ctl));
    HZ_BL_ALLOC(S->red.partials, sizeof(double) * kMaxRedBlocks * kMaxRedValues);
    HZ_BL_ALLOC(S->red.counter, 256);
    HZ_CUDA(cudaMemset(S->red.counter, 0, 256));
    HZ_CUDA(cudaMemset(S->st, 0, sizeof(BiState<double2>)));
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
    HZ_TRY(is_ff_kind(S->kind) ? bl_build_graph<float4>(S, A, g) : bl_build_graph<double2>(S, A, g));
    HZ_CUDA(cudaGraphInstantiate(&S->exec, g, 0));
    *out = S;
    return HZ_OK;
}

// one BiCGStab(l) solve on operator `op` (A itself, or its Jacobi-scaled
// copy with the scalings in c); restart once like BiCGStab
hz_status bl_solve(hz_mat *op, int ell, const Ctl &c, Info *out, int *restarts, cudaStream_t s) {
    BlSolver *S = nullptr;
    HZ_TRY(bl_get_solver(op, ell, &S));
    *S->hctl = c;
    S->hctl->op_scale = S->op_scale;
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
