// spmv.cu -- matrix handles, SpMV variant selection (row-length histogram
// and optional timing-based autotuning), SELL-C-sigma construction and the
// hz_zspmv / hz_cspmv entry points.
#include <algorithm>
#include <climits>
#include <cmath>
#include <numeric>
#include <vector>

#include "spmv.cuh"

namespace hz {

// ---------------------------------------------------------------------------
__global__ void k_rebase(int n, const int *in, int *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = in[i] - 1;
}

__global__ void k_to_c64(int64_t n, const double2 *__restrict__ in, float2 *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = to_c64(in[i]);
}

// SELL slot values from the CSR values through the slot -> CSR map
__global__ void k_sell_gather(int64_t slots, const int *__restrict__ src, const double2 *__restrict__ val,
                              double2 *__restrict__ sval, float2 *__restrict__ sval32, float4 *__restrict__ svff) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < slots;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int k = src[i];
        const double2 v = k >= 0 ? val[k] : make_double2(0.0, 0.0);
        sval[i] = v;
        if (sval32) sval32[i] = to_c64(v);
        if (svff) svff[i] = split_ff(v);
    }
}

// ---------------------------------------------------------------------------
// Packed binary64 stream of the row blocks (HZ_SPMV_FLAT64P).  Built from
// the CSR arrays at creation and on every value refresh by three kernels,
// one warp per row block with the lane runs of the block-flat kernel
// (lane l: entries [c0, c1), U per lane).

// per group of kD64Group steps: 32 x its steps if one of its entries has a
// nonzero imaginary part (the slots it needs in pk_im), else 0
__global__ void k_pk_count(int nfblk, const int *__restrict__ fblk_k, const int *__restrict__ gbase,
                           const double2 *__restrict__ val, int *__restrict__ gim) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nfblk; b += nw) {
        const int kb = fblk_k[b], ke = fblk_k[b + 1], U = (ke - kb + 31) >> 5;
        const int c0 = min(ke, kb + lane * U), c1 = min(ke, c0 + U), g0 = gbase[b];
        for (int u0 = 0; u0 < U; u0 += kD64Group) {
            const int ue = min(U, u0 + kD64Group);
            bool cplx = false;
            for (int u = u0; u < ue; ++u)
                if (c0 + u < c1 && !zero_bits(val[c0 + u].y)) cplx = true;
            const bool any = __any_sync(0xffffffffu, cplx);
            if (lane == 0) gim[g0 + u0 / kD64Group] = any ? 32 * (ue - u0) : 0;
        }
    }
}

// the counts -> exclusive prefix sums, the offsets of the complex groups'
// parts in pk_im (-1 for a real group); one CTA, chunks of consecutive groups
// per thread, the chunk sums scanned in shared memory
constexpr int kPkScanThreads = 1024;
__global__ void __launch_bounds__(kPkScanThreads) k_pk_scan(int ng, int *__restrict__ gim) {
    __shared__ int part[kPkScanThreads];
    const int t = threadIdx.x;
    const int per = (ng + kPkScanThreads - 1) / kPkScanThreads;
    const int lo = min(ng, t * per), hi = min(ng, lo + per);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += gim[i];
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < kPkScanThreads; off <<= 1) {   // inclusive scan (Hillis-Steele)
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - sum;
    for (int i = lo; i < hi; ++i) {
        const int c = gim[i];
        gim[i] = c ? run : -1;
        run += c;
    }
}

// slot pk_base[b] + 32 u + l <- entry u of lane l's run (column -1, value 0
// past its end); imaginary parts of complex groups at their offset
__global__ void k_pk_fill(int nfblk, const int *__restrict__ fblk_k, const int *__restrict__ base,
                          const int *__restrict__ gbase, const int *__restrict__ gim, const int *__restrict__ col,
                          const double2 *__restrict__ val, int *__restrict__ pcol, double *__restrict__ pre,
                          double *__restrict__ pim) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nfblk; b += nw) {
        const int kb = fblk_k[b], ke = fblk_k[b + 1], U = (ke - kb + 31) >> 5;
        const int c0 = min(ke, kb + lane * U), c1 = min(ke, c0 + U), P = base[b], g0 = gbase[b];
        for (int u = 0; u < U; ++u) {
            const int k = c0 + u, slot = P + 32 * u + lane;
            const bool in = k < c1;
            const double2 a = in ? val[k] : make_double2(0.0, 0.0);
            pcol[slot] = in ? col[k] : -1;
            pre[slot] = a.x;
            const int o = gim[g0 + u / kD64Group];
            if (o >= 0) pim[o + 32 * (u % kD64Group) + lane] = a.y;
        }
    }
}

static hz_status pk_refresh(hz_mat *A, cudaStream_t s) {
    if (!A->pk_re) return HZ_OK;
    DevInfo d;
    HZ_TRY(dev_info(&d));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)A->nfblk + 7) / 8, (int64_t)d.num_sms * 8));
    k_pk_count<<<grid, 256, 0, s>>>(A->nfblk, A->fblk_k, A->pk_gbase, A->val, A->pk_gim);
    HZ_CUDA(cudaGetLastError());
    k_pk_scan<<<1, kPkScanThreads, 0, s>>>(A->pk_groups, A->pk_gim);
    HZ_CUDA(cudaGetLastError());
    k_pk_fill<<<grid, 256, 0, s>>>(A->nfblk, A->fblk_k, A->pk_base, A->pk_gbase, A->pk_gim, A->col, A->val,
                                   A->pk_col, A->pk_re, A->pk_im);
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
}

// smallest and largest binary exponent (IEEE field minus bias) over the
// nonzero real and imaginary parts of the values: out[0] = min, out[1] = max
// (out[0] = INT_MAX, out[1] = INT_MIN on entry); a non-finite part counts as
// exponent 1024
__global__ void k_exp_range(int64_t n, const double2 *__restrict__ val, int *out) {
    int lo = INT32_MAX, hi = INT32_MIN;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = val[i];
        const double c[2] = {v.x, v.y};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const unsigned hw = (unsigned)__double2hiint(c[q]), lw = (unsigned)__double2loint(c[q]);
            if (((hw & 0x7fffffffu) | lw) == 0u) continue;   // a zero splits exactly
            const int e = (int)((hw >> 20) & 0x7ffu) - 1023;
            lo = min(lo, e);
            hi = max(hi, e);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out, lo);
        atomicMax(out + 1, hi);
    }
}

__global__ void k_split_ff(int64_t n, const double2 *__restrict__ x, float4 *__restrict__ xff) {
    pdl_release();   // a programmatic dependent (the SpMV) may start streaming the matrix
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        xff[i] = split_ff(x[i]);
}

cudaError_t split_ff_vec(int n, const double2 *x, float4 *xff, cudaStream_t s) {
    DevInfo d;
    if (dev_info(&d) != HZ_OK) return cudaErrorUnknown;
    if (n > 0) k_split_ff<<<stream_grid(d, n, 256, 8), 256, 0, s>>>(n, x, xff);
    return cudaGetLastError();
}

template <>
MatView<double2> mat_view<double2>(const hz_mat *A) {
    MatView<double2> v{};
    v.n = A->n; v.rowptr = A->rowptr; v.col = A->col; v.val = A->val; v.vff = A->val_ff; v.svff = A->sell_vff;
    v.nfblk = A->nfblk; v.fblk = A->fblk; v.fblk_k = A->fblk_k; v.nfblk_t = A->nfblk_t; v.fblk_t = A->fblk_t; v.colp = A->col_pad; v.fault = A->fault;
    v.nchunks = A->sell_nchunks; v.chunk_off = A->sell_chunk_off; v.chunk_w = A->sell_chunk_w;
    v.perm = A->sell_perm; v.scol = A->sell_col; v.sval = A->sell_val;
    v.pk_base = A->pk_base; v.pk_gbase = A->pk_gbase; v.pk_gim = A->pk_gim; v.pk_col = A->pk_col;
    v.pk_re = A->pk_re; v.pk_im = A->pk_im;
    return v;
}

template <>
MatView<float2> mat_view<float2>(const hz_mat *A) {
    MatView<float2> v{};
    v.n = A->n; v.rowptr = A->rowptr; v.col = A->col; v.val = A->val32;
    v.nfblk = A->nfblk; v.fblk = A->fblk; v.fblk_k = A->fblk_k;
    v.nchunks = A->sell_nchunks; v.chunk_off = A->sell_chunk_off; v.chunk_w = A->sell_chunk_w;
    v.perm = A->sell_perm; v.scol = A->sell_col; v.sval = A->sell_val32;
    return v;
}

int spmv_grid(const hz_mat *A, int kind, int group, int blocks_per_sm_cap) {
    DevInfo d;
    if (dev_info(&d) != HZ_OK) return 1;
    if (kind == HZ_SPMV_FF_FLAT || kind == HZ_SPMV_FF_TMA || is_flat64(kind)) {
        // persistent: exactly the CTAs that fit at once (blocks are taken
        // grid-stride, so CTAs beyond one wave would only add a tail)
        static int occ_flat = 0, occ_tma = 0, occ_d64 = 0, occ_d64p = 0;
        int &occ = kind == HZ_SPMV_FF_TMA ? occ_tma
                   : kind == HZ_SPMV_FLAT64 ? occ_d64
                   : kind == HZ_SPMV_FLAT64P ? occ_d64p
                                             : occ_flat;
        if (occ == 0) {
            cudaError_t e;
            if (kind == HZ_SPMV_FF_TMA) {
                cudaFuncSetAttribute(k_spmv_fft<EpiStore<double2>>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_fft<EpiStore<double2>>, kFlatThreads, 0);
            } else if (kind == HZ_SPMV_FLAT64) {
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_d64b<EpiStore<double2>, false>,
                                                                  kFlatThreads, 0);
            } else if (kind == HZ_SPMV_FLAT64P) {
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_d64b<EpiStore<double2>, true>,
                                                                  kFlatThreads, 0);
            } else {
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_ffb<EpiStore<double2>>, kFlatThreads, 0);
            }
            if (e != cudaSuccess || occ < 1) occ = 1;
        }
        const int wpc = kFlatThreads / 32;
        int64_t g = std::min<int64_t>(((kind == HZ_SPMV_FF_TMA ? A->nfblk_t : A->nfblk) + wpc - 1) / wpc,
                                      (int64_t)d.num_sms * occ);
        return (int)std::max<int64_t>(1, std::min<int64_t>(g, kMaxRedBlocks));
    }
    const bool sell = kind == HZ_SPMV_SELL || kind == HZ_SPMV_SELL_FF;
    int64_t threads = sell ? (int64_t)A->sell_nchunks * 32 : (int64_t)A->n * group;
    return stream_grid(d, threads, kSpmvBlock, blocks_per_sm_cap);
}

int c64_flat_grid(const hz_mat *A) {
    DevInfo d;
    if (dev_info(&d) != HZ_OK) return 1;
    static int occ = 0;
    if (occ == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_c64b<EpiStore<float2>>, kFlatThreads, 0) !=
             cudaSuccess || occ < 1))
        occ = 1;
    const int64_t g = std::min<int64_t>(A->nfblk, (int64_t)d.num_sms * occ);
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, kMaxRedBlocks));
}

// lanes per row from the row-length histogram: about four entries per lane,
// rounded to a power of two in [2, 32]
static int pick_group(double mean_row) {
    int w = 2;
    while (w < 32 && w * 4 < mean_row) w *= 2;
    return w;
}

static hz_status build_sell(hz_mat *A, cudaStream_t s, const std::vector<int> &rp,
                            const std::vector<int> &cl, int sigma) {
    const int n = A->n;
    const int nchunks = (n + kSellC - 1) / kSellC;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    for (int w0 = 0; w0 < n; w0 += sigma) {
        const int w1 = std::min(n, w0 + sigma);
        std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int a, int b) {
            return (rp[a + 1] - rp[a]) > (rp[b + 1] - rp[b]);
        });
    }
    std::vector<int> perm((size_t)nchunks * kSellC, -1), cw(nchunks), coff(nchunks + 1);
    int64_t slots = 0;
    for (int c = 0; c < nchunks; ++c) {
        int w = 0;
        for (int l = 0; l < kSellC; ++l) {
            const int r = c * kSellC + l;
            if (r < n) {
                perm[(size_t)c * kSellC + l] = order[r];
                w = std::max(w, rp[order[r] + 1] - rp[order[r]]);
            }
        }
        cw[c] = w;
        coff[c] = (int)slots;
        slots += (int64_t)w * kSellC;
        if (slots > INT32_MAX) { set_error("SELL copy exceeds 2^31 slots"); return HZ_ERR_ARG; }
    }
    coff[nchunks] = (int)slots;
    std::vector<int> scol(slots, -1), ssrc(slots, -1);
    for (int c = 0; c < nchunks; ++c)
        for (int l = 0; l < kSellC; ++l) {
            const int row = perm[(size_t)c * kSellC + l];
            if (row < 0) continue;
            for (int j = 0; j < rp[row + 1] - rp[row]; ++j) {
                const int64_t slot = coff[c] + (int64_t)j * kSellC + l;
                scol[slot] = cl[rp[row] + j];
                ssrc[slot] = rp[row] + j;
            }
        }
    A->sell_nchunks = nchunks;
    A->sell_sigma = sigma;
    A->sell_slots = slots;
    HZ_CUDA(cudaMalloc(&A->sell_chunk_off, sizeof(int) * (nchunks + 1)));
    HZ_CUDA(cudaMalloc(&A->sell_chunk_w, sizeof(int) * std::max(nchunks, 1)));
    HZ_CUDA(cudaMalloc(&A->sell_perm, sizeof(int) * std::max<size_t>(perm.size(), 1)));
    HZ_CUDA(cudaMalloc(&A->sell_col, sizeof(int) * std::max<int64_t>(slots, 1)));
    HZ_CUDA(cudaMalloc(&A->sell_src, sizeof(int) * std::max<int64_t>(slots, 1)));
    HZ_CUDA(cudaMalloc(&A->sell_val, sizeof(double2) * std::max<int64_t>(slots, 1)));
    HZ_CUDA(cudaMemcpyAsync(A->sell_chunk_off, coff.data(), sizeof(int) * (nchunks + 1), cudaMemcpyHostToDevice, s));
    if (nchunks) {
        HZ_CUDA(cudaMemcpyAsync(A->sell_chunk_w, cw.data(), sizeof(int) * nchunks, cudaMemcpyHostToDevice, s));
        HZ_CUDA(cudaMemcpyAsync(A->sell_perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice, s));
    }
    if (slots) {
        HZ_CUDA(cudaMemcpyAsync(A->sell_col, scol.data(), sizeof(int) * slots, cudaMemcpyHostToDevice, s));
        HZ_CUDA(cudaMemcpyAsync(A->sell_src, ssrc.data(), sizeof(int) * slots, cudaMemcpyHostToDevice, s));
    }
    HZ_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
    return HZ_OK;
}

static hz_status refresh(hz_mat *A, cudaStream_t s) {
    DevInfo d;
    HZ_TRY(dev_info(&d));
    if (A->val32 && A->nnz) {
        k_to_c64<<<stream_grid(d, A->nnz, 256, 8), 256, 0, s>>>(A->nnz, A->val, A->val32);
        HZ_CUDA(cudaGetLastError());
    }
    if (A->val_ff && A->nnz) {
        k_split_ff<<<stream_grid(d, A->nnz, 256, 8), 256, 0, s>>>(A->nnz, A->val, A->val_ff);
        HZ_CUDA(cudaGetLastError());
    }
    if (A->sell_val && A->sell_slots) {
        k_sell_gather<<<stream_grid(d, A->sell_slots, 256, 8), 256, 0, s>>>(
            A->sell_slots, A->sell_src, A->val, A->sell_val, A->sell_val32, A->sell_vff);
        HZ_CUDA(cudaGetLastError());
    }
    return pk_refresh(A, s);
}

hz_status ensure_c64(hz_mat *A, cudaStream_t s) {
    if (A->val32) return HZ_OK;
    HZ_CUDA(cudaMalloc(&A->val32, sizeof(float2) * std::max(A->nnz, 1)));
    if (A->sell_val) HZ_CUDA(cudaMalloc(&A->sell_val32, sizeof(float2) * std::max<int64_t>(A->sell_slots, 1)));
    HZ_TRY(refresh(A, s));
    HZ_CUDA(cudaStreamSynchronize(s));
    return HZ_OK;
}

static hz_status autotune(hz_mat *A, cudaStream_t s) {
    if (A->n == 0) return HZ_OK;
    double2 *x = nullptr, *y = nullptr;
    HZ_CUDA(cudaMalloc(&x, sizeof(double2) * A->n));
    HZ_CUDA(cudaMalloc(&y, sizeof(double2) * A->n));
    HZ_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * A->n, s));
    cudaEvent_t e0, e1;
    HZ_CUDA(cudaEventCreate(&e0));
    HZ_CUDA(cudaEventCreate(&e1));
    std::vector<std::pair<int, int>> cand;
    for (int w : {2, 4, 8, 16, 32}) cand.push_back({HZ_SPMV_CSR_VECTOR, w});
    if (A->sell_val) cand.push_back({HZ_SPMV_SELL, 0});
    if (A->val_ff)
        for (int w : {2, 4, 8, 16, 32}) cand.push_back({HZ_SPMV_FF, w});
    if (A->sell_vff) cand.push_back({HZ_SPMV_SELL_FF, 0});
    if (A->fblk) cand.push_back({HZ_SPMV_FLAT64, 0});
    if (A->pk_re) cand.push_back({HZ_SPMV_FLAT64P, 0});
    if (A->val_ff && A->fblk) cand.push_back({HZ_SPMV_FF_FLAT, 0});
    if (A->col_pad) cand.push_back({HZ_SPMV_FF_TMA, 0});
    float best = 1e30f, best_cv = 1e30f;   // over all kinds; over the binary64 CSR-vector groups
    int group_cv = A->group;
    MatView<double2> V = mat_view<double2>(A);
    EpiStore<double2> epi{y};
    hz_status st = HZ_OK;
    for (auto &c : cand) {
        const int grid = spmv_grid(A, c.first, c.second);
        float tms[5];
        for (int rep = -1; rep < 5; ++rep) {
            cudaEventRecord(e0, s);
            if (is_ff_kind(c.first))
                launch_spmv_ff(c.first, c.second, V, A->x_ff, epi, RedScratch{}, grid, s);
            else launch_spmv<double2>(c.first, c.second, V, x, epi, RedScratch{}, grid, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = HZ_ERR_CUDA; break; }
            if (rep >= 0) cudaEventElapsedTime(&tms[rep], e0, e1);
        }
        if (st != HZ_OK) break;
        std::sort(tms, tms + 5);
        if (c.first == HZ_SPMV_CSR_VECTOR && tms[2] < best_cv) {
            best_cv = tms[2];
            group_cv = c.second;
        }
        if (tms[2] < best) {
            best = tms[2];
            A->spmv_kind = c.first;
            if (c.first == HZ_SPMV_CSR_VECTOR || c.first == HZ_SPMV_FF) A->group = c.second;
        }
    }
    // the lanes per row of the fastest binary64 CSR-vector product: the row
    // tile of this matrix's items in the persistent batched solver (and of
    // the CSR-vector kinds), whichever kind won overall
    if (A->spmv_kind != HZ_SPMV_FF) A->group = group_cv;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    if (st != HZ_OK) { set_error("SpMV autotuning launch failed"); return st; }
    return HZ_OK;
}

void free_solvers(hz_mat *A);

}  // namespace hz

using namespace hz;

extern "C" HZ_API hz_status hz_csr_create(hz_mat **out, int32_t n, int32_t nnz, const int32_t *d_rowptr,
                                          const int32_t *d_col, const hz_z *d_val, int32_t index_base,
                                          uint32_t flags, void *stream) {
    HZ_CHECK(out != nullptr, "hz_csr_create: null output handle");
    *out = nullptr;
    HZ_CHECK(n >= 0 && nnz >= 0, "hz_csr_create: negative size");
    HZ_CHECK(n <= kMaxCsrSize && nnz <= kMaxCsrSize, "hz_csr_create: n and nnz must be at most 2^31 - 4097");
    HZ_CHECK(index_base == 0 || index_base == 1, "hz_csr_create: index_base must be 0 or 1");
    HZ_CHECK(d_rowptr != nullptr, "hz_csr_create: null rowptr");
    HZ_CHECK(nnz == 0 || (d_col != nullptr && d_val != nullptr), "hz_csr_create: null col/val");
    // the kernels read values with 16-byte vector loads and copies
    HZ_CHECK(((uintptr_t)d_val & 15u) == 0 && ((uintptr_t)d_col & 3u) == 0 && ((uintptr_t)d_rowptr & 3u) == 0,
             "hz_csr_create: d_val must be 16-byte aligned, d_col and d_rowptr 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    hz_mat *A = new hz_mat();
    int dev = 0;
    cudaGetDevice(&dev);
    A->device = dev;
    A->n = n;
    A->nnz = nnz;
    A->val = (double2 *)d_val;
    auto fail = [&](hz_status st) { hz_mat_destroy(A); return st; };
    if (index_base == 1) {
        if (cudaMalloc(&A->own_rowptr, sizeof(int) * (n + 1)) != cudaSuccess ||
            cudaMalloc(&A->own_col, sizeof(int) * std::max(nnz, 1)) != cudaSuccess) {
            set_error("hz_csr_create: allocation failed");
            return fail(HZ_ERR_ALLOC);
        }
        k_rebase<<<64, 256, 0, s>>>(n + 1, d_rowptr, A->own_rowptr);
        if (nnz) k_rebase<<<256, 256, 0, s>>>(nnz, d_col, A->own_col);
        A->rowptr = A->own_rowptr;
        A->col = A->own_col;
    } else {
        A->rowptr = d_rowptr;
        A->col = d_col;
    }
    std::vector<int> rp(n + 1);
    if (cudaMemcpyAsync(rp.data(), A->rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("hz_csr_create: cannot read rowptr (is it a device pointer?)");
        return fail(HZ_ERR_CUDA);
    }
    const bool need_cols = (flags & (HZ_FLAG_VALIDATE | HZ_FLAG_SELL)) != 0;
    std::vector<int> cl;
    if (flags & HZ_FLAG_VALIDATE) {
        if (rp[0] != 0 || rp[n] != nnz) {
            set_error("hz_csr_create: rowptr[0] must be the base and rowptr[n] must equal nnz + base");
            return fail(HZ_ERR_ARG);
        }
        for (int i = 0; i < n; ++i)
            if (rp[i + 1] < rp[i]) {
                set_error("hz_csr_create: rowptr is not monotone at row " + std::to_string(i));
                return fail(HZ_ERR_ARG);
            }
    } else if (rp[n] != nnz) {
        set_error("hz_csr_create: rowptr[n] does not match nnz");
        return fail(HZ_ERR_ARG);
    }
    if (need_cols && nnz) {
        cl.resize(nnz);
        if (cudaMemcpy(cl.data(), A->col, sizeof(int) * nnz, cudaMemcpyDeviceToHost) != cudaSuccess) {
            set_error("hz_csr_create: cannot read col");
            return fail(HZ_ERR_CUDA);
        }
        if (flags & HZ_FLAG_VALIDATE)
            for (int k = 0; k < nnz; ++k)
                if (cl[k] < 0 || cl[k] >= n) {
                    set_error("hz_csr_create: column index out of range at entry " + std::to_string(k));
                    return fail(HZ_ERR_ARG);
                }
    }
    int mx = 0, mn = n ? INT32_MAX : 0;
    for (int i = 0; i < n; ++i) {
        const int l = rp[i + 1] - rp[i];
        mx = std::max(mx, l);
        mn = std::min(mn, l);
    }
    A->max_row = mx;
    A->min_row = mn;
    A->mean_row = n ? (double)nnz / n : 0.0;
    A->group = pick_group(A->mean_row);
    // row blocks for the block-flat kernels: greedy runs of at most
    // kFlatRows complete rows with at most `cap` entries; a longer row is
    // a block of its own
    // (and, for dev_k, the first entry of every block boundary row)
    std::vector<int> fb_keep;
    auto row_blocks = [&](int cap, int32_t **dev, int32_t *count, int32_t **dev_k) {
        std::vector<int> fb{0};
        for (int r = 0; r < n;) {
            int r1 = r + 1;
            while (r1 < n && r1 - r < kFlatRows && rp[r1 + 1] - rp[r] <= cap) ++r1;
            fb.push_back(r1);
            r = r1;
        }
        *count = (int32_t)fb.size() - 1;
        if (cudaMalloc(dev, sizeof(int) * fb.size()) != cudaSuccess ||
            cudaMemcpy(*dev, fb.data(), sizeof(int) * fb.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return false;
        if (!dev_k) return true;
        fb_keep = fb;
        std::vector<int> fk(fb.size());
        for (size_t b = 0; b < fb.size(); ++b) fk[b] = rp[fb[b]];
        return cudaMalloc(dev_k, sizeof(int) * fk.size()) == cudaSuccess &&
               cudaMemcpy(*dev_k, fk.data(), sizeof(int) * fk.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!row_blocks(kFlatCap, &A->fblk, &A->nfblk, &A->fblk_k)) {
        set_error("hz_csr_create: allocation failed");
        return fail(HZ_ERR_ALLOC);
    }
    // the packed binary64 stream of these blocks: U = ceil(entries / 32)
    // steps of 32 slots per block, groups of kD64Group steps (skipped when
    // the slots would not fit 31-bit offsets)
    {
        const int nb = A->nfblk;
        std::vector<int> pb(nb + 1), pg(nb + 1);
        int64_t P = 0, G = 0;
        for (int b = 0; b < nb; ++b) {
            const int64_t U = ((int64_t)rp[fb_keep[b + 1]] - rp[fb_keep[b]] + 31) / 32;
            pb[b] = (int)std::min<int64_t>(P, INT32_MAX);
            pg[b] = (int)std::min<int64_t>(G, INT32_MAX);
            P += 32 * U;
            G += (U + kD64Group - 1) / kD64Group;
        }
        if (P < INT32_MAX - 32) {
            pb[nb] = (int)P;
            pg[nb] = (int)G;
            A->pk_slots = P;
            A->pk_groups = (int32_t)G;
            if (cudaMalloc(&A->pk_base, sizeof(int) * (nb + 1)) != cudaSuccess ||
                cudaMalloc(&A->pk_gbase, sizeof(int) * (nb + 1)) != cudaSuccess ||
                cudaMalloc(&A->pk_gim, sizeof(int) * std::max<int64_t>(G, 1)) != cudaSuccess ||
                cudaMalloc(&A->pk_col, sizeof(int) * std::max<int64_t>(P, 1)) != cudaSuccess ||
                cudaMalloc(&A->pk_re, sizeof(double) * std::max<int64_t>(P, 1)) != cudaSuccess ||
                cudaMalloc(&A->pk_im, sizeof(double) * std::max<int64_t>(P, 1)) != cudaSuccess ||
                cudaMemcpy(A->pk_base, pb.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(A->pk_gbase, pg.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
                set_error("hz_csr_create: allocation failed");
                return fail(HZ_ERR_ALLOC);
            }
        }
    }
    A->spmv_kind = A->pk_re ? HZ_SPMV_FLAT64P : HZ_SPMV_FLAT64;
    hz_status st;
    if (flags & HZ_FLAG_SELL) {
        if ((st = build_sell(A, s, rp, cl, 1024)) != HZ_OK) return fail(st);
        A->spmv_kind = HZ_SPMV_SELL;
    }
    if (flags & HZ_FLAG_C64) {
        if (cudaMalloc(&A->val32, sizeof(float2) * std::max(nnz, 1)) != cudaSuccess ||
            (A->sell_val && cudaMalloc(&A->sell_val32, sizeof(float2) * std::max<int64_t>(A->sell_slots, 1)) !=
                                cudaSuccess)) {
            set_error("hz_csr_create: allocation failed");
            return fail(HZ_ERR_ALLOC);
        }
    }
    if (flags & HZ_FLAG_FF) {
        if (cudaMalloc(&A->val_ff, sizeof(float4) * std::max(nnz, 1)) != cudaSuccess ||
            cudaMalloc(&A->x_ff, sizeof(float4) * std::max(n, 1)) != cudaSuccess) {
            set_error("hz_csr_create: allocation failed");
            return fail(HZ_ERR_ALLOC);
        }
        if (n) cudaMemsetAsync(A->x_ff, 0, sizeof(float4) * n, s);
        if (A->sell_val) {
            if (cudaMalloc(&A->sell_vff, sizeof(float4) * std::max<int64_t>(A->sell_slots, 1)) != cudaSuccess) {
                set_error("hz_csr_create: allocation failed");
                return fail(HZ_ERR_ALLOC);
            }
        }
        if (!row_blocks(kTmaCap, &A->fblk_t, &A->nfblk_t, nullptr)) {
            set_error("hz_csr_create: allocation failed");
            return fail(HZ_ERR_ALLOC);
        }
        // padded column copy (16-byte aligned, 8 spare zero entries) for the
        // bulk-copy kernel, which reads whole 16-byte units around each block
        if (cudaMalloc(&A->col_pad, sizeof(int) * ((size_t)nnz + 8)) != cudaSuccess ||
            cudaMalloc(&A->fault, sizeof(int)) != cudaSuccess) {
            set_error("hz_csr_create: allocation failed");
            return fail(HZ_ERR_ALLOC);
        }
        if (nnz) cudaMemcpyAsync(A->col_pad, A->col, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(A->col_pad + nnz, 0, sizeof(int) * 8, s);
        cudaMemsetAsync(A->fault, 0, sizeof(int), s);
        // the double-float split keeps 48 bits only while every value lies in
        // [2^-100, 2^100] (both parts normal binary32 numbers); a matrix with
        // values outside that range keeps the binary64 kind
        bool in_range = true;
        if (nnz) {
            int *d_er = nullptr, h_er[2] = {INT32_MAX, INT32_MIN};
            DevInfo di;
            if (dev_info(&di) != HZ_OK || cudaMalloc(&d_er, 2 * sizeof(int)) != cudaSuccess) {
                set_error("hz_csr_create: allocation failed");
                return fail(HZ_ERR_ALLOC);
            }
            cudaMemcpyAsync(d_er, h_er, 2 * sizeof(int), cudaMemcpyHostToDevice, s);
            k_exp_range<<<stream_grid(di, nnz, 256, 8), 256, 0, s>>>(nnz, A->val, d_er);
            const cudaError_t e1 = cudaMemcpyAsync(h_er, d_er, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
            const cudaError_t e2 = cudaStreamSynchronize(s);
            cudaFree(d_er);
            if (e1 != cudaSuccess || e2 != cudaSuccess) {
                set_error("hz_csr_create: value range check failed");
                return fail(HZ_ERR_CUDA);
            }
            in_range = h_er[0] >= kFFMinExp && h_er[1] <= kFFMaxExp;
        }
        A->ff_range_ok = in_range;
        A->spmv_kind = in_range ? HZ_SPMV_FF_FLAT : A->pk_re ? HZ_SPMV_FLAT64P : HZ_SPMV_FLAT64;
    }
    if ((st = refresh(A, s)) != HZ_OK) return fail(st);
    if (flags & HZ_FLAG_AUTOTUNE) {
        if ((st = autotune(A, s)) != HZ_OK) return fail(st);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("hz_csr_create: stream error");
        return fail(HZ_ERR_CUDA);
    }
    *out = A;
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_mat_destroy(hz_mat *A) {
    if (!A) return HZ_OK;
    cudaDeviceSynchronize();
    free_solvers(A);
    free_jacobi(A);
    cudaFree(A->own_rowptr);
    cudaFree(A->own_col);
    cudaFree(A->sell_chunk_off);
    cudaFree(A->sell_chunk_w);
    cudaFree(A->sell_perm);
    cudaFree(A->sell_col);
    cudaFree(A->sell_src);
    cudaFree(A->sell_val);
    cudaFree(A->sell_vff);
    cudaFree(A->fblk);
    cudaFree(A->fblk_k);
    cudaFree(A->pk_base);
    cudaFree(A->pk_gbase);
    cudaFree(A->pk_gim);
    cudaFree(A->pk_col);
    cudaFree(A->pk_re);
    cudaFree(A->pk_im);
    cudaFree(A->fblk_t);
    cudaFree(A->col_pad);
    cudaFree(A->fault);
    cudaFree(A->sell_val32);
    cudaFree(A->val32);
    cudaFree(A->val_ff);
    cudaFree(A->x_ff);
    cudaFree(A->diag_pos);
    delete A;
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_mat_query(const hz_mat *A, hz_mat_props *p) {
    HZ_CHECK(A && p, "hz_mat_query: null argument");
    p->n = A->n;
    p->nnz = A->nnz;
    p->max_row = A->max_row;
    p->min_row = A->min_row;
    p->mean_row = A->mean_row;
    p->spmv_kind = A->spmv_kind;
    p->group = A->group;
    p->sell_slots = A->sell_slots;
    p->sell_sigma = A->sell_sigma;
    p->has_c64 = A->val32 != nullptr;
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_mat_check(const hz_mat *A, void *stream) {
    HZ_CHECK(A, "hz_mat_check: null handle");
    if (!A->fault) return HZ_OK;
    int f = 0;
    HZ_CUDA(cudaMemcpyAsync(&f, A->fault, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    HZ_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (f) {
        set_error("hz_mat_check: a bulk copy of the matrix stream did not complete within its wait limit");
        return HZ_ERR_TIMEOUT;
    }
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_mat_refresh_values(hz_mat *A, void *stream) {
    HZ_CHECK(A, "hz_mat_refresh_values: null handle");
    free_jacobi(A);   // the scaled copy is rebuilt from the new values on the next use
    return refresh(A, (cudaStream_t)stream);
}

extern "C" HZ_API hz_status hz_zspmv(const hz_mat *A, const hz_z *d_x, hz_z *d_y, void *stream) {
    HZ_CHECK(A, "hz_zspmv: null handle");
    if (A->n == 0) return HZ_OK;
    HZ_CHECK(d_x && d_y, "hz_zspmv: null vector");
    HZ_CHECK((const void *)d_x != (const void *)d_y, "hz_zspmv: x and y must not alias");
    HZ_CHECK((((uintptr_t)d_x | (uintptr_t)d_y) & 15u) == 0, "hz_zspmv: x and y must be 16-byte aligned");
    const int grid = spmv_grid(A, A->spmv_kind, A->group);
    EpiStore<double2> epi{(double2 *)d_y};
    if (is_ff_kind(A->spmv_kind)) {
        HZ_CUDA(split_ff_vec(A->n, (const double2 *)d_x, A->x_ff, (cudaStream_t)stream));
        if (A->spmv_kind == HZ_SPMV_FF_FLAT && kFlatPipe) {
            // programmatic dependent of the split: the matrix stream starts
            // while the split drains; x is gathered after griddepcontrol.wait
            HZ_CUDA(launch_pdl(k_spmv_ffb<EpiStore<double2>, true>, grid, kFlatThreads, (cudaStream_t)stream,
                               mat_view<double2>(A), (const float4 *)A->x_ff, epi, RedScratch{}));
            return HZ_OK;
        }
        HZ_CUDA(launch_spmv_ff(A->spmv_kind, A->group, mat_view<double2>(A), A->x_ff, epi,
                               RedScratch{}, grid, (cudaStream_t)stream));
        return HZ_OK;
    }
    HZ_CUDA(launch_spmv<double2>(A->spmv_kind, A->group, mat_view<double2>(A), (const double2 *)d_x, epi,
                                 RedScratch{}, grid, (cudaStream_t)stream));
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_cspmv(hz_mat *A, const hz_c *d_x, hz_c *d_y, void *stream) {
    HZ_CHECK(A, "hz_cspmv: null handle");
    if (A->n == 0) return HZ_OK;
    HZ_CHECK(d_x && d_y, "hz_cspmv: null vector");
    HZ_CHECK((const void *)d_x != (const void *)d_y, "hz_cspmv: x and y must not alias");
    HZ_TRY(ensure_c64(A, (cudaStream_t)stream));
    if (A->fblk && is_flat64(d64_kind(A, A->spmv_kind))) {
        // the block-flat kinds: the block-flat complex64 kernel
        EpiStore<float2> epi{(float2 *)d_y};
        HZ_CUDA(launch_k(false, k_spmv_c64b<EpiStore<float2>>, c64_flat_grid(A), kFlatThreads, (cudaStream_t)stream,
                         mat_view<float2>(A), (const float2 *)d_x, epi, RedScratch{}));
        return HZ_OK;
    }
    const int kind = (A->spmv_kind == HZ_SPMV_SELL || A->spmv_kind == HZ_SPMV_SELL_FF) ? HZ_SPMV_SELL
                                                                                     : HZ_SPMV_CSR_VECTOR;
    const int grid = spmv_grid(A, kind, A->group);
    EpiStore<float2> epi{(float2 *)d_y};
    HZ_CUDA(launch_spmv<float2>(kind, A->group, mat_view<float2>(A), (const float2 *)d_x, epi, RedScratch{}, grid,
                                (cudaStream_t)stream));
    return HZ_OK;
}

extern "C" HZ_API hz_status hz_mat_set_spmv(hz_mat *A, int32_t kind, int32_t group) {
    HZ_CHECK(A, "hz_mat_set_spmv: null handle");
    if (kind == HZ_SPMV_SELL) {
        HZ_CHECK(A->sell_val != nullptr, "hz_mat_set_spmv: the handle has no SELL copy (HZ_FLAG_SELL)");
        A->spmv_kind = HZ_SPMV_SELL;
        return HZ_OK;
    }
    if (kind == HZ_SPMV_FLAT64) {
        A->spmv_kind = kind;
        return HZ_OK;
    }
    if (kind == HZ_SPMV_FLAT64P) {
        HZ_CHECK(A->pk_re != nullptr, "hz_mat_set_spmv: the handle has no packed binary64 stream");
        A->spmv_kind = kind;
        return HZ_OK;
    }
    if (kind == HZ_SPMV_FF_FLAT || kind == HZ_SPMV_FF_TMA) {
        HZ_CHECK(A->val_ff != nullptr, "hz_mat_set_spmv: the handle has no double-float copy (HZ_FLAG_FF)");
        A->spmv_kind = kind;
        return HZ_OK;
    }
    if (kind == HZ_SPMV_SELL_FF) {
        HZ_CHECK(A->sell_vff != nullptr,
                 "hz_mat_set_spmv: the handle has no double-float SELL copy (HZ_FLAG_SELL | HZ_FLAG_FF)");
        A->spmv_kind = HZ_SPMV_SELL_FF;
        return HZ_OK;
    }
    HZ_CHECK(kind == HZ_SPMV_CSR_VECTOR || kind == HZ_SPMV_FF, "hz_mat_set_spmv: unknown kind");
    HZ_CHECK(kind != HZ_SPMV_FF || A->val_ff != nullptr,
             "hz_mat_set_spmv: the handle has no double-float copy (HZ_FLAG_FF)");
    HZ_CHECK(group == 2 || group == 4 || group == 8 || group == 16 || group == 32,
             "hz_mat_set_spmv: group must be 2, 4, 8, 16 or 32");
    A->spmv_kind = kind;
    A->group = group;
    return HZ_OK;
}
