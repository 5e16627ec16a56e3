// spmv.cuh -- complex CSR / SELL-C-sigma sparse matrix-vector product cores
// with fused epilogues (Section 6 of the paper: y = A x on CSR storage).
//
// Row i of y is sum_{k = rowptr[i]}^{rowptr[i+1]-1} val[k] * x[col[k]].
//
// CSR-vector: a group of W lanes (W in {2,4,8,16,32}) owns one row at a
// time; lane l accumulates entries beg+l, beg+l+W, ... with four FMAs per
// complex multiply-accumulate, then the group folds its partial sums with
// xor shuffles.  The matrix streams through L2 with evict-first hints and
// bypasses L1; the gathered x goes through the read-only cache.
//
// SELL-C-sigma (C = 32): rows are sorted by length inside windows of sigma
// rows and packed in chunks of 32 rows stored column-major, so one warp
// reads 32 consecutive slots per step; slot columns of -1 are padding.
//
// Epilogue functors see every finished row once (on one lane) and may store
// it, transform it, and add to NV per-thread reduction values that the
// kernel folds into one grid total (single pass, deterministic order).
#pragma once

#include <type_traits>

#include "arith.cuh"

namespace hz {

constexpr int kSpmvBlock = 256;
constexpr int kSellC = 32;
#ifndef HZ_FF_UNROLL
#define HZ_FF_UNROLL 4
#endif
constexpr int kFFUnroll = HZ_FF_UNROLL;
#ifndef HZ_FF_MIN_BLOCKS
#define HZ_FF_MIN_BLOCKS 1
#endif
#ifndef HZ_FF_CONTIG
#define HZ_FF_CONTIG 0
#endif
#ifndef HZ_FF_TRANSPOSE
#define HZ_FF_TRANSPOSE 0
#endif
constexpr bool kFFContig = HZ_FF_CONTIG != 0;        // contiguous row range per block
constexpr bool kFFTranspose = HZ_FF_TRANSPOSE != 0;  // lane-transposed row outputs
// block-flat double-float kernel: one warp per row block, kFlatU entries per
// lane per pass, so a row block holds up to kFlatCap = 32 * kFlatU entries
#ifndef HZ_FLAT_THREADS
#define HZ_FLAT_THREADS 128
#endif
#ifndef HZ_FLAT_U
#define HZ_FLAT_U 16
#endif
#ifndef HZ_FLAT_GROUP
#define HZ_FLAT_GROUP 8
#endif
constexpr int kFlatThreads = HZ_FLAT_THREADS;   // warps per CTA = kFlatThreads / 32
constexpr int kFlatU = HZ_FLAT_U;
constexpr int kFlatGroup = HZ_FLAT_GROUP;       // entries per lane whose loads are in flight together
constexpr int kFlatCap = 32 * kFlatU;           // entries per warp row block
constexpr int kFlatRows = 32;                   // rows per row block (one per lane in phase 2)
static_assert(kFlatU % kFlatGroup == 0, "kFlatU must be a multiple of kFlatGroup");
#ifndef HZ_FLAT_CONTIG
#define HZ_FLAT_CONTIG 0
#endif
constexpr bool kFlatContig = HZ_FLAT_CONTIG != 0;   // contiguous block range per CTA
#ifndef HZ_FLAT_PIPE
#define HZ_FLAT_PIPE 1
#endif
constexpr bool kFlatPipe = HZ_FLAT_PIPE != 0;       // column stream one group ahead
#ifndef HZ_FLAT_MIN_BLOCKS
#define HZ_FLAT_MIN_BLOCKS 4
#endif
// resident CTAs per SM asked of the register allocator: four (<= 128
// registers) is what the 32 KB slabs allow anyway, and it keeps the solver
// epilogues with a prefetched operand from dropping to three
constexpr int kFlatMinBlocks = HZ_FLAT_MIN_BLOCKS;

template <class T>
struct MatView {
    int n;
    const int *rowptr;
    const int *col;
    const T *val;
    // SELL-C-sigma (used when the kernel's W == 0)
    int nchunks;
    const int *chunk_off;
    const int *chunk_w;
    const int *perm;
    const int *scol;
    const T *sval;
    // double-float split values (used by the ff kernels), CSR and SELL order
    const float4 *vff;
    const float4 *svff;
    // row blocks of the block-flat double-float kernels: block b holds the
    // complete rows [fblk[b], fblk[b+1]) (<= 32 rows and kFlatCap entries, or
    // one longer row); fblk_t the same with kTmaCap for the bulk-copy kernel
    int nfblk;
    const int *fblk;
    const int *fblk_k;   // rowptr[fblk[b]]: a block's entry range without a dependent load
    int nfblk_t;
    const int *fblk_t;
    // padded copy of col read by the bulk-copy kernel, and its fault word
    const int *colp;
    int *fault;
    // packed binary64 stream of the row blocks (see hz_mat::pk_*)
    const int *pk_base;
    const int *pk_gbase;
    const int *pk_gim;
    const int *pk_col;
    const double *pk_re;
    const double *pk_im;
};

// Epilogue interface (every fused SpMV epilogue provides):
//   using Acc, R;  static constexpr int NV;  static constexpr bool kFFRow;
//   static void zero(Acc &);  static R total(const Acc &);
//   bool skip() const;                       grid-uniform early exit
//   void on_skip() const;                    run by one thread when skip() held
//   void row(int i, Y y, Acc (&acc)[N]) const;  Y = T, or float4 if kFFRow
//   void finish(R (&tot)[N]) const;          thread 0 of the last block
template <int W, class T, class Epi, int NV>
__device__ __forceinline__ void csr_rows(const MatView<T> &A, const T *__restrict__ x, const Epi &epi,
                                         typename Epi::Acc (&acc)[NV]) {
    const int lane = threadIdx.x & (W - 1);
    const unsigned gmask =
        (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << ((threadIdx.x & 31) & ~(W - 1)));
    const int groups = (gridDim.x * blockDim.x) / W;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) / W; row < A.n; row += groups) {
        const int beg = __ldg(A.rowptr + row), end = __ldg(A.rowptr + row + 1);
        T y = czero<T>();
        for (int k = beg + lane; k < end; k += W) {
            const T a = ld_stream(A.val + k);
            const int c = ld_stream(A.col + k);
            cmac(y, a, __ldg(x + c));
        }
#pragma unroll
        for (int off = W / 2; off > 0; off >>= 1) {
            y.x += __shfl_xor_sync(gmask, y.x, off, W);
            y.y += __shfl_xor_sync(gmask, y.y, off, W);
        }
        if (lane == 0) epi.row(row, y, acc);
    }
}

template <class T, class Epi, int NV>
__device__ __forceinline__ void sell_rows(const MatView<T> &A, const T *__restrict__ x, const Epi &epi,
                                          typename Epi::Acc (&acc)[NV]) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < A.nchunks; c += warps) {
        const int off = __ldg(A.chunk_off + c), w = __ldg(A.chunk_w + c);
        const int row = __ldg(A.perm + c * kSellC + lane);
        T y = czero<T>();
        for (int j = 0; j < w; ++j) {
            const int slot = off + j * kSellC + lane;
            const int cc = ld_stream(A.scol + slot);
            if (cc >= 0) cmac(y, ld_stream(A.sval + slot), __ldg(x + cc));
        }
        if (row >= 0) epi.row(row, y, acc);
    }
}

// row result handed to the epilogue: ff pair, or binary64 rounded once
template <class Epi, int NV>
__device__ __forceinline__ void ff_row_out(const Epi &epi, int row, float sr, float cr, float si, float ci,
                                           typename Epi::Acc (&acc)[NV]) {
    if constexpr (Epi::kFFRow) {
        const float2 r = ff_norm(sr, cr), i = ff_norm(si, ci);
        epi.row(row, make_float4(r.x, r.y, i.x, i.y), acc);
    } else {
        epi.row(row, make_double2(join_d(sr, cr), join_d(si, ci)), acc);
    }
}

// Double-float row core: the same CSR-vector schedule, with the binary64
// multiply-accumulate replaced by ff_mac on the binary32 pipes (four real
// ff products per complex entry) and an ff fold across the group's lanes.
// x is the ff split of the vector.  The row result goes to the epilogue as
// a normalized ff pair (kFFRow) or rounded once to binary64 as hi + lo.
template <int W, class Epi, int NV>
__device__ __forceinline__ void csr_rows_ff(const MatView<double2> &A, const float4 *__restrict__ x,
                                            const Epi &epi, typename Epi::Acc (&acc)[NV]) {
    const int lane = threadIdx.x & (W - 1);
    const unsigned gmask =
        (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << ((threadIdx.x & 31) & ~(W - 1)));
    const uint64_t pol = pol_evict_first();
    int row0, rstep, r_end;
    if constexpr (kFFContig) {
        // each block owns one contiguous range of rows, walked blockDim/W
        // rows at a time (x reuse between neighbouring rows stays in L1)
        rstep = blockDim.x / W;
        int chunk = (A.n + gridDim.x - 1) / gridDim.x;
        chunk = (chunk + rstep - 1) / rstep * rstep;
        row0 = blockIdx.x * chunk + (int)threadIdx.x / W;
        r_end = min(A.n, (blockIdx.x + 1) * chunk);
    } else {
        rstep = (gridDim.x * blockDim.x) / W;
        row0 = (blockIdx.x * blockDim.x + threadIdx.x) / W;
        r_end = A.n;
    }
    // with kFFTranspose, lane q of a group keeps the result of every W-th row
    // the group finishes (q = k mod W), so the output conversion and the
    // epilogue run once per W rows on all lanes instead of on one lane per row
    float ksr = 0.f, kcr = 0.f, ksi = 0.f, kci = 0.f;
    int krow = -1, q = 0;
    for (int row = row0; row < r_end; row += rstep) {
        const int beg = __ldg(A.rowptr + row), end = __ldg(A.rowptr + row + 1);
        float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
        // kFFUnroll entries per lane per step: all their loads are issued
        // before the first dependent gather, so each lane keeps several
        // HBM requests in flight instead of one.  Slots past the row end
        // hold zeros and add exact zeros (no divergent exit).
        for (int k0 = beg + lane; k0 < end; k0 += W * kFFUnroll) {
            int c[kFFUnroll];
            float4 a[kFFUnroll], v[kFFUnroll];
#pragma unroll
            for (int u = 0; u < kFFUnroll; ++u) {
                const int k = k0 + u * W;
                c[u] = k < end ? ld_stream(A.col + k, pol) : -1;
                a[u] = k < end ? ld_stream(A.vff + k, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kFFUnroll; ++u) v[u] = c[u] >= 0 ? __ldg(x + c[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < kFFUnroll; ++u) {
                ff_mac(sr, cr, a[u].x, a[u].y, v[u].x, v[u].y);
                ff_mac(sr, cr, -a[u].z, -a[u].w, v[u].z, v[u].w);
                ff_mac(si, ci, a[u].x, a[u].y, v[u].z, v[u].w);
                ff_mac(si, ci, a[u].z, a[u].w, v[u].x, v[u].y);
            }
        }
#pragma unroll
        for (int off = W / 2; off > 0; off >>= 1) {
            const float s2 = __shfl_xor_sync(gmask, sr, off, W), c2 = __shfl_xor_sync(gmask, cr, off, W);
            const float s3 = __shfl_xor_sync(gmask, si, off, W), c3 = __shfl_xor_sync(gmask, ci, off, W);
            ff_acc(sr, cr, s2);
            cr = __fadd_rn(cr, c2);
            ff_acc(si, ci, s3);
            ci = __fadd_rn(ci, c3);
        }
        if constexpr (kFFTranspose) {
            // the xor fold leaves the row total on every lane of the group
            if (lane == q) { ksr = sr; kcr = cr; ksi = si; kci = ci; krow = row; }
            if (++q == W) {
                if (krow >= 0) ff_row_out<Epi, NV>(epi, krow, ksr, kcr, ksi, kci, acc);
                q = 0;
                krow = -1;
            }
        } else {
            if (lane == 0) ff_row_out<Epi, NV>(epi, row, sr, cr, si, ci, acc);
        }
    }
    if constexpr (kFFTranspose) {
        if (krow >= 0) ff_row_out<Epi, NV>(epi, krow, ksr, kcr, ksi, kci, acc);
    }
}

// Double-float SELL-C-sigma core: one lane per row, 32 rows per chunk stored
// column-major, so each step of a warp reads 32 consecutive slots (512
// contiguous bytes of values).  kFFUnroll slots per lane are loaded before
// the first dependent gather.  No cross-lane fold, and the binary64 output
// conversion covers 32 rows per instruction.  Padding slots hold value 0 and
// column -1 (no gather; they add exact zeros).
template <class Epi, int NV>
__device__ __forceinline__ void sell_rows_ff(const MatView<double2> &A, const float4 *__restrict__ x,
                                             const Epi &epi, typename Epi::Acc (&acc)[NV]) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < A.nchunks; c += warps) {
        const int off = __ldg(A.chunk_off + c), w = __ldg(A.chunk_w + c);
        const int row = __ldg(A.perm + c * kSellC + lane);
        float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
        for (int j0 = 0; j0 < w; j0 += kFFUnroll) {
            int cc[kFFUnroll];
            float4 a[kFFUnroll], v[kFFUnroll];
#pragma unroll
            for (int u = 0; u < kFFUnroll; ++u) {
                const int slot = off + (j0 + u) * kSellC + lane;
                const bool in = j0 + u < w;
                cc[u] = in ? ld_stream(A.scol + slot) : -1;
                a[u] = in ? ld_stream(A.svff + slot) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kFFUnroll; ++u) v[u] = cc[u] >= 0 ? __ldg(x + cc[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < kFFUnroll; ++u) {
                ff_mac(sr, cr, a[u].x, a[u].y, v[u].x, v[u].y);
                ff_mac(sr, cr, -a[u].z, -a[u].w, v[u].z, v[u].w);
                ff_mac(si, ci, a[u].x, a[u].y, v[u].z, v[u].w);
                ff_mac(si, ci, a[u].z, a[u].w, v[u].x, v[u].y);
            }
        }
        if (row >= 0) ff_row_out<Epi, NV>(epi, row, sr, cr, si, ci, acc);
    }
}

// row result from packed accumulators S = (re_hi, im_hi), C = (re_lo, im_lo):
// normalised ff pair (kFFRow, both halves by one packed TwoSum) or binary64
// Optional prefetch of an epilogue's per-row operand: an epilogue that reads
// one vector entry per row may declare `using Pre`, `Pre pre(int row) const`
// and a row() that takes the loaded value as a fourth argument.  The
// pipelined block-flat core issues those loads (and the row bounds) together
// with the last group of a row block's entries, so they arrive while that
// group's values and gathers are in flight instead of after the row sums.
struct NoPre {};
template <class E, class = void>
struct PreOf {
    using T = NoPre;
    static constexpr bool kHas = false;
};
template <class E>
struct PreOf<E, std::void_t<typename E::Pre>> {
    using T = typename E::Pre;
    static constexpr bool kHas = true;
};
template <class Epi>
__device__ __forceinline__ typename PreOf<Epi>::T epi_pre(const Epi &epi, int row) {
    if constexpr (PreOf<Epi>::kHas) return epi.pre(row);
    else return NoPre{};
}
template <class Epi, class Y, int NV>
__device__ __forceinline__ void epi_row(const Epi &epi, int row, Y y, typename Epi::Acc (&acc)[NV],
                                        const typename PreOf<Epi>::T &pf) {
    if constexpr (PreOf<Epi>::kHas) epi.row(row, y, acc, pf);
    else epi.row(row, y, acc);
}

template <class Epi, int NV>
__device__ __forceinline__ void ff_row_out2(const Epi &epi, int row, f32x2 S, f32x2 C,
                                            typename Epi::Acc (&acc)[NV], const typename PreOf<Epi>::T &pf) {
    if constexpr (Epi::kFFRow) {
        f32x2 h, l;
        two_sum2(S, C, h, l);
        float hr, hi, lr, li;
        upk2(h, hr, hi);
        upk2(l, lr, li);
        epi_row(epi, row, make_float4(hr, lr, hi, li), acc, pf);
    } else {
        float sr, si, cr, ci;
        upk2(S, sr, si);
        upk2(C, cr, ci);
        epi_row(epi, row, make_double2(join_d(sr, cr), join_d(si, ci)), acc, pf);
    }
}

// Phase 2 of the block-flat kernels: lane j sums the products of row r0 + j
// (+32, ...) held in prod[] for entries [kc, kend) and hands finished rows to
// the epilogue.  A single row longer than one chunk is summed over several
// chunks, lane 0 carrying (LS, LC) until the chunk that ends at ke.
// phase 2 of a row block: lane j sums row r0 + j (a block has at most 32
// rows) over entries [rb, re) clipped to the chunk [kc, kend); rb, re and the
// epilogue operand pf were loaded for that row by the caller
template <class Epi, int NV>
__device__ __forceinline__ void flat_row_sums(const float4 *prod, int r0, int r1, int kc, int kend, int ke,
                                              bool long_row, f32x2 &LS, f32x2 &LC, const Epi &epi,
                                              typename Epi::Acc (&acc)[NV], int rb, int re,
                                              const typename PreOf<Epi>::T &pf) {
    const int row = r0 + (threadIdx.x & 31);
    if (row >= r1) return;
    const int beg = max(rb, kc), end = min(re, kend);
    f32x2 S = 0ull, C = 0ull;   // +0.0f in both lanes
    for (int k = beg; k < end; ++k) ff_cacc(S, C, prod[k - kc]);
    if (long_row) {
        f32x2 t, e;
        two_sum2(LS, S, t, e);
        LS = t;
        LC = add2(LC, add2(e, C));
        if (kend == ke) ff_row_out2<Epi, NV>(epi, row, LS, LC, acc, pf);
    } else {
        ff_row_out2<Epi, NV>(epi, row, S, C, acc, pf);
    }
}

// the same, loading the row bounds and the epilogue operand itself
template <class Epi, int NV>
__device__ __forceinline__ void flat_row_sums(const MatView<double2> &A, const float4 *prod, int r0, int r1,
                                              int kc, int kend, int ke, bool long_row, f32x2 &LS, f32x2 &LC,
                                              const Epi &epi, typename Epi::Acc (&acc)[NV]) {
    const int row = r0 + (threadIdx.x & 31);
    int rb = 0, re = 0;
    typename PreOf<Epi>::T pf{};
    if (row < r1) {
        rb = __ldg(A.rowptr + row);
        re = __ldg(A.rowptr + row + 1);
        pf = epi_pre(epi, row);
    }
    flat_row_sums<Epi, NV>(prod, r0, r1, kc, kend, ke, long_row, LS, LC, epi, acc, rb, re, pf);
}

// Block-flat double-float core, one warp per row block (complete rows: at
// most 32 rows and kFlatCap = 32*kFlatU entries, or a single longer row).
// Two phases:
//  1. lane l takes entries kb + l + 32*u (coalesced loads, every lane busy),
//     forms each entry's complex product a*x in double-float (ff_cprod) and
//     stores it to the warp's slab of shared memory; the kFlatU entries of a
//     lane go in groups of kFlatGroup (loads of a group, then its gathers,
//     then its products);
//  2. lane j sums the products of row r0 + j from the slab (packed pairs,
//     one pass since a block has at most 32 rows) and hands the row to the
//     epilogue.
// Row boundaries never enter the streaming phase, which runs like a flat
// gather-stream; warps need only __syncwarp.  A single row longer than
// kFlatCap is processed in kFlatCap-entry passes, lane 0 carrying its sum.
template <class Epi, int NV>
__device__ __forceinline__ void flat_rows_ff(const MatView<double2> &A, const float4 *__restrict__ x,
                                             const Epi &epi, typename Epi::Acc (&acc)[NV], float4 *slab) {
    const uint64_t pol = pol_evict_first();
    const int lane = threadIdx.x & 31;
    float4 *prod = slab + (threadIdx.x >> 5) * kFlatCap;
    int b_first, b_end, b_step;
    if constexpr (kFlatContig) {
        // each CTA walks one contiguous range of row blocks, its warps
        // interleaved, so neighbouring blocks (which gather overlapping x
        // ranges under a bandwidth-reducing ordering) meet in the same L1
        const int per = (A.nfblk + gridDim.x - 1) / gridDim.x;
        b_first = blockIdx.x * per + (threadIdx.x >> 5);
        b_end = min(A.nfblk, (blockIdx.x + 1) * per);
        b_step = blockDim.x >> 5;
    } else {
        b_first = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        b_end = A.nfblk;
        b_step = gridDim.x * (blockDim.x >> 5);
    }
    for (int b = b_first; b < b_end; b += b_step) {
        const int r0 = __ldg(A.fblk + b), r1 = __ldg(A.fblk + b + 1);
        const int kb = __ldg(A.rowptr + r0), ke = __ldg(A.rowptr + r1);
        const bool long_row = r1 - r0 == 1 && ke - kb > kFlatCap;
        f32x2 LS = 0ull, LC = 0ull;   // long-row carry (lane 0)
        for (int kc = kb;; kc += kFlatCap) {
            const int kend = min(ke, kc + kFlatCap);
            // phase 1: products
#pragma unroll 1
            for (int g = 0; g < kFlatU; g += kFlatGroup) {
                int c[kFlatGroup];
                float4 a[kFlatGroup], v[kFlatGroup];
#pragma unroll
                for (int u = 0; u < kFlatGroup; ++u) {
                    const int k = kc + lane + 32 * (g + u);
                    c[u] = k < kend ? ld_stream(A.col + k, pol) : -1;
                    a[u] = k < kend ? ld_stream(A.vff + k, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < kFlatGroup; ++u)
                    v[u] = c[u] >= 0 ? __ldg(x + c[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < kFlatGroup; ++u)
                    if (c[u] >= 0) prod[lane + 32 * (g + u)] = ff_cprod(a[u], v[u]);
                if (kc + 32 * (g + kFlatGroup) >= kend) break;
            }
            __syncwarp();
            // phase 2: row sums (rows clipped to this pass's entries)
            flat_row_sums<Epi, NV>(A, prod, r0, r1, kc, kend, ke, long_row, LS, LC, epi, acc);
            __syncwarp();
            if (kend >= ke) break;
        }
    }
}

// The same kernel with the column stream one group ahead: the columns of the
// next group (in this chunk, the next chunk of a long row, or the warp's next
// row block) are loaded while the current group's values and x gathers are in
// flight, so a group waits for one memory latency instead of a column load
// followed by a dependent gather.  With kLateX the kernel was launched as a
// programmatic dependent of the kernel that writes x: it streams its first
// columns and values before waiting for that kernel (griddepcontrol.wait)
// and only then gathers x.
template <class Epi, int NV, bool kLateX = false>
__device__ __forceinline__ void flat_rows_ff_pipe(const MatView<double2> &A, const float4 *__restrict__ x,
                                                  const Epi &epi, typename Epi::Acc (&acc)[NV], float4 *slab) {
    const uint64_t pol = pol_evict_first();
    const int lane = threadIdx.x & 31;
    float4 *prod = slab + (threadIdx.x >> 5) * kFlatCap;
    const int step = gridDim.x * (blockDim.x >> 5);
    // group = entries [kg, kg + 32 * kFlatGroup) of chunk [kc, kend) of
    // row block b = rows [r0, r1), entries [kb, ke)
    struct Group {
        int b, r0, r1, kb, ke, kc, kend, kg;
    };
    // a block's bounds come from four independent loads (fblk_k holds the
    // rowptr entries of the block boundaries) issued one block ahead, so the
    // switch to the next block never waits on them
    struct Meta {
        int b, r0, r1, kb, ke;
    };
    auto block_meta = [&](int b) {
        Meta m{b, 0, 0, 0, 0};
        if (b < A.nfblk) {
            m.r0 = __ldg(A.fblk + b);
            m.r1 = __ldg(A.fblk + b + 1);
            m.kb = __ldg(A.fblk_k + b);
            m.ke = __ldg(A.fblk_k + b + 1);
        }
        return m;
    };
    auto block_group = [&](const Meta &m) {
        Group q;
        q.b = m.b;
        q.r0 = m.r0;
        q.r1 = m.r1;
        q.kb = m.kb;
        q.ke = m.ke;
        q.kc = q.kg = m.kb;
        q.kend = min(m.ke, m.kb + kFlatCap);
        return q;
    };
    auto load_cols = [&](const Group &q, int (&c)[kFlatGroup]) {
#pragma unroll
        for (int u = 0; u < kFlatGroup; ++u) {
            const int k = q.kg + lane + 32 * u;
            c[u] = (q.b < A.nfblk && k < q.kend) ? ld_stream(A.col + k, pol) : -1;
        }
    };
    const int b0 = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b0 >= A.nfblk) return;
    Group cur = block_group(block_meta(b0));
    Meta ahead = block_meta(b0 + step);   // the warp's next block
    int cn[kFlatGroup];
    load_cols(cur, cn);
    f32x2 LS = 0ull, LC = 0ull;   // long-row carry (lane 0)
    bool x_ready = !kLateX;
    for (;;) {
        int c[kFlatGroup];
        float4 a[kFlatGroup], v[kFlatGroup];
#pragma unroll
        for (int u = 0; u < kFlatGroup; ++u) {
            c[u] = cn[u];
            const int k = cur.kg + lane + 32 * u;
            a[u] = c[u] >= 0 ? ld_stream(A.vff + k, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if constexpr (kLateX) {
            if (!x_ready) {
                pdl_wait();
                x_ready = true;
            }
        }
#pragma unroll
        for (int u = 0; u < kFlatGroup; ++u) v[u] = c[u] >= 0 ? __ldg(x + c[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
        // the last group of a chunk also fetches what its row sums need: this
        // lane's row bounds and the epilogue's operand for that row
        const bool chunk_done = cur.kg + 32 * kFlatGroup >= cur.kend;
        int rb = 0, re = 0;
        typename PreOf<Epi>::T pf{};
        if (chunk_done && cur.r0 + lane < cur.r1) {
            rb = __ldg(A.rowptr + cur.r0 + lane);
            re = __ldg(A.rowptr + cur.r0 + lane + 1);
            pf = epi_pre(epi, cur.r0 + lane);
        }
        // the next group, and its columns
        Group nxt = cur;
        if (!chunk_done) {
            nxt.kg = cur.kg + 32 * kFlatGroup;
        } else if (cur.kend < cur.ke) {   // next pass over the same long row
            nxt.kc = nxt.kg = cur.kend;
            nxt.kend = min(cur.ke, cur.kend + kFlatCap);
        } else {
            nxt = block_group(ahead);
            ahead = block_meta(nxt.b + step);
        }
        load_cols(nxt, cn);
#pragma unroll
        for (int u = 0; u < kFlatGroup; ++u)
            if (c[u] >= 0) prod[cur.kg - cur.kc + lane + 32 * u] = ff_cprod(a[u], v[u]);
        if (chunk_done) {
            __syncwarp();
            const bool long_row = cur.r1 - cur.r0 == 1 && cur.ke - cur.kb > kFlatCap;
            if (long_row && cur.kc == cur.kb) LS = LC = 0ull;
            flat_row_sums<Epi, NV>(prod, cur.r0, cur.r1, cur.kc, cur.kend, cur.ke, long_row, LS, LC, epi, acc, rb, re,
                                   pf);
            __syncwarp();
        }
        if (nxt.b >= A.nfblk) break;
        cur = nxt;
    }
}

// ---------------------------------------------------------------------------
// Block-flat double-float core with the matrix stream staged by bulk copies.
//
// The same row blocks and arithmetic as flat_rows_ff, but a warp's entries
// (values and columns) reach shared memory through cp.async.bulk issued one
// chunk ahead: while the warp gathers x and forms the products of chunk j,
// the copy engine already moves chunk j+1 into the warp's other stage.  Its
// row blocks (fblk_t) hold at most kTmaCap entries so that two stages of
// four warps fit beside each other; a chunk is a row block, or a
// kTmaCap-entry piece of a longer single row.
// The products overwrite the values in place (each lane reads and writes its
// own slots), and phase 2 sums them per row as before.
//
// Every wait on a stage is bounded (kStageWaitNs of wall time); on expiry
// the warp records the fault in A.fault, waits (bounded again) for its copy
// still in flight, and stops.  The row outputs are then incomplete and the
// fault word tells the host so.
constexpr int kTmaU = 8;
constexpr int kTmaCap = 32 * kTmaU;   // entries per chunk of the bulk-copy kernel
struct alignas(16) FlatStage {
    float4 val[kTmaCap];   // values of the chunk, later its products
    int col[kTmaCap + 8];  // columns from the 16-byte boundary below the chunk
};
constexpr int kTmaWarps = kFlatThreads / 32;
constexpr uint64_t kStageWaitNs = 1000000000ull;

template <class Epi, int NV>
__device__ __forceinline__ void flat_rows_ff_tma(const MatView<double2> &A, const float4 *__restrict__ x,
                                                 const Epi &epi, typename Epi::Acc (&acc)[NV],
                                                 FlatStage *stg, uint64_t *bar) {
    const uint64_t pol = pol_evict_first();
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * kTmaWarps;
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_init_fence();
    }
    __syncwarp();
    // chunk = entries [kc, kend) of row block b = rows [r0, r1), entries [kb, ke)
    struct Chunk {
        int b, r0, r1, kb, ke, kc, kend;
    };
    auto block_chunk = [&](int b) {
        Chunk c;
        c.b = b;
        c.r0 = c.r1 = c.kb = c.ke = c.kc = c.kend = 0;
        if (b < A.nfblk_t) {
            c.r0 = __ldg(A.fblk_t + b);
            c.r1 = __ldg(A.fblk_t + b + 1);
            c.kb = __ldg(A.rowptr + c.r0);
            c.ke = __ldg(A.rowptr + c.r1);
            c.kc = c.kb;
            c.kend = min(c.ke, c.kb + kTmaCap);
        }
        return c;
    };
    auto issue = [&](const Chunk &c, int s) {
        if (lane != 0) return;
        const int cnt = c.kend - c.kc;
        if (cnt == 0) {   // rows without entries: complete the phase with no copy
            mbar_arrive(bar + s);
            return;
        }
        const int ca = c.kc & ~3, ce = (c.kend + 3) & ~3;
        const unsigned bv = 16u * (unsigned)cnt, bc = 4u * (unsigned)(ce - ca);
        mbar_arrive_tx(bar + s, bv + bc);
        bulk_load(stg[s].val, A.vff + c.kc, bv, bar + s, pol);
        bulk_load(stg[s].col, A.colp + ca, bc, bar + s, pol);
    };
    Chunk cur = block_chunk(blockIdx.x * kTmaWarps + (threadIdx.x >> 5));
    if (cur.b >= A.nfblk_t) return;
    issue(cur, 0);
    unsigned phase = 0;   // bit s: parity of stage s's next completion
    int s = 0;
    f32x2 LS = 0ull, LC = 0ull;   // long-row carry (lane 0)
    for (;;) {
        Chunk nxt;
        if (cur.kend < cur.ke) {   // next piece of the same long row
            nxt = cur;
            nxt.kc = cur.kend;
            nxt.kend = min(cur.ke, cur.kend + kTmaCap);
        } else {
            nxt = block_chunk(cur.b + nwarps);
        }
        const bool more = nxt.b < A.nfblk_t;
        if (more) issue(nxt, s ^ 1);
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar + s, (phase >> s) & 1u, kStageWaitNs));
        phase ^= 1u << s;
        if (!ok) {
            if (lane == 0) {
                atomicExch(A.fault, 1);
                mbar_wait_bounded(bar + s, ((phase >> s) & 1u) ^ 1u, kStageWaitNs);
                if (more) mbar_wait_bounded(bar + (s ^ 1), (phase >> (s ^ 1)) & 1u, kStageWaitNs);
            }
            __syncwarp();
            return;
        }
        FlatStage &S = stg[s];
        const int cnt = cur.kend - cur.kc, off = cur.kc & 3;
        // phase 1: products
        int c[kTmaU];
        float4 v[kTmaU];
#pragma unroll
        for (int u = 0; u < kTmaU; ++u) {
            const int k = lane + 32 * u;
            c[u] = k < cnt ? S.col[off + k] : -1;
        }
#pragma unroll
        for (int u = 0; u < kTmaU; ++u) v[u] = c[u] >= 0 ? __ldg(x + c[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kTmaU; ++u) {
            const int k = lane + 32 * u;
            if (c[u] >= 0) S.val[k] = ff_cprod(S.val[k], v[u]);
        }
        __syncwarp();
        // phase 2: row sums (rows clipped to this chunk's entries)
        const bool long_row = cur.r1 - cur.r0 == 1 && cur.ke - cur.kb > kTmaCap;
        if (long_row && cur.kc == cur.kb) LS = LC = 0ull;
        flat_row_sums<Epi, NV>(A, S.val, cur.r0, cur.r1, cur.kc, cur.kend, cur.ke, long_row, LS, LC, epi, acc);
        // the copy issued at the top of the next iteration refills this
        // stage: order this lane's reads and writes of it before that copy
        fence_async_smem();
        __syncwarp();
        if (!more) break;
        cur = nxt;
        s ^= 1;
    }
}

// ---------------------------------------------------------------------------
// Block-flat binary64 core with contiguous lane runs (HZ_SPMV_FLAT64 on the
// caller's CSR arrays; HZ_SPMV_FLAT64P, the default, on the handle's packed
// copy of the row blocks, whose slots hold step u of the 32 lane runs
// side by side so every load is coalesced, and whose groups without a
// nonzero imaginary part store none).
//
// On GB300 the binary64 pipe retires about 1.7 lanes per SM per clock, and a
// warp instruction occupies it for the same time whether 32 lanes or one are
// active, so a binary64 SpMV is bound by the number of binary64 warp
// instructions, not by the number of multiply-adds.  A group of lanes per
// row leaves lanes idle at every row end and folds partial sums with extra
// additions; here every lane of a warp runs one contiguous stretch of
// ceil(nnz_block / 32) entries of its row block and accumulates it with four
// FMAs per entry (the minimum for a complex multiply-accumulate), switching
// rows inside its stretch as the row pointers say.  A row that crosses the
// boundary between two lanes' stretches is finished in phase 2 from the
// lanes' partial sums: the tail of the lane where it starts, the whole
// stretch of every lane in between and the head of the lane where it ends,
// added in that order (storage order of the entries).  Row blocks are those
// of the block-flat double-float kernel (<= 32 complete rows and <= 512
// entries, or one longer row), so phase 2 is one row per lane.
//
// Helmholtz operators with a real wavenumber are real away from their
// impedance boundary (stiffness and mass entries); where a whole group of a
// warp (kD64Group entries per lane) holds values with zero imaginary parts,
// the group takes two FMAs per entry instead of four.  The skipped terms are
// exact zeros for finite x, so the sums are the same numbers (up to the sign
// of a zero result); an infinite or NaN x turns the skipped 0 * x into NaN,
// which the lane applies to its partial sum when it flushes the run.
struct alignas(16) D64Seg {
    double2 head[32];   // lane l: its first run when that run's row began in an earlier lane
    double2 tail[32];   // lane l: its last run when that run's row continues in a later lane
    double2 full[32];   // rows that lie inside one lane's stretch, by row offset
    int rp[33];         // row pointers of the block's rows (rp[nr] = end of the block)
};
#ifndef HZ_D64_GROUP
#define HZ_D64_GROUP 8
#endif
constexpr int kD64Group = HZ_D64_GROUP;   // entries per lane whose loads are in flight together
#ifndef HZ_D64_MIN_BLOCKS
#define HZ_D64_MIN_BLOCKS 4
#endif
constexpr int kD64MinBlocks = HZ_D64_MIN_BLOCKS;   // resident CTAs per SM asked of the register allocator
#ifndef HZ_D64_TWO_ACC
#define HZ_D64_TWO_ACC 1
#endif
constexpr bool kD64TwoAcc = HZ_D64_TWO_ACC != 0;   // even / odd entries of a group in two accumulators
#ifndef HZ_D64_REAL_GROUPS
#define HZ_D64_REAL_GROUPS 1
#endif
constexpr bool kD64RealGroups = HZ_D64_REAL_GROUPS != 0;   // two FMAs per entry for real-valued groups
#ifndef HZ_D64_PIPE
#define HZ_D64_PIPE 1
#endif
constexpr bool kD64Pipe = HZ_D64_PIPE != 0;   // column stream one group ahead
#ifndef HZ_D64_ROW_AHEAD
#define HZ_D64_ROW_AHEAD 1
#endif
constexpr bool kD64RowAhead = HZ_D64_ROW_AHEAD != 0;   // row pointers and epilogue operands one block ahead

// +0 or -0, by the bit pattern (integer pipe; a binary64 compare would
// occupy the binary64 pipe like an FMA)
__device__ __forceinline__ bool zero_bits(double v) {
    return ((__double2hiint(v) & 0x7fffffff) | __double2loint(v)) == 0;
}

// finite (exponent field not all ones), by the bit pattern
__device__ __forceinline__ bool finite1(double v) { return (__double2hiint(v) & 0x7ff00000) != 0x7ff00000; }

__device__ __forceinline__ double2 ld_stream_l1(const double2 *ptr, uint64_t pol) {
    double2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_stream_l1(const double *ptr, uint64_t pol) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ int ld_stream_l1(const int *ptr, uint64_t pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}

// The warp takes row blocks b0, b0 + step, ... below bend (a kernel of its
// own: grid-stride over all blocks; the batched solver: one block per warp
// of a work item).
// G: steps per group (the packed stream's groups are kD64Group steps).
template <class Epi, int NV, bool PK, int G = kD64Group>
__device__ __forceinline__ void flat_rows_d64(const MatView<double2> &A, const double2 *__restrict__ x,
                                              const Epi &epi, typename Epi::Acc (&acc)[NV], D64Seg *sg, int b0,
                                              int step, int bend) {
    static_assert(!PK || G == kD64Group, "the packed stream is laid out in groups of kD64Group steps");
    const uint64_t pol = pol_evict_first();
    const int lane = threadIdx.x & 31;
    // a row block's bounds and this lane's stretch [c0, c1) of its entries
    // [kb, ke) (U entries per lane); packed: its first slot P and first group gb
    struct Blk {
        int b, r0, r1, kb, ke, U, c0, c1, P, gb;
    };
    auto blk = [&](int bb) {
        Blk m{bb, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (bb < bend) {
            m.r0 = __ldg(A.fblk + bb);
            m.r1 = __ldg(A.fblk + bb + 1);
            m.kb = __ldg(A.fblk_k + bb);
            m.ke = __ldg(A.fblk_k + bb + 1);
            m.U = (m.ke - m.kb + 31) >> 5;
            m.c0 = min(m.ke, m.kb + lane * m.U);
            m.c1 = min(m.ke, m.c0 + m.U);
            if constexpr (PK) {
                m.P = __ldg(A.pk_base + bb);
                m.gb = __ldg(A.pk_gbase + bb);
            }
        }
        return m;
    };
    // the columns of steps [u0, u0 + G) of block m's lane runs (-1 past the
    // run's end) and, packed, where the group keeps its imaginary parts
    // (-1: nowhere, all are zero); CSR order: entries c0 + u0 + u
    auto cols = [&](const Blk &m, int u0, int (&c)[G], int &gim) {
        if constexpr (PK) {
#pragma unroll
            for (int u = 0; u < G; ++u)
                c[u] = u0 + u < m.U ? ld_stream_l1(A.pk_col + m.P + 32 * (u0 + u) + lane, pol) : -1;
            gim = u0 < m.U ? __ldg(A.pk_gim + m.gb + u0 / G) : -1;
        } else {
            const int k0 = m.c0 + u0;
#pragma unroll
            for (int u = 0; u < G; ++u) c[u] = k0 + u < m.c1 ? ld_stream_l1(A.col + k0 + u, pol) : -1;
            gim = 0;
        }
    };
    Blk cur = blk(b0), ahead = blk(b0 + step);
    // the column stream runs one group ahead (into the next row block at the
    // end of one), so a group's x gathers wait for one load, not two; each
    // lane's row pointer and epilogue operand come one row block ahead
    int cn[G], gn = -1;
    if (kD64Pipe) cols(cur, 0, cn, gn);
    auto row_start = [&](const Blk &m) { return lane < m.r1 - m.r0 ? __ldg(A.rowptr + m.r0 + lane) : 0; };
    auto row_pre = [&](const Blk &m) {
        typename PreOf<Epi>::T q{};
        if (lane < m.r1 - m.r0) q = epi_pre(epi, m.r0 + lane);
        return q;
    };
    int rp_cur = kD64RowAhead ? row_start(cur) : 0;
    typename PreOf<Epi>::T pf_cur = kD64RowAhead ? row_pre(cur) : typename PreOf<Epi>::T{};
    for (int b = b0; b < bend; b += step) {
        const int r0 = cur.r0, r1 = cur.r1, kb = cur.kb, ke = cur.ke;
        const int nr = r1 - r0;
        if (!kD64RowAhead) {
            rp_cur = row_start(cur);
            pf_cur = row_pre(cur);
        }
        const typename PreOf<Epi>::T pf = pf_cur;
        if (lane < nr) sg->rp[lane] = rp_cur;
        if (lane == 0) sg->rp[nr] = ke;
        __syncwarp();
        if (kD64RowAhead && ahead.b < bend) {
            rp_cur = row_start(ahead);
            pf_cur = row_pre(ahead);
        }
        const int U = cur.U, c0 = cur.c0, c1 = cur.c1;
        // the row holding c0: the last j < nr with rp[j] <= c0 (rows without
        // entries before it are skipped, since their rp equals the next one's)
        int j = 0;
        if (c0 < c1) {
            int hi = nr - 1;
            while (j < hi) {
                const int mid = (j + hi + 1) >> 1;
                if (sg->rp[mid] <= c0) j = mid;
                else hi = mid - 1;
            }
        }
        int nxt = sg->rp[j + 1];   // first entry of the next row (> c0)
        int seg0 = c0;             // first entry of the current run
        double2 s = make_double2(0.0, 0.0), s2 = make_double2(0.0, 0.0);
        bool nan_re = false, nan_im = false;   // a real group met a non-finite x (see below)
        // a finished run [beg, end) of row jj: a head, a tail, or a whole row
        auto flush = [&](int jj, int beg, int end) {
            if (beg == end) return;
            double2 t = cadd(s, s2);
            if (nan_re) t.x = __longlong_as_double(0x7ff8000000000000ll);
            if (nan_im) t.y = __longlong_as_double(0x7ff8000000000000ll);
            if (beg == c0 && sg->rp[jj] < c0) sg->head[lane] = t;
            else if (end == c1 && sg->rp[jj + 1] > c1) sg->tail[lane] = t;
            else sg->full[jj] = t;
        };
#pragma unroll 1
        for (int u0 = 0; u0 < U; u0 += G) {
            const int k0 = c0 + u0;
            int c[G], gim;
            double ar[G], ai[G];
            double2 v[G];
            if constexpr (kD64Pipe) {
#pragma unroll
                for (int u = 0; u < G; ++u) c[u] = cn[u];
                gim = gn;
            } else {
                cols(cur, u0, c, gim);
            }
            if constexpr (PK) {
                // coalesced: step u of all 32 lanes is 32 consecutive slots
#pragma unroll
                for (int u = 0; u < G; ++u)
                    ar[u] = u0 + u < U ? ld_stream_l1(A.pk_re + cur.P + 32 * (u0 + u) + lane, pol) : 0.0;
                if (gim >= 0) {
#pragma unroll
                    for (int u = 0; u < G; ++u)
                        ai[u] = u0 + u < U ? ld_stream_l1(A.pk_im + gim + 32 * u + lane, pol) : 0.0;
                } else {
#pragma unroll
                    for (int u = 0; u < G; ++u) ai[u] = 0.0;
                }
            } else {
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    const double2 a = k0 + u < c1 ? ld_stream_l1(A.val + k0 + u, pol) : make_double2(0.0, 0.0);
                    ar[u] = a.x;
                    ai[u] = a.y;
                }
            }
            if constexpr (kD64Pipe) {
                if (u0 + G < U) cols(cur, u0 + G, cn, gn);
                else cols(ahead, 0, cn, gn);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) v[u] = c[u] >= 0 ? __ldg(x + c[u]) : make_double2(0.0, 0.0);
            // a group of the warp whose values all have a zero imaginary part
            // needs two FMAs per entry, not four: the terms -Im(a) Im(x) and
            // Im(a) Re(x) are exact zeros.  Packed, the stream says so; else
            // it is decided on the values alone, after the gathers are
            // issued, so neither waits for the other
            bool all_real;
            if constexpr (PK) {
                all_real = gim < 0;
            } else {
                bool real = true;
#pragma unroll
                for (int u = 0; u < G; ++u) real = real && zero_bits(ai[u]);
                all_real = kD64RealGroups && __all_sync(0xffffffffu, real);
            }
            auto run = [&](auto real_tag) {
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    const int k = k0 + u;
                    if (k < c1) {
                        while (k == nxt && j < nr - 1) {   // row j ends before entry k
                            flush(j, seg0, k);
                            ++j;
                            nxt = sg->rp[j + 1];
                            s = s2 = make_double2(0.0, 0.0);
                            nan_re = nan_im = false;
                            seg0 = k;
                        }
                        // even and odd entries of the group go to two
                        // accumulators: two dependent FMA chains per lane
                        double2 &q = (kD64TwoAcc && (u & 1)) ? s2 : s;
                        if constexpr (decltype(real_tag)::value) {
                            q.x = fma(ar[u], v[u].x, q.x);
                            q.y = fma(ar[u], v[u].y, q.y);
                            // the skipped 0 * Im(x) and 0 * Re(x) are NaN for a
                            // non-finite x: remembered and applied at the flush
                            nan_re = nan_re || !finite1(v[u].y);
                            nan_im = nan_im || !finite1(v[u].x);
                        } else {
                            cmac(q, make_double2(ar[u], ai[u]), v[u]);
                        }
                    }
                }
            };
            if (all_real) run(std::true_type{});
            else run(std::false_type{});
        }
        // a block without entries ran no group: the next block's columns
        if (kD64Pipe && U == 0) cols(ahead, 0, cn, gn);
        if (c0 < c1) flush(j, seg0, c1);
        __syncwarp();
        // phase 2: lane j finishes row r0 + j
        if (lane < nr) {
            const int rb = sg->rp[lane], re = sg->rp[lane + 1];
            double2 y = make_double2(0.0, 0.0);
            if (re > rb) {
                // (clamped: with monotone row pointers both are in 0..31 already)
                const int la = min(31, max(0, (rb - kb) / U)), lb = min(31, max(la, (re - 1 - kb) / U));
                if (la == lb) {
                    y = sg->full[lane];
                } else {
                    y = sg->tail[la];
                    for (int l = la + 1; l < lb; ++l) y = cadd(y, sg->head[l]);
                    y = cadd(y, sg->head[lb]);
                }
            }
            epi_row(epi, r0 + lane, y, acc, pf);
        }
        __syncwarp();
        cur = ahead;
        ahead = blk(b + 2 * step);
    }
}

// per-thread accumulators -> one grid total -> epi.finish (last block)
template <class Epi, int NV>
__device__ __forceinline__ void spmv_reduce(const Epi &epi, typename Epi::Acc (&acc)[NV], RedScratch red) {
    using R = typename Epi::R;
    R tot[NV];
    if (grid_reduce_acc(acc, red, tot, [](const typename Epi::Acc &a) { return Epi::total(a); })) {
        if (threadIdx.x == 0) epi.finish(tot);
    }
}

// the block-flat binary64 kernel (kFlatThreads threads, row blocks, contiguous lane runs)
template <class Epi, bool PK = false>
__global__ void __launch_bounds__(kFlatThreads, kD64MinBlocks) k_spmv_d64b(MatView<double2> A,
                                                                            const double2 *__restrict__ x, Epi epi,
                                                                            RedScratch red) {
    __shared__ D64Seg seg[kFlatThreads / 32];
    constexpr int NV = Epi::NV > 0 ? Epi::NV : 1;
    pdl_wait();
    pdl_release();
    if (epi.skip()) {   // grid-uniform early exit; one thread reports it to the epilogue
        if (blockIdx.x == 0 && threadIdx.x == 0) epi.on_skip();
        return;
    }
    typename Epi::Acc acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) Epi::zero(acc[j]);
    const int wpc = blockDim.x >> 5;
    flat_rows_d64<Epi, NV, PK>(A, x, epi, acc, &seg[threadIdx.x >> 5], blockIdx.x * wpc + (threadIdx.x >> 5),
                               gridDim.x * wpc, A.nfblk);
    if constexpr (Epi::NV > 0) spmv_reduce<Epi, NV>(epi, acc, red);
}


template <int W, class T, class Epi>
__global__ void __launch_bounds__(kSpmvBlock) k_spmv(MatView<T> A, const T *__restrict__ x, Epi epi,
                                                     RedScratch red) {
    constexpr int NV = Epi::NV > 0 ? Epi::NV : 1;
    pdl_wait();
    pdl_release();
    if (epi.skip()) {   // grid-uniform early exit; one thread reports it to the epilogue
        if (blockIdx.x == 0 && threadIdx.x == 0) epi.on_skip();
        return;
    }
    typename Epi::Acc acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) Epi::zero(acc[j]);
    if constexpr (W == 0) sell_rows<T, Epi, NV>(A, x, epi, acc);
    else csr_rows<W, T, Epi, NV>(A, x, epi, acc);
    if constexpr (Epi::NV > 0) spmv_reduce<Epi, NV>(epi, acc, red);
}

// the same kernel on the double-float path (x given as its ff split)
template <int W, class Epi>
__global__ void __launch_bounds__(kSpmvBlock, HZ_FF_MIN_BLOCKS) k_spmv_ff(MatView<double2> A, const float4 *__restrict__ x, Epi epi,
                                                        RedScratch red) {
    constexpr int NV = Epi::NV > 0 ? Epi::NV : 1;
    pdl_wait();
    pdl_release();
    if (epi.skip()) {   // grid-uniform early exit; one thread reports it to the epilogue
        if (blockIdx.x == 0 && threadIdx.x == 0) epi.on_skip();
        return;
    }
    typename Epi::Acc acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) Epi::zero(acc[j]);
    if constexpr (W == 0) sell_rows_ff<Epi, NV>(A, x, epi, acc);
    else csr_rows_ff<W, Epi, NV>(A, x, epi, acc);
    if constexpr (Epi::NV > 0) spmv_reduce<Epi, NV>(epi, acc, red);
}

// the block-flat double-float kernel (kFlatThreads threads, row blocks);
// kLateX: see flat_rows_ff_pipe (only for epilogues that read nothing the
// preceding kernel writes, and skip() == false)
template <class Epi, bool kLateX = false>
__global__ void __launch_bounds__(kFlatThreads, kFlatMinBlocks) k_spmv_ffb(MatView<double2> A, const float4 *__restrict__ x, Epi epi,
                                                           RedScratch red) {
    __shared__ float4 prod[(kFlatThreads / 32) * kFlatCap];   // one slab per warp
    constexpr int NV = Epi::NV > 0 ? Epi::NV : 1;
    static_assert(!kLateX || kFlatPipe, "the late wait needs the pipelined core");
    if constexpr (!kLateX) pdl_wait();
    pdl_release();
    if (epi.skip()) {   // grid-uniform early exit; one thread reports it to the epilogue
        if (blockIdx.x == 0 && threadIdx.x == 0) epi.on_skip();
        return;
    }
    typename Epi::Acc acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) Epi::zero(acc[j]);
    if constexpr (kFlatPipe) flat_rows_ff_pipe<Epi, NV, kLateX>(A, x, epi, acc, prod);
    else flat_rows_ff<Epi, NV>(A, x, epi, acc, prod);
    if constexpr (kLateX) pdl_wait();   // a warp without row blocks still waits before leaving
    if constexpr (Epi::NV > 0) spmv_reduce<Epi, NV>(epi, acc, red);
}

// the block-flat double-float kernel with bulk-copy staging (kFlatThreads
// threads; two stages of FlatStage per warp)
template <class Epi>
__global__ void __launch_bounds__(kFlatThreads) k_spmv_fft(MatView<double2> A, const float4 *__restrict__ x, Epi epi,
                                                           RedScratch red) {
    __shared__ FlatStage stg[kTmaWarps][2];
    __shared__ uint64_t bar[kTmaWarps][2];
    constexpr int NV = Epi::NV > 0 ? Epi::NV : 1;
    pdl_wait();
    pdl_release();
    if (epi.skip()) {   // grid-uniform early exit; one thread reports it to the epilogue
        if (blockIdx.x == 0 && threadIdx.x == 0) epi.on_skip();
        return;
    }
    typename Epi::Acc acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) Epi::zero(acc[j]);
    const int w = threadIdx.x >> 5;
    flat_rows_ff_tma<Epi, NV>(A, x, epi, acc, stg[w], bar[w]);
    if constexpr (Epi::NV > 0) spmv_reduce<Epi, NV>(epi, acc, red);
}

// ---------------------------------------------------------------------------
// Block-flat complex64 kernel: the row blocks and two phases of the
// double-float kernel with complex64 values (the mixed solver's inner
// operator) and plain binary32 arithmetic: phase 1 forms a_k x_col(k) (four
// FMA-pipe operations) into the warp's slab, phase 2 sums each row in
// storage order.
template <class Epi, int NV>
__device__ __forceinline__ void flat_rows_c64(const MatView<float2> &A, const float2 *__restrict__ x, const Epi &epi,
                                              typename Epi::Acc (&acc)[NV], float2 *slab) {
    const uint64_t pol = pol_evict_first();
    const int lane = threadIdx.x & 31;
    float2 *prod = slab + (threadIdx.x >> 5) * kFlatCap;
    const int step = gridDim.x * (blockDim.x >> 5);
    // the schedule of flat_rows_ff_pipe: columns one group ahead, the next
    // block's bounds one block ahead, row bounds with a chunk's last group
    struct Group {
        int b, r0, r1, kb, ke, kc, kend, kg;
    };
    struct Meta {
        int b, r0, r1, kb, ke;
    };
    auto block_meta = [&](int b) {
        Meta m{b, 0, 0, 0, 0};
        if (b < A.nfblk) {
            m.r0 = __ldg(A.fblk + b);
            m.r1 = __ldg(A.fblk + b + 1);
            m.kb = __ldg(A.fblk_k + b);
            m.ke = __ldg(A.fblk_k + b + 1);
        }
        return m;
    };
    auto block_group = [&](const Meta &m) {
        Group q;
        q.b = m.b;
        q.r0 = m.r0;
        q.r1 = m.r1;
        q.kb = m.kb;
        q.ke = m.ke;
        q.kc = q.kg = m.kb;
        q.kend = min(m.ke, m.kb + kFlatCap);
        return q;
    };
    auto load_cols = [&](const Group &q, int (&c)[kFlatGroup]) {
#pragma unroll
        for (int u = 0; u < kFlatGroup; ++u) {
            const int k = q.kg + lane + 32 * u;
            c[u] = (q.b < A.nfblk && k < q.kend) ? ld_stream(A.col + k, pol) : -1;
        }
    };
    const int b0 = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b0 >= A.nfblk) return;
    Group cur = block_group(block_meta(b0));
    Meta ahead = block_meta(b0 + step);
    int cn[kFlatGroup];
    load_cols(cur, cn);
    float2 carry = make_float2(0.f, 0.f);   // long-row carry (lane 0)
    for (;;) {
        int c[kFlatGroup];
        float2 a[kFlatGroup], v[kFlatGroup];
#pragma unroll
        for (int u = 0; u < kFlatGroup; ++u) {
            c[u] = cn[u];
            const int k = cur.kg + lane + 32 * u;
            a[u] = c[u] >= 0 ? ld_stream(A.val + k) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kFlatGroup; ++u) v[u] = c[u] >= 0 ? __ldg(x + c[u]) : make_float2(0.f, 0.f);
        const bool chunk_done = cur.kg + 32 * kFlatGroup >= cur.kend;
        int rb = 0, re = 0;
        if (chunk_done && cur.r0 + lane < cur.r1) {
            rb = __ldg(A.rowptr + cur.r0 + lane);
            re = __ldg(A.rowptr + cur.r0 + lane + 1);
        }
        Group nxt = cur;
        if (!chunk_done) {
            nxt.kg = cur.kg + 32 * kFlatGroup;
        } else if (cur.kend < cur.ke) {   // next pass over the same long row
            nxt.kc = nxt.kg = cur.kend;
            nxt.kend = min(cur.ke, cur.kend + kFlatCap);
        } else {
            nxt = block_group(ahead);
            ahead = block_meta(nxt.b + step);
        }
        load_cols(nxt, cn);
#pragma unroll
        for (int u = 0; u < kFlatGroup; ++u)
            if (c[u] >= 0) prod[cur.kg - cur.kc + lane + 32 * u] = cmul(a[u], v[u]);
        if (chunk_done) {
            __syncwarp();
            const bool long_row = cur.r1 - cur.r0 == 1 && cur.ke - cur.kb > kFlatCap;
            if (long_row && cur.kc == cur.kb) carry = make_float2(0.f, 0.f);
            const int row = cur.r0 + lane;
            if (row < cur.r1) {
                const int beg = max(rb, cur.kc), end = min(re, cur.kend);
                float2 y = make_float2(0.f, 0.f);
                for (int k = beg; k < end; ++k) {
                    const float2 q = prod[k - cur.kc];
                    y.x += q.x;
                    y.y += q.y;
                }
                if (long_row) {
                    carry.x += y.x;
                    carry.y += y.y;
                    if (cur.kend == cur.ke) epi.row(row, carry, acc);
                } else {
                    epi.row(row, y, acc);
                }
            }
            __syncwarp();
        }
        if (nxt.b >= A.nfblk) break;
        cur = nxt;
    }
}

template <class Epi>
__global__ void __launch_bounds__(kFlatThreads) k_spmv_c64b(MatView<float2> A, const float2 *__restrict__ x, Epi epi,
                                                            RedScratch red) {
    __shared__ float2 prod[(kFlatThreads / 32) * kFlatCap];   // one slab per warp
    constexpr int NV = Epi::NV > 0 ? Epi::NV : 1;
    pdl_wait();
    pdl_release();
    if (epi.skip()) {
        if (blockIdx.x == 0 && threadIdx.x == 0) epi.on_skip();
        return;
    }
    typename Epi::Acc acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) Epi::zero(acc[j]);
    flat_rows_c64<Epi, NV>(A, x, epi, acc, prod);
    if constexpr (Epi::NV > 0) spmv_reduce<Epi, NV>(epi, acc, red);
}

// grid of k_spmv_c64b: the CTAs that fit at once
int c64_flat_grid(const hz_mat *A);

// binary64 -> double-float split of a vector (xff[i] = split_ff(x[i])), on stream s
cudaError_t split_ff_vec(int n, const double2 *x, float4 *xff, cudaStream_t s);

// ---------------------------------------------------------------------------
// plain store epilogue: y[i] = (A x)_i
template <class T>
struct EpiStore {
    using R = typename Cplx<T>::R;
    using Acc = R;
    static constexpr int NV = 0;
    static constexpr bool kFFRow = false;
    T *y;
    __device__ static void zero(Acc &a) { a = Acc(0); }
    __device__ static R total(const Acc &a) { return a; }
    __device__ bool skip() const { return false; }
    __device__ void on_skip() const {}
    template <int N> __device__ void row(int i, T v, Acc (&)[N]) const { y[i] = v; }
    template <int N> __device__ void finish(R (&)[N]) const {}
};

// plain or programmatic-dependent launch of kernel k
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    if (pdl) return launch_pdl(k, grid, block, s, args...);
    k<<<grid, block, 0, s>>>(((KArgs)args)...);
    return cudaGetLastError();
}

// launch helper: picks the template instance for the handle's variant
template <class T, class Epi>
cudaError_t launch_spmv(int kind, int group, const MatView<T> &A, const T *x, const Epi &epi,
                        RedScratch red, int grid, cudaStream_t s, bool pdl = false) {
    if constexpr (std::is_same<T, double2>::value) {
        if (kind == HZ_SPMV_FLAT64) {
            launch_k(pdl, k_spmv_d64b<Epi, false>, grid, kFlatThreads, s, A, x, epi, red);
            return cudaGetLastError();
        }
        if (kind == HZ_SPMV_FLAT64P) {
            launch_k(pdl, k_spmv_d64b<Epi, true>, grid, kFlatThreads, s, A, x, epi, red);
            return cudaGetLastError();
        }
    }
    if (kind == HZ_SPMV_SELL) {
        launch_k(pdl, k_spmv<0, T, Epi>, grid, kSpmvBlock, s, A, x, epi, red);
    } else {
        switch (group) {
            case 2: launch_k(pdl, k_spmv<2, T, Epi>, grid, kSpmvBlock, s, A, x, epi, red); break;
            case 4: launch_k(pdl, k_spmv<4, T, Epi>, grid, kSpmvBlock, s, A, x, epi, red); break;
            case 8: launch_k(pdl, k_spmv<8, T, Epi>, grid, kSpmvBlock, s, A, x, epi, red); break;
            case 16: launch_k(pdl, k_spmv<16, T, Epi>, grid, kSpmvBlock, s, A, x, epi, red); break;
            default: launch_k(pdl, k_spmv<32, T, Epi>, grid, kSpmvBlock, s, A, x, epi, red); break;
        }
    }
    return cudaGetLastError();
}

// double-float kernels by handle kind: HZ_SPMV_FF_FLAT (row blocks),
// HZ_SPMV_SELL_FF, or HZ_SPMV_FF (CSR-vector with `group` lanes per row)
template <class Epi>
cudaError_t launch_spmv_ff(int kind, int group, const MatView<double2> &A, const float4 *xff, const Epi &epi,
                           RedScratch red, int grid, cudaStream_t s, bool pdl = false) {
    if (kind == HZ_SPMV_FF_FLAT) {
        launch_k(pdl, k_spmv_ffb<Epi>, grid, kFlatThreads, s, A, xff, epi, red);
        return cudaGetLastError();
    }
    if (kind == HZ_SPMV_FF_TMA) {
        static bool carveout = false;   // ask for the largest shared-memory carveout once
        if (!carveout) {
            cudaFuncSetAttribute(k_spmv_fft<Epi>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
            carveout = true;
        }
        launch_k(pdl, k_spmv_fft<Epi>, grid, kFlatThreads, s, A, xff, epi, red);
        return cudaGetLastError();
    }
    if (kind == HZ_SPMV_SELL_FF) {
        launch_k(pdl, k_spmv_ff<0, Epi>, grid, kSpmvBlock, s, A, xff, epi, red);
        return cudaGetLastError();
    }
    switch (group) {
        case 2: launch_k(pdl, k_spmv_ff<2, Epi>, grid, kSpmvBlock, s, A, xff, epi, red); break;
        case 4: launch_k(pdl, k_spmv_ff<4, Epi>, grid, kSpmvBlock, s, A, xff, epi, red); break;
        case 8: launch_k(pdl, k_spmv_ff<8, Epi>, grid, kSpmvBlock, s, A, xff, epi, red); break;
        case 16: launch_k(pdl, k_spmv_ff<16, Epi>, grid, kSpmvBlock, s, A, xff, epi, red); break;
        default: launch_k(pdl, k_spmv_ff<32, Epi>, grid, kSpmvBlock, s, A, xff, epi, red); break;
    }
    return cudaGetLastError();
}

// grid for a fused SpMV: enough blocks to cover the rows once, capped at a
// whole number of waves over the SMs (the row loop is grid-stride); the
// block-flat kinds get exactly the CTAs that fit at once.
int spmv_grid(const hz_mat *A, int kind, int group, int blocks_per_sm_cap = 8);

// the binary64 (and complex64) kernel family that stands for a handle's
// kind when a solver runs in binary64: the SELL kinds -> HZ_SPMV_SELL, the
// CSR-vector kinds -> HZ_SPMV_CSR_VECTOR, HZ_SPMV_FLAT64 -> itself, the other
// block-flat kinds -> HZ_SPMV_FLAT64P where the handle has its packed stream
// (else HZ_SPMV_FLAT64; the row blocks exist for every handle)
inline int d64_kind(const hz_mat *A, int kind) {
    if (kind == HZ_SPMV_SELL || kind == HZ_SPMV_SELL_FF) return HZ_SPMV_SELL;
    if (kind == HZ_SPMV_CSR_VECTOR || kind == HZ_SPMV_FF) return HZ_SPMV_CSR_VECTOR;
    if (kind == HZ_SPMV_FLAT64) return HZ_SPMV_FLAT64;
    return A->pk_re ? HZ_SPMV_FLAT64P : HZ_SPMV_FLAT64;
}
// the binary64 block-flat kinds
inline bool is_flat64(int kind) { return kind == HZ_SPMV_FLAT64 || kind == HZ_SPMV_FLAT64P; }

template <class T>
MatView<T> mat_view(const hz_mat *A);

}  // namespace hz
