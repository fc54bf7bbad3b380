// Krylov kernel templates shared by the FP64 and FP32 translation units.
//
// Krylov solvers started from the subspace guess (the solve of Algorithm 1; the
// paper uses GMRES for general matrices and names CG for SPD ones, Section 1).
//
// Restarted GMRES(R) with CGS2 Arnoldi.  One Arnoldi step j is four
// streaming kernels over the n rows:
//   K5a w = A v_j                 software-pipelined warp-tile CSR product
//   K5b h1 = V_j^T w              column-segment dots over all warps
//   K7a w -= V_j h1, h2 = V_j^T w fused: each basis element is read once
//   K7b w -= V_j h2, v_{j+1} = w (unnormalised), ||w||^2; the last block then
//       forms the Hessenberg column h1 + h2, applies the Givens rotations,
//       updates the residual estimate and decides whether the cycle ends.
// Reductions end in a deterministic last-block pass.  On this GPU a
// warp-wide FP64 instruction occupies a sub-partition's FP64 unit for many
// cycles, so the CGS kernels are specialised on the exact number of basis
// columns and issue exactly the algorithmic count of FP64 operations.
// Basis columns are stored unnormalised with sigma_k = 1/||.|| kept on the
// device, so no extra pass rescales them.  A cycle (R steps, the basis update
// x += V y and the true residual of the new iterate) is captured once as a
// CUDA graph; kernels after the end of a cycle return at once.
//
// The same templates run the FP32 inner solve of mixed precision (system
// A32 d = rhs32 from d = 0, FP32 vectors and FP32 dot accumulation; the
// Hessenberg and rotations stay FP64).
#pragma once

#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace sa {

enum { ST_OK = 0, ST_NOT_CONVERGED = 1, ST_BREAKDOWN = -4, ST_NONFINITE = -5 };
enum { CNT_START = 0, CNT_DOT = 1, CNT_PASS2 = 2, CNT_PASS3 = 3, CNT_RES = 4, CNT_REFINE = 5 };

struct SysF64 {
    using T = double;
    using V = double;
    __device__ static const double* val(const DevArgs* a) { return a->val64; }
    __device__ static const double* rhs(const DevArgs* a) { return a->b; }
    __device__ static double* x(const DevArgs* a) { return a->x; }
};
struct SysF32 {
    using T = float;
    using V = float;
    __device__ static const float* val(const DevArgs* a) { return a->val32; }
    __device__ static const float* rhs(const DevArgs* a) { return a->rhs32; }
    __device__ static float* x(const DevArgs* a) { return reinterpret_cast<float*>(a->d); }
};

constexpr int kWarps = kStreamBlock / 32;
constexpr int kTile = kTileStage;              // pipelined tiles: (value, x) staging
constexpr int kTileP = kTileChunks * 32;       // single-stage tiles: product staging

// ---------------------------------------------------------------------------
// Cycle start: r = rhs - A x written to basis column 0, beta = ||r||.  With
// first != 0 the solve is initialised (||rhs||, target, iteration count; the
// FP32 inner solve also zeroes d, so r = rhs).
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock, 1)
gmres_start_kernel(const DevArgs* __restrict__ a, KState* ks, typename Sys::T* V,
                   typename Sys::T* partial, int first) {
    using T = typename Sys::T;
    if (!first && ks->finished) return;
    __shared__ T sprod[kWarps * kTileP];
    __shared__ T scratch[kWarps * 2];
    __shared__ T red[2];
    const int n = a->n, nnz = a->nnz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T* x = Sys::x(a);
    const T* rhs = Sys::rhs(a);
    const bool zero_x = first && (sizeof(T) == 4);
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    T acc[2] = {0, 0};
    for (int r0 = lo + warp * 32; r0 < hi; r0 += kWarps * 32) {
        T ax = 0;
        if (!zero_x)
            ax = warp_tile_spmv<T>(a->rowptr, a->colind, Sys::val(a), x, n, nnz, r0,
                                   sprod + warp * kTileP, &ks->bad_index);
        const int row = r0 + lane;
        if (row < n) {
            const T bi = rhs[row];
            const T r = bi - ax;
            V[row] = r;
            if (zero_x) x[row] = 0;
            acc[0] += r * r;
            acc[1] += bi * bi;
        }
    }
    block_sum<T, 2>(acc, 2, red, scratch);
    if (threadIdx.x < 2) partial[blockIdx.x * 2 + threadIdx.x] = red[threadIdx.x];
    if (last_block_arrive(&ks->counter[CNT_START])) {
        __shared__ double tot[2];
        reduce_blocks(partial, gridDim.x, 2, 2, tot);
        if (threadIdx.x == 0) {
            const double beta = sqrt(tot[0]);
            if (first) {
                ks->bnorm = sqrt(tot[1]);
                ks->target = a->tol * ks->bnorm;
                ks->iters = 0;
                ks->status = ST_OK;
                ks->first_relres = rel_residual(beta, ks->bnorm);
            }
            ks->last_jdone = first ? 0 : ks->jdone;
            ks->beta = beta;
            ks->g[0] = beta;
            ks->sigma[0] = beta > 0.0 ? 1.0 / beta : 0.0;
            ks->jdone = 0;
            ks->cycle_over = 0;
            ks->finished = 0;
            if (!isfinite(beta)) {
                ks->status = ST_NONFINITE;
                ks->finished = 1;
            } else if (beta <= ks->target) {
                ks->status = ST_OK;
                ks->finished = 1;
            } else if (ks->iters >= a->max_iters) {
                ks->status = ST_NOT_CONVERGED;
                ks->finished = 1;
            }
            if (ks->finished) ks->cycle_over = 1;
            ks->counter[CNT_START] = 0;
        }
    }
}

// Lane l of every warp holds, for K <= 32, the warp partial of column l % K
// after warp_reduce_scatter; the block partial of column k (k < nk) is the
// sum over warps in warp order.  32 < K <= 64 is handled as two halves of 32,
// the upper one padded with zeros past column K - 1.
template <typename T, int K>
__device__ __forceinline__ void block_columns(T (&part)[K], int nk, T* wsum /* kWarps * K */,
                                              T* out /* global, K */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (K <= 32 && (K & (K - 1)) == 0) {
        const T c = warp_reduce_scatter<T, K>(part);
        if (lane < K) wsum[warp * K + lane] = c;
    } else if constexpr (K < 32) {
        constexpr int P = K <= 8 ? 8 : (K <= 16 ? 16 : 32);   // next power of two
        T v[P];
#pragma unroll
        for (int i = 0; i < P; ++i) v[i] = i < K ? part[i] : (T)0;
        const T c = warp_reduce_scatter<T, P>(v);
        if (lane < K) wsum[warp * K + lane] = c;
    } else {
        static_assert(K <= 64, "at most 64 columns");
        T lo[32], hi[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            lo[i] = part[i];
            hi[i] = 32 + i < K ? part[32 + i] : (T)0;
        }
        const T cl = warp_reduce_scatter<T, 32>(lo);
        const T ch = warp_reduce_scatter<T, 32>(hi);
        wsum[warp * K + lane] = cl;
        if (32 + lane < K) wsum[warp * K + 32 + lane] = ch;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        T s = wsum[k];
        for (int w = 1; w < kWarps; ++w) s += wsum[w * K + k];
        out[k] = s;
    }
}

// ---------------------------------------------------------------------------
// K5a: w = sigma_j A vstored_j.  Software-pipelined warp tiles (the row range
// of tile k+2, the CSR loads of tile k+1 and the gathers of tile k in flight
// together), no reduction, so the block can be large.
constexpr int kSpmvBlock = 768;
constexpr int kSpmvWarps = kSpmvBlock / 32;

// SELL-32 product: warp per 32-row slice (lane = row), the slice's entries
// stored column-major and padded to its widest row (padding has column -1).
// G slices per warp and iteration (3 in FP32, 2 in FP64): the slice offsets
// (or, when every slice has the same width, offsets computed from the slice
// index, with no load), then all index and value loads of the G slices and
// the epilogue's own row operands (issued before the gathers, so they are in
// flight together), then all gathers, then each row is summed in CSR order
// with exactly one fused multiply-add per stored entry (the FMA chain is
// unrolled for the slice's exact width, so padding costs no arithmetic).
// Slices wider than kSellW use a plain loop.
constexpr int kSellW = 5;

template <typename T, int W>
__device__ __forceinline__ T sell_dot(const T (&v)[kSellW], const T (&xv)[kSellW]) {
    T a = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) a = fma(v[k], xv[k], a);
    return a;
}

template <typename T>
__device__ __forceinline__ T sell_dot_w(int w, const T (&v)[kSellW], const T (&xv)[kSellW]) {
    switch (w) {
        case 1: return sell_dot<T, 1>(v, xv);
        case 2: return sell_dot<T, 2>(v, xv);
        case 3: return sell_dot<T, 3>(v, xv);
        case 4: return sell_dot<T, 4>(v, xv);
        case 5: return sell_dot<T, 5>(v, xv);
        default: return (T)0;
    }
}

// x2 != NULL: the gathered operand is x[c] * x2[c].
template <typename T>
__device__ __forceinline__ T sell_row_loop(const int* __restrict__ col, const T* __restrict__ val,
                                           const T* __restrict__ x, const T* __restrict__ x2,
                                           int n, int o, int w, int& flag) {
    const int lane = threadIdx.x & 31;
    T a = 0;
    for (int k = 0; k < w; ++k) {
        const int c = __ldg(col + o + k * 32 + lane);
        if ((unsigned)c < (unsigned)n) a = fma(__ldg(val + o + k * 32 + lane), x2 ? x[c] * x2[c] : x[c], a);
        else if (c >= 0) flag = 1;
    }
    return a;
}

// Row results of a SELL product go through an epilogue: pre(row) loads the
// row operands the epilogue needs (issued early), epi(row, (A x)_row, pre)
// writes the results; kSlices > 0 overrides the slices per warp and
// iteration (epilogues with many row operands take fewer).  An epilogue with
// a member x2 (and kProd = true) makes the product gather x[c] * x2[c]
// instead of x[c]: A (x .* x2) without forming x .* x2.
struct NoPre {};

template <class E, class = void>
struct GatherProd {
    static constexpr bool value = false;
};
template <class E>
struct GatherProd<E, decltype((void)E::kProd)> {
    static constexpr bool value = E::kProd;
};
template <class E, typename T>
__device__ __forceinline__ const T* gather_x2(const E& e) {
    if constexpr (GatherProd<E>::value) return e.x2;
    else return nullptr;
}

template <typename T>
struct ScaleEpi {
    T* y;
    T scale;
    static constexpr int kSlices = 0;    // slices per warp and iteration: the default
    using Pre = NoPre;
    __device__ Pre pre(int) const { return {}; }
    __device__ void operator()(int r, T ax, const Pre&) const { y[r] = ax * scale; }
};

template <typename T, typename Epi>
__device__ __forceinline__ void sell_rows(const int* __restrict__ off,
                                          const int* __restrict__ col,
                                          const T* __restrict__ val,
                                          const T* __restrict__ x, int n, int lo, int hi,
                                          int nwarps, int ellw, int keep, int* bad,
                                          const Epi& epi) {
    // An empty range (a trailing block when the grid covers more than n rows)
    // has no slice: lo = hi = n would otherwise map to the last partial slice
    // and repeat rows that another block owns.
    if (lo >= hi) return;
    constexpr int G = Epi::kSlices > 0 ? Epi::kSlices : (sizeof(T) == 4 ? 3 : 2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s_lo = lo >> 5, s_hi = (hi + 31) >> 5;
    const uint64_t pol = l2_policy(keep != 0);
    int flag = 0;
    for (int s0 = s_lo + warp; s0 < s_hi; s0 += G * nwarps) {
        int o[G], w[G], r[G];
        bool row_ok[G];
        typename Epi::Pre pre[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int sl = s0 + g * nwarps;
            const bool live = sl < s_hi;
            r[g] = sl * 32 + lane;
            row_ok[g] = live && r[g] < hi;
            if (ellw > 0) {
                o[g] = live ? sl * 32 * ellw : 0;
                w[g] = live ? ellw : 0;
            } else {
                o[g] = live ? __ldg(off + sl) : 0;
                w[g] = live ? (__ldg(off + sl + 1) - o[g]) >> 5 : 0;
            }
        }
        bool fast = true;
#pragma unroll
        for (int g = 0; g < G; ++g) fast = fast && w[g] <= kSellW;
        T ax[G];
        if (fast) {
            int c[G][kSellW];
            T v[G][kSellW], xv[G][kSellW];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int k = 0; k < kSellW; ++k)
                    c[g][k] = k < w[g] ? ld_hint(col + o[g] + k * 32 + lane, pol) : -1;
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int k = 0; k < kSellW; ++k)
                    v[g][k] = k < w[g] ? ld_hint(val + o[g] + k * 32 + lane, pol) : (T)0;
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (row_ok[g]) pre[g] = epi.pre(r[g]);
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int k = 0; k < kSellW; ++k) {
                    xv[g][k] = (unsigned)c[g][k] < (unsigned)n ? x[c[g][k]] : (T)0;
                    if constexpr (GatherProd<Epi>::value)
                        xv[g][k] *= (unsigned)c[g][k] < (unsigned)n ? epi.x2[c[g][k]] : (T)0;
                    if (c[g][k] >= n) flag = 1;
                }
#pragma unroll
            for (int g = 0; g < G; ++g) ax[g] = sell_dot_w<T>(w[g], v[g], xv[g]);
        } else {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (row_ok[g]) pre[g] = epi.pre(r[g]);
                ax[g] = w[g] > 0 ? sell_row_loop<T>(col, val, x, gather_x2<Epi, T>(epi), n, o[g],
                                                    w[g], flag)
                                 : (T)0;
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (row_ok[g]) epi(r[g], ax[g], pre[g]);
    }
    if (flag) atomicOr(bad, 1);
}

template <typename T>
__device__ __forceinline__ void sell_spmv_rows(const int* __restrict__ off,
                                               const int* __restrict__ col,
                                               const T* __restrict__ val,
                                               const T* __restrict__ x, int n, int lo, int hi,
                                               T scale, T* __restrict__ y, int nwarps, int ellw,
                                               int keep, int* bad) {
    sell_rows<T>(off, col, val, x, n, lo, hi, nwarps, ellw, keep, bad, ScaleEpi<T>{y, scale});
}

template <class Sys>
__global__ void __launch_bounds__(kSpmvBlock, 1)
arnoldi_spmv_kernel(const DevArgs* __restrict__ a, const KState* __restrict__ ks,
                    const typename Sys::T* __restrict__ V, size_t ldv,
                    typename Sys::T* __restrict__ w, int j, const typename Sys::T* src) {
    using T = typename Sys::T;
    if (ks->cycle_over) return;
    extern __shared__ unsigned char dsm[];
    T* sprod = reinterpret_cast<T*>(dsm);                   // kSpmvWarps * kTile
    const int n = a->n, nnz = a->nnz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // w = A v_j, v_j = sigma_j times the stored column, or (right
    // preconditioning) w = A z with z = M^{-1} v_j already formed in src.
    const T sig = src ? (T)1 : (T)ks->sigma[j];
    const T* vj = src ? src : V + (size_t)j * ldv;
    const T* val = Sys::val(a);
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    if (a->sell_off) {
        sell_spmv_rows<T>(a->sell_off, a->sell_col, reinterpret_cast<const T*>(a->sell_val), vj, n,
                          lo, hi, sig, w, kSpmvWarps, a->sell_w, a->sell_keep,
                          const_cast<int*>(&ks->bad_index));
        return;
    }
    const int step = kSpmvWarps * 32;
    int r0 = lo + warp * 32;
    TileRows ta = tile_rows(a->rowptr, n, nnz, r0, hi);
    TileRows tb = tile_rows(a->rowptr, n, nnz, r0 + step, hi);
    TileData<T> da, db;
    tile_span(ta, n, r0);
    tile_load(a->colind, val, ta, da);
    for (; r0 < hi; r0 += step) {
        const TileRows tc = tile_rows(a->rowptr, n, nnz, r0 + 2 * step, hi);
        tile_span(tb, n, r0 + step);
        if (r0 + step < hi) tile_load(a->colind, val, tb, db);
        const T ax = tile_finish<T>(a->colind, val, vj, n, ta, da, sprod + warp * kTile,
                                    const_cast<int*>(&ks->bad_index));
        const int row = r0 + lane;
        if (row < hi) w[row] = ax * sig;
        ta = tb;
        da = db;
        tb = tc;
    }
}

// K5b: h1 = sigma_k (V_stored^T w)_k for k <= j.  Work items (column k, row
// segment g) spread over all warps (nseg segments per column so that small
// bases still use every warp); each lane keeps eight accumulators, combined
// in a fixed order, then the warp butterfly; segments are summed in segment
// order.  With more columns than warps the row-parallel K5b' below takes
// over.  Here and in K5b', K7a and K7b the basis columns are read with
// streaming loads (evict-first in L2), which keeps the matrix in L2 for the
// product of the next Arnoldi step.
constexpr int kDotBlock = 768;
constexpr int kDotWarps = kDotBlock / 32;
constexpr int kDotRowsMin = kDotWarps + 1;   // first nk taken by K5b' (measured: slower below)

template <class Sys>
__global__ void __launch_bounds__(kDotBlock, 1)
arnoldi_dot_kernel(const DevArgs* __restrict__ a, KState* ks,
                   const typename Sys::T* __restrict__ V, size_t ldv,
                   const typename Sys::T* __restrict__ w, typename Sys::T* partial, int j,
                   int stride) {
    using T = typename Sys::T;
    if (ks->cycle_over) return;
    __shared__ T segsum[kMaxBasis * kDotWarps];
    __shared__ T colsum[kMaxBasis];
    const int n = a->n, nk = j + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    const int nseg = max(1, kDotWarps / nk);
    const int seglen = (((hi - lo) + nseg - 1) / nseg + 31) & ~31;
    for (int item = warp; item < nk * nseg; item += kDotWarps) {
        const int k = item / nseg, g = item - k * nseg;
        const int s0 = lo + g * seglen, s1 = min(hi, s0 + seglen);
        const T* vk = V + (size_t)k * ldv;
        T acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = 0;
        int i = s0 + lane;
        for (; i + 7 * 32 < s1; i += 8 * 32) {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = fma(__ldcs(vk + i + u * 32), w[i + u * 32], acc[u]);
        }
        for (; i < s1; i += 32) acc[0] = fma(__ldcs(vk + i), w[i], acc[0]);
        const T t = warp_sum(((acc[0] + acc[1]) + (acc[2] + acc[3])) +
                             ((acc[4] + acc[5]) + (acc[6] + acc[7])));
        if (lane == 0) segsum[k * kDotWarps + g] = t;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        T t = segsum[k * kDotWarps];
        for (int g = 1; g < nseg; ++g) t += segsum[k * kDotWarps + g];
        colsum[k] = t;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nk; k += blockDim.x) partial[(size_t)blockIdx.x * stride + k] = colsum[k];
    if (last_block_arrive(&ks->counter[CNT_DOT])) {
        __shared__ double tot[kMaxBasis];
        reduce_blocks(partial, gridDim.x, stride, nk, tot);
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            const double hk = ks->sigma[k] * tot[k];
            ks->h1[k] = hk;
            ks->c1[k] = ks->sigma[k] * hk;
        }
        if (threadIdx.x == 0) ks->counter[CNT_DOT] = 0;
    }
}

// K7a: w -= V_stored c1; h2 = sigma_k (V_stored^T w)_k.  NK (the number of
// basis columns) is a compile-time constant, so the row loop issues exactly
// 2 NK FP64 fused multiply-adds per row and no predicated-off ones (on this
// GPU one warp-wide FP64 instruction occupies a sub-partition's FP64 unit for
// many cycles, so the instruction count, not latency, bounds the kernel).
// ROWS rows per thread and iteration keep >= 16 loads in flight; the dot
// partials accumulate per thread and are reduce-scattered over the warp once.
template <class Sys, int NK>
__global__ void __launch_bounds__(kStreamBlock, 1)
arnoldi_pass2_kernel(const DevArgs* __restrict__ a, KState* ks,
                     const typename Sys::T* __restrict__ V, size_t ldv,
                     typename Sys::T* __restrict__ w, typename Sys::T* partial, int j) {
    using T = typename Sys::T;
    if (ks->cycle_over) return;
    __shared__ T cf[NK];
    __shared__ T wsum[kWarps * NK];
    const int n = a->n;
    const int nk = NK;
    for (int k = threadIdx.x; k < NK; k += blockDim.x) cf[k] = (T)ks->c1[k];
    __syncthreads();
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    T part[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) part[k] = 0;
    constexpr int ROWS = NK >= 16 ? 1 : (16 + NK - 1) / NK;
    const int bd = blockDim.x;
    for (int i0 = lo + threadIdx.x; i0 < hi; i0 += ROWS * bd) {
        T vv[ROWS][NK];
        T r[ROWS];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const int i = min(i0 + u * bd, hi - 1);
#pragma unroll
            for (int k = 0; k < NK; ++k) vv[u][k] = __ldcs(V + (size_t)k * ldv + i);
            r[u] = w[i];
        }
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
#pragma unroll
            for (int k = 0; k < NK; ++k) r[u] = fma(-vv[u][k], cf[k], r[u]);
        }
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const int i = i0 + u * bd;
            if (i < hi) {
                w[i] = r[u];
#pragma unroll
                for (int k = 0; k < NK; ++k) part[k] = fma(vv[u][k], r[u], part[k]);
            }
        }
    }
    block_columns<T, NK>(part, nk, wsum, partial + (size_t)blockIdx.x * kMaxBasis);
    if (last_block_arrive(&ks->counter[CNT_PASS2])) {
        __shared__ double tot[NK];
        reduce_blocks(partial, gridDim.x, kMaxBasis, nk, tot);
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            const double hk = ks->sigma[k] * tot[k];
            ks->h2[k] = hk;
            ks->c2[k] = ks->sigma[k] * hk;
        }
        if (threadIdx.x == 0) ks->counter[CNT_PASS2] = 0;
    }
}

// K5b' (nk > kDotWarps): the same h1 = sigma_k (V_stored^T w)_k, row-parallel
// like K7a: each thread reads a row of all NK columns and w once and keeps NK
// partial sums; the warp reduce-scatter and the block's warps in order, then
// the blocks in order in the last block.  With one column per warp item, K5b
// would leave a warp with a whole extra column after the others finish, and
// on this GPU a warp-wide FP64 add holds a sub-partition's FP64 pipe for tens
// of cycles, so splitting columns into more segments costs as much in
// per-item reductions as it saves.
template <class Sys, int NK>
__global__ void __launch_bounds__(kStreamBlock, 1)
arnoldi_dot_rows_kernel(const DevArgs* __restrict__ a, KState* ks,
                        const typename Sys::T* __restrict__ V, size_t ldv,
                        const typename Sys::T* __restrict__ w, typename Sys::T* partial, int j) {
    using T = typename Sys::T;
    if (ks->cycle_over) return;
    __shared__ T wsum[kWarps * NK];
    const int n = a->n;
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    T part[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) part[k] = 0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        T vv[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) vv[k] = __ldcs(V + (size_t)k * ldv + i);
        const T wi = w[i];
#pragma unroll
        for (int k = 0; k < NK; ++k) part[k] = fma(vv[k], wi, part[k]);
    }
    block_columns<T, NK>(part, NK, wsum, partial + (size_t)blockIdx.x * kMaxBasis);
    if (last_block_arrive(&ks->counter[CNT_DOT])) {
        __shared__ double tot[NK];
        reduce_blocks(partial, gridDim.x, kMaxBasis, NK, tot);
        for (int k = threadIdx.x; k < NK; k += blockDim.x) {
            const double hk = ks->sigma[k] * tot[k];
            ks->h1[k] = hk;
            ks->c1[k] = ks->sigma[k] * hk;
        }
        if (threadIdx.x == 0) ks->counter[CNT_DOT] = 0;
    }
}

// Last block of K7b, all threads: Hessenberg column j = h1 + h2 with
// h_{j+1,j} = ||w||, the previous Givens rotations applied to it, the new
// rotation, the residual estimate |g_{j+1}| and the end-of-cycle decision;
// at the end of a cycle the triangular system R y = g is solved by warp 0
// (column-oriented back substitution from shared memory) and sigma_k y_k
// stored for the basis update.  Everything is staged in shared memory, so
// thread 0's serial part touches no global memory.
template <typename T>
__device__ inline void arnoldi_finish(KState* ks, const DevArgs* a, int j, int R,
                                     const T* __restrict__ partial, int nblk) {
    __shared__ double hc[kMaxBasis + 1];
    __shared__ double cs_s[kMaxRestart], sn_s[kMaxRestart];
    __shared__ double Hs[kMaxBasis * kMaxRestart];
    __shared__ double hn2_s;
    __shared__ int end_cycle, k_s, ok_s;
    const int tid = threadIdx.x, nk = j + 1;
    if (tid < 32) {
        // ||w||^2: the block partials summed by warp 0 in block order (as
        // reduce_blocks does) ...
        T v = 0;
        for (int b = tid; b < nblk; b += 32) v += __ldcg(partial + b);
        v = warp_sum(v);
        if (tid == 0) hn2_s = (double)v;
    } else {
        // ... while the other warps load the new column and the previous
        // rotations (one L2 round trip overlapped with the other).
        const int t = tid - 32, nt = blockDim.x - 32;
        for (int i = t; i < nk; i += nt) hc[i] = ks->h1[i] + ks->h2[i];
        for (int i = t; i < j; i += nt) {
            cs_s[i] = ks->cs[i];
            sn_s[i] = ks->sn[i];
        }
    }
    __syncthreads();
    const double hn2 = hn2_s;
    // The serial part (the previous rotations applied to the new column) is
    // one dependent FP64 chain; everything that does not depend on it runs
    // beside it: ||h||^2 over warp 0 before lane 0 starts the chain, and
    // h_{j+1,j} = ||w|| with its reciprocal in warp 1 (FP64 square roots and
    // divisions are long sequences of FP64 operations on this GPU).
    __shared__ double hh_s, hn_s, hninv_s;
    if (tid < 32) {
        double v = 0.0;
        for (int i = tid; i < nk; i += 32) v += hc[i] * hc[i];
        v = warp_sum(v);
        if (tid == 0) {
            hh_s = v;
            // The rotated entry i + 1 is carried in a register: the chain is
            // one FP64 multiply-add per rotation, no shared-memory round trip.
            double carry = hc[0];
            for (int i = 0; i < j; ++i) {
                const double hi1 = hc[i + 1];
                hc[i] = cs_s[i] * carry + sn_s[i] * hi1;
                carry = -sn_s[i] * carry + cs_s[i] * hi1;
            }
            hc[j] = carry;
        }
    } else if (tid == 32) {
        const double hn = sqrt(hn2);
        hn_s = hn;
        hninv_s = hn > 0.0 ? 1.0 / hn : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        const double hn = hn_s, hh = hh_s;
        hc[j + 1] = hn;
        const double av = hc[j], bv = hn;
        const double rr = hypot(av, bv);
        double c = 1.0, sv = 0.0;
        if (rr != 0.0) {
            const double rinv = 1.0 / rr;
            c = av * rinv;
            sv = bv * rinv;
        }
        ks->cs[j] = c;
        ks->sn[j] = sv;
        hc[j] = rr;
        hc[j + 1] = 0.0;
        const double gj = ks->g[j];
        const double gj1 = -sv * gj;
        ks->g[j + 1] = gj1;
        ks->g[j] = c * gj;
        ks->iters += 1;
        ks->sigma[j + 1] = hninv_s;
        const bool nonfinite = !isfinite(hn) || !isfinite(gj1);
        // Breakdown: ||w|| <= 1e-14 ||(h, ||w||)||, compared in squares.
        const bool happy = hn * hn <= 1e-28 * (hh + hn * hn);
        const bool conv = fabs(gj1) <= ks->target;
        const int e = nonfinite || happy || conv || ks->iters >= a->max_iters || j == R - 1;
        end_cycle = e;
        k_s = j + 1;
        ok_s = 1;
        if (e) {
            ks->cycle_over = 1;
            ks->jdone = j + 1;
            if (nonfinite) {
                ks->status = ST_NONFINITE;
                ks->finished = 1;
                ok_s = 0;
            }
        }
    }
    __syncthreads();
    double* Hcol = ks->H + (size_t)j * kMaxBasis;
    for (int i = tid; i <= j + 1; i += blockDim.x) Hcol[i] = hc[i];
    if (!end_cycle) return;
    const int k = k_s;
    for (int i = tid; i < kMaxBasis; i += blockDim.x) ks->cy[i] = 0.0;
    if (!ok_s) return;
    // Upper triangle of H (columns 0..k-1; column j is the one just formed).
    for (int idx = tid; idx < k * k; idx += blockDim.x) {
        const int col = idx / k, row = idx - col * k;
        Hs[col * kMaxBasis + row] = (col == j) ? hc[row] : ks->H[(size_t)col * kMaxBasis + row];
    }
    __syncthreads();
    if (tid < 32) {
        const int lane = tid;
        bool sing = false;
        for (int i = lane; i < k; i += 32) sing |= (Hs[i * kMaxBasis + i] == 0.0);
        sing = __any_sync(0xffffffffu, sing);
        if (sing) {
            if (lane == 0) {
                ks->status = ST_BREAKDOWN;
                ks->finished = 1;
            }
            return;
        }
        // Lane l owns rows l and l + 32; acc starts at g and loses H[row][i] y_i.
        // The diagonal's reciprocals are formed lane-parallel first, so the
        // dependent chain holds a multiplication per row, not a division.
        __shared__ double rdiag[kMaxRestart + 1];
        for (int i = lane; i < k; i += 32) rdiag[i] = 1.0 / Hs[i * kMaxBasis + i];
        __syncwarp();
        double acc0 = lane < k ? ks->g[lane] : 0.0;
        double acc1 = lane + 32 < k ? ks->g[lane + 32] : 0.0;
        double y0 = 0.0, y1 = 0.0;
        for (int i = k - 1; i >= 0; --i) {
            const double own = (i < 32) ? acc0 : acc1;
            double yi = __shfl_sync(0xffffffffu, own, i & 31) * rdiag[i];
            if (lane == (i & 31)) {
                if (i < 32) y0 = yi; else y1 = yi;
            }
            if (lane < i) acc0 -= Hs[i * kMaxBasis + lane] * yi;
            if (lane + 32 < i) acc1 -= Hs[i * kMaxBasis + lane + 32] * yi;
        }
        if (lane < k) ks->cy[lane] = ks->sigma[lane] * y0;
        if (lane + 32 < k) ks->cy[lane + 32] = ks->sigma[lane + 32] * y1;
    }
}

// K7b: w -= V_stored c2, stored as basis column j+1; ||w||^2; then K8.
// NK is a compile-time constant: all column loads of two rows per thread are
// issued before the nk + 1 FP64 fused multiply-adds per row (measured faster
// than four or eight rows per thread for nk >= 2; four rows spilled registers
// at nk = 18..23).
template <class Sys, int NK>
__global__ void __launch_bounds__(kStreamBlock, 1)
arnoldi_pass3_kernel(const DevArgs* __restrict__ a, KState* ks, typename Sys::T* __restrict__ V,
                     size_t ldv, const typename Sys::T* __restrict__ w, typename Sys::T* partial,
                     int j, int R) {
    using T = typename Sys::T;
    if (ks->cycle_over) return;
    __shared__ T cf[NK];
    __shared__ T scratch[kWarps];
    __shared__ T red[1];
    const int n = a->n;
    for (int k = threadIdx.x; k < NK; k += blockDim.x) cf[k] = (T)ks->c2[k];
    __syncthreads();
    T* vout = V + (size_t)(j + 1) * ldv;
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    T part[1] = {0};
    const int bd = blockDim.x;
    constexpr int ROWS = 2;
    for (int i0 = lo + threadIdx.x; i0 < hi; i0 += ROWS * bd) {
        T vv[ROWS][NK];
        T r[ROWS];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const int i = min(i0 + u * bd, hi - 1);
#pragma unroll
            for (int k = 0; k < NK; ++k) vv[u][k] = __ldcs(V + (size_t)k * ldv + i);
            r[u] = w[i];
        }
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
#pragma unroll
            for (int k = 0; k < NK; ++k) r[u] = fma(-vv[u][k], cf[k], r[u]);
            const int i = i0 + u * bd;
            if (i < hi) {
                vout[i] = r[u];
                part[0] = fma(r[u], r[u], part[0]);
            }
        }
    }
    block_sum<T, 1>(part, 1, red, scratch);
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
    if (last_block_arrive(&ks->counter[CNT_PASS3])) {
        if (threadIdx.x == 0) ks->counter[CNT_PASS3] = 0;
        arnoldi_finish(ks, a, j, R, partial, (int)gridDim.x);
    }
}

// x += V_stored cy (the GMRES correction of the finished cycle).
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock, 1)
gmres_update_kernel(const DevArgs* __restrict__ a, const KState* ks,
                    const typename Sys::T* __restrict__ V, size_t ldv) {
    using T = typename Sys::T;
    if (ks->status != ST_OK && ks->status != ST_NOT_CONVERGED) return;
    if (ks->finished) return;
    __shared__ T cy[kMaxBasis];
    __shared__ int kk;
    if (threadIdx.x == 0) kk = ks->jdone;
    for (int k = threadIdx.x; k < kMaxBasis; k += blockDim.x) cy[k] = (T)ks->cy[k];
    __syncthreads();
    const int k = kk, n = a->n;
    T* x = Sys::x(a);
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        // Eight independent column loads in flight per thread (streaming
        // loads); the multiply-adds keep the column order.
        T acc = 0;
        int l = 0;
        for (; l + 8 <= k; l += 8) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcs(V + (size_t)(l + u) * ldv + i);
#pragma unroll
            for (int u = 0; u < 8; ++u) acc = fma(v[u], cy[l + u], acc);
        }
        for (; l < k; ++l) acc = fma(__ldcs(V + (size_t)l * ldv + i), cy[l], acc);
        x[i] += acc;
    }
}

#include "precond_kernels.cuh"

template <class Sys>
static void launch_start(const DevArgs* a, KState* ks, typename Sys::T* V, typename Sys::T* partial,
                         int nblk, int first, cudaStream_t st) {
    gmres_start_kernel<Sys><<<nblk, kStreamBlock, 0, st>>>(a, ks, V, partial, first);
}

template <class Sys>
static size_t spmv_smem() {
    using T = typename Sys::T;
    const size_t bytes = sizeof(T) * (size_t)kSpmvWarps * kTile;
    // The attribute is per device: set it on every call (cheap, host only).
    cudaFuncSetAttribute(arnoldi_spmv_kernel<Sys>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bytes);
    return bytes;
}

#include "krylov_f32_kernels.cuh"

// Records ev[*k] (when timing events are supplied) and advances *k.
inline void mark(cudaEvent_t* ev, int* k, cudaStream_t st) {
    if (ev) cudaEventRecordWithFlags(ev[(*k)++], st, cudaEventRecordExternal);
}

template <class Sys>
static const typename Sys::T* launch_precond(const DevArgs* a, KState* ks,
                                             const PrecondArgs<typename Sys::T>& pc,
                                             const typename Sys::T* u, int sig_idx, int phase,
                                             int nblk, cudaStream_t st, cudaEvent_t* ev, int* k) {
    using T = typename Sys::T;
    if (pc.sweeps == 1) {
        precond_scale_kernel<Sys><<<nblk, kStreamBlock, 0, st>>>(a, ks, u, sig_idx, pc.dinv,
                                                                 pc.omega, pc.za, phase, pc.cheb,
                                                                 pc.tab, pc.dvec);
        mark(ev, k, st);
        return pc.za;
    }
    // Sweep 1 forms z_1 from u itself (no scale kernel), then sweeps 2 .. d-1.
    T* cur = pc.za;
    T* nxt = pc.zb;
    for (int sw = 1; sw < pc.sweeps; ++sw) {
        const int last = sw == pc.sweeps - 1;
        const T* zin = sw == 1 ? u : cur;
        T* zout = sw == 1 ? cur : nxt;
        if (pc.cheb && sw == 1)
            precond_sweep_kernel<Sys, 1, 1><<<nblk, kSpmvBlock, 0, st>>>(
                a, ks, u, sig_idx, pc.dinv, pc.omega, zin, zout, phase, sw, pc.tab, pc.dvec, last);
        else if (pc.cheb)
            precond_sweep_kernel<Sys, 1, 0><<<nblk, kSpmvBlock, 0, st>>>(
                a, ks, u, sig_idx, pc.dinv, pc.omega, zin, zout, phase, sw, pc.tab, pc.dvec, last);
        else if (sw == 1)
            precond_sweep_kernel<Sys, 0, 1><<<nblk, kSpmvBlock, 0, st>>>(
                a, ks, u, sig_idx, pc.dinv, pc.omega, zin, zout, phase, sw, pc.tab, pc.dvec, last);
        else
            precond_sweep_kernel<Sys, 0, 0><<<nblk, kSpmvBlock, 0, st>>>(
                a, ks, u, sig_idx, pc.dinv, pc.omega, zin, zout, phase, sw, pc.tab, pc.dvec, last);
        if (last) mark(ev, k, st);     // one event pair around the application's sweeps
        if (sw > 1) {
            T* tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
    }
    return cur;
}

template <class Sys, int NK>
static void launch_step(const DevArgs* a, KState* ks, typename Sys::T* V, size_t ldv,
                        typename Sys::T* w, typename Sys::T* partial, int nblk, int j, int R,
                        cudaStream_t st, cudaEvent_t* ev, int* k,
                        const PrecondArgs<typename Sys::T>& pc) {
    const typename Sys::T* src = nullptr;
    if (pc.sweeps > 0)
        src = launch_precond<Sys>(a, ks, pc, V + (size_t)j * ldv, j, 0, nblk, st, ev, k);
    if constexpr (sizeof(typename Sys::T) == 4) {
        f32_spmv_dot_kernel<NK><<<nblk, kStreamBlock, 0, st>>>(a, ks, V, ldv, w, partial, j, src);
        mark(ev, k, st);
        f32_pass2_kernel<NK><<<nblk, kStreamBlock, 0, st>>>(a, ks, V, ldv, w, partial, j);
        mark(ev, k, st);
        f32_pass3_kernel<NK><<<nblk, kStreamBlock, 0, st>>>(a, ks, V, ldv, w, partial, j, R);
        mark(ev, k, st);
    } else {
        arnoldi_spmv_kernel<Sys><<<nblk, kSpmvBlock, spmv_smem<Sys>(), st>>>(a, ks, V, ldv, w, j, src);
        mark(ev, k, st);
        if constexpr (NK >= kDotRowsMin)
            arnoldi_dot_rows_kernel<Sys, NK><<<nblk, kStreamBlock, 0, st>>>(a, ks, V, ldv, w, partial, j);
        else
            arnoldi_dot_kernel<Sys><<<nblk, kDotBlock, 0, st>>>(a, ks, V, ldv, w, partial, j, kMaxBasis);
        mark(ev, k, st);
        arnoldi_pass2_kernel<Sys, NK><<<nblk, kStreamBlock, 0, st>>>(a, ks, V, ldv, w, partial, j);
        mark(ev, k, st);
        arnoldi_pass3_kernel<Sys, NK><<<nblk, kStreamBlock, 0, st>>>(a, ks, V, ldv, w, partial, j, R);
        mark(ev, k, st);
    }
}

template <class Sys, int NK>
struct StepTable {
    static void launch(int nk, const DevArgs* a, KState* ks, typename Sys::T* V, size_t ldv,
                       typename Sys::T* w, typename Sys::T* partial, int nblk, int j, int R,
                       cudaStream_t st, cudaEvent_t* ev, int* k,
                       const PrecondArgs<typename Sys::T>& pc) {
        if (nk == NK)
            launch_step<Sys, NK>(a, ks, V, ldv, w, partial, nblk, j, R, st, ev, k, pc);
        else
            StepTable<Sys, NK + 1>::launch(nk, a, ks, V, ldv, w, partial, nblk, j, R, st, ev, k, pc);
    }
};
template <class Sys>
struct StepTable<Sys, kMaxRestart + 1> {
    static void launch(int, const DevArgs*, KState*, typename Sys::T*, size_t, typename Sys::T*,
                       typename Sys::T*, int, int, int, cudaStream_t, cudaEvent_t*, int*,
                       const PrecondArgs<typename Sys::T>&) {}
};

// One restart cycle.  With `ev` (cycle_marks + 1 timing events) an event is
// recorded before the first kernel and after every kernel, except that a
// preconditioner application's consecutive sweeps share one pair of events:
// with S = step_kernels + (1 with a preconditioner) marks per Arnoldi step j,
// S j is the preconditioner, then SpMV, first-pass dots, pass 2, pass 3
// (FP32: SpMV with the dots, pass 2, pass 3); from S R the update (one
// kernel, or combine + preconditioner + axpy), then the restart residual.
template <class Sys>
static void launch_cycle(const DevArgs* a, KState* ks, typename Sys::T* V, size_t ldv,
                         typename Sys::T* w, typename Sys::T* partial, int nblk, int R,
                         cudaStream_t st, int* launches, cudaEvent_t* ev,
                         const PrecondArgs<typename Sys::T>& pc) {
    int k = 0;
    mark(ev, &k, st);
    for (int j = 0; j < R; ++j)
        StepTable<Sys, 1>::launch(j + 1, a, ks, V, ldv, w, partial, nblk, j, R, st, ev, &k, pc);
    if (pc.sweeps > 0) {
        gmres_combine_kernel<Sys><<<nblk, kStreamBlock, 0, st>>>(a, ks, V, ldv, pc.t);
        mark(ev, &k, st);
        const typename Sys::T* z = launch_precond<Sys>(a, ks, pc, pc.t, -1, 1, nblk, st, ev, &k);
        gmres_axpy_kernel<Sys><<<nblk, kStreamBlock, 0, st>>>(a, ks, z);
        mark(ev, &k, st);
    } else {
        gmres_update_kernel<Sys><<<nblk, kStreamBlock, 0, st>>>(a, ks, V, ldv);
        mark(ev, &k, st);
    }
    gmres_start_kernel<Sys><<<nblk, kStreamBlock, 0, st>>>(a, ks, V, partial, 0);
    mark(ev, &k, st);
    if (launches) *launches = cycle_kernels(R, pc.sweeps, sizeof(typename Sys::T) == 4);
}

}  // namespace sa
