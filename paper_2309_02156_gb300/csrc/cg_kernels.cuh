// Grid-wide conjugate gradients (Hestenes-Stiefel) for large SPD systems:
// every SM works on the iteration, three streaming kernels per iteration
// (product with the direction and p^T A p; the x / r update and r^T r; the new
// direction), captured as a CUDA graph of several iterations.  Scalars live
// in the solve's KState (FP64); reductions end in the deterministic
// last-block pass.  The conventions are the single-block CG's: an iteration
// is one product; when the recursive residual passes the test the true
// residual b - A x is formed (on the host's request, between graph launches)
// and the solve either ends or restarts from it, the count continuing;
// p^T A p <= 0 is a breakdown.  Included by krylov.cu after the Krylov
// kernel templates it builds on.
#pragma once

namespace sa {

// Slots of KState::g used by the CG scalars; KState::jdone = 1 asks the host
// for the true-residual check (jdone lies in the state tail the host reads).
enum { CG_RR = 0, CG_ALPHA = 1, CG_BETA = 2 };

template <typename T>
struct CgProduct {                   // q[r] = (A p)[r], acc += p[r] (A p)[r]
    T* q;
    const T* p;
    T* acc;
    static constexpr int kSlices = 0;
    struct Pre { T p; };
    __device__ Pre pre(int r) const { return {p[r]}; }
    __device__ void operator()(int r, T ax, const Pre& o) const {
        q[r] = ax;
        *acc = fma(o.p, ax, *acc);
    }
    __device__ void operator()(int r, T ax) const { (*this)(r, ax, pre(r)); }
};

template <typename T>
struct CgResidual {                  // r[i] = b[i] - (A x)[i] (and p = r), acc += r^2
    T* r;
    T* p;
    const T* b;
    T* acc;
    static constexpr int kSlices = 0;
    struct Pre { T b; };
    __device__ Pre pre(int i) const { return {b[i]}; }
    __device__ void operator()(int i, T ax, const Pre& o) const {
        const T ri = o.b - ax;
        r[i] = ri;
        if (p) p[i] = ri;
        *acc = fma(ri, ri, *acc);
    }
    __device__ void operator()(int i, T ax) const { (*this)(i, ax, pre(i)); }
};

// Product over the block's rows [lo, hi): the SELL-32 copy when present,
// CSR rows (one per thread) otherwise.  Each row reaches the epilogue once.
template <class Sys, typename Epi>
__device__ __forceinline__ void cg_product(const DevArgs* __restrict__ a, KState* ks,
                                           const typename Sys::T* x, int lo, int hi,
                                           const Epi& epi) {
    using T = typename Sys::T;
    const int n = a->n;
    if (a->sell_off) {
        sell_rows<T>(a->sell_off, a->sell_col, reinterpret_cast<const T*>(a->sell_val), x, n, lo,
                     hi, kWarps, a->sell_w, a->sell_keep, &ks->bad_index, epi);
        return;
    }
    const T* val = Sys::val(a);
    int flag = 0;
    for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) {
        T ax = 0;
        for (int e = a->rowptr[r]; e < a->rowptr[r + 1]; ++e) {
            const int c = a->colind[e];
            if ((unsigned)c < (unsigned)n) ax = fma(val[e], x[c], ax);
            else flag = 1;
        }
        epi(r, ax);
    }
    if (flag) atomicOr(&ks->bad_index, 1);
}

// Start: r = b - A x (FP32 inner solves: x = 0, r = b), p = r, ||r||^2,
// ||b||^2; the last block initialises the solve.
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock, 1)
cgg_start_kernel(const DevArgs* __restrict__ a, KState* ks, typename Sys::T* r,
                 typename Sys::T* p, typename Sys::T* partial, int zero_x) {
    using T = typename Sys::T;
    __shared__ T scratch[kWarps * 2];
    __shared__ T red[2];
    T* x = Sys::x(a);
    const T* b = Sys::rhs(a);
    int lo, hi;
    block_rows(a->n, gridDim.x, blockIdx.x, lo, hi);
    T acc[2] = {0, 0};
    if (zero_x) {
        for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const T bi = b[i];
            x[i] = 0;
            r[i] = bi;
            p[i] = bi;
            acc[0] = fma(bi, bi, acc[0]);
        }
        acc[1] = acc[0];
    } else {
        cg_product<Sys>(a, ks, x, lo, hi, CgResidual<T>{r, p, b, &acc[0]});
        for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) acc[1] = fma(b[i], b[i], acc[1]);
    }
    block_sum<T, 2>(acc, 2, red, scratch);
    if (threadIdx.x < 2) partial[blockIdx.x * 2 + threadIdx.x] = red[threadIdx.x];
    if (last_block_arrive(&ks->counter[CNT_START])) {
        __shared__ double tot[2];
        reduce_blocks(partial, gridDim.x, 2, 2, tot);
        if (threadIdx.x == 0) {
            const double rr = tot[0], bnorm = sqrt(tot[1]);
            ks->bnorm = bnorm;
            ks->target = a->tol * bnorm;
            ks->first_relres = rel_residual(sqrt(rr), bnorm);
            ks->beta = sqrt(rr);
            ks->g[CG_RR] = rr;
            ks->iters = 0;
            ks->jdone = 0;
            ks->status = ST_OK;
            ks->finished = 0;
            if (!isfinite(rr) || !isfinite(bnorm)) {
                ks->status = ST_NONFINITE;
                ks->finished = 1;
            } else if (sqrt(rr) <= ks->target) {
                ks->finished = 1;
            } else if (a->max_iters <= 0) {
                ks->status = ST_NOT_CONVERGED;
                ks->finished = 1;
            }
            ks->cycle_over = ks->finished;
            ks->counter[CNT_START] = 0;
        }
    }
}

// q = A p and p^T q; the last block forms alpha = r^T r / p^T q.
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock, 1)
cgg_product_kernel(const DevArgs* __restrict__ a, KState* ks, const typename Sys::T* __restrict__ p,
                   typename Sys::T* __restrict__ q, typename Sys::T* partial) {
    using T = typename Sys::T;
    if (ks->cycle_over) return;
    __shared__ T scratch[kWarps];
    __shared__ T red[1];
    int lo, hi;
    block_rows(a->n, gridDim.x, blockIdx.x, lo, hi);
    T acc[1] = {0};
    cg_product<Sys>(a, ks, p, lo, hi, CgProduct<T>{q, p, &acc[0]});
    block_sum<T, 1>(acc, 1, red, scratch);
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
    if (last_block_arrive(&ks->counter[CNT_DOT])) {
        __shared__ double tot[1];
        reduce_blocks(partial, gridDim.x, 1, 1, tot);
        if (threadIdx.x == 0) {
            const double pq = tot[0];
            if (!(pq > 0.0)) {
                ks->status = isfinite(pq) ? ST_BREAKDOWN : ST_NONFINITE;
                ks->finished = 1;
                ks->cycle_over = 1;
            } else {
                ks->g[CG_ALPHA] = ks->g[CG_RR] / pq;
            }
            ks->counter[CNT_DOT] = 0;
        }
    }
}

// x += alpha p, r -= alpha q, r^T r; the last block counts the iteration and
// decides: non-finite, converged recursively (the host then checks the true
// residual), iteration cap, or beta for the next direction.
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock, 1)
cgg_update_kernel(const DevArgs* __restrict__ a, KState* ks, const typename Sys::T* __restrict__ p,
                  const typename Sys::T* __restrict__ q, typename Sys::T* __restrict__ r,
                  typename Sys::T* partial) {
    using T = typename Sys::T;
    if (ks->cycle_over) return;
    __shared__ T scratch[kWarps];
    __shared__ T red[1];
    const T alpha = (T)ks->g[CG_ALPHA];
    T* x = Sys::x(a);
    int lo, hi;
    block_rows(a->n, gridDim.x, blockIdx.x, lo, hi);
    T acc[1] = {0};
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const T ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc[0] = fma(ri, ri, acc[0]);
    }
    block_sum<T, 1>(acc, 1, red, scratch);
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
    if (last_block_arrive(&ks->counter[CNT_PASS2])) {
        __shared__ double tot[1];
        reduce_blocks(partial, gridDim.x, 1, 1, tot);
        if (threadIdx.x == 0) {
            const double rr = tot[0];
            ks->iters += 1;
            if (!isfinite(rr)) {
                ks->status = ST_NONFINITE;
                ks->finished = 1;
                ks->cycle_over = 1;
            } else if (sqrt(rr) <= ks->target) {
                ks->jdone = 1;                 // true-residual check requested
                ks->cycle_over = 1;
            } else if (ks->iters >= a->max_iters) {
                ks->status = ST_NOT_CONVERGED;
                ks->finished = 1;
                ks->cycle_over = 1;
            } else {
                ks->g[CG_BETA] = rr / ks->g[CG_RR];
                ks->g[CG_RR] = rr;
            }
            ks->counter[CNT_PASS2] = 0;
        }
    }
}

// p = r + beta p.
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock)
cgg_direction_kernel(const DevArgs* __restrict__ a, const KState* ks,
                     const typename Sys::T* __restrict__ r, typename Sys::T* __restrict__ p) {
    using T = typename Sys::T;
    if (ks->cycle_over) return;
    const T beta = (T)ks->g[CG_BETA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a->n; i += gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], r[i]);
}

// True residual r = b - A x and its norm (into beta).  check != 0: the
// convergence check -- the solve ends if it passes; otherwise CG restarts
// from it (p = r, r^T r) unless the iteration cap is reached.
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock, 1)
cgg_true_residual_kernel(const DevArgs* __restrict__ a, KState* ks, typename Sys::T* r,
                         typename Sys::T* p, typename Sys::T* partial, int check) {
    using T = typename Sys::T;
    __shared__ T scratch[kWarps];
    __shared__ T red[1];
    int lo, hi;
    block_rows(a->n, gridDim.x, blockIdx.x, lo, hi);
    T acc[1] = {0};
    cg_product<Sys>(a, ks, Sys::x(a), lo, hi,
                    CgResidual<T>{r, check ? p : nullptr, Sys::rhs(a), &acc[0]});
    block_sum<T, 1>(acc, 1, red, scratch);
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
    if (last_block_arrive(&ks->counter[CNT_RES])) {
        __shared__ double tot[1];
        reduce_blocks(partial, gridDim.x, 1, 1, tot);
        if (threadIdx.x == 0) {
            const double rr = tot[0];
            ks->beta = sqrt(rr);
            if (check) {
                ks->jdone = 0;
                if (!isfinite(rr)) {
                    ks->status = ST_NONFINITE;
                    ks->finished = 1;
                } else if (sqrt(rr) <= ks->target) {
                    ks->finished = 1;
                } else if (ks->iters >= a->max_iters) {
                    ks->status = ST_NOT_CONVERGED;
                    ks->finished = 1;
                } else {
                    ks->g[CG_RR] = rr;          // restart from the true residual
                }
                ks->cycle_over = ks->finished;
            }
            ks->counter[CNT_RES] = 0;
        }
    }
}

// The graph body: `iters` CG iterations (three kernels each); kernels after
// the end of the solve or a check request return at once.
template <class Sys>
static void launch_cg_iterations(const DevArgs* a, KState* ks, typename Sys::T* r, typename Sys::T* p,
                                 typename Sys::T* q, typename Sys::T* partial, int nblk, int iters,
                                 cudaStream_t st) {
    for (int k = 0; k < iters; ++k) {
        cgg_product_kernel<Sys><<<nblk, kStreamBlock, 0, st>>>(a, ks, p, q, partial);
        cgg_update_kernel<Sys><<<nblk, kStreamBlock, 0, st>>>(a, ks, p, q, r, partial);
        cgg_direction_kernel<Sys><<<nblk, kStreamBlock, 0, st>>>(a, ks, r, p);
    }
}

}  // namespace sa
