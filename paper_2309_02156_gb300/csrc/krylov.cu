// Krylov solvers on the FP64 system, the mixed-precision outer loop and the
// single-block CG.  The kernel templates live in krylov_kernels.cuh.
#include <math.h>

#include "krylov_kernels.cuh"
#include "cg_kernels.cuh"

namespace sa {

int stream_grid(int n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int need = (n + kStreamBlock - 1) / kStreamBlock;
    return need < sms ? (need > 0 ? need : 1) : sms;
}

// ---------------------------------------------------------------------------
// ||b - A x|| and ||b|| (FP64); x_override replaces a->x when not NULL.
__global__ void __launch_bounds__(kStreamBlock, 1)
residual_norm_kernel(const DevArgs* __restrict__ a, KState* ks, double* partial,
                     const double* x_override) {
    __shared__ double sprod[kWarps * kTileP];
    __shared__ double scratch[kWarps * 2];
    __shared__ double red[2];
    const int n = a->n, nnz = a->nnz;
    const double* x = x_override ? x_override : a->x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    double acc[2] = {0.0, 0.0};
    for (int r0 = lo + warp * 32; r0 < hi; r0 += kWarps * 32) {
        const double ax = warp_tile_spmv<double>(a->rowptr, a->colind, a->val64, x, n, nnz, r0,
                                                 sprod + warp * kTileP, &ks->bad_index);
        const int row = r0 + lane;
        if (row < n) {
            const double bi = a->b[row];
            const double r = bi - ax;
            acc[0] += r * r;
            acc[1] += bi * bi;
        }
    }
    block_sum<double, 2>(acc, 2, red, scratch);
    if (threadIdx.x < 2) partial[blockIdx.x * 2 + threadIdx.x] = red[threadIdx.x];
    if (last_block_arrive(&ks->counter[CNT_RES])) {
        __shared__ double tot[2];
        reduce_blocks(partial, gridDim.x, 2, 2, tot);
        if (threadIdx.x == 0) {
            ks->beta = sqrt(tot[0]);
            ks->bnorm = sqrt(tot[1]);
            ks->first_relres = rel_residual(sqrt(tot[0]), sqrt(tot[1]));
            ks->counter[CNT_RES] = 0;
        }
    }
}

void launch_residual_norm(const DevArgs* a, KState* ks, double* partial, int nblk,
                          const double* x_override, cudaStream_t st) {
    residual_norm_kernel<<<nblk, kStreamBlock, 0, st>>>(a, ks, partial, x_override);
}

void launch_gmres_start_f64(const DevArgs* a, KState* ks, double* V, size_t, double* partial,
                            int nblk, int first, cudaStream_t st) {
    launch_start<SysF64>(a, ks, V, partial, nblk, first, st);
}
void launch_gmres_cycle_f64(const DevArgs* a, KState* ks, double* V, size_t ldv, double* w,
                            double* partial, int nblk, int R, cudaStream_t st, int* launches,
                            cudaEvent_t* ev, int sweeps, double omega, const double* dinv,
                            double* za, double* zb, double* t, const ChebConfig* cheb, double* dvec) {
    PrecondArgs<double> pc;
    pc.sweeps = sweeps;
    pc.omega = omega;
    pc.dinv = dinv;
    pc.za = za;
    pc.zb = zb;
    pc.t = t;
    if (cheb && cheb->on) {
        pc.cheb = 1;
        pc.tab = cheb->tab;
        pc.dvec = dvec;
    }
    launch_cycle<SysF64>(a, ks, V, ldv, w, partial, nblk, R, st, launches, ev, pc);
}
void launch_cheb_table(double* tab, double lfix, double ratio, int sweeps, cudaStream_t st) {
    cheb_table_kernel<<<1, 32, 0, st>>>(tab, lfix, ratio, sweeps);
}
void launch_diag_inv_f64(const DevArgs* a, double* dinv, int n, cudaStream_t st,
                         unsigned long long* bound) {
    int b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    diag_inv_kernel<SysF64><<<b > 0 ? b : 1, 256, 0, st>>>(a, dinv, bound);
}
// ---------------------------------------------------------------------------
// CSR -> SELL-32 conversion (once per solve; the GMRES cycles then run ~10^3
// products on the same matrix).  Slice s holds rows 32 s .. 32 s + 31; its
// width is its longest row; entry k of row 32 s + l sits at
// off[s] + 32 k + l.  Padding entries have column -1 and value 0.
__global__ void sell_width_kernel(const int* __restrict__ rowptr, int n, int nnz, int* width) {
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int ns = (n + 31) >> 5;
    if (s >= ns) return;
    const int row = s * 32 + lane;
    int len = 0;
    if (row < n) {
        const int rs = max(0, min(rowptr[row], nnz));
        const int re = max(rs, min(rowptr[row + 1], nnz));
        len = re - rs;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if (lane == 0) width[s] = len;
}

// Exclusive scan of 32 * width over the slices by one block (off[ns] = total,
// off[ns + 1] = the widest slice).
__global__ void sell_scan_kernel(const int* __restrict__ width, int ns, int* off) {
    __shared__ long long wsum[32];
    __shared__ long long carry;
    __shared__ int wmax;
    if (threadIdx.x == 0) {
        carry = 0;
        wmax = 0;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < ns; s += blockDim.x) atomicMax(&wmax, width[s]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < ns; base += blockDim.x) {
        const int s = base + threadIdx.x;
        long long v = s < ns ? 32LL * width[s] : 0;
        long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        long long before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        const long long excl = carry + before + incl - v;
        if (s < ns) off[s] = (int)min(excl, (long long)0x7fffffff);
        __syncthreads();
        if (threadIdx.x == 0) {
            long long tot = 0;
            for (int w = 0; w < nw; ++w) tot += wsum[w];
            carry += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[ns] = (int)min(carry, (long long)0x7fffffff);
        off[ns + 1] = wmax;
    }
}

// Every slice padded to width w: off[s] = 32 w s for s <= ns.
__global__ void sell_uniform_kernel(int ns, int w, int* off) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= ns; s += gridDim.x * blockDim.x)
        off[s] = 32 * w * s;
}

template <typename VT>
__global__ void sell_fill_kernel(const int* __restrict__ rowptr, const int* __restrict__ colind,
                                 const VT* __restrict__ val, int n, int nnz,
                                 const int* __restrict__ off, int* col_out, VT* val_out) {
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int ns = (n + 31) >> 5;
    if (s >= ns) return;
    const int o = off[s], w = (off[s + 1] - o) >> 5;
    const int row = s * 32 + lane;
    int rs = 0, re = 0;
    if (row < n) {
        rs = max(0, min(rowptr[row], nnz));
        re = max(rs, min(rowptr[row + 1], nnz));
    }
    for (int k = 0; k < w; ++k) {
        const int e = rs + k;
        const bool ok = e < re;
        col_out[o + k * 32 + lane] = ok ? colind[e] : -1;
        val_out[o + k * 32 + lane] = ok ? val[e] : (VT)0;
    }
}

void launch_sell_layout(const int* rowptr, int n, int nnz, int* width, int* off, cudaStream_t st) {
    const int ns = (n + 31) / 32;
    sell_width_kernel<<<(ns + 7) / 8, 256, 0, st>>>(rowptr, n, nnz, width);
    sell_scan_kernel<<<1, 1024, 0, st>>>(width, ns, off);
}

void launch_sell_uniform(int n, int w, int* off, cudaStream_t st) {
    const int ns = (n + 31) / 32;
    sell_uniform_kernel<<<(ns + 256) / 256, 256, 0, st>>>(ns, w, off);
}

void launch_sell_fill_f64(const int* rowptr, const int* colind, const double* val, int n, int nnz,
                          const int* off, int* col, double* v, cudaStream_t st) {
    const int ns = (n + 31) / 32;
    sell_fill_kernel<double><<<(ns + 7) / 8, 256, 0, st>>>(rowptr, colind, val, n, nnz, off, col, v);
}

void launch_sell_fill_f32(const int* rowptr, const int* colind, const float* val, int n, int nnz,
                          const int* off, int* col, float* v, cudaStream_t st) {
    const int ns = (n + 31) / 32;
    sell_fill_kernel<float><<<(ns + 7) / 8, 256, 0, st>>>(rowptr, colind, val, n, nnz, off, col, v);
}

// ---------------------------------------------------------------------------
// Mixed precision: r = b - A64 x in FP64 (into r64), beta = ||r||, ||b||.
__global__ void __launch_bounds__(kStreamBlock, 1)
refine_residual_kernel(const DevArgs* __restrict__ a, KState* ks, double* r64, double* partial) {
    __shared__ double sprod[kWarps * kTileP];
    __shared__ double scratch[kWarps * 2];
    __shared__ double red[2];
    const int n = a->n, nnz = a->nnz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    double acc[2] = {0.0, 0.0};
    for (int r0 = lo + warp * 32; r0 < hi; r0 += kWarps * 32) {
        const double ax = warp_tile_spmv<double>(a->rowptr, a->colind, a->val64, a->x, n, nnz, r0,
                                                 sprod + warp * kTileP, &ks->bad_index);
        const int row = r0 + lane;
        if (row < n) {
            const double bi = a->b[row];
            const double r = bi - ax;
            r64[row] = r;
            acc[0] += r * r;
            acc[1] += bi * bi;
        }
    }
    block_sum<double, 2>(acc, 2, red, scratch);
    if (threadIdx.x < 2) partial[blockIdx.x * 2 + threadIdx.x] = red[threadIdx.x];
    if (last_block_arrive(&ks->counter[CNT_REFINE])) {
        __shared__ double tot[2];
        reduce_blocks(partial, gridDim.x, 2, 2, tot);
        if (threadIdx.x == 0) {
            ks->beta = sqrt(tot[0]);
            ks->bnorm = sqrt(tot[1]);
            ks->target = a->tol * ks->bnorm;
            ks->counter[CNT_REFINE] = 0;
        }
    }
}

void launch_refine_residual(const DevArgs* a, KState* ks, double* r64, double* partial, int nblk,
                            cudaStream_t st) {
    refine_residual_kernel<<<nblk, kStreamBlock, 0, st>>>(a, ks, r64, partial);
}

// rhs32 = r / ||r|| in FP32: the inner equation is A d = r / ||r|| and the
// correction ||r|| d, the same solve in exact arithmetic (the inner tolerance
// is relative), with the FP32 right-hand side and its dot products in range
// whatever the scale of b.
__global__ void refine_scale_kernel(const double* __restrict__ r64, const KState* __restrict__ ks,
                                    float* __restrict__ rhs32, int n) {
    const double inv = 1.0 / ks->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        rhs32[i] = (float)(r64[i] * inv);
}

void launch_refine_scale(const double* r64, const KState* ks, float* rhs32, int n, cudaStream_t st) {
    int b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    refine_scale_kernel<<<b > 0 ? b : 1, 256, 0, st>>>(r64, ks, rhs32, n);
}

// x += ||r|| d (FP64 += the FP32 correction of the inner solve on r / ||r||;
// ||r|| = outer->beta, the residual norm the right-hand side was scaled by).
__global__ void refine_update_kernel(const DevArgs* __restrict__ a, const KState* __restrict__ outer) {
    const int n = a->n;
    const float* d = reinterpret_cast<const float*>(a->d);
    const double beta = outer->beta;
    double* x = a->x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] = fma(beta, (double)d[i], x[i]);
}

void launch_refine_update(const DevArgs* a, const KState* outer, cudaStream_t st) {
    refine_update_kernel<<<152 * 8, 256, 0, st>>>(a, outer);
}

__global__ void round_f32_kernel(const double* __restrict__ src, float* __restrict__ dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

void launch_round_f32(const double* src, float* dst, int n, cudaStream_t st) {
    int b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    round_f32_kernel<<<b, 256, 0, st>>>(src, dst, n);
}

// ---------------------------------------------------------------------------
// CG in one thread block: the whole iteration runs on the device with block
// barriers only (no launches, no host round trips).  Meant for small and
// medium systems; the batched form runs one such solve per sequence.
template <class Sys>
__device__ __forceinline__ typename Sys::T csr_row(const DevArgs* a, const typename Sys::T* x,
                                                   int i, int n, int nnz, int& bad) {
    using T = typename Sys::T;
    const T* val = Sys::val(a);
    int rs = max(0, min(a->rowptr[i], nnz));
    int re = max(rs, min(a->rowptr[i + 1], nnz));
    T acc = 0;
    for (int e = rs; e < re; ++e) {
        const int c = a->colind[e];
        if ((unsigned)c < (unsigned)n)
            acc += val[e] * x[c];
        else
            bad = 1;
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ T block_total(T v, T* sred) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sred[warp] = v;
    __syncthreads();
    T t = 0;
    for (int w = 0; w < nw; ++w) t += sred[w];
    return t;
}

template <class Sys>
__global__ void __launch_bounds__(1024)
cg_block_kernel(const DevArgs* __restrict__ a, KState* ks, typename Sys::T* r, typename Sys::T* p,
                typename Sys::T* q) {
    using T = typename Sys::T;
    __shared__ T sred[32];
    const int n = a->n, nnz = a->nnz, tid = threadIdx.x, bd = blockDim.x;
    T* x = Sys::x(a);
    const T* b = Sys::rhs(a);
    int bad = 0;
    const bool zero_x = sizeof(T) == 4;      // the FP32 inner solve starts from d = 0
    if (zero_x)
        for (int i = tid; i < n; i += bd) x[i] = 0;
    __syncthreads();
    T rr_l = 0, bb_l = 0;
    for (int i = tid; i < n; i += bd) {
        const T ri = b[i] - (zero_x ? (T)0 : csr_row<Sys>(a, x, i, n, nnz, bad));
        r[i] = ri;
        p[i] = ri;
        rr_l += ri * ri;
        bb_l += b[i] * b[i];
    }
    T rr = block_total(rr_l, sred);
    const T bb = block_total(bb_l, sred);
    const double bnorm = sqrt((double)bb);
    const double target = a->tol * bnorm;
    const double first = rel_residual(sqrt((double)rr), bnorm);
    int it = 0, status = ST_OK;
    if (!isfinite((double)rr) || !isfinite(bnorm)) {
        status = ST_NONFINITE;
    } else if (sqrt((double)rr) > target) {
        for (;;) {
            if (it >= a->max_iters) {
                status = ST_NOT_CONVERGED;
                break;
            }
            __syncthreads();
            T pq_l = 0;
            for (int i = tid; i < n; i += bd) {
                const T qi = csr_row<Sys>(a, p, i, n, nnz, bad);
                q[i] = qi;
                pq_l += p[i] * qi;
            }
            const T pq = block_total(pq_l, sred);
            if (!(pq > 0)) {
                status = isfinite((double)pq) ? ST_BREAKDOWN : ST_NONFINITE;
                break;
            }
            const T alpha = rr / pq;
            T rn_l = 0;
            for (int i = tid; i < n; i += bd) {
                x[i] += alpha * p[i];
                const T ri = r[i] - alpha * q[i];
                r[i] = ri;
                rn_l += ri * ri;
            }
            const T rr_new = block_total(rn_l, sred);
            ++it;
            if (!isfinite((double)rr_new)) {
                status = ST_NONFINITE;
                break;
            }
            if (sqrt((double)rr_new) <= target) {
                __syncthreads();
                T t_l = 0;
                for (int i = tid; i < n; i += bd) {
                    const T ri = b[i] - csr_row<Sys>(a, x, i, n, nnz, bad);
                    r[i] = ri;
                    t_l += ri * ri;
                }
                rr = block_total(t_l, sred);
                if (sqrt((double)rr) <= target) break;
                for (int i = tid; i < n; i += bd) p[i] = r[i];
                continue;
            }
            const T beta = rr_new / rr;
            rr = rr_new;
            for (int i = tid; i < n; i += bd) p[i] = r[i] + beta * p[i];
        }
    }
    if (bad) atomicOr(&ks->bad_index, 1);
    __syncthreads();
    // Final true residual (reported, and used by the refinement loop).
    T f_l = 0;
    for (int i = tid; i < n; i += bd) {
        const T ri = b[i] - csr_row<Sys>(a, x, i, n, nnz, bad);
        f_l += ri * ri;
    }
    const T ff = block_total(f_l, sred);
    if (tid == 0) {
        ks->iters = it;
        ks->status = status;
        ks->bnorm = bnorm;
        ks->target = target;
        ks->first_relres = first;
        ks->beta = sqrt((double)ff);
        ks->finished = 1;
        ks->cycle_over = 1;
    }
}

void launch_cg_block_f64(const DevArgs* a, KState* ks, double* r, double* p, double* q,
                         cudaStream_t st) {
    cg_block_kernel<SysF64><<<1, 1024, 0, st>>>(a, ks, r, p, q);
}
void launch_cg_block_f32(const DevArgs* a, KState* ks, float* r, float* p, float* q,
                         cudaStream_t st) {
    cg_block_kernel<SysF32><<<1, 1024, 0, st>>>(a, ks, r, p, q);
}

void launch_cgg_start_f64(const DevArgs* a, KState* ks, double* r, double* p, double* partial,
                          int nblk, cudaStream_t st) {
    cgg_start_kernel<SysF64><<<nblk, kStreamBlock, 0, st>>>(a, ks, r, p, partial, 0);
}
void launch_cgg_start_f32(const DevArgs* a, KState* ks, float* r, float* p, float* partial,
                          int nblk, cudaStream_t st) {
    cgg_start_kernel<SysF32><<<nblk, kStreamBlock, 0, st>>>(a, ks, r, p, partial, 1);
}
void launch_cgg_iterations_f64(const DevArgs* a, KState* ks, double* r, double* p, double* q,
                               double* partial, int nblk, int iters, cudaStream_t st) {
    launch_cg_iterations<SysF64>(a, ks, r, p, q, partial, nblk, iters, st);
}
void launch_cgg_iterations_f32(const DevArgs* a, KState* ks, float* r, float* p, float* q,
                               float* partial, int nblk, int iters, cudaStream_t st) {
    launch_cg_iterations<SysF32>(a, ks, r, p, q, partial, nblk, iters, st);
}
void launch_cgg_true_residual_f64(const DevArgs* a, KState* ks, double* r, double* p,
                                  double* partial, int nblk, int check, cudaStream_t st) {
    cgg_true_residual_kernel<SysF64><<<nblk, kStreamBlock, 0, st>>>(a, ks, r, p, partial, check);
}
void launch_cgg_true_residual_f32(const DevArgs* a, KState* ks, float* r, float* p,
                                  float* partial, int nblk, int check, cudaStream_t st) {
    cgg_true_residual_kernel<SysF32><<<nblk, kStreamBlock, 0, st>>>(a, ks, r, p, partial, check);
}

}  // namespace sa
