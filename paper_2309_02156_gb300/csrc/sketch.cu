// Sparse-sign row sketch and the sketched block W = S [A X | b].
//
// S (s x n) has zeta nonzeros +-1/sqrt(zeta) per column.  Column j draws its
// candidate rows from SplitMix64 outputs 256 j + c + 1 (c = 0, 1, ...):
// row = ((h >> 32) * s) >> 32, sign = bit 0 of h, repeated rows skipped; if
// 256 candidates fall short, the smallest unused rows are taken with sign +1.
// The sketch replaces the n-row reduced least-squares problem of Algorithm 1
// (min ||A(t_i) X y - b(t_i)||) by its s-row image; the paper itself
// sketches columns instead (Section 2.2), so this construction is this
// library's own.
//
// Layout: the history ring X is row-major, n rows of ldx >= M values (slot k
// of row i at X[i * ldx + k]), so the M values a CSR neighbour contributes are
// one contiguous read.  W is row-major s x (M + 1): W[q * (M+1) + k] for
// history slot k < M and W[q * (M+1) + M] for b.
#include "common.cuh"
#include "internal.h"

namespace sa {

__global__ void sketch_columns_kernel(int n, int s, int zeta, uint64_t seed,
                                      uint16_t* packed, int32_t* rows_out, int8_t* signs_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int rows[kMaxZeta];
    int sg[kMaxZeta];
    int cnt = 0;
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    for (int c = 0; c < 256 && cnt < zeta; ++c) {
        const uint64_t ctr = (uint64_t)j * 256ull + (uint64_t)(c + 1);
        const uint64_t h = mix64(seed + ctr * gamma);
        const int q = (int)(((h >> 32) * (uint64_t)s) >> 32);
        bool dup = false;
        for (int k = 0; k < cnt; ++k) dup |= (rows[k] == q);
        if (!dup) {
            rows[cnt] = q;
            sg[cnt] = (h & 1ull) ? -1 : 1;
            ++cnt;
        }
    }
    for (int q = 0; cnt < zeta && q < s; ++q) {      // exhausted: smallest unused rows
        bool used = false;
        for (int k = 0; k < cnt; ++k) used |= (rows[k] == q);
        if (!used) {
            rows[cnt] = q;
            sg[cnt] = 1;
            ++cnt;
        }
    }
    for (int k = 0; k < zeta; ++k) {
        if (packed) packed[(size_t)j * zeta + k] = (uint16_t)(rows[k] | (sg[k] < 0 ? 0x8000 : 0));
        if (rows_out) rows_out[(size_t)j * zeta + k] = rows[k];
        if (signs_out) signs_out[(size_t)j * zeta + k] = (int8_t)sg[k];
    }
}

void launch_sketch_columns(int n, int s, int zeta, uint64_t seed, uint16_t* packed,
                           int32_t* rows, int8_t* signs, cudaStream_t st) {
    const int threads = 256;
    sketch_columns_kernel<<<(n + threads - 1) / threads, threads, 0, st>>>(
        n, s, zeta, seed, packed, rows, signs);
}

// One pass over A and X: for each row r, Y_r = [(A X)_r | b_r] (lane k holds
// column k) and W += S[:, r] Y_r.  Every warp accumulates a private s x (M+1)
// copy of W in shared memory (lane k owns column k, so there are no write
// conflicts and the order of additions is fixed), processing its rows four
// at a time to keep loads in flight.  The block's warps are then summed in
// warp order and written to partial[blk] (s*(M+1) values, then ||b||^2 of the
// block's rows).  Values are accumulated as +-Y and scaled by 1/sqrt(zeta)
// once, in the final reduction.
template <typename T, typename XT>
__global__ void __launch_bounds__(128)
sketch_spmm_kernel(const int* __restrict__ rowptr, const int* __restrict__ colind,
                   const T* __restrict__ val, const XT* __restrict__ X, int ldx,
                   const double* __restrict__ b, const uint16_t* __restrict__ sk,
                   int n, int nnz, int M, int s, int zeta, T* __restrict__ partial, int* bad) {
    extern __shared__ unsigned char smem_raw[];
    T* Ws = reinterpret_cast<T*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int ncol = M + 1;
    const int wsz = s * ncol;
    T* Ww = Ws + warp * wsz;
    for (int i = lane; i < wsz; i += 32) Ww[i] = 0;
    __syncwarp();
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    double bb = 0.0;
    int flag = 0;
    constexpr int R = 4;
    for (int base = lo + warp * R; base < hi; base += nw * R) {
        T y[R];
        int rs[R], re[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int r = base + u;
            rs[u] = re[u] = 0;
            if (r < hi) {
                rs[u] = max(0, min(__ldg(rowptr + r), nnz));
                re[u] = max(rs[u], min(__ldg(rowptr + r + 1), nnz));
            }
            y[u] = 0;
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int r = base + u;
            if (r >= hi) continue;
            if (lane < M) {
                T acc = 0;
                for (int e = rs[u]; e < re[u]; ++e) {
                    const int c = __ldg(colind + e);
                    if ((unsigned)c < (unsigned)n)
                        acc += __ldg(val + e) * (T)__ldg(X + (size_t)c * ldx + lane);
                    else
                        flag = 1;
                }
                y[u] = acc;
            } else if (lane == M) {
                const double bv = __ldg(b + r);
                y[u] = (T)bv;
                bb += bv * bv;
            }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int r = base + u;
            if (r >= hi) continue;
            for (int k = 0; k < zeta; ++k) {
                const unsigned e = __ldg(sk + (size_t)r * zeta + k);
                const int q = e & 0x7fff;
                if (lane < ncol) {
                    T* dst = Ww + q * ncol + lane;
                    *dst = (e & 0x8000) ? *dst - y[u] : *dst + y[u];
                }
            }
            __syncwarp();
        }
    }
    if (flag) atomicOr(bad, 1);
    __syncthreads();
    T* out = partial + (size_t)blockIdx.x * (wsz + 1);
    for (int i = threadIdx.x; i < wsz; i += blockDim.x) {
        T acc = Ws[i];
        for (int w = 1; w < nw; ++w) acc += Ws[w * wsz + i];
        out[i] = acc;
    }
    // ||b||^2 of this block: only lane M of each warp holds a value.
    __shared__ double bbs[32];
    if (lane == M) bbs[warp] = bb;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += bbs[w];
        out[wsz] = (T)t;
    }
}

// W[i] = (1/sqrt(zeta)) * sum over blocks of partial[blk][i] (fixed order);
// W[wsz] = ||b||^2 (not scaled).  One thread per entry.
template <typename T>
__global__ void sketch_reduce_kernel(const T* __restrict__ partial, int nblk, int wsz,
                                     double inv_sqrt_zeta, double* __restrict__ W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > wsz) return;
    T acc = sum_over_blocks(partial, nblk, wsz + 1, i);
    W[i] = (i < wsz) ? (double)acc * inv_sqrt_zeta : (double)acc;
}

int sketch_grid(int n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nblk = sms * 2;
    const int need = (n + 127) / 128;
    return nblk < need ? nblk : (need > 0 ? need : 1);
}

template <typename T, typename XT>
static void launch_sketch_impl(const int* rowptr, const int* colind, const T* val, const XT* X,
                               int ldx, const double* b, const uint16_t* sk, int n, int nnz,
                               int M, int s, int zeta, T* partial, int nblk, double* W, int* bad,
                               cudaStream_t st) {
    const int wsz = s * (M + 1);
    const size_t smem = (size_t)4 * wsz * sizeof(T);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(sketch_spmm_kernel<T, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        attr_set = true;
    }
    sketch_spmm_kernel<T, XT><<<nblk, 128, smem, st>>>(rowptr, colind, val, X, ldx, b, sk, n, nnz,
                                                        M, s, zeta, partial, bad);
    const double inv = 1.0 / sqrt((double)zeta);
    sketch_reduce_kernel<T><<<(wsz + 1 + 127) / 128, 128, 0, st>>>(partial, nblk, wsz, inv, W);
}

void launch_sketch_f64(const int* rowptr, const int* colind, const double* val, const double* X,
                       int ldx, const double* b, const uint16_t* sk, int n, int nnz, int M, int s,
                       int zeta, double* partial, int nblk, double* W, int* bad, cudaStream_t st) {
    launch_sketch_impl<double, double>(rowptr, colind, val, X, ldx, b, sk, n, nnz, M, s, zeta,
                                       partial, nblk, W, bad, st);
}

void launch_sketch_f32(const int* rowptr, const int* colind, const float* val, const float* X,
                       int ldx, const double* b, const uint16_t* sk, int n, int nnz, int M, int s,
                       int zeta, float* partial, int nblk, double* W, int* bad, cudaStream_t st) {
    launch_sketch_impl<float, float>(rowptr, colind, val, X, ldx, b, sk, n, nnz, M, s, zeta,
                                     partial, nblk, W, bad, st);
}

}  // namespace sa
