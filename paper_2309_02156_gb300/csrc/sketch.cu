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

// Sketch entries of column j (row j of A), in acceptance order, packed as
// row | sign << 15 (sign bit set for -1).
__device__ __forceinline__ void sketch_column_packed(int j, int s, int zeta, uint64_t seed,
                                                     uint16_t* out) {
    uint64_t taken0 = 0, taken1 = 0;                  // rows already taken (s <= 128)
    int cnt = 0;
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    for (int c = 0; c < 256 && cnt < zeta; ++c) {
        const uint64_t ctr = (uint64_t)j * 256ull + (uint64_t)(c + 1);
        const uint64_t h = mix64(seed + ctr * gamma);
        const int q = (int)(((h >> 32) * (uint64_t)s) >> 32);
        const uint64_t bit = 1ull << (q & 63);
        const bool dup = ((q < 64 ? taken0 : taken1) & bit) != 0;
        if (!dup) {
            if (q < 64) taken0 |= bit; else taken1 |= bit;
            out[cnt] = (uint16_t)(q | ((h & 1ull) ? 0x8000 : 0));
            ++cnt;
        }
    }
    for (int q = 0; cnt < zeta && q < s; ++q) {      // exhausted: smallest unused rows
        const uint64_t bit = 1ull << (q & 63);
        if (((q < 64 ? taken0 : taken1) & bit) == 0) {
            if (q < 64) taken0 |= bit; else taken1 |= bit;
            out[cnt] = (uint16_t)q;
            ++cnt;
        }
    }
}

__global__ void sketch_columns_kernel(int n, int s, int zeta, uint64_t seed,
                                      uint16_t* packed, int32_t* rows_out, int8_t* signs_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint16_t e[kMaxZeta];
    sketch_column_packed(j, s, zeta, seed, e);
    for (int k = 0; k < zeta; ++k) {
        if (packed) packed[(size_t)j * zeta + k] = e[k];
        if (rows_out) rows_out[(size_t)j * zeta + k] = e[k] & 0x7fff;
        if (signs_out) signs_out[(size_t)j * zeta + k] = (e[k] & 0x8000) ? (int8_t)-1 : (int8_t)1;
    }
}

void launch_sketch_columns(int n, int s, int zeta, uint64_t seed, uint16_t* packed,
                           int32_t* rows, int8_t* signs, cudaStream_t st) {
    const int threads = 256;
    sketch_columns_kernel<<<(n + threads - 1) / threads, threads, 0, st>>>(
        n, s, zeta, seed, packed, rows, signs);
}

namespace {

constexpr int kSkWarps = 4;          // warps per block of the sketch kernel
constexpr int kSkStage = 256;        // CSR entries of a 32-row tile staged in shared memory
constexpr int kSkFastRow = 5;        // rows up to this many entries take the unrolled path
constexpr int kSkValueBits = 52;     // |quantised value| < 2^52 (the bits of an FP64 mantissa)

// Bytes of one warp's shared region: integer accumulator (s x ncol), the
// tile's Y (32 x ncol doubles), staged CSR values and columns, sketch entries.
__host__ __device__ inline size_t sketch_warp_bytes(int s, int ncol) {
    return 8 * (size_t)s * ncol + 8 * 32 * (size_t)ncol + 12 * (size_t)kSkStage +
           2 * 32 * (size_t)kMaxZeta;
}

// y (finite) as a fixed-point integer with F fraction bits, rounded to
// nearest (halves away from zero), by integer operations on its bits.  The
// caller guarantees |y| 2^F < 2^kSkValueBits.
__device__ __forceinline__ long long quantize(double y, int F) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(y);
    const int eb = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = bits & 0xfffffffffffffull;
    if (eb) mant |= 1ull << 52;
    const int sh = (eb ? eb - 1075 : -1074) + F;
    unsigned long long r;
    if (sh >= 0) {
        r = mant << sh;
    } else if (sh > -64) {
        const int d = -sh;
        r = (mant + (1ull << (d - 1))) >> d;
    } else {
        r = 0;
    }
    const long long v = (long long)r;
    return (bits >> 63) ? -v : v;
}

// w / 2^d rounded to nearest (halves up), for an accumulator |w| < 2^63.
__device__ __forceinline__ long long shift_round(long long w, int d) {
    if (d <= 0) return w;
    if (d >= 63) return 0;
    return (w + (1ll << (d - 1))) >> d;
}

}  // namespace

// W += S[:, r] Yq[r, :] for the tile's rows (integers; Wi and Yq row-major
// with ncol columns).  The zeta x ncol (sketch entry, column) pairs of a row
// are spread over the warp's lanes, P per lane; the pairs of one row hit
// distinct accumulators, so a lane reads all of its P, then writes them back,
// and the warp moves to the next row together.
template <int P>
__device__ __forceinline__ void scatter_rows(long long* Wi, const long long* Yq,
                                             const uint16_t* skS, int ncol, int zeta, int cnt) {
    const int lane = threadIdx.x & 31;
    int zz[P], kk[P];
    bool ok[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const int p = lane + 32 * i;
        ok[i] = p < zeta * ncol;
        zz[i] = ok[i] ? p / ncol : 0;
        kk[i] = ok[i] ? p - zz[i] * ncol : 0;
    }
    for (int r = 0; r < cnt; ++r) {
        int off[P];
        long long cur[P];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (ok[i]) {
                const unsigned e = skS[r * kMaxZeta + zz[i]];
                const long long v = Yq[r * ncol + kk[i]];
                off[i] = (int)(e & 0x7fff) * ncol + kk[i];
                cur[i] = Wi[off[i]] + ((e & 0x8000) ? -v : v);
            }
        }
#pragma unroll
        for (int i = 0; i < P; ++i)
            if (ok[i]) Wi[off[i]] = cur[i];
        __syncwarp();
    }
}

// W = S [A X | b] in one pass over A and X, with S generated on the fly.
//
// The grid's warps take 32-row tiles in turn.  For a tile it stages the rows' CSR entries,
// generates the rows' sketch columns (zeta entries each), and forms
// Y = [A X | b] with the 32 x M products spread over all 32 lanes (lane l
// computes entries l, l + 32, ... in row-major order, several at once).  The
// scatter W += S[:, r] Y_r then runs in exact integer arithmetic: lane k turns
// column k of the tile into fixed-point integers (a per-column scale with
// values below 2^52, chosen from the running maximum of the column; when a
// larger value arrives the accumulated column is shifted to the new scale),
// and the warp adds +-v into its private 64-bit accumulator at the zeta
// sketch rows of each row.  Integer sums do not depend on their order, so the result is
// deterministic, and the sketch's zeta (M+1) additions per row leave the
// FP64 pipe (the limiting unit of this GPU for FP64 work) to the products;
// the additions of one row are spread over all lanes (scatter_rows).
// At the end the block's warps are converted back to FP64 and summed in warp
// order into partial[blk] (s (M+1) values); a column with a non-finite value
// becomes NaN.  A warp takes at most 33 tiles (grid sizing), so an
// accumulator holds at most 1056 terms below 2^52 and stays below 2^63.
template <typename T, typename XT, int P>
__global__ void __launch_bounds__(kSkWarps * 32)
sketch_block_kernel(const int* __restrict__ rowptr, const int* __restrict__ colind,
                    const T* __restrict__ val, const XT* __restrict__ X, int ldx,
                    const double* __restrict__ b, int n, int nnz, int M, int s, int zeta,
                    uint64_t seed, double* __restrict__ partial, int* bad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int Fsh[kSkWarps][32];
    __shared__ int stat[kSkWarps][32];      // bit 0: column has values, bit 1: non-finite
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncol = M + 1, wsz = s * ncol;
    unsigned char* base_ptr = smem_raw + (size_t)warp * sketch_warp_bytes(s, ncol);
    long long* Wi = reinterpret_cast<long long*>(base_ptr);
    double* Ys = reinterpret_cast<double*>(Wi + wsz);
    T* valS = reinterpret_cast<T*>(Ys + 32 * ncol);
    int* colS = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(valS) + 8 * kSkStage);
    uint16_t* skS = reinterpret_cast<uint16_t*>(colS + kSkStage);
    for (int i = lane; i < wsz; i += 32) Wi[i] = 0;
    int F = 0, has = 0, nonfinite = 0, flag = 0;
    // This lane's first product entry in the row-major 32 x M tile, and the
    // step to the next one (32 entries further).
    const int r_first = lane / M, k_first = lane - (lane / M) * M;
    const int dr = 32 / M, dk = 32 - (32 / M) * M;
    // Tiles are dealt to the grid's warps cyclically, so that at any time the
    // whole GPU works on one window of consecutive rows and the X rows a
    // stencil shares between rows far apart (r and r +- the grid side) are
    // still in L2 when their second reader comes.
    const int hi = n;
    const long long ntiles = ((long long)n + 31) / 32;
    for (long long tile = (long long)blockIdx.x * kSkWarps + warp; tile < ntiles;
         tile += (long long)gridDim.x * kSkWarps) {
        const int base = (int)(tile * 32);
        const int cnt = min(32, hi - base);
        int rs = 0, re = 0;
        if (lane < cnt) {
            rs = max(0, min(__ldg(rowptr + base + lane), nnz));
            re = max(rs, min(__ldg(rowptr + base + lane + 1), nnz));
            sketch_column_packed(base + lane, s, zeta, seed, skS + lane * kMaxZeta);
        }
        const int e0 = __shfl_sync(0xffffffffu, rs, 0);
        const int e1 = max(e0, __shfl_sync(0xffffffffu, re, cnt - 1));
        const bool staged = e1 - e0 <= kSkStage;
        if (staged) {
            for (int e = e0 + lane; e < e1; e += 32) {
                colS[e - e0] = __ldg(colind + e);
                valS[e - e0] = __ldg(val + e);
            }
        }
        if (lane < 32) Ys[lane * ncol + M] = lane < cnt ? __ldg(b + base + lane) : 0.0;
        __syncwarp();
        // Y[:, 0:M] = A X for the tile's rows, four entries per lane at a time.
        int r = r_first, k = k_first;
        for (int j = 0; j < M; j += 4) {
            int rr[4], kk[4], st[4], ln[4];
            T acc[4];
            int maxlen = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                rr[u] = r;
                kk[u] = k;
                const int srow = min(r, 31);
                const int a = __shfl_sync(0xffffffffu, rs, srow);
                const int z = __shfl_sync(0xffffffffu, re, srow);
                const bool live = (j + u < M) && r < cnt;
                st[u] = a;
                ln[u] = live ? z - a : 0;
                maxlen = max(maxlen, ln[u]);
                acc[u] = 0;
                k += dk;
                r += dr;
                if (k >= M) {
                    k -= M;
                    r += 1;
                }
            }
            if (maxlen <= kSkFastRow) {
                // Rows of at most kSkFastRow entries: every load of the four
                // entries is issued before the first product.
                T xv[4][kSkFastRow], vv[4][kSkFastRow];
#pragma unroll
                for (int t = 0; t < kSkFastRow; ++t) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        xv[u][t] = 0;
                        vv[u][t] = 0;
                        if (t < ln[u]) {
                            const int e = st[u] + t;
                            const int c = staged ? colS[e - e0] : __ldg(colind + e);
                            if ((unsigned)c < (unsigned)n) {
                                vv[u][t] = staged ? valS[e - e0] : __ldg(val + e);
                                xv[u][t] = (T)__ldg(X + (size_t)c * ldx + kk[u]);
                            } else {
                                flag = 1;
                            }
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < kSkFastRow; ++t) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (t < ln[u]) acc[u] = fma(vv[u][t], xv[u][t], acc[u]);
                }
            } else {
                for (int t = 0; t < maxlen; ++t) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (t < ln[u]) {
                            const int e = st[u] + t;
                            const int c = staged ? colS[e - e0] : __ldg(colind + e);
                            const T v = staged ? valS[e - e0] : __ldg(val + e);
                            if ((unsigned)c < (unsigned)n)
                                acc[u] = fma(v, (T)__ldg(X + (size_t)c * ldx + kk[u]), acc[u]);
                            else
                                flag = 1;
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j + u < M && rr[u] < 32) Ys[rr[u] * ncol + kk[u]] = rr[u] < cnt ? (double)acc[u] : 0.0;
        }
        __syncwarp();
        long long* Yq = reinterpret_cast<long long*>(Ys);     // quantised in place
        if (lane < ncol) {
            // Column scale from the tile's largest magnitude, then the column
            // as fixed-point integers (zeros for a column with no finite scale).
            unsigned long long mx = 0;
            for (int q = 0; q < cnt; ++q) {
                const unsigned long long a =
                    (unsigned long long)__double_as_longlong(Ys[q * ncol + lane]) & 0x7fffffffffffffffull;
                mx = a > mx ? a : mx;
            }
            if (mx >= 0x7ff0000000000000ull) nonfinite = 1;
            const bool use = mx != 0 && !nonfinite;
            if (use) {
                const int emax = (int)(mx >> 52) - 1023;          // mx < 2^(emax + 1)
                const int Fn = (kSkValueBits - 1) - emax;
                if (!has) {
                    F = Fn;
                    has = 1;
                } else if (Fn < F) {
                    const int d = F - Fn;
                    for (int q = 0; q < s; ++q) Wi[q * ncol + lane] = shift_round(Wi[q * ncol + lane], d);
                    F = Fn;
                }
            }
            for (int q = 0; q < 32; ++q)
                Yq[q * ncol + lane] = (use && q < cnt) ? quantize(Ys[q * ncol + lane], F) : 0;
        }
        __syncwarp();
        scatter_rows<P>(Wi, Yq, skS, ncol, zeta, cnt);
        __syncwarp();
    }
    if (flag) atomicOr(bad, 1);
    Fsh[warp][lane] = F;
    stat[warp][lane] = has | (nonfinite << 1);
    __syncthreads();
    double* out = partial + (size_t)blockIdx.x * wsz;
    for (int i = threadIdx.x; i < wsz; i += blockDim.x) {
        const int k = i % ncol;
        double acc = 0.0;
        bool nan = false;
        for (int w = 0; w < kSkWarps; ++w) {
            const int sw = stat[w][k];
            nan |= (sw & 2) != 0;
            if (sw & 1) {
                const long long* Ww = reinterpret_cast<const long long*>(
                    smem_raw + (size_t)w * sketch_warp_bytes(s, ncol));
                acc += scalbn((double)Ww[i], -Fsh[w][k]);
            }
        }
        out[i] = nan ? __longlong_as_double(0x7ff8000000000000ll) : acc;
    }
}

// W[i] = (1/sqrt(zeta)) * sum over blocks of partial[blk][i] (fixed order).
__global__ void sketch_reduce_kernel(const double* __restrict__ partial, int nblk, int wsz,
                                     double inv_sqrt_zeta, double* __restrict__ W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= wsz) return;
    W[i] = sum_over_blocks(partial, nblk, wsz, i) * inv_sqrt_zeta;
}

// Blocks of the sketch kernel: two per SM, more when needed so that no warp
// takes more than 33 tiles of 32 rows (so its accumulators stay below 2^63),
// never more than one per 128 rows.
int sketch_grid(int n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nblk = sms * 2;
    const int by_rows = (int)(((long long)n + 4095) / 4096);
    if (by_rows > nblk) nblk = by_rows;
    const int need = (n + 127) / 128;
    return nblk < need ? nblk : (need > 0 ? need : 1);
}

size_t sketch_partial_doubles(int n, int s, int M) {
    return (size_t)sketch_grid(n) * s * (M + 1);
}

// Kernel for P = ceil(zeta (M+1) / 32) scatter pairs per lane.
template <typename T, typename XT, int P>
static void launch_sketch_p(const int* rowptr, const int* colind, const T* val, const XT* X,
                            int ldx, const double* b, int n, int nnz, int M, int s, int zeta,
                            uint64_t seed, double* partial, int nblk, int* bad, cudaStream_t st) {
    const size_t smem = kSkWarps * sketch_warp_bytes(s, M + 1);
    // The attribute is per device: set it on every call (cheap, host only).
    cudaFuncSetAttribute(sketch_block_kernel<T, XT, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    sketch_block_kernel<T, XT, P><<<nblk, kSkWarps * 32, smem, st>>>(
        rowptr, colind, val, X, ldx, b, n, nnz, M, s, zeta, seed, partial, bad);
}

template <typename T, typename XT>
static void launch_sketch_impl(const int* rowptr, const int* colind, const T* val, const XT* X,
                               int ldx, const double* b, int n, int nnz, int M, int s, int zeta,
                               uint64_t seed, double* partial, int nblk, double* W, int* bad,
                               cudaStream_t st) {
    const int wsz = s * (M + 1);
#define SA_SK(PP)                                                                           \
    launch_sketch_p<T, XT, PP>(rowptr, colind, val, X, ldx, b, n, nnz, M, s, zeta, seed, \
                               partial, nblk, bad, st)
    switch ((zeta * (M + 1) + 31) / 32) {
        case 1: SA_SK(1); break;
        case 2: SA_SK(2); break;
        case 3: SA_SK(3); break;
        case 4: SA_SK(4); break;
        case 5: SA_SK(5); break;
        case 6: SA_SK(6); break;
        case 7: SA_SK(7); break;
        case 8: SA_SK(8); break;
        case 9: case 10: SA_SK(10); break;
        case 11: case 12: SA_SK(12); break;
        default: SA_SK(16); break;
    }
#undef SA_SK
    const double inv = 1.0 / sqrt((double)zeta);
    sketch_reduce_kernel<<<(wsz + 127) / 128, 128, 0, st>>>(partial, nblk, wsz, inv, W);
}

void launch_sketch_f64(const int* rowptr, const int* colind, const double* val, const double* X,
                       int ldx, const double* b, int n, int nnz, int M, int s, int zeta,
                       uint64_t seed, double* partial, int nblk, double* W, int* bad,
                       cudaStream_t st) {
    launch_sketch_impl<double, double>(rowptr, colind, val, X, ldx, b, n, nnz, M, s, zeta, seed,
                                       partial, nblk, W, bad, st);
}

void launch_sketch_f32(const int* rowptr, const int* colind, const float* val, const float* X,
                       int ldx, const double* b, int n, int nnz, int M, int s, int zeta,
                       uint64_t seed, double* partial, int nblk, double* W, int* bad,
                       cudaStream_t st) {
    launch_sketch_impl<float, float>(rowptr, colind, val, X, ldx, b, n, nnz, M, s, zeta, seed,
                                     partial, nblk, W, bad, st);
}

}  // namespace sa
