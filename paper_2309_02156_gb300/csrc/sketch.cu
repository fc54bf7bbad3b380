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
#include <algorithm>

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

constexpr int kSkTeamWarps = 4;      // warps of a team (one 32-row tile at a time)
constexpr int kSkTeamThreads = kSkTeamWarps * 32;
constexpr int kSkMaxTeams = 8;       // teams per block (one block per SM)
constexpr int kSkRowsPerWarp = 8;    // rows of a tile per warp
constexpr int kSkWarpStage = 64;     // CSR entries of a warp's rows staged in shared memory
constexpr int kSkFastRow = 5;        // rows up to this many entries take the unrolled path
constexpr int kSkU = 2;              // product entries per lane in flight (32 warps per SM: 64 registers)
constexpr int kSkValueBits = 52;     // |quantised value| < 2^52 (the bits of an FP64 mantissa)
constexpr int kSkMaxTiles = 33;      // tiles per team: <= 33 * 32 terms per accumulator, < 2^63
constexpr size_t kSkSmemCap = 220 * 1024;

// Bytes of one team's shared region: integer accumulator (s x ncol), the
// tile's Y (32 x ncol doubles, quantised in place), per warp the staged CSR
// values (8 bytes each) and columns, the tile's sketch entries, and per
// column the fixed-point exponent and status.
__host__ __device__ inline size_t sketch_team_bytes(int s, int ncol) {
    return 8 * (size_t)s * ncol + 8 * 32 * (size_t)ncol +
           (size_t)kSkTeamWarps * kSkWarpStage * 12 + 2 * 32 * (size_t)kMaxZeta +
           8 * (size_t)ncol;
}

int sketch_teams(int s, int ncol) {
    const size_t t = kSkSmemCap / sketch_team_bytes(s, ncol);
    return t < 1 ? 1 : (t > (size_t)kSkMaxTeams ? kSkMaxTeams : (int)t);
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

__device__ __forceinline__ void team_sync(int team) {
    asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(kSkTeamThreads) : "memory");
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

}  // namespace

// W = S [A X | b] in one pass over A and X, with S generated on the fly.
//
// A block (one per SM) runs up to eight teams of four warps; each team takes
// 32-row tiles in turn (tiles are dealt to the grid's teams cyclically, so
// that at any time the whole GPU works on one window of consecutive rows and
// the X rows a stencil shares between rows far apart, r and r +- the grid
// side, are still in L2 when their second reader comes).  For a tile:
//  (a) warp w takes rows 8w .. 8w+7: their CSR entries (staged in shared
//      memory) and sketch columns (zeta entries each, generated from the
//      counters), and b;
//  (b) it forms Y = A X on those rows, the 8 x M products spread over its
//      lanes, four at a time;
//  (c) the warps split the M + 1 columns: for each, the tile's largest
//      magnitude sets a fixed-point scale (values below 2^52, chosen from the
//      running maximum of the column; when a larger value arrives the
//      accumulated column is shifted to the new scale) and the column is
//      turned into integers;
//  (d) the team adds +-v into its 64-bit accumulator at the zeta sketch rows
//      of each row (shared-memory atomics: integer sums do not depend on
//      their order, so the result is deterministic), leaving the FP64 pipe
//      (the limiting unit of this GPU for FP64 work) to the products.
// At the end the block's teams are converted back to FP64 and summed in team
// order into partial[blk] (s (M+1) values); a column with a non-finite value
// becomes NaN.  A team takes at most kSkMaxTiles tiles (grid sizing), so an
// accumulator holds at most 1056 terms below 2^52 and stays below 2^63.
template <typename T, typename XT>
__global__ void __launch_bounds__(kSkMaxTeams * kSkTeamThreads, 1)
sketch_block_kernel(const int* __restrict__ rowptr, const int* __restrict__ colind,
                    const T* __restrict__ val, const XT* __restrict__ X, int ldx,
                    const double* __restrict__ b, int n, int nnz, int M, int s, int zeta,
                    uint64_t seed, double* __restrict__ partial, int* bad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nteams = blockDim.x / kSkTeamThreads;
    const int team = threadIdx.x / kSkTeamThreads, tt = threadIdx.x % kSkTeamThreads;
    const int tw = tt >> 5, lane = threadIdx.x & 31;
    const int ncol = M + 1, wsz = s * ncol;
    const size_t tb = sketch_team_bytes(s, ncol);
    unsigned char* base_ptr = smem_raw + (size_t)team * tb;
    long long* Wi = reinterpret_cast<long long*>(base_ptr);
    double* Ys = reinterpret_cast<double*>(Wi + wsz);
    unsigned char* stg = reinterpret_cast<unsigned char*>(Ys + 32 * ncol);
    T* valW = reinterpret_cast<T*>(stg + (size_t)tw * kSkWarpStage * 8);
    int* colW = reinterpret_cast<int*>(stg + (size_t)kSkTeamWarps * kSkWarpStage * 8) +
                tw * kSkWarpStage;
    uint16_t* skS = reinterpret_cast<uint16_t*>(stg + (size_t)kSkTeamWarps * kSkWarpStage * 12);
    int* Fk = reinterpret_cast<int*>(skS + 32 * kMaxZeta);
    int* stk = Fk + ncol;                    // bit 0: column has values, bit 1: non-finite
    // (entry, column) of the flat index q = z (M + 1) + k of a row's scatter pairs
    __shared__ int zk[kMaxZeta * (kMaxM + 1)];
    const int per_row = zeta * ncol;
    for (int q = threadIdx.x; q < per_row; q += blockDim.x) zk[q] = ((q / ncol) << 8) | (q % ncol);
    for (int i = tt; i < wsz; i += kSkTeamThreads) Wi[i] = 0;
    for (int k = tt; k < ncol; k += kSkTeamThreads) {
        Fk[k] = 0;
        stk[k] = 0;
    }
    __syncthreads();
    int flag = 0;
    const int nent = kSkRowsPerWarp * M;
    const long long ntiles = ((long long)n + 31) / 32;
    for (long long tile = (long long)blockIdx.x * nteams + team; tile < ntiles;
         tile += (long long)gridDim.x * nteams) {
        const int row0 = (int)(tile * 32);
        const int cnt = min(32, n - row0);
        const int r0 = row0 + tw * kSkRowsPerWarp;
        const int wcnt = max(0, min(kSkRowsPerWarp, n - r0));
        // (a) this warp's rows
        int rs = 0, re = 0;
        if (lane < wcnt) {
            rs = max(0, min(__ldg(rowptr + r0 + lane), nnz));
            re = max(rs, min(__ldg(rowptr + r0 + lane + 1), nnz));
            sketch_column_packed(r0 + lane, s, zeta, seed,
                                 skS + (tw * kSkRowsPerWarp + lane) * kMaxZeta);
        }
        const int e0 = __shfl_sync(0xffffffffu, rs, 0);
        const int e1 = max(e0, __shfl_sync(0xffffffffu, re, max(wcnt - 1, 0)));
        const bool staged = e1 - e0 <= kSkWarpStage;
        if (staged) {
            for (int e = e0 + lane; e < e1; e += 32) {
                colW[e - e0] = __ldg(colind + e);
                valW[e - e0] = __ldg(val + e);
            }
        }
        if (lane < kSkRowsPerWarp)
            Ys[(tw * kSkRowsPerWarp + lane) * ncol + M] = lane < wcnt ? __ldg(b + r0 + lane) : 0.0;
        __syncwarp();
        // (b) Y[:, 0:M] = A X on the warp's rows, kSkU entries per lane at a time
        // (the loop is uniform over the warp: the shuffles need every lane)
        for (int eb0 = 0; eb0 < nent; eb0 += kSkU * 32) {
            const int eb = eb0 + lane;
            int rr[kSkU], kk[kSkU], st[kSkU], ln[kSkU];
            T acc[kSkU];
            int maxlen = 0;
#pragma unroll
            for (int u = 0; u < kSkU; ++u) {
                const int e = eb + 32 * u;
                const bool in = e < nent;
                const int r = in ? e / M : 0;
                rr[u] = r;
                kk[u] = in ? e - r * M : 0;
                const int a = __shfl_sync(0xffffffffu, rs, r);
                const int z = __shfl_sync(0xffffffffu, re, r);
                st[u] = a;
                ln[u] = (in && r < wcnt) ? z - a : 0;
                maxlen = max(maxlen, ln[u]);
                acc[u] = 0;
            }
            if (maxlen <= kSkFastRow) {
                T xv[kSkU][kSkFastRow], vv[kSkU][kSkFastRow];
#pragma unroll
                for (int t = 0; t < kSkFastRow; ++t) {
#pragma unroll
                    for (int u = 0; u < kSkU; ++u) {
                        xv[u][t] = 0;
                        vv[u][t] = 0;
                        if (t < ln[u]) {
                            const int e = st[u] + t;
                            const int c = staged ? colW[e - e0] : __ldg(colind + e);
                            if ((unsigned)c < (unsigned)n) {
                                vv[u][t] = staged ? valW[e - e0] : __ldg(val + e);
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
                    for (int u = 0; u < kSkU; ++u)
                        if (t < ln[u]) acc[u] = fma(vv[u][t], xv[u][t], acc[u]);
                }
            } else {
                for (int t = 0; t < maxlen; ++t) {
#pragma unroll
                    for (int u = 0; u < kSkU; ++u) {
                        if (t < ln[u]) {
                            const int e = st[u] + t;
                            const int c = staged ? colW[e - e0] : __ldg(colind + e);
                            const T v = staged ? valW[e - e0] : __ldg(val + e);
                            if ((unsigned)c < (unsigned)n)
                                acc[u] = fma(v, (T)__ldg(X + (size_t)c * ldx + kk[u]), acc[u]);
                            else
                                flag = 1;
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kSkU; ++u)
                if (eb + 32 * u < nent)
                    Ys[(tw * kSkRowsPerWarp + rr[u]) * ncol + kk[u]] =
                        rr[u] < wcnt ? (double)acc[u] : 0.0;
        }
        team_sync(team);
        // (c) column scales and fixed-point values; warp tw owns columns tw, tw + 4, ...
        long long* Yq = reinterpret_cast<long long*>(Ys);
        for (int k = tw; k < ncol; k += kSkTeamWarps) {
            const double y = Ys[lane * ncol + k];
            const unsigned long long mx = warp_max_u64(
                lane < cnt ? ((unsigned long long)__double_as_longlong(y) & 0x7fffffffffffffffull)
                           : 0ull);
            const bool nonfinite = mx >= 0x7ff0000000000000ull;
            const bool use = mx != 0 && !nonfinite;
            const int has = stk[k] & 1;
            int F = Fk[k];
            if (use) {
                const int emax = (int)(mx >> 52) - 1023;          // mx < 2^(emax + 1)
                const int Fn = (kSkValueBits - 1) - emax;
                if (!has) {
                    F = Fn;
                } else if (Fn < F) {
                    const int d = F - Fn;
                    for (int q = lane; q < s; q += 32)
                        Wi[q * ncol + k] = shift_round(Wi[q * ncol + k], d);
                    F = Fn;
                }
            }
            Yq[lane * ncol + k] = (use && lane < cnt) ? quantize(y, F) : 0;
            __syncwarp();
            if (lane == 0) {
                Fk[k] = F;
                stk[k] |= (use ? 1 : 0) | (nonfinite ? 2 : 0);
            }
        }
        team_sync(team);
        // (d) W += S[:, r] Yq[r, :] for the tile's rows (integer atomics); the
        // (row, sketch entry, column) triples are walked with the (entry,
        // column) of each flat index taken from the block's table zk.
        {
            int r = 0, q = tt;
            while (q >= per_row) {
                q -= per_row;
                ++r;
            }
            for (; r < cnt;) {
                const int t = zk[q];
                const int z = t >> 8, k = t & 0xff;
                const long long v = Yq[r * ncol + k];
                if (v != 0) {
                    const unsigned e = skS[r * kMaxZeta + z];
                    atomicAdd(reinterpret_cast<unsigned long long*>(&Wi[(int)(e & 0x7fff) * ncol + k]),
                              (unsigned long long)((e & 0x8000) ? -v : v));
                }
                q += kSkTeamThreads;
                while (q >= per_row) {
                    q -= per_row;
                    ++r;
                }
            }
        }
        team_sync(team);
    }
    if (flag) atomicOr(bad, 1);
    __syncthreads();
    double* out = partial + (size_t)blockIdx.x * wsz;
    for (int i = threadIdx.x; i < wsz; i += blockDim.x) {
        const int k = i % ncol;
        double acc = 0.0;
        bool nan = false;
        for (int t = 0; t < nteams; ++t) {
            const unsigned char* tp = smem_raw + (size_t)t * tb;
            const long long* Wt = reinterpret_cast<const long long*>(tp);
            const int* Ft = reinterpret_cast<const int*>(tp + 8 * (size_t)wsz + 8 * 32 * (size_t)ncol +
                                                         (size_t)kSkTeamWarps * kSkWarpStage * 12 +
                                                         2 * 32 * (size_t)kMaxZeta);
            const int st = Ft[ncol + k];
            nan |= (st & 2) != 0;
            if (st & 1) acc += scalbn((double)Wt[i], -Ft[k]);
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

// Blocks of the sketch kernel: one per SM, more when needed so that no team
// takes more than kSkMaxTiles tiles of 32 rows (its accumulators stay below
// 2^63), never more than the tiles need.
int sketch_grid(int n, int s, int M) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int teams = sketch_teams(s, M + 1);
    const long long ntiles = ((long long)n + 31) / 32;
    long long nblk = std::min<long long>(sms, (ntiles + teams - 1) / teams);
    const long long need = (ntiles + (long long)kSkMaxTiles * teams - 1) / ((long long)kSkMaxTiles * teams);
    if (need > nblk) nblk = need;
    return nblk > 0 ? (int)nblk : 1;
}

size_t sketch_partial_doubles(int n, int s, int M) {
    return (size_t)sketch_grid(n, s, M) * s * (M + 1);
}

template <typename T, typename XT>
static void launch_sketch_impl(const int* rowptr, const int* colind, const T* val, const XT* X,
                               int ldx, const double* b, int n, int nnz, int M, int s, int zeta,
                               uint64_t seed, double* partial, int nblk, double* W, int* bad,
                               cudaStream_t st) {
    const int wsz = s * (M + 1);
    // Teams for these columns (at least as many as the grid was sized for,
    // so that no team takes more than kSkMaxTiles tiles).
    const int teams = sketch_teams(s, M + 1);
    const size_t smem = (size_t)teams * sketch_team_bytes(s, M + 1);
    // The attribute is per device: set it on every call (cheap, host only).
    cudaFuncSetAttribute(sketch_block_kernel<T, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    sketch_block_kernel<T, XT><<<nblk, teams * kSkTeamThreads, smem, st>>>(
        rowptr, colind, val, X, ldx, b, n, nnz, M, s, zeta, seed, partial, bad);
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
