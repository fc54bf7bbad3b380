// Device helpers shared by the seqaccel kernels (sm_103a).
//
// Reductions are deterministic: every partial sum has a fixed owner and is
// combined in a fixed order (warp butterfly, then warps in index order, then
// blocks in index order by the last block to finish), so results do not
// depend on scheduling and repeat bit for bit from run to run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sa {

constexpr int kWarp = 32;
constexpr int kMaxBasis = 65;     // GMRES restart <= 64 -> at most 65 basis vectors
constexpr int kMaxRestart = 64;
constexpr int kMaxM = 31;         // history length (M + 1 <= 32 lanes in the sketch kernel)
constexpr int kMaxS = 128;        // sketch rows
constexpr int kMaxZeta = 16;
constexpr int kKernelsPerStep = 4; // SpMV, first-pass dots, CGS pass 2, CGS pass 3
constexpr int kStreamBlock = 384; // threads per block of the streaming kernels (one block per SM)
constexpr int kTileChunks = 8;    // CSR entries of a 32-row tile loaded up front: 8 x 32
constexpr int kTileStage = 2 * kTileChunks * 32;   // shared staging per warp (values, x)
constexpr int kChebTab = 2 + 2 * 32;   // Chebyshev coefficient table (degree <= 32)

// Device-side copy of the per-call arguments.  The CUDA graphs of a context
// take a pointer to this struct, so one captured graph serves every call.
struct DevArgs {
    const int* rowptr;
    const int* colind;
    const double* val64;
    const float* val32;
    const double* b;
    double* x;          // FP64 iterate (GMRES/CG on the FP64 system, or the
                        // refinement iterate in mixed precision)
    void* d;            // inner correction vector (mixed precision, FP32)
    const float* rhs32; // inner right-hand side (mixed precision)
    const int* sell_off;   // SELL-32 copy of the matrix used inside GMRES cycles
    const int* sell_col;   // (slice offsets, column indices, values; NULL: use CSR)
    const void* sell_val;
    int n;
    int nnz;
    int max_iters;
    int sell_w;         // every SELL slice has this width (offsets = 32 w s); 0: read them
    int sell_keep;      // 1: load the SELL arrays with L2 evict-last priority (they fit in L2)
    int pad1;
    double tol;         // relative tolerance of this solve
};

// State of one restarted GMRES / CG solve, kept on the device.
struct KState {
    double sigma[kMaxBasis];        // stored basis column k = v_k / sigma_k
    double h1[kMaxBasis];           // first CGS pass coefficients
    double h2[kMaxBasis];           // second CGS pass coefficients
    double c1[kMaxBasis];           // sigma_k * h1_k (applied to stored columns)
    double c2[kMaxBasis];           // sigma_k * h2_k
    double H[kMaxBasis * kMaxRestart];  // rotated Hessenberg, column-major (ld kMaxBasis)
    double cs[kMaxRestart];
    double sn[kMaxRestart];
    double g[kMaxBasis];
    double cy[kMaxBasis];           // sigma_k * y_k for the basis update
    double beta;                    // ||r|| at the last cycle start
    double bnorm;                   // ||b||
    double target;                  // tol * ||b||
    double first_relres;            // relative residual of the starting vector
    int cycle_over;                 // 1: Arnoldi steps of this cycle are finished
    int finished;                   // 1: the solve is over (see status)
    int jdone;                      // Arnoldi steps in the current cycle
    int iters;                      // iterations of this solve
    int status;                     // seq_status
    int bad_index;                  // a CSR column index fell outside [0, n)
    int last_jdone;                 // Arnoldi steps of the cycle that just ended
    int pad1;
    unsigned counter[8];            // last-block counters, one per kernel kind
};

// Loads with an L2 eviction priority (createpolicy + ld.global.nc.L2::cache_hint):
// evict_last keeps a matrix that is read again by the next kernels (the
// sweeps and products of one Arnoldi step) resident in L2 while vectors
// stream past it.
__device__ __forceinline__ uint64_t l2_policy(bool keep) {
    uint64_t p;
    if (keep)
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else
        asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int ld_hint(const int* ptr, uint64_t pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_hint(const float* ptr, uint64_t pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_hint(const double* ptr, uint64_t pol) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum K per-thread values over the block; on return red[k] (shared, >= K
// entries) holds the block total of value k.  blockDim.x is a multiple of 32.
template <typename T, int K>
__device__ __forceinline__ void block_sum(T (&v)[K], int nk, T* red, T* scratch /* nwarps*K */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (k < nk) {
            T s = warp_sum(v[k]);
            if (lane == 0) scratch[warp * K + k] = s;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        T s = scratch[k];
        for (int w = 1; w < nw; ++w) s += scratch[w * K + k];
        red[k] = s;
    }
    __syncthreads();
}

// Returns true (in every thread) in the block that arrives last.  Each block
// must have written its partials (by any of its threads) before calling.
__device__ __forceinline__ bool last_block_arrive(unsigned* counter) {
    __shared__ int am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last != 0;
}

// Sum partial[blk * stride + k] over blocks 0..nblk-1 in index order, for
// k < nk, by the threads of one block (one k per thread, four interleaved
// accumulators combined in a fixed order).  Reads bypass L1.
template <typename T>
__device__ __forceinline__ T sum_over_blocks(const T* partial, int nblk, int stride, int k) {
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int b = 0;
    for (; b + 3 < nblk; b += 4) {
        a0 += __ldcg(partial + (size_t)(b + 0) * stride + k);
        a1 += __ldcg(partial + (size_t)(b + 1) * stride + k);
        a2 += __ldcg(partial + (size_t)(b + 2) * stride + k);
        a3 += __ldcg(partial + (size_t)(b + 3) * stride + k);
    }
    for (; b < nblk; ++b) a0 += __ldcg(partial + (size_t)b * stride + k);
    return (a0 + a1) + (a2 + a3);
}

// SplitMix64 output finaliser (Steele, Lea, Flood 2014; variant-13 mixer).
// ||r|| / ||b||, or ||r|| itself when b = 0 (the relative residual is then
// undefined; x = 0 is the exact solution and has residual 0).
__host__ __device__ __forceinline__ double rel_residual(double rnorm, double bnorm) {
    return bnorm > 0.0 ? rnorm / bnorm : rnorm;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Rows [lo, hi) owned by block `blk` when n rows are split into `nblk`
// contiguous chunks whose length is a multiple of 32.
__device__ __forceinline__ void block_rows(int n, int nblk, int blk, int& lo, int& hi) {
    int chunk = (n + nblk - 1) / nblk;
    chunk = (chunk + 31) & ~31;
    lo = min(n, blk * chunk);
    hi = min(n, lo + chunk);
}

// (A x)[row] for the 32 consecutive rows r0 .. r0+31 of one warp, lane l
// returning row r0 + l (0 past the end).  The tile's nonzeros [e0, e1) are
// loaded with coalesced reads, all of them up front when they fit in
// kTileChunks x 32 entries (the usual case: stencil rows hold ~5 entries),
// otherwise chunk by chunk.  Products are staged in shared memory (sprod:
// kTileChunks * 32 entries per warp) and each lane sums the entries of its own
// row in CSR order.  Column indices outside [0, n) contribute 0 and raise *bad.
// XL2: read x through L2 only (x is written by other thread blocks of the
// same launch).
template <typename Acc, typename VT, typename XT, bool XL2 = false>
__device__ __forceinline__ Acc warp_tile_spmv(const int* __restrict__ rowptr,
                                              const int* __restrict__ colind,
                                              const VT* __restrict__ val,
                                              const XT* __restrict__ x, int n, int nnz,
                                              int r0, Acc* sprod, int* bad) {
    const int lane = threadIdx.x & 31;
    const int row = r0 + lane;
    int rs = 0, re = 0;
    if (row < n) {
        rs = __ldg(rowptr + row);
        re = __ldg(rowptr + row + 1);
        rs = max(0, min(rs, nnz));
        re = max(rs, min(re, nnz));
    }
    const int last = min(31, n - 1 - r0);
    const int e0 = __shfl_sync(0xffffffffu, rs, 0);
    const int e1 = max(e0, __shfl_sync(0xffffffffu, re, last));
    Acc acc = 0;
    int flag = 0;
    if (e1 - e0 <= kTileChunks * 32) {
        int cc[kTileChunks];
        VT vv[kTileChunks];
#pragma unroll
        for (int q = 0; q < kTileChunks; ++q) {
            const int e = e0 + q * 32 + lane;
            cc[q] = e < e1 ? __ldg(colind + e) : 0;
        }
#pragma unroll
        for (int q = 0; q < kTileChunks; ++q) {
            const int e = e0 + q * 32 + lane;
            vv[q] = e < e1 ? __ldg(val + e) : (VT)0;
        }
#pragma unroll
        for (int q = 0; q < kTileChunks; ++q) {
            const int e = e0 + q * 32 + lane;
            Acc prod = 0;
            if (e < e1) {
                if ((unsigned)cc[q] < (unsigned)n)
                    prod = (Acc)vv[q] * (Acc)(XL2 ? __ldcg(x + cc[q]) : x[cc[q]]);
                else
                    flag = 1;
            }
            sprod[q * 32 + lane] = prod;
        }
        __syncwarp();
        const int lo = max(rs, e0), hi = min(re, e1);
        for (int e = lo; e < hi; ++e) acc += sprod[e - e0];
        __syncwarp();
    } else {
        for (int base = e0; base < e1; base += 32) {
            const int e = base + lane;
            Acc prod = 0;
            if (e < e1) {
                const int c = __ldg(colind + e);
                if ((unsigned)c < (unsigned)n)
                    prod = (Acc)__ldg(val + e) * (Acc)(XL2 ? __ldcg(x + c) : x[c]);
                else
                    flag = 1;
            }
            sprod[lane] = prod;
            __syncwarp();
            const int lo = max(rs, base), hi = min(re, base + 32);
            for (int k = lo; k < hi; ++k) acc += sprod[k - base];
            __syncwarp();
        }
    }
    if (flag) atomicOr(bad, 1);
    return acc;
}

// Software-pipelined warp tiles.  A tile's CSR row range is fetched one
// stage ahead of its column/value loads, which are fetched one stage ahead of
// the gathers and sums, so three tiles' loads are in flight per warp.
struct TileRows {
    int rs, re;     // this lane's row range, clamped to [0, nnz]
    int e0, e1;     // the tile's entry range
};

__device__ __forceinline__ TileRows tile_rows(const int* __restrict__ rowptr, int n, int nnz,
                                              int r0, int hi) {
    const int lane = threadIdx.x & 31;
    const int row = r0 + lane;
    TileRows t;
    t.rs = t.re = 0;
    if (r0 < hi && row < n) {
        t.rs = max(0, min(__ldg(rowptr + row), nnz));
        t.re = max(t.rs, min(__ldg(rowptr + row + 1), nnz));
    }
    return t;
}

__device__ __forceinline__ void tile_span(TileRows& t, int n, int r0) {
    const int last = max(0, min(31, n - 1 - r0));
    t.e0 = __shfl_sync(0xffffffffu, t.rs, 0);
    t.e1 = max(t.e0, __shfl_sync(0xffffffffu, t.re, last));
}

template <typename VT>
struct TileData {
    int cc[kTileChunks];
    VT vv[kTileChunks];
};

template <typename VT>
__device__ __forceinline__ void tile_load(const int* __restrict__ colind, const VT* __restrict__ val,
                                          const TileRows& t, TileData<VT>& d) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < kTileChunks; ++q) {
        const int e = t.e0 + q * 32 + lane;
        d.cc[q] = e < t.e1 ? __ldg(colind + e) : 0;
    }
#pragma unroll
    for (int q = 0; q < kTileChunks; ++q) {
        const int e = t.e0 + q * 32 + lane;
        d.vv[q] = e < t.e1 ? __ldg(val + e) : (VT)0;
    }
}

// Gathers, products and per-row sums of a tile whose loads are in `d`; rows
// with more than kTileChunks x 32 entries in the tile fall back to a chunked
// loop over the CSR arrays.
template <typename Acc, typename VT, typename XT>
__device__ __forceinline__ Acc tile_finish(const int* __restrict__ colind,
                                           const VT* __restrict__ val, const XT* __restrict__ x,
                                           int n, const TileRows& t, const TileData<VT>& d,
                                           Acc* sprod, int* bad) {
    const int lane = threadIdx.x & 31;
    Acc acc = 0;
    int flag = 0;
    if (t.e1 - t.e0 <= kTileChunks * 32) {
        // Stage (value, x[col]) pairs; the row's lane then forms its sum with
        // one fused multiply-add per entry, in CSR order.
        Acc* sval = sprod;
        Acc* sx = sprod + kTileChunks * 32;
#pragma unroll
        for (int q = 0; q < kTileChunks; ++q) {
            const int e = t.e0 + q * 32 + lane;
            Acc xv = 0;
            if (e < t.e1) {
                if ((unsigned)d.cc[q] < (unsigned)n)
                    xv = (Acc)x[d.cc[q]];
                else
                    flag = 1;
            }
            sval[q * 32 + lane] = (Acc)d.vv[q];
            sx[q * 32 + lane] = xv;
        }
        __syncwarp();
        const int lo = max(t.rs, t.e0), hi = min(t.re, t.e1);
        for (int e = lo; e < hi; ++e) acc = fma(sval[e - t.e0], sx[e - t.e0], acc);
        __syncwarp();
    } else {
        for (int base = t.e0; base < t.e1; base += 32) {
            const int e = base + lane;
            Acc prod = 0;
            if (e < t.e1) {
                const int c = __ldg(colind + e);
                if ((unsigned)c < (unsigned)n)
                    prod = (Acc)__ldg(val + e) * (Acc)x[c];
                else
                    flag = 1;
            }
            sprod[lane] = prod;
            __syncwarp();
            const int lo = max(t.rs, base), hi = min(t.re, base + 32);
            for (int k = lo; k < hi; ++k) acc += sprod[k - base];
            __syncwarp();
        }
    }
    if (flag) atomicOr(bad, 1);
    return acc;
}

// Warp reduce-scatter of K <= 32 per-lane values: returns, in lane l, the
// warp-wide sum of value (l % K).  Halves of the lane range are folded while
// they exceed K, then a recursive-halving exchange leaves one value per lane
// (a fixed pattern: the result does not depend on scheduling).
template <typename T, int K>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[K]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 16; s >= K; s >>= 1) {
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], s);
    }
#pragma unroll
    for (int s = K / 2; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            const T send = upper ? v[i] : v[i + s];
            const T keep = upper ? v[i + s] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0];
}

// Last block: dst[k] = sum over blocks b of partial[b * stride + k] for
// k < nk.  Warp w handles k = w, w + nw, ...; lane l adds blocks l, l+32, ...
// in order, then the warp butterfly.  Ends with __syncthreads().
template <typename T>
__device__ __forceinline__ void reduce_blocks(const T* partial, int nblk, int stride, int nk,
                                              double* dst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < nk; k += nw) {
        T a = 0;
        for (int b = lane; b < nblk; b += 32) a += __ldcg(partial + (size_t)b * stride + k);
        a = warp_sum(a);
        if (lane == 0) dst[k] = (double)a;
    }
    __syncthreads();
}

}  // namespace sa
