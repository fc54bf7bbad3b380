// seq_sketch_block_noalloc: the sketched block W = S [A X | b] computed
// without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// need W -- code inside a host callback or a real-time loop that must not
// block in the allocator (cudaMalloc may synchronise the device), and hosts
// that give the GPU's memory to their own pool or fix the library's memory
// budget up front, so that an allocation made later would fail.  They pass
// their own inputs and output; the only scratch the kernels use (one partial
// block of W per thread block) lives in a file-scope device array of fixed
// size.
//
// Limits and sharing:
//   * s * (M + 1) <= kNoAllocSlots (4096: s <= 128 with M <= 31), zeta <= 16;
//     larger requests return SEQ_EINVAL before any GPU work.
//   * The scratch array holds kNoAllocBlocks x (kNoAllocSlots + 1) + 1
//     doubles (about 5 MB); every GPU that loads the library keeps it until
//     the process exits.
//   * Every call uses the same array: calls that overlap on the GPU (for
//     example on two streams at once) race on it.  It keeps the last call's
//     contents; each call writes every partial slot it later reads and
//     clears the error word first, so nothing else needs clearing.
//   * The first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before any stream capture.
//   * Each call ends by copying the column-index flag to the host and
//     synchronising the caller's stream.
//
// The sketch is the same sparse-sign S as everywhere in the library (column
// j: zeta distinct rows from SplitMix64 outputs 256 j + c + 1, row =
// ((h >> 32) s) >> 32, sign = bit 0 of h, entries +-1/sqrt(zeta)), generated
// here on the fly, so no sketch buffer is needed either.
#include <mutex>

#include "../../include/seqaccel.h"
#include "common.cuh"

namespace {

constexpr int kNoAllocSlots = 4096;   // s * (M + 1) at most
constexpr int kNoAllocBlocks = 152;   // thread blocks (one partial each)
constexpr int kNoAllocThreads = 128;  // 4 warps
constexpr int kNoAllocWarps = kNoAllocThreads / 32;

// Partials of every block, then one word for the column-index flag.
__device__ __align__(256) double g_noalloc_scratch[kNoAllocBlocks * (kNoAllocSlots + 1) + 1];

std::mutex g_mu;
double* g_scratch_ptr[128] = {nullptr};

// Sketch entries of column (row of A) j, packed as row | sign << 15.
__device__ __forceinline__ void sketch_column(int j, int s, int zeta, uint64_t seed,
                                              uint16_t* out) {
    int rows[sa::kMaxZeta];
    int cnt = 0;
    for (int c = 0; c < 256 && cnt < zeta; ++c) {
        const uint64_t h = sa::mix64(seed + ((uint64_t)j * 256ull + (uint64_t)(c + 1)) *
                                                0x9E3779B97F4A7C15ull);
        const int q = (int)(((h >> 32) * (uint64_t)s) >> 32);
        bool dup = false;
        for (int k = 0; k < cnt; ++k) dup |= rows[k] == q;
        if (!dup) {
            rows[cnt] = q;
            out[cnt] = (uint16_t)(q | ((h & 1ull) ? 0x8000 : 0));
            ++cnt;
        }
    }
    for (int q = 0; cnt < zeta && q < s; ++q) {
        bool used = false;
        for (int k = 0; k < cnt; ++k) used |= rows[k] == q;
        if (!used) {
            rows[cnt] = q;
            out[cnt] = (uint16_t)q;
            ++cnt;
        }
    }
}

// Per block: rows [lo, hi) in batches of 32 per warp.  Lane l first builds
// the sketch column of row base + l in shared memory, then the warp walks the
// batch row by row with lane k owning column k of Y = [A X | b] and of the
// warp's private copy of W (fixed order, no atomics).  The block's warps are
// summed in warp order into the block's slot of the scratch array.
__global__ void __launch_bounds__(kNoAllocThreads)
noalloc_sketch_kernel(const int* __restrict__ rowptr, const int* __restrict__ colind,
                      const double* __restrict__ val, const double* __restrict__ X, int ldx,
                      const double* __restrict__ b, int n, int nnz, int M, int s, int zeta,
                      uint64_t seed, double* __restrict__ partial, int* bad) {
    extern __shared__ double wsm[];                       // kNoAllocWarps * s * (M+1)
    __shared__ uint16_t sks[kNoAllocWarps][32][sa::kMaxZeta];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncol = M + 1, wsz = s * ncol;
    double* Ww = wsm + warp * wsz;
    for (int i = lane; i < wsz; i += 32) Ww[i] = 0.0;
    int lo, hi;
    sa::block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    double bb = 0.0;
    int flag = 0;
    for (int base = lo + warp * 32; base < hi; base += kNoAllocWarps * 32) {
        if (base + lane < hi) sketch_column(base + lane, s, zeta, seed, sks[warp][lane]);
        __syncwarp();
        const int cnt = min(32, hi - base);
        for (int u = 0; u < cnt; ++u) {
            const int r = base + u;
            double y = 0.0;
            if (lane < M) {
                const int rs = max(0, min(__ldg(rowptr + r), nnz));
                const int re = max(rs, min(__ldg(rowptr + r + 1), nnz));
                for (int e = rs; e < re; ++e) {
                    const int c = __ldg(colind + e);
                    if ((unsigned)c < (unsigned)n)
                        y = fma(__ldg(val + e), __ldg(X + (size_t)c * ldx + lane), y);
                    else
                        flag = 1;
                }
            } else if (lane == M) {
                y = __ldg(b + r);
                bb = fma(y, y, bb);
            }
            if (lane < ncol) {
                for (int k = 0; k < zeta; ++k) {
                    const unsigned e = sks[warp][u][k];
                    double* dst = Ww + (e & 0x7fff) * ncol + lane;
                    *dst = (e & 0x8000) ? *dst - y : *dst + y;
                }
            }
        }
        __syncwarp();
    }
    if (flag) atomicOr(bad, 1);
    __syncthreads();
    double* out = partial + (size_t)blockIdx.x * (kNoAllocSlots + 1);
    for (int i = threadIdx.x; i < wsz; i += blockDim.x) {
        double acc = wsm[i];
        for (int w = 1; w < kNoAllocWarps; ++w) acc += wsm[w * wsz + i];
        out[i] = acc;
    }
    __shared__ double bbs[kNoAllocWarps];
    if (lane == M) bbs[warp] = bb;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNoAllocWarps; ++w) t += bbs[w];
        out[kNoAllocSlots] = t;
    }
}

// W[i] = sum over blocks (in block order) of partial[blk][i] / sqrt(zeta).
__global__ void noalloc_reduce_kernel(const double* __restrict__ partial, int nblk, int wsz,
                                      double inv_sqrt_zeta, double* __restrict__ W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= wsz) return;
    double acc = 0.0;
    for (int blk = 0; blk < nblk; ++blk) acc += partial[(size_t)blk * (kNoAllocSlots + 1) + i];
    W[i] = acc * inv_sqrt_zeta;
}

// Device address of the scratch array for the current device (looked up once
// per device, with that device current).
int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return SEQ_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SEQ_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return SEQ_OK;
}

// Column-index errors are reported through the scratch array's last word
// (cleared by each call) and read back after the call.
__global__ void noalloc_clear_flag(int* flag) { *flag = 0; }

}  // namespace

extern "C" int seq_sketch_block_noalloc(int32_t n, int32_t nnz, const int32_t* rowptr,
                                        const int32_t* colind, const double* values,
                                        const double* X, int32_t ldx, int32_t M,
                                        const double* b, int32_t s, int32_t zeta, uint64_t seed,
                                        double* W_dev, void* cuda_stream) {
    if (n <= 0 || nnz < 0 || !rowptr || (nnz > 0 && (!colind || !values)) || !X || !b || !W_dev)
        return SEQ_EINVAL;
    if (M < 1 || M > sa::kMaxM || ldx < M || s < 1 || zeta < 1 || zeta > s ||
        zeta > sa::kMaxZeta || (long long)s * (M + 1) > kNoAllocSlots || s > 32767)
        return SEQ_EINVAL;
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != SEQ_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nblk = (n + 127) / 128;
    if (nblk > kNoAllocBlocks) nblk = kNoAllocBlocks;
    if (nblk > sms && sms > 0) nblk = sms;
    const int wsz = s * (M + 1);
    const size_t smem = sizeof(double) * (size_t)kNoAllocWarps * wsz;
    if (cudaFuncSetAttribute(noalloc_sketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return SEQ_ECUDA;
    }
    int* flag = reinterpret_cast<int*>(scratch + (size_t)kNoAllocBlocks * (kNoAllocSlots + 1));
    noalloc_clear_flag<<<1, 1, 0, st>>>(flag);
    noalloc_sketch_kernel<<<nblk, kNoAllocThreads, smem, st>>>(rowptr, colind, values, X, ldx, b, n,
                                                              nnz, M, s, zeta, seed, scratch, flag);
    noalloc_reduce_kernel<<<(wsz + 127) / 128, 128, 0, st>>>(scratch, nblk, wsz,
                                                            1.0 / sqrt((double)zeta), W_dev);
    if (cudaGetLastError() != cudaSuccess) return SEQ_ECUDA;
    int hflag = 0;
    if (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SEQ_ECUDA;
    return hflag ? SEQ_EINVAL : SEQ_OK;
}
