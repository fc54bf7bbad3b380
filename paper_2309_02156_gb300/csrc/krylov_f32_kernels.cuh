// FP32 Arnoldi kernels of the mixed-precision inner solves (part of the
// Krylov kernel templates; included by krylov_kernels.cuh after the SELL
// product, the reductions and the Arnoldi finish step they build on).
#pragma once
// (Textually included inside namespace sa.)

// ---------------------------------------------------------------------------
// FP32 CGS kernels (inner solves of the mixed forms).  In FP32 the passes are
// bound by memory, not by arithmetic, so they are organised for bytes in
// flight: each thread owns VW consecutive rows and reads them from every
// basis column with one VW-wide vector load (a warp reads 32 VW 4-byte values
// of a column per instruction), U vectors per iteration; the row-parallel
// layout replaces the column-segment dot kernel of FP64.  Rows past the last
// full vector of the block's range are handled one per thread.  Reductions:
// per-thread partials over its rows, warp reduce-scatter, warps in order,
// blocks in order in the last block (deterministic).  The basis columns are
// read with streaming loads (ld.global.cs, evict-first in L2): each pass
// reads them once, so they leave L2 before the matrix does and the product
// of the next Arnoldi step finds the matrix there.
template <int VW> struct F32x;
template <> struct F32x<1> {
    using type = float;
    __device__ static void get(const float* p, float (&o)[1]) { o[0] = *p; }
    __device__ static void stream(const float* p, float (&o)[1]) { o[0] = __ldcs(p); }
    __device__ static void put(float* p, const float (&o)[1]) { *p = o[0]; }
};
template <> struct F32x<2> {
    using type = float2;
    __device__ static void get(const float* p, float (&o)[2]) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        o[0] = v.x; o[1] = v.y;
    }
    __device__ static void stream(const float* p, float (&o)[2]) {
        const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
    __device__ static void put(float* p, const float (&o)[2]) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    }
};
template <> struct F32x<4> {
    using type = float4;
    __device__ static void get(const float* p, float (&o)[4]) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ static void stream(const float* p, float (&o)[4]) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ static void put(float* p, const float (&o)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
// Per thread and iteration about 64 floats (256 bytes) in flight: one block
// of 12 warps per SM (the partial sums of NK columns need the registers) has
// to hide the memory latency with bytes per thread, not with warps.
template <int NK> struct F32Shape {
    static constexpr int VW = NK >= 32 ? 1 : (NK >= 20 ? 2 : 4);
    static constexpr int per = (NK + 1) * VW;                 // floats loaded per vector
    static constexpr int U0 = per >= 64 ? 1 : (64 + per - 1) / per;
    static constexpr int U = (U0 > 1 && U0 * per > 96) ? U0 - 1 : U0;
};

// MODE 0: part[k] = sum v_k w (first CGS pass, h1).
// MODE 1: r = w - sum_k v_k c1_k, w = r, part[k] = sum v_k r (fused pass 2).
// MODE 2: r = w - sum_k v_k c2_k, v_{j+1} = r, part[0] = sum r^2 (pass 3).
template <int NK, int MODE>
__device__ __forceinline__ void f32_rows(const float* __restrict__ V, size_t ldv, float* w,
                                         float* vout, const float* cf, int lo, int hi,
                                         float (&part)[NK]) {
    constexpr int VW = F32Shape<NK>::VW, U = F32Shape<NK>::U;
    using X = F32x<VW>;
    const int bd = blockDim.x;
    const int hv = lo + ((hi - lo) / VW) * VW;               // end of the full vectors
    for (int i0 = lo + threadIdx.x * VW; i0 < hv; i0 += U * bd * VW) {
        float vv[U][NK][VW];
        float r[U][VW];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = min(i0 + u * bd * VW, hv - VW);
#pragma unroll
            for (int k = 0; k < NK; ++k) X::stream(V + (size_t)k * ldv + i, vv[u][k]);
            X::get(w + i, r[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * bd * VW;
            if (i >= hv) continue;
            if constexpr (MODE == 0) {
#pragma unroll
                for (int k = 0; k < NK; ++k)
#pragma unroll
                    for (int e = 0; e < VW; ++e) part[k] = fmaf(vv[u][k][e], r[u][e], part[k]);
            } else {
#pragma unroll
                for (int e = 0; e < VW; ++e)
#pragma unroll
                    for (int k = 0; k < NK; ++k) r[u][e] = fmaf(-vv[u][k][e], cf[k], r[u][e]);
                if constexpr (MODE == 1) {
                    X::put(w + i, r[u]);
#pragma unroll
                    for (int k = 0; k < NK; ++k)
#pragma unroll
                        for (int e = 0; e < VW; ++e) part[k] = fmaf(vv[u][k][e], r[u][e], part[k]);
                } else {
                    X::put(vout + i, r[u]);
#pragma unroll
                    for (int e = 0; e < VW; ++e) part[0] = fmaf(r[u][e], r[u][e], part[0]);
                }
            }
        }
    }
    for (int i = hv + threadIdx.x; i < hi; i += bd) {        // ragged tail, one row per thread
        float rr = w[i];
        if constexpr (MODE == 0) {
#pragma unroll
            for (int k = 0; k < NK; ++k) part[k] = fmaf(V[(size_t)k * ldv + i], rr, part[k]);
        } else {
            float vk[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) vk[k] = V[(size_t)k * ldv + i];
#pragma unroll
            for (int k = 0; k < NK; ++k) rr = fmaf(-vk[k], cf[k], rr);
            if constexpr (MODE == 1) {
                w[i] = rr;
#pragma unroll
                for (int k = 0; k < NK; ++k) part[k] = fmaf(vk[k], rr, part[k]);
            } else {
                vout[i] = rr;
                part[0] = fmaf(rr, rr, part[0]);
            }
        }
    }
}

// FP32 w = A v_j (or A src, the preconditioned vector) fused with the first
// CGS pass h1 = V^T w: each block forms w on its own rows (SELL-32 product,
// warp per slice), then, after a block barrier, reads those rows back (from
// cache) together with the basis columns.  Saves a launch and a pass over w.
template <int NK>
__global__ void __launch_bounds__(kStreamBlock, 1)
f32_spmv_dot_kernel(const DevArgs* __restrict__ a, KState* ks, const float* __restrict__ V,
                    size_t ldv, float* __restrict__ w, float* partial, int j, const float* src) {
    __shared__ float wsum[kWarps * NK];
    const int over = ks->cycle_over;
    const float sig = src ? 1.f : (float)ks->sigma[j];
    if (over) return;
    const int n = a->n;
    const float* vj = src ? src : V + (size_t)j * ldv;
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    if (a->sell_off) {
        sell_spmv_rows<float>(a->sell_off, a->sell_col, reinterpret_cast<const float*>(a->sell_val),
                              vj, n, lo, hi, sig, w, kWarps, a->sell_w, a->sell_keep,
                              &ks->bad_index);
    } else {                                      // no SELL copy: CSR, one row per thread
        const float* val = a->val32;
        int flag = 0;
        for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) {
            float acc = 0.f;
            for (int e = a->rowptr[r]; e < a->rowptr[r + 1]; ++e) {
                const int c = a->colind[e];
                if ((unsigned)c < (unsigned)n) acc = fmaf(val[e], vj[c], acc);
                else flag = 1;
            }
            w[r] = acc * sig;
        }
        if (flag) atomicOr(&ks->bad_index, 1);
    }
    __syncthreads();
    float part[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) part[k] = 0.f;
    f32_rows<NK, 0>(V, ldv, w, nullptr, nullptr, lo, hi, part);
    block_columns<float, NK>(part, NK, wsum, partial + (size_t)blockIdx.x * kMaxBasis);
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

template <int NK>
__global__ void __launch_bounds__(kStreamBlock, 1)
f32_pass2_kernel(const DevArgs* __restrict__ a, KState* ks, const float* __restrict__ V, size_t ldv,
                 float* __restrict__ w, float* partial, int j) {
    __shared__ float cf[NK];
    __shared__ float wsum[kWarps * NK];
    // The end-of-cycle flag and the coefficients are loaded together (one
    // latency); every thread sees the same flag, so the return is uniform.
    const int over = ks->cycle_over;
    for (int k = threadIdx.x; k < NK; k += blockDim.x) cf[k] = (float)ks->c1[k];
    if (over) return;
    __syncthreads();
    int lo, hi;
    block_rows(a->n, gridDim.x, blockIdx.x, lo, hi);
    float part[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) part[k] = 0.f;
    f32_rows<NK, 1>(V, ldv, w, nullptr, cf, lo, hi, part);
    block_columns<float, NK>(part, NK, wsum, partial + (size_t)blockIdx.x * kMaxBasis);
    if (last_block_arrive(&ks->counter[CNT_PASS2])) {
        __shared__ double tot[NK];
        reduce_blocks(partial, gridDim.x, kMaxBasis, NK, tot);
        for (int k = threadIdx.x; k < NK; k += blockDim.x) {
            const double hk = ks->sigma[k] * tot[k];
            ks->h2[k] = hk;
            ks->c2[k] = ks->sigma[k] * hk;
        }
        if (threadIdx.x == 0) ks->counter[CNT_PASS2] = 0;
    }
}

template <int NK>
__global__ void __launch_bounds__(kStreamBlock, 1)
f32_pass3_kernel(const DevArgs* __restrict__ a, KState* ks, float* __restrict__ V, size_t ldv,
                 const float* __restrict__ w, float* partial, int j, int R) {
    __shared__ float cf[NK];
    __shared__ float scratch[kWarps];
    __shared__ float red[1];
    const int over = ks->cycle_over;
    for (int k = threadIdx.x; k < NK; k += blockDim.x) cf[k] = (float)ks->c2[k];
    if (over) return;
    __syncthreads();
    int lo, hi;
    block_rows(a->n, gridDim.x, blockIdx.x, lo, hi);
    float part[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) part[k] = 0.f;
    f32_rows<NK, 2>(V, ldv, const_cast<float*>(w), V + (size_t)(j + 1) * ldv, cf, lo, hi, part);
    float p1[1] = {part[0]};
    block_sum<float, 1>(p1, 1, red, scratch);
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
    if (last_block_arrive(&ks->counter[CNT_PASS3])) {
        if (threadIdx.x == 0) ks->counter[CNT_PASS3] = 0;
        arnoldi_finish(ks, a, j, R, partial, (int)gridDim.x);
    }
}
