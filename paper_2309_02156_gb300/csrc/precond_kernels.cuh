// Right-preconditioning kernels of the restarted GMRES (part of the Krylov
// kernel templates; included by krylov_kernels.cuh after the SELL product and
// the Arnoldi kernels it builds on).
#pragma once
// (Textually included inside namespace sa.)

// ---------------------------------------------------------------------------
// Right preconditioning (optional): GMRES runs on A M^{-1}, the cycle's
// correction is x += M^{-1} (V y), so the residual GMRES minimises and tests
// is the true one.  M^{-1} u = `sweeps` damped Jacobi sweeps on A z = u from
// z = 0:  z_1 = omega D^{-1} u,  z_{k+1} = z_k + omega D^{-1} (u - A z_k)
// (a fixed polynomial in D^{-1} A times D^{-1}).  Phase 0 kernels belong to an
// Arnoldi step (skipped once the cycle is over), phase 1 kernels to the basis
// update (skipped like the update).
__device__ __forceinline__ bool update_skipped(const KState* ks) {
    return (ks->status != ST_OK && ks->status != ST_NOT_CONVERGED) || ks->finished;
}
__device__ __forceinline__ bool precond_skipped(const KState* ks, int phase) {
    return phase == 0 ? ks->cycle_over != 0 : update_skipped(ks);
}

// dinv = 1 / diag(A) in the system's precision (1 where the diagonal is
// missing or zero).
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock)
diag_inv_kernel(const DevArgs* __restrict__ a, typename Sys::T* __restrict__ dinv) {
    using T = typename Sys::T;
    const T* val = Sys::val(a);
    const int n = a->n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T d = 0;
        for (int e = a->rowptr[i]; e < a->rowptr[i + 1]; ++e)
            if (a->colind[e] == i) d = val[e];
        dinv[i] = d != (T)0 ? (T)1 / d : (T)1;
    }
}

// z = (omega dinv) (s u), s = sigma_{sig_idx} (a stored basis column) or 1.
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock)
precond_scale_kernel(const DevArgs* __restrict__ a, const KState* __restrict__ ks,
                     const typename Sys::T* __restrict__ u, int sig_idx,
                     const typename Sys::T* __restrict__ dinv, double omega,
                     typename Sys::T* __restrict__ z, int phase) {
    using T = typename Sys::T;
    if (precond_skipped(ks, phase)) return;
    const T sc = sig_idx >= 0 ? (T)ks->sigma[sig_idx] : (T)1, om = (T)omega;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a->n; i += gridDim.x * blockDim.x)
        z[i] = (om * dinv[i]) * (sc * u[i]);
}

template <typename T>
struct SweepEpi {
    const T* zin;
    const T* u;
    const T* dinv;
    T sc, om;
    T* zout;
    struct Pre { T z, u, d; };
    __device__ Pre pre(int r) const { return {zin[r], u[r], dinv[r]}; }
    __device__ void operator()(int r, T ax, const Pre& o) const {
        zout[r] = o.z + (om * o.d) * (sc * o.u - ax);
    }
    __device__ void operator()(int r, T ax) const { (*this)(r, ax, pre(r)); }
};

// z_out = z_in + (omega dinv) (s u - A z_in).
template <class Sys>
__global__ void __launch_bounds__(kSpmvBlock, 1)
precond_sweep_kernel(const DevArgs* __restrict__ a, KState* ks, const typename Sys::T* __restrict__ u,
                     int sig_idx, const typename Sys::T* __restrict__ dinv, double omega,
                     const typename Sys::T* __restrict__ zin, typename Sys::T* __restrict__ zout,
                     int phase) {
    using T = typename Sys::T;
    if (precond_skipped(ks, phase)) return;
    const T sc = sig_idx >= 0 ? (T)ks->sigma[sig_idx] : (T)1, om = (T)omega;
    const int n = a->n;
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    const SweepEpi<T> epi{zin, u, dinv, sc, om, zout};
    if (a->sell_off) {
        sell_rows<T>(a->sell_off, a->sell_col, reinterpret_cast<const T*>(a->sell_val), zin, n, lo,
                     hi, kSpmvWarps, a->sell_w, a->sell_keep, &ks->bad_index, epi);
        return;
    }
    const T* val = Sys::val(a);
    int flag = 0;
    for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) {
        T ax = 0;
        for (int e = a->rowptr[r]; e < a->rowptr[r + 1]; ++e) {
            const int c = a->colind[e];
            if ((unsigned)c < (unsigned)n) ax = fma(val[e], zin[c], ax);
            else flag = 1;
        }
        epi(r, ax);
    }
    if (flag) atomicOr(&ks->bad_index, 1);
}

// t = V_stored cy (the cycle's correction before preconditioning).
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock, 1)
gmres_combine_kernel(const DevArgs* __restrict__ a, const KState* ks,
                     const typename Sys::T* __restrict__ V, size_t ldv, typename Sys::T* __restrict__ t) {
    using T = typename Sys::T;
    if (update_skipped(ks)) return;
    __shared__ T cy[kMaxBasis];
    __shared__ int kk;
    if (threadIdx.x == 0) kk = ks->jdone;
    for (int k = threadIdx.x; k < kMaxBasis; k += blockDim.x) cy[k] = (T)ks->cy[k];
    __syncthreads();
    const int k = kk, n = a->n;
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        T acc = 0;
        for (int l = 0; l < k; ++l) acc = fma(V[(size_t)l * ldv + i], cy[l], acc);
        t[i] = acc;
    }
}

// x += z.
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock)
gmres_axpy_kernel(const DevArgs* __restrict__ a, const KState* ks, const typename Sys::T* __restrict__ z) {
    using T = typename Sys::T;
    if (update_skipped(ks)) return;
    T* x = Sys::x(a);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a->n; i += gridDim.x * blockDim.x)
        x[i] += z[i];
}

template <typename T>
struct PrecondArgs {
    int sweeps = 0;            // 0: no preconditioner
    double omega = 1.0;
    const T* dinv = nullptr;
    T* za = nullptr;           // sweep ping-pong vectors
    T* zb = nullptr;
    T* t = nullptr;            // correction before preconditioning
};

// Applies M^{-1} to s u (phase 0: u = basis column sig_idx; phase 1: u = t);
// returns the vector holding the result.
template <class Sys>
static const typename Sys::T* launch_precond(const DevArgs* a, KState* ks,
                                             const PrecondArgs<typename Sys::T>& pc,
                                             const typename Sys::T* u, int sig_idx, int phase,
                                             int nblk, cudaStream_t st, cudaEvent_t* ev, int* k);
