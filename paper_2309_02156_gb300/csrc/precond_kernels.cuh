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
// (a fixed polynomial in D^{-1} A times D^{-1}), or the Chebyshev polynomial
// of the same degree on [lmax / ratio, lmax] of the spectrum of D^{-1} A,
// applied by the Chebyshev iteration's three-term recurrence (one product
// with A per step, like a sweep; one more vector d):
//   d_0 = D^{-1} u / theta, z_1 = d_0,
//   d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^{-1} (u - A z_k), z_{k+1} = z_k + d_k,
// with theta, delta the centre and half-width of the interval, sigma =
// theta / delta, rho_0 = 1 / sigma, rho_k = 1 / (2 sigma - rho_{k-1}); lmax is
// Gershgorin's bound max_i sum_j |a_ij| / |a_ii| unless the caller fixes it.
// Phase 0 kernels belong to an
// Arnoldi step (skipped once the cycle is over), phase 1 kernels to the basis
// update (skipped like the update).
__device__ __forceinline__ bool update_skipped(const KState* ks) {
    return (ks->status != ST_OK && ks->status != ST_NOT_CONVERGED) || ks->finished;
}
__device__ __forceinline__ bool precond_skipped(const KState* ks, int phase) {
    return phase == 0 ? ks->cycle_over != 0 : update_skipped(ks);
}

// dinv = 1 / diag(A) in the system's precision (1 where the diagonal is
// missing or zero); with bound != NULL also max_i (sum_j |a_ij|) / |a_ii| in
// FP64 (row sums in CSR order; the maximum is taken on the bit patterns of
// the non-negative doubles, which order like the values; *bound starts at 0).
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock)
diag_inv_kernel(const DevArgs* __restrict__ a, typename Sys::T* __restrict__ dinv,
                unsigned long long* bound) {
    using T = typename Sys::T;
    const T* val = Sys::val(a);
    const int n = a->n;
    unsigned long long mx = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T d = 0;
        double rs = 0.0;
        for (int e = a->rowptr[i]; e < a->rowptr[i + 1]; ++e) {
            if (a->colind[e] == i) d = val[e];
            rs += fabs((double)val[e]);
        }
        dinv[i] = d != (T)0 ? (T)1 / d : (T)1;
        const double g = rs / (d != (T)0 ? fabs((double)d) : 1.0);
        const unsigned long long gb = (unsigned long long)__double_as_longlong(g);
        mx = gb > mx ? gb : mx;
    }
    if (bound) atomicMax(bound, mx);
}

// Chebyshev coefficients of step k (k >= 1): c1 = rho_k rho_{k-1}, c2 = 2 rho_k
// / delta; step 0 scales by 1 / theta (c2 = 1 / theta).  FP64, from the
// interval [lmax / ratio, lmax].
struct ChebStep {
    double c1, c2;
};
__device__ __forceinline__ ChebStep cheb_step(double lmax, double ratio, int k) {
    const double lmin = lmax / ratio;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    if (k == 0) return {0.0, 1.0 / theta};
    const double sigma = theta / delta;
    double rho_prev = 1.0 / sigma, rho = rho_prev;
    for (int i = 1; i <= k; ++i) {
        rho = 1.0 / (2.0 * sigma - rho_prev);
        if (i < k) rho_prev = rho;
    }
    return {rho * rho_prev, 2.0 * rho / delta};
}

// Coefficient table of the Chebyshev preconditioner, formed once per solve by
// one thread (FP64 divisions are slow on this GPU: the sweeps only load it):
// tab[0] the Gershgorin bound (bits, from the dinv kernel), tab[1] = 1 / theta,
// tab[2k] = c1_k and tab[2k + 1] = c2_k for steps k = 1 .. sweeps - 1; lmax =
// lfix when the caller fixes it, else the bound.
static __global__ void cheb_table_kernel(double* tab, double lfix, double ratio, int sweeps) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double bound = __longlong_as_double(*reinterpret_cast<const long long*>(tab));
    const double lmax = lfix > 0.0 ? lfix : bound;
    tab[1] = cheb_step(lmax, ratio, 0).c2;
    for (int k = 1; k < sweeps && 2 * k + 1 < kChebTab; ++k) {
        const ChebStep c = cheb_step(lmax, ratio, k);
        tab[2 * k] = c.c1;
        tab[2 * k + 1] = c.c2;
    }
}

// Jacobi: z = (omega dinv) (s u); Chebyshev: d = z = dinv (s u) / theta.
// s = sigma_{sig_idx} (a stored basis column) or 1.  Four independent
// elements per thread and iteration.
template <class Sys>
__global__ void __launch_bounds__(kStreamBlock)
precond_scale_kernel(const DevArgs* __restrict__ a, const KState* __restrict__ ks,
                     const typename Sys::T* __restrict__ u, int sig_idx,
                     const typename Sys::T* __restrict__ dinv, double omega,
                     typename Sys::T* __restrict__ z, int phase, int cheb,
                     const double* __restrict__ tab, typename Sys::T* __restrict__ dvec) {
    using T = typename Sys::T;
    if (precond_skipped(ks, phase)) return;
    const T sc = sig_idx >= 0 ? (T)ks->sigma[sig_idx] : (T)1;
    const T om = cheb ? (T)tab[1] : (T)omega;
    const int n = a->n, stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        T uu[4], dd[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + q * stride;
            uu[q] = i < n ? u[i] : (T)0;
            dd[q] = i < n ? dinv[i] : (T)0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + q * stride;
            if (i < n) {
                const T zi = (om * dd[q]) * (sc * uu[q]);
                z[i] = zi;
                if (cheb) dvec[i] = zi;
            }
        }
    }
}

template <typename T>
struct SweepEpi {
    const T* zin;
    const T* u;
    const T* dinv;
    T sc, om;
    T* zout;
    static constexpr int kSlices = 0;
    struct Pre { T z, u, d; };
    __device__ Pre pre(int r) const { return {zin[r], u[r], dinv[r]}; }
    __device__ void operator()(int r, T ax, const Pre& o) const {
        zout[r] = o.z + (om * o.d) * (sc * o.u - ax);
    }
    __device__ void operator()(int r, T ax) const { (*this)(r, ax, pre(r)); }
};

// Chebyshev step: d = c1 d + c2 dinv (s u - A z_in), z_out = z_in + d (d is
// not stored at the last step: dout = NULL).
template <typename T>
struct ChebEpi {
    const T* zin;
    const T* u;
    const T* dinv;
    const T* dvec;
    T* dout;
    T sc, c1, c2;
    T* zout;
    static constexpr int kSlices = 2;
    struct Pre { T z, u, d, dv; };
    __device__ Pre pre(int r) const { return {zin[r], u[r], dinv[r], dvec[r]}; }
    __device__ void operator()(int r, T ax, const Pre& o) const {
        const T dn = c1 * o.dv + c2 * (o.d * (sc * o.u - ax));
        if (dout) dout[r] = dn;
        zout[r] = o.z + dn;
    }
    __device__ void operator()(int r, T ax) const { (*this)(r, ax, pre(r)); }
};

// First sweep with the scale step folded in: z_1 = om (dinv (s u)) is a
// pointwise function of u, so the product gathers u[c] dinv[c] (A z_1 = om s
// A (dinv .* u)) and the row forms z_1 itself.  Jacobi: om = omega, z_out =
// z_1 + om dinv (s u - A z_1).  Chebyshev: om = 1 / theta, d_0 = z_1, d_1 = c1
// d_0 + c2 dinv (s u - A z_1), z_out = z_1 + d_1.
template <typename T, int CHEB>
struct FirstEpi {
    const T* u;
    const T* dinv;
    const T* x2;                         // = dinv: the gather's second factor
    T* dout;
    T sc, om, c1, c2;
    T* zout;
    static constexpr int kSlices = CHEB ? 2 : 0;
    static constexpr bool kProd = true;
    struct Pre { T u, d; };
    __device__ Pre pre(int r) const { return {u[r], dinv[r]}; }
    __device__ void operator()(int r, T ax, const Pre& o) const {
        const T su = sc * o.u;
        const T z1 = (om * o.d) * su;
        const T az = (om * sc) * ax;
        if constexpr (CHEB != 0) {
            const T dn = c1 * z1 + c2 * (o.d * (su - az));
            if (dout) dout[r] = dn;
            zout[r] = z1 + dn;
        } else {
            zout[r] = z1 + (om * o.d) * (su - az);
        }
    }
    __device__ void operator()(int r, T ax) const { (*this)(r, ax, pre(r)); }
};

template <class Sys, typename Epi>
__device__ __forceinline__ void precond_rows(const DevArgs* __restrict__ a, KState* ks,
                                             const typename Sys::T* __restrict__ zin, const Epi& epi) {
    using T = typename Sys::T;
    const int n = a->n;
    int lo, hi;
    block_rows(n, gridDim.x, blockIdx.x, lo, hi);
    if (a->sell_off) {
        sell_rows<T>(a->sell_off, a->sell_col, reinterpret_cast<const T*>(a->sell_val), zin, n, lo,
                     hi, (int)(blockDim.x >> 5), a->sell_w, a->sell_keep, &ks->bad_index, epi);
        return;
    }
    const T* val = Sys::val(a);
    const T* x2 = gather_x2<Epi, T>(epi);
    int flag = 0;
    for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) {
        T ax = 0;
        for (int e = a->rowptr[r]; e < a->rowptr[r + 1]; ++e) {
            const int c = a->colind[e];
            if ((unsigned)c < (unsigned)n) ax = fma(val[e], x2 ? zin[c] * x2[c] : zin[c], ax);
            else flag = 1;
        }
        epi(r, ax);
    }
    if (flag) atomicOr(&ks->bad_index, 1);
}

// Sweep k (k >= 1) of the preconditioner.  Jacobi: z_out = z_in + (omega
// dinv) (s u - A z_in); Chebyshev: the recurrence step above.  FIRST: sweep 1
// with the scale step folded in (z_in is not read; see FirstEpi).  last: the
// final sweep of the application (Chebyshev does not store d there).
template <class Sys, int CHEB, int FIRST>
__global__ void __launch_bounds__(kSpmvBlock, 1)
precond_sweep_kernel(const DevArgs* __restrict__ a, KState* ks, const typename Sys::T* __restrict__ u,
                     int sig_idx, const typename Sys::T* __restrict__ dinv, double omega,
                     const typename Sys::T* __restrict__ zin, typename Sys::T* __restrict__ zout,
                     int phase, int k, const double* __restrict__ tab,
                     typename Sys::T* __restrict__ dvec, int last) {
    using T = typename Sys::T;
    if (precond_skipped(ks, phase)) return;
    const T sc = sig_idx >= 0 ? (T)ks->sigma[sig_idx] : (T)1;
    T* dout = last ? nullptr : dvec;
    if constexpr (FIRST != 0) {
        const T om = CHEB ? (T)tab[1] : (T)omega;
        const T c1 = CHEB ? (T)tab[2] : (T)0, c2 = CHEB ? (T)tab[3] : (T)0;
        const FirstEpi<T, CHEB> epi{u, dinv, dinv, dout, sc, om, c1, c2, zout};
        precond_rows<Sys>(a, ks, u, epi);
    } else if constexpr (CHEB != 0) {
        const ChebEpi<T> epi{zin, u, dinv, dvec, dout, sc, (T)tab[2 * k], (T)tab[2 * k + 1], zout};
        precond_rows<Sys>(a, ks, zin, epi);
    } else {
        const SweepEpi<T> epi{zin, u, dinv, sc, (T)omega, zout};
        precond_rows<Sys>(a, ks, zin, epi);
    }
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
    int cheb = 0;              // 1: Chebyshev polynomial instead of Jacobi sweeps
    const double* tab = nullptr;   // its coefficient table (cheb_table_kernel)
    T* dvec = nullptr;         // Chebyshev recurrence vector
};

// Applies M^{-1} to s u (phase 0: u = basis column sig_idx; phase 1: u = t);
// returns the vector holding the result.
template <class Sys>
static const typename Sys::T* launch_precond(const DevArgs* a, KState* ks,
                                             const PrecondArgs<typename Sys::T>& pc,
                                             const typename Sys::T* u, int sig_idx, int phase,
                                             int nblk, cudaStream_t st, cudaEvent_t* ev, int* k);
