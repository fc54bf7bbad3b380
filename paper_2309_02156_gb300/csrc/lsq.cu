// Reduced least squares and guess expansion (Algorithm 1).
//
// y = argmin ||W1 y - wb||_2 for the s x m sketched block, solved by one
// thread block in FP64 with column scaling, Householder QR with
// Businger-Golub column pivoting (largest remaining column 2-norm, ties to
// the lowest index), reflectors alpha = -sign(x_0) ||x|| (sign(0) = +1), rank
// truncation at |R_kk| <= tau |R_00| and back substitution; then x0 = X y.
// The history columns are nearly dependent (the paper's Theorem 1 shows their
// singular values decay geometrically), which is why the factorisation is
// rank revealing.
#include "common.cuh"
#include "internal.h"

namespace sa {

__global__ void __launch_bounds__(256)
lsq_kernel(const double* __restrict__ W, int s, int M, int m, int oldest, double tau, LsqOut* out) {
    extern __shared__ double sm[];
    double* B = sm;              // s x m, column-major (scaled, factorised in place)
    double* Wo = B + s * m;      // s x m, column-major (unscaled copy)
    double* c = Wo + s * m;      // right-hand side, transformed
    double* cb = c + s;          // right-hand side, original
    double* v = cb + s;          // Householder vector
    double* d = v + s;           // column scales
    double* nrm = d + m;
    double* rdiag = nrm + m;
    double* z = rdiag + m;
    double* ylog = z + m;
    double* red = ylog + m;      // 32 doubles
    __shared__ int perm[kMaxM], live[kMaxM];
    __shared__ double sh_normx, sh_vtv;
    __shared__ int sh_p, sh_rank;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int bd = blockDim.x;
    const int ncol = M + 1;

    for (int i = tid; i < s * m; i += bd) {
        const int l = i / s, q = i - l * s;
        Wo[i] = W[q * ncol + (oldest + l) % M];
    }
    for (int q = tid; q < s; q += bd) c[q] = cb[q] = W[q * ncol + M];
    __syncthreads();
    for (int l = warp; l < m; l += nw) {
        double a = 0.0;
        for (int q = lane; q < s; q += 32) a += Wo[l * s + q] * Wo[l * s + q];
        a = warp_sum(a);
        if (lane == 0) d[l] = sqrt(a);
    }
    __syncthreads();
    for (int i = tid; i < s * m; i += bd) {
        const int l = i / s;
        B[i] = d[l] > 0.0 ? Wo[i] / d[l] : 0.0;
    }
    if (tid < m) {
        perm[tid] = tid;
        live[tid] = d[tid] > 0.0;
    }
    __syncthreads();

    const int steps = min(s, m);
    int kdone = 0;
    for (int k = 0; k < steps; ++k) {
        for (int l = k + warp; l < m; l += nw) {
            double a = 0.0;
            for (int q = k + lane; q < s; q += 32) a += B[l * s + q] * B[l * s + q];
            a = warp_sum(a);
            if (lane == 0) nrm[l] = live[perm[l]] ? sqrt(a) : -1.0;
        }
        __syncthreads();
        if (tid == 0) {
            int p = k;
            double best = nrm[k];
            for (int l = k + 1; l < m; ++l)
                if (nrm[l] > best) { best = nrm[l]; p = l; }
            sh_p = p;
        }
        __syncthreads();
        const int p = sh_p;
        if (p != k) {
            for (int q = tid; q < s; q += bd) {
                const double t = B[k * s + q];
                B[k * s + q] = B[p * s + q];
                B[p * s + q] = t;
            }
            if (tid == 0) {
                const int t = perm[k];
                perm[k] = perm[p];
                perm[p] = t;
            }
        }
        __syncthreads();
        if (warp == 0) {
            double a = 0.0;
            for (int q = k + lane; q < s; q += 32) a += B[k * s + q] * B[k * s + q];
            a = warp_sum(a);
            if (lane == 0) sh_normx = sqrt(a);
        }
        __syncthreads();
        const double normx = sh_normx;
        if (normx == 0.0 || !live[perm[k]]) break;
        const double alpha = B[k * s + k] >= 0.0 ? -normx : normx;
        for (int q = k + tid; q < s; q += bd) v[q] = B[k * s + q] - (q == k ? alpha : 0.0);
        __syncthreads();
        if (warp == 0) {
            double a = 0.0;
            for (int q = k + lane; q < s; q += 32) a += v[q] * v[q];
            a = warp_sum(a);
            if (lane == 0) sh_vtv = a;
        }
        __syncthreads();
        const double vtv = sh_vtv;
        if (vtv > 0.0) {
            for (int l = k + 1 + warp; l <= m; l += nw) {      // l == m: right-hand side
                double* col = (l < m) ? B + l * s : c;
                double a = 0.0;
                for (int q = k + lane; q < s; q += 32) a += v[q] * col[q];
                a = warp_sum(a);
                const double t = (2.0 / vtv) * a;
                for (int q = k + lane; q < s; q += 32) col[q] -= v[q] * t;
            }
        }
        __syncthreads();
        for (int q = k + tid; q < s; q += bd) B[k * s + q] = (q == k) ? alpha : 0.0;
        if (tid == 0) rdiag[k] = alpha;
        kdone = k + 1;
        __syncthreads();
    }

    if (tid == 0) {
        int r = 0;
        if (kdone > 0 && rdiag[0] != 0.0) {
            const double lim = tau * fabs(rdiag[0]);
            while (r < kdone && fabs(rdiag[r]) > lim) ++r;
        }
        for (int i = r - 1; i >= 0; --i) {
            double acc = 0.0;
            for (int j = i + 1; j < r; ++j) acc += B[j * s + i] * z[j];
            z[i] = (c[i] - acc) / B[i * s + i];
        }
        for (int l = 0; l < m; ++l) ylog[l] = 0.0;
        for (int i = 0; i < r; ++i) {
            const int l = perm[i];
            ylog[l] = live[l] ? z[i] / d[l] : 0.0;
        }
        sh_rank = r;
    }
    __syncthreads();
    // rho_s = ||Wo y - cb||.
    double part = 0.0;
    for (int q = tid; q < s; q += bd) {
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc += Wo[l * s + q] * ylog[l];
        const double e = acc - cb[q];
        part += e * e;
    }
    part = warp_sum(part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red[w];
        out->rho = sqrt(t);
        out->rank = sh_rank;
        out->m = m;
    }
    for (int k = tid; k < kMaxM; k += bd) {
        out->y_logical[k] = k < m ? ylog[k] : 0.0;
        out->y_phys[k] = 0.0;
    }
    __syncthreads();
    for (int l = tid; l < m; l += bd) out->y_phys[(oldest + l) % M] = ylog[l];
    for (int i = tid; i < s * (m + 1); i += bd) {
        const int q = i / (m + 1), l = i - q * (m + 1);
        out->W_logical[i] = (l < m) ? Wo[l * s + q] : cb[q];
    }
}

void launch_lsq(const double* W, int s, int M, int m, int oldest_slot, double tau, LsqOut* out,
                cudaStream_t st) {
    const size_t smem = sizeof(double) * (2 * (size_t)s * m + 3 * (size_t)s + 5 * (size_t)m + 32);
    // The attribute is per device: set it on every call (cheap, host only).
    cudaFuncSetAttribute(lsq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    lsq_kernel<<<1, 256, smem, st>>>(W, s, M, m, oldest_slot, tau, out);
}

// x0 = X y with FP64 accumulation (X in FP64 or FP32; slots of unused or
// truncated columns carry y = 0).
template <typename XT>
__global__ void expand_kernel(const XT* __restrict__ X, int ldx, int n, int M,
                              const LsqOut* __restrict__ lo, double* __restrict__ x0) {
    __shared__ double ys[kMaxM];
    if (threadIdx.x < kMaxM) ys[threadIdx.x] = threadIdx.x < M ? lo->y_phys[threadIdx.x] : 0.0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const XT* row = X + (size_t)i * ldx;
        double acc = 0.0;
        for (int k = 0; k < M; ++k) acc += (double)row[k] * ys[k];
        x0[i] = acc;
    }
}

template <typename XT>
__global__ void copy_slot_kernel(const XT* __restrict__ X, int ldx, int n, int slot,
                                 double* __restrict__ x0) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x0[i] = (double)X[(size_t)i * ldx + slot];
}

template <typename XT>
__global__ void push_kernel(const double* __restrict__ x, int n, XT* __restrict__ X, int ldx, int slot) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        X[(size_t)i * ldx + slot] = (XT)x[i];
}

static int ew_grid(int n) {
    int b = (n + 255) / 256;
    return b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8;
}

void launch_expand_f64(const double* X, int ldx, int n, int M, const LsqOut* lo, double* x0,
                       cudaStream_t st) {
    expand_kernel<double><<<ew_grid(n), 256, 0, st>>>(X, ldx, n, M, lo, x0);
}
void launch_expand_f32(const float* X, int ldx, int n, int M, const LsqOut* lo, double* x0,
                       cudaStream_t st) {
    expand_kernel<float><<<ew_grid(n), 256, 0, st>>>(X, ldx, n, M, lo, x0);
}
void launch_copy_slot_f64(const double* X, int ldx, int n, int slot, double* x0, cudaStream_t st) {
    copy_slot_kernel<double><<<ew_grid(n), 256, 0, st>>>(X, ldx, n, slot, x0);
}
void launch_copy_slot_f32(const float* X, int ldx, int n, int slot, double* x0, cudaStream_t st) {
    copy_slot_kernel<float><<<ew_grid(n), 256, 0, st>>>(X, ldx, n, slot, x0);
}
void launch_push_f64(const double* x, int n, double* X, int ldx, int slot, cudaStream_t st) {
    push_kernel<double><<<ew_grid(n), 256, 0, st>>>(x, n, X, ldx, slot);
}
void launch_push_f32(const double* x, int n, float* X, int ldx, int slot, cudaStream_t st) {
    push_kernel<float><<<ew_grid(n), 256, 0, st>>>(x, n, X, ldx, slot);
}

}  // namespace sa
