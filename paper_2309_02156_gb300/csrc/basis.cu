// Compressed bases of span(X) for the guess (Section 2): POD (Algorithm 2)
// and the randomised range finder with progressive updates (Algorithm 4).
//
// POD.  Q_POD spans X V_k, where V_k holds the k leading eigenvectors of the
// Gram matrix G = X^T X (the snapshot form of the truncated SVD: the left
// singular vectors are X v_j / sigma_j).  G is formed in one pass over the
// history (FP64, deterministic block partials), its eigendecomposition by a
// parallel cyclic Jacobi method in one block (round-robin pair ordering,
// Golub-Van Loan's symmetric 2x2 Schur rotation).  The guess then needs no
// pass of its own over A: the sketched block of the whole history
// W = S [A X | b] is already formed, and S A (X V_k) = (S A X) V_k, so the
// reduced problem is min ||W1 V_k c - wb|| (s x k), solved by the same
// pivoted-QR least squares, and x0 = X (V_k c).
//
// Randomised range finder.  Omega = X Z (n x m, row-major, FP64) is formed
// from scratch with a Gaussian Z and, at every push of a new
// solution, updated in the same pass that writes the solution into the ring:
// Omega[r,:] = (Omega[r,:] - x_leaving[r] z_1) + x_new[r] z_new (the
// progressive update of Algorithm 4).
// Z is kept per ring slot, so "moving the rows of Z up" is the ring's index
// arithmetic.  The guess sketches A Omega (m columns instead of M) and
// solves the reduced least squares; x0 = Omega c.
//
// Gaussian draw k of a context: Box-Muller on SplitMix64 outputs 2k+1 and
// 2k+2 of the stream seeded with seed XOR 0x52414E44 (u1 = ((h1 >> 11) + 1)
// 2^-53, u2 = (h2 >> 11) 2^-53, g = sqrt(-2 ln u1) cos(2 pi u2)).
#include "common.cuh"
#include "internal.h"

namespace sa {
namespace {

constexpr int kGramThreads = 256;
constexpr int kGramTile = 64;
constexpr int kMaxPairs = kMaxM * (kMaxM + 1) / 2;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ double gauss_draw(uint64_t gseed, uint64_t k) {
    const uint64_t h1 = mix64(gseed + (2 * k + 1) * kGamma);
    const uint64_t h2 = mix64(gseed + (2 * k + 2) * kGamma);
    const double u1 = (double)((h1 >> 11) + 1) * 0x1p-53;
    const double u2 = (double)(h2 >> 11) * 0x1p-53;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Z rows of a from-scratch Omega: logical column l (ring slot (oldest+l) % M)
// takes draws start + l m .. start + l m + m - 1.
__global__ void rand_draw_z_kernel(double* Zs, int M, int mi, int oldest, int m, uint64_t gseed,
                                   uint64_t start) {
    for (int i = threadIdx.x; i < mi * m; i += blockDim.x) {
        const int l = i / m, j = i - l * m;
        Zs[((oldest + l) % M) * m + j] = gauss_draw(gseed, start + (uint64_t)i);
    }
}

// Omega = X Z over the mi history columns (oldest first); one row per thread.
__global__ void rand_scratch_kernel(const double* __restrict__ X, int ldx, int n, int M, int mi,
                                    int oldest, const double* __restrict__ Zs, int m,
                                    double* __restrict__ Om, int ldo) {
    __shared__ double z[kMaxM * kMaxM];
    __shared__ int slot[kMaxM];
    for (int i = threadIdx.x; i < mi * m; i += blockDim.x) {
        const int l = i / m, j = i - l * m;
        z[i] = Zs[((oldest + l) % M) * m + j];
    }
    if (threadIdx.x < mi) slot[threadIdx.x] = (oldest + threadIdx.x) % M;
    __syncthreads();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        double acc[kMaxM];
#pragma unroll
        for (int j = 0; j < kMaxM; ++j) acc[j] = 0.0;
        const double* xr = X + (size_t)r * ldx;
        for (int l = 0; l < mi; ++l) {
            const double xv = xr[slot[l]];
#pragma unroll
            for (int j = 0; j < kMaxM; ++j)
                if (j < m) acc[j] = fma(xv, z[l * m + j], acc[j]);
        }
        double* o = Om + (size_t)r * ldo;
#pragma unroll
        for (int j = 0; j < kMaxM; ++j)
            if (j < ldo) o[j] = j < m ? acc[j] : 0.0;
    }
}

// The progressive update fused with the push: Omega[r,:] = (Omega[r,:] - x_old[r] z_old)
// + x_new[r] z_new and X[r, slot] = x_new[r] (x_old = the slot's previous
// content when `remove`, else nothing is removed).
__global__ void rand_push_kernel(const double* __restrict__ x, int n, double* __restrict__ X, int ldx,
                                 int slot, int remove, const double* __restrict__ Zs, int m,
                                 uint64_t gseed, uint64_t start, double* __restrict__ Om, int ldo) {
    __shared__ double zo[kMaxM], zn[kMaxM];
    if (threadIdx.x < m) {
        zo[threadIdx.x] = remove ? Zs[slot * m + threadIdx.x] : 0.0;
        zn[threadIdx.x] = gauss_draw(gseed, start + threadIdx.x);
    }
    __syncthreads();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const double xn = x[r];
        double* xs = X + (size_t)r * ldx + slot;
        const double xo = remove ? *xs : 0.0;
        double* o = Om + (size_t)r * ldo;
        for (int j = 0; j < m; ++j) o[j] = fma(xn, zn[j], fma(-xo, zo[j], o[j]));
        *xs = xn;
    }
}

// The new row of Z, stored in the slot after every block has read the old one.
__global__ void rand_store_z_kernel(double* Zs, int slot, int m, uint64_t gseed, uint64_t start) {
    if (threadIdx.x < m) Zs[slot * m + threadIdx.x] = gauss_draw(gseed, start + threadIdx.x);
}

// G = X^T X over the mi history columns (logical order).  Each block sums its
// rows for the upper-triangle pairs (a <= b) it owns; the last block to
// finish adds the block partials in block order and writes G (mi x mi).
__global__ void __launch_bounds__(kGramThreads)
gram_kernel(const double* __restrict__ X, int ldx, int n, int M, int mi, int oldest,
            double* __restrict__ partial, unsigned* counter, double* __restrict__ G) {
    __shared__ double tile[kGramTile * 32];
    const int tid = threadIdx.x, npairs = mi * (mi + 1) / 2;
    int sa_[2], sb_[2], pa[2], pb[2];
    double acc[2] = {0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        int p = tid + k * kGramThreads, a = 0;
        pa[k] = pb[k] = -1;
        sa_[k] = sb_[k] = 0;
        if (p < npairs) {
            while (p >= mi - a) {      // row a of the upper triangle holds mi - a pairs
                p -= mi - a;
                ++a;
            }
            pa[k] = a;
            pb[k] = a + p;
            sa_[k] = (oldest + pa[k]) % M;
            sb_[k] = (oldest + pb[k]) % M;
        }
    }
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int lo = min(n, blockIdx.x * per), hi = min(n, lo + per);
    for (int r0 = lo; r0 < hi; r0 += kGramTile) {
        const int rows = min(kGramTile, hi - r0);
        const double* src = X + (size_t)r0 * ldx;
        for (int i = tid; i < rows * ldx; i += kGramThreads) tile[i] = src[i];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (pa[k] >= 0)
                for (int rr = 0; rr < rows; ++rr)
                    acc[k] = fma(tile[rr * ldx + sa_[k]], tile[rr * ldx + sb_[k]], acc[k]);
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 2; ++k)
        if (pa[k] >= 0) partial[(size_t)blockIdx.x * kMaxPairs + tid + k * kGramThreads] = acc[k];
    if (last_block_arrive(counter)) {
        for (int p = tid; p < npairs; p += kGramThreads) {
            double s = 0.0;
            for (int blk = 0; blk < (int)gridDim.x; ++blk) s += partial[(size_t)blk * kMaxPairs + p];
            int a = 0, q = p;
            while (q >= mi - a) {
                q -= mi - a;
                ++a;
            }
            const int b = a + q;
            G[a * mi + b] = s;
            G[b * mi + a] = s;
        }
        if (tid == 0) *counter = 0u;
    }
}

// Eigendecomposition of the symmetric G (k x k, k <= 31) by the cyclic
// Jacobi method with the round-robin ordering (k/2 disjoint rotations per
// round, applied to rows, then columns, then to V), at most `max_sweeps`
// sweeps, stopping once the off-diagonal mass is below (1e-15)^2 of ||G||_F^2.
// Writes the `kk` leading eigenvectors (eigenvalues descending, ties to the
// lower index) to Vk (k x kk, column-major) and all eigenvalues (descending)
// to lam.
__global__ void __launch_bounds__(512)
jacobi_eig_kernel(const double* __restrict__ Gin, int k, int kk, int max_sweeps,
                  double* __restrict__ Vk, double* __restrict__ lam, int* sweeps_out) {
    __shared__ double G[32][33], V[32][33];
    __shared__ double cs[16], sn[16];
    __shared__ int pp[16], qq[16], arr[32];
    __shared__ int done, order[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int P = (k + 1) & ~1;                  // players (a dummy when k is odd)
    for (int i = tid; i < 32 * 32; i += nt) {
        const int r = i / 32, c = i % 32;
        G[r][c] = (r < k && c < k) ? Gin[r * k + c] : 0.0;
        V[r][c] = (r == c) ? 1.0 : 0.0;
    }
    if (tid == 0) done = 0;
    __syncthreads();
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // convergence test
        if (tid < 32) {
            double off = 0.0, tot = 0.0;
            for (int c = 0; c < k; ++c) {
                const double g = tid < k ? G[tid][c] : 0.0;
                tot += g * g;
                if (c != tid) off += g * g;
            }
            off = warp_sum(off);
            tot = warp_sum(tot);
            if (tid == 0) done = (off <= 1e-30 * tot) || tot == 0.0;
        }
        __syncthreads();
        if (done) break;
        for (int round = 0; round < P - 1; ++round) {
            if (tid < P) arr[tid] = tid == 0 ? 0 : (round + tid - 1) % (P - 1) + 1;
            __syncthreads();
            if (tid < P / 2) {
                int p = arr[tid], q = arr[P - 1 - tid];
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                double c = 1.0, s = 0.0;
                if (q < k) {
                    const double apq = G[p][q];
                    if (apq != 0.0) {
                        const double tau = (G[q][q] - G[p][p]) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                cs[tid] = c;
                sn[tid] = s;
                pp[tid] = p;
                qq[tid] = q < k ? q : p;     // a dummy pair rotates nothing
            }
            __syncthreads();
            const int npair = P / 2;
            for (int i = tid; i < npair * k; i += nt) {          // rows: J^T G
                const int pr = i / k, j = i - pr * k;
                const int p = pp[pr], q = qq[pr];
                if (p == q) continue;
                const double c = cs[pr], s = sn[pr];
                const double gp = G[p][j], gq = G[q][j];
                G[p][j] = c * gp - s * gq;
                G[q][j] = s * gp + c * gq;
            }
            __syncthreads();
            for (int i = tid; i < npair * k; i += nt) {          // columns: G J and V J
                const int pr = i / k, j = i - pr * k;
                const int p = pp[pr], q = qq[pr];
                if (p == q) continue;
                const double c = cs[pr], s = sn[pr];
                const double gp = G[j][p], gq = G[j][q];
                G[j][p] = c * gp - s * gq;
                G[j][q] = s * gp + c * gq;
                const double vp = V[j][p], vq = V[j][q];
                V[j][p] = c * vp - s * vq;
                V[j][q] = s * vp + c * vq;
            }
            __syncthreads();
            if (tid < npair && pp[tid] != qq[tid]) {              // exact zero of the pivot
                G[pp[tid]][qq[tid]] = 0.0;
                G[qq[tid]][pp[tid]] = 0.0;
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        for (int i = 0; i < k; ++i) order[i] = i;
        for (int i = 0; i < k; ++i) {          // selection of the largest remaining, ties lowest
            int best = i;
            for (int j = i + 1; j < k; ++j)
                if (G[order[j]][order[j]] > G[order[best]][order[best]]) best = j;
            const int t = order[i];
            order[i] = order[best];
            order[best] = t;
        }
        if (sweeps_out) *sweeps_out = sweep;
    }
    __syncthreads();
    for (int i = tid; i < k; i += nt) lam[i] = G[order[i]][order[i]];
    for (int i = tid; i < k * kk; i += nt) {
        const int c = i / k, r = i - c * k;
        Vk[c * k + r] = V[r][order[c]];
    }
}

// Reduced block W' = [W1 V_k | wb] (s x (kk+1), row-major) from the sketched
// block of the whole history (W: s x (M+1), ring slots, b last).
__global__ void pod_project_kernel(const double* __restrict__ W, int s, int M, int mi, int oldest,
                                   const double* __restrict__ Vk, int kk, double* __restrict__ Wp) {
    const int nc = kk + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s * nc; i += gridDim.x * blockDim.x) {
        const int q = i / nc, c = i - q * nc;
        double v;
        if (c < kk) {
            v = 0.0;
            for (int l = 0; l < mi; ++l) v = fma(W[q * (M + 1) + (oldest + l) % M], Vk[c * mi + l], v);
        } else {
            v = W[q * (M + 1) + M];
        }
        Wp[i] = v;
    }
}

// History coefficients y = V_k c in ring-slot order for the expansion
// x0 = X y; the reduced problem's block and c stay as the diagnostics.
__global__ void pod_coeff_kernel(const LsqOut* __restrict__ red, const double* __restrict__ Vk, int mi,
                                 int kk, int M, int oldest, LsqOut* __restrict__ out) {
    const int tid = threadIdx.x;
    double y = 0.0;
    if (tid < mi)
        for (int c = 0; c < kk; ++c) y = fma(Vk[c * mi + tid], red->y_logical[c], y);
    if (tid < kMaxM) {
        out->y_logical[tid] = tid < kk ? red->y_logical[tid] : 0.0;
        out->y_phys[tid] = 0.0;
    }
    __syncthreads();
    if (tid < mi) out->y_phys[(oldest + tid) % M] = y;
    for (int i = tid; i < kMaxS * (kMaxM + 1); i += blockDim.x) out->W_logical[i] = red->W_logical[i];
    if (tid == 0) {
        out->rho = red->rho;
        out->rank = red->rank;
        out->m = kk;
    }
}

int ew_blocks(int n) {
    const int b = (n + 255) / 256;
    return b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8;
}

}  // namespace

int gram_grid() { return 2 * 152; }
size_t gram_partial_doubles() { return (size_t)gram_grid() * kMaxPairs; }

void launch_rand_scratch(const double* X, int ldx, int n, int M, int mi, int oldest, double* Zs, int m,
                         uint64_t gseed, uint64_t start, double* Om, int ldo, cudaStream_t st) {
    rand_draw_z_kernel<<<1, 256, 0, st>>>(Zs, M, mi, oldest, m, gseed, start);
    rand_scratch_kernel<<<ew_blocks(n), 256, 0, st>>>(X, ldx, n, M, mi, oldest, Zs, m, Om, ldo);
}

void launch_rand_push(const double* x, int n, double* X, int ldx, int slot, int remove, double* Zs,
                      int m, uint64_t gseed, uint64_t start, double* Om, int ldo, cudaStream_t st) {
    rand_push_kernel<<<ew_blocks(n), 256, 0, st>>>(x, n, X, ldx, slot, remove, Zs, m, gseed, start, Om, ldo);
    rand_store_z_kernel<<<1, 32, 0, st>>>(Zs, slot, m, gseed, start);
}

void launch_pod_basis(const double* X, int ldx, int n, int M, int mi, int oldest, int kk,
                      double* partial, unsigned* counter, double* G, double* Vk, double* lam,
                      int* sweeps, cudaStream_t st) {
    gram_kernel<<<gram_grid(), kGramThreads, 0, st>>>(X, ldx, n, M, mi, oldest, partial, counter, G);
    jacobi_eig_kernel<<<1, 512, 0, st>>>(G, mi, kk, 40, Vk, lam, sweeps);
}

void launch_pod_reduce(const double* W, int s, int M, int mi, int oldest, const double* Vk, int kk,
                       double* Wp, cudaStream_t st) {
    pod_project_kernel<<<(s * (kk + 1) + 255) / 256, 256, 0, st>>>(W, s, M, mi, oldest, Vk, kk, Wp);
}

void launch_pod_coeff(const LsqOut* red, const double* Vk, int mi, int kk, int M, int oldest,
                      LsqOut* out, cudaStream_t st) {
    pod_coeff_kernel<<<1, 256, 0, st>>>(red, Vk, mi, kk, M, oldest, out);
}

}  // namespace sa
