// Learned coefficient predictor: a small MLP that predicts the history
// coefficients y of the guess from the coefficient vectors of the previous
// four systems and the sketched residual of the linearly extrapolated guess
// (the paper computes y by least squares every step, Algorithm 1; this
// is the learned variant, with the sketched least squares as fallback).
//
// Network: 4M+s -> H -> H -> M, GELU (erf form), weights stored FP32 (master)
// and rounded to bfloat16 (round to nearest even) for every forward and
// backward pass, FP32 arithmetic and accumulation.  Output head:
// y_hat = shift(y_{i-1}) + sigma_out * d.  Loss per sample:
// (y_hat - y)^T (W1^T W1) (y_hat - y) / ||wb||^2, the excess sketched residual
// over the least-squares minimum.  Adam (bias-corrected).  Every reduction
// (GEMM dot products, batch sums) runs in a fixed order: training is
// deterministic.
//
// Sample layout (FP32, stride in + out + out*out + 1):
//   [features (in) | target y (out) | G = W1^T W1 (out x out) | ||wb||].
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/seqaccel.h"
#include "common.cuh"
#include "internal.h"
#include "mlp_internal.h"

#include <cuda_bf16.h>

namespace sa {
namespace {

constexpr int TB = 16;   // GEMM tile

__device__ __forceinline__ float gelu_f(float u) { return 0.5f * u * (1.0f + erff(u * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float u) {
    return 0.5f * (1.0f + erff(u * 0.70710678118654752f)) +
           u * expf(-0.5f * u * u) * 0.39894228040143268f;
}
__device__ __forceinline__ float bf(uint16_t v) {
    return __bfloat162float(__ushort_as_bfloat16(v));
}

// Y = X W^T + b (X: B x K fp32, W: N x K bf16); optional H = GELU(Y).
__global__ void linear_fwd(const float* __restrict__ X, int ldx, const uint16_t* __restrict__ W,
                           const float* __restrict__ bias, int B, int N, int K, float* A, float* H) {
    __shared__ float xs[TB][TB + 1], ws[TB][TB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * TB + ty, col = blockIdx.x * TB + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += TB) {
        xs[ty][tx] = (row < B && k0 + tx < K) ? X[(size_t)row * ldx + k0 + tx] : 0.f;
        const int wn = blockIdx.x * TB + ty;
        ws[ty][tx] = (wn < N && k0 + tx < K) ? bf(W[(size_t)wn * K + k0 + tx]) : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TB; ++k) acc = fmaf(xs[ty][k], ws[tx][k], acc);
        __syncthreads();
    }
    if (row < B && col < N) {
        const float a = acc + bias[col];
        A[(size_t)row * N + col] = a;
        if (H) H[(size_t)row * N + col] = gelu_f(a);
    }
}

// dX = (dY W) * GELU'(Apre)   (dY: B x N, W: N x K bf16, dX: B x K)
__global__ void linear_bwd_input(const float* __restrict__ dY, const uint16_t* __restrict__ W,
                                 const float* __restrict__ Apre, int B, int N, int K, float* dX) {
    __shared__ float ds[TB][TB + 1], ws[TB][TB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * TB + ty, col = blockIdx.x * TB + tx;
    float acc = 0.f;
    for (int n0 = 0; n0 < N; n0 += TB) {
        ds[ty][tx] = (row < B && n0 + tx < N) ? dY[(size_t)row * N + n0 + tx] : 0.f;
        const int wk = blockIdx.x * TB + tx;
        ws[ty][tx] = (n0 + ty < N && wk < K) ? bf(W[(size_t)(n0 + ty) * K + wk]) : 0.f;
        __syncthreads();
#pragma unroll
        for (int n = 0; n < TB; ++n) acc = fmaf(ds[ty][n], ws[n][tx], acc);
        __syncthreads();
    }
    if (row < B && col < K) {
        const float g = Apre ? gelu_d(Apre[(size_t)row * K + col]) : 1.f;
        dX[(size_t)row * K + col] = acc * g;
    }
}

// dW = dY^T X (N x K), db = sum_b dY (b in order)
__global__ void linear_bwd_weight(const float* __restrict__ dY, const float* __restrict__ X, int ldx,
                                  int B, int N, int K, float* dW, float* db) {
    __shared__ float ds[TB][TB + 1], xs[TB][TB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int n = blockIdx.y * TB + ty, k = blockIdx.x * TB + tx;
    float acc = 0.f, bacc = 0.f;
    for (int b0 = 0; b0 < B; b0 += TB) {
        ds[ty][tx] = (b0 + tx < B && blockIdx.y * TB + ty < N) ? dY[(size_t)(b0 + tx) * N + blockIdx.y * TB + ty] : 0.f;
        xs[ty][tx] = (b0 + ty < B && k < K) ? X[(size_t)(b0 + ty) * ldx + k] : 0.f;
        __syncthreads();
#pragma unroll
        for (int b = 0; b < TB; ++b) acc = fmaf(ds[ty][b], xs[b][tx], acc);
        if (blockIdx.x == 0 && tx == 0) {
            for (int b = 0; b < TB; ++b) bacc += ds[ty][b];
        }
        __syncthreads();
    }
    if (n < N && k < K) dW[(size_t)n * K + k] = acc;
    if (blockIdx.x == 0 && tx == 0 && n < N) db[n] = bacc;
}

__global__ void normalize_kernel(const float* __restrict__ S, int stride, int B, int in,
                                 const float* __restrict__ mu, const float* __restrict__ sd, float* z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * in) return;
    const int b = i / in, f = i - b * in;
    z[i] = (S[(size_t)b * stride + f] - mu[f]) / sd[f];
}

// y = base + sigma * d; for training also the loss gradient and per-sample loss.
__global__ void head_kernel(const float* __restrict__ S, int stride, int B, int out,
                            const float* __restrict__ d, const float* __restrict__ sig, int in,
                            float* y, float* dd, float* loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float* s = S + (size_t)b * stride;
    float yy[kMaxM];
    for (int j = 0; j < out; ++j) {
        yy[j] = s[j] + sig[j] * d[(size_t)b * out + j];
        y[(size_t)b * out + j] = yy[j];
    }
    if (!dd) return;
    const float* T = s + in;
    const float* G = T + out;
    const float nb = s[in + out + out * out];
    const float inv = 1.f / (nb * nb);
    float l = 0.f;
    for (int j = 0; j < out; ++j) {
        float ge = 0.f;
        for (int k = 0; k < out; ++k) ge = fmaf(G[j * out + k], yy[k] - T[k], ge);
        l = fmaf(yy[j] - T[j], ge, l);
        dd[(size_t)b * out + j] = (2.f / (float)B) * ge * inv * sig[j];
    }
    loss[b] = l * inv;
}

__global__ void sum_kernel(const float* __restrict__ v, int n, float* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += v[i];
    *out = s / (float)n;
}

__global__ void adam_kernel(float* P, const float* __restrict__ G, float* M, float* V, size_t n,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.f - b1) * g;
        const float v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ P, uint16_t* W, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        W[i] = __bfloat16_as_ushort(__float2bfloat16_rn(P[i]));
}

// He-uniform weights from SplitMix64 outputs offset+1 .., biases zero.
__global__ void he_init_kernel(float* W, size_t n, int fan_in, uint64_t seed, uint64_t offset) {
    const double bound = sqrt(6.0 / (double)fan_in);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint64_t h = mix64(seed + (offset + i + 1) * 0x9E3779B97F4A7C15ull);
        const double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
        W[i] = (float)((2.0 * u - 1.0) * bound);
    }
}

__global__ void gather_kernel(const float* __restrict__ S, const int* __restrict__ idx, int B,
                              int stride, float* out) {
    const size_t total = (size_t)B * stride;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / stride);
        out[i] = S[(size_t)idx[b] * stride + (i - (size_t)b * stride)];
    }
}

// Per-feature mean/std over the samples, and per-output std of (target - base).
__global__ void norm_stats_kernel(const float* __restrict__ S, int stride, int count, int in,
                                  int out, float* mu, float* sd, float* sig) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < in) {
        double s = 0, s2 = 0;
        for (int b = 0; b < count; ++b) {
            const double v = S[(size_t)b * stride + f];
            s += v;
            s2 += v * v;
        }
        const double m = s / count, var = fmax(s2 / count - m * m, 0.0);
        mu[f] = (float)m;
        sd[f] = (float)fmax(sqrt(var), 1e-6);
    } else if (f < in + out) {
        const int j = f - in;
        double s2 = 0;
        for (int b = 0; b < count; ++b) {
            const double v = S[(size_t)b * stride + in + j] - S[(size_t)b * stride + j];
            s2 += v * v;
        }
        sig[j] = (float)fmax(sqrt(s2 / count), 1e-6);
    }
}

}  // namespace

// ---- pieces used by the learned guess in api.cu ----------------------------

// Training sample of the current guess: features from the sketched block of
// the current window and the previous coefficient vectors (ring, newest
// first), target = the least-squares y, G = W1^T W1, ||wb||.
__global__ void learned_sample_kernel(const LsqOut* __restrict__ lo, int s, int M,
                                      const double* __restrict__ yring, float* sample) {
    __shared__ double Wl[kMaxS * (kMaxM + 1)];
    const int ncol = M + 1, in = 4 * M + s, tid = threadIdx.x;
    for (int i = tid; i < s * ncol; i += blockDim.x) Wl[i] = lo->W_logical[i];
    __syncthreads();
    __shared__ double nb;
    if (tid == 0) {
        double t = 0;
        for (int q = 0; q < s; ++q) t += Wl[q * ncol + M] * Wl[q * ncol + M];
        nb = sqrt(t);
    }
    __syncthreads();
    for (int k = 1; k <= 4; ++k)
        for (int j = tid; j < M; j += blockDim.x) {
            const int src = j + k;
            sample[(k - 1) * M + j] = src < M ? (float)yring[(k - 1) * kMaxM + src] : 0.f;
        }
    for (int q = tid; q < s; q += blockDim.x) {
        const double e = 2.0 * Wl[q * ncol + M - 1] - (M >= 2 ? Wl[q * ncol + M - 2] : 0.0) - Wl[q * ncol + M];
        sample[4 * M + q] = (float)(e / nb);
    }
    for (int j = tid; j < M; j += blockDim.x) sample[in + j] = (float)lo->y_logical[j];
    for (int jk = tid; jk < M * M; jk += blockDim.x) {
        const int j = jk / M, k = jk - j * M;
        double g = 0;
        for (int q = 0; q < s; ++q) g += Wl[q * ncol + j] * Wl[q * ncol + k];
        sample[in + M + jk] = (float)g;
    }
    if (tid == 0) sample[in + M + M * M] = (float)nb;
}

// Choose between the network's prediction and the least-squares solution:
// the network's y is used unless its sketched residual exceeds 1.5 times the
// least-squares one.  Writes the chosen y into lo (logical and physical).
__global__ void learned_select_kernel(LsqOut* lo, int s, int M, int oldest, const float* __restrict__ yhat,
                                      int* used_net, double* rho_net_out) {
    __shared__ double part[32];
    const int ncol = M + 1, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double acc = 0;
    for (int q = tid; q < s; q += blockDim.x) {
        double r = -lo->W_logical[q * ncol + M];
        for (int j = 0; j < M; ++j) r += lo->W_logical[q * ncol + j] * (double)yhat[j];
        acc += r * r;
    }
    acc = warp_sum(acc);
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    __shared__ int use;
    if (tid == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        const double rho_net = sqrt(t);
        use = rho_net <= 1.5 * lo->rho;
        *rho_net_out = rho_net;
        if (use) lo->rho = rho_net;
        *used_net = use;
    }
    __syncthreads();
    if (use) {
        for (int j = tid; j < M; j += blockDim.x) {
            lo->y_logical[j] = (double)yhat[j];
            lo->y_phys[(oldest + j) % M] = (double)yhat[j];
        }
    }
}

// Ring of the last four coefficient vectors (newest first), in the frame of
// the window they were computed for.
__global__ void yring_push_kernel(double* yring, const LsqOut* __restrict__ lo, int M) {
    const int j = threadIdx.x;
    if (j >= M) return;
    for (int k = 3; k >= 1; --k) yring[k * kMaxM + j] = yring[(k - 1) * kMaxM + j];
    yring[j] = lo->y_logical[j];
}

void launch_learned_sample(const LsqOut* lo, int s, int M, const double* yring, float* sample,
                           cudaStream_t st) {
    learned_sample_kernel<<<1, 256, 0, st>>>(lo, s, M, yring, sample);
}
void launch_learned_select(LsqOut* lo, int s, int M, int oldest, const float* yhat, int* used,
                           double* rho_net, cudaStream_t st) {
    learned_select_kernel<<<1, 128, 0, st>>>(lo, s, M, oldest, yhat, used, rho_net);
}
void launch_yring_push(double* yring, const LsqOut* lo, int M, cudaStream_t st) {
    yring_push_kernel<<<1, 32, 0, st>>>(yring, lo, M);
}

}  // namespace sa

using namespace sa;

struct seq_mlp {
    int M, s, in, hid, out, bmax, stride;
    cudaStream_t stream;
    size_t oW1, ob1, oW2, ob2, oW3, ob3, np;
    float *P = nullptr, *G = nullptr, *Mm = nullptr, *Vv = nullptr;
    uint16_t* Wb = nullptr;            // bf16 W1 | W2 | W3
    float *mu = nullptr, *sd = nullptr, *sig = nullptr;
    float *z, *a1, *h1, *a2, *h2, *d, *y, *dd, *dh2, *dh1, *loss, *batch, *scalar;
    int* idx = nullptr;
    int t = 0;
    std::vector<void*> allocs;
};

namespace {

int mlp_alloc(seq_mlp* m, void** p, size_t bytes) {
    if (cudaMalloc(p, bytes ? bytes : 4) != cudaSuccess) {
        cudaGetLastError();
        return SEQ_ENOMEM;
    }
    m->allocs.push_back(*p);
    return SEQ_OK;
}

void refresh_bf16(seq_mlp* m) {
    const size_t n1 = (size_t)m->hid * m->in, n2 = (size_t)m->hid * m->hid, n3 = (size_t)m->out * m->hid;
    to_bf16_kernel<<<64, 256, 0, m->stream>>>(m->P + m->oW1, m->Wb, n1);
    to_bf16_kernel<<<64, 256, 0, m->stream>>>(m->P + m->oW2, m->Wb + n1, n2);
    to_bf16_kernel<<<16, 256, 0, m->stream>>>(m->P + m->oW3, m->Wb + n1 + n2, n3);
}

// Forward pass on B samples (rows of S with the sample stride).
void mlp_forward(seq_mlp* m, const float* S, int stride, int B, cudaStream_t st) {
    const size_t n1 = (size_t)m->hid * m->in, n2 = (size_t)m->hid * m->hid;
    normalize_kernel<<<(B * m->in + 255) / 256, 256, 0, st>>>(S, stride, B, m->in, m->mu, m->sd, m->z);
    dim3 blk(TB, TB);
    linear_fwd<<<dim3((m->hid + TB - 1) / TB, (B + TB - 1) / TB), blk, 0, st>>>(
        m->z, m->in, m->Wb, m->P + m->ob1, B, m->hid, m->in, m->a1, m->h1);
    linear_fwd<<<dim3((m->hid + TB - 1) / TB, (B + TB - 1) / TB), blk, 0, st>>>(
        m->h1, m->hid, m->Wb + n1, m->P + m->ob2, B, m->hid, m->hid, m->a2, m->h2);
    linear_fwd<<<dim3((m->out + TB - 1) / TB, (B + TB - 1) / TB), blk, 0, st>>>(
        m->h2, m->hid, m->Wb + n1 + n2, m->P + m->ob3, B, m->out, m->hid, m->d, nullptr);
}

// Loss and gradients (into m->G) on B samples.
void mlp_backward(seq_mlp* m, const float* S, int stride, int B) {
    const size_t n1 = (size_t)m->hid * m->in, n2 = (size_t)m->hid * m->hid;
    head_kernel<<<(B + 127) / 128, 128, 0, m->stream>>>(S, stride, B, m->out, m->d, m->sig, m->in, m->y,
                                                        m->dd, m->loss);
    dim3 blk(TB, TB);
    linear_bwd_weight<<<dim3((m->hid + TB - 1) / TB, (m->out + TB - 1) / TB), blk, 0, m->stream>>>(
        m->dd, m->h2, m->hid, B, m->out, m->hid, m->G + m->oW3, m->G + m->ob3);
    linear_bwd_input<<<dim3((m->hid + TB - 1) / TB, (B + TB - 1) / TB), blk, 0, m->stream>>>(
        m->dd, m->Wb + n1 + n2, m->a2, B, m->out, m->hid, m->dh2);
    linear_bwd_weight<<<dim3((m->hid + TB - 1) / TB, (m->hid + TB - 1) / TB), blk, 0, m->stream>>>(
        m->dh2, m->h1, m->hid, B, m->hid, m->hid, m->G + m->oW2, m->G + m->ob2);
    linear_bwd_input<<<dim3((m->hid + TB - 1) / TB, (B + TB - 1) / TB), blk, 0, m->stream>>>(
        m->dh2, m->Wb + n1, m->a1, B, m->hid, m->hid, m->dh1);
    linear_bwd_weight<<<dim3((m->in + TB - 1) / TB, (m->hid + TB - 1) / TB), blk, 0, m->stream>>>(
        m->dh1, m->z, m->in, B, m->hid, m->in, m->G + m->oW1, m->G + m->ob1);
    sum_kernel<<<1, 1, 0, m->stream>>>(m->loss, B, m->scalar);
}

}  // namespace

namespace sa {
// Prediction on stream st (the predictor's activations are reused: not
// concurrently with training on another stream).
void mlp_predict_dev(seq_mlp* m, const float* features, int B, float* y, cudaStream_t st) {
    mlp_forward(m, features, m->stride, B, st);
    head_kernel<<<(B + 127) / 128, 128, 0, st>>>(features, m->stride, B, m->out, m->d, m->sig,
                                                 m->in, y, nullptr, nullptr);
}
int mlp_stride(const seq_mlp* m) { return m->stride; }
int mlp_dims_ok(const seq_mlp* m, int M, int s) { return m && m->M == M && m->s == s; }
int mlp_hidden(const seq_mlp* m) { return m ? m->hid : 0; }
int mlp_max_batch(const seq_mlp* m) { return m ? m->bmax : 0; }
}  // namespace sa

extern "C" {

int seq_mlp_create(int32_t M, int32_t s, int32_t hidden, int32_t max_batch, uint64_t seed,
                   void* cuda_stream, seq_mlp** out) {
    if (!out) return SEQ_EINVAL;
    *out = nullptr;
    if (M < 2 || M > kMaxM || s < M + 1 || s > kMaxS || hidden < 1 || hidden > 4096 ||
        max_batch < 1 || max_batch > 65536)
        return SEQ_EINVAL;
    seq_mlp* m = new seq_mlp();
    m->M = M;
    m->s = s;
    m->in = 4 * M + s;
    m->hid = hidden;
    m->out = M;
    m->bmax = max_batch;
    m->stride = m->in + M + M * M + 1;
    m->stream = (cudaStream_t)cuda_stream;
    m->oW1 = 0;
    m->ob1 = m->oW1 + (size_t)m->hid * m->in;
    m->oW2 = m->ob1 + m->hid;
    m->ob2 = m->oW2 + (size_t)m->hid * m->hid;
    m->oW3 = m->ob2 + m->hid;
    m->ob3 = m->oW3 + (size_t)m->out * m->hid;
    m->np = m->ob3 + m->out;
    int rc = SEQ_OK;
    void* p;
    auto A = [&](float** dst, size_t nfl) {
        if (rc == SEQ_OK) {
            rc = mlp_alloc(m, &p, nfl * sizeof(float));
            *dst = (float*)p;
        }
    };
    A(&m->P, m->np);
    A(&m->G, m->np);
    A(&m->Mm, m->np);
    A(&m->Vv, m->np);
    A(&m->mu, m->in);
    A(&m->sd, m->in);
    A(&m->sig, m->out);
    const size_t B = m->bmax;
    A(&m->z, B * m->in);
    A(&m->a1, B * m->hid);
    A(&m->h1, B * m->hid);
    A(&m->a2, B * m->hid);
    A(&m->h2, B * m->hid);
    A(&m->d, B * m->out);
    A(&m->y, B * m->out);
    A(&m->dd, B * m->out);
    A(&m->dh2, B * m->hid);
    A(&m->dh1, B * m->hid);
    A(&m->loss, B);
    A(&m->batch, B * m->stride);
    A(&m->scalar, 4);
    if (rc == SEQ_OK) {
        rc = mlp_alloc(m, &p, sizeof(uint16_t) * ((size_t)m->hid * m->in + (size_t)m->hid * m->hid +
                                                   (size_t)m->out * m->hid));
        m->Wb = (uint16_t*)p;
    }
    if (rc == SEQ_OK) {
        rc = mlp_alloc(m, &p, sizeof(int) * B);
        m->idx = (int*)p;
    }
    if (rc != SEQ_OK) {
        seq_mlp_destroy(m);
        return rc;
    }
    cudaMemsetAsync(m->P, 0, sizeof(float) * m->np, m->stream);
    cudaMemsetAsync(m->Mm, 0, sizeof(float) * m->np, m->stream);
    cudaMemsetAsync(m->Vv, 0, sizeof(float) * m->np, m->stream);
    he_init_kernel<<<64, 256, 0, m->stream>>>(m->P + m->oW1, (size_t)m->hid * m->in, m->in, seed, 0);
    he_init_kernel<<<64, 256, 0, m->stream>>>(m->P + m->oW2, (size_t)m->hid * m->hid, m->hid, seed,
                                              (uint64_t)m->hid * m->in);
    he_init_kernel<<<16, 256, 0, m->stream>>>(m->P + m->oW3, (size_t)m->out * m->hid, m->hid, seed,
                                              (uint64_t)m->hid * m->in + (uint64_t)m->hid * m->hid);
    std::vector<float> ones(m->in, 1.f);
    cudaMemsetAsync(m->mu, 0, sizeof(float) * m->in, m->stream);
    cudaMemcpy(m->sd, ones.data(), sizeof(float) * m->in, cudaMemcpyHostToDevice);
    cudaMemcpy(m->sig, ones.data(), sizeof(float) * m->out, cudaMemcpyHostToDevice);
    refresh_bf16(m);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        seq_mlp_destroy(m);
        return SEQ_ECUDA;
    }
    *out = m;
    return SEQ_OK;
}

int seq_mlp_destroy(seq_mlp* m) {
    if (!m) return SEQ_OK;
    cudaStreamSynchronize(m->stream);
    for (void* p : m->allocs) cudaFree(p);
    delete m;
    return SEQ_OK;
}

int seq_mlp_param_count(const seq_mlp* m) { return m ? (int)m->np : 0; }

int seq_mlp_get_params(seq_mlp* m, float* params_host, float* norm_host) {
    if (!m) return SEQ_EINVAL;
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return SEQ_ECUDA;
    if (params_host && cudaMemcpy(params_host, m->P, sizeof(float) * m->np, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SEQ_ECUDA;
    if (norm_host) {
        if (cudaMemcpy(norm_host, m->mu, sizeof(float) * m->in, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(norm_host + m->in, m->sd, sizeof(float) * m->in, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(norm_host + 2 * m->in, m->sig, sizeof(float) * m->out, cudaMemcpyDeviceToHost) != cudaSuccess)
            return SEQ_ECUDA;
    }
    return SEQ_OK;
}

int seq_mlp_set_params(seq_mlp* m, const float* params_host, const float* norm_host) {
    if (!m) return SEQ_EINVAL;
    if (params_host && cudaMemcpyAsync(m->P, params_host, sizeof(float) * m->np, cudaMemcpyHostToDevice,
                                       m->stream) != cudaSuccess)
        return SEQ_ECUDA;
    if (norm_host) {
        cudaMemcpyAsync(m->mu, norm_host, sizeof(float) * m->in, cudaMemcpyHostToDevice, m->stream);
        cudaMemcpyAsync(m->sd, norm_host + m->in, sizeof(float) * m->in, cudaMemcpyHostToDevice, m->stream);
        cudaMemcpyAsync(m->sig, norm_host + 2 * m->in, sizeof(float) * m->out, cudaMemcpyHostToDevice, m->stream);
    }
    refresh_bf16(m);
    m->t = 0;
    cudaMemsetAsync(m->Mm, 0, sizeof(float) * m->np, m->stream);
    cudaMemsetAsync(m->Vv, 0, sizeof(float) * m->np, m->stream);
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? SEQ_OK : SEQ_ECUDA;
}

int seq_mlp_fit_normalization(seq_mlp* m, const float* samples_dev, int32_t count) {
    if (!m || !samples_dev || count < 1) return SEQ_EINVAL;
    norm_stats_kernel<<<(m->in + m->out + 127) / 128, 128, 0, m->stream>>>(samples_dev, m->stride, count,
                                                                          m->in, m->out, m->mu, m->sd, m->sig);
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? SEQ_OK : SEQ_ECUDA;
}

int seq_mlp_loss_grad(seq_mlp* m, const float* samples_dev, int32_t B, float* loss_host,
                      float* grads_host) {
    if (!m || !samples_dev || B < 1 || B > m->bmax) return SEQ_EINVAL;
    mlp_forward(m, samples_dev, m->stride, B, m->stream);
    mlp_backward(m, samples_dev, m->stride, B);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return SEQ_ECUDA;
    if (loss_host && cudaMemcpy(loss_host, m->scalar, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SEQ_ECUDA;
    if (grads_host && cudaMemcpy(grads_host, m->G, sizeof(float) * m->np, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SEQ_ECUDA;
    return SEQ_OK;
}

int seq_mlp_train(seq_mlp* m, const float* samples_dev, int32_t count, int32_t epochs, int32_t batch,
                  float lr, uint64_t seed, float* losses_host) {
    if (!m || !samples_dev || count < 1 || epochs < 0 || batch < 1 || batch > m->bmax || !(lr > 0))
        return SEQ_EINVAL;
    std::vector<int> perm(count);
    std::vector<float> ep_loss(epochs > 0 ? epochs : 1, 0.f);
    uint64_t ctr = 0;
    for (int e = 0; e < epochs; ++e) {
        for (int i = 0; i < count; ++i) perm[i] = i;
        for (int i = count - 1; i > 0; --i) {          // Fisher-Yates with SplitMix64 draws
            uint64_t z = seed + (++ctr) * 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            const int j = (int)(((z >> 32) * (uint64_t)(i + 1)) >> 32);
            std::swap(perm[i], perm[j]);
        }
        double acc = 0;
        int nb = 0;
        for (int b0 = 0; b0 + batch <= count; b0 += batch) {
            cudaMemcpyAsync(m->idx, perm.data() + b0, sizeof(int) * batch, cudaMemcpyHostToDevice, m->stream);
            gather_kernel<<<128, 256, 0, m->stream>>>(samples_dev, m->idx, batch, m->stride, m->batch);
            mlp_forward(m, m->batch, m->stride, batch, m->stream);
            mlp_backward(m, m->batch, m->stride, batch);
            m->t += 1;
            const float c1 = 1.f - powf(0.9f, (float)m->t), c2 = 1.f - powf(0.999f, (float)m->t);
            adam_kernel<<<256, 256, 0, m->stream>>>(m->P, m->G, m->Mm, m->Vv, m->np, lr, 0.9f, 0.999f,
                                                    1e-8f, c1, c2);
            refresh_bf16(m);
            float l = 0.f;
            cudaMemcpyAsync(&l, m->scalar, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
            if (cudaStreamSynchronize(m->stream) != cudaSuccess) return SEQ_ECUDA;
            acc += l;
            ++nb;
        }
        ep_loss[e] = nb ? (float)(acc / nb) : 0.f;
    }
    if (losses_host && epochs > 0) memcpy(losses_host, ep_loss.data(), sizeof(float) * epochs);
    return cudaGetLastError() == cudaSuccess ? SEQ_OK : SEQ_ECUDA;
}

int seq_mlp_predict(seq_mlp* m, const float* samples_dev, int32_t B, float* y_dev) {
    if (!m || !samples_dev || !y_dev || B < 1 || B > m->bmax) return SEQ_EINVAL;
    mlp_predict_dev(m, samples_dev, B, y_dev, m->stream);
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? SEQ_OK : SEQ_ECUDA;
}

}  // extern "C"
