// Batched form: many independent sequences advance one time step in a single
// persistent launch (captured in a CUDA graph; one graph launch per step).
//
// Each thread block pulls sequences from a device work queue (largest first
// by default, the order the autotuner picked otherwise) and runs the whole
// step of one sequence with block barriers only -- there is no grid-wide
// wait anywhere, so blocks never spin on one another:
//   1. guess (Algorithm 1): W = S [A X | b] accumulated in shared
//      memory (the sparse-sign S generated on the fly from its counters),
//      the column-scaled pivoted Householder least squares in shared memory,
//      x0 = X y with FP64 accumulation;
//   2. FP64 iterative refinement around FP32 CG (the solve): r = b - A x in FP64,
//      inner CG on A32 d = r to a relative tolerance
//      max(inner_tol, theta tol ||b|| / ||r||), x += d, until ||r|| <= tol ||b||;
//   3. push x into the sequence's history ring (FP64).
// Inputs per step are device arrays owned by the caller; the per-sequence
// descriptors live in a device array refreshed by seq_batch_step.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/seqaccel.h"
#include "common.cuh"
#include "internal.h"

namespace sa {
namespace {

constexpr int kBatchMaxM = 16;
constexpr int kBatchMaxS = 64;
constexpr int kSketchWarps = 8;           // warps with a private copy of W
constexpr double kTheta = 0.5;
constexpr int kOk = 0;

struct BatchSeq {
    // fixed for the life of the batch
    int n, nnz, M, s, zeta, ldx;
    uint64_t seed;
    const int* rowptr;
    const int* colind;
    double* X;                             // history ring, n x ldx (FP64)
    float* val32;                          // zeros (source of the SELL padding fill)
    const int* soff;                       // SELL-32 copy of the pattern for the FP32 CG:
    const int* scol;                       //   slice offsets, padded column indices,
    float* sval;                           //   values refreshed every step (FP32)
    float *r, *p, *q, *d;                  // FP32 CG vectors (16-byte aligned, stride nv)
    // per step
    const double* val;
    const double* b;
    double* x;
    // state and outputs
    int pushes;
    int iters, refinements, status, history_cols, rank;
    double guess_relres, sketch_resid, final_relres;
};

struct BatchParams {
    double tol;
    double inner_tol;
    int max_iters;
    int commit;          // 1: push the solution into the history and keep the state
};

template <typename T>
__device__ __forceinline__ T btotal(T v, T* sred) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sred[warp] = v;
    __syncthreads();
    T t = 0;
    for (int w = 0; w < nw; ++w) t += sred[w];
    return t;
}

template <typename VT, typename XT, typename Acc>
__device__ __forceinline__ Acc row_dot(const int* __restrict__ rowptr, const int* __restrict__ colind,
                                       const VT* __restrict__ val, const XT* x, int i, int n,
                                       int nnz, int& bad) {
    const int rs = max(0, min(rowptr[i], nnz));
    const int re = max(rs, min(rowptr[i + 1], nnz));
    Acc acc = 0;
    for (int e = rs; e < re; ++e) {
        const int c = colind[e];
        if ((unsigned)c < (unsigned)n)
            acc = fma((Acc)val[e], (Acc)x[c], acc);
        else
            bad = 1;
    }
    return acc;
}

__device__ void sketch_column_b(int j, int s, int zeta, uint64_t seed, uint16_t* out) {
    int rows[kMaxZeta];
    int cnt = 0;
    for (int c = 0; c < 256 && cnt < zeta; ++c) {
        const uint64_t h = mix64(seed + ((uint64_t)j * 256ull + (uint64_t)(c + 1)) *
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

// The sketched block W (s x (M+1), physical history slots, b last) of rows
// [r_lo, r_hi) of one sequence, summed into Wsum (shared).  Warps
// 0..kSketchWarps-1 keep private copies; rows are taken in batches of 32 per
// warp, lane l building the sketch column of row base + l; the copies are
// added in warp order.
__device__ void block_sketch(const BatchSeq& q, double* Wpriv, uint16_t* sks, double* Wsum,
                             int& bad, int r_lo, int r_hi) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncol = q.M + 1, wsz = q.s * ncol;
    const int nsw = min(kSketchWarps, (int)(blockDim.x >> 5));
    for (int i = threadIdx.x; i < nsw * wsz; i += blockDim.x) Wpriv[i] = 0.0;
    __syncthreads();
    if (warp < nsw) {
        double* Ww = Wpriv + warp * wsz;
        uint16_t* sk = sks + warp * 32 * kMaxZeta;
        for (int base = r_lo + warp * 32; base < r_hi; base += nsw * 32) {
            if (base + lane < r_hi) sketch_column_b(base + lane, q.s, q.zeta, q.seed, sk + lane * kMaxZeta);
            __syncwarp();
            const int cnt = min(32, r_hi - base);
            for (int u = 0; u < cnt; ++u) {
                const int r = base + u;
                double y = 0.0;
                if (lane < q.M) {
                    const int rs = max(0, min(q.rowptr[r], q.nnz));
                    const int re = max(rs, min(q.rowptr[r + 1], q.nnz));
                    for (int e = rs; e < re; ++e) {
                        const int c = q.colind[e];
                        if ((unsigned)c < (unsigned)q.n)
                            y = fma(q.val[e], q.X[(size_t)c * q.ldx + lane], y);
                        else
                            bad = 1;
                    }
                } else if (lane == q.M) {
                    y = q.b[r];
                }
                if (lane < ncol) {
                    for (int k = 0; k < q.zeta; ++k) {
                        const unsigned e = sk[u * kMaxZeta + k];
                        double* dst = Ww + (e & 0x7fff) * ncol + lane;
                        *dst = (e & 0x8000) ? *dst - y : *dst + y;
                    }
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    const double inv = 1.0 / sqrt((double)q.zeta);
    for (int i = threadIdx.x; i < wsz; i += blockDim.x) {
        double acc = Wpriv[i];
        for (int w = 1; w < nsw; ++w) acc += Wpriv[w * wsz + i];
        Wsum[i] = acc * inv;
    }
    __syncthreads();
}

// Column-scaled, pivoted Householder least squares of the s x m block (the
// same steps as the single-sequence kernel), all in shared memory.  Returns
// y per physical slot in yphys (zeros for unused or truncated slots).
__device__ void block_lsq(const double* Wsum, int s, int M, int m, int oldest, double tau,
                          double* ws, double* yphys, int* rank_out, double* rho_out) {
    double* B = ws;               // s*m
    double* Wo = B + s * m;       // s*m
    double* c = Wo + s * m;       // s
    double* cb = c + s;           // s
    double* v = cb + s;           // s
    double* d = v + s;            // m
    double* nrm = d + m;          // m
    double* rdiag = nrm + m;      // m
    double* z = rdiag + m;        // m
    double* ylog = z + m;         // m
    __shared__ int perm[kBatchMaxM], live[kBatchMaxM];
    __shared__ double sh_normx, sh_vtv, sh_rho[32];
    __shared__ int sh_p, sh_rank;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int bd = blockDim.x, ncol = M + 1;
    for (int i = tid; i < s * m; i += bd) {
        const int l = i / s, qq = i - l * s;
        Wo[i] = Wsum[qq * ncol + (oldest + l) % M];
    }
    for (int qq = tid; qq < s; qq += bd) c[qq] = cb[qq] = Wsum[qq * ncol + M];
    __syncthreads();
    for (int l = warp; l < m; l += nw) {
        double a = 0.0;
        for (int qq = lane; qq < s; qq += 32) a += Wo[l * s + qq] * Wo[l * s + qq];
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
            for (int qq = k + lane; qq < s; qq += 32) a += B[l * s + qq] * B[l * s + qq];
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
            for (int qq = tid; qq < s; qq += bd) {
                const double t = B[k * s + qq];
                B[k * s + qq] = B[p * s + qq];
                B[p * s + qq] = t;
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
            for (int qq = k + lane; qq < s; qq += 32) a += B[k * s + qq] * B[k * s + qq];
            a = warp_sum(a);
            if (lane == 0) sh_normx = sqrt(a);
        }
        __syncthreads();
        const double normx = sh_normx;
        if (normx == 0.0 || !live[perm[k]]) break;
        const double alpha = B[k * s + k] >= 0.0 ? -normx : normx;
        for (int qq = k + tid; qq < s; qq += bd) v[qq] = B[k * s + qq] - (qq == k ? alpha : 0.0);
        __syncthreads();
        if (warp == 0) {
            double a = 0.0;
            for (int qq = k + lane; qq < s; qq += 32) a += v[qq] * v[qq];
            a = warp_sum(a);
            if (lane == 0) sh_vtv = a;
        }
        __syncthreads();
        const double vtv = sh_vtv;
        if (vtv > 0.0) {
            for (int l = k + 1 + warp; l <= m; l += nw) {
                double* col = (l < m) ? B + l * s : c;
                double a = 0.0;
                for (int qq = k + lane; qq < s; qq += 32) a += v[qq] * col[qq];
                a = warp_sum(a);
                const double t = (2.0 / vtv) * a;
                for (int qq = k + lane; qq < s; qq += 32) col[qq] -= v[qq] * t;
            }
        }
        __syncthreads();
        for (int qq = k + tid; qq < s; qq += bd) B[k * s + qq] = (qq == k) ? alpha : 0.0;
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
    double part = 0.0;
    for (int qq = tid; qq < s; qq += bd) {
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc += Wo[l * s + qq] * ylog[l];
        const double e = acc - cb[qq];
        part += e * e;
    }
    part = warp_sum(part);
    if (lane == 0) sh_rho[warp] = part;
    __syncthreads();
    if (tid < M) yphys[tid] = 0.0;
    __syncthreads();
    for (int l = tid; l < m; l += bd) yphys[(oldest + l) % M] = ylog[l];
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sh_rho[w];
        *rho_out = sqrt(t);
        *rank_out = sh_rank;
    }
    __syncthreads();
}

// FP32 CG on A32 d = rhs (d from 0) to ||rhs - A32 d|| <= itol ||rhs||, in
// one block; returns iterations (negative status on breakdown).
// FP32 SELL-32 product of one sequence by a whole block: warp per 32-row
// slice (lane = row); for every slice the index and value loads are issued
// first (coalesced), then the gathers, then the row sums in CSR order.  Padding (column -1) costs no arithmetic; a
// column >= n is skipped and flagged.  Row results go to epi(row, value).
constexpr int kBW = 5;      // 5-point stencils: every slice fits; wider rows take the loop

// Slices [s_lo, s_hi); rows outside [r_lo, r_hi) were written by other
// thread blocks of the launch and are read through L2 only.
template <typename Epi>
__device__ __forceinline__ void bsell_spmv(const BatchSeq& q, const float* __restrict__ x, int nw,
                                           int* bad, Epi& epi, int s_lo, int s_hi, int r_lo,
                                           int r_hi) {
    // Two slices per warp and iteration: both slices' index and value loads
    // and the epilogue's row operand are in flight together, then the gathers.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n = q.n;
    const int ns = s_hi;
    int flag = 0;
    for (int sl0 = s_lo + warp; sl0 < ns; sl0 += 2 * nw) {
        int o[2], w[2], r[2];
        bool live[2];
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const int sl = sl0 + g * nw;
            live[g] = sl < ns;
            o[g] = live[g] ? q.soff[sl] : 0;
            w[g] = live[g] ? (q.soff[sl + 1] - o[g]) >> 5 : 0;
            r[g] = sl * 32 + lane;
        }
        float a[2] = {0.f, 0.f};
        typename Epi::Pre pre[2];
#pragma unroll
        for (int g = 0; g < 2; ++g)
            if (live[g] && r[g] < n) pre[g] = epi.pre(r[g]);
        if (w[0] <= kBW && w[1] <= kBW) {
            int c[2][kBW];
            float v[2][kBW], xv[2][kBW];
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int k = 0; k < kBW; ++k) {
                    c[g][k] = k < w[g] ? q.scol[o[g] + k * 32 + lane] : -1;
                    v[g][k] = k < w[g] ? q.sval[o[g] + k * 32 + lane] : 0.f;
                }
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int k = 0; k < kBW; ++k) {
                    const int cc = c[g][k];
                    xv[g][k] = (unsigned)cc < (unsigned)n
                                   ? (cc >= r_lo && cc < r_hi ? x[cc] : __ldcg(x + cc))
                                   : 0.f;
                    flag |= cc >= n;
                }
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int k = 0; k < kBW; ++k)
                    if (k < w[g]) a[g] = fmaf(v[g][k], xv[g][k], a[g]);
        } else {
#pragma unroll
            for (int g = 0; g < 2; ++g)
                for (int k = 0; k < w[g]; ++k) {
                    const int cc = q.scol[o[g] + k * 32 + lane];
                    if ((unsigned)cc < (unsigned)n)
                        a[g] = fmaf(q.sval[o[g] + k * 32 + lane],
                                    cc >= r_lo && cc < r_hi ? x[cc] : __ldcg(x + cc), a[g]);
                    else
                        flag |= cc >= n;
                }
        }
#pragma unroll
        for (int g = 0; g < 2; ++g)
            if (live[g] && r[g] < n) epi(r[g], a[g], pre[g]);
    }
    if (flag) atomicOr(bad, 1);
}

struct CgProductEpi {
    float* qv;
    const float* p;
    float acc;
    using Pre = float;
    __device__ float pre(int r) const { return p[r]; }
    __device__ void operator()(int r, float a, float pr) {
        qv[r] = a;
        acc = fmaf(pr, a, acc);
    }
};

__device__ int block_cg32(const BatchSeq& q, double itol, int max_iters, float* sred, float* stage,
                          int* sbad, int& status) {
    // Vector phases use 16-byte loads over the first 4 floor(n / 4) entries
    // (the vectors are 16-byte aligned), then the ragged tail.
    const int n4 = q.n >> 2;
    float4* r4 = reinterpret_cast<float4*>(q.r);
    float4* p4 = reinterpret_cast<float4*>(q.p);
    float4* q4 = reinterpret_cast<float4*>(q.q);
    float4* d4 = reinterpret_cast<float4*>(q.d);
    (void)stage;
    const int n = q.n, tid = threadIdx.x, bd = blockDim.x;
    const int nw = bd >> 5;
    float rr_l = 0.f;
    for (int i = tid; i < n4; i += bd) {
        const float4 ri = r4[i];
        d4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        p4[i] = ri;
        rr_l = fmaf(ri.x, ri.x, rr_l);
        rr_l = fmaf(ri.y, ri.y, rr_l);
        rr_l = fmaf(ri.z, ri.z, rr_l);
        rr_l = fmaf(ri.w, ri.w, rr_l);
    }
    for (int i = 4 * n4 + tid; i < n; i += bd) {
        const float ri = q.r[i];
        q.d[i] = 0.f;
        q.p[i] = ri;
        rr_l = fmaf(ri, ri, rr_l);
    }
    float rr = btotal(rr_l, sred);
    // The stopping test ||r|| <= itol ||rhs|| on squares in FP32 (an FP64
    // square root per thread and iteration would cost microseconds of the
    // FP64 pipe on this GPU).
    const float target2 = (float)(itol * itol * (double)rr);
    int it = 0;
    status = kOk;
    if (!(rr > 0.f)) return 0;
    while (rr > target2) {
        if (it >= max_iters) {
            status = 1;
            break;
        }
        __syncthreads();
        CgProductEpi epi{q.q, q.p, 0.f};
        bsell_spmv(q, q.p, nw, sbad, epi, 0, (n + 31) >> 5, 0, n);
        const float pq = btotal(epi.acc, sred);
        if (!(pq > 0.f)) {
            status = isfinite(pq) ? -4 : -5;
            break;
        }
        const float alpha = rr / pq;
        float rn_l = 0.f;
        // Two float4 groups per thread and iteration, all loads issued before
        // the stores, so that twice the bytes are in flight per thread.
        for (int i = tid; i < n4; i += 2 * bd) {
            const int i1 = i + bd;
            const bool two = i1 < n4;
            float4 pv[2], qv[2], dv[2], rv[2];
            pv[0] = p4[i];
            qv[0] = q4[i];
            dv[0] = d4[i];
            rv[0] = r4[i];
            if (two) {
                pv[1] = p4[i1];
                qv[1] = q4[i1];
                dv[1] = d4[i1];
                rv[1] = r4[i1];
            }
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (g == 1 && !two) break;
                dv[g].x = fmaf(alpha, pv[g].x, dv[g].x);
                dv[g].y = fmaf(alpha, pv[g].y, dv[g].y);
                dv[g].z = fmaf(alpha, pv[g].z, dv[g].z);
                dv[g].w = fmaf(alpha, pv[g].w, dv[g].w);
                rv[g].x = fmaf(-alpha, qv[g].x, rv[g].x);
                rv[g].y = fmaf(-alpha, qv[g].y, rv[g].y);
                rv[g].z = fmaf(-alpha, qv[g].z, rv[g].z);
                rv[g].w = fmaf(-alpha, qv[g].w, rv[g].w);
                rn_l = fmaf(rv[g].x, rv[g].x, rn_l);
                rn_l = fmaf(rv[g].y, rv[g].y, rn_l);
                rn_l = fmaf(rv[g].z, rv[g].z, rn_l);
                rn_l = fmaf(rv[g].w, rv[g].w, rn_l);
            }
            d4[i] = dv[0];
            r4[i] = rv[0];
            if (two) {
                d4[i1] = dv[1];
                r4[i1] = rv[1];
            }
        }
        for (int i = 4 * n4 + tid; i < n; i += bd) {
            q.d[i] = fmaf(alpha, q.p[i], q.d[i]);
            const float ri = fmaf(-alpha, q.q[i], q.r[i]);
            q.r[i] = ri;
            rn_l = fmaf(ri, ri, rn_l);
        }
        const float rr_new = btotal(rn_l, sred);
        ++it;
        const float beta = rr_new / rr;
        rr = rr_new;
        for (int i = tid; i < n4; i += 2 * bd) {
            const int i1 = i + bd;
            const bool two = i1 < n4;
            float4 rv[2], pv[2];
            rv[0] = r4[i];
            pv[0] = p4[i];
            if (two) {
                rv[1] = r4[i1];
                pv[1] = p4[i1];
            }
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                pv[g].x = fmaf(beta, pv[g].x, rv[g].x);
                pv[g].y = fmaf(beta, pv[g].y, rv[g].y);
                pv[g].z = fmaf(beta, pv[g].z, rv[g].z);
                pv[g].w = fmaf(beta, pv[g].w, rv[g].w);
            }
            p4[i] = pv[0];
            if (two) p4[i1] = pv[1];
        }
        for (int i = 4 * n4 + tid; i < n; i += bd) q.p[i] = fmaf(beta, q.p[i], q.r[i]);
    }
    __syncthreads();
    return it;
}

// ---------------------------------------------------------------------------
// Cluster form: a thread-block cluster of C CTAs (one per SM) takes each
// sequence, CTA k owning a contiguous range of its 32-row slices.  Fewer
// sequences are in flight at once (one per cluster instead of one per SM), so
// their working sets stay in L2 between CG iterations.  Block totals are
// combined across the cluster through distributed shared memory: every CTA
// reads the C partial sums in rank order, so all CTAs hold bitwise the same
// total and take the same branches -- every cluster barrier below is reached
// by all CTAs the same number of times.
__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cl_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Cluster barrier; writes before it (shared and global) are visible after it.
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\t"
                 "barrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_map(const void* p, unsigned rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ double cl_ld(const double* p, unsigned rank) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(cl_map(p, rank)) : "memory");
    return v;
}
__device__ __forceinline__ float cl_ld(const float* p, unsigned rank) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(cl_map(p, rank)) : "memory");
    return v;
}
__device__ __forceinline__ int cl_ld(const int* p, unsigned rank) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(cl_map(p, rank)) : "memory");
    return v;
}

// Sum over the cluster of one block total per CTA (every thread gets it).
// slot: two shared words used alternately (par), bc: a shared word.
template <typename T>
__device__ __forceinline__ T cl_total(T blocktotal, T* slot, T* bc, int& par) {
    if (threadIdx.x == 0) slot[par] = blocktotal;
    cl_sync();
    if (threadIdx.x < 32) {
        const unsigned nr = cl_size();
        const T v = threadIdx.x < nr ? cl_ld(&slot[par], threadIdx.x) : (T)0;
        T t = 0;
        for (unsigned r = 0; r < nr; ++r) t += __shfl_sync(0xffffffffu, v, r);
        if (threadIdx.x == 0) *bc = t;
    }
    __syncthreads();
    const T t = *bc;
    par ^= 1;
    return t;
}

struct ClRed {
    double* dslot;
    double* dbc;
    float* fslot;
    float* fbc;
    int dpar, fpar;
};

// FP32 CG of block_cg32 on the rows [r_lo, r_hi) (slices [s_lo, s_hi)) of
// this CTA, totals over the cluster.
__device__ int cluster_cg32(const BatchSeq& q, double itol, int max_iters, float* sred, int* sbad,
                            int s_lo, int s_hi, int r_lo, int r_hi, ClRed& red, int& status) {
    const int i4lo = r_lo >> 2, i4hi = r_hi >> 2;
    float4* r4 = reinterpret_cast<float4*>(q.r);
    float4* p4 = reinterpret_cast<float4*>(q.p);
    float4* q4 = reinterpret_cast<float4*>(q.q);
    float4* d4 = reinterpret_cast<float4*>(q.d);
    const int tid = threadIdx.x, bd = blockDim.x, nw = bd >> 5;
    float rr_l = 0.f;
    for (int i = i4lo + tid; i < i4hi; i += bd) {
        const float4 ri = r4[i];
        d4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        p4[i] = ri;
        rr_l = fmaf(ri.x, ri.x, rr_l);
        rr_l = fmaf(ri.y, ri.y, rr_l);
        rr_l = fmaf(ri.z, ri.z, rr_l);
        rr_l = fmaf(ri.w, ri.w, rr_l);
    }
    for (int i = max(r_lo, 4 * i4hi) + tid; i < r_hi; i += bd) {
        const float ri = q.r[i];
        q.d[i] = 0.f;
        q.p[i] = ri;
        rr_l = fmaf(ri, ri, rr_l);
    }
    float rr = cl_total(btotal(rr_l, sred), red.fslot, red.fbc, red.fpar);
    const float target2 = (float)(itol * itol * (double)rr);
    int it = 0;
    status = kOk;
    if (!(rr > 0.f)) return 0;
    while (rr > target2) {
        if (it >= max_iters) {
            status = 1;
            break;
        }
        __syncthreads();
        CgProductEpi epi{q.q, q.p, 0.f};
        bsell_spmv(q, q.p, nw, sbad, epi, s_lo, s_hi, r_lo, r_hi);
        const float pq = cl_total(btotal(epi.acc, sred), red.fslot, red.fbc, red.fpar);
        if (!(pq > 0.f)) {
            status = isfinite(pq) ? -4 : -5;
            break;
        }
        const float alpha = rr / pq;
        float rn_l = 0.f;
        for (int i = i4lo + tid; i < i4hi; i += bd) {
            const float4 pv = p4[i], qv = q4[i];
            float4 dv = d4[i], rv = r4[i];
            dv.x = fmaf(alpha, pv.x, dv.x);
            dv.y = fmaf(alpha, pv.y, dv.y);
            dv.z = fmaf(alpha, pv.z, dv.z);
            dv.w = fmaf(alpha, pv.w, dv.w);
            rv.x = fmaf(-alpha, qv.x, rv.x);
            rv.y = fmaf(-alpha, qv.y, rv.y);
            rv.z = fmaf(-alpha, qv.z, rv.z);
            rv.w = fmaf(-alpha, qv.w, rv.w);
            d4[i] = dv;
            r4[i] = rv;
            rn_l = fmaf(rv.x, rv.x, rn_l);
            rn_l = fmaf(rv.y, rv.y, rn_l);
            rn_l = fmaf(rv.z, rv.z, rn_l);
            rn_l = fmaf(rv.w, rv.w, rn_l);
        }
        for (int i = max(r_lo, 4 * i4hi) + tid; i < r_hi; i += bd) {
            q.d[i] = fmaf(alpha, q.p[i], q.d[i]);
            const float ri = fmaf(-alpha, q.q[i], q.r[i]);
            q.r[i] = ri;
            rn_l = fmaf(ri, ri, rn_l);
        }
        const float rr_new = cl_total(btotal(rn_l, sred), red.fslot, red.fbc, red.fpar);
        ++it;
        const float beta = rr_new / rr;
        rr = rr_new;
        for (int i = i4lo + tid; i < i4hi; i += bd) {
            const float4 rv = r4[i];
            float4 pv = p4[i];
            pv.x = fmaf(beta, pv.x, rv.x);
            pv.y = fmaf(beta, pv.y, rv.y);
            pv.z = fmaf(beta, pv.z, rv.z);
            pv.w = fmaf(beta, pv.w, rv.w);
            p4[i] = pv;
        }
        for (int i = max(r_lo, 4 * i4hi) + tid; i < r_hi; i += bd) q.p[i] = fmaf(beta, q.p[i], q.r[i]);
        cl_sync();    // the new direction is complete before the next product gathers it
    }
    __syncthreads();
    return it;
}

// Shared-memory bytes of one block for sequences with at most s rows of
// sketch and M history columns.
size_t batch_smem_bytes(int s, int M) {
    const int ncol = M + 1, wsz = s * ncol;
    size_t d = (size_t)kSketchWarps * wsz + wsz + (2 * s * M + 3 * s + 5 * M) + kBatchMaxM;
    const size_t guess = d * sizeof(double) + (size_t)kSketchWarps * 32 * kMaxZeta * sizeof(uint16_t);
    const size_t stage = sizeof(double) * 32 * (size_t)kTileChunks * 32;   // up to 32 warps
    return guess > stage ? guess : stage;
}

// One time step of every sequence.  Blocks take sequences from the queue
// until it is empty; each sequence is processed by one block from start to
// end (no inter-block waiting).  MAXT: the largest block size the
// instantiation is launched with at one block per SM, which sets its register
// budget (65,536 / MAXT, at most 255): 1024 -> 64, 512 -> 128, 256 -> 255.
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
batched_step_kernel(BatchSeq* seqs, const int* __restrict__ order, int count, int* queue,
                    const BatchParams* __restrict__ prm) {
    extern __shared__ double smem[];
    __shared__ int sidx;
    __shared__ double dred[32];
    __shared__ float fred[32];
    __shared__ int sbad;
    const int tid = threadIdx.x, bd = blockDim.x;
    const BatchParams P = *prm;
    for (;;) {
        if (tid == 0) {
            sidx = atomicAdd(queue, 1);
            sbad = 0;
        }
        __syncthreads();
        const int idx = sidx;
        if (idx >= count) break;
        BatchSeq& gq = seqs[order[idx]];
        const BatchSeq q = gq;
        const int n = q.n, M = q.M, s = q.s;
        const int m = min(q.pushes, M);
        int bad = 0, rank = 0;
        double rho = 0.0;
        // 1. guess
        double* Wpriv = smem;
        double* Wsum = Wpriv + kSketchWarps * s * (M + 1);
        double* ws = Wsum + s * (M + 1);
        double* yphys = ws + (2 * s * M + 3 * s + 5 * M);
        uint16_t* sks = reinterpret_cast<uint16_t*>(yphys + kBatchMaxM);
        if (m == 0) {
            for (int i = tid; i < n; i += bd) q.x[i] = 0.0;
        } else {
            block_sketch(q, Wpriv, sks, Wsum, bad, 0, n);
            block_lsq(Wsum, s, M, m, (q.pushes - m) % M, 1e-12, ws, yphys, &rank, &rho);
            for (int i = tid; i < n; i += bd) {
                const double* row = q.X + (size_t)i * q.ldx;
                double acc = 0.0;
                for (int k = 0; k < M; ++k) acc = fma(row[k], yphys[k], acc);
                q.x[i] = acc;
            }
        }
        // This step's values into the SELL copy (FP32): entry k of row i goes
        // to soff[i / 32] + 32 k + i % 32.
        for (int i = tid; i < n; i += bd) {
            const int e0 = q.rowptr[i], e1 = q.rowptr[i + 1];
            float* dst = q.sval + q.soff[i >> 5] + (i & 31);
            for (int e = e0; e < e1; ++e) dst[(e - e0) * 32] = (float)q.val[e];
        }
        __syncthreads();
        // Warp-tile staging for the products (aliases the guess workspace).
        double* stage_d = smem;
        float* stage_f = reinterpret_cast<float*>(smem);
        const int lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
        // 2. FP64 refinement around FP32 CG
        double bb_l = 0.0;
        for (int i = tid; i < n; i += bd) bb_l = fma(q.b[i], q.b[i], bb_l);
        const double bnorm = sqrt(btotal(bb_l, dred));
        const double target = P.tol * bnorm;
        int total = 0, nref = 0, status = kOk;
        double rn = 0.0, first = 0.0;
        for (int pass = 0;; ++pass) {
            double rr_l = 0.0;
            for (int r0 = warp * 32; r0 < n; r0 += nw * 32) {
                const double ax = warp_tile_spmv<double>(q.rowptr, q.colind, q.val, q.x, n, q.nnz, r0,
                                                         stage_d + warp * kTileChunks * 32, &sbad);
                const int i = r0 + lane;
                if (i < n) {
                    const double ri = q.b[i] - ax;
                    q.r[i] = (float)ri;
                    rr_l = fma(ri, ri, rr_l);
                }
            }
            rn = sqrt(btotal(rr_l, dred));
            if (pass == 0) first = bnorm > 0.0 ? rn / bnorm : rn;
            if (!isfinite(rn)) {
                status = -5;
                break;
            }
            if (rn <= target) break;
            if (total >= P.max_iters || nref >= 100) {
                status = 1;
                break;
            }
            const double itol = fmax(P.inner_tol, kTheta * target / rn);
            int st = kOk;
            total += block_cg32(q, itol, P.max_iters - total, fred, stage_f, &sbad, st);
            ++nref;
            if (st < 0) {
                status = st;
                break;
            }
            for (int i = tid; i < n; i += bd) q.x[i] += (double)q.d[i];
            __syncthreads();
        }
        // 3. push
        if (P.commit && status >= 0) {
            const int slot = q.pushes % M;
            for (int i = tid; i < n; i += bd) q.X[(size_t)i * q.ldx + slot] = q.x[i];
        }
        if (bad) atomicOr(&sbad, 1);
        __syncthreads();
        if (tid == 0) {
            if (P.commit && status >= 0) gq.pushes = q.pushes + 1;
            gq.iters = total;
            gq.refinements = nref;
            gq.status = sbad ? -1 : status;
            gq.history_cols = m;
            gq.rank = rank;
            gq.guess_relres = first;
            gq.sketch_resid = rho;
            gq.final_relres = bnorm > 0.0 ? rn / bnorm : rn;
        }
        __syncthreads();
    }
}

// Shared-memory bytes of one CTA of the cluster form: the single-block layout
// plus the cluster total of W.
size_t batch_cluster_smem_bytes(int s, int M) {
    const size_t base = batch_smem_bytes(s, M);
    const int wsz = s * (M + 1);
    const size_t d = (size_t)kSketchWarps * wsz + wsz + (2 * s * M + 3 * s + 5 * M) + kBatchMaxM;
    const size_t guess = d * sizeof(double) + (size_t)kSketchWarps * 32 * kMaxZeta * sizeof(uint16_t);
    const size_t need = guess + (size_t)wsz * sizeof(double);
    return base > need ? base : need;
}

// One time step of every sequence, one cluster per sequence (see cl_sync and
// cl_total above).  The steps and their arithmetic are those of
// batched_step_kernel; rows are split over the cluster's CTAs and block
// totals (the sketch W, norms, CG dot products) are summed over the cluster.
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
batched_cluster_kernel(BatchSeq* seqs, const int* __restrict__ order, int count, int* queue,
                       const BatchParams* __restrict__ prm) {
    extern __shared__ double smem[];
    __shared__ int s_take, s_idx;
    __shared__ double dred[32];
    __shared__ float fred[32];
    __shared__ int sbad;
    __shared__ double dslot[2], dbc;
    __shared__ float fslot[2], fbc;
    const int tid = threadIdx.x, bd = blockDim.x;
    const unsigned rk = cl_rank(), nr = cl_size();
    const BatchParams P = *prm;
    ClRed red{dslot, &dbc, fslot, &fbc, 0, 0};
    for (;;) {
        if (rk == 0 && tid == 0) s_take = atomicAdd(queue, 1);
        if (tid == 0) sbad = 0;
        cl_sync();
        if (tid == 0) s_idx = cl_ld(&s_take, 0);
        __syncthreads();
        const int idx = s_idx;
        if (idx >= count) break;
        BatchSeq& gq = seqs[order[idx]];
        const BatchSeq q = gq;
        const int n = q.n, M = q.M, s = q.s;
        const int m = min(q.pushes, M);
        // This CTA's slices and rows.
        const int ns = (n + 31) >> 5;
        const int per = (ns + (int)nr - 1) / (int)nr;
        const int s_lo = min(ns, (int)rk * per), s_hi = min(ns, s_lo + per);
        const int r_lo = s_lo * 32, r_hi = min(n, s_hi * 32);
        int bad = 0, rank = 0;
        double rho = 0.0;
        // 1. guess
        const int ncol = M + 1, wsz = s * ncol;
        double* Wpriv = smem;
        double* Wsum = Wpriv + kSketchWarps * wsz;
        double* ws = Wsum + wsz;
        double* yphys = ws + (2 * s * M + 3 * s + 5 * M);
        uint16_t* sks = reinterpret_cast<uint16_t*>(yphys + kBatchMaxM);
        double* Wtot = reinterpret_cast<double*>(sks + kSketchWarps * 32 * kMaxZeta);
        if (m == 0) {
            for (int i = r_lo + tid; i < r_hi; i += bd) q.x[i] = 0.0;
        } else {
            block_sketch(q, Wpriv, sks, Wsum, bad, r_lo, r_hi);
            cl_sync();
            for (int i = tid; i < wsz; i += bd) {
                double t = 0.0;
                for (unsigned r = 0; r < nr; ++r) t += cl_ld(&Wsum[i], r);
                Wtot[i] = t;
            }
            cl_sync();   // every CTA has read the partial sums before they are overwritten
            block_lsq(Wtot, s, M, m, (q.pushes - m) % M, 1e-12, ws, yphys, &rank, &rho);
            for (int i = r_lo + tid; i < r_hi; i += bd) {
                const double* row = q.X + (size_t)i * q.ldx;
                double acc = 0.0;
                for (int k = 0; k < M; ++k) acc = fma(row[k], yphys[k], acc);
                q.x[i] = acc;
            }
        }
        // This step's values into the SELL copy (FP32), own rows.
        for (int i = r_lo + tid; i < r_hi; i += bd) {
            const int e0 = q.rowptr[i], e1 = q.rowptr[i + 1];
            float* dst = q.sval + q.soff[i >> 5] + (i & 31);
            for (int e = e0; e < e1; ++e) dst[(e - e0) * 32] = (float)q.val[e];
        }
        __syncthreads();
        double* stage_d = smem;
        const int lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
        // 2. FP64 refinement around FP32 CG (the x of other CTAs is complete
        // after the cluster total below)
        double bb_l = 0.0;
        for (int i = r_lo + tid; i < r_hi; i += bd) bb_l = fma(q.b[i], q.b[i], bb_l);
        const double bnorm = sqrt(cl_total(btotal(bb_l, dred), red.dslot, red.dbc, red.dpar));
        const double target = P.tol * bnorm;
        int total = 0, nref = 0, status = kOk;
        double rn = 0.0, first = 0.0;
        for (int pass = 0;; ++pass) {
            double rr_l = 0.0;
            for (int r0 = r_lo + warp * 32; r0 < r_hi; r0 += nw * 32) {
                const double ax = warp_tile_spmv<double, double, double, true>(
                    q.rowptr, q.colind, q.val, q.x, n, q.nnz, r0, stage_d + warp * kTileChunks * 32,
                    &sbad);
                const int i = r0 + lane;
                if (i < r_hi) {
                    const double ri = q.b[i] - ax;
                    q.r[i] = (float)ri;
                    rr_l = fma(ri, ri, rr_l);
                }
            }
            rn = sqrt(cl_total(btotal(rr_l, dred), red.dslot, red.dbc, red.dpar));
            if (pass == 0) first = bnorm > 0.0 ? rn / bnorm : rn;
            if (!isfinite(rn)) {
                status = -5;
                break;
            }
            if (rn <= target) break;
            if (total >= P.max_iters || nref >= 100) {
                status = 1;
                break;
            }
            const double itol = fmax(P.inner_tol, kTheta * target / rn);
            int st = kOk;
            total += cluster_cg32(q, itol, P.max_iters - total, fred, &sbad, s_lo, s_hi, r_lo, r_hi,
                                  red, st);
            ++nref;
            if (st < 0) {
                status = st;
                break;
            }
            for (int i = r_lo + tid; i < r_hi; i += bd) q.x[i] += (double)q.d[i];
            cl_sync();   // x complete before the next residual gathers it
        }
        // 3. push (own rows)
        if (P.commit && status >= 0) {
            const int slot = q.pushes % M;
            for (int i = r_lo + tid; i < r_hi; i += bd) q.X[(size_t)i * q.ldx + slot] = q.x[i];
        }
        if (bad) atomicOr(&sbad, 1);
        __syncthreads();
        const double anybad = cl_total((double)(sbad != 0), red.dslot, red.dbc, red.dpar);
        if (rk == 0 && tid == 0) {
            if (P.commit && status >= 0) gq.pushes = q.pushes + 1;
            gq.iters = total;
            gq.refinements = nref;
            gq.status = anybad > 0.0 ? -1 : status;
            gq.history_cols = m;
            gq.rank = rank;
            gq.guess_relres = first;
            gq.sketch_resid = rho;
            gq.final_relres = bnorm > 0.0 ? rn / bnorm : rn;
        }
        __syncthreads();
    }
    cl_sync();   // no CTA leaves while another may still read its shared memory
}

// The instantiation whose register budget fits `threads` x `blocks_per_sm`
// threads on one SM.
using StepKernel = void (*)(BatchSeq*, const int*, int, int*, const BatchParams*);
StepKernel step_kernel_for(int threads, int blocks_per_sm) {
    const int t = threads * blocks_per_sm;
    return t <= 256 ? batched_step_kernel<256> : t <= 512 ? batched_step_kernel<512>
                                                           : batched_step_kernel<1024>;
}

StepKernel cluster_kernel_for(int threads) {
    return threads <= 256 ? batched_cluster_kernel<256> : threads <= 512 ? batched_cluster_kernel<512>
                                                                        : batched_cluster_kernel<1024>;
}

__global__ void batch_push_kernel(const double* __restrict__ x, int n, double* X, int ldx, int slot) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        X[(size_t)i * ldx + slot] = x[i];
}

}  // namespace
}  // namespace sa

using namespace sa;

struct seq_batch {
    int count = 0, M = 0, s = 0, zeta = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    std::vector<BatchSeq> host;           // mirror of the device descriptors
    BatchSeq* h_pinned = nullptr;
    BatchSeq* d_seqs = nullptr;
    BatchParams* h_prm = nullptr;
    BatchParams* d_prm = nullptr;
    int* d_order = nullptr;
    int* d_queue = nullptr;
    std::vector<void*> allocs;
    int threads = 512, blocks_per_sm = 1, order_kind = 0;  // 0: largest first, 1: given order
    int cluster = 1;                      // CTAs per sequence (1: one block per sequence)
    size_t smem_cluster = 0;
    int autopush = 1;
    cudaGraphExec_t graph = nullptr;
    size_t smem = 0;
    int sms = 0;
};

namespace {

int batch_alloc(seq_batch* bt, void** p, size_t bytes) {
    if (cudaMalloc(p, bytes ? bytes : 1) != cudaSuccess) {
        cudaGetLastError();
        return SEQ_ENOMEM;
    }
    bt->allocs.push_back(*p);
    return SEQ_OK;
}

int batch_order(seq_batch* bt) {
    std::vector<int> ord(bt->count);
    for (int k = 0; k < bt->count; ++k) ord[k] = k;
    if (bt->order_kind == 0)
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
            return (long long)bt->host[a].nnz > (long long)bt->host[b].nnz;
        });
    if (cudaMemcpyAsync(bt->d_order, ord.data(), sizeof(int) * bt->count, cudaMemcpyHostToDevice,
                        bt->stream) != cudaSuccess)
        return SEQ_ECUDA;
    return cudaStreamSynchronize(bt->stream) == cudaSuccess ? SEQ_OK : SEQ_ECUDA;
}

// Launch configuration of the cluster form: clusters of bt->cluster CTAs, one
// CTA per SM, as many clusters as fit at once.  Returns the grid (0: none fits).
int cluster_grid(seq_batch* bt, StepKernel kern) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = bt->cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(bt->cluster * bt->sms);
    cfg.blockDim = dim3(bt->threads);
    cfg.dynamicSmemBytes = bt->smem_cluster;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, (const void*)kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // one CTA per SM
    nc = std::min(nc, bt->sms / bt->cluster);
    return nc * bt->cluster;
}

int batch_capture(seq_batch* bt) {
    if (bt->graph) {
        cudaGraphExecDestroy(bt->graph);
        bt->graph = nullptr;
    }
    const bool cl = bt->cluster > 1;
    const StepKernel kern = cl ? cluster_kernel_for(bt->threads)
                               : step_kernel_for(bt->threads, bt->blocks_per_sm);
    const size_t smem = cl ? bt->smem_cluster : bt->smem;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return SEQ_ECUDA;
    }
    int grid = bt->sms * bt->blocks_per_sm;
    if (cl) {
        if (bt->cluster > 8 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess) {
            cudaGetLastError();
            return SEQ_ECUDA;
        }
        grid = cluster_grid(bt, kern);
        if (grid <= 0) return SEQ_ECUDA;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return SEQ_ECUDA;
    cudaMemsetAsync(bt->d_queue, 0, sizeof(int), bt->cap);
    if (cl) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = bt->cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(bt->threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = bt->cap;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, kern, bt->d_seqs, (const int*)bt->d_order, bt->count, bt->d_queue,
                           (const BatchParams*)bt->d_prm);
    } else {
        kern<<<grid, bt->threads, smem, bt->cap>>>(bt->d_seqs, bt->d_order, bt->count, bt->d_queue,
                                                   bt->d_prm);
    }
    if (cudaStreamEndCapture(bt->cap, &g) != cudaSuccess) {
        cudaGetLastError();
        return SEQ_ECUDA;
    }
    cudaError_t e = cudaGraphInstantiate(&bt->graph, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? SEQ_OK : SEQ_ECUDA;
}

// Upload descriptors and parameters, launch the captured step, read back.
int batch_run(seq_batch* bt, const double* const* values, const double* const* b,
              double* const* x, double tol, int commit) {
    for (int k = 0; k < bt->count; ++k) {
        if (!values[k] || !b[k] || !x[k]) return SEQ_EINVAL;
        bt->host[k].val = values[k];
        bt->host[k].b = b[k];
        bt->host[k].x = x[k];
    }
    memcpy(bt->h_pinned, bt->host.data(), sizeof(BatchSeq) * bt->count);
    bt->h_prm->tol = tol;
    bt->h_prm->commit = commit;
    cudaMemcpyAsync(bt->d_seqs, bt->h_pinned, sizeof(BatchSeq) * bt->count,
                    cudaMemcpyHostToDevice, bt->stream);
    cudaMemcpyAsync(bt->d_prm, bt->h_prm, sizeof(BatchParams), cudaMemcpyHostToDevice, bt->stream);
    if (cudaGraphLaunch(bt->graph, bt->stream) != cudaSuccess) return SEQ_ECUDA;
    cudaMemcpyAsync(bt->h_pinned, bt->d_seqs, sizeof(BatchSeq) * bt->count,
                    cudaMemcpyDeviceToHost, bt->stream);
    if (cudaStreamSynchronize(bt->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return SEQ_ECUDA;
    memcpy(bt->host.data(), bt->h_pinned, sizeof(BatchSeq) * bt->count);
    return SEQ_OK;
}

}  // namespace

extern "C" {

int seq_batch_create(int32_t count, const seq_csr* patterns, int32_t M, int32_t s, int32_t zeta,
                     uint64_t seed, int32_t max_iters, double inner_tol, void* cuda_stream,
                     seq_batch** out) {
    if (!out) return SEQ_EINVAL;
    *out = nullptr;
    if (count <= 0 || !patterns || M < 1 || M > kBatchMaxM || s < M + 1 || s > kBatchMaxS ||
        zeta < 1 || zeta > s || zeta > kMaxZeta || max_iters < 0)
        return SEQ_EINVAL;
    for (int k = 0; k < count; ++k)
        if (patterns[k].n <= 0 || patterns[k].nnz < 0 || !patterns[k].rowptr ||
            (patterns[k].nnz > 0 && !patterns[k].colind))
            return SEQ_EINVAL;
    seq_batch* bt = new seq_batch();
    bt->count = count;
    bt->M = M;
    bt->s = s;
    bt->zeta = zeta;
    bt->stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&bt->sms, cudaDevAttrMultiProcessorCount, dev);
    bt->smem = batch_smem_bytes(s, M);
    bt->smem_cluster = batch_cluster_smem_bytes(s, M);
    bt->host.resize(count);
    int rc = SEQ_OK;
    const int ldx = (M + 1) & ~1;
    for (int k = 0; k < count && rc == SEQ_OK; ++k) {
        BatchSeq& q = bt->host[k];
        memset(&q, 0, sizeof(q));
        q.n = patterns[k].n;
        q.nnz = patterns[k].nnz;
        q.M = M;
        q.s = s;
        q.zeta = zeta;
        q.ldx = ldx;
        q.seed = seed + (uint64_t)k;
        q.rowptr = patterns[k].rowptr;
        q.colind = patterns[k].colind;
        void* p = nullptr;
        rc = batch_alloc(bt, &p, sizeof(double) * (size_t)q.n * ldx);
        if (rc) break;
        q.X = (double*)p;
        cudaMemsetAsync(q.X, 0, sizeof(double) * (size_t)q.n * ldx, bt->stream);
        rc = batch_alloc(bt, &p, sizeof(float) * (size_t)(q.nnz > 0 ? q.nnz : 1));
        if (rc) break;
        q.val32 = (float*)p;
        cudaMemsetAsync(q.val32, 0, sizeof(float) * (size_t)(q.nnz > 0 ? q.nnz : 1), bt->stream);
        // SELL-32 copy of the pattern (column indices once; the values are
        // written by the step kernel; padding stays column -1, value 0).
        const int ns = (q.n + 31) / 32;
        rc = batch_alloc(bt, &p, sizeof(int) * (size_t)ns);
        if (rc) break;
        int* width = (int*)p;
        rc = batch_alloc(bt, &p, sizeof(int) * (size_t)(ns + 2));     // + total, widest slice
        if (rc) break;
        int* off = (int*)p;
        launch_sell_layout(q.rowptr, q.n, q.nnz, width, off, bt->stream);
        int total = 0;
        if (cudaMemcpyAsync(&total, off + ns, sizeof(int), cudaMemcpyDeviceToHost, bt->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(bt->stream) != cudaSuccess) {
            rc = SEQ_ECUDA;
            break;
        }
        if (total < 0 || (long long)total > 2LL * q.nnz + 64LL * ns) {
            rc = SEQ_EINVAL;
            break;
        }
        rc = batch_alloc(bt, &p, sizeof(int) * (size_t)(total > 0 ? total : 1));
        if (rc) break;
        int* scol = (int*)p;
        rc = batch_alloc(bt, &p, sizeof(float) * (size_t)(total > 0 ? total : 1));
        if (rc) break;
        float* sval = (float*)p;
        launch_sell_fill_f32(q.rowptr, q.colind, q.val32, q.n, q.nnz, off, scol, sval, bt->stream);
        q.soff = off;
        q.scol = scol;
        q.sval = sval;
        const size_t nv = ((size_t)q.n + 3) & ~(size_t)3;     // 16-byte aligned vectors
        rc = batch_alloc(bt, &p, sizeof(float) * 4 * nv);
        if (rc) break;
        q.r = (float*)p;
        q.p = q.r + nv;
        q.q = q.p + nv;
        q.d = q.q + nv;
    }
    void* p = nullptr;
    if (rc == SEQ_OK) rc = batch_alloc(bt, &p, sizeof(BatchSeq) * count), bt->d_seqs = (BatchSeq*)p;
    if (rc == SEQ_OK) rc = batch_alloc(bt, &p, sizeof(BatchParams)), bt->d_prm = (BatchParams*)p;
    if (rc == SEQ_OK) rc = batch_alloc(bt, &p, sizeof(int) * count), bt->d_order = (int*)p;
    if (rc == SEQ_OK) rc = batch_alloc(bt, &p, sizeof(int)), bt->d_queue = (int*)p;
    if (rc == SEQ_OK && (cudaMallocHost(&bt->h_pinned, sizeof(BatchSeq) * count) != cudaSuccess ||
                         cudaMallocHost(&bt->h_prm, sizeof(BatchParams)) != cudaSuccess))
        rc = SEQ_ENOMEM;
    if (rc == SEQ_OK && cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking) != cudaSuccess)
        rc = SEQ_ECUDA;
    if (rc == SEQ_OK) {
        bt->h_prm->tol = 1e-8;
        bt->h_prm->inner_tol = inner_tol > 0 ? inner_tol : 1e-2;
        bt->h_prm->max_iters = max_iters;
        bt->h_prm->commit = 1;
        rc = batch_order(bt);
    }
    if (rc == SEQ_OK) rc = batch_capture(bt);
    if (rc != SEQ_OK) {
        cudaGetLastError();
        seq_batch_destroy(bt);
        return rc;
    }
    *out = bt;
    return SEQ_OK;
}

int seq_batch_destroy(seq_batch* bt) {
    if (!bt) return SEQ_OK;
    cudaStreamSynchronize(bt->stream);
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    for (void* p : bt->allocs) cudaFree(p);
    if (bt->h_pinned) cudaFreeHost(bt->h_pinned);
    if (bt->h_prm) cudaFreeHost(bt->h_prm);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    delete bt;
    return SEQ_OK;
}

int seq_batch_step(seq_batch* bt, const double* const* values, const double* const* b,
                   double* const* x, double tol, seq_info* infos) {
    if (!bt || !values || !b || !x || !(tol > 0)) return SEQ_EINVAL;
    int rc = batch_run(bt, values, b, x, tol, bt->autopush);
    if (rc) return rc;
    int worst = SEQ_OK;
    for (int k = 0; k < bt->count; ++k) {
        const BatchSeq& q = bt->host[k];
        if (infos) {
            seq_info& in = infos[k];
            memset(&in, 0, sizeof(in));
            in.iters = q.iters;
            in.refinements = q.refinements;
            in.history_cols = q.history_cols;
            in.rank = q.rank;
            in.guess_relres = q.guess_relres;
            in.sketch_resid = q.sketch_resid;
            in.final_relres = q.final_relres;
            in.status = q.status;
            in.launches = (k == 0) ? 1 : 0;
            in.net_resid = -1.0;
        }
        if (q.status < 0) worst = q.status;
        else if (q.status > 0 && worst == SEQ_OK) worst = q.status;
    }
    return worst;
}

int seq_batch_autotune(seq_batch* bt, const double* const* values, const double* const* b,
                       double* const* x, double tol, int32_t* chosen) {
    if (!bt || !values || !b || !x || !(tol > 0)) return SEQ_EINVAL;
    const int thr[3] = {256, 512, 1024};
    const int cls[3] = {1, 4, 8};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bt_thr = bt->threads, bt_bps = bt->blocks_per_sm, bt_ord = bt->order_kind;
    int bt_cl = bt->cluster;
    for (int ci = 0; ci < 3; ++ci) {
        const int cl = cls[ci];
        for (int oi = 0; oi < 2; ++oi) {
            for (int ti = 0; ti < 3; ++ti) {
                for (int bps = 1; bps <= 2; ++bps) {
                    if (cl > 1 && (bps > 1 || thr[ti] < 512)) continue;
                    const size_t smem = cl > 1 ? bt->smem_cluster : bt->smem;
                    if ((size_t)bps * smem > 220 * 1024) continue;
                    bt->threads = thr[ti];
                    bt->blocks_per_sm = bps;
                    bt->order_kind = oi;
                    bt->cluster = cl;
                    const StepKernel kern =
                        cl > 1 ? cluster_kernel_for(thr[ti]) : step_kernel_for(thr[ti], bps);
                    int nb = 0;
                    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem) != cudaSuccess ||
                        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, thr[ti], smem) !=
                            cudaSuccess ||
                        nb < bps || (cl > 1 && cluster_grid(bt, kern) <= 0)) {
                        cudaGetLastError();
                        continue;
                    }
                    if (batch_order(bt) || batch_capture(bt)) continue;
                    cudaEventRecord(e0, bt->stream);
                    const int rc = batch_run(bt, values, b, x, tol, 0);
                    cudaEventRecord(e1, bt->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rc == SEQ_OK && ms < best) {
                        best = ms;
                        bt_thr = thr[ti];
                        bt_bps = bps;
                        bt_ord = oi;
                        bt_cl = cl;
                    }
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bt->threads = bt_thr;
    bt->blocks_per_sm = bt_bps;
    bt->order_kind = bt_ord;
    bt->cluster = bt_cl;
    int rc = batch_order(bt);
    if (!rc) rc = batch_capture(bt);
    if (chosen) {
        chosen[0] = bt->threads;
        chosen[1] = bt->blocks_per_sm;
        chosen[2] = bt->order_kind;
    }
    return rc;
}

int seq_batch_set_autopush(seq_batch* bt, int32_t on) {
    if (!bt) return SEQ_EINVAL;
    bt->autopush = on ? 1 : 0;
    return SEQ_OK;
}

int seq_batch_push(seq_batch* bt, int32_t k, const double* x_dev) {
    if (!bt || k < 0 || k >= bt->count || !x_dev) return SEQ_EINVAL;
    BatchSeq& q = bt->host[k];
    const int slot = q.pushes % q.M;
    int blocks = (q.n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    batch_push_kernel<<<blocks, 256, 0, bt->stream>>>(x_dev, q.n, q.X, q.ldx, slot);
    if (cudaGetLastError() != cudaSuccess) return SEQ_ECUDA;
    q.pushes += 1;
    return SEQ_OK;
}

int seq_batch_set_schedule(seq_batch* bt, int32_t threads, int32_t blocks_per_sm,
                           int32_t order_kind) {
    if (!bt || (threads != 256 && threads != 512 && threads != 1024) || blocks_per_sm < 1 ||
        blocks_per_sm > 2 || order_kind < 0 || order_kind > 1)
        return SEQ_EINVAL;
    bt->threads = threads;
    bt->blocks_per_sm = blocks_per_sm;
    bt->order_kind = order_kind;
    bt->cluster = 1;
    int rc = batch_order(bt);
    if (!rc) rc = batch_capture(bt);
    return rc;
}

int seq_batch_set_cluster(seq_batch* bt, int32_t ctas, int32_t threads, int32_t order_kind) {
    if (!bt || (ctas != 1 && ctas != 2 && ctas != 4 && ctas != 8) ||
        (threads != 256 && threads != 512 && threads != 1024) || order_kind < 0 || order_kind > 1)
        return SEQ_EINVAL;
    bt->cluster = ctas;
    bt->threads = threads;
    bt->blocks_per_sm = 1;
    bt->order_kind = order_kind;
    int rc = batch_order(bt);
    if (!rc) rc = batch_capture(bt);
    return rc;
}

int seq_batch_get_schedule(const seq_batch* bt, int32_t* out) {
    if (!bt || !out) return SEQ_EINVAL;
    out[0] = bt->threads;
    out[1] = bt->blocks_per_sm;
    out[2] = bt->order_kind;
    out[3] = bt->cluster;
    return SEQ_OK;
}

}  // extern "C"
