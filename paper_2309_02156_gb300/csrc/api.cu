// C-ABI of libseqaccel (declared in include/seqaccel.h): context management
// and the host orchestration of the guess of Algorithm 1 and the Krylov
// solve that follows it.  Device memory is allocated once per context; every
// call is ordered on the context's stream and synchronises only where a
// seq_info is returned (once per GMRES restart cycle inside seq_solve).
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/seqaccel.h"
#include "common.cuh"
#include "internal.h"
#include "mlp_internal.h"

using namespace sa;

struct seq_ctx {
    seq_config cfg;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;      // private stream used only for graph capture
    int dev = 0;
    bool mixed = false;              // FP32 inner Krylov inside FP64 refinement
    bool hist32 = false;             // FP32 history and sketch (SEQ_MIXED)
    int ldx = 0;
    void* X = nullptr;               // history ring, n x ldx (double or float)
    int pushes = 0;
    double* sk_partial = nullptr;    // per-block partial sketched blocks
    int sk_nblk = 0;
    double* W = nullptr;             // s*(M+1) + 1
    LsqOut* lsq = nullptr;
    LsqOut* lsq_host = nullptr;      // pinned
    int nblk = 0;
    double* kpartial = nullptr;      // nblk * 80 doubles (per-block partial sums)
    size_t ldv = 0;
    void* V = nullptr;               // (restart+1) x ldv basis (GMRES)
    void* w = nullptr;
    void* r = nullptr;               // CG vectors
    void* p = nullptr;
    void* q = nullptr;
    float* val32 = nullptr;          // rounded matrix values (mixed, when not supplied)
    int val32_cap = 0;
    float* rhs32 = nullptr;
    double* r64 = nullptr;           // FP64 residual of the refinement (mixed precision)
    float* d = nullptr;
    DevArgs* d_args = nullptr;       // outer (FP64) system
    DevArgs* h_args = nullptr;       // pinned staging
    DevArgs* d_args_in = nullptr;    // inner (FP32) system
    DevArgs* h_args_in = nullptr;
    KState* ks = nullptr;            // outer / FP64 solve state
    KState* ks_in = nullptr;         // inner solve state
    KState* h_ks = nullptr;          // pinned mirror of the state tail
    int* sell_width = nullptr;       // SELL-32 copy of A used by the GMRES cycles
    int* sell_off = nullptr;
    int* sell_col = nullptr;
    void* sell_val = nullptr;
    size_t sell_cap = 0;             // entries allocated
    int* h_int = nullptr;            // pinned scratch words (SELL total and widest slice)
    bool sell_ok = false;
    int sell_w = 0;                  // uniform SELL slice width (0: slices differ)
    int sell_keep = 0;               // SELL arrays small enough to keep in L2 (evict-last loads)
    double* yring = nullptr;         // last four coefficient vectors (newest first)
    int yring_valid = 0;             // consecutive full-history guesses in the ring
    long long yring_pushes = -1;     // pushes at the newest ring entry
    seq_mlp* mlp = nullptr;          // learned predictor (SEQ_GUESS_LEARNED)
    seq_mlp* mlp_owned = nullptr;    // predictor created by seq_learned_train / _load
    float* sample = nullptr;         // features / target of the last full guess
    float* yhat = nullptr;
    int* used_net = nullptr;
    int* h_used = nullptr;
    bool sample_ready = false;
    double* Om = nullptr;            // RAND: Omega, n x ldo row-major
    int ldo = 0;
    double* Zs = nullptr;            // RAND: Z row of every ring slot (M x basis_m)
    uint64_t gseed = 0;
    uint64_t gdraws = 0;             // Gaussian values drawn so far
    bool om_valid = false;
    int om_updates = 0;
    double* gpart = nullptr;         // POD: Gram partials, Gram, eigenvectors, eigenvalues
    unsigned* gcount = nullptr;
    double* G = nullptr;
    double* Vk = nullptr;
    double* lam = nullptr;
    int* sweeps = nullptr;
    double* Wp = nullptr;            // POD: reduced block [W1 V_k | wb]
    LsqOut* lsq_red = nullptr;
    int pod_mi = 0, pod_kk = 0;
    void* dinv = nullptr;            // preconditioner: 1 / diag(A) and sweep vectors
    void* za = nullptr;
    void* zb = nullptr;
    void* tprec = nullptr;
    void* pc_d = nullptr;            // Chebyshev recurrence vector
    double* pc_tab = nullptr;        // Chebyshev: Gershgorin bound (bits) and coefficients
    cudaGraphExec_t cycle = nullptr;
    cudaGraphExec_t cg_graph = nullptr;     // grid-wide CG iterations (large systems)
    cudaGraphExec_t cycle_prof = nullptr;   // same cycle with timing events between kernels
    std::vector<cudaEvent_t> ev;
    bool profiling = false;
    seq_kernel_stat stats[SEQ_K_COUNT];
    int cycle_launches = 0;
    int launches = 0;
    std::string err;
};

namespace {

const size_t kTailOff = offsetof(KState, beta);
const size_t kTailLen = offsetof(KState, counter) - offsetof(KState, beta);

int fail(seq_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, SEQ_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int round_up(int v, int m) { return (v + m - 1) / m * m; }

int check_csr(seq_ctx* ctx, const seq_csr* A) {
    if (!A) return fail(ctx, SEQ_EINVAL, "A is NULL");
    if (A->n != ctx->cfg.n) return fail(ctx, SEQ_EINVAL, "A->n differs from the context's n");
    if (A->nnz < 0) return fail(ctx, SEQ_EINVAL, "A->nnz < 0");
    if (!A->rowptr || (A->nnz > 0 && (!A->colind || !A->values)))
        return fail(ctx, SEQ_EINVAL, "A has a NULL array");
    return SEQ_OK;
}

// Copy the state tail (beta .. bad_index) of a device KState into h_ks.
int read_tail(seq_ctx* ctx, const KState* ks) {
    CK(cudaMemcpyAsync(reinterpret_cast<char*>(ctx->h_ks) + kTailOff,
                       reinterpret_cast<const char*>(ks) + kTailOff, kTailLen,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SEQ_OK;
}

int set_args(seq_ctx* ctx, const seq_csr* A, const double* b, double* x, double tol,
             int max_iters) {
    DevArgs* h = ctx->h_args;
    memset(h, 0, sizeof(DevArgs));
    h->rowptr = A->rowptr;
    h->colind = A->colind;
    h->val64 = A->values;
    h->val32 = A->values_f32 ? A->values_f32 : ctx->val32;
    h->b = b;
    h->x = x;
    h->d = ctx->d;
    h->rhs32 = ctx->rhs32;
    h->sell_off = ctx->sell_ok ? ctx->sell_off : nullptr;
    h->sell_col = ctx->sell_ok ? ctx->sell_col : nullptr;
    h->sell_val = ctx->sell_ok ? ctx->sell_val : nullptr;
    h->sell_w = ctx->sell_ok ? ctx->sell_w : 0;
    h->sell_keep = ctx->sell_ok ? ctx->sell_keep : 0;
    h->n = A->n;
    h->nnz = A->nnz;
    h->max_iters = max_iters;
    h->tol = tol;
    CK(cudaMemcpyAsync(ctx->d_args, h, sizeof(DevArgs), cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->mixed) {
        memcpy(ctx->h_args_in, h, sizeof(DevArgs));
        CK(cudaMemcpyAsync(ctx->d_args_in, ctx->h_args_in, sizeof(DevArgs),
                           cudaMemcpyHostToDevice, ctx->stream));
    }
    return SEQ_OK;
}

int ensure_val32(seq_ctx* ctx, const seq_csr* A) {
    if (!ctx->mixed || A->values_f32) return SEQ_OK;
    if (A->nnz > ctx->val32_cap) {
        if (ctx->val32) cudaFree(ctx->val32);
        ctx->val32 = nullptr;
        ctx->val32_cap = 0;
        if (cudaMalloc(&ctx->val32, sizeof(float) * (size_t)(A->nnz > 0 ? A->nnz : 1)) != cudaSuccess)
            return fail(ctx, SEQ_ENOMEM, "cannot allocate the FP32 copy of A");
        ctx->val32_cap = A->nnz;
    }
    launch_round_f32(A->values, ctx->val32, A->nnz, ctx->stream);
    ctx->launches += 1;
    return SEQ_OK;
}

// SELL-32 copy of the matrix for the GMRES cycles (values in FP64, or the
// FP32 copy in mixed precision).  Sized with one small synchronisation; kept
// off (CSR is used) when padding would more than double the storage.
int build_sell(seq_ctx* ctx, const seq_csr* A) {
    ctx->sell_ok = false;
    const int n = A->n, ns = (n + 31) / 32;
    launch_sell_layout(A->rowptr, n, A->nnz, ctx->sell_width, ctx->sell_off, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->h_int, ctx->sell_off + ns, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    long long total = ctx->h_int[0];
    const long long wmax = ctx->h_int[1];
    ctx->sell_w = 0;
    if (total <= 0 || total >= 0x7fffffffLL || total > 2LL * A->nnz + 64LL * ns) return SEQ_OK;
    // When padding every slice to the widest costs at most 5% more storage,
    // use one width: the products then compute slice offsets instead of
    // loading them (one dependent load less per slice).
    if (wmax > 0 && 32LL * ns * wmax <= total + total / 20 && 32LL * ns * wmax < 0x7fffffffLL) {
        launch_sell_uniform(n, (int)wmax, ctx->sell_off, ctx->stream);
        ctx->launches += 1;
        total = 32LL * ns * wmax;
        ctx->h_int[0] = (int)total;
        ctx->sell_w = (int)wmax;
    }
    const size_t el = ctx->mixed ? sizeof(float) : sizeof(double);
    if ((size_t)total > ctx->sell_cap) {
        if (ctx->sell_col) cudaFree(ctx->sell_col);
        if (ctx->sell_val) cudaFree(ctx->sell_val);
        ctx->sell_col = nullptr;
        ctx->sell_val = nullptr;
        ctx->sell_cap = 0;
        if (cudaMalloc(&ctx->sell_col, sizeof(int) * (size_t)total) != cudaSuccess ||
            cudaMalloc(&ctx->sell_val, el * (size_t)total) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SEQ_ENOMEM, "cannot allocate the SELL-32 copy of A");
        }
        ctx->sell_cap = (size_t)total;
    }
    if (ctx->mixed) {
        const float* v32 = A->values_f32 ? A->values_f32 : ctx->val32;
        launch_sell_fill_f32(A->rowptr, A->colind, v32, n, A->nnz, ctx->sell_off, ctx->sell_col,
                             (float*)ctx->sell_val, ctx->stream);
    } else {
        launch_sell_fill_f64(A->rowptr, A->colind, A->values, n, A->nnz, ctx->sell_off,
                             ctx->sell_col, (double*)ctx->sell_val, ctx->stream);
    }
    ctx->launches += 3;
    CK(cudaGetLastError());
    ctx->sell_ok = true;
    // Every Arnoldi step reads the matrix several times (the product and, when
    // preconditioned, every sweep): keep it in L2 when it takes at most half.
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->dev);
    const double sell_bytes = (4.0 + (double)el) * (double)total + 4.0 * (ns + 1);
    ctx->sell_keep = l2 > 0 && sell_bytes <= 0.5 * (double)l2;
    return SEQ_OK;
}

// Capture one restart cycle as a CUDA graph (once per context); the profiled
// variant carries an event record node between consecutive kernels.
int capture_cycle(seq_ctx* ctx, bool prof) {
    cudaGraphExec_t* exec = prof ? &ctx->cycle_prof : &ctx->cycle;
    if (*exec) return SEQ_OK;
    const int R = ctx->cfg.restart;
    cudaEvent_t* ev = nullptr;
    const int sw = ctx->cfg.precond_sweeps;
    const double om = ctx->cfg.precond_omega;
    if (prof) {
        if (ctx->ev.empty()) {
            ctx->ev.resize(cycle_marks(R, sw, ctx->mixed) + 1);
            for (auto& e : ctx->ev) CK(cudaEventCreate(&e));
        }
        ev = ctx->ev.data();
    }
    const ChebConfig cheb{ctx->cfg.precond_kind == 1, ctx->pc_tab};
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    if (!ctx->mixed)
        launch_gmres_cycle_f64(ctx->d_args, ctx->ks, (double*)ctx->V, ctx->ldv, (double*)ctx->w,
                               ctx->kpartial, ctx->nblk, R, ctx->cap, &ctx->cycle_launches, ev, sw,
                               om, (const double*)ctx->dinv, (double*)ctx->za, (double*)ctx->zb,
                               (double*)ctx->tprec, &cheb, (double*)ctx->pc_d);
    else
        launch_gmres_cycle_f32(ctx->d_args_in, ctx->ks_in, (float*)ctx->V, ctx->ldv,
                               (float*)ctx->w, (float*)ctx->kpartial, ctx->nblk, R, ctx->cap,
                               &ctx->cycle_launches, ev, sw, om, (const float*)ctx->dinv,
                               (float*)ctx->za, (float*)ctx->zb, (float*)ctx->tprec, &cheb,
                               (float*)ctx->pc_d);
    CK(cudaStreamEndCapture(ctx->cap, &g));
    cudaError_t e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *exec = nullptr;
        return fail(ctx, SEQ_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    return SEQ_OK;
}

// launches kernels of one kind between events ev0 and ev0 + 1.
void add_stat(seq_ctx* ctx, int kind, int ev0, double bytes, double flops, int launches = 1) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[ev0], ctx->ev[ev0 + 1]) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    seq_kernel_stat& st = ctx->stats[kind];
    st.launches += launches;
    st.ms += ms;
    st.bytes += bytes;
    st.flops += flops;
}

// Per-kind time and algorithmic traffic of the cycle that just ran (each
// operand counted once: CSR arrays, gathered vector, basis columns, outputs).
void account_cycle(seq_ctx* ctx, bool f32, int jd, bool updated, int nnz) {
    const double n = ctx->cfg.n, E = f32 ? 4.0 : 8.0, R = ctx->cfg.restart;
    const double csr = 4.0 * (n + 1) + (4.0 + E) * nnz;
    // The cycle's products read the SELL-32 copy when it exists (padded index
    // and value arrays plus the slice offsets), the CSR arrays otherwise.
    const double ns = (ctx->cfg.n + 31) / 32;
    const double spmv_mat = ctx->sell_ok ? 4.0 * (ns + 1) + (4.0 + E) * (double)*ctx->h_int : csr;
    const int sw = ctx->cfg.precond_sweeps;
    const int pk = precond_kernels(sw);
    const int pm = sw > 0 ? 1 : 0;                   // one mark per preconditioner application
    const int S = step_kernels(f32) + pm;
    // Preconditioner of degree d > 1: the first sweep reads the matrix, u
    // (gathered; the same array as its row operand) and dinv and writes z;
    // each later sweep reads the matrix, z (gathered), u, dinv and writes the
    // next z.  Chebyshev also writes d at every sweep but the last and reads
    // it at every sweep but the first.  Degree 1: the scale reads u, dinv and
    // writes z (and d).  The application's sweeps share one pair of events.
    const double cv = ctx->cfg.precond_kind == 1 ? 1.0 : 0.0;
    auto precond = [&](int ev0) {
        if (sw == 1) {
            add_stat(ctx, SEQ_K_PRECOND, ev0, (3.0 + cv) * E * n, 2.0 * n);
            return;
        }
        double bytes = 0.0, flops = 0.0;
        for (int k = 1; k < sw; ++k) {
            const double dv = cv * ((k > 1 ? 1.0 : 0.0) + (k < sw - 1 ? 1.0 : 0.0));
            bytes += spmv_mat + ((k == 1 ? 3.0 : 4.0) + dv) * E * n;
            flops += 2.0 * nnz + (k == 1 ? 6.0 + 2.0 * cv : 4.0 + 3.0 * cv) * n;
        }
        add_stat(ctx, SEQ_K_PRECOND, ev0, bytes, flops, pk);
    };
    for (int j = 0; j < jd; ++j) {
        const double nk = j + 1;
        int e = S * j + pm;
        if (sw > 0) precond(S * j);
        if (f32) {
            // fused SpMV + first-pass dots: matrix, gathered vector, w written
            // once, basis columns 0..j (w re-read from cache, not counted)
            add_stat(ctx, SEQ_K_SPMV, e, spmv_mat + E * n * (nk + 2), 2.0 * nnz + n + 2.0 * n * nk);
            e -= 1;
        } else {
            add_stat(ctx, SEQ_K_SPMV, e, spmv_mat + 2.0 * E * n, 2.0 * nnz + n);
            add_stat(ctx, SEQ_K_CGS_DOT, e + 1, E * n * (nk + 1), 2.0 * n * nk);
        }
        add_stat(ctx, SEQ_K_CGS_PASS2, e + 2, E * n * (nk + 2), 4.0 * n * nk);
        add_stat(ctx, SEQ_K_CGS_PASS3, e + 3, E * n * (nk + 2), 2.0 * n * nk + 2.0 * n);
    }
    int u = S * (int)R;
    if (sw > 0) {
        if (updated) {
            add_stat(ctx, SEQ_K_UPDATE, u, E * n * (jd + 1), 2.0 * n * jd);
            precond(u + 1);
            add_stat(ctx, SEQ_K_UPDATE, u + 2, 3.0 * E * n, n);
        }
        u += 3;
    } else {
        if (updated) add_stat(ctx, SEQ_K_UPDATE, u, E * n * (jd + 2), 2.0 * n * jd);
        u += 1;
    }
    add_stat(ctx, SEQ_K_RESTART, u, csr + 3.0 * E * n, 2.0 * nnz + 4.0 * n);
}

// One restarted GMRES solve on the system bound to (args, ks); `f32` selects
// the FP32 inner kernels.  Returns a seq_status; h_ks holds the final tail.
int run_gmres(seq_ctx* ctx, bool f32) {
    KState* ks = f32 ? ctx->ks_in : ctx->ks;
    if (!f32)
        launch_gmres_start_f64(ctx->d_args, ks, (double*)ctx->V, ctx->ldv, ctx->kpartial,
                               ctx->nblk, 1, ctx->stream);
    else
        launch_gmres_start_f32(ctx->d_args_in, ks, (float*)ctx->V, ctx->ldv,
                               (float*)ctx->kpartial, ctx->nblk, 1, ctx->stream);
    ctx->launches += 1;
    CK(cudaGetLastError());
    int rc = read_tail(ctx, ks);
    if (rc) return rc;
    const bool prof = ctx->profiling;
    rc = capture_cycle(ctx, prof);
    if (rc) return rc;
    cudaGraphExec_t exec = prof ? ctx->cycle_prof : ctx->cycle;
    const int nnz = f32 ? ctx->h_args_in->nnz : ctx->h_args->nnz;
    // The iteration cap bounds the number of cycles: each unfinished cycle
    // performs at least one Arnoldi step.
    const long max_cycles = (long)ctx->cfg.max_iters + 2;
    long cycles = 0;
    while (!ctx->h_ks->finished) {
        if (++cycles > max_cycles) return fail(ctx, SEQ_ETIMEOUT, "GMRES cycle bound exceeded");
        CK(cudaGraphLaunch(exec, ctx->stream));
        ctx->launches += ctx->cycle_launches;
        rc = read_tail(ctx, ks);
        if (rc) return rc;
        if (prof) {
            const bool err = ctx->h_ks->status == SEQ_EBREAKDOWN || ctx->h_ks->status == SEQ_ENONFINITE;
            account_cycle(ctx, f32, err ? ctx->h_ks->jdone : ctx->h_ks->last_jdone, !err, nnz);
        }
    }
    return SEQ_OK;
}

// Grid-wide CG on the system bound to (args, ks) (FP32: the inner solve from
// d = 0): the start kernel, then graph launches of kGridCgGraphIters
// iterations; between launches the host answers a true-residual check
// request (KState::jdone) with the check kernel.  Ends with the true
// residual of the final iterate in ks->beta.
int run_cg_grid(seq_ctx* ctx, bool f32) {
    KState* ks = f32 ? ctx->ks_in : ctx->ks;
    const DevArgs* args = f32 ? ctx->d_args_in : ctx->d_args;
    if (f32)
        launch_cgg_start_f32(args, ks, (float*)ctx->r, (float*)ctx->p, (float*)ctx->kpartial,
                             ctx->nblk, ctx->stream);
    else
        launch_cgg_start_f64(args, ks, (double*)ctx->r, (double*)ctx->p, ctx->kpartial, ctx->nblk,
                             ctx->stream);
    ctx->launches += 1;
    CK(cudaGetLastError());
    int rc = read_tail(ctx, ks);
    if (rc) return rc;
    if (!ctx->cg_graph) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
        if (f32)
            launch_cgg_iterations_f32(args, ks, (float*)ctx->r, (float*)ctx->p, (float*)ctx->q,
                                      (float*)ctx->kpartial, ctx->nblk, kGridCgGraphIters, ctx->cap);
        else
            launch_cgg_iterations_f64(args, ks, (double*)ctx->r, (double*)ctx->p, (double*)ctx->q,
                                      ctx->kpartial, ctx->nblk, kGridCgGraphIters, ctx->cap);
        CK(cudaStreamEndCapture(ctx->cap, &g));
        cudaError_t e = cudaGraphInstantiate(&ctx->cg_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ctx->cg_graph = nullptr;
            return fail(ctx, SEQ_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
    }
    // Every graph launch performs at least one iteration or ends the solve,
    // and every check either ends it or is followed by a launch.
    const long max_rounds = 2L * ((long)ctx->cfg.max_iters + 2);
    long rounds = 0;
    while (!ctx->h_ks->finished) {
        if (++rounds > max_rounds) return fail(ctx, SEQ_ETIMEOUT, "CG round bound exceeded");
        if (ctx->h_ks->jdone) {
            if (f32)
                launch_cgg_true_residual_f32(args, ks, (float*)ctx->r, (float*)ctx->p,
                                             (float*)ctx->kpartial, ctx->nblk, 1, ctx->stream);
            else
                launch_cgg_true_residual_f64(args, ks, (double*)ctx->r, (double*)ctx->p,
                                             ctx->kpartial, ctx->nblk, 1, ctx->stream);
            ctx->launches += 1;
        } else {
            CK(cudaGraphLaunch(ctx->cg_graph, ctx->stream));
            ctx->launches += 3 * kGridCgGraphIters;
        }
        CK(cudaGetLastError());
        rc = read_tail(ctx, ks);
        if (rc) return rc;
    }
    if (f32)
        launch_cgg_true_residual_f32(args, ks, (float*)ctx->r, nullptr, (float*)ctx->kpartial,
                                     ctx->nblk, 0, ctx->stream);
    else
        launch_cgg_true_residual_f64(args, ks, (double*)ctx->r, nullptr, ctx->kpartial, ctx->nblk,
                                     0, ctx->stream);
    ctx->launches += 1;
    CK(cudaGetLastError());
    return read_tail(ctx, ks);
}

void fill_info(seq_info* info, const KState* t) {
    if (!info) return;
    info->guess_relres = t->first_relres;
    info->final_relres = rel_residual(t->beta, t->bnorm);
    info->iters = t->iters;
    info->status = t->status;
}

}  // namespace

extern "C" {

int seq_create(const seq_config* cfg, void* cuda_stream, seq_ctx** out) {
    if (!out) return SEQ_EINVAL;
    *out = nullptr;
    if (!cfg) return SEQ_EINVAL;
    const seq_config& c = *cfg;
    if (c.n <= 0 || c.M < 1 || c.M > kMaxM || c.s < c.M + 1 || c.s > kMaxS || c.zeta < 1 ||
        c.zeta > c.s || c.zeta > kMaxZeta || c.restart < 1 || c.restart > kMaxRestart ||
        c.max_iters < 0 || (c.precision < SEQ_F64 || c.precision > SEQ_MIXED_KRYLOV) ||
        c.guess < SEQ_GUESS_ZERO || c.guess > SEQ_GUESS_RAND ||
        (c.krylov != SEQ_CG && c.krylov != SEQ_GMRES))
        return SEQ_EINVAL;
    const bool compressed = c.guess == SEQ_GUESS_POD || c.guess == SEQ_GUESS_RAND;
    if (compressed && (c.basis_m < 1 || c.basis_m > c.M || c.refresh < 0 || c.precision == SEQ_MIXED))
        return SEQ_EINVAL;
    if (c.precond_sweeps < 0 || c.precond_sweeps > 32 || c.precond_omega < 0.0 ||
        c.precond_omega >= 2.0 || (c.precond_sweeps > 0 && c.krylov != SEQ_GMRES) ||
        c.precond_kind < 0 || c.precond_kind > 1 || !(c.precond_ratio == 0.0 || c.precond_ratio > 1.0) ||
        !(c.precond_lmax >= 0.0))
        return SEQ_EINVAL;
    seq_ctx* ctx = new seq_ctx();
    memset(ctx->stats, 0, sizeof(ctx->stats));
    ctx->cfg = c;
    if (ctx->cfg.inner_tol <= 0) ctx->cfg.inner_tol = 1e-2;
    if (ctx->cfg.rank_tol <= 0) ctx->cfg.rank_tol = c.precision == SEQ_MIXED ? 1e-5 : 1e-12;
    if (ctx->cfg.refresh <= 0) ctx->cfg.refresh = 50;
    if (ctx->cfg.precond_omega <= 0.0) ctx->cfg.precond_omega = 0.8;
    if (ctx->cfg.precond_ratio <= 0.0) ctx->cfg.precond_ratio = 30.0;
    ctx->mixed = c.precision != SEQ_F64;
    ctx->hist32 = c.precision == SEQ_MIXED;
    ctx->stream = (cudaStream_t)cuda_stream;
    const int n = c.n, M = c.M, s = c.s;
    const size_t el = ctx->mixed ? sizeof(float) : sizeof(double);     // Krylov vectors
    const size_t elh = ctx->hist32 ? sizeof(float) : sizeof(double);  // history and sketch
    ctx->ldx = ctx->hist32 ? round_up(M, 8) : round_up(M, 4);
    bool ok = cudaGetDevice(&ctx->dev) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaMalloc(&ctx->X, elh * (size_t)n * ctx->ldx) == cudaSuccess;
    ok = ok && cudaMemsetAsync(ctx->X, 0, elh * (size_t)n * ctx->ldx, ctx->stream) == cudaSuccess;
    ctx->sk_nblk = sketch_grid(n, s, M);
    ok = ok && cudaMalloc(&ctx->sk_partial, sizeof(double) * sketch_partial_doubles(n, s, M)) == cudaSuccess;
    ok = ok && cudaMalloc(&ctx->W, sizeof(double) * (s * (M + 1) + 1)) == cudaSuccess;
    ok = ok && cudaMalloc(&ctx->lsq, sizeof(LsqOut)) == cudaSuccess;
    ok = ok && cudaMallocHost(&ctx->lsq_host, sizeof(LsqOut)) == cudaSuccess;
    ctx->nblk = stream_grid(n);
    ok = ok && cudaMalloc(&ctx->kpartial, sizeof(double) * (size_t)ctx->nblk * 80) == cudaSuccess;
    ctx->ldv = (size_t)round_up(n, 64);
    if (c.krylov == SEQ_GMRES) {
        ok = ok && cudaMalloc(&ctx->V, el * ctx->ldv * (c.restart + 1)) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->w, el * ctx->ldv) == cudaSuccess;
    } else {
        ok = ok && cudaMalloc(&ctx->r, el * (size_t)n) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->p, el * (size_t)n) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->q, el * (size_t)n) == cudaSuccess;
    }
    if (ctx->mixed) {
        ok = ok && cudaMalloc(&ctx->rhs32, sizeof(float) * (size_t)n) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->r64, sizeof(double) * (size_t)n) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->d, sizeof(float) * (size_t)n) == cudaSuccess;
    }
    if (c.krylov == SEQ_GMRES || n >= kGridCgMinRows) {     // SELL-32 copy for the cycles
        const int ns = (n + 31) / 32;
        ok = ok && cudaMalloc(&ctx->sell_width, sizeof(int) * (size_t)ns) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->sell_off, sizeof(int) * (size_t)(ns + 2)) == cudaSuccess;
    }
    ok = ok && cudaMallocHost(&ctx->h_int, 2 * sizeof(int)) == cudaSuccess;
    {
        const int in = 4 * M + s, stride = in + M + M * M + 1;
        ok = ok && cudaMalloc(&ctx->yring, sizeof(double) * 4 * kMaxM) == cudaSuccess;
        ok = ok && cudaMemsetAsync(ctx->yring, 0, sizeof(double) * 4 * kMaxM, ctx->stream) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->sample, sizeof(float) * stride) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->yhat, sizeof(float) * kMaxM) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->used_net, 16) == cudaSuccess;     // int flag | double rho
        ok = ok && cudaMallocHost(&ctx->h_used, 16) == cudaSuccess;
    }
    if (c.precond_sweeps > 0) {
        ok = ok && cudaMalloc(&ctx->dinv, el * (size_t)n) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->za, el * (size_t)n) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->zb, el * (size_t)n) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->tprec, el * (size_t)n) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->pc_tab, sizeof(double) * kChebTab) == cudaSuccess;
        if (c.precond_kind == 1)
            ok = ok && cudaMalloc(&ctx->pc_d, el * (size_t)n) == cudaSuccess;
    }
    if (c.guess == SEQ_GUESS_RAND) {
        ctx->ldo = round_up(c.basis_m, 4);
        ctx->gseed = c.seed ^ 0x52414E44ull;
        ok = ok && cudaMalloc(&ctx->Om, sizeof(double) * (size_t)n * ctx->ldo) == cudaSuccess;
        ok = ok && cudaMemsetAsync(ctx->Om, 0, sizeof(double) * (size_t)n * ctx->ldo, ctx->stream) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->Zs, sizeof(double) * M * c.basis_m) == cudaSuccess;
    }
    if (c.guess == SEQ_GUESS_POD) {
        ok = ok && cudaMalloc(&ctx->gpart, sizeof(double) * gram_partial_doubles()) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->gcount, sizeof(unsigned)) == cudaSuccess;
        ok = ok && cudaMemsetAsync(ctx->gcount, 0, sizeof(unsigned), ctx->stream) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->G, sizeof(double) * kMaxM * kMaxM) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->Vk, sizeof(double) * kMaxM * kMaxM) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->lam, sizeof(double) * kMaxM) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->sweeps, sizeof(int)) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->Wp, sizeof(double) * s * (kMaxM + 1)) == cudaSuccess;
        ok = ok && cudaMalloc(&ctx->lsq_red, sizeof(LsqOut)) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&ctx->d_args, sizeof(DevArgs)) == cudaSuccess;
    ok = ok && cudaMallocHost(&ctx->h_args, sizeof(DevArgs)) == cudaSuccess;
    ok = ok && cudaMalloc(&ctx->d_args_in, sizeof(DevArgs)) == cudaSuccess;
    ok = ok && cudaMallocHost(&ctx->h_args_in, sizeof(DevArgs)) == cudaSuccess;
    ok = ok && cudaMalloc(&ctx->ks, sizeof(KState)) == cudaSuccess;
    ok = ok && cudaMalloc(&ctx->ks_in, sizeof(KState)) == cudaSuccess;
    ok = ok && cudaMallocHost(&ctx->h_ks, sizeof(KState)) == cudaSuccess;
    ok = ok && cudaMemsetAsync(ctx->ks, 0, sizeof(KState), ctx->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(ctx->ks_in, 0, sizeof(KState), ctx->stream) == cudaSuccess;
    if (ok) ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(ctx->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        seq_destroy(ctx);
        return SEQ_ENOMEM;
    }
    *out = ctx;
    return SEQ_OK;
}

int seq_destroy(seq_ctx* ctx) {
    if (!ctx) return SEQ_OK;
    if (ctx->stream || true) cudaStreamSynchronize(ctx->stream);
    if (ctx->cycle) cudaGraphExecDestroy(ctx->cycle);
    if (ctx->cg_graph) cudaGraphExecDestroy(ctx->cg_graph);
    if (ctx->cycle_prof) cudaGraphExecDestroy(ctx->cycle_prof);
    for (auto e : ctx->ev) cudaEventDestroy(e);
    if (ctx->mlp_owned) seq_mlp_destroy(ctx->mlp_owned);
    void* dev_ptrs[] = {ctx->X, ctx->sk_partial, ctx->W, ctx->lsq, ctx->kpartial,
                        ctx->V, ctx->w, ctx->r, ctx->p, ctx->q, ctx->val32, ctx->rhs32, ctx->r64, ctx->d,
                        ctx->d_args, ctx->d_args_in, ctx->ks, ctx->ks_in, ctx->sell_width,
                        ctx->sell_off, ctx->sell_col, ctx->sell_val, ctx->yring, ctx->sample,
                        ctx->yhat, ctx->used_net, ctx->Om, ctx->Zs, ctx->gpart, ctx->gcount,
                        ctx->G, ctx->Vk, ctx->lam, ctx->sweeps, ctx->Wp, ctx->lsq_red,
                        ctx->dinv, ctx->za, ctx->zb, ctx->tprec, ctx->pc_d, ctx->pc_tab};
    for (void* p : dev_ptrs)
        if (p) cudaFree(p);
    void* host_ptrs[] = {ctx->lsq_host, ctx->h_args, ctx->h_args_in, ctx->h_ks, ctx->h_int,
                         ctx->h_used};
    for (void* p : host_ptrs)
        if (p) cudaFreeHost(p);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    delete ctx;
    return SEQ_OK;
}

int seq_push_solution(seq_ctx* ctx, const double* x_dev) {
    if (!ctx || !x_dev) return fail(ctx, SEQ_EINVAL, "NULL argument");
    const int slot = ctx->pushes % ctx->cfg.M;
    if (ctx->cfg.guess == SEQ_GUESS_RAND && ctx->om_valid) {
        // The progressive update of Algorithm 4, fused with the push.
        const int mb = ctx->cfg.basis_m;
        launch_rand_push(x_dev, ctx->cfg.n, (double*)ctx->X, ctx->ldx, slot,
                         ctx->pushes >= ctx->cfg.M, ctx->Zs, mb, ctx->gseed, ctx->gdraws, ctx->Om,
                         ctx->ldo, ctx->stream);
        CK(cudaGetLastError());
        ctx->gdraws += (uint64_t)mb;
        ctx->om_updates += 1;
        ctx->pushes += 1;
        ctx->launches = 2;
        return SEQ_OK;
    }
    if (ctx->hist32)
        launch_push_f32(x_dev, ctx->cfg.n, (float*)ctx->X, ctx->ldx, slot, ctx->stream);
    else
        launch_push_f64(x_dev, ctx->cfg.n, (double*)ctx->X, ctx->ldx, slot, ctx->stream);
    CK(cudaGetLastError());
    ctx->pushes += 1;
    ctx->launches = 1;
    return SEQ_OK;
}

int seq_history_size(const seq_ctx* ctx) {
    if (!ctx) return 0;
    return ctx->pushes < ctx->cfg.M ? ctx->pushes : ctx->cfg.M;
}

int seq_guess(seq_ctx* ctx, const seq_csr* A, const double* b_dev, double* x0_dev, seq_info* info) {
    if (!ctx) return SEQ_EINVAL;
    ctx->err.clear();
    ctx->launches = 0;
    int rc = check_csr(ctx, A);
    if (rc) return rc;
    if (!b_dev || !x0_dev) return fail(ctx, SEQ_EINVAL, "NULL vector");
    const seq_config& c = ctx->cfg;
    const int n = c.n, M = c.M;
    const int m = seq_history_size(ctx);
    int mode = c.guess;
    const bool learned = mode == SEQ_GUESS_LEARNED;
    if (learned) mode = SEQ_GUESS_SKETCH;
    bool predicted = false;          // the network's y was computed (and tested)
    ctx->sample_ready = false;
    ctx->sell_ok = false;            // the SELL copy belongs to the last seq_solve's matrix
    if (m == 0 && mode != SEQ_GUESS_ZERO) mode = SEQ_GUESS_ZERO;
    CK(cudaMemsetAsync(ctx->ks, 0, sizeof(KState), ctx->stream));
    int rank = 0;
    double rho = 0.0;
    int basis_cols = m;              // columns of the reduced problem
    if (mode == SEQ_GUESS_ZERO) {
        CK(cudaMemsetAsync(x0_dev, 0, sizeof(double) * (size_t)n, ctx->stream));
    } else if (mode == SEQ_GUESS_PREV) {
        const int slot = (ctx->pushes - 1) % M;
        if (ctx->hist32)
            launch_copy_slot_f32((const float*)ctx->X, ctx->ldx, n, slot, x0_dev, ctx->stream);
        else
            launch_copy_slot_f64((const double*)ctx->X, ctx->ldx, n, slot, x0_dev, ctx->stream);
        ctx->launches += 1;
    } else if (mode == SEQ_GUESS_POD || mode == SEQ_GUESS_RAND) {
        int* bad = &ctx->ks->bad_index;
        const int oldest = (ctx->pushes - m) % M;
        const int mb = c.basis_m;
        const double* X = (const double*)ctx->X;
        if (mode == SEQ_GUESS_POD) {
            // Algorithm 2 in snapshot form; the reduced problem from W = S[AX|b].
            const int kk = mb < m ? mb : m;
            launch_sketch_f64(A->rowptr, A->colind, A->values, X, ctx->ldx, b_dev, n, A->nnz, M,
                              c.s, c.zeta, c.seed, ctx->sk_partial, ctx->sk_nblk,
                              ctx->W, bad, ctx->stream);
            launch_pod_basis(X, ctx->ldx, n, M, m, oldest, kk, ctx->gpart, ctx->gcount, ctx->G,
                             ctx->Vk, ctx->lam, ctx->sweeps, ctx->stream);
            launch_pod_reduce(ctx->W, c.s, M, m, oldest, ctx->Vk, kk, ctx->Wp, ctx->stream);
            launch_lsq(ctx->Wp, c.s, kk, kk, 0, c.rank_tol, ctx->lsq_red, ctx->stream);
            launch_pod_coeff(ctx->lsq_red, ctx->Vk, m, kk, M, oldest, ctx->lsq, ctx->stream);
            launch_expand_f64(X, ctx->ldx, n, M, ctx->lsq, x0_dev, ctx->stream);
            ctx->launches += 8;
            ctx->pod_mi = m;
            ctx->pod_kk = kk;
            basis_cols = kk;
        } else {
            // Algorithm 4: Omega from scratch when due, then the reduced problem
            // over span(Omega).
            if (!ctx->om_valid || ctx->om_updates >= c.refresh) {
                launch_rand_scratch(X, ctx->ldx, n, M, m, oldest, ctx->Zs, mb, ctx->gseed,
                                    ctx->gdraws, ctx->Om, ctx->ldo, ctx->stream);
                ctx->gdraws += (uint64_t)m * mb;
                ctx->om_valid = true;
                ctx->om_updates = 0;
                ctx->launches += 2;
            }
            launch_sketch_f64(A->rowptr, A->colind, A->values, ctx->Om, ctx->ldo, b_dev, n,
                              A->nnz, mb, c.s, c.zeta, c.seed, ctx->sk_partial, ctx->sk_nblk,
                              ctx->W, bad, ctx->stream);
            launch_lsq(ctx->W, c.s, mb, mb, 0, c.rank_tol, ctx->lsq, ctx->stream);
            launch_expand_f64(ctx->Om, ctx->ldo, n, mb, ctx->lsq, x0_dev, ctx->stream);
            ctx->launches += 4;
            basis_cols = mb;
        }
        CK(cudaMemcpyAsync(ctx->lsq_host, ctx->lsq, offsetof(LsqOut, W_logical),
                           cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(&ctx->lsq_host->rho, &ctx->lsq->rho,
                           sizeof(LsqOut) - offsetof(LsqOut, rho), cudaMemcpyDeviceToHost,
                           ctx->stream));
    } else {
        int* bad = &ctx->ks->bad_index;
        if (ctx->hist32) {
            rc = ensure_val32(ctx, A);
            if (rc) return rc;
            const float* v32 = A->values_f32 ? A->values_f32 : ctx->val32;
            launch_sketch_f32(A->rowptr, A->colind, v32, (const float*)ctx->X, ctx->ldx, b_dev,
                              n, A->nnz, M, c.s, c.zeta, c.seed, ctx->sk_partial, ctx->sk_nblk,
                              ctx->W, bad, ctx->stream);
        } else {
            launch_sketch_f64(A->rowptr, A->colind, A->values, (const double*)ctx->X, ctx->ldx,
                              b_dev, n, A->nnz, M, c.s, c.zeta, c.seed, ctx->sk_partial,
                              ctx->sk_nblk, ctx->W, bad, ctx->stream);
        }
        const int oldest = (ctx->pushes - m) % M;
        launch_lsq(ctx->W, c.s, M, m, oldest, c.rank_tol, ctx->lsq, ctx->stream);
        ctx->launches += 1;
        if (ctx->pushes != ctx->yring_pushes + 1) ctx->yring_valid = 0;   // window moved by != 1
        if (m == M && ctx->yring_valid >= 4 && M >= 2) {
            // Features and target of this guess (training sample), and the
            // learned prediction with its fallback to least squares.
            launch_learned_sample(ctx->lsq, c.s, M, ctx->yring, ctx->sample, ctx->stream);
            ctx->sample_ready = true;
            ctx->launches += 1;
        }
        // The ring keeps the least-squares coefficients (the training
        // targets), pushed before the network's choice can replace them.
        if (m == M) {
            launch_yring_push(ctx->yring, ctx->lsq, M, ctx->stream);
            ctx->yring_valid += 1;
            ctx->yring_pushes = ctx->pushes;
            ctx->launches += 1;
        } else {
            ctx->yring_valid = 0;
        }
        if (ctx->sample_ready) {
            if (learned && ctx->mlp && mlp_dims_ok(ctx->mlp, M, c.s)) {
                mlp_predict_dev(ctx->mlp, ctx->sample, 1, ctx->yhat, ctx->stream);
                launch_learned_select(ctx->lsq, c.s, M, oldest, ctx->yhat, ctx->used_net,
                                      (double*)(ctx->used_net + 2), ctx->stream);
                CK(cudaMemcpyAsync(ctx->h_used, ctx->used_net, 16, cudaMemcpyDeviceToHost,
                                   ctx->stream));
                ctx->launches += 6;
                predicted = true;   // used or rejected: read after the synchronisation
            }
        }
        if (ctx->hist32)
            launch_expand_f32((const float*)ctx->X, ctx->ldx, n, M, ctx->lsq, x0_dev, ctx->stream);
        else
            launch_expand_f64((const double*)ctx->X, ctx->ldx, n, M, ctx->lsq, x0_dev, ctx->stream);
        ctx->launches += 3;
        CK(cudaMemcpyAsync(ctx->lsq_host, ctx->lsq, offsetof(LsqOut, W_logical),
                           cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(&ctx->lsq_host->rho, &ctx->lsq->rho,
                           sizeof(LsqOut) - offsetof(LsqOut, rho), cudaMemcpyDeviceToHost,
                           ctx->stream));
    }
    rc = set_args(ctx, A, b_dev, x0_dev, 1.0, 0);
    if (rc) return rc;
    launch_residual_norm(ctx->d_args, ctx->ks, ctx->kpartial, ctx->nblk, nullptr, ctx->stream);
    ctx->launches += 1;
    CK(cudaGetLastError());
    rc = read_tail(ctx, ctx->ks);
    if (rc) return rc;
    const bool reduced = mode == SEQ_GUESS_SKETCH || mode == SEQ_GUESS_POD || mode == SEQ_GUESS_RAND;
    if (reduced) {
        rank = ctx->lsq_host->rank;
        rho = ctx->lsq_host->rho;
    }
    if (info) {
        memset(info, 0, sizeof(seq_info));
        info->history_cols = mode == SEQ_GUESS_ZERO ? 0 : (mode == SEQ_GUESS_PREV ? 1 : m);
        info->rank = rank;
        info->sketch_resid = rho;
        info->guess_relres = ctx->h_ks->first_relres;
        info->final_relres = ctx->h_ks->first_relres;
        info->launches = ctx->launches;
        info->net_resid = predicted ? *(const double*)(ctx->h_used + 2) : -1.0;
    }
    ctx->lsq_host->m = reduced ? basis_cols : 0;
    const bool fallback = predicted && *ctx->h_used == 0;   // the network's y was rejected
    if (ctx->h_ks->bad_index) {
        if (info) info->status = SEQ_EINVAL;
        return fail(ctx, SEQ_EINVAL, "CSR column index outside [0, n)");
    }
    if (!isfinite(ctx->h_ks->first_relres)) {
        if (info) info->status = SEQ_ENONFINITE;
        return fail(ctx, SEQ_ENONFINITE, "non-finite residual of the guess");
    }
    if (fallback) {
        if (info) info->status = SEQ_FALLBACK_USED;
        return SEQ_FALLBACK_USED;
    }
    return SEQ_OK;
}

int seq_set_learned(seq_ctx* ctx, seq_mlp* mlp) {
    if (!ctx) return SEQ_EINVAL;
    if (mlp && !mlp_dims_ok(mlp, ctx->cfg.M, ctx->cfg.s))
        return fail(ctx, SEQ_EINVAL, "predictor dimensions differ from the context's M and s");
    if (ctx->mlp_owned && ctx->mlp_owned != mlp) {     // a network the context made itself
        seq_mlp_destroy(ctx->mlp_owned);
        ctx->mlp_owned = nullptr;
    }
    ctx->mlp = mlp;
    return SEQ_OK;
}

namespace {
constexpr int32_t kLearnedMagic = 0x4C514553;
constexpr int kLearnedHidden = 256;
constexpr int kLearnedBatch = 32;

// FP32 values in a serialised predictor of hidden width H (parameters, then
// feature mean, feature std and output scale).
size_t learned_floats(int M, int s, int H) {
    const size_t in = 4 * (size_t)M + s;
    const size_t np = (size_t)H * in + H + (size_t)H * H + H + (size_t)M * H + M;
    return np + 2 * in + M;
}
}  // namespace

int seq_learned_train(seq_ctx* ctx, const float* dataset_dev, int32_t count, int32_t epochs,
                      uint64_t seed) {
    if (!ctx) return SEQ_EINVAL;
    ctx->err.clear();
    if (!dataset_dev || count < 1 || epochs < 0 || ctx->cfg.M < 2)
        return fail(ctx, SEQ_EINVAL, "seq_learned_train: bad argument (or M < 2)");
    seq_mlp* m = ctx->mlp;
    if (!m) {
        int rc = seq_mlp_create(ctx->cfg.M, ctx->cfg.s, kLearnedHidden, kLearnedBatch, seed,
                                ctx->stream, &m);
        if (rc) return fail(ctx, rc, "seq_learned_train: cannot create the predictor");
        ctx->mlp = ctx->mlp_owned = m;
    }
    int batch = count < kLearnedBatch ? count : kLearnedBatch;
    if (batch > mlp_max_batch(m)) batch = mlp_max_batch(m);
    int rc = seq_mlp_fit_normalization(m, dataset_dev, count);
    if (rc) return fail(ctx, rc, "seq_learned_train: normalisation failed");
    rc = seq_mlp_train(m, dataset_dev, count, epochs, batch, 1e-3f, seed, nullptr);
    if (rc) return fail(ctx, rc, "seq_learned_train: training failed");
    return SEQ_OK;
}

int seq_learned_save(seq_ctx* ctx, void* weights_host, size_t bytes, size_t* needed) {
    if (!ctx) return SEQ_EINVAL;
    if (!ctx->mlp) return fail(ctx, SEQ_EINVAL, "seq_learned_save: no predictor attached");
    const int M = ctx->cfg.M, s = ctx->cfg.s, H = mlp_hidden(ctx->mlp);
    const size_t need = 16 + sizeof(float) * learned_floats(M, s, H);
    if (needed) *needed = need;
    if (!weights_host) return SEQ_OK;
    if (bytes < need) return fail(ctx, SEQ_EINVAL, "seq_learned_save: buffer too small");
    int32_t hdr[4] = {kLearnedMagic, M, s, H};
    memcpy(weights_host, hdr, sizeof(hdr));
    float* body = reinterpret_cast<float*>(static_cast<char*>(weights_host) + 16);
    const int np = seq_mlp_param_count(ctx->mlp);
    int rc = seq_mlp_get_params(ctx->mlp, body, body + np);
    return rc ? fail(ctx, rc, "seq_learned_save: cannot read the parameters") : SEQ_OK;
}

int seq_learned_load(seq_ctx* ctx, const void* weights_host, size_t bytes) {
    if (!ctx) return SEQ_EINVAL;
    ctx->err.clear();
    if (!weights_host || bytes < 16) return fail(ctx, SEQ_EINVAL, "seq_learned_load: no header");
    int32_t hdr[4];
    memcpy(hdr, weights_host, sizeof(hdr));
    const int M = ctx->cfg.M, s = ctx->cfg.s, H = hdr[3];
    if (hdr[0] != kLearnedMagic || hdr[1] != M || hdr[2] != s || H < 1 || H > 4096)
        return fail(ctx, SEQ_EINVAL, "seq_learned_load: header does not match the context");
    if (bytes != 16 + sizeof(float) * learned_floats(M, s, H))
        return fail(ctx, SEQ_EINVAL, "seq_learned_load: size does not match the header");
    seq_mlp* m = ctx->mlp;
    if (!m || mlp_hidden(m) != H) {
        int rc = seq_mlp_create(M, s, H, kLearnedBatch, 0, ctx->stream, &m);
        if (rc) return fail(ctx, rc, "seq_learned_load: cannot create the predictor");
        if (ctx->mlp_owned) seq_mlp_destroy(ctx->mlp_owned);
        ctx->mlp = ctx->mlp_owned = m;
    }
    const float* body = reinterpret_cast<const float*>(static_cast<const char*>(weights_host) + 16);
    const int np = seq_mlp_param_count(m);
    int rc = seq_mlp_set_params(m, body, body + np);
    return rc ? fail(ctx, rc, "seq_learned_load: cannot write the parameters") : SEQ_OK;
}

int seq_last_sample(seq_ctx* ctx, float* sample_dev) {
    if (!ctx || !sample_dev) return SEQ_EINVAL;
    if (!ctx->sample_ready) return fail(ctx, SEQ_EINVAL, "no sample: the last guess lacked a full history");
    const int M = ctx->cfg.M, stride = 4 * M + ctx->cfg.s + M + M * M + 1;
    CK(cudaMemcpyAsync(sample_dev, ctx->sample, sizeof(float) * stride, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SEQ_OK;
}

int seq_solve(seq_ctx* ctx, const seq_csr* A, const double* b_dev, double tol, double* x_dev,
              seq_info* info) {
    if (!ctx) return SEQ_EINVAL;
    ctx->err.clear();
    ctx->launches = 0;
    int rc = check_csr(ctx, A);
    if (rc) return rc;
    if (!b_dev || !x_dev) return fail(ctx, SEQ_EINVAL, "NULL vector");
    if (!(tol > 0.0)) return fail(ctx, SEQ_EINVAL, "tol must be > 0");
    const seq_config& c = ctx->cfg;
    if (info) {
        memset(info, 0, sizeof(seq_info));
        info->net_resid = -1.0;
    }
    CK(cudaMemsetAsync(ctx->ks, 0, sizeof(KState), ctx->stream));
    CK(cudaMemsetAsync(ctx->ks_in, 0, sizeof(KState), ctx->stream));
    rc = ensure_val32(ctx, A);
    if (rc) return rc;
    const bool grid_cg = c.krylov == SEQ_CG && c.n >= kGridCgMinRows;
    if (c.krylov == SEQ_GMRES || grid_cg) {
        rc = build_sell(ctx, A);
        if (rc) return rc;
    }
    rc = set_args(ctx, A, b_dev, x_dev, tol, c.max_iters);
    if (rc) return rc;
    if (c.precond_sweeps > 0) {
        unsigned long long* bound = reinterpret_cast<unsigned long long*>(ctx->pc_tab);
        CK(cudaMemsetAsync(ctx->pc_tab, 0, sizeof(double) * kChebTab, ctx->stream));
        if (!ctx->mixed)
            launch_diag_inv_f64(ctx->d_args, (double*)ctx->dinv, c.n, ctx->stream, bound);
        else
            launch_diag_inv_f32(ctx->d_args_in, (float*)ctx->dinv, c.n, ctx->stream, bound);
        if (c.precond_kind == 1) {
            launch_cheb_table(ctx->pc_tab, c.precond_lmax, c.precond_ratio, c.precond_sweeps,
                              ctx->stream);
            ctx->launches += 1;
        }
        ctx->launches += 1;
        CK(cudaGetLastError());
    }
    int status = SEQ_OK;
    if (!ctx->mixed) {
        if (c.krylov == SEQ_GMRES) {
            rc = run_gmres(ctx, false);
            if (rc) return rc;
        } else if (grid_cg) {
            rc = run_cg_grid(ctx, false);
            if (rc) return rc;
        } else {
            launch_cg_block_f64(ctx->d_args, ctx->ks, (double*)ctx->r, (double*)ctx->p,
                                (double*)ctx->q, ctx->stream);
            ctx->launches += 1;
            CK(cudaGetLastError());
            rc = read_tail(ctx, ctx->ks);
            if (rc) return rc;
        }
        fill_info(info, ctx->h_ks);
        status = ctx->h_ks->status;
    } else {
        // FP64 iterative refinement around FP32 inner solves.
        const double theta = 0.5;
        int total = 0, refinements = 0;
        launch_refine_residual(ctx->d_args, ctx->ks, ctx->r64, ctx->kpartial, ctx->nblk,
                               ctx->stream);
        ctx->launches += 1;
        CK(cudaGetLastError());
        rc = read_tail(ctx, ctx->ks);
        if (rc) return rc;
        const double bnorm = ctx->h_ks->bnorm, target = ctx->h_ks->target;
        const double first = rel_residual(ctx->h_ks->beta, bnorm);
        double beta = ctx->h_ks->beta;
        int bad = ctx->h_ks->bad_index;
        status = SEQ_OK;
        // A GMRES inner solve is one restart cycle: every restart then starts
        // from the FP64 residual (an FP32 residual has rounding noise of about
        // u32 cond(A) ||r||, which stalls restarts on ill-conditioned systems).
        // Each refinement costs at least one iteration, so max_iters bounds them.
        const int max_ref = c.krylov == SEQ_GMRES ? c.max_iters + 1 : 100;
        while (!(beta <= target)) {           // a NaN residual enters and is reported
            if (!isfinite(beta)) {
                status = SEQ_ENONFINITE;
                break;
            }
            if (total >= c.max_iters || refinements >= max_ref) {
                status = SEQ_NOT_CONVERGED;
                break;
            }
            launch_refine_scale(ctx->r64, ctx->ks, ctx->rhs32, ctx->cfg.n, ctx->stream);
            ctx->launches += 1;
            DevArgs* hi = ctx->h_args_in;
            hi->tol = fmax(c.inner_tol, theta * target / beta);
            hi->max_iters = c.max_iters - total;
            if (c.krylov == SEQ_GMRES && hi->max_iters > c.restart) hi->max_iters = c.restart;
            CK(cudaMemcpyAsync(ctx->d_args_in, hi, sizeof(DevArgs), cudaMemcpyHostToDevice,
                               ctx->stream));
            if (c.krylov == SEQ_GMRES) {
                rc = run_gmres(ctx, true);
                if (rc) return rc;
            } else if (grid_cg) {
                rc = run_cg_grid(ctx, true);
                if (rc) return rc;
            } else {
                launch_cg_block_f32(ctx->d_args_in, ctx->ks_in, (float*)ctx->r, (float*)ctx->p,
                                    (float*)ctx->q, ctx->stream);
                ctx->launches += 1;
                CK(cudaGetLastError());
                rc = read_tail(ctx, ctx->ks_in);
                if (rc) return rc;
            }
            bad |= ctx->h_ks->bad_index;
            total += ctx->h_ks->iters;
            refinements += 1;
            const int ist = ctx->h_ks->status;
            if (ist == SEQ_EBREAKDOWN || ist == SEQ_ENONFINITE) {
                status = ist;
                break;
            }
            launch_refine_update(ctx->d_args, ctx->ks, ctx->stream);
            launch_refine_residual(ctx->d_args, ctx->ks, ctx->r64, ctx->kpartial, ctx->nblk,
                                   ctx->stream);
            ctx->launches += 2;
            CK(cudaGetLastError());
            rc = read_tail(ctx, ctx->ks);
            if (rc) return rc;
            beta = ctx->h_ks->beta;
            bad |= ctx->h_ks->bad_index;
        }
        if (info) {
            info->iters = total;
            info->refinements = refinements;
            info->guess_relres = first;
            info->final_relres = rel_residual(beta, bnorm);
            info->status = status;
        }
        if (bad) status = SEQ_EINVAL;
    }
    if (info) info->launches = ctx->launches;
    if (ctx->h_ks->bad_index) {
        if (info) info->status = SEQ_EINVAL;
        return fail(ctx, SEQ_EINVAL, "CSR column index outside [0, n)");
    }
    if (status == SEQ_NOT_CONVERGED) ctx->err = "iteration cap reached";
    return status;
}

int seq_set_profiling(seq_ctx* ctx, int on) {
    if (!ctx) return SEQ_EINVAL;
    ctx->profiling = on != 0;
    return SEQ_OK;
}

int seq_kernel_stats(seq_ctx* ctx, seq_kernel_stat* out, int reset) {
    if (!ctx || !out) return SEQ_EINVAL;
    memcpy(out, ctx->stats, sizeof(ctx->stats));
    if (reset) memset(ctx->stats, 0, sizeof(ctx->stats));
    return SEQ_OK;
}

const char* seq_last_error(const seq_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

int seq_last_sketch(seq_ctx* ctx, double* W_host, double* y_host) {
    if (!ctx) return SEQ_EINVAL;
    const int m = ctx->lsq_host->m;
    CK(cudaStreamSynchronize(ctx->stream));
    if (W_host && m > 0)
        CK(cudaMemcpy(W_host, ctx->lsq->W_logical, sizeof(double) * ctx->cfg.s * (m + 1),
                      cudaMemcpyDeviceToHost));
    if (y_host && m > 0)
        CK(cudaMemcpy(y_host, ctx->lsq->y_logical, sizeof(double) * m, cudaMemcpyDeviceToHost));
    return SEQ_OK;
}

int seq_rand_state(seq_ctx* ctx, double* omega_host, double* Z_host, uint64_t* draws,
                   int32_t* updates) {
    if (!ctx) return SEQ_EINVAL;
    if (ctx->cfg.guess != SEQ_GUESS_RAND || !ctx->om_valid)
        return fail(ctx, SEQ_EINVAL, "no Omega: not in RAND mode or no guess yet");
    const int n = ctx->cfg.n, M = ctx->cfg.M, mb = ctx->cfg.basis_m;
    const int mi = seq_history_size(ctx), oldest = (ctx->pushes - mi) % M;
    CK(cudaStreamSynchronize(ctx->stream));
    if (omega_host)
        CK(cudaMemcpy2D(omega_host, sizeof(double) * mb, ctx->Om, sizeof(double) * ctx->ldo,
                        sizeof(double) * mb, n, cudaMemcpyDeviceToHost));
    if (Z_host) {
        std::vector<double> z((size_t)M * mb);
        CK(cudaMemcpy(z.data(), ctx->Zs, sizeof(double) * z.size(), cudaMemcpyDeviceToHost));
        for (int l = 0; l < mi; ++l)
            memcpy(Z_host + (size_t)l * mb, z.data() + (size_t)((oldest + l) % M) * mb, sizeof(double) * mb);
    }
    if (draws) *draws = ctx->gdraws;
    if (updates) *updates = ctx->om_updates;
    return SEQ_OK;
}

int seq_pod_state(seq_ctx* ctx, double* V_host, double* lam_host, int32_t* dims) {
    if (!ctx) return SEQ_EINVAL;
    if (ctx->cfg.guess != SEQ_GUESS_POD) return fail(ctx, SEQ_EINVAL, "not in POD mode");
    CK(cudaStreamSynchronize(ctx->stream));
    const int mi = ctx->pod_mi, kk = ctx->pod_kk;
    if (V_host && mi > 0)
        CK(cudaMemcpy(V_host, ctx->Vk, sizeof(double) * mi * kk, cudaMemcpyDeviceToHost));
    if (lam_host && mi > 0)
        CK(cudaMemcpy(lam_host, ctx->lam, sizeof(double) * mi, cudaMemcpyDeviceToHost));
    if (dims) {
        dims[0] = mi;
        dims[1] = kk;
        dims[2] = 0;
        if (mi > 0) CK(cudaMemcpy(&dims[2], ctx->sweeps, sizeof(int), cudaMemcpyDeviceToHost));
    }
    return SEQ_OK;
}

int seq_sketch_columns(int32_t n, int32_t s, int32_t zeta, uint64_t seed, int32_t* rows_dev,
                       int8_t* signs_dev, void* cuda_stream) {
    if (n <= 0 || s < 1 || s > kMaxS || zeta < 1 || zeta > s || zeta > kMaxZeta || !rows_dev ||
        !signs_dev)
        return SEQ_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    launch_sketch_columns(n, s, zeta, seed, nullptr, rows_dev, signs_dev, st);
    if (cudaGetLastError() != cudaSuccess) return SEQ_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? SEQ_OK : SEQ_ECUDA;
}

int seq_probe_fp64_peak(void* cuda_stream, double* tflops) {
    if (!tflops) return SEQ_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SEQ_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256, iters = 1 << 13;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return SEQ_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        launch_fp64_probe(out, blocks, threads, iters, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return SEQ_ECUDA;
    // 8 independent FMA chains per thread, 2 flops each.
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
    return SEQ_OK;
}

}  // extern "C"
