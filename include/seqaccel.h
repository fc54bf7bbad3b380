/*
 * seqaccel — subspace-accelerated solution of a sequence of sparse linear
 * systems A(t_i) x(t_i) = b(t_i), i = 0, 1, 2, ... on one GPU (sm_103a).
 *
 * Method (Guido, Kressner, Ricci, arXiv 2309.02156):
 *   Section 1, eq. (1)   the systems arrive one at a time;
 *   Section 2            history X = [x(t_{i-M}) | ... | x(t_{i-1})], shifted
 *                        by one column per system;
 *   Algorithm 1          guess = argmin over span(X) of ||A(t_i) s - b(t_i)||_2,
 *                        then the Krylov solver starts from it.
 * Here the reduced least-squares problem of Algorithm 1 is sketched
 * with a sparse-sign matrix S (s x n, zeta nonzeros of +-1/sqrt(zeta) per
 * column, generated from SplitMix64 counters):
 *   W = S [A X | b],  y = argmin ||W[:, :m] y - W[:, m]||_2 (pivoted Householder
 *   QR, rank truncation), x0 = X y;
 * then CG (SPD) or restarted GMRES with CGS2 Arnoldi (Section 1, the solve of
 * Algorithm 1) runs from x0 to ||b - A x|| <= tol ||b||.
 *
 * Conventions for every entry point
 *   - Pointers named *_dev are DEVICE pointers owned by the caller and only
 *     borrowed for the duration of the call; pointers named *_host are host
 *     pointers.  Vectors are dense, contiguous, length n.
 *   - All work is ordered on the CUDA stream given to seq_create.  Calls that
 *     return a seq_info synchronise that stream before returning.
 *   - Matrices are CSR with int32 row pointers (n+1) and column indices (nnz);
 *     column indices outside [0, n) are skipped by the kernels and reported as
 *     SEQ_EINVAL.
 *   - Return values are seq_status codes; no exception or abort crosses the
 *     boundary.  seq_last_error() describes the last failure of a context.
 *   - A context is not thread safe; distinct contexts are independent.
 */
#ifndef SEQACCEL_H
#define SEQACCEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct seq_ctx seq_ctx;

typedef enum {
    SEQ_OK = 0,               /* converged / done                              */
    SEQ_NOT_CONVERGED = 1,    /* iteration cap reached; x holds the last iterate */
    SEQ_FALLBACK_USED = 2,    /* learned guess rejected, sketched LS used        */
    SEQ_EINVAL = -1,          /* bad argument or malformed CSR                   */
    SEQ_ENOMEM = -2,          /* device or pinned allocation failed              */
    SEQ_ECUDA = -3,           /* a CUDA runtime call failed                      */
    SEQ_EBREAKDOWN = -4,      /* CG p^T A p <= 0, or a singular Hessenberg       */
    SEQ_ENONFINITE = -5,      /* NaN or Inf met in a residual norm               */
    SEQ_ETIMEOUT = -6         /* a bounded device-side wait expired              */
} seq_status;

typedef enum {
    SEQ_F64 = 0,          /* FP64 everywhere                                            */
    SEQ_MIXED = 1,        /* FP32 values, history, sketch and inner Krylov; FP64 QR,
                             refinement residual b - A x and convergence test         */
    SEQ_MIXED_KRYLOV = 2  /* FP64 history, sketch, QR and guess; FP32 inner Krylov
                             inside FP64 iterative refinement                         */
} seq_precision;

typedef enum {
    SEQ_GUESS_ZERO = 0,     /* x0 = 0                                                  */
    SEQ_GUESS_PREV = 1,     /* x0 = x(t_{i-1}), the paper's baseline (Sections 4-5)    */
    SEQ_GUESS_SKETCH = 2,   /* x0 = X y, y from the sketched least squares (Alg. 1)    */
    SEQ_GUESS_LEARNED = 3,  /* y predicted by the coefficient MLP, sketched LS fallback */
    SEQ_GUESS_POD = 4,      /* Algorithm 1 over span(Q_POD), Q_POD = the basis_m leading
                               left singular vectors of X (Algorithm 2)               */
    SEQ_GUESS_RAND = 5      /* Algorithm 1 over span(Omega), Omega = X Z with a Gaussian
                               Z (n x basis_m), updated progressively at every push and
                               recomputed every `refresh` updates (Algorithm 4)       */
} seq_guess_mode;

typedef enum { SEQ_CG = 0, SEQ_GMRES = 1 } seq_krylov;

typedef struct {
    int32_t n;                 /* rows = columns                                  */
    int32_t nnz;               /* stored entries                                  */
    const int32_t* rowptr;     /* device, n+1, rowptr[0] = 0, non-decreasing      */
    const int32_t* colind;     /* device, nnz                                     */
    const double* values;      /* device, nnz, FP64                               */
    const float* values_f32;   /* device, nnz, FP32 copy used by the FP32 inner
                                  solves (and the FP32 sketch of SEQ_MIXED); NULL:
                                  the library rounds `values`                      */
} seq_csr;

typedef struct {
    int32_t n;            /* unknowns per system                                   */
    int32_t M;            /* history length, 1..31                                 */
    int32_t s;            /* sketch rows, M+1..128                                  */
    int32_t zeta;         /* nonzeros per sketch column, 1..min(s, 16)             */
    uint64_t seed;        /* sketch seed (S is fixed for the life of the context)  */
    int32_t precision;    /* seq_precision                                         */
    int32_t guess;        /* seq_guess_mode                                        */
    int32_t krylov;       /* seq_krylov                                            */
    int32_t restart;      /* GMRES restart length, 1..64                           */
    int32_t max_iters;    /* Krylov iteration cap per solve (inner iterations in
                             the mixed modes)                                      */
    double inner_tol;     /* mixed modes: floor of the inner relative tolerance;
                             0 selects 1e-2                                        */
    double rank_tol;      /* QR truncation tau; 0 selects 1e-12 for an FP64 sketch
                             or 1e-5 for an FP32 sketch (SEQ_MIXED)                */
    int32_t basis_m;      /* SEQ_GUESS_POD / SEQ_GUESS_RAND: basis size m, 1..M
                             (ignored by the other modes)                          */
    int32_t refresh;      /* SEQ_GUESS_RAND: progressive updates between from-scratch
                             computations of Omega; 0 selects 50 (Section 4)       */
    int32_t precond_sweeps; /* GMRES only: right preconditioner M^{-1} = this many
                             damped Jacobi sweeps on A z = u from z = 0 (0: none,
                             at most 32); the minimised and tested residual stays
                             the true one (x = x0 + M^{-1} V y)                   */
    double precond_omega; /* sweep weight omega in (0, 2); 0 selects 0.8          */
    int32_t precond_kind; /* 0: the damped Jacobi sweeps above; 1: the Chebyshev
                             polynomial of degree precond_sweeps on the interval
                             [lmax / precond_ratio, lmax] of the spectrum of
                             D^{-1} A (the minimax residual polynomial on it,
                             applied by the Chebyshev iteration from z = 0: the
                             cost of as many sweeps plus one vector)           */
    double precond_ratio; /* Chebyshev: lmax / lmin > 1; 0 selects 30             */
    double precond_lmax;  /* Chebyshev: lmax; 0: Gershgorin's bound
                             max_i sum_j |a_ij| / |a_ii|, formed at every solve   */
} seq_config;

typedef struct {
    int32_t iters;          /* Krylov iterations (inner iterations summed, mixed modes) */
    int32_t refinements;    /* FP64 refinement steps (mixed modes)                      */
    int32_t history_cols;   /* history columns the guess used                          */
    int32_t rank;           /* columns kept by the pivoted QR                           */
    double guess_relres;    /* ||b - A x0|| / ||b|| of the starting vector              */
    double sketch_resid;    /* ||W1 y - wb||_2 (sketched residual)                      */
    double final_relres;    /* true ||b - A x|| / ||b|| at exit (seq_solve)             */
    int32_t status;         /* seq_status of the call                                   */
    int32_t launches;       /* kernels this call launched (graph nodes included)        */
    double net_resid;       /* SEQ_GUESS_LEARNED: sketched residual ||W1 y_net - S b|| of
                               the network's y, whether used or rejected; -1 when no
                               prediction was made (history not full)               */
} seq_info;

/* Create a context for one sequence (Section 2: one history X per sequence).
 * Allocates the history ring (n x M), per-block partial sketched blocks, the
 * Krylov workspace (GMRES: n x (restart+1) basis) and small device state.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: SEQ_EINVAL (cfg out of range), SEQ_ENOMEM, SEQ_ECUDA.  *out is NULL
 * on failure. */
int seq_create(const seq_config* cfg, void* cuda_stream, seq_ctx** out);

/* Free everything the context owns.  NULL is accepted. */
int seq_destroy(seq_ctx* ctx);

/* Append x(t_i) to the history and drop the oldest column once M are held
 * (Section 2.1: each time step the oldest solution leaves X and the newest
 * one is appended).  x_dev: device, n FP64 values (rounded to FP32 in
 * SEQ_MIXED).  Stream-ordered; does not synchronise. */
int seq_push_solution(seq_ctx* ctx, const double* x_dev);

/* Number of history columns currently held (0..M). */
int seq_history_size(const seq_ctx* ctx);

/* Initial guess for A x = b (the guess of Algorithm 1, with the sketched reduced
 * problem; or the guess mode chosen in the config).  Writes x0_dev (device, n
 * FP64).  With an empty history x0 = 0; with m < M columns the m available
 * ones are used.  Fills info (guess_relres, sketch_resid, rank, history_cols;
 * net_resid in SEQ_GUESS_LEARNED).  guess_relres is ||b - A x0|| / ||b||, or
 * ||b - A x0|| when b = 0.  Synchronises the stream.
 * Returns SEQ_OK, or SEQ_FALLBACK_USED (learned mode: the network's y was
 * rejected and the least-squares y used; x0 is valid).
 * Errors: SEQ_EINVAL (bad argument or column index), SEQ_ENONFINITE (NaN or
 * Inf in the residual of the guess), SEQ_ECUDA. */
int seq_guess(seq_ctx* ctx, const seq_csr* A, const double* b_dev,
              double* x0_dev, seq_info* info);

/* Krylov solve from x_dev (the solve of Algorithm 1): on entry x_dev holds the
 * starting vector, on exit the iterate with ||b - A x|| <= tol ||b|| (status
 * SEQ_OK) or the last iterate (SEQ_NOT_CONVERGED after max_iters iterations).
 * CG or GMRES(restart) with CGS2 per the config, optionally right-
 * preconditioned (precond_sweeps); the mixed precisions run FP32 inner solves
 * inside FP64 iterative refinement of the true residual (a GMRES inner solve
 * is one restart cycle).  CG runs in one thread block for n < 65,536 and on
 * the whole GPU above (three kernels per iteration, captured as a CUDA graph
 * of 16 iterations); the algorithm and its stopping test are the same.  With b = 0 the
 * test is ||b - A x|| <= 0 and x = 0 passes it.  Does not push x.
 * Synchronises.
 * Errors: SEQ_EINVAL, SEQ_EBREAKDOWN (CG p^T A p <= 0, singular Hessenberg),
 * SEQ_ENONFINITE (NaN or Inf met), SEQ_ETIMEOUT (host cycle bound), SEQ_ECUDA. */
int seq_solve(seq_ctx* ctx, const seq_csr* A, const double* b_dev, double tol,
              double* x_dev, seq_info* info);

/* Description of the last error of ctx ("" if none).  Valid until the next
 * call on ctx. */
const char* seq_last_error(const seq_ctx* ctx);

/* The sketched block and coefficients of the last seq_guess, in logical
 * history order (oldest column first): W_host (s x (m+1), row-major, b last)
 * and y_host (m), where m = info.history_cols of that call.  In the POD and
 * RAND modes they are the reduced problem's block [S A B | S b] and its
 * coefficients c over the basis B (X V_k, resp. Omega), m = basis columns.
 * Either pointer may be NULL.  Diagnostic; synchronises. */
int seq_last_sketch(seq_ctx* ctx, double* W_host, double* y_host);

/* Algorithm 4 state of a SEQ_GUESS_RAND context (diagnostic; synchronises):
 * omega_host (n x basis_m, row-major), Z_host (history_size x basis_m, oldest
 * history column first), the number of Gaussian values drawn so far and the
 * progressive updates since the last from-scratch Omega.  Any pointer may be
 * NULL.  SEQ_EINVAL if the context is not in RAND mode or Omega was never
 * formed. */
int seq_rand_state(seq_ctx* ctx, double* omega_host, double* Z_host, uint64_t* draws,
                   int32_t* updates);

/* Algorithm 2 state of the last SEQ_GUESS_POD guess (diagnostic; synchronises):
 * V_host (m_i x k, column-major: the k leading eigenvectors of X^T X over the
 * m_i history columns, oldest first), lam_host (m_i eigenvalues, descending),
 * dims[0] = m_i, dims[1] = k, dims[2] = Jacobi sweeps.  Pointers may be NULL. */
int seq_pod_state(seq_ctx* ctx, double* V_host, double* lam_host, int32_t* dims);

/* Materialise the sparse-sign sketch used by every context with the same
 * (n, s, zeta, seed): for column j, rows_dev[j*zeta + k] and signs_dev[j*zeta + k]
 * (+1/-1) in acceptance order (see the oracle's definition: candidates are
 * SplitMix64 outputs 256 j + c + 1, row = ((h >> 32) s) >> 32, sign = bit 0,
 * duplicates skipped).  1 <= zeta <= min(s, 16), s <= 128 (SEQ_EINVAL otherwise).
 * Device pointers; stream-ordered; synchronises. */
int seq_sketch_columns(int32_t n, int32_t s, int32_t zeta, uint64_t seed,
                       int32_t* rows_dev, int8_t* signs_dev, void* cuda_stream);

/* Kernel kinds reported by seq_kernel_stats (the GMRES cycle of the solve of
 * Algorithm 1, and the stages of the guess). */
typedef enum {
    SEQ_K_SPMV = 0,       /* w = A v_j (FP32 inner solves: fused with the first CGS pass) */
    SEQ_K_CGS_DOT = 1,    /* first classical Gram-Schmidt pass h1 = V^T w               */
    SEQ_K_CGS_PASS2 = 2,  /* w -= V h1 fused with the second pass h2 = V^T w             */
    SEQ_K_CGS_PASS3 = 3,  /* w -= V h2, ||w||, Givens update (basis column j+1)          */
    SEQ_K_UPDATE = 4,     /* x += V y at the end of a restart cycle                      */
    SEQ_K_RESTART = 5,    /* r = b - A x, ||r|| at a cycle start                         */
    SEQ_K_PRECOND = 6,    /* preconditioner kernels (scale and Jacobi sweeps)            */
    SEQ_K_COUNT = 7
} seq_kernel_kind;

typedef struct {
    int64_t launches;     /* launches that did work                               */
    double ms;            /* summed device time between the launch's boundary events */
    double bytes;         /* summed algorithmic DRAM bytes (each operand once)    */
    double flops;         /* summed algorithmic floating-point operations         */
} seq_kernel_stat;

/* Turn per-kernel timing of seq_solve on (on != 0) or off.  When on, the GMRES
 * cycle graph records a CUDA event between consecutive kernels (on the
 * context's stream), and seq_kernel_stats accumulates, per kernel kind, the
 * device time and the algorithmic traffic of every launch that did work.  The
 * events add a small overhead to each cycle.  GMRES only. */
int seq_set_profiling(seq_ctx* ctx, int on);

/* Copy the accumulated per-kind statistics into out[SEQ_K_COUNT]; reset != 0
 * clears them afterwards. */
int seq_kernel_stats(seq_ctx* ctx, seq_kernel_stat* out, int reset);

/* Measure this device's FP64 fused multiply-add throughput (TFLOP/s, counting
 * 2 flops per FMA) with a register-only kernel of about 50 ms.  Used as the
 * arithmetic roof of the FP64 kernels.  Synchronises. */
int seq_probe_fp64_peak(void* cuda_stream, double* tflops);

/* ---- Learned coefficient predictor (SEQ_GUESS_LEARNED) ----
 *
 * Not in the paper (Algorithm 1 solves for y every step).  A small MLP,
 * 4M+s -> H -> H -> M with GELU, bfloat16 weights and FP32 accumulation,
 * predicts y from the previous four coefficient vectors (shifted into the
 * current window) and the sketched residual of the linear extrapolation
 * 2 x(t_{i-1}) - x(t_{i-2}); y_hat = shift(y_{i-1}) + sigma_out * net.  In
 * SEQ_GUESS_LEARNED, seq_guess uses y_hat unless its sketched residual
 * exceeds 1.5 times that of the least-squares y, in which case it falls back
 * to least squares and returns SEQ_FALLBACK_USED.
 *
 * Training data: after every seq_guess with a full history and four previous
 * guesses, seq_last_sample writes the sample of that guess, FP32, stride
 * (4M+s) + M + M*M + 1: [features | least-squares y | W1^T W1 | ||S b||].
 * Loss of a sample: (y_hat - y)^T W1^T W1 (y_hat - y) / ||S b||^2 (the
 * excess sketched residual).  Training runs on the GPU (hand-written forward
 * and backward kernels, Adam). */
typedef struct seq_mlp seq_mlp;

/* He-uniform weights from SplitMix64 counters (seed), zero biases, identity
 * normalisation.  max_batch bounds the batch of train / loss_grad / predict. */
int seq_mlp_create(int32_t M, int32_t s, int32_t hidden, int32_t max_batch, uint64_t seed,
                   void* cuda_stream, seq_mlp** out);
int seq_mlp_destroy(seq_mlp* mlp);
/* Number of FP32 parameters: W1 (H x (4M+s)), b1, W2 (H x H), b2, W3 (M x H), b3. */
int seq_mlp_param_count(const seq_mlp* mlp);
/* Host copies of the parameters (param_count floats, layout above) and of the
 * normalisation (feature mean, feature std, output scale: 2(4M+s) + M floats);
 * either pointer may be NULL.  set also resets the Adam state. */
int seq_mlp_get_params(seq_mlp* mlp, float* params_host, float* norm_host);
int seq_mlp_set_params(seq_mlp* mlp, const float* params_host, const float* norm_host);
/* Feature mean/std and output scale from count samples (device). */
int seq_mlp_fit_normalization(seq_mlp* mlp, const float* samples_dev, int32_t count);
/* Batch-mean loss and its gradient (host, param_count floats) on B samples,
 * without updating. */
int seq_mlp_loss_grad(seq_mlp* mlp, const float* samples_dev, int32_t B, float* loss_host,
                      float* grads_host);
/* epochs of Adam (lr) over count samples in shuffled batches (SplitMix64 seed);
 * losses_host (epochs floats, may be NULL) receives the mean loss per epoch. */
int seq_mlp_train(seq_mlp* mlp, const float* samples_dev, int32_t count, int32_t epochs,
                  int32_t batch, float lr, uint64_t seed, float* losses_host);
/* y_hat (B x M, device) for B samples (device, sample stride; only the
 * features part is read). */
int seq_mlp_predict(seq_mlp* mlp, const float* samples_dev, int32_t B, float* y_dev);
/* Attach (or detach with NULL) a predictor to a context.  The caller keeps
 * ownership of mlp; a predictor the context created itself (seq_learned_train
 * or seq_learned_load) is freed when it is detached or replaced. */
int seq_set_learned(seq_ctx* ctx, seq_mlp* mlp);
/* Sample of the last seq_guess into sample_dev (device); SEQ_EINVAL if that
 * guess had no full history or fewer than four previous guesses. */
int seq_last_sample(seq_ctx* ctx, float* sample_dev);

/* Context-level entry points of the learned form.  Not in the paper (its
 * Algorithm 1 solves for y by least squares at every step); they wrap the
 * seq_mlp object above for the common case of one network per sequence.
 *
 * Train the context's predictor on `count` samples (device, the
 * seq_last_sample layout, stride (4M+s) + M + M*M + 1 floats): if none is
 * attached, the context creates and owns one (hidden width 256, He-uniform
 * initialisation from `seed`); then the normalisation is fitted to the
 * samples and `epochs` epochs of Adam run (learning rate 1e-3, batches of
 * min(32, count) samples shuffled with `seed`).  Equivalent to seq_mlp_create
 * (M, s, 256, 32, seed) + seq_mlp_fit_normalization + seq_mlp_train(epochs,
 * 32, 1e-3, seed) on a fresh network, and the trained network is attached
 * (seq_set_learned).  Synchronises.
 * Errors: SEQ_EINVAL (count < 1, epochs < 0, NULL samples, M < 2),
 * SEQ_ENOMEM, SEQ_ECUDA. */
int seq_learned_train(seq_ctx* ctx, const float* dataset_dev, int32_t count, int32_t epochs,
                      uint64_t seed);

/* Serialised predictor: a 16-byte header of four int32 (0x4C514553, M, s,
 * hidden width H), then the seq_mlp_get_params parameters and normalisation
 * as FP32 (param_count + 2(4M+s) + M floats), host byte order.
 * seq_learned_save writes the attached predictor into weights_host (bytes
 * available) and the size it needs into *needed (may be NULL; weights_host
 * NULL only queries the size).  SEQ_EINVAL without a predictor or when bytes
 * is too small. */
int seq_learned_save(seq_ctx* ctx, void* weights_host, size_t bytes, size_t* needed);

/* Load a serialised predictor (the seq_learned_save layout) into the
 * context: into the attached network when its M, s and H match the header,
 * else into a new network owned by the context (the one it replaces is
 * detached; an owned one is freed).  The Adam state starts from zero.
 * Errors: SEQ_EINVAL (bad header, M or s different from the context's, size
 * not matching the header), SEQ_ENOMEM, SEQ_ECUDA. */
int seq_learned_load(seq_ctx* ctx, const void* weights_host, size_t bytes);

/* ---- Batched form: many independent sequences, one persistent launch per step ----
 *
 * Each sequence k has its own history (M columns, FP64), sketch (seed + k)
 * and fixed sparsity pattern; every step, for every sequence: the sketched
 * guess (Algorithm 1), then FP64 iterative refinement around FP32 CG (the
 * sequences are SPD) to ||b - A x|| <= tol ||b|| (the solve), then the
 * push.  One thread block processes one sequence at a time, taking sequences
 * from a device queue; the step is a single kernel launch captured in a CUDA
 * graph.  Limits: M <= 16, s <= 64, zeta <= min(s, 16). */
typedef struct seq_batch seq_batch;

/* patterns (host array of count seq_csr; device rowptr/colind, values ignored)
 * stay borrowed for the life of the batch.  Allocates per sequence the
 * history (n x M FP64), an FP32 copy of the values and four FP32 vectors.
 * The default schedule is 512 threads, one block per SM, largest first. */
int seq_batch_create(int32_t count, const seq_csr* patterns, int32_t M, int32_t s, int32_t zeta,
                     uint64_t seed, int32_t max_iters, double inner_tol, void* cuda_stream,
                     seq_batch** out);
int seq_batch_destroy(seq_batch* batch);

/* One time step.  values, b, x: host arrays of count device pointers (the
 * step's matrix values in the pattern's CSR order, right-hand side, solution
 * output).  infos (host array of count, or NULL) receives per-sequence
 * results.  Returns the worst status.  Synchronises the stream. */
int seq_batch_step(seq_batch* batch, const double* const* values, const double* const* b,
                   double* const* x, double tol, seq_info* infos);

/* Autotuner: times one non-committing step (no history update) for every
 * schedule (threads per block 256/512/1024, one or two blocks per SM,
 * largest-first or given queue order, one block or a cluster of 4 or 8 CTAs
 * per sequence) on these inputs and keeps the fastest; chosen (3 ints, may be
 * NULL) receives threads, blocks per SM and order (seq_batch_get_schedule
 * also gives the cluster size). */
int seq_batch_autotune(seq_batch* batch, const double* const* values, const double* const* b,
                       double* const* x, double tol, int32_t* chosen);

/* Append x_dev (device, n_k FP64 values) to sequence k's history, as
 * seq_push_solution does for one sequence (steps push automatically; this
 * primes a history from solutions computed elsewhere).  Stream-ordered. */
int seq_batch_push(seq_batch* batch, int32_t k, const double* x_dev);

/* on = 0: seq_batch_step leaves the histories unchanged (the caller pushes
 * with seq_batch_push); on = 1 (default): every step pushes its solutions. */
int seq_batch_set_autopush(seq_batch* batch, int32_t on);

/* Fix the schedule explicitly (e.g. one the autotuner picked earlier); one
 * block per sequence. */
int seq_batch_set_schedule(seq_batch* batch, int32_t threads, int32_t blocks_per_sm,
                           int32_t order_kind);

/* Cluster schedule: each sequence is taken by a thread-block cluster of ctas
 * (1, 2, 4 or 8) CTAs, one per SM, each owning a contiguous range of the
 * sequence's rows; block sums are combined over the cluster through
 * distributed shared memory (same steps and arithmetic, rows split).  Fewer
 * sequences are in flight at once, so their working sets stay in L2 between
 * CG iterations.  ctas = 1 is the one-block schedule with `threads`.  The
 * autotuner also tries clusters of 4 and 8 (512 and 1024 threads). */
int seq_batch_set_cluster(seq_batch* batch, int32_t ctas, int32_t threads, int32_t order_kind);

/* The schedule in use: out[0] threads per block, out[1] blocks per SM,
 * out[2] order (0 largest first, 1 given), out[3] CTAs per sequence. */
int seq_batch_get_schedule(const seq_batch* batch, int32_t* out);

/* The sketched block W = S [A X | b] computed without allocating any device
 * memory.  The paper has no counterpart: this is a deployment variant of the
 * sketch step for callers that cannot call cudaMalloc where they need W --
 * host callbacks and real-time loops that must not block in the allocator
 * (cudaMalloc can synchronise the device and take milliseconds), and hosts
 * that hand the GPU's memory to their own pool or fix the library's memory
 * budget up front, so that a later allocation would fail.
 *
 * Inputs (device): CSR A (n rows, nnz entries), X (n x M, row i at
 * X[i * ldx .. i * ldx + M - 1], column k is the k-th history vector), b (n).
 * Output (device): W_dev, s x (M + 1) row-major, column k < M = S A X[:, k],
 * column M = S b, with the same sparse-sign S (n, s, zeta, seed) as the rest
 * of the library (entries +-1/sqrt(zeta)).
 * Limits: s * (M + 1) <= 4096, M <= 31, zeta <= min(s, 16); larger sizes
 * return SEQ_EINVAL before any GPU work.  Column indices outside [0, n) give
 * SEQ_EINVAL after the call; the next call starts from a cleared flag.
 * Scratch: a fixed device array of about 5 MB defined in the library, held by
 * every GPU that loads the library until the process exits.  All calls share
 * it and it keeps the last call's contents; calls that overlap on the GPU
 * race on it.  The first call on a device looks up the array's address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture.  Each call ends by reading the column-index
 * flag back to the host and synchronising cuda_stream. */
int seq_sketch_block_noalloc(int32_t n, int32_t nnz, const int32_t* rowptr, const int32_t* colind,
                             const double* values, const double* X, int32_t ldx, int32_t M,
                             const double* b, int32_t s, int32_t zeta, uint64_t seed,
                             double* W_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SEQACCEL_H */
