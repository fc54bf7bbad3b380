// Host-side launchers of the seqaccel kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sa {

// sketch.cu
int sketch_grid(int n, int s, int M);   // blocks of launch_sketch_* for up to M columns
size_t sketch_partial_doubles(int n, int s, int M);   // partial buffer of launch_sketch_*
void launch_sketch_columns(int n, int s, int zeta, uint64_t seed, uint16_t* packed,
                           int32_t* rows, int8_t* signs, cudaStream_t st);
// W = S [A X | b] (s x (M+1), row-major, scaled by 1/sqrt(zeta)) with the sparse-sign S
// of (n, s, zeta, seed) generated on the fly; partial: sketch_partial_doubles doubles.
void launch_sketch_f64(const int* rowptr, const int* colind, const double* val, const double* X,
                       int ldx, const double* b, int n, int nnz, int M, int s, int zeta,
                       uint64_t seed, double* partial, int nblk, double* W, int* bad,
                       cudaStream_t st);
void launch_sketch_f32(const int* rowptr, const int* colind, const float* val, const float* X,
                       int ldx, const double* b, int n, int nnz, int M, int s, int zeta,
                       uint64_t seed, double* partial, int nblk, double* W, int* bad,
                       cudaStream_t st);

// lsq.cu
struct LsqOut {
    double y_logical[kMaxM];
    double y_phys[kMaxM];
    double W_logical[kMaxS * (kMaxM + 1)];   // s x (m+1), row-major, b last
    double rho;
    int rank;
    int m;
};
void launch_lsq(const double* W, int s, int M, int m, int oldest_slot, double tau, LsqOut* out,
                cudaStream_t st);
void launch_expand_f64(const double* X, int ldx, int n, int M, const LsqOut* lo, double* x0,
                       cudaStream_t st);
void launch_expand_f32(const float* X, int ldx, int n, int M, const LsqOut* lo, double* x0,
                       cudaStream_t st);
void launch_copy_slot_f64(const double* X, int ldx, int n, int slot, double* x0, cudaStream_t st);
void launch_copy_slot_f32(const float* X, int ldx, int n, int slot, double* x0, cudaStream_t st);
void launch_push_f64(const double* x, int n, double* X, int ldx, int slot, cudaStream_t st);
void launch_push_f32(const double* x, int n, float* X, int ldx, int slot, cudaStream_t st);

// basis.cu: POD (Algorithm 2) and randomised range finder (Algorithm 4)
int gram_grid();
size_t gram_partial_doubles();
void launch_rand_scratch(const double* X, int ldx, int n, int M, int mi, int oldest, double* Zs, int m,
                         uint64_t gseed, uint64_t start, double* Om, int ldo, cudaStream_t st);
void launch_rand_push(const double* x, int n, double* X, int ldx, int slot, int remove, double* Zs,
                      int m, uint64_t gseed, uint64_t start, double* Om, int ldo, cudaStream_t st);
void launch_pod_basis(const double* X, int ldx, int n, int M, int mi, int oldest, int kk,
                      double* partial, unsigned* counter, double* G, double* Vk, double* lam,
                      int* sweeps, cudaStream_t st);
void launch_pod_reduce(const double* W, int s, int M, int mi, int oldest, const double* Vk, int kk,
                       double* Wp, cudaStream_t st);
void launch_pod_coeff(const LsqOut* red, const double* Vk, int mi, int kk, int M, int oldest,
                      LsqOut* out, cudaStream_t st);

// krylov.cu
int stream_grid(int n);
// Arnoldi kernels per step: FP64 SpMV, first-pass dots, pass 2, pass 3; FP32
// fuses the SpMV with the first-pass dots.
inline int step_kernels(bool f32) { return f32 ? kKernelsPerStep - 1 : kKernelsPerStep; }
// Kernels of one preconditioner application of degree `sweeps`: the scale
// kernel alone for one sweep, else sweeps - 1 sweep kernels (the first forms
// the scaled start vector itself).
inline int precond_kernels(int sweeps) { return sweeps <= 1 ? sweeps : sweeps - 1; }
// Kernels of one restart cycle: per Arnoldi step the preconditioner's kernels
// and the Arnoldi kernels; then the update (combine, preconditioner, axpy; or
// one update kernel) and the restart residual.
inline int cycle_kernels(int R, int sweeps, bool f32) {
    const int pk = precond_kernels(sweeps);
    return (step_kernels(f32) + pk) * R + (sweeps > 0 ? pk + 2 : 1) + 1;
}
// Timing marks of a profiled cycle: one per kernel, one per preconditioner
// application (its sweeps run back to back between two events).
inline int cycle_marks(int R, int sweeps, bool f32) {
    const int pm = sweeps > 0 ? 1 : 0;
    return (step_kernels(f32) + pm) * R + (sweeps > 0 ? 3 : 1) + 1;
}
// ||b - A x|| and ||b|| of FP64 vectors; results in st->beta, st->bnorm and
// st->first_relres = beta / bnorm.
void launch_residual_norm(const DevArgs* a, KState* ks, double* partial, int nblk,
                          const double* x_override, cudaStream_t st);
// Restarted GMRES(R) with CGS2 on the FP64 system: the start kernel and one
// full cycle (R Arnoldi steps, basis update, residual of the updated iterate).
void launch_gmres_start_f64(const DevArgs* a, KState* ks, double* V, size_t ldv, double* partial,
                            int nblk, int first, cudaStream_t st);
// Right preconditioning (sweeps > 0): M^{-1} = `sweeps` damped Jacobi sweeps
// with weight omega and dinv = 1 / diag(A), or (cheb->on) the Chebyshev
// polynomial of degree `sweeps` on [lmax / ratio, lmax] of D^{-1} A, whose
// coefficients launch_cheb_table writes into cheb->tab once per solve (after
// launch_diag_inv_* has left the Gershgorin bound in its first word); za, zb,
// t, dvec: n-vectors of scratch.
struct ChebConfig {
    int on;
    const double* tab;                    // kChebTab doubles
};
void launch_cheb_table(double* tab, double lfix, double ratio, int sweeps, cudaStream_t st);
void launch_gmres_cycle_f64(const DevArgs* a, KState* ks, double* V, size_t ldv, double* w,
                            double* partial, int nblk, int R, cudaStream_t st, int* launches,
                            cudaEvent_t* ev = nullptr, int sweeps = 0, double omega = 1.0,
                            const double* dinv = nullptr, double* za = nullptr,
                            double* zb = nullptr, double* t = nullptr,
                            const ChebConfig* cheb = nullptr, double* dvec = nullptr);
// dinv = 1 / diag(A); with bound (zeroed by the caller) also the Gershgorin
// bound max_i sum_j |a_ij| / |a_ii| as the bits of a double.
void launch_diag_inv_f64(const DevArgs* a, double* dinv, int n, cudaStream_t st,
                         unsigned long long* bound = nullptr);
// Same on the FP32 inner system A32 d = rhs32 (mixed precision).
void launch_gmres_start_f32(const DevArgs* a, KState* ks, float* V, size_t ldv, float* partial,
                            int nblk, int first, cudaStream_t st);
void launch_gmres_cycle_f32(const DevArgs* a, KState* ks, float* V, size_t ldv, float* w,
                            float* partial, int nblk, int R, cudaStream_t st, int* launches,
                            cudaEvent_t* ev = nullptr, int sweeps = 0, double omega = 1.0,
                            const float* dinv = nullptr, float* za = nullptr,
                            float* zb = nullptr, float* t = nullptr,
                            const ChebConfig* cheb = nullptr, float* dvec = nullptr);
void launch_diag_inv_f32(const DevArgs* a, float* dinv, int n, cudaStream_t st,
                         unsigned long long* bound = nullptr);
// Mixed precision outer step: the FP64 residual r = b - A64 x (into r64) with
// st->beta = ||r|| and ||b||; the FP32 right-hand side rhs32 = r / ||r||; and
// after the inner solve x += ||r|| d (FP64 += FP32).
void launch_refine_residual(const DevArgs* a, KState* ks, double* r64, double* partial, int nblk,
                            cudaStream_t st);
void launch_refine_scale(const double* r64, const KState* ks, float* rhs32, int n, cudaStream_t st);
void launch_refine_update(const DevArgs* a, const KState* outer, cudaStream_t st);
// Single-block CG (T = double: FP64 system; the kernel loops on the device).
void launch_cg_block_f64(const DevArgs* a, KState* ks, double* r, double* p, double* q,
                         cudaStream_t st);
void launch_cg_block_f32(const DevArgs* a, KState* ks, float* r, float* p, float* q,
                         cudaStream_t st);
void launch_round_f32(const double* src, float* dst, int n, cudaStream_t st);
// Grid-wide CG for large systems (all SMs; three kernels per iteration): the
// start (FP32: from x = 0), `iters` iterations (the body of a CUDA graph), and
// the true residual (check != 0: convergence check and restart).
constexpr int kGridCgMinRows = 65536;
constexpr int kGridCgGraphIters = 16;
void launch_cgg_start_f64(const DevArgs* a, KState* ks, double* r, double* p, double* partial,
                          int nblk, cudaStream_t st);
void launch_cgg_start_f32(const DevArgs* a, KState* ks, float* r, float* p, float* partial,
                          int nblk, cudaStream_t st);
void launch_cgg_iterations_f64(const DevArgs* a, KState* ks, double* r, double* p, double* q,
                               double* partial, int nblk, int iters, cudaStream_t st);
void launch_cgg_iterations_f32(const DevArgs* a, KState* ks, float* r, float* p, float* q,
                               float* partial, int nblk, int iters, cudaStream_t st);
void launch_cgg_true_residual_f64(const DevArgs* a, KState* ks, double* r, double* p,
                                  double* partial, int nblk, int check, cudaStream_t st);
void launch_cgg_true_residual_f32(const DevArgs* a, KState* ks, float* r, float* p,
                                  float* partial, int nblk, int check, cudaStream_t st);
// CSR -> SELL-32 (slice widths and offsets, then the padded arrays).
// off needs (n + 31) / 32 + 2 entries: off[ns] = total, off[ns + 1] = widest slice.
void launch_sell_layout(const int* rowptr, int n, int nnz, int* width, int* off, cudaStream_t st);
// Re-layout with every slice of width w (off[s] = 32 w s).
void launch_sell_uniform(int n, int w, int* off, cudaStream_t st);
void launch_sell_fill_f64(const int* rowptr, const int* colind, const double* val, int n, int nnz,
                          const int* off, int* col, double* v, cudaStream_t st);
void launch_sell_fill_f32(const int* rowptr, const int* colind, const float* val, int n, int nnz,
                          const int* off, int* col, float* v, cudaStream_t st);

// probe.cu
void launch_fp64_probe(double* out, int blocks, int threads, int iters, cudaStream_t st);

}  // namespace sa
