// Learned predictor pieces shared between mlp.cu and api.cu (internal).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

struct seq_mlp;

namespace sa {
void launch_learned_sample(const LsqOut* lo, int s, int M, const double* yring, float* sample,
                           cudaStream_t st);
void launch_learned_select(LsqOut* lo, int s, int M, int oldest, const float* yhat, int* used,
                           double* rho_net, cudaStream_t st);
void launch_yring_push(double* yring, const LsqOut* lo, int M, cudaStream_t st);
void mlp_predict_dev(seq_mlp* m, const float* features, int B, float* y, cudaStream_t st);
int mlp_stride(const seq_mlp* m);
int mlp_dims_ok(const seq_mlp* m, int M, int s);
int mlp_hidden(const seq_mlp* m);
int mlp_max_batch(const seq_mlp* m);
}  // namespace sa
