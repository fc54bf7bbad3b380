// FP64 FMA throughput probe: the arithmetic roof of the FP64 kernels.
// Register-only, eight independent dependency chains per thread, bounded
// iteration count; the result is stored so the work cannot be removed.
#include "internal.h"

namespace sa {

__global__ void fp64_probe_kernel(double* out, double a, double b, int iters) {
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

void launch_fp64_probe(double* out, int blocks, int threads, int iters, cudaStream_t st) {
    fp64_probe_kernel<<<blocks, threads, 0, st>>>(out, 0.999999, 1e-7, iters);
}

}  // namespace sa
