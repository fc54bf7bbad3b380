// FP32 instantiation of the restarted GMRES kernels (inner solves of the
// mixed-precision form).  The kernel templates live in krylov_kernels.cuh.
#include "krylov_kernels.cuh"

namespace sa {

void launch_gmres_start_f32(const DevArgs* a, KState* ks, float* V, size_t, float* partial,
                            int nblk, int first, cudaStream_t st) {
    launch_start<SysF32>(a, ks, V, partial, nblk, first, st);
}
void launch_gmres_cycle_f32(const DevArgs* a, KState* ks, float* V, size_t ldv, float* w,
                            float* partial, int nblk, int R, cudaStream_t st, int* launches,
                            cudaEvent_t* ev) {
    launch_cycle<SysF32>(a, ks, V, ldv, w, partial, nblk, R, st, launches, ev);
}

}  // namespace sa
