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
                            cudaEvent_t* ev, int sweeps, double omega, const float* dinv,
                            float* za, float* zb, float* t, const ChebConfig* cheb, float* dvec) {
    PrecondArgs<float> pc;
    pc.sweeps = sweeps;
    pc.omega = omega;
    pc.dinv = dinv;
    pc.za = za;
    pc.zb = zb;
    pc.t = t;
    if (cheb && cheb->on) {
        pc.cheb = 1;
        pc.tab = cheb->tab;
        pc.dvec = dvec;
    }
    launch_cycle<SysF32>(a, ks, V, ldv, w, partial, nblk, R, st, launches, ev, pc);
}
void launch_diag_inv_f32(const DevArgs* a, float* dinv, int n, cudaStream_t st,
                         unsigned long long* bound) {
    int b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    diag_inv_kernel<SysF32><<<b > 0 ? b : 1, 256, 0, st>>>(a, dinv, bound);
}

}  // namespace sa
