// hase_step_f14.cu -- the fused step kernel, family 14: the one-thread emission with line of sight for 5 to 8 agents, windows of two words a plane, CTAs of up to 384 threads (168 registers).
#include "hase_step.cuh"

namespace hase {

cudaError_t opt_in_f14(int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step_kernel<384, 1, 14>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_kernel<384, 1, 14>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

cudaError_t launch_f14(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem, cudaStream_t st) {
    if (threads > 384u) return cudaErrorInvalidConfiguration;
    step_kernel<384, 1, 14><<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hase
