// hase_step_f15.cu -- the fused step kernel, family 15: the one-thread emission with line of sight for 9 to 12 agents, windows of two words a plane, CTAs of up to 384 threads (168 registers).
#include "hase_step.cuh"

namespace hase {

cudaError_t opt_in_f15(int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step_kernel<384, 1, 15>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_kernel<384, 1, 15>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

cudaError_t launch_f15(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem, cudaStream_t st) {
    if (threads > 384u) return cudaErrorInvalidConfiguration;
    step_kernel<384, 1, 15><<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hase
