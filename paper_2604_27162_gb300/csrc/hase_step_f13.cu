// hase_step_f13.cu -- the fused step kernel, family 13: the one-thread emission with line of sight for 1 to 4 agents, windows of two words a plane, CTAs of up to 384 threads (168 registers).
#include "hase_step.cuh"

namespace hase {

cudaError_t opt_in_f13(int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step_kernel<384, 1, 13>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_kernel<384, 1, 13>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

cudaError_t launch_f13(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem, cudaStream_t st) {
    if (threads > 384u) return cudaErrorInvalidConfiguration;
    step_kernel<384, 1, 13><<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hase
