// hase_step_f1.cu -- the fused step kernel, family 1: the one-thread emission for 1 to 4 agents, CTAs of up to 384 threads (168 registers).
#include "hase_step.cuh"

namespace hase {

cudaError_t opt_in_f1(int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step_kernel<384, 1, 1>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_kernel<384, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

cudaError_t launch_f1(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem, cudaStream_t st) {
    if (threads > 384u) return cudaErrorInvalidConfiguration;
    step_kernel<384, 1, 1><<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hase
