// hase_step_f12.cu -- the fused step kernel, family 12: the one-thread emission with line of sight for 13 to 16 agents (one-word windows), CTAs of up to 384 threads (168 registers).
#include "hase_step.cuh"

namespace hase {

cudaError_t opt_in_f12(int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step_kernel<384, 1, 12>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_kernel<384, 1, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

cudaError_t launch_f12(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem, cudaStream_t st) {
    if (threads > 384u) return cudaErrorInvalidConfiguration;
    step_kernel<384, 1, 12><<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hase
