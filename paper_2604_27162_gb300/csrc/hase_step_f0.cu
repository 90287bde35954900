// hase_step_f0.cu -- the fused step kernel, family 0: the general emission (one lane per agent), CTAs of up to 512 threads.
#include "hase_step.cuh"

namespace hase {

cudaError_t opt_in_f0(int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step_kernel<512, 1, 0>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_kernel<512, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

cudaError_t launch_f0(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem, cudaStream_t st) {
    if (threads > 512u) return cudaErrorInvalidConfiguration;
    step_kernel<512, 1, 0><<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hase
