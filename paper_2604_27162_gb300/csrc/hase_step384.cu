// hase_step384.cu -- the fused step kernel for CTAs of up to 384 threads.
#include "hase_step.cuh"

namespace hase {

cudaError_t opt_in_step384(int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step_kernel<384, 1>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_kernel<384, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

cudaError_t launch_step384(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem,
                           cudaStream_t st) {
    step_kernel<384, 1><<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hase
