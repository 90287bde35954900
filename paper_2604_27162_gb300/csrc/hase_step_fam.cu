// hase_step_fam.cu -- one kernel family of the fused step, compiled once per
// family with -DHASE_FAM=<0..16> (the families are compiled in parallel):
//
//   family 0       the general emission (one lane per agent), CTAs of up to
//                  512 threads (128 registers);
//   families 1-16  the one-thread emission: 1-4, 5-8, 9-12 and 13-16 agents
//                  with one word a plane (1-4), two words a plane (5-8), line
//                  of sight with one word (9-12) and two words (13-16); CTAs
//                  of up to 384 threads (168 registers).
//
// Families 1-8 also have the streaming form (stream_kernel, hase_stream.cuh),
// used when no centralized observation or fog of war is exported.
#include "hase_step.cuh"
#include "hase_stream.cuh"

#ifndef HASE_FAM
#error "compile with -DHASE_FAM=<family>"
#endif

namespace hase {

#define HASE_CAT2(a, b) a##b
#define HASE_CAT(a, b) HASE_CAT2(a, b)

constexpr int kFam = HASE_FAM;
constexpr int kFamThreads = kFam == 0 ? 512 : 384;
#define HASE_FAM_STREAM (HASE_FAM >= 1 && HASE_FAM <= 8)

template <typename K>
static cudaError_t opt_in_kernel(K kernel, int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// All the dynamic shared memory a block may have beside the kernel's static share.
cudaError_t HASE_CAT(opt_in_f, HASE_FAM)(int optin) {
    cudaError_t e = opt_in_kernel(step_kernel<kFamThreads, 1, kFam>, optin);
#if HASE_FAM_STREAM
    if (e == cudaSuccess) e = opt_in_kernel(stream_kernel<384, kFam>, optin);
#endif
    return e;
}

cudaError_t HASE_CAT(launch_f, HASE_FAM)(const StepParams& p, uint32_t n_groups, uint32_t threads, uint32_t smem,
                                        cudaStream_t st) {
    if (threads > (uint32_t)kFamThreads) return cudaErrorInvalidConfiguration;
    step_kernel<kFamThreads, 1, kFam><<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t HASE_CAT(launch_stream_f, HASE_FAM)(const StepParams& p, uint32_t n_groups, uint32_t threads,
                                               uint32_t smem, cudaStream_t st) {
#if HASE_FAM_STREAM
    if (threads > 384u) return cudaErrorInvalidConfiguration;
    stream_kernel<384, kFam><<<n_groups, threads, smem, st>>>(p);
    return cudaGetLastError();
#else
    (void)p;
    (void)n_groups;
    (void)threads;
    (void)smem;
    (void)st;
    return cudaErrorInvalidValue;
#endif
}

}  // namespace hase
