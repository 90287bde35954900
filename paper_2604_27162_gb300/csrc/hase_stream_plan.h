// hase_stream_plan.h -- launch-shape helper of the streaming step form
// (stream_kernel), shared by the host API and the kernel.
#pragma once

#include <stdint.h>

namespace hase {

// Warp ids of the streaming form's roles for n_dyn dynamics warps in a CTA
// of n_warps (>= n_dyn + 2): dynamics warp d at bits [4d, 4d + 4), the action
// warp at bits [16, 20); every other warp emits.  spread = 0 puts the
// dynamics on ids 0, 4, 8, 12 (one SM sub-partition: warp w runs on
// sub-partition w mod 4), spread = 1 on ids 0, 4, 1, 5 (two), spread = 2 on
// ids 0, 1, 2, 3 (one each); ids 0, 1, 2, 3 when the CTA is too small.  The
// action warp takes the lowest free id.
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t stream_dyn_ids(int n_dyn, int n_warps, int spread) {
    const uint8_t one[4] = {0, 4, 8, 12}, two[4] = {0, 4, 1, 5};
    uint32_t ids = 0, used = 0;
    for (int d = 0; d < n_dyn; ++d) {
        int id = spread == 2 ? d : (spread ? two[d] : one[d]);
        if (4 * (n_dyn - 1) >= n_warps) id = d;
        ids |= (uint32_t)id << (4 * d);
        used |= 1u << id;
    }
    int act = 0;
    while ((used >> act) & 1u) ++act;
    return ids | ((uint32_t)act << 16);
}

}  // namespace hase
