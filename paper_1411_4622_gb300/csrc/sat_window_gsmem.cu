// The windowed kernel on groups of 2 or 4 warps per chain with the residual
// band in shared memory, without the near-tie count.
#include "sat_window_inst.cuh"

namespace satpila {

SweepFn window_group_smem_kernel(int rt, int jmax, int kmax, int warps_per_chain) {
    return window_group_smem_kernel_impl<false>(rt, jmax, kmax, warps_per_chain);
}

}  // namespace satpila
