// The windowed kernel on groups of 2 or 4 warps per chain with the residual
// band in shared memory, counting near-tie decisions (SAT_FLAG_NEAR_TIES).
#include "sat_window_inst.cuh"

namespace satpila {

SweepFn window_group_smem_kernel_nt(int rt, int jmax, int kmax, int warps_per_chain) {
    return window_group_smem_kernel_impl<true>(rt, jmax, kmax, warps_per_chain);
}

}  // namespace satpila
