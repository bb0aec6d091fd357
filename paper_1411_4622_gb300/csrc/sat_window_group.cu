// The windowed kernel on groups of 2 or 4 warps per chain, without the
// near-tie count.
#include "sat_window_inst.cuh"

namespace satpila {

SweepFn window_group_kernel(int rt, int jmax, int kmax, int warps_per_chain) {
    return window_group_kernel_impl<false>(rt, jmax, kmax, warps_per_chain);
}

}  // namespace satpila
