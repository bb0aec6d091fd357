// The windowed kernels (one warp per chain, and the hybrid) that also count
// near-tie decisions (SAT_FLAG_NEAR_TIES).
#include "sat_window_inst.cuh"

namespace satpila {

SweepFn window_kernel_nt(int rt, bool smem, int jmax, int kmax) {
    return window_kernel_impl<true>(rt, smem, jmax, kmax);
}
SweepFn hybrid_kernel_nt(int rt, int jmax, int kmax) { return hybrid_kernel_impl<true>(rt, jmax, kmax); }

}  // namespace satpila
