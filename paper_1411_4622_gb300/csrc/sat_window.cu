// The windowed kernels (one warp per chain, and the hybrid) without the
// near-tie count.
#include "sat_window_inst.cuh"

namespace satpila {

SweepFn window_kernel(int rt, bool smem, int jmax, int kmax) { return window_kernel_impl<false>(rt, smem, jmax, kmax); }
SweepFn hybrid_kernel(int rt, int jmax, int kmax) { return hybrid_kernel_impl<false>(rt, jmax, kmax); }

}  // namespace satpila
