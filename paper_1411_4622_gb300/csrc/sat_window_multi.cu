// The windowed kernel on groups of 4 warps per chain over chains of several
// tables in one launch (the serving engine's classes of one image size):
// up to 512 angles (four records per lane), up to 8 estimates, residual in
// global memory.
#include "sat_window_inst.cuh"

namespace satpila {

SweepFn window_multi_kernel(int rt) {
    switch (rt) {
        case PILA_F32: return sat_window_group_kernel<PILA_F32, 4, 8, 4, false, false, true>;
        case PILA_F16: return sat_window_group_kernel<PILA_F16, 4, 8, 4, false, false, true>;
        case PILA_U8: return sat_window_group_kernel<PILA_U8, 4, 8, 4, false, false, true>;
        default: return nullptr;
    }
}

}  // namespace satpila
