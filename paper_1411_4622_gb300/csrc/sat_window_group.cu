// Instantiations of the windowed annealing kernel for chains on groups of 2
// or 4 warps (residual in global memory), for FP32, FP16 and one-byte tables.
#include "sat_window.cuh"

namespace satpila {

using SweepFn = void (*)(const SatArgs);

#define SAT_WGRP(RT, J, K, W) sat_window_group_kernel<RT, J, K, W>
#define SAT_WGRP_K(RT, J, W) {SAT_WGRP(RT, J, 4, W), SAT_WGRP(RT, J, 8, W), SAT_WGRP(RT, J, 32, W)}

SweepFn window_group_kernel(int rt, int jmax, int kmax, int warps_per_chain) {
    const int kk = kmax == 4 ? 0 : kmax == 8 ? 1 : kmax == 32 ? 2 : -1;
    const int jj = jmax == 2 ? 0 : jmax == 4 ? 1 : -1;
    const int ww = warps_per_chain == 2 ? 0 : warps_per_chain == 4 ? 1 : -1;
    if (kk < 0 || jj < 0 || ww < 0) return nullptr;
    if (rt == PILA_U8) {  // four records per 16-byte chunk: always 4 per lane
        if (jmax != 4) return nullptr;
        static const SweepFn u8[2][3] = {SAT_WGRP_K(PILA_U8, 4, 2), SAT_WGRP_K(PILA_U8, 4, 4)};
        return u8[ww][kk];
    }
    if (rt != PILA_F16 && rt != PILA_F32) return nullptr;
    static const SweepFn t16[2][2][3] = {{SAT_WGRP_K(PILA_F16, 2, 2), SAT_WGRP_K(PILA_F16, 4, 2)},
                                         {SAT_WGRP_K(PILA_F16, 2, 4), SAT_WGRP_K(PILA_F16, 4, 4)}};
    static const SweepFn t32[2][2][3] = {{SAT_WGRP_K(PILA_F32, 2, 2), SAT_WGRP_K(PILA_F32, 4, 2)},
                                         {SAT_WGRP_K(PILA_F32, 2, 4), SAT_WGRP_K(PILA_F32, 4, 4)}};
    return rt == PILA_F16 ? t16[ww][jj][kk] : t32[ww][jj][kk];
}

}  // namespace satpila
