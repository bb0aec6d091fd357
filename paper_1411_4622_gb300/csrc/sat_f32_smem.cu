// Instantiations of the annealing sweep kernel: F32 records, residual in smem.
#include "sat_sweep.cuh"

namespace satpila {

#define SAT_K(J, K) sat_sweep_kernel<false, true, J, K>
using SweepFn = void (*)(const SatArgs);

SweepFn sweep_kernel_f32_smem(int jmax, int kmax) {
    const int kk = kmax == 4 ? 0 : kmax == 8 ? 1 : kmax == 32 ? 2 : -1;
    static const SweepFn table[4][3] = {{SAT_K(2, 4), SAT_K(2, 8), SAT_K(2, 32)},
                                        {SAT_K(4, 4), SAT_K(4, 8), SAT_K(4, 32)},
                                        {SAT_K(8, 4), SAT_K(8, 8), SAT_K(8, 32)},
                                        {SAT_K(16, 4), SAT_K(16, 8), SAT_K(16, 32)}};
    const int jj = jmax == 2 ? 0 : jmax == 4 ? 1 : jmax == 8 ? 2 : jmax == 16 ? 3 : -1;
    if (jj < 0 || kk < 0) return nullptr;
    return table[jj][kk];
}

}  // namespace satpila
