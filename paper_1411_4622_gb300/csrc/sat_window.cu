// Instantiations of the windowed annealing kernel (one warp per chain,
// residual in shared memory).
#include "sat_window.cuh"

namespace satpila {

using SweepFn = void (*)(const SatArgs);

#define SAT_W(F16, J, K) sat_window_kernel<F16, true, J, K>
#define SAT_WG(F16, J, K) sat_window_kernel<F16, false, J, K>

SweepFn window_kernel(bool f16, bool smem, int jmax, int kmax) {
    const int kk = kmax == 4 ? 0 : kmax == 8 ? 1 : kmax == 32 ? 2 : -1;
    const int jj = jmax == 2 ? 0 : jmax == 4 ? 1 : -1;
    if (kk < 0 || jj < 0) return nullptr;
    if (!smem) {
        static const SweepFn g16[2][3] = {{SAT_WG(true, 2, 4), SAT_WG(true, 2, 8), SAT_WG(true, 2, 32)},
                                          {SAT_WG(true, 4, 4), SAT_WG(true, 4, 8), SAT_WG(true, 4, 32)}};
        static const SweepFn g32[2][3] = {{SAT_WG(false, 2, 4), SAT_WG(false, 2, 8), SAT_WG(false, 2, 32)},
                                          {SAT_WG(false, 4, 4), SAT_WG(false, 4, 8), SAT_WG(false, 4, 32)}};
        return f16 ? g16[jj][kk] : g32[jj][kk];
    }
    static const SweepFn t16[2][3] = {{SAT_W(true, 2, 4), SAT_W(true, 2, 8), SAT_W(true, 2, 32)},
                                      {SAT_W(true, 4, 4), SAT_W(true, 4, 8), SAT_W(true, 4, 32)}};
    static const SweepFn t32[2][3] = {{SAT_W(false, 2, 4), SAT_W(false, 2, 8), SAT_W(false, 2, 32)},
                                      {SAT_W(false, 4, 4), SAT_W(false, 4, 8), SAT_W(false, 4, 32)}};
    return f16 ? t16[jj][kk] : t32[jj][kk];
}

#define SAT_H(F16, J, K) sat_hybrid_kernel<F16, J, K>

SweepFn hybrid_kernel(bool f16, int jmax, int kmax) {
    const int kk = kmax == 4 ? 0 : kmax == 8 ? 1 : kmax == 32 ? 2 : -1;
    const int jj = jmax == 2 ? 0 : jmax == 4 ? 1 : -1;
    if (kk < 0 || jj < 0) return nullptr;
    static const SweepFn t16[2][3] = {{SAT_H(true, 2, 4), SAT_H(true, 2, 8), SAT_H(true, 2, 32)},
                                      {SAT_H(true, 4, 4), SAT_H(true, 4, 8), SAT_H(true, 4, 32)}};
    static const SweepFn t32[2][3] = {{SAT_H(false, 2, 4), SAT_H(false, 2, 8), SAT_H(false, 2, 32)},
                                      {SAT_H(false, 4, 4), SAT_H(false, 4, 8), SAT_H(false, 4, 32)}};
    return f16 ? t16[jj][kk] : t32[jj][kk];
}

}  // namespace satpila
