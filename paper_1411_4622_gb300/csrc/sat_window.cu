// Instantiations of the windowed annealing kernel (one warp per chain,
// residual in shared memory or global memory) for FP32, FP16 and one-byte
// tables (the last with 4 records per lane only).
#include "sat_window.cuh"

namespace satpila {

using SweepFn = void (*)(const SatArgs);

#define SAT_W(RT, J, K) sat_window_kernel<RT, true, J, K>
#define SAT_WG(RT, J, K) sat_window_kernel<RT, false, J, K>

SweepFn window_kernel(int rt, bool smem, int jmax, int kmax) {
    const int kk = kmax == 4 ? 0 : kmax == 8 ? 1 : kmax == 32 ? 2 : -1;
    const int jj = jmax == 2 ? 0 : jmax == 4 ? 1 : -1;
    if (kk < 0 || jj < 0) return nullptr;
    if (rt == PILA_U8) {
        if (jmax != 4) return nullptr;
        static const SweepFn u8[2][3] = {{SAT_WG(PILA_U8, 4, 4), SAT_WG(PILA_U8, 4, 8), SAT_WG(PILA_U8, 4, 32)},
                                         {SAT_W(PILA_U8, 4, 4), SAT_W(PILA_U8, 4, 8), SAT_W(PILA_U8, 4, 32)}};
        return u8[smem ? 1 : 0][kk];
    }
    const bool f16 = rt == PILA_F16;
    if (!smem) {
        static const SweepFn g16[2][3] = {{SAT_WG(PILA_F16, 2, 4), SAT_WG(PILA_F16, 2, 8), SAT_WG(PILA_F16, 2, 32)},
                                          {SAT_WG(PILA_F16, 4, 4), SAT_WG(PILA_F16, 4, 8), SAT_WG(PILA_F16, 4, 32)}};
        static const SweepFn g32[2][3] = {{SAT_WG(PILA_F32, 2, 4), SAT_WG(PILA_F32, 2, 8), SAT_WG(PILA_F32, 2, 32)},
                                          {SAT_WG(PILA_F32, 4, 4), SAT_WG(PILA_F32, 4, 8), SAT_WG(PILA_F32, 4, 32)}};
        return f16 ? g16[jj][kk] : g32[jj][kk];
    }
    static const SweepFn t16[2][3] = {{SAT_W(PILA_F16, 2, 4), SAT_W(PILA_F16, 2, 8), SAT_W(PILA_F16, 2, 32)},
                                      {SAT_W(PILA_F16, 4, 4), SAT_W(PILA_F16, 4, 8), SAT_W(PILA_F16, 4, 32)}};
    static const SweepFn t32[2][3] = {{SAT_W(PILA_F32, 2, 4), SAT_W(PILA_F32, 2, 8), SAT_W(PILA_F32, 2, 32)},
                                      {SAT_W(PILA_F32, 4, 4), SAT_W(PILA_F32, 4, 8), SAT_W(PILA_F32, 4, 32)}};
    return f16 ? t16[jj][kk] : t32[jj][kk];
}

#define SAT_H(RT, J, K) sat_hybrid_kernel<RT, J, K>

SweepFn hybrid_kernel(int rt, int jmax, int kmax) {
    const int kk = kmax == 4 ? 0 : kmax == 8 ? 1 : kmax == 32 ? 2 : -1;
    const int jj = jmax == 2 ? 0 : jmax == 4 ? 1 : -1;
    if (kk < 0 || jj < 0 || rt == PILA_U8) return nullptr;
    static const SweepFn t16[2][3] = {{SAT_H(PILA_F16, 2, 4), SAT_H(PILA_F16, 2, 8), SAT_H(PILA_F16, 2, 32)},
                                      {SAT_H(PILA_F16, 4, 4), SAT_H(PILA_F16, 4, 8), SAT_H(PILA_F16, 4, 32)}};
    static const SweepFn t32[2][3] = {{SAT_H(PILA_F32, 2, 4), SAT_H(PILA_F32, 2, 8), SAT_H(PILA_F32, 2, 32)},
                                      {SAT_H(PILA_F32, 4, 4), SAT_H(PILA_F32, 4, 8), SAT_H(PILA_F32, 4, 32)}};
    return rt == PILA_F16 ? t16[jj][kk] : t32[jj][kk];
}

}  // namespace satpila
