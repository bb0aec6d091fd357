// Tables of the windowed annealing kernels: one warp per chain (residual in
// shared memory or global memory), the hybrid of both, and groups of 2 or 4
// warps per chain (residual in global memory), for FP32, FP16 and one-byte
// tables (the last with 4 records per lane only).  NT: the kernels that also
// count near-tie decisions.  Each translation unit instantiates one table for
// one NT, so that nvcc compiles them in parallel.
#pragma once
#include "sat_window.cuh"

namespace satpila {

using SweepFn = void (*)(const SatArgs);

inline int kmax_slot(int kmax) { return kmax == 4 ? 0 : kmax == 8 ? 1 : kmax == 32 ? 2 : -1; }
inline int jmax_slot(int jmax) { return jmax == 2 ? 0 : jmax == 4 ? 1 : -1; }

template <bool NT>
SweepFn window_kernel_impl(int rt, bool smem, int jmax, int kmax) {
#define SAT_W(RT, J, K) sat_window_kernel<RT, true, J, K, NT>
#define SAT_WG(RT, J, K) sat_window_kernel<RT, false, J, K, NT>
    const int kk = kmax_slot(kmax), jj = jmax_slot(jmax);
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
#undef SAT_W
#undef SAT_WG
}

template <bool NT>
SweepFn hybrid_kernel_impl(int rt, int jmax, int kmax) {
#define SAT_H(RT, J, K) sat_hybrid_kernel<RT, J, K, NT>
    const int kk = kmax_slot(kmax), jj = jmax_slot(jmax);
    if (kk < 0 || jj < 0 || rt == PILA_U8) return nullptr;
    static const SweepFn t16[2][3] = {{SAT_H(PILA_F16, 2, 4), SAT_H(PILA_F16, 2, 8), SAT_H(PILA_F16, 2, 32)},
                                      {SAT_H(PILA_F16, 4, 4), SAT_H(PILA_F16, 4, 8), SAT_H(PILA_F16, 4, 32)}};
    static const SweepFn t32[2][3] = {{SAT_H(PILA_F32, 2, 4), SAT_H(PILA_F32, 2, 8), SAT_H(PILA_F32, 2, 32)},
                                      {SAT_H(PILA_F32, 4, 4), SAT_H(PILA_F32, 4, 8), SAT_H(PILA_F32, 4, 32)}};
    return rt == PILA_F16 ? t16[jj][kk] : t32[jj][kk];
#undef SAT_H
}

template <bool NT>
SweepFn window_group_kernel_impl(int rt, int jmax, int kmax, int warps_per_chain) {
#define SAT_WGRP(RT, J, K, W) sat_window_group_kernel<RT, J, K, W, NT>
#define SAT_WGRP_K(RT, J, W) {SAT_WGRP(RT, J, 4, W), SAT_WGRP(RT, J, 8, W), SAT_WGRP(RT, J, 32, W)}
    const int kk = kmax_slot(kmax), jj = jmax_slot(jmax);
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
#undef SAT_WGRP_K
#undef SAT_WGRP
}

// The windowed kernel on groups of 2 or 4 warps per chain with the residual
// band in shared memory (FP32 and FP16 tables).
template <bool NT>
SweepFn window_group_smem_kernel_impl(int rt, int jmax, int kmax, int warps_per_chain) {
#define SAT_WGS(RT, J, K, W) sat_window_group_kernel<RT, J, K, W, NT, true>
#define SAT_WGS_K(RT, J, W) {SAT_WGS(RT, J, 4, W), SAT_WGS(RT, J, 8, W), SAT_WGS(RT, J, 32, W)}
    const int kk = kmax_slot(kmax), jj = jmax_slot(jmax);
    const int ww = warps_per_chain == 2 ? 0 : warps_per_chain == 4 ? 1 : -1;
    if (kk < 0 || jj < 0 || ww < 0 || (rt != PILA_F16 && rt != PILA_F32)) return nullptr;
    static const SweepFn t16[2][2][3] = {{SAT_WGS_K(PILA_F16, 2, 2), SAT_WGS_K(PILA_F16, 4, 2)},
                                         {SAT_WGS_K(PILA_F16, 2, 4), SAT_WGS_K(PILA_F16, 4, 4)}};
    static const SweepFn t32[2][2][3] = {{SAT_WGS_K(PILA_F32, 2, 2), SAT_WGS_K(PILA_F32, 4, 2)},
                                         {SAT_WGS_K(PILA_F32, 2, 4), SAT_WGS_K(PILA_F32, 4, 4)}};
    return rt == PILA_F16 ? t16[ww][jj][kk] : t32[ww][jj][kk];
#undef SAT_WGS_K
#undef SAT_WGS
}

}  // namespace satpila
