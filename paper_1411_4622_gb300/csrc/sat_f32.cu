// Instantiations of the annealing sweep kernel for F32 PILA records.
#include "sat_sweep.cuh"

namespace satpila {

cudaError_t launch_sweep_f32(bool smem, int jmax, const SatArgs& a, int grid, int warps, size_t smem_bytes,
                               cudaStream_t s) {
    void (*k)(const SatArgs) = nullptr;
    switch (jmax) {
        case 4: k = smem ? sat_sweep_kernel<false, true, 4> : sat_sweep_kernel<false, false, 4>; break;
        case 8: k = smem ? sat_sweep_kernel<false, true, 8> : sat_sweep_kernel<false, false, 8>; break;
        case 12: k = smem ? sat_sweep_kernel<false, true, 12> : sat_sweep_kernel<false, false, 12>; break;
        case 16: k = smem ? sat_sweep_kernel<false, true, 16> : sat_sweep_kernel<false, false, 16>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    k<<<grid, warps * 32, smem_bytes, s>>>(a);
    return cudaGetLastError();
}

int sweep_blocks_per_sm_f32(bool smem, int jmax, int warps, size_t smem_bytes) {
    void (*k)(const SatArgs) = nullptr;
    switch (jmax) {
        case 4: k = smem ? sat_sweep_kernel<false, true, 4> : sat_sweep_kernel<false, false, 4>; break;
        case 8: k = smem ? sat_sweep_kernel<false, true, 8> : sat_sweep_kernel<false, false, 8>; break;
        case 12: k = smem ? sat_sweep_kernel<false, true, 12> : sat_sweep_kernel<false, false, 12>; break;
        case 16: k = smem ? sat_sweep_kernel<false, true, 16> : sat_sweep_kernel<false, false, 16>; break;
        default: return 0;
    }
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem_bytes) != cudaSuccess) return 0;
    return nb;
}

}  // namespace satpila
