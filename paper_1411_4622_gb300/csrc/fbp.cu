// Filtered back-projection, for the start image, beta and the spatial
// constraint that Step 1, Step 2 and Fig. 9 take from an FBP
// reconstruction.  The paper does not give its filter; the discrete Ram-Lak
// (ramp) filter for unit bin spacing is used:
//   h(0) = 1/4, h(k) = -1/(pi^2 k^2) for odd k, 0 for even k != 0;
//   q_u(k) = sum_k' p_u(k') h(k - k');
//   f(x, y) = (pi / U) sum_u q_u(x cos theta_u + y sin theta_u),
// q_u linearly interpolated between bin centres (zero outside).
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace satpila {
namespace {

constexpr float kInvPi2 = 0.101321183642337771443f;  // 1 / pi^2

__global__ void ramlak_kernel(const float* sino, long long n_rows, int B, float* out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_rows * B) return;
    const long long row = idx / B;
    const int k = (int)(idx % B);
    const float* p = sino + row * B;
    float acc = 0.25f * p[k];
    // odd offsets d = k - k' only
    for (int kp = (k & 1) ? 0 : 1; kp < B; kp += 2) {
        const float d = (float)(k - kp);
        acc = fmaf(p[kp], -kInvPi2 / (d * d), acc);
    }
    out[idx] = acc;
}

__global__ void backproject_kernel(const float* q, long long n_items, int n, int U, int B, const double* cs,
                                   const double* sn, float* img) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long P = (long long)n * n;
    if (idx >= n_items * P) return;
    const long long item = idx / P;
    const int pix = (int)(idx % P), i = pix / n, j = pix % n;
    const float x = (float)j - 0.5f * (float)(n - 1), y = 0.5f * (float)(n - 1) - (float)i;
    const float* qi = q + item * (long long)U * B;
    float acc = 0.0f;
    for (int u = 0; u < U; ++u) {
        const float pos = fmaf(x, (float)cs[u], fmaf(y, (float)sn[u], 0.5f * (float)(B - 1)));
        const float k0f = floorf(pos);
        const float a = pos - k0f;
        const int k0 = (int)k0f;
        const float* row = qi + (long long)u * B;
        const float v0 = (k0 >= 0 && k0 < B) ? row[k0] : 0.0f;
        const float v1 = (k0 + 1 >= 0 && k0 + 1 < B) ? row[k0 + 1] : 0.0f;
        acc += fmaf(a, v1 - v0, v0);
    }
    img[idx] = acc * (3.14159265358979323846f / (float)U);
}

// Per image: beta = max, the start image clipped to [0, beta] on the
// constrained space, the space itself = pixels above frac * max.
__global__ void prior_kernel(const float* img, int P, float frac, float* init, uint8_t* mask, float* beta) {
    const int item = blockIdx.x;
    const float* f = img + (long long)item * P;
    __shared__ float red[32];
    float m = -INFINITY;
    for (int q = threadIdx.x; q < P; q += blockDim.x) m = fmaxf(m, f[q]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    const float mx = fmaxf(m, 0.0f);
    const float thr = frac * mx;
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
        const bool in = f[q] > thr;
        if (mask) mask[(long long)item * P + q] = in ? 1 : 0;
        if (init) init[(long long)item * P + q] = in ? fminf(fmaxf(f[q], 0.0f), mx) : 0.0f;
    }
    if (beta && threadIdx.x == 0) beta[item] = mx;
}

}  // namespace
}  // namespace satpila

using namespace satpila;

extern "C" int fbp(int32_t n, int32_t n_angles, int32_t n_bins, const double* angles_rad, int32_t n_items,
                   const float* sino, float* images, void* stream) {
    if (n < 1 || n_angles < 1 || n_bins < 1 || n_items < 0 || !sino || !images)
        return fail(SATPILA_ERR_INVALID_ARG, "fbp: bad argument");
    if (!is_device_pointer(sino) || !is_device_pointer(images))
        return fail(SATPILA_ERR_INVALID_ARG, "fbp: sino and images must be device memory");
    if (n_items == 0) return SATPILA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> tab(2 * (size_t)n_angles);
    for (int u = 0; u < n_angles; ++u) {
        const double th = angles_rad ? angles_rad[u] : M_PI * (double)u / (double)n_angles;
        double c = std::cos(th), sn = std::sin(th);
        if (std::fabs(c) < 1e-12) c = 0.0;
        if (std::fabs(sn) < 1e-12) sn = 0.0;
        tab[u] = c;
        tab[n_angles + u] = sn;
    }
    const long long rows = (long long)n_items * n_angles, cells = rows * n_bins;
    void* ws = nullptr;
    SP_CUDA(cudaMalloc(&ws, tab.size() * 8 + (size_t)cells * 4));
    double* d_tab = (double*)ws;
    float* q = (float*)((char*)ws + tab.size() * 8);
    cudaError_t e = cudaMemcpyAsync(d_tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        ramlak_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(sino, rows, n_bins, q);
        e = cudaGetLastError();
    }
    const long long px = (long long)n_items * n * n;
    if (e == cudaSuccess) {
        backproject_kernel<<<(unsigned)((px + 255) / 256), 256, 0, s>>>(q, n_items, n, n_angles, n_bins, d_tab,
                                                                       d_tab + n_angles, images);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ws);
    if (e != cudaSuccess) return cuda_fail(e, "fbp");
    return SATPILA_OK;
}

extern "C" int fbp_prior(int32_t n, int32_t n_items, const float* images, float mask_frac, float* init,
                         uint8_t* mask, float* beta, void* stream) {
    if (n < 1 || n_items < 0 || !images || !(mask_frac >= 0.0f && mask_frac < 1.0f))
        return fail(SATPILA_ERR_INVALID_ARG, "fbp_prior: bad argument");
    for (const void* ptr : {(const void*)images, (const void*)init, (const void*)mask, (const void*)beta})
        if (ptr && !is_device_pointer(ptr)) return fail(SATPILA_ERR_INVALID_ARG, "fbp_prior: buffers must be device memory");
    if (n_items == 0) return SATPILA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    prior_kernel<<<n_items, 256, 0, s>>>(images, n * n, mask_frac, init, mask, beta);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "fbp_prior");
    return SATPILA_OK;
}
