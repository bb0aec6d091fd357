// SIRT with PILA, Eqs. (10)-(11) of Sec. III-D:
//   f(i,j) += relax * (1/U) * sum_u (P_m - P_c)(alpha_u, k) / W(u, k) * l_u
// with W(u, k) = sum of l^2 along ray (u, k) over the reconstruction space.
// A pixel crossed by two rays of one angle takes both rays' terms; rays with
// W = 0 contribute nothing; only reconstruction-space pixels change.
//
// SIMULTANEOUS: per pass, the projector writes the correction
//   c(u, k) = (P_m - P_c)(u, k) / W(u, k) for all rays at once; then one warp
//   per pixel gathers c over its PILA row (lanes = angles, coalesced records)
//   and a fixed-order butterfly sum updates the pixel (deterministic).
// SEQUENTIAL: the paper's description: one warp per slice walks the
//   reconstruction space in raster order; each pixel's update is written into
//   the residual through the PILA (Eq. (6)) before the next pixel is read.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace satpila {
namespace {

__global__ void sirt_backproject_kernel(const unsigned char* table, int f16, long long row_records, int U, int B,
                                        const int32_t* list, int n_list, const float* corr, long long corr_stride,
                                        float* img, long long img_stride, float scale) {
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int slice = blockIdx.y;
    if (gw >= n_list) return;
    const int p = list[gw];
    const float* c = corr + (long long)slice * corr_stride;
    float acc = 0.0f;
    for (int u = lane; u < U; u += 32) {
        const long long rec = (long long)p * row_records + u;
        const Entry2 e = decode_rec(table, rec, f16);
        if (e.l0 != 0.0f) acc = fmaf(c[u * B + e.k0], e.l0, acc);
        if (e.l1 != 0.0f) acc = fmaf(c[u * B + e.k1], e.l1, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) img[(long long)slice * img_stride + p] += scale * acc;
}

// One warp per slice; residual r = P_c - P_m in global memory.
__global__ void sirt_sequential_kernel(const unsigned char* table, int f16, long long row_records, int U, int B,
                                       const int32_t* list, int n_list, const float* w, float* resid,
                                       long long resid_stride, float* img, long long img_stride, float scale,
                                       int n_slices) {
    const int lane = threadIdx.x & 31;
    const int slice = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (slice >= n_slices) return;
    float* r = resid + (long long)slice * resid_stride;
    float* f = img + (long long)slice * img_stride;
    for (int q = 0; q < n_list; ++q) {
        const int p = list[q];
        float acc = 0.0f;
        for (int u = lane; u < U; u += 32) {
            const long long rec = (long long)p * row_records + u;
            const Entry2 e = decode_rec(table, rec, f16);
            if (e.l0 != 0.0f) {
                const float wv = w[u * B + e.k0];
                if (wv > 0.0f) acc = fmaf(-r[u * B + e.k0] / wv, e.l0, acc);
            }
            if (e.l1 != 0.0f) {
                const float wv = w[u * B + e.k1];
                if (wv > 0.0f) acc = fmaf(-r[u * B + e.k1] / wv, e.l1, acc);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const float d = scale * acc;
        if (lane == 0) f[p] += d;
        for (int u = lane; u < U; u += 32) {
            const long long rec = (long long)p * row_records + u;
            const Entry2 e = decode_rec(table, rec, f16);
            if (e.l0 != 0.0f) r[u * B + e.k0] = fmaf(d, e.l0, r[u * B + e.k0]);
            if (e.l1 != 0.0f) r[u * B + e.k1] = fmaf(d, e.l1, r[u * B + e.k1]);
        }
        __syncwarp();
    }
}

__global__ void scatter_costs_kernel(const double* src, double* dst, int n_slices, int n_iter, int it) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_slices) dst[(long long)i * n_iter + it] = src[i];
}

}  // namespace
}  // namespace satpila

using namespace satpila;

extern "C" int sirt_run(const satpila_pila* p_const, int32_t n_slices, const float* sino_meas, float* images,
                        const sirt_params* prm, double* costs, void* stream) {
    satpila_pila* p = const_cast<satpila_pila*>(p_const);
    if (!p || !prm || n_slices < 0) return fail(SATPILA_ERR_INVALID_ARG, "sirt_run: bad argument");
    if (prm->n_iter < 0 || (prm->mode != SIRT_SIMULTANEOUS && prm->mode != SIRT_SEQUENTIAL))
        return fail(SATPILA_ERR_INVALID_ARG, "sirt_run: bad n_iter or mode");
    if (n_slices == 0 || prm->n_iter == 0) return SATPILA_OK;
    if (!sino_meas || !images) return fail(SATPILA_ERR_INVALID_ARG, "sirt_run: null data pointer");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_factor(p, s);
    if (rc != SATPILA_OK) return rc;
    const long long P = (long long)p->n * p->n, cells = (long long)p->U * p->B;
    const int n_iter = prm->n_iter;
    if (p->B > projector_max_bins()) return fail(SATPILA_ERR_INVALID_ARG, "sirt_run: too many bins");
    const int G = p->U;  // per-angle partial sums of each slice's cost

    const bool dev_s = is_device_pointer(sino_meas), dev_i = is_device_pointer(images);
    const bool dev_c = costs ? is_device_pointer(costs) : true;
    const float* d_sino = sino_meas;
    float* d_img = images;
    double* d_costs = costs;
    void* ws = nullptr;
    const size_t bytes_sino = dev_s ? 0 : (size_t)n_slices * cells * 4;
    const size_t bytes_img = dev_i ? 0 : (size_t)n_slices * P * 4;
    const size_t bytes_costs = (size_t)n_slices * n_iter * 8;
    const size_t o_sino = 0, o_img = (bytes_sino + 255) / 256 * 256, o_costs = o_img + (bytes_img + 255) / 256 * 256;
    const size_t o_corr = o_costs + (bytes_costs + 255) / 256 * 256;
    const size_t o_psq = o_corr + ((size_t)n_slices * cells * 4 + 255) / 256 * 256;
    const size_t o_cost = o_psq + ((size_t)n_slices * G * 8 + 255) / 256 * 256;
    const size_t o_proj = o_cost + ((size_t)n_slices * 8 + 255) / 256 * 256;
    const bool rays = p->d_ray_off && !projector_forced_pixel();
    const size_t proj_ws = rays ? ray_ws_bytes(n_slices, p->U, p->B, p->n) : projector_ws_bytes(n_slices, p->U, p->B, p->n);
    const size_t total = o_proj + proj_ws;
    SP_CUDA(cudaMalloc(&ws, total));
    char* b = (char*)ws;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess && !dev_s) {
        d_sino = (const float*)(b + o_sino);
        e = cudaMemcpyAsync((void*)d_sino, sino_meas, bytes_sino, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess && !dev_i) {
        d_img = (float*)(b + o_img);
        e = cudaMemcpyAsync(d_img, images, bytes_img, cudaMemcpyHostToDevice, s);
    }
    if (!dev_c) d_costs = (double*)(b + o_costs);
    float* corr = (float*)(b + o_corr);
    double* psq = (double*)(b + o_psq);
    double* cost_now = (double*)(b + o_cost);

    ProjArgs pa{};
    pa.table = p->d_table;
    pa.f16 = p->precision;
    pa.row_records = p->row_records;
    pa.n = p->n;
    pa.U = p->U;
    pa.B = p->B;
    pa.img = d_img;
    pa.img_stride = P;
    pa.pm = d_sino;
    pa.pm_stride = cells;
    pa.resid = corr;
    pa.resid_stride = cells;
    pa.w = p->d_w32;
    pa.part_sq = psq;
    if (rays) use_ray_projector(pa, p, b + o_proj);
    else pa.ws = proj_ws ? b + o_proj : nullptr;
    ReduceArgs ra{};
    ra.n_items = n_slices;
    ra.n_rows = G;
    ra.part_sq = psq;
    ra.inv_cells = 1.0 / (double)cells;
    ra.cost_out = cost_now;
    ra.cost_stride = 1;
    const float scale = prm->relax / (float)p->U;
    auto record_cost = [&](int it) -> cudaError_t {
        cudaError_t err = launch_reduce(ra, s);
        if (err == cudaSuccess && d_costs) {
            scatter_costs_kernel<<<(n_slices + 127) / 128, 128, 0, s>>>(cost_now, d_costs, n_slices, n_iter, it);
            err = cudaGetLastError();
        }
        return err;
    };
    if (prm->mode == SIRT_SIMULTANEOUS) {
        pa.mode = PROJ_SIRT;
        for (int it = 0; it <= n_iter && e == cudaSuccess; ++it) {
            e = launch_projector(pa, n_slices, s);
            if (e == cudaSuccess && it > 0) e = record_cost(it - 1);
            if (e == cudaSuccess && it < n_iter) {
                const long long threads = (long long)p->n_mask * 32;
                dim3 grid((unsigned)((threads + 255) / 256), n_slices);
                if (p->n_mask > 0)
                    sirt_backproject_kernel<<<grid, 256, 0, s>>>(p->d_table, pa.f16, p->row_records, p->U, p->B,
                                                                 p->d_list, p->n_mask, corr, cells, d_img, P, scale);
                e = cudaGetLastError();
            }
        }
    } else {
        pa.mode = PROJ_RESYNC;  // corr buffer holds the residual P_c - P_m
        pa.drift = 0;
        e = launch_projector(pa, n_slices, s);
        for (int it = 0; it < n_iter && e == cudaSuccess; ++it) {
            const int threads = n_slices * 32;
            sirt_sequential_kernel<<<(threads + 127) / 128, 128, 0, s>>>(p->d_table, pa.f16, p->row_records, p->U,
                                                                         p->B, p->d_list, p->n_mask, p->d_w32, corr,
                                                                         cells, d_img, P, scale, n_slices);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = launch_projector(pa, n_slices, s);  // fresh residual and cost
            if (e == cudaSuccess) e = record_cost(it);
        }
    }
    if (e == cudaSuccess && !dev_i) e = cudaMemcpyAsync(images, d_img, bytes_img, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && costs && !dev_c) e = cudaMemcpyAsync(costs, d_costs, bytes_costs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ws);
    if (e != cudaSuccess) return cuda_fail(e, "sirt_run");
    return SATPILA_OK;
}

// ---- SIRT without any allocation -------------------------------------------
//
// For callers that must not allocate device memory during the call:
// processes that run inside a fixed memory budget handed to them at
// start-up, hosts whose own allocator has reserved all device memory, and
// loops that cannot take the device-wide synchronisation an allocation or
// release may cause.  The scratch that sirt_run allocates per call lives instead
// in one statically sized device array of this library, which every GPU that
// loads the library keeps for the life of the process.

namespace satpila {
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[SATPILA_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[64] = {};

// Device address of the static scratch on the current device.  The array's
// name on the host is only a stand-in for the symbol, so the address comes
// from the runtime, once per device (on that device's first call).
int noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "sirt_run_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(SATPILA_ERR_INVALID_ARG, "sirt_run_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "sirt_run_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SATPILA_OK;
}

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace satpila

extern "C" int sirt_run_noalloc(const satpila_pila* p, int32_t n_slices, const float* sino_meas, float* images,
                                const sirt_params* prm, double* costs, void* stream) {
    if (!p || !prm || n_slices < 0) return fail(SATPILA_ERR_INVALID_ARG, "sirt_run_noalloc: bad argument");
    if (prm->n_iter < 0 || (prm->mode != SIRT_SIMULTANEOUS && prm->mode != SIRT_SEQUENTIAL))
        return fail(SATPILA_ERR_INVALID_ARG, "sirt_run_noalloc: bad n_iter or mode");
    if (n_slices == 0 || prm->n_iter == 0) return SATPILA_OK;
    if (!sino_meas || !images) return fail(SATPILA_ERR_INVALID_ARG, "sirt_run_noalloc: null data pointer");
    if (!is_device_pointer(sino_meas) || !is_device_pointer(images) || (costs && !is_device_pointer(costs)))
        return fail(SATPILA_ERR_INVALID_ARG, "sirt_run_noalloc: data must be in device memory");
    cudaStream_t s = (cudaStream_t)stream;
    const long long P = (long long)p->n * p->n, cells = (long long)p->U * p->B;
    const int n_iter = prm->n_iter;
    if (p->B > projector_max_bins()) return fail(SATPILA_ERR_INVALID_ARG, "sirt_run_noalloc: too many bins");
    const int G = p->U;  // per-angle partial sums of each slice's cost
    // Scratch layout: correction or residual, partial sums, costs, and the
    // factor matrix when the table has not cached one.
    const bool own_w = p->d_w32 == nullptr;
    const size_t o_corr = 0;
    const size_t o_psq = o_corr + round256((size_t)n_slices * cells * 4);
    const size_t o_cost = o_psq + round256((size_t)n_slices * G * 8);
    const size_t o_w64 = o_cost + round256((size_t)n_slices * 8);
    const size_t o_w32 = o_w64 + (own_w ? round256((size_t)cells * 8) : 0);
    const size_t o_proj = o_w32 + (own_w ? round256((size_t)cells * 4) : 0);
    size_t total = o_proj;
    if (total > (size_t)SATPILA_NOALLOC_SCRATCH_BYTES)
        return fail(SATPILA_ERR_INVALID_ARG, "sirt_run_noalloc: the problem needs " + std::to_string(total) +
                                                 " bytes of scratch, more than the static " +
                                                 std::to_string((size_t)SATPILA_NOALLOC_SCRATCH_BYTES));
    // the projector's workspace (pixel chunks for few slices) when it fits
    const size_t proj_ws = projector_ws_bytes(n_slices, p->U, p->B, p->n);
    const bool chunk_ws = proj_ws > 0 && total + proj_ws <= (size_t)SATPILA_NOALLOC_SCRATCH_BYTES;
    if (chunk_ws) total += proj_ws;
    void* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc != SATPILA_OK) return rc;
    char* b = (char*)base;
    float* corr = (float*)(b + o_corr);
    double* psq = (double*)(b + o_psq);
    double* cost_now = (double*)(b + o_cost);
    // The array keeps the previous call's contents: start from zero.
    cudaError_t e = cudaMemsetAsync(base, 0, total, s);

    ProjArgs pa{};
    pa.table = p->d_table;
    pa.f16 = p->precision;
    pa.row_records = p->row_records;
    pa.n = p->n;
    pa.U = p->U;
    pa.B = p->B;
    pa.ws = chunk_ws ? b + o_proj : nullptr;
    const float* w32 = p->d_w32;
    if (e == cudaSuccess && own_w) {
        ProjArgs fa = pa;
        fa.mode = PROJ_FACTOR;
        fa.mask = p->d_mask;
        fa.out64 = (double*)(b + o_w64);
        fa.out32 = (float*)(b + o_w32);
        e = launch_projector(fa, 1, s);
        w32 = fa.out32;
    }
    pa.img = images;
    pa.img_stride = P;
    pa.pm = sino_meas;
    pa.pm_stride = cells;
    pa.resid = corr;
    pa.resid_stride = cells;
    pa.w = w32;
    pa.part_sq = psq;
    ReduceArgs ra{};
    ra.n_items = n_slices;
    ra.n_rows = G;
    ra.part_sq = psq;
    ra.inv_cells = 1.0 / (double)cells;
    ra.cost_out = cost_now;
    ra.cost_stride = 1;
    const float scale = prm->relax / (float)p->U;
    auto record_cost = [&](int it) -> cudaError_t {
        cudaError_t err = launch_reduce(ra, s);
        if (err == cudaSuccess && costs) {
            scatter_costs_kernel<<<(n_slices + 127) / 128, 128, 0, s>>>(cost_now, costs, n_slices, n_iter, it);
            err = cudaGetLastError();
        }
        return err;
    };
    if (prm->mode == SIRT_SIMULTANEOUS) {
        pa.mode = PROJ_SIRT;
        for (int it = 0; it <= n_iter && e == cudaSuccess; ++it) {
            e = launch_projector(pa, n_slices, s);
            if (e == cudaSuccess && it > 0) e = record_cost(it - 1);
            if (e == cudaSuccess && it < n_iter && p->n_mask > 0) {
                const long long threads = (long long)p->n_mask * 32;
                dim3 grid((unsigned)((threads + 255) / 256), n_slices);
                sirt_backproject_kernel<<<grid, 256, 0, s>>>(p->d_table, pa.f16, p->row_records, p->U, p->B,
                                                             p->d_list, p->n_mask, corr, cells, images, P, scale);
                e = cudaGetLastError();
            }
        }
    } else {
        pa.mode = PROJ_RESYNC;
        pa.drift = 0;
        e = e == cudaSuccess ? launch_projector(pa, n_slices, s) : e;
        for (int it = 0; it < n_iter && e == cudaSuccess; ++it) {
            const int threads = n_slices * 32;
            sirt_sequential_kernel<<<(threads + 127) / 128, 128, 0, s>>>(p->d_table, pa.f16, p->row_records, p->U,
                                                                         p->B, p->d_list, p->n_mask, w32, corr, cells,
                                                                         images, P, scale, n_slices);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = launch_projector(pa, n_slices, s);
            if (e == cudaSuccess) e = record_cost(it);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "sirt_run_noalloc");
    return SATPILA_OK;
}
