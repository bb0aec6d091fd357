// Forward projection through the PILA (the DRT of Eq. (1) with the stored
// lengths), used for: the FP64 residual resync and final cost of the
// annealer (Eq. (4)), the public pila_forward call, the SIRT factor matrix
// (Sec. III-D, lengths squared over the reconstruction space) and the SIRT
// correction of Eq. (11).
//
// Design: one CTA per (image, group of angles) holds a shared-memory
// accumulator for its [angles][bins] block.  Warps walk the pixels, lanes the
// angles of a pixel's PILA row (coalesced record loads), and every product
// f * l is added as an exact 64-bit fixed-point integer (integer units; the
// FP64 units of this part are scarce).  Integer addition is associative, so
// the result does not depend on the order of the shared-memory atomics:
// the projection is deterministic and at least as accurate as an FP64 sum.
// The fraction bits are chosen per image from max|f| so nothing overflows.
#include <cmath>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace satpila {
namespace {

constexpr int kProjThreads = 512;
constexpr int kProjSmemBudget = 200 * 1024;

__device__ double block_sum_fixed_order(double v, double* red) {
    const int tid = threadIdx.x;
    red[tid] = v;
    __syncthreads();
    for (int w = kProjThreads / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__device__ float block_max(float v, float* red) {
    const int tid = threadIdx.x;
    red[tid] = v;
    __syncthreads();
    for (int w = kProjThreads / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] = fmaxf(red[tid], red[tid + w]);
        __syncthreads();
    }
    const float r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kProjThreads) projector_kernel(ProjArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    long long* acc = reinterpret_cast<long long*>(smem_raw);
    __shared__ double red_d[kProjThreads];
    __shared__ float red_f[kProjThreads];

    const int item = blockIdx.y, grp = blockIdx.x;
    const int u0 = grp * a.angles_per_group;
    const int A = min(a.angles_per_group, a.U - u0);
    const int B = a.B;
    const long long P = (long long)a.n * a.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* img = a.img ? a.img + (long long)item * a.img_stride : nullptr;

    for (int e = tid; e < A * B; e += kProjThreads) acc[e] = 0;

    // Fraction bits from a bound on |P| (every ray is at most sqrt(2)*n + 2 long).
    double bound;
    if (a.mode == PROJ_FACTOR) {
        bound = 2.0 * (1.4142135623730951 * a.n + 2.0);
    } else {
        float m = 0.0f;
        for (long long q = tid; q < P; q += kProjThreads) m = fmaxf(m, fabsf(img[q]));
        m = block_max(m, red_f);
        bound = 1.5 * (double)m * (1.4142135623730951 * a.n + 2.0);
    }
    const int F = fixed_point_bits(bound);
    __syncthreads();

    const int nwarps = kProjThreads / 32;
    for (long long q = warp; q < P; q += nwarps) {
        float f;
        if (a.mode == PROJ_FACTOR) f = a.mask[q] ? 1.0f : 0.0f;
        else f = img[q];
        if (f == 0.0f) continue;
        const long long row = q * a.row_records;
        for (int ul = lane; ul < A; ul += 32) {
            const long long rec = row + u0 + ul;
            const Entry2 e = decode_rec(a.table, rec, a.f16);
            if (e.l0 != 0.0f) {
                const long long t = a.mode == PROJ_FACTOR ? fixed_product(e.l0, e.l0, F) : fixed_product(f, e.l0, F);
                atomicAdd(reinterpret_cast<unsigned long long*>(&acc[ul * B + e.k0]), (unsigned long long)t);
            }
            if (e.l1 != 0.0f) {
                const long long t = a.mode == PROJ_FACTOR ? fixed_product(e.l1, e.l1, F) : fixed_product(f, e.l1, F);
                atomicAdd(reinterpret_cast<unsigned long long*>(&acc[ul * B + e.k1]), (unsigned long long)t);
            }
        }
    }
    __syncthreads();

    double sq = 0.0;
    float drift = 0.0f;
    for (int e = tid; e < A * B; e += kProjThreads) {
        const int ul = e / B, k = e - ul * B;
        const long long cell = (long long)(u0 + ul) * B + k;
        const double val = ldexp((double)acc[e], -F);
        switch (a.mode) {
            case PROJ_FORWARD:
                a.out64[(long long)item * a.out_stride + cell] = val;
                break;
            case PROJ_FACTOR:
                a.out64[cell] = val;
                a.out32[cell] = (float)val;
                break;
            case PROJ_RESYNC: {
                const double r = val - (double)a.pm[(long long)item * a.pm_stride + cell];
                const float rf = (float)r;
                const int pitch = a.resid_pitch > 0 ? a.resid_pitch : B;
                float* dst = a.resid + (long long)item * a.resid_stride + (long long)(u0 + ul) * pitch + k;
                if (a.drift) drift = fmaxf(drift, fabsf(rf - *dst));
                *dst = rf;
                sq += r * r;
                break;
            }
            case PROJ_SIRT: {
                const double r = val - (double)a.pm[(long long)item * a.pm_stride + cell];
                const float w = a.w[cell];
                a.resid[(long long)item * a.resid_stride + cell] = w > 0.0f ? (float)(-r / (double)w) : 0.0f;
                sq += r * r;
                break;
            }
        }
    }
    if (a.part_sq) {
        const double s = block_sum_fixed_order(sq, red_d);
        if (tid == 0) a.part_sq[(long long)item * a.n_groups + grp] = s;
    }
    if (a.part_drift) {
        const float d = block_max(drift, red_f);
        if (tid == 0) a.part_drift[(long long)item * a.n_groups + grp] = d;
    }
}

__global__ void reduce_kernel(ReduceArgs a) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= a.n_items) return;
    double s = 0.0;
    float d = 0.0f;
    for (int g = 0; g < a.n_groups; ++g) {
        s += a.part_sq[(long long)item * a.n_groups + g];
        if (a.part_drift) d = fmaxf(d, a.part_drift[(long long)item * a.n_groups + g]);
    }
    if (a.S_out) a.S_out[item] = s;
    if (a.cost_out) a.cost_out[(long long)item * a.cost_stride] = sqrt(s * a.inv_cells);
    if (a.drift_max && a.part_drift) a.drift_max[item] = fmax(a.drift_max[item], (double)d);
}

}  // namespace

int projector_smem_bytes(int angles_per_group, int B) { return angles_per_group * B * (int)sizeof(long long); }

int projector_plan(int U, int B, int* angles_per_group, int* n_groups) {
    int A = kProjSmemBudget / (B * (int)sizeof(long long));
    if (A < 1) return SATPILA_ERR_INVALID_ARG;
    if (A > U) A = U;
    // balance the groups
    const int G = (U + A - 1) / A;
    A = (U + G - 1) / G;
    *angles_per_group = A;
    *n_groups = G;
    return SATPILA_OK;
}

// The projector's shared-memory limit, set once per device (before any
// stream capture that launches it).
cudaError_t prepare_projector() {
    static std::mutex mu;
    static uint64_t done = 0;  // bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && (done >> dev) & 1u) return cudaSuccess;
    e = cudaFuncSetAttribute(projector_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kProjSmemBudget);
    if (e == cudaSuccess && dev < 64) done |= 1ull << dev;
    return e;
}

cudaError_t launch_projector(const ProjArgs& a, int n_items, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const int smem = projector_smem_bytes(a.angles_per_group, a.B);
    cudaError_t e = prepare_projector();
    if (e != cudaSuccess) return e;
    dim3 grid(a.n_groups, n_items);
    projector_kernel<<<grid, kProjThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t s) {
    if (a.n_items <= 0) return cudaSuccess;
    reduce_kernel<<<(a.n_items + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

// Builds the SIRT factor matrix of a PILA on first use.
int ensure_factor(satpila_pila* p, cudaStream_t s) {
    if (p->d_w64) return SATPILA_OK;
    const size_t cells = (size_t)p->U * p->B;
    SP_CUDA(cudaMalloc(&p->d_w64, cells * sizeof(double)));
    SP_CUDA(cudaMalloc(&p->d_w32, cells * sizeof(float)));
    ProjArgs a{};
    a.table = p->d_table;
    a.f16 = p->precision;
    a.row_records = p->row_records;
    a.n = p->n;
    a.U = p->U;
    a.B = p->B;
    if (projector_plan(p->U, p->B, &a.angles_per_group, &a.n_groups) != SATPILA_OK)
        return fail(SATPILA_ERR_INVALID_ARG, "too many bins for the projector");
    a.mode = PROJ_FACTOR;
    a.mask = p->d_mask;
    a.out64 = p->d_w64;
    a.out32 = p->d_w32;
    SP_CUDA(launch_projector(a, 1, s));
    return SATPILA_OK;
}

}  // namespace satpila

using namespace satpila;

extern "C" int pila_forward(const satpila_pila* p, int32_t n_images, const float* images, double* sino,
                            void* stream) {
    if (!p || n_images < 0 || (n_images > 0 && (!images || !sino)))
        return fail(SATPILA_ERR_INVALID_ARG, "pila_forward: bad argument");
    if (n_images == 0) return SATPILA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const long long P = (long long)p->n * p->n, cells = (long long)p->U * p->B;
    const bool dev_i = is_device_pointer(images), dev_o = is_device_pointer(sino);
    const float* di = images;
    double* dout = sino;
    float* tmp_i = nullptr;
    double* tmp_o = nullptr;
    if (!dev_i) {
        SP_CUDA(cudaMalloc(&tmp_i, (size_t)n_images * P * sizeof(float)));
        SP_CUDA(cudaMemcpyAsync(tmp_i, images, (size_t)n_images * P * sizeof(float), cudaMemcpyHostToDevice, s));
        di = tmp_i;
    }
    if (!dev_o) {
        SP_CUDA(cudaMalloc(&tmp_o, (size_t)n_images * cells * sizeof(double)));
        dout = tmp_o;
    }
    ProjArgs a{};
    a.table = p->d_table;
    a.f16 = p->precision;
    a.row_records = p->row_records;
    a.n = p->n;
    a.U = p->U;
    a.B = p->B;
    if (projector_plan(p->U, p->B, &a.angles_per_group, &a.n_groups) != SATPILA_OK)
        return fail(SATPILA_ERR_INVALID_ARG, "pila_forward: too many bins");
    a.mode = PROJ_FORWARD;
    a.img = di;
    a.img_stride = P;
    a.out64 = dout;
    a.out_stride = cells;
    cudaError_t e = launch_projector(a, n_images, s);
    if (e == cudaSuccess && !dev_o)
        e = cudaMemcpyAsync(sino, dout, (size_t)n_images * cells * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && (!dev_i || !dev_o)) e = cudaStreamSynchronize(s);
    if (tmp_i) cudaFree(tmp_i);
    if (tmp_o) cudaFree(tmp_o);
    if (e != cudaSuccess) return cuda_fail(e, "pila_forward");
    return SATPILA_OK;
}

extern "C" int pila_sirt_factor(const satpila_pila* p, double* w, void* stream) {
    if (!p || !w) return fail(SATPILA_ERR_INVALID_ARG, "pila_sirt_factor: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_factor(const_cast<satpila_pila*>(p), s);
    if (rc != SATPILA_OK) return rc;
    const size_t bytes = (size_t)p->U * p->B * sizeof(double);
    SP_CUDA(cudaMemcpyAsync(w, p->d_w64, bytes, is_device_pointer(w) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    return SATPILA_OK;
}
