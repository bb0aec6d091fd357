// PILA construction (Eq. (5), Sec. II-B) and the table-level API calls.
//
// One thread per (pixel, angle) record.  The chord of a line through a unit
// square depends only on its distance t to the square's centre along the
// line's normal: with a = |cos|, b = |sin|, the square projects onto the
// normal as a trapezoid of half-width (a+b)/2, flat top of half-width
// |a-b|/2 and height 1/max(a,b).  The rays crossing the pixel are the bins
// whose centre lies in [s_p - (a+b)/2, s_p + (a+b)/2) (half-open, so a ray
// on an edge belongs to the pixel on its +s side); since a+b <= sqrt(2) < 2
// there are at most two, on consecutive bins.  FP64 arithmetic, rounded once
// to the record's precision.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "sat_host.h"

namespace satpila {
namespace {

// One thread per (angle u, pixel p): threads of a block span consecutive
// angles (coalesced record writes), blocks step through the pixels.  The
// per-angle terms (a, b, half-width, plateau half-width, plateau height, a*b)
// are the same FP64 expressions for every pixel, so they are formed once.
__global__ void pila_build_kernel(unsigned char* table, int f16, int row_records, int n, int U, int B,
                                  const double* cs, const double* sn, unsigned long long* entries) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = n * n;  // at most 2^30
    double c = 0.0, s = 0.0, half = 0.0, flat = 0.0, height = 0.0, ab = 0.0;
    if (u < U) {
        c = cs[u];
        s = sn[u];
        const double a = fabs(c), b = fabs(s);
        half = 0.5 * (a + b);
        flat = 0.5 * fabs(a - b);
        height = 1.0 / fmax(a, b);
        ab = a * b;
    }
    const double centre = 0.5 * (B - 1);
    unsigned long long count = 0;
    if (u < row_records) {
        for (int p = blockIdx.y; p < P; p += gridDim.y) {
            int cnt = 0;
            int kk[2] = {0, 0};
            double ll[2] = {0.0, 0.0};
            if (u < U) {
                const int i = p / n, j = p - i * n;
                const double x = (double)j - 0.5 * (n - 1), y = 0.5 * (n - 1) - (double)i;
                const double sp = x * c + y * s;
                const double kfirst = ceil(sp - half + centre);
                for (int t = 0; t < 2; ++t) {
                    const double kd = kfirst + t;
                    const double d = (kd - centre) - sp;
                    if (d < -half || d >= half) continue;
                    const double dist = fabs(d);
                    const double l = dist <= flat ? height : (half - dist) / ab;
                    if (!(l >= 1e-12)) continue;
                    if (kd < 0.0 || kd >= (double)B) continue;
                    kk[cnt] = (int)kd;
                    ll[cnt] = l;
                    ++cnt;
                }
            }
            if (cnt == 0) kk[0] = kk[1] = 0;
            if (cnt == 1) kk[1] = kk[0];
            const long long idx = (long long)p * row_records + u;
            if (f16 == PILA_U8) {
                // lengths times 180, rounded (at most round(sqrt 2 * 180) = 255)
                const uint32_t q0 = (uint32_t)fmin(255.0, rint(ll[0] * 180.0));
                const uint32_t q1 = (uint32_t)fmin(255.0, rint(ll[1] * 180.0));
                reinterpret_cast<uint32_t*>(table)[idx] = ((uint32_t)(uint16_t)kk[0]) | (q0 << 16) | (q1 << 24);
                count += (q0 != 0u) + (q1 != 0u);
            } else if (f16) {
                const __half h0 = __double2half(ll[0]), h1 = __double2half(ll[1]);
                const uint32_t bins = ((uint32_t)(uint16_t)kk[0]) | ((uint32_t)(uint16_t)kk[1] << 16);
                const uint32_t lens = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
                reinterpret_cast<uint2*>(table)[idx] = make_uint2(bins, lens);
                count += (__half2float(h0) != 0.0f) + (__half2float(h1) != 0.0f);
            } else {
                const float f0 = (float)ll[0], f1 = (float)ll[1];
                reinterpret_cast<uint4*>(table)[idx] =
                    make_uint4((uint32_t)kk[0], (uint32_t)kk[1], __float_as_uint(f0), __float_as_uint(f1));
                count += (f0 != 0.0f) + (f1 != 0.0f);
            }
        }
    }
    // warp-level count of non-empty entries
    for (int o = 16; o > 0; o >>= 1) count += __shfl_xor_sync(0xffffffffu, count, o);
    if ((threadIdx.x & 31) == 0 && count) atomicAdd(entries, count);
}

// Per pixel, the sum of its stored lengths squared (sum l^2 of Eq. (7)'s
// (df l)^2 term), accumulated in FP64 in angle order and rounded once.
__global__ void pila_hsum_kernel(const unsigned char* table, int f16, int row_records, int U, long long P,
                                 float* hsum) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double acc = 0.0;
    for (int u = 0; u < U; ++u) {
        const long long rec = p * row_records + u;
        const Entry2 e = decode_rec(table, rec, f16);
        acc += (double)e.l0 * e.l0 + (double)e.l1 * e.l1;
    }
    hsum[p] = (float)acc;
}

// Smallest and largest cell an annealing move can touch: over the records of
// the reconstruction-space pixels, bin k0 and the cell k0 + 1 that the second
// entry of a record addresses.  Threads span angles, blocks step through the
// list; one pair of atomics per block.
__global__ void pila_band_kernel(const unsigned char* table, int f16, int row_records, int U, const int32_t* list,
                                 int n_list, int* lohi) {
    int lo = 0x7fffffff, hi = -1;
    for (int u = threadIdx.x; u < U; u += blockDim.x)
        for (int q = blockIdx.x; q < n_list; q += gridDim.x) {
            const Entry2 e = decode_rec(table, (long long)list[q] * row_records + u, f16);
            lo = min(lo, e.k0);
            hi = max(hi, e.k0 + 1);
        }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ int red[2][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = lo;
        red[1][warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = min(lo, red[0][w]);
            hi = max(hi, red[1][w]);
        }
        if (hi >= 0) {
            atomicMin(&lohi[0], lo);
            atomicMax(&lohi[1], hi);
        }
    }
}

__global__ void pila_export_kernel(const unsigned char* table, int f16, int row_records, int U, long long P,
                                   int32_t* bins, float* lens) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P * U) return;
    const long long p = idx / U;
    const int u = (int)(idx % U);
    const long long rec = p * row_records + u;
    const Entry2 e = decode_rec(table, rec, f16);
    bins[idx * 2] = e.l0 != 0.0f ? e.k0 : -1;
    bins[idx * 2 + 1] = e.l1 != 0.0f ? e.k1 : -1;
    lens[idx * 2] = e.l0;
    lens[idx * 2 + 1] = e.l1;
}

}  // namespace
}  // namespace satpila

using namespace satpila;

extern "C" int pila_build(const pila_geom* g, int32_t precision, void* stream, satpila_pila** out) {
    return satpila::pila_build_in(g, precision, (cudaStream_t)stream, nullptr, out);
}

int satpila::pila_build_in(const pila_geom* g, int32_t precision, cudaStream_t stream, cudaMemPool_t pool,
                           satpila_pila** out, bool ray_index) {
    if (!g || !out) return fail(SATPILA_ERR_INVALID_ARG, "pila_build: null argument");
    *out = nullptr;
    if (g->n < 1 || g->n_angles < 1 || g->n_bins < 1)
        return fail(SATPILA_ERR_INVALID_ARG, "pila_build: n, n_angles and n_bins must be >= 1");
    if (precision != PILA_F32 && precision != PILA_F16 && precision != PILA_U8)
        return fail(SATPILA_ERR_INVALID_ARG, "pila_build: precision must be PILA_F32, PILA_F16 or PILA_U8");
    if (precision != PILA_F32 && g->n_bins > 32767)
        return fail(SATPILA_ERR_INVALID_ARG, "pila_build: 16-bit bins need n_bins <= 32767");
    if ((long long)g->n * g->n > (1LL << 30))
        return fail(SATPILA_ERR_INVALID_ARG, "pila_build: image too large");
    cudaStream_t s = stream;
    auto* p = new satpila_pila();
    cudaGetDevice(&p->device);
    p->pool = pool;
    p->alloc_stream = pool ? s : nullptr;
    p->n = g->n;
    p->U = g->n_angles;
    p->B = g->n_bins;
    p->precision = precision;
    p->record_bytes = precision == PILA_U8 ? 4 : precision == PILA_F16 ? 8 : 16;
    // rows are whole 16-byte chunks
    p->row_records = (p->U + 16 / p->record_bytes - 1) / (16 / p->record_bytes) * (16 / p->record_bytes);
    p->row_bytes = (int64_t)p->row_records * p->record_bytes;
    const long long P = (long long)p->n * p->n;
    p->table_bytes = P * p->row_bytes;

    // angle tables (FP64, exact zeros for |v| < 1e-12)
    std::vector<double> cs(p->U), sn(p->U);
    for (int u = 0; u < p->U; ++u) {
        const double th = g->angles_rad ? g->angles_rad[u] : M_PI * (double)u / (double)p->U;
        cs[u] = std::cos(th);
        sn[u] = std::sin(th);
        if (std::fabs(cs[u]) < 1e-12) cs[u] = 0.0;
        if (std::fabs(sn[u]) < 1e-12) sn[u] = 0.0;
    }
    // reconstruction-space list
    std::vector<uint8_t> mask(P, 1);
    std::vector<int32_t> list;
    list.reserve(P);
    for (long long q = 0; q < P; ++q) {
        if (g->mask) mask[q] = g->mask[q] ? 1 : 0;
        if (mask[q]) list.push_back((int32_t)q);
    }
    p->n_mask = (int)list.size();

    auto cleanup = [&](int code, const std::string& msg) {
        pila_free(p);
        return fail(code, msg);
    };
    auto dalloc = [&](auto** ptr, size_t bytes) {
        void* v = nullptr;
        const cudaError_t e = pool ? cudaMallocFromPoolAsync(&v, bytes, pool, s) : cudaMalloc(&v, bytes);
        *ptr = static_cast<std::remove_pointer_t<decltype(ptr)>>(v);
        return e == cudaSuccess;
    };
    unsigned long long* d_entries = nullptr;  // entry count, then the band bounds
    if (!dalloc(&p->d_table, p->table_bytes) || !dalloc(&p->d_list, std::max<size_t>(1, list.size()) * 4) ||
        !dalloc(&p->d_mask, P) || !dalloc(&p->d_cos, p->U * sizeof(double)) ||
        !dalloc(&p->d_sin, p->U * sizeof(double)) || !dalloc(&p->d_hsum, P * sizeof(float)) ||
        !dalloc(&d_entries, 2 * sizeof(unsigned long long))) {
        cudaGetLastError();
        if (d_entries) pool ? cudaFreeAsync(d_entries, s) : cudaFree(d_entries);
        return cleanup(SATPILA_ERR_OOM, "pila_build: device allocation failed");
    }
    cudaError_t e = cudaSuccess;
    if (!list.empty())
        e = cudaMemcpyAsync(p->d_list, list.data(), list.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_mask, mask.data(), P, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_cos, cs.data(), p->U * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_sin, sn.data(), p->U * sizeof(double), cudaMemcpyHostToDevice, s);
    const int band_init[2] = {0x7fffffff, -1};
    if (e == cudaSuccess) e = cudaMemsetAsync(d_entries, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_entries + 1, band_init, sizeof(band_init), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const int threads = 128;
        const dim3 grid((unsigned)((p->row_records + threads - 1) / threads), (unsigned)std::min<long long>(P, 8192));
        pila_build_kernel<<<grid, threads, 0, s>>>(p->d_table, precision, p->row_records, p->n, p->U, p->B,
                                                   p->d_cos, p->d_sin, d_entries);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        pila_hsum_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(p->d_table, precision,
                                                                     p->row_records, p->U, P, p->d_hsum);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !list.empty()) {
        const int threads = p->U >= 256 ? 256 : (p->U + 31) / 32 * 32;
        pila_band_kernel<<<(unsigned)std::min<size_t>(list.size(), 4096), threads, 0, s>>>(
            p->d_table, precision, p->row_records, p->U, p->d_list, (int)list.size(),
            reinterpret_cast<int*>(d_entries + 1));
        e = cudaGetLastError();
    }
    unsigned long long entries[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(entries, d_entries, sizeof(entries), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (pool) cudaFreeAsync(d_entries, s);
    else cudaFree(d_entries);
    if (e != cudaSuccess) {
        const std::string msg = std::string("pila_build: ") + cudaGetErrorString(e);
        return cleanup(SATPILA_ERR_CUDA, msg);
    }
    p->entries = (int64_t)entries[0];
    int band[2];
    std::memcpy(band, &entries[1], sizeof(band));
    if (list.empty() || band[1] < band[0]) band[0] = 0, band[1] = 1;
    p->band_lo = std::max(0, band[0]);
    p->band_hi = std::min(p->B, band[1]);
    if (ray_index) {
        const int rc = build_ray_index(p, s, pool);
        if (rc != SATPILA_OK) {
            const std::string msg = satpila_last_error();
            return cleanup(rc, msg);
        }
    }
    *out = p;
    return SATPILA_OK;
}

extern "C" int pila_free(satpila_pila* p) {
    if (!p) return SATPILA_OK;
    sat_cache_purge(p);
    void* bufs[] = {p->d_table, p->d_list, p->d_mask, p->d_cos, p->d_sin, p->d_hsum, p->d_ray_off, p->d_ray_ent};
    for (void* b : bufs) {
        if (!b) continue;
        if (p->pool) cudaFreeAsync(b, p->alloc_stream);
        else cudaFree(b);
    }
    if (p->d_w64) cudaFree(p->d_w64);  // SIRT factor: ordinary allocations
    if (p->d_w32) cudaFree(p->d_w32);
    delete p;
    return SATPILA_OK;
}

extern "C" int pila_info(const satpila_pila* p, pila_info_t* info) {
    if (!p || !info) return fail(SATPILA_ERR_INVALID_ARG, "pila_info: null argument");
    info->n = p->n;
    info->n_angles = p->U;
    info->n_bins = p->B;
    info->precision = p->precision;
    info->n_mask = p->n_mask;
    info->record_bytes = p->record_bytes;
    info->row_records = p->row_records;
    info->pad = 0;
    info->table_bytes = p->table_bytes;
    info->entries = p->entries;
    return SATPILA_OK;
}

extern "C" int pila_export(const satpila_pila* p, int32_t* bins, float* lens, void* stream) {
    if (!p || !bins || !lens) return fail(SATPILA_ERR_INVALID_ARG, "pila_export: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const long long P = (long long)p->n * p->n;
    const size_t cnt = (size_t)P * p->U * 2;
    const bool dev_b = is_device_pointer(bins), dev_l = is_device_pointer(lens);
    int32_t* db = bins;
    float* dl = lens;
    if (!dev_b) SP_CUDA(cudaMalloc(&db, cnt * sizeof(int32_t)));
    if (!dev_l) SP_CUDA(cudaMalloc(&dl, cnt * sizeof(float)));
    const long long total = P * p->U;
    pila_export_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(p->d_table, p->precision,
                                                                       p->row_records, p->U, P, db, dl);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !dev_b) e = cudaMemcpyAsync(bins, db, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && !dev_l) e = cudaMemcpyAsync(lens, dl, cnt * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (!dev_b) cudaFree(db);
    if (!dev_l) cudaFree(dl);
    if (e != cudaSuccess) return cuda_fail(e, "pila_export");
    return SATPILA_OK;
}
