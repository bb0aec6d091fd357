// Ray-major index of the PILA (Eq. (5) stored the other way round): for every
// ray (u, k), the pixels it crosses with their stored lengths.  The table is
// pixel-major, which suits the annealing move (one pixel, all angles); a
// forward projection (Eq. (1)) sums along rays, and with this index one warp
// can sum a ray in registers instead of scattering pixel terms into shared
// accumulators.  Built once per table from the records themselves, so the
// lengths are exactly the stored (dequantised) values (kept as significand and
// exponent, the two parts of the exact term).
//
// Steps: count the entries of every ray (one thread per record), exclusive
// scan, place the entries (per-ray cursors), then sort each ray by pixel so
// that consecutive entries read nearby image words.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace satpila {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 4;
constexpr int kScanBlock = kScanThreads * kScanPerThread;
constexpr int kSortThreads = 256;
constexpr int kSortMax = 4096;  // longest ray the shared-memory sort takes (a ray crosses at most 2n pixels)

// Threads span angles (as the table build does), blocks step through pixels.
template <bool FILL>
__global__ void ray_place_kernel(const unsigned char* table, int prec, int row_records, int n, int U, int B,
                                 uint32_t* cursor, uint2* ent) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    const int P = n * n;
    for (int p = blockIdx.y; p < P; p += gridDim.y) {
        const Entry2 e = decode_rec(table, (long long)p * row_records + u, prec);
        const uint32_t ray = (uint32_t)u * (uint32_t)B;
        if (e.l0 != 0.0f) {
            const uint32_t at = atomicAdd(&cursor[ray + e.k0], 1u);
            if (FILL) ent[at] = make_uint2((uint32_t)p, __float_as_uint(e.l0));
        }
        if (e.l1 != 0.0f) {
            const uint32_t at = atomicAdd(&cursor[ray + e.k1], 1u);
            if (FILL) ent[at] = make_uint2((uint32_t)p, __float_as_uint(e.l1));
        }
    }
}

// Exclusive scan, step 1: each block scans kScanBlock counts and leaves its
// total in sums[block].
__global__ void __launch_bounds__(kScanThreads) scan_block_kernel(const uint32_t* in, uint32_t* out, uint32_t* sums,
                                                                  long long n) {
    __shared__ uint32_t s[kScanThreads];
    const long long base = (long long)blockIdx.x * kScanBlock + (long long)threadIdx.x * kScanPerThread;
    uint32_t v[kScanPerThread];
    uint32_t mine = 0;
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        v[j] = base + j < n ? in[base + j] : 0u;
        mine += v[j];
    }
    s[threadIdx.x] = mine;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        const uint32_t t = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = s[threadIdx.x] - mine;
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = s[kScanThreads - 1];
}

// Step 2: one block turns the block totals into exclusive offsets, in
// chunks of kScanThreads with a running carry.
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint32_t* sums, int nb) {
    __shared__ uint32_t s[kScanThreads];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += kScanThreads) {
        const int i = c0 + threadIdx.x;
        const uint32_t v = i < nb ? sums[i] : 0u;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < kScanThreads; off <<= 1) {
            const uint32_t t = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0u;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) sums[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry += s[kScanThreads - 1];
        __syncthreads();
    }
}

// Step 3: offsets = block offset + in-block offset; the cursors start there.
__global__ void scan_add_kernel(uint32_t* out, uint32_t* cursor, const uint32_t* sums, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t v = out[i] + sums[i / kScanBlock];
    out[i] = v;
    cursor[i] = v;
}

// One block per ray: bitonic sort of its entries by pixel (keys pixel << 32 |
// length bits; a pixel meets a ray at most once, so keys are distinct).
__global__ void __launch_bounds__(kSortThreads) ray_sort_kernel(const uint32_t* off, uint2* ent) {
    __shared__ unsigned long long key[kSortMax];
    const long long ray = blockIdx.x;
    const uint32_t e0 = off[ray], len = off[ray + 1] - e0;
    if (len < 2 || len > (uint32_t)kSortMax) return;
    int N = 2;
    while ((uint32_t)N < len) N <<= 1;
    for (int i = threadIdx.x; i < N; i += kSortThreads) {
        if ((uint32_t)i < len) {
            const uint2 v = ent[e0 + i];
            key[i] = ((unsigned long long)v.x << 32) | v.y;
        } else {
            key[i] = ~0ull;
        }
    }
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += kSortThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = key[i], b = key[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        key[i] = b;
                        key[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; (uint32_t)i < len; i += kSortThreads)
        ent[e0 + i] = make_uint2((uint32_t)(key[i] >> 32), (uint32_t)key[i]);
}

// Last step: each entry's length from float32 bits to the form the
// projector's exact terms take: its significand (hidden bit set) shifted left
// by 7, with the biased exponent in the 7 low bits freed (a stored length is
// at most sqrt 2, so the exponent is below 128).
__global__ void ray_pack_kernel(uint2* ent, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t b = ent[i].y;
    ent[i].y = (((b & 0x7fffffu) | 0x800000u) << 7) | ((b >> 23) & 0x7fu);
}

}  // namespace

int build_ray_index(satpila_pila* p, cudaStream_t s, cudaMemPool_t pool) {
    const long long rays = (long long)p->U * p->B;
    if (p->entries >= (int64_t)0xffffffffLL || rays + 1 >= (long long)0xffffffffLL) return SATPILA_OK;  // too large: no index
    const long long nb = (rays + kScanBlock - 1) / kScanBlock;
    auto dalloc = [&](auto** ptr, size_t bytes) {
        void* v = nullptr;
        const cudaError_t e = pool ? cudaMallocFromPoolAsync(&v, bytes, pool, s) : cudaMalloc(&v, bytes);
        *ptr = static_cast<std::remove_pointer_t<decltype(ptr)>>(v);
        return e == cudaSuccess;
    };
    auto dfree = [&](void* v) {
        if (v) pool ? cudaFreeAsync(v, s) : cudaFree(v);
    };
    uint32_t* cnt = nullptr;  // counts, then cursors
    uint32_t* sums = nullptr;
    if (!dalloc(&p->d_ray_off, (size_t)(rays + 1) * 4) ||
        !dalloc(&p->d_ray_ent, (size_t)std::max<int64_t>(1, p->entries) * sizeof(uint2)) ||
        !dalloc(&cnt, (size_t)rays * 4) || !dalloc(&sums, (size_t)nb * 4)) {
        cudaGetLastError();
        dfree(cnt);
        dfree(sums);
        return fail(SATPILA_ERR_OOM, "pila_build: ray index allocation failed");
    }
    p->ray_bytes = (rays + 1) * 4 + p->entries * (int64_t)sizeof(uint2);
    const uint32_t total = (uint32_t)p->entries;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)rays * 4, s);
    const int threads = 128;
    const dim3 grid((unsigned)((p->U + threads - 1) / threads),
                    (unsigned)std::min<long long>((long long)p->n * p->n, 8192));
    if (e == cudaSuccess) {
        ray_place_kernel<false><<<grid, threads, 0, s>>>(p->d_table, p->precision, p->row_records, p->n, p->U, p->B,
                                                         cnt, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        scan_block_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(cnt, p->d_ray_off, sums, rays);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        scan_sums_kernel<<<1, kScanThreads, 0, s>>>(sums, (int)nb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        scan_add_kernel<<<(unsigned)((rays + 255) / 256), 256, 0, s>>>(p->d_ray_off, cnt, sums, rays);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_ray_off + rays, &total, 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        ray_place_kernel<true><<<grid, threads, 0, s>>>(p->d_table, p->precision, p->row_records, p->n, p->U, p->B,
                                                        cnt, p->d_ray_ent);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ray_sort_kernel<<<(unsigned)rays, kSortThreads, 0, s>>>(p->d_ray_off, p->d_ray_ent);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && total > 0) {
        ray_pack_kernel<<<(total + 255) / 256, 256, 0, s>>>(p->d_ray_ent, total);
        e = cudaGetLastError();
    }
    // `total` is read by the copy above before the call returns
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(cnt);
    dfree(sums);
    if (e != cudaSuccess) return cuda_fail(e, "pila_build: ray index");
    return SATPILA_OK;
}

}  // namespace satpila
