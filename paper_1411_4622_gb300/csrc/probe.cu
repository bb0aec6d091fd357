// Memory-level probes: the read rates that bound the annealer's gathers, measured on the running GPU.
//
// The move reads three kinds of bytes: the pixel's PILA row (consecutive 16-byte chunks of one record row, from L2
// when the table fits there, else from HBM), the residual cells of its entries (one 32-byte sector per record,
// scattered over the chain's residual: shared memory, L2 or HBM) and two image words.  A copy-bandwidth figure is
// the right denominator for none of them except a table streamed from HBM, so these probes time each access pattern
// by itself:
//   - stream: consecutive 16-byte loads (whole lines per warp), as the PILA rows are read;
//   - sector: one 32-byte sector at a pseudo-random place per load, as the residual cells are read;
//   - shared-memory 4-byte loads, conflict-free or at pseudo-random words.
// Every global load bypasses L1 (ld.global.cg), so a buffer that fits in L2 measures L2 and one many times larger
// than L2 measures HBM.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace satpila {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 8;       // independent loads in flight per thread
constexpr int kSmemWords = 8192;      // 32 KB shared-memory array of the smem probe (static limit 48 KB)

// 32-bit integer hash (the finaliser of MurmurHash3): spreads consecutive
// inputs over the whole word, so sector indices look random to the memory.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

// Each warp gathers inside its own region of region_sectors sectors (region
// w mod n_regions for global warp w), as a chain's warps gather inside that
// chain's residual; one region spanning the buffer scatters over all of it.
__global__ void __launch_bounds__(kProbeThreads) probe_sector_kernel(const uint4* buf, uint32_t region_sectors,
                                                                     uint32_t n_regions, int iters, uint32_t seed,
                                                                     uint32_t* sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t base = (uint64_t)((t >> 5) % n_regions) * region_sectors;
    uint32_t h = mix32(t ^ seed);
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
        uint4 v[kProbeUnroll];
#pragma unroll
        for (int j = 0; j < kProbeUnroll; ++j) {
            h = mix32(h + 0x9E3779B9u);
            const uint64_t s = base + __umulhi(h, region_sectors);  // a sector of the warp's region
            v[j] = __ldcg(buf + 2ull * s);
        }
#pragma unroll
        for (int j = 0; j < kProbeUnroll; ++j) acc ^= v[j].x ^ v[j].w;
    }
    if (acc == 0x9E3779B9u) sink[t & 1023u] = acc;  // keeps the loads; practically never taken
}

__global__ void __launch_bounds__(kProbeThreads) probe_stream_kernel(const uint4* buf, uint64_t n_chunks, int iters,
                                                                     uint32_t* sink) {
    // i stays in [0, n_chunks): it starts reduced and advances by less than n_chunks
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) % n_chunks;
    uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) % n_chunks;
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
        uint4 v[kProbeUnroll];
#pragma unroll
        for (int j = 0; j < kProbeUnroll; ++j) {
            v[j] = __ldcg(buf + i);
            i += stride;
            if (i >= n_chunks) i -= n_chunks;
        }
#pragma unroll
        for (int j = 0; j < kProbeUnroll; ++j) acc ^= v[j].x ^ v[j].w;
    }
    if (acc == 0x9E3779B9u) sink[threadIdx.x] = acc;
}

// kind 0: lane i of every load reads bank i (conflict-free); kind 1: each
// lane reads a pseudo-random word of the array.  (h >> 19) keeps 13 bits:
// a word index below kSmemWords.
__global__ void __launch_bounds__(kProbeThreads) probe_smem_kernel(int kind, int iters, uint32_t* sink) {
    __shared__ uint32_t words[kSmemWords];
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    for (uint32_t i = tid; i < kSmemWords; i += kProbeThreads) words[i] = i * 2654435761u;
    __syncthreads();
    uint32_t acc = 0;
    uint32_t h = mix32(blockIdx.x * kProbeThreads + tid);
    uint32_t base = (tid >> 5) * 1024u;
    for (int it = 0; it < iters; ++it) {
        uint32_t v[kProbeUnroll];
        if (kind == 0) {
#pragma unroll
            for (int j = 0; j < kProbeUnroll; ++j) v[j] = words[(base + 32u * j + lane) & (kSmemWords - 1)];
            base += 32u * kProbeUnroll;
        } else {
#pragma unroll
            for (int j = 0; j < kProbeUnroll; ++j) {
                h = h * 1664525u + 1013904223u;  // LCG step (Numerical Recipes constants)
                v[j] = words[(h >> 19) & (kSmemWords - 1)];
            }
        }
#pragma unroll
        for (int j = 0; j < kProbeUnroll; ++j) acc += v[j];
    }
    if (acc == 0x9E3779B9u) sink[tid] = acc;
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, sms);
}

// One untimed launch, then the timed one; returns its milliseconds.
template <typename Launch>
int time_launch(Launch launch, cudaStream_t s, float* ms) {
    cudaEvent_t e0, e1;
    SP_CUDA(cudaEventCreate(&e0));
    SP_CUDA(cudaEventCreate(&e1));
    cudaError_t e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "probe launch");
    return SATPILA_OK;
}

uint32_t* probe_sink() {
    static uint32_t* sink[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!sink[dev] && cudaMalloc(&sink[dev], 1024 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return sink[dev];
}

}  // namespace
}  // namespace satpila

using namespace satpila;

extern "C" int satpila_probe_read(const void* buf, uint64_t bytes, int32_t kind, uint64_t region_bytes,
                                  uint64_t loads, double* gbs, void* stream) {
    if (!buf || !gbs || bytes < 4096 || (reinterpret_cast<uintptr_t>(buf) & 15u) != 0 || loads == 0)
        return fail(SATPILA_ERR_INVALID_ARG, "satpila_probe_read: bad argument");
    if (kind != SATPILA_PROBE_STREAM && kind != SATPILA_PROBE_SECTOR)
        return fail(SATPILA_ERR_INVALID_ARG, "satpila_probe_read: unknown kind");
    if (!is_device_pointer(buf)) return fail(SATPILA_ERR_INVALID_ARG, "satpila_probe_read: buf must be device memory");
    const uint64_t sectors = bytes / 32;
    const uint64_t region = region_bytes == 0 ? sectors : std::min<uint64_t>(region_bytes / 32, sectors);
    if (kind == SATPILA_PROBE_SECTOR && (region == 0 || region > 0xffffffffull || sectors / region > 0xffffffffull))
        return fail(SATPILA_ERR_INVALID_ARG, "satpila_probe_read: regions of 32 bytes to 2^32 sectors");
    uint32_t* sink = probe_sink();
    if (!sink) return fail(SATPILA_ERR_OOM, "satpila_probe_read: sink");
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = sm_count() * 8;
    const uint64_t per_launch = (uint64_t)grid * kProbeThreads * kProbeUnroll;
    const int iters = (int)std::max<uint64_t>(1, std::min<uint64_t>((loads + per_launch - 1) / per_launch, 1u << 20));
    const uint4* b4 = static_cast<const uint4*>(buf);
    float ms = 0.0f;
    int rc;
    if (kind == SATPILA_PROBE_SECTOR) {
        rc = time_launch([&]() {
            probe_sector_kernel<<<grid, kProbeThreads, 0, s>>>(b4, (uint32_t)region, (uint32_t)(sectors / region),
                                                               iters, 12345u, sink);
            return cudaGetLastError();
        }, s, &ms);
    } else {
        const uint64_t chunks = bytes / 16;
        rc = time_launch([&]() {
            probe_stream_kernel<<<grid, kProbeThreads, 0, s>>>(b4, chunks, iters, sink);
            return cudaGetLastError();
        }, s, &ms);
    }
    if (rc != SATPILA_OK) return rc;
    const double bytes_read = (double)per_launch * iters * (kind == SATPILA_PROBE_SECTOR ? 32.0 : 16.0);
    *gbs = ms > 0.0f ? bytes_read / (ms * 1e-3) / 1e9 : 0.0;
    return SATPILA_OK;
}

extern "C" int satpila_probe_smem(int32_t kind, uint64_t loads, double* gbs, void* stream) {
    if (!gbs || loads == 0 || (kind != 0 && kind != 1))
        return fail(SATPILA_ERR_INVALID_ARG, "satpila_probe_smem: bad argument");
    uint32_t* sink = probe_sink();
    if (!sink) return fail(SATPILA_ERR_OOM, "satpila_probe_smem: sink");
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = sm_count() * 8;
    const uint64_t per_launch = (uint64_t)grid * kProbeThreads * kProbeUnroll;
    const int iters = (int)std::max<uint64_t>(1, std::min<uint64_t>((loads + per_launch - 1) / per_launch, 1u << 20));
    float ms = 0.0f;
    const int rc = time_launch([&]() {
        probe_smem_kernel<<<grid, kProbeThreads, 0, s>>>(kind, iters, sink);
        return cudaGetLastError();
    }, s, &ms);
    if (rc != SATPILA_OK) return rc;
    *gbs = ms > 0.0f ? (double)per_launch * iters * 4.0 / (ms * 1e-3) / 1e9 : 0.0;
    return SATPILA_OK;
}
