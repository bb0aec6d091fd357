// Device helpers shared by the satpila kernels (sm_103a).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "satpila.h"

namespace satpila {

constexpr uint32_t kStreamSat = 1u;  // Philox stream id of the annealing moves
constexpr uint32_t kStreamT0 = 2u;   // Philox stream id of the Eq. (8) samples
constexpr int kMaxK = 32;            // most BoME estimates per move
constexpr int kMaxStages = 8;        // deepest PILA-row prefetch ring
constexpr uint32_t kWaitSpins = 1u << 22;  // bound on every device-side wait loop

// Philox4x32 with 10 rounds (Salmon et al., SC'11): per round two 32x32->64
// products of counter words with fixed multipliers, mixed with the other
// counter words and the key; the key advances by a Weyl increment.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Uniform in (0, 1): an odd multiple of 2^-24, exact in FP32.
__device__ __forceinline__ float unit_uniform(uint32_t x) {
    return (float)((x >> 9) * 2u + 1u) * 0x1p-24f;
}

// floor(x * m / 2^32): uniform index in [0, m).
__device__ __forceinline__ uint32_t pick_index(uint32_t x, uint32_t m) { return __umulhi(x, m); }

__device__ __forceinline__ uint2 chain_key(unsigned long long seed) {
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// ---- shared-memory barriers and bulk copies (inline PTX) -------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) accesses of the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> this CTA's shared memory, completion counted on bar.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for a barrier phase (at most kWaitSpins polls and 2 s of wall
// time); false if the bound ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t i = 0; i < kWaitSpins; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// st.global.cg of v under a predicate, without a branch around it.
__device__ __forceinline__ void stcg_if(bool pred, float* p, float v) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.global.cg.f32 [%1], %2;\n\t}" ::"r"((int)pred),
        "l"(p), "f"(v)
        : "memory");
}

// The same prefetch under a predicate, without a branch around it (the
// address is not touched when pred is false).
__device__ __forceinline__ void prefetch_l1_if(bool pred, const void* p) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q prefetch.global.L1 [%1];\n\t}" ::"r"((int)pred),
        "l"(p));
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Records one error code (the first one wins).
__device__ __forceinline__ void raise_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// ---- PILA records ------------------------------------------------------------

struct Entry2 {
    int k0, k1;
    float l0, l1;
};

__device__ __forceinline__ Entry2 decode_f32(uint4 v) {
    return Entry2{(int)v.x, (int)v.y, __uint_as_float(v.z), __uint_as_float(v.w)};
}

__device__ __forceinline__ Entry2 decode_f16(uint32_t bins, uint32_t lens) {
    Entry2 e;
    e.k0 = (int)(int16_t)(bins & 0xffffu);
    e.k1 = (int)(int16_t)(bins >> 16);
    e.l0 = __half2float(__ushort_as_half((unsigned short)(lens & 0xffffu)));
    e.l1 = __half2float(__ushort_as_half((unsigned short)(lens >> 16)));
    return e;
}

// Record of the one-byte table (the storage Sec. II-B describes): bits 0-15
// the bin of entry 0 (entry 1, when present, sits on the next bin), bits
// 16-23 and 24-31 the two lengths times 180, rounded.  A stored length is
// q * fl(1/180), the same value wherever the table is read.
constexpr float kU8Unit = 1.0f / 180.0f;

__device__ __forceinline__ Entry2 decode_u8(uint32_t v) {
    Entry2 e;
    e.k0 = (int)(v & 0xffffu);
    e.l0 = (float)((v >> 16) & 0xffu) * kU8Unit;
    e.l1 = (float)(v >> 24) * kU8Unit;
    e.k1 = e.l1 != 0.0f ? e.k0 + 1 : e.k0;
    return e;
}

// Record rec of a table of precision prec (PILA_F32, PILA_F16, PILA_U8).
__device__ __forceinline__ Entry2 decode_rec(const unsigned char* table, long long rec, int prec) {
    if (prec == PILA_F16) {
        const uint2 v = reinterpret_cast<const uint2*>(table)[rec];
        return decode_f16(v.x, v.y);
    }
    if (prec == PILA_U8) return decode_u8(reinterpret_cast<const uint32_t*>(table)[rec]);
    return decode_f32(reinterpret_cast<const uint4*>(table)[rec]);
}

// ---- exact fixed-point accumulation ------------------------------------------

// Fraction bits F such that sum of |terms| <= bound stays below 2^61.
__device__ __forceinline__ int fixed_point_bits(double bound) {
    if (!(bound > 0.0)) return 0;
    int ex;
    frexp(bound, &ex);  // bound < 2^ex
    return 61 - ex;
}

}  // namespace satpila
