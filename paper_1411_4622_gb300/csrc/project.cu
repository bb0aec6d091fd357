// Forward projection through the PILA (the DRT of Eq. (1) with the stored
// lengths), used for: the FP64 residual resync and final cost of the
// annealer (Eq. (4)), the public pila_forward call, the SIRT factor matrix
// (Sec. III-D, lengths squared over the reconstruction space) and the SIRT
// correction of Eq. (11).
//
// Design: one CTA per (image, group of up to 16 angles) holds a shared-memory
// accumulator for its [angles][bins] block.  Warps walk the pixels, each lane
// one (pixel, angle) pair of the group (a pixel's records of the group are
// contiguous), and every product f * l is added as an exact 64-bit
// fixed-point integer (integer units; the FP64 units of this part are
// scarce).  Groups are as wide as the number of CTAs allows.  Integer addition is associative, so
// the result does not depend on the order of the shared-memory atomics:
// the projection is deterministic and at least as accurate as an FP64 sum.
// The fraction bits are chosen per image from max|f| so nothing overflows.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace satpila {
namespace {

constexpr int kProjThreads = 512;
constexpr int kProjSmemBudget = 200 * 1024;

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

// A float split for exact fixed-point products: significand (with the
// hidden bit), exponent of its last bit, sign.
struct FixedSplit {
    uint32_t m;
    int x;
    uint32_t neg;
};

__device__ __forceinline__ FixedSplit fixed_split(float a) {
    const uint32_t ba = __float_as_uint(a);
    const uint32_t ea = (ba >> 23) & 0xffu;
    FixedSplit s;
    s.m = ba & 0x7fffffu;
    s.x = -149;
    if (ea) {
        s.m |= 0x800000u;
        s.x = (int)ea - 150;
    }
    s.neg = ba >> 31;
    return s;
}

// round(a * l * 2^F) for a split a and a positive normal float l (every
// stored length is one: at least 1e-12, or a decoded half or byte): the
// 48-bit product of the significands shifted by the combined exponent (round
// half away from zero), on the integer units.  F keeps it from overflowing.
__device__ __forceinline__ long long fixed_mul(const FixedSplit& a, float l, int F) {
    const uint32_t bl = __float_as_uint(l);
    const uint32_t ml = (bl & 0x7fffffu) | 0x800000u;
    const int e = a.x + (int)((bl >> 23) & 0xffu) - 150 + F;
    const unsigned long long m = (unsigned long long)a.m * (unsigned long long)ml;
    unsigned long long v;
    if (e >= 0) {
        v = m << e;
    } else if (e > -64) {
        const int sh = -e;
        v = (m >> sh) + ((m >> (sh - 1)) & 1ull);
    } else {
        v = 0ull;
    }
    return a.neg ? -(long long)v : (long long)v;
}

// Adds f * l (or l * l for the factor matrix) to bin k of an accumulator row.
__device__ __forceinline__ void add_entry(long long* row, int k, const FixedSplit& fs, float l, int F, bool factor) {
    const long long t = fixed_mul(factor ? fixed_split(l) : fs, l, F);
    atomicAdd(reinterpret_cast<unsigned long long*>(&row[k]), (unsigned long long)t);
}

// Offset of cell (u, k) in a residual whose rows (u, u + il) are stored in
// interleaved pairs of 8-cell blocks (the annealer's layout for residuals it
// gathers from global memory; the same formula as its kernels use).
__device__ __forceinline__ long long resid_cell_at(int u, int k, int pitch, int il) {
    const int ls = il == 4 ? 2 : il == 2 ? 1 : 0;
    const long long pair = ((long long)(u >> (ls + 1)) << ls) + (u & (il - 1));
    return pair * 2 * pitch + (((u >> ls) & 1) << 3) + k + (k & ~7);
}

// Outputs of cell (u, k) of image item from its fixed-point sum; returns
// P_c - P_m (RESYNC, SIRT; else 0), whose square the row sums add with one
// rounding (an explicit fused multiply-add, the same in every path), and,
// for RESYNC, the drift.
__device__ __forceinline__ double cell_output(const ProjArgs& a, int item, int u, int k, long long raw, int F,
                                              float* drift) {
    const int B = a.B;
    const long long cell = (long long)u * B + k;
    const double val = ldexp((double)raw, -F);
    switch (a.mode) {
        case PROJ_FORWARD:
            a.out64[(long long)item * a.out_stride + cell] = val;
            return 0.0;
        case PROJ_FACTOR:
            a.out64[cell] = val;
            a.out32[cell] = (float)val;
            return 0.0;
        case PROJ_RESYNC: {
            const double r = val - (double)a.pm[(long long)item * a.pm_stride + cell];
            const float rf = (float)r;
            const int pitch = a.resid_pitch > 0 ? a.resid_pitch : B;
            // plain rows, or pairs of rows interleaved by 8-cell blocks (the
            // layout of the annealer's global-memory residuals)
            const long long at = a.resid_il ? resid_cell_at(u, k, pitch, a.resid_il) : (long long)u * pitch + k;
            float* dst = a.resid + (long long)item * a.resid_stride + at;
            if (a.drift) *drift = fabsf(rf - *dst);
            *dst = rf;
            return r;
        }
        default: {  // PROJ_SIRT
            const double r = val - (double)a.pm[(long long)item * a.pm_stride + cell];
            const float w = a.w[cell];
            a.resid[(long long)item * a.resid_stride + cell] = w > 0.0f ? (float)(-r / (double)w) : 0.0f;
            return r;
        }
    }
}

// A row's sum of squares and drift in a fixed order: lane partials over
// k = lane, lane + 32, ... ascending, then a butterfly; lane 0 stores them.
__device__ __forceinline__ void store_row_sums(const ProjArgs& a, int item, int u, double sq, float drift,
                                               int lane) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
        drift = fmaxf(drift, __shfl_xor_sync(0xffffffffu, drift, o));
    }
    if (lane == 0) {
        if (a.part_sq) a.part_sq[(long long)item * a.U + u] = sq;
        if (a.part_drift) a.part_drift[(long long)item * a.U + u] = drift;
    }
}

// Outputs of angle row u from its fixed-point sums src[0..B), one warp.
__device__ __forceinline__ void finish_row(const ProjArgs& a, int item, int u, int F, const long long* src,
                                           int lane) {
    double sq = 0.0;
    float drift = 0.0f;
    for (int k = lane; k < a.B; k += 32) {
        float d = 0.0f;
        const double r = cell_output(a, item, u, k, src[k], F, &d);
        sq = __fma_rn(r, r, sq);
        drift = fmaxf(drift, d);
    }
    store_row_sums(a, item, u, sq, drift, lane);
}

constexpr int kScaleParts = 32;  // blocks per image finding max|f| in chunked launches

__device__ __forceinline__ int fraction_bits_of_max(const ProjArgs& a, float m) {
    if (a.mode == PROJ_FACTOR) return fixed_point_bits(2.0 * (1.4142135623730951 * a.n + 2.0));
    return fixed_point_bits(1.5 * (double)m * (1.4142135623730951 * a.n + 2.0));
}

// Fraction bits of image item's sums, from a bound on |P| (every ray is at
// most sqrt(2)*n + 2 long).  All threads of the block must call it.
__device__ int item_fraction_bits(const ProjArgs& a, int item, float* red) {
    if (a.mode == PROJ_FACTOR) return fraction_bits_of_max(a, 0.0f);
    const float* img = a.img + (long long)item * a.img_stride;
    const long long P = (long long)a.n * a.n;
    float m = 0.0f;
    for (long long q = threadIdx.x; q < P; q += blockDim.x) m = fmaxf(m, fabsf(img[q]));
    return fraction_bits_of_max(a, block_max(m, red));
}

// The same bits from the kScaleParts partial maxima of a chunked launch
// (called by a whole warp).
__device__ __forceinline__ int item_fraction_bits_parts(const ProjArgs& a, int item, int lane) {
    float m = a.max_parts[(long long)item * kScaleParts + lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    return fraction_bits_of_max(a, m);
}

// Chunked launches: max|f| of each image in kScaleParts pieces.
__global__ void __launch_bounds__(kProjThreads) proj_scale_kernel(ProjArgs a) {
    __shared__ float red_f[kProjThreads];
    const int item = blockIdx.y, part = blockIdx.x;
    const long long P = (long long)a.n * a.n;
    const long long per = (P + kScaleParts - 1) / kScaleParts;
    const long long q0 = part * per, q1 = min(P, q0 + per);
    float m = 0.0f;
    if (a.mode != PROJ_FACTOR) {
        const float* img = a.img + (long long)item * a.img_stride;
        for (long long q = q0 + threadIdx.x; q < q1; q += kProjThreads) m = fmaxf(m, fabsf(img[q]));
    }
    m = block_max(m, red_f);
    if (threadIdx.x == 0) a.max_parts[(long long)item * kScaleParts + part] = m;
}

// One CTA per (group of 2^l angles, image, pixel chunk).  A warp takes
// 32 >> l pixels of the chunk at a time, one per lane slot (a slot's lanes
// are the group's angles); the slots walk far-apart parts of the chunk,
// starting at different columns, so that lanes of one angle rarely add to the
// same bin.  Four steps are loaded before any is added, to overlap their
// loads.  With one chunk the CTA finishes its rows itself; with several it
// adds its sums to the image's rows in acc_global (exact integer adds, so the
// order does not matter) and proj_finish_kernel finishes them.
__global__ void __launch_bounds__(kProjThreads) projector_kernel(ProjArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    long long* acc = reinterpret_cast<long long*>(smem_raw);
    __shared__ float red_f[kProjThreads];

    const int item = blockIdx.y, grp = blockIdx.x, chunk = blockIdx.z;
    const int u0 = grp * a.angles_per_group;
    const int A = min(a.angles_per_group, a.U - u0);
    const int B = a.B;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool factor = a.mode == PROJ_FACTOR;
    const float* img = a.img ? a.img + (long long)item * a.img_stride : nullptr;

    for (int e = tid; e < A * B; e += kProjThreads) acc[e] = 0;
    __shared__ int F_sh;
    if (a.chunks > 1) {
        if (warp == 0) {
            const int f = item_fraction_bits_parts(a, item, lane);
            if (lane == 0) F_sh = f;
        }
    } else {
        const int f = item_fraction_bits(a, item, red_f);
        if (tid == 0) F_sh = f;
    }
    __syncthreads();
    const int F = F_sh;

    // pixel indices fit in 32 bits (pila_build caps n * n at 2^30)
    const int Pi = a.n * a.n;
    const int per = (Pi + a.chunks - 1) / a.chunks;
    const int c0 = chunk * per, c1 = min(Pi, c0 + per);
    const int nwarps = kProjThreads / 32;
    const int la = a.lanes_log2;
    const int ps = lane >> la, ul = lane & ((1 << la) - 1);
    const int slots = 32 >> la;
    const int L = (c1 - c0 + slots - 1) / slots;  // pixels per slot
    const bool on = ul < A;
    const long long col = (long long)u0 + ul;
    long long* row = acc + ul * B;
    auto pixel_of = [&](int b) -> int {
        int off = b + 7 * ps;
        if (off >= L) off -= L;
        if (off >= L) off %= L;
        return c0 + ps * L + off;
    };
    constexpr int kSteps = 4;  // pixel steps loaded before their adds
    for (int b = warp; b < L; b += kSteps * nwarps) {
        float f[kSteps];
        Entry2 e[kSteps];
#pragma unroll
        for (int t = 0; t < kSteps; ++t) {
            const int bt = b + t * nwarps;
            const int q = bt < L ? pixel_of(bt) : c1;
            f[t] = 0.0f;
            e[t] = Entry2{0, 0, 0.0f, 0.0f};
            if (on && q < c1) {
                f[t] = factor ? (a.mask[q] ? 1.0f : 0.0f) : img[q];
                e[t] = decode_rec(a.table, (long long)q * a.row_records + col, a.f16);
            }
        }
#pragma unroll
        for (int t = 0; t < kSteps; ++t) {
            if (f[t] != 0.0f) {
                const FixedSplit st = fixed_split(f[t]);
                if (e[t].l0 != 0.0f) add_entry(row, e[t].k0, st, e[t].l0, F, factor);
                if (e[t].l1 != 0.0f) add_entry(row, e[t].k1, st, e[t].l1, F, factor);
            }
        }
    }
    __syncthreads();

    if (a.chunks == 1) {
        for (int r = warp; r < A; r += nwarps) finish_row(a, item, u0 + r, F, acc + r * B, lane);
    } else {
        // the chunk's sums, rows u0 .. u0 + A - 1 (contiguous), into its own slice
        long long* dst = a.partial + (((long long)item * a.chunks + chunk) * a.U + u0) * B;
        for (int e = tid; e < A * B; e += kProjThreads) dst[e] = acc[e];
    }
}

// Chunked launches, step 1: one thread per cell sums the chunks' slices
// (exact integer adds), writes the outputs, and leaves the cell's residual
// and drift in slice 0 and 1 of the cell (read by step 2 only).
__global__ void proj_finish_cells_kernel(ProjArgs a) {
    const int item = blockIdx.y;
    const long long cells = (long long)a.U * a.B;
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ int F_sh;
    if (threadIdx.x < 32) {  // the whole first warp, before any thread leaves
        const int f = item_fraction_bits_parts(a, item, threadIdx.x);
        if (threadIdx.x == 0) F_sh = f;
    }
    __syncthreads();
    if (cell >= cells) return;
    long long* src = a.partial + (long long)item * a.chunks * cells + cell;
    long long raw = 0;
    for (int c = 0; c < a.chunks; ++c) raw += src[c * cells];
    const int u = (int)(cell / a.B), k = (int)(cell - (long long)u * a.B);
    float drift = 0.0f;
    const double r = cell_output(a, item, u, k, raw, F_sh, &drift);
    src[0] = __double_as_longlong(r);
    src[cells] = (long long)__float_as_int(drift);
}

// Step 2: one warp per angle row, the row sums in the same fixed order as an
// unchunked launch.
constexpr int kFinishWarps = 4;
__global__ void __launch_bounds__(32 * kFinishWarps) proj_finish_rows_kernel(ProjArgs a) {
    const int item = blockIdx.y, lane = threadIdx.x & 31;
    const int u = blockIdx.x * kFinishWarps + (threadIdx.x >> 5);
    if (u >= a.U) return;
    const long long cells = (long long)a.U * a.B;
    const long long* src = a.partial + (long long)item * a.chunks * cells + (long long)u * a.B;
    double sq = 0.0;
    float drift = 0.0f;
    for (int k = lane; k < a.B; k += 32) {
        const double r = __longlong_as_double(src[k]);
        sq = __fma_rn(r, r, sq);
        drift = fmaxf(drift, __int_as_float((int)src[cells + k]));
    }
    store_row_sums(a, item, u, sq, drift, lane);
}

// ---- ray-driven projector ---------------------------------------------------
//
// With the table's ray-major index (rays.cu) a forward projection sums along
// rays, so each sum stays in a register: no shared accumulators, no atomics.
// The terms are the same exact fixed-point products as above (the fraction
// bits F of an image come from the same bound), and integer addition is
// associative, so every sum is bit-identical to the pixel-driven
// projector's.  The sums go to a workspace [item][U][B] and finish_rows_kernel
// forms the outputs and the per-angle sums of squares with finish_row, the
// function (and so the order) of the unchunked pixel-driven launch.
//
// Many images: a block of 4 warps takes 4 consecutive angles of one group of
// 32 images and 32 consecutive bins (the four warps' rays cross nearly the
// same pixels, so their image loads share L1 lines); lane = image.  The
// images are first transposed to [group][P][32], so that one pixel's values
// for the 32 images are one 128-byte line.  Few images: one warp per
// (image, ray), lanes over the ray's entries, a butterfly of the sums.

constexpr int kImageLanesMin = 24;  // images from which the image-lanes form runs
constexpr int kRowWarps = 4;        // angles per block of ray_rows_kernel
constexpr int kRowBins = 32;        // bins per block of ray_rows_kernel
constexpr int kRowUnroll = 16;      // index entries loaded before their terms

// 64-bit right shift by s, 0 for s >= 64 (PTX clamps the shift amount).
__device__ __forceinline__ unsigned long long shr_clamp(unsigned long long x, uint32_t s) {
    unsigned long long r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}

// fixed_mul(fixed_split(f), l, F) from the bits of f and l, with
// ebias = F - 300: the term's exponent is (max(ef, 1) - 150) + (el - 150) + F
// = max(ef, 1) + el + ebias.  Equal to fixed_mul: for
// e >= 0 the product shifted left, else rounded half away from zero; e <= 14
// always (every term is below 2^61 and a product of normal significands is
// at least 2^46), so (m << 15) >> (14 - e) = floor(m 2^(e+1)) never loses a
// high bit, and shifts of 64 or more give 0.
__device__ __forceinline__ long long fixed_term_bits(uint32_t bf, uint32_t bl, int ebias) {
    const uint32_t ef = (bf >> 23) & 0xffu;
    const uint32_t mf = (bf & 0x7fffffu) | (ef ? 0x800000u : 0u);
    const int e = (int)max(ef, 1u) + (int)((bl >> 23) & 0xffu) + ebias;
    const unsigned long long m = (unsigned long long)mf * (unsigned long long)((bl & 0x7fffffu) | 0x800000u);
    const unsigned long long t = shr_clamp(m << 15, (uint32_t)(14 - e));
    const unsigned long long v = (t + 1ull) >> 1;
    return (bf >> 31) ? -(long long)v : (long long)v;
}

__device__ __forceinline__ long long fixed_term(float f, float l, int F) {
    return fixed_term_bits(__float_as_uint(f), __float_as_uint(l), F - 300);
}

// The two forms above for a length in the ray index's packed form y = ml << 7
// | el (ml its 24-bit significand, el its biased exponent): the product of the
// significands comes out already shifted by 15, from (mf << 8) * (ml << 7).
__device__ __forceinline__ long long fixed_term_packed(uint32_t bf, uint32_t y, int ebias) {
    const uint32_t ef = (bf >> 23) & 0xffu;
    const uint32_t mf8 = ((bf << 8) & 0x7fffff00u) | (ef ? 0x80000000u : 0u);
    const int e = (int)max(ef, 1u) + (int)(y & 0x7fu) + ebias;
    const unsigned long long t = shr_clamp((unsigned long long)mf8 * (unsigned long long)(y & ~0x7fu), (uint32_t)(14 - e));
    const unsigned long long v = (t + 1ull) >> 1;
    return (bf >> 31) ? -(long long)v : (long long)v;
}

// The same term for a non-negative image value (its sign bit clear) of an
// image whose F is at most 124: the hidden bit is set even for a zero or
// subnormal f (ef = 0), but its exponent ef + el + ebias is then at most
// 127 + 124 - 300 = -49 (l < 2), and a product below 2^48 times 2^-49 rounds
// to 0, which is what the exact form gives for such f.
__device__ __forceinline__ long long fixed_term_nonneg_packed(uint32_t bf, uint32_t y, int ebias) {
    const int e = (int)(bf >> 23) + (int)(y & 0x7fu) + ebias;
    const unsigned long long t =
        shr_clamp((unsigned long long)((bf << 8) | 0x80000000u) * (unsigned long long)(y & ~0x7fu), (uint32_t)(14 - e));
    return (long long)((t + 1ull) >> 1);
}

// float32 length of a packed index entry
__device__ __forceinline__ float packed_length(uint32_t y) {
    return __uint_as_float(((y >> 7) & 0x7fffffu) | ((y & 0x7fu) << 23));
}

// T[g][p][lane] = image (32 g + lane) at pixel p (-0 as +0: the same term),
// 0 past the last image; neg_group[g] = 1 if the group holds a negative value.
__global__ void transpose_images_kernel(const ProjArgs a, int n_items, long long P) {
    __shared__ float tile[32][33];
    const int g = blockIdx.y;
    const long long p0 = (long long)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    bool neg = false;
    for (int r = ty; r < 32; r += 8) {
        const int item = g * 32 + r;
        const long long p = p0 + tx;
        const float v = (item < n_items && p < P) ? __fadd_rn(a.img[(long long)item * a.img_stride + p], 0.0f) : 0.0f;
        neg = neg || v < 0.0f;
        tile[r][tx] = v;
    }
    if (__syncthreads_or(neg) && tx == 0 && ty == 0) atomicOr(&a.neg_group[g], 1);
    for (int r = ty; r < 32; r += 8) {
        const long long p = p0 + r;
        if (p < P) a.timg[((long long)g * P + p) * 32 + tx] = tile[tx][r];
    }
}

// The warp's rays: bins k0 .. k1-1 of angle row `off`, lane = image.
template <bool NONNEG>
__device__ __forceinline__ void ray_rows_sum(const ProjArgs& a, const float* T, const uint32_t* off, int k0, int k1,
                                             int ebias, long long* out, bool live) {
    uint32_t e1 = off[k0];
    for (int k = k0; k < k1; ++k) {
        uint32_t e = e1;
        e1 = off[k + 1];
        long long acc = 0;
        for (; e + kRowUnroll <= e1; e += kRowUnroll) {
            uint2 en[kRowUnroll];
            uint32_t f[kRowUnroll];
#pragma unroll
            for (int j = 0; j < kRowUnroll; ++j) en[j] = a.ray_ent[e + j];
#pragma unroll
            for (int j = 0; j < kRowUnroll; ++j) f[j] = __float_as_uint(T[(long long)en[j].x * 32]);
#pragma unroll
            for (int j = 0; j < kRowUnroll; ++j)
                acc += NONNEG ? fixed_term_nonneg_packed(f[j], en[j].y, ebias) : fixed_term_packed(f[j], en[j].y, ebias);
        }
        for (; e < e1; ++e) {
            const uint2 en = a.ray_ent[e];
            const uint32_t f = __float_as_uint(T[(long long)en.x * 32]);
            acc += NONNEG ? fixed_term_nonneg_packed(f, en.y, ebias) : fixed_term_packed(f, en.y, ebias);
        }
        if (live) out[k] = acc;
    }
}

// Block (group g, bin chunk c, angle quad q), g slowest so that the blocks
// running at once share one group's transposed images in L2; warp w takes
// angle 4q + w, bins 32c .. 32c + 31, lane = image.
__global__ void __launch_bounds__(32 * kRowWarps) ray_rows_kernel(const ProjArgs a, int n_items, int quads,
                                                                  int chunks) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long blk = blockIdx.x;
    const int g = (int)(blk / ((long long)chunks * quads));
    const int rem = (int)(blk - (long long)g * chunks * quads);
    const int c = rem / quads, u = (rem - c * quads) * kRowWarps + warp;
    if (u >= a.U) return;
    const int item = g * 32 + lane;
    float m = 0.0f;
    if (item < n_items)
        for (int q = 0; q < kScaleParts; ++q) m = fmaxf(m, a.max_parts[(long long)item * kScaleParts + q]);
    const int F = fraction_bits_of_max(a, m);
    const int ebias = F - 300;  // the lane's image's F, as fixed_term folds it
    const long long P = (long long)a.n * a.n;
    const float* T = a.timg + (long long)g * P * 32 + lane;
    const uint32_t* off = a.ray_off + (long long)u * a.B;
    long long* out = a.partial + ((long long)item * a.U + u) * a.B;
    const int k0 = c * kRowBins, k1 = min(a.B, k0 + kRowBins);
    const bool live = item < n_items;
    // the short form needs every lane's image free of negative values and F <= 124
    if (__all_sync(0xffffffffu, F <= 124) && a.neg_group[g] == 0)
        ray_rows_sum<true>(a, T, off, k0, k1, ebias, out, live);
    else
        ray_rows_sum<false>(a, T, off, k0, k1, ebias, out, live);
}

// One warp per (image, ray), image-major; lanes over the ray's entries.
__global__ void __launch_bounds__(256) ray_cells_kernel(const ProjArgs a, int n_items) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long rays = (long long)a.U * a.B;
    if (w >= rays * n_items) return;
    const int item = (int)(w / rays);
    const long long ray = w - (long long)item * rays;
    const int F = item_fraction_bits_parts(a, item, lane);
    const bool factor = a.mode == PROJ_FACTOR;
    const float* img = factor ? nullptr : a.img + (long long)item * a.img_stride;
    long long acc = 0;
    const uint32_t e1 = a.ray_off[ray + 1];
    for (uint32_t e = a.ray_off[ray] + lane; e < e1; e += 32) {
        const uint2 en = a.ray_ent[e];
        const float l = packed_length(en.y);
        const float f = factor ? (a.mask[en.x] ? l : 0.0f) : img[en.x];
        acc += fixed_term(f, l, F);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) a.partial[(long long)item * rays + ray] = acc;
}

// One warp per (image, angle row): outputs and row sums from the sums.
constexpr int kRowsPerBlock = 4;
__global__ void __launch_bounds__(32 * kRowsPerBlock) finish_rows_kernel(const ProjArgs a, int n_items) {
    const int item = blockIdx.y, lane = threadIdx.x & 31;
    const int u = blockIdx.x * kRowsPerBlock + (threadIdx.x >> 5);
    if (u >= a.U || item >= n_items) return;
    const int F = item_fraction_bits_parts(a, item, lane);
    finish_row(a, item, u, F, a.partial + ((long long)item * a.U + u) * a.B, lane);
}

// One warp per item: lane partials over u = lane, lane + 32, ... in order,
// then a butterfly (a fixed order).
__global__ void reduce_kernel(ReduceArgs a) {
    const int item = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (item >= a.n_items) return;
    double s = 0.0;
    float d = 0.0f;
    for (int u = lane; u < a.n_rows; u += 32) {
        s += a.part_sq[(long long)item * a.n_rows + u];
        if (a.part_drift) d = fmaxf(d, a.part_drift[(long long)item * a.n_rows + u]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
    }
    if (lane != 0) return;
    if (a.S_out) a.S_out[item] = s;
    if (a.cost_out) a.cost_out[(long long)item * a.cost_stride] = sqrt(s * a.inv_cells);
    if (a.drift_max && a.part_drift) a.drift_max[item] = fmax(a.drift_max[item], (double)d);
}

}  // namespace

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int projector_smem_bytes(int angles_per_group, int B) { return angles_per_group * B * (int)sizeof(long long); }

int projector_max_bins() { return kProjSmemBudget / (int)sizeof(long long); }

int projector_plan(int U, int B, int n, long long n_items, bool can_chunk, int* angles_per_group, int* n_groups,
                   int* lanes_log2, int* chunks) {
    int amax = kProjSmemBudget / (B * (int)sizeof(long long));
    if (amax < 1) return SATPILA_ERR_INVALID_ARG;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
    const long long target = 2LL * sms;  // CTAs wanted
    int l = 4;
    while ((1 << l) > amax) --l;
    long long G = (U + (1 << l) - 1) >> l;
    *chunks = 1;
    if (n_items * G < target) {
        const long long P = (long long)n * n;
        if (can_chunk && P / 1024 >= 2) {
            // split the pixels: chunks of at least 1024 pixels, several CTAs per SM
            const long long want = 4 * target;
            *chunks = (int)std::max(2LL, std::min((want + n_items * G - 1) / (n_items * G), P / 1024));
        } else {
            // narrower groups: the widest that still gives enough CTAs
            while (l > 0 && n_items * ((U + (1 << l) - 1) >> l) < target) --l;
            G = (U + (1 << l) - 1) >> l;
        }
    }
    *angles_per_group = 1 << l;
    *n_groups = (int)G;
    *lanes_log2 = l;
    return SATPILA_OK;
}

size_t projector_ws_bytes(long long n_items, int U, int B, int n) {
    int A = 0, G = 0, l = 0, chunks = 1;
    if (projector_plan(U, B, n, n_items, true, &A, &G, &l, &chunks) != SATPILA_OK || chunks <= 1) return 0;
    return round_up((size_t)n_items * chunks * U * B * sizeof(long long), 256) +
           round_up((size_t)n_items * kScaleParts * sizeof(float), 256);
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

// [item][U][B] sums, the transposed images and a flag per group (many
// images), the max|f| parts.
size_t ray_ws_bytes(long long n_items, int U, int B, int n) {
    const long long P = (long long)n * n, cells = (long long)U * B;
    const long long groups = (n_items + 31) / 32;
    const size_t timg = n_items >= kImageLanesMin ? (size_t)groups * P * 32 * sizeof(float) : 0;
    return round_up((size_t)n_items * cells * sizeof(long long), 256) + round_up(timg, 256) +
           round_up((size_t)n_items * kScaleParts * sizeof(float), 256) + round_up((size_t)groups * sizeof(int), 256);
}

// SATPILA_PROJECTOR=pixel in the environment selects the pixel-driven
// projector wherever the ray-driven one could run (to compare the two).
bool projector_forced_pixel() {
    const char* v = std::getenv("SATPILA_PROJECTOR");
    return v && std::strcmp(v, "pixel") == 0;
}

void use_ray_projector(ProjArgs& a, const satpila_pila* p, void* ws) {
    a.ray_off = p->d_ray_off;
    a.ray_ent = p->d_ray_ent;
    a.ray_ws = p->d_ray_off ? ws : nullptr;
}

namespace {

cudaError_t launch_ray_projector(ProjArgs& a, int n_items, cudaStream_t s) {
    const long long P = (long long)a.n * a.n, cells = (long long)a.U * a.B;
    const bool lanes_are_images = n_items >= kImageLanesMin;
    const size_t sums = round_up((size_t)n_items * cells * sizeof(long long), 256);
    const size_t timg = lanes_are_images ? round_up((size_t)((n_items + 31) / 32) * P * 32 * sizeof(float), 256) : 0;
    char* ws = static_cast<char*>(a.ray_ws);
    const int groups = (n_items + 31) / 32;
    a.partial = reinterpret_cast<long long*>(ws);
    a.timg = reinterpret_cast<float*>(ws + sums);
    a.max_parts = reinterpret_cast<float*>(ws + sums + timg);
    a.neg_group = reinterpret_cast<int*>(ws + sums + timg + round_up((size_t)n_items * kScaleParts * sizeof(float), 256));
    cudaError_t e;
    proj_scale_kernel<<<dim3(kScaleParts, n_items), kProjThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (lanes_are_images) {
        if ((e = cudaMemsetAsync(a.neg_group, 0, (size_t)groups * sizeof(int), s)) != cudaSuccess) return e;
        transpose_images_kernel<<<dim3((unsigned)((P + 31) / 32), groups), dim3(32, 8), 0, s>>>(a, n_items, P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int quads = (a.U + kRowWarps - 1) / kRowWarps, chunks = (a.B + kRowBins - 1) / kRowBins;
        const long long blocks = (long long)groups * chunks * quads;
        ray_rows_kernel<<<(unsigned)blocks, 32 * kRowWarps, 0, s>>>(a, n_items, quads, chunks);
    } else {
        const long long warps = cells * n_items;
        ray_cells_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(a, n_items);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    finish_rows_kernel<<<dim3((a.U + kRowsPerBlock - 1) / kRowsPerBlock, n_items), 32 * kRowsPerBlock, 0, s>>>(
        a, n_items);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_projector(ProjArgs& a, int n_items, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    if (a.ray_off && a.ray_ent && a.ray_ws && !projector_forced_pixel()) return launch_ray_projector(a, n_items, s);
    if (projector_plan(a.U, a.B, a.n, n_items, a.ws != nullptr, &a.angles_per_group, &a.n_groups, &a.lanes_log2,
                       &a.chunks) != SATPILA_OK)
        return cudaErrorInvalidValue;
    a.partial = nullptr;
    a.max_parts = nullptr;
    if (a.chunks > 1) {
        a.partial = reinterpret_cast<long long*>(a.ws);
        a.max_parts = reinterpret_cast<float*>(reinterpret_cast<char*>(a.ws) +
                                               round_up((size_t)n_items * a.chunks * a.U * a.B * sizeof(long long), 256));
    }
    const int smem = projector_smem_bytes(a.angles_per_group, a.B);
    cudaError_t e = prepare_projector();
    if (e != cudaSuccess) return e;
    if (a.chunks > 1) {
        proj_scale_kernel<<<dim3(kScaleParts, n_items), kProjThreads, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    projector_kernel<<<dim3(a.n_groups, n_items, a.chunks), kProjThreads, smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.chunks > 1) {
        const long long cells = (long long)a.U * a.B;
        proj_finish_cells_kernel<<<dim3((unsigned)((cells + 255) / 256), n_items), 256, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        proj_finish_rows_kernel<<<dim3((a.U + kFinishWarps - 1) / kFinishWarps, n_items), 32 * kFinishWarps, 0, s>>>(a);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t s) {
    if (a.n_items <= 0) return cudaSuccess;
    reduce_kernel<<<(unsigned)((a.n_items + 3) / 4), 128, 0, s>>>(a);
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
    if (p->B > projector_max_bins()) return fail(SATPILA_ERR_INVALID_ARG, "too many bins for the projector");
    a.mode = PROJ_FACTOR;
    a.mask = p->d_mask;
    a.out64 = p->d_w64;
    a.out32 = p->d_w32;
    void* ws = nullptr;
    if (p->d_ray_off) SP_CUDA(cudaMallocAsync(&ws, ray_ws_bytes(1, p->U, p->B, p->n), s));
    use_ray_projector(a, p, ws);
    cudaError_t e = launch_projector(a, 1, s);
    if (ws) {
        const cudaError_t ef = cudaFreeAsync(ws, s);
        if (e == cudaSuccess) e = ef;
    }
    SP_CUDA(e);
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
    if (p->B > projector_max_bins()) return fail(SATPILA_ERR_INVALID_ARG, "pila_forward: too many bins");
    a.mode = PROJ_FORWARD;
    a.img = di;
    a.img_stride = P;
    a.out64 = dout;
    a.out_stride = cells;
    cudaError_t e = cudaSuccess;
    void* ws = nullptr;
    int A = 0, G = 0, l = 0, chunks = 1;
    if (p->d_ray_off && !projector_forced_pixel()) {
        // the ray-driven projector's workspace, stream-ordered
        e = cudaMallocAsync(&ws, ray_ws_bytes(n_images, p->U, p->B, p->n), s);
        use_ray_projector(a, p, ws);
    } else if (projector_plan(p->U, p->B, p->n, n_images, true, &A, &G, &l, &chunks) == SATPILA_OK && chunks > 1) {
        // few images: a stream-ordered workspace lets their pixels spread over more CTAs
        e = cudaMallocAsync(&ws, projector_ws_bytes(n_images, p->U, p->B, p->n), s);
        a.ws = ws;
    }
    if (e == cudaSuccess) e = launch_projector(a, n_images, s);
    if (ws) {
        const cudaError_t ef = cudaFreeAsync(ws, s);
        if (e == cudaSuccess) e = ef;
    }
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
