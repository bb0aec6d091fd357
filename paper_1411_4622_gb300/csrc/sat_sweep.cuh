// The annealing move of Secs. II-A/II-B/III-B on sm_103a.
//
// A group of W warps runs one chain; a chain is strictly sequential (move
// m+1 sees move m's update).  Within a move the 32*W lanes split the
// projection angles: each lane owns a fixed set of angles for the whole run,
// so every residual cell is only ever read and written by one thread and no
// atomics are needed.
//
// Per move m (Step 2 -> Step 4):
//   * pixel and estimates come from Philox4x32-10, key = seed + chain,
//     counter (stage, move, block, 1): draw 0 picks the pixel, draw 1 is the
//     acceptance number N1, draw 2+e the value of estimate e (Eq. (3) read as
//     the uniform law on [max(0, f-beta), min(beta, f+beta)]);
//   * each lane copies its own 16-byte chunks of the pixel's PILA row
//     (Eq. (5)) into shared memory with cp.async, D-1 moves ahead (pixel
//     choice does not depend on the chain's state);
//   * the Eq. (7) sum of every estimate is dS = df * (2g + df*h) with
//     g = sum r*l over the residual r = P_c - P_m and h = sum l^2 (a per-pixel
//     constant of the table); the best estimate (BoME) is the smallest dS,
//     lowest index on ties;
//   * Step 4 compares x = dS/(B*U) with T L (2C + T L), L = -ln N1, which is
//     N1 < exp(-(C' - C)/T) rearranged;
//   * on acceptance each lane applies Eq. (6) to its own residual cells.
// The chain's only loop-carried dependence is kept to a few instructions:
// move m+1's g is split as Gs + df(m) * OV, where Gs sums the residual as
// gathered before move m's update and OV sums the products of the two moves'
// lengths on shared cells; both are reduced across the group while move m is
// still being decided.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace satpila {

// Per-chain control of a batch whose chains are at different points of their
// own schedules (the serving engine); sat_run passes none and uses the
// batch-wide values.
struct ChainCtl {
    unsigned long long seed;  // Philox key of the chain
    double t0, tn;            // as in sat_params (t0 <= 0: Eq. (8); tn < 0: T0 / 1000)
    int stage0;               // stages the chain ran before this launch
    int n_sweeps;             // length of the chain's schedule
    int schedule;             // SAT_SCHED_*
    int t0_samples;           // Q of Eq. (8)
};

struct SatArgs {
    const unsigned char* table;  // PILA records [P][row_records]
    long long row_stride;        // bytes between pixel rows
    int row_chunks;              // 16-byte chunks per row
    const float* hsum;           // [P] sum of squared stored lengths of each pixel
    int n, U, B;
    int pitch;                   // residual row pitch (B + 1 rounded up to 4: a private pad cell per row)
    int band_lo;                 // windowed kernel, shared-memory residual: first bin kept (multiple of 4)
    int band_pitch;              //   bins kept per row (multiple of 4)
    long long band_floats;       //   U * band_pitch cells, then 2 dummy cells per lane
    const int32_t* list;         // reconstruction-space pixels (NULL: identity)
    int n_list;
    int moves;                   // M moves per stage
    int K;                       // estimates per move
    float beta;
    float inv_BU;
    double inv_BU_d;
    int D;                       // PILA rows in flight (3..kMaxStages)
    int W;                       // warps per chain (1, 2 or 4)
    int stage_bytes;             // bytes of one stage buffer
    int group_smem_bytes;        // shared memory per chain group (per shared-memory warp in the hybrid kernel)
    int hybrid_smem_warps;       // hybrid kernel: warps with a shared-memory residual
    int hybrid_glob_bytes;       // hybrid kernel: shared memory of each global-residual warp
    long long resid_floats;      // per-chain residual stride (floats, multiple of 4)
    int n_chains;
    float* resid;                // [n_chains][resid_floats]
    float* img;                  // [n_chains][img_stride]
    long long img_stride;
    double* S;                   // [n_chains] running sum of squared residuals
    const double* T0;            // [n_chains]
    const double* TN;            // [n_chains]
    unsigned long long seed;
    unsigned long long* accepted;  // [n_chains]
    int* progress;               // [n_chains] next stage to run
    int schedule, n_sweeps_total;
    int sweep_begin, sweep_end, sweeps_per_task, n_tasks;
    int* task_counter;
    int* error;
    double* sweep_cost;          // [n_chains][n_sweeps_total] or NULL
    sat_trace_rec* trace;
    int trace_chain;
    long long trace_cap;
    const ChainCtl* ctl;         // [n_chains] or NULL
    int* claim;                  // windowed kernels: [n_chains] 1 while a warp runs the chain, or NULL
    unsigned long long wait_ns;  // bound on a wait for a chain's earlier stages (and for a chain to claim)
    unsigned* ties;              // [n_chains] near-tie decisions (windowed kernels built to count them)
    int stall_chain;             // test hook: this chain's first task is never reported done (-1: none)
    int resid_il;                // 0: plain residual rows; 1, 2, 4: rows u and u + resid_il interleaved (resid_row_base)
    // A launch over chains of several tables (the serving engine's classes):
    // the per-class arguments (table, geometry, move rules and the class's
    // chain arrays), and for each chain of the launch its class and its index
    // there.  The launch's own fields then hold the task queue, the progress
    // flags (indexed by the launch's chain number), the error word and the
    // shared-memory layout.  NULL: one table.
    const SatArgs* classes;
    const int2* chain_map;       // [n_chains]
};

// Residual rows in global memory are stored plainly (cell (u, k) at
// u * pitch + k) or, for layouts that gather their cells from global memory,
// in pairs of rows (u, u + s) interleaved by 8-cell (32-byte) blocks:
// [row u, cells 8b..8b+7][row u + s, cells 8b..8b+7] for b = 0, 1, ... (pitch
// a multiple of 8).  A DRAM access fetches 64 bytes, so a cell's access also
// brings the same bins of an angle s steps away, which the same move mostly
// needs (a pixel's bin moves by about one bin per angle step).  s is the
// number of records per 16-byte chunk of the table (1 FP32, 2 FP16, 4 one-byte):
// the lanes of one warp instruction then hold the two rows of a pair in
// neighbouring lanes, so both halves of the 64 bytes travel in one request.
// Cell (u, k) sits at resid_row_base(u) + k + (k & ~7) in that layout.
__host__ __device__ __forceinline__ int resid_row_base(int u, int pitch, int il) {
    if (!il) return u * pitch;
    const int ls = il == 4 ? 2 : il == 2 ? 1 : 0;  // log2 of the pair stride s
    const int pair = ((u >> (ls + 1)) << ls) + (u & (il - 1));
    return pair * 2 * pitch + (((u >> ls) & 1) << 3);
}
__host__ __device__ __forceinline__ int resid_cell(int row_base, int k, int il) {
    return row_base + k + (il ? (k & ~7) : 0);
}
// First cell after the rows (the lanes' dummy cells follow).
__host__ __device__ __forceinline__ int resid_rows_end(int U, int pitch, int il) {
    return il ? (U + 2 * il - 1) / (2 * il) * (2 * il) * pitch : U * pitch;
}

// True unless the task just run is the stalled chain's first (test hook).
__device__ __forceinline__ bool report_progress(const SatArgs& a, int c, int s0) {
    return !(c == a.stall_chain && s0 == a.sweep_begin);
}

constexpr int kSatMaxWarps = 8;
constexpr int kMaxGroupWarps = 4;
constexpr int kBatch = 8;       // moves per block of random draws (per-move pipelined kernel)
constexpr int kDrawRing = 3 * kBatch;  // the batch in use, the next one, and one being drawn
// Windowed kernels: 16 moves per block when a move takes at most two Philox
// blocks (K <= 4), so that one warp-wide pass fills every lane; 8 otherwise.
// Their ring holds 4 blocks (a power of two, so that a move's slot is one
// AND): the block in use, the next one, one being drawn, one spare.
__host__ __device__ constexpr int batch_moves(int kmax) { return kmax <= 4 ? 32 : 8; }
__host__ __device__ constexpr int ring_slots(int kmax) { return 4 * batch_moves(kmax); }
// Bytes of one warp's draw ring for kmax estimates: the pixel of each slot,
// then the draw words of each slot (a multiple of 16 bytes; room for the
// windowed kernels' ring, which the pipelined kernel's fits in).
__host__ __device__ constexpr int draw_ring_bytes(int kmax) {
    return ring_slots(kmax) * (4 * ((kmax + 2 + 3) / 4) + 1) * 4;
}
// Shared memory of a chain group: header, one draw ring per warp, then the
// PILA-row stages and (when resident) the residual.
constexpr int kPartSlots = 8;   // window sums a warp of a group publishes per window (windowed kernel)
constexpr int kPartOffset = 64;  // GroupShared::part: [2][kMaxGroupWarps][kPartSlots] floats
constexpr int kFlagsOffset = kPartOffset + 2 * kMaxGroupWarps * kPartSlots * 4;  // GroupShared::flags: 8 ints
constexpr int kGroupHeader = kFlagsOffset + 64;
__host__ __device__ constexpr int group_ring_bytes(int W, int kmax) { return kGroupHeader + W * draw_ring_bytes(kmax); }

__device__ __forceinline__ double stage_temperature(int schedule, double t0, double tn, int s, int n_sweeps) {
    const double N = (double)n_sweeps, n = (double)s;
    if (schedule == SAT_SCHED_GEOMETRIC) return t0 <= 0.0 ? 0.0 : t0 * pow(tn / t0, n / N);
    if (schedule == SAT_SCHED_CUBIC) return t0 - n * n * n * (t0 - tn) / (N * N * N);
    return t0 - n * (t0 - tn) / N;
}

// Lane-owned decoded records of one move.  Entry 1 always sits on bin k + 1
// (the builder stores consecutive bins), so only bin 0 is kept.
template <int JMAX>
struct Recs {
    int k[JMAX];
    float l0[JMAX], l1[JMAX];
};

template <bool F16, int JMAX>
__host__ __device__ constexpr int chunks_per_lane() { return F16 ? JMAX / 2 : JMAX; }

// Record index of slot j of group lane gl (= lane + 32 * warp-in-group).
template <bool F16>
__device__ __forceinline__ int record_of(int gl, int W, int j) {
    return F16 ? 2 * (gl + 32 * W * (j / 2)) + (j & 1) : gl + 32 * W * j;
}

template <bool F16, int JMAX>
__device__ __forceinline__ void decode_stage(const unsigned char* stage, int gl, int W, Recs<JMAX>& r) {
    const uint4* q4 = reinterpret_cast<const uint4*>(stage);
    if constexpr (F16) {
#pragma unroll
        for (int i = 0; i < JMAX / 2; ++i) {
            const uint4 v = q4[gl + 32 * W * i];
            const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
            const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.w));
            r.k[2 * i] = (int)(v.x & 0xffffu);
            r.l0[2 * i] = a.x;
            r.l1[2 * i] = a.y;
            r.k[2 * i + 1] = (int)(v.z & 0xffffu);
            r.l0[2 * i + 1] = b.x;
            r.l1[2 * i + 1] = b.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < JMAX; ++i) {
            const uint4 v = q4[gl + 32 * W * i];
            r.k[i] = (int)v.x;
            r.l0[i] = __uint_as_float(v.z);
            r.l1[i] = __uint_as_float(v.w);
        }
    }
}

// Record-type-generic forms (RT = PILA_F32, PILA_F16 or PILA_U8): records per
// 16-byte chunk, the lane's chunks, the record of a lane slot, decoding.
template <int RT>
__host__ __device__ constexpr int recs_per_chunk() { return RT == PILA_U8 ? 4 : RT == PILA_F16 ? 2 : 1; }

template <int RT, int JMAX>
__host__ __device__ constexpr int rt_chunks_per_lane() { return JMAX / recs_per_chunk<RT>(); }

template <int RT>
__device__ __forceinline__ int rt_record_of(int gl, int W, int j) {
    constexpr int r = recs_per_chunk<RT>();
    return r * (gl + 32 * W * (j / r)) + (j % r);
}

template <int RT, int JMAX>
__device__ __forceinline__ void rt_decode_stage(const unsigned char* stage, int gl, int W, Recs<JMAX>& r) {
    if constexpr (RT == PILA_U8) {
        const uint4* q4 = reinterpret_cast<const uint4*>(stage);
#pragma unroll
        for (int i = 0; i < JMAX / 4; ++i) {
            const uint4 v = q4[gl + 32 * W * i];
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                r.k[4 * i + q] = (int)(w[q] & 0xffffu);
                r.l0[4 * i + q] = (float)((w[q] >> 16) & 0xffu) * kU8Unit;
                r.l1[4 * i + q] = (float)(w[q] >> 24) * kU8Unit;
            }
        }
    } else {
        decode_stage<RT == PILA_F16, JMAX>(stage, gl, W, r);
    }
}

struct GroupShared {
    uint64_t* bar;         // one barrier: the residual's bulk copy at task start
    float* part;           // partial window sums per parity (pipelined: [2][kMaxGroupWarps][4]; windowed:
                           // [2][kMaxGroupWarps][kPartSlots])
    volatile int* flags;   // [0] task, [2] progress-wait result
    uint32_t* draws;       // this warp's ring [kDrawRing][4 * blocks]: raw Philox words
    int* pix;              // this warp's ring [kDrawRing]: pixel of each move
    unsigned char* stages;
};

// Named barrier of the chain group (ids 1.. ; id 0 is the CTA barrier).
__device__ __forceinline__ void group_sync(int id, int W) {
    if (W == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(32 * W) : "memory");
    }
}

__device__ __forceinline__ void cp_async_16_pred(bool pred, void* smem_dst, const void* src) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %0, 0;\n\t"
        "@p cp.async.cg.shared.global [%1], [%2], 16;\n\t}" ::"r"((uint32_t)pred),
        "r"(smem_u32(smem_dst)), "l"(src)
        : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Waits until at most n of this thread's copy groups are still pending.
__device__ __forceinline__ void cp_async_wait_pending(int n) {
    switch (n) {
        case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    }
}

// The lane's chunks of a pixel's row into a stage (one copy group).
template <bool F16, int JMAX>
__device__ __forceinline__ void fetch_row(const SatArgs& a, unsigned char* stage, int p, int gl, int W) {
    const unsigned char* row = a.table + (long long)p * a.row_stride;
#pragma unroll
    for (int i = 0; i < chunks_per_lane<F16, JMAX>(); ++i) {
        const int q = gl + 32 * W * i;
        cp_async_16_pred(q < a.row_chunks, stage + 16 * q, row + 16 * (q < a.row_chunks ? q : 0));
    }
    cp_async_commit();
}

template <int KMAX>
__host__ __device__ constexpr int draw_words() { return 4 * ((KMAX + 2 + 3) / 4); }

// Random draws of moves [first, first + kBatch) of stage s into this warp's
// ring: one warp-wide Philox pass per 32 (move, block) units, raw words
// stored as they come.  Draw d = 4*block + word: d = 0 the pixel, d = 1 the
// acceptance number N1, d = 2 + e the uniform of estimate e.  A pixel of a
// masked reconstruction space is looked up in the pixel list; `late` keeps
// that lookup in a register (stored by settle_pixels a few moves later) so
// the load latency stays off the move loop.
struct PendingPixel {
    int slot[3];  // ring slots, or -1 (a lane draws at most one pixel per pass, three passes)
    int value[3];
};

template <int KMAX, int BATCH = kBatch, int RING = kDrawRing>
__device__ __forceinline__ void draw_batch(const SatArgs& a, const GroupShared& G, int s, int first, uint2 key,
                                           int lane, bool late, PendingPixel& pend) {
    constexpr int kWords = draw_words<KMAX>();
    // Philox blocks per move: for the build's estimate capacity when it is at
    // most 8 (a compile-time count, so the unit's move and block come by shifts;
    // blocks past the call's K are drawn and never read, and a pass costs the
    // same with them), else for the call's K.
    const int nblk = KMAX <= 8 ? (KMAX + 2 + 3) / 4 : (a.K + 2 + 3) / 4;
    const int units = BATCH * nblk;  // <= 72 (16 x 2 or 8 x 9 at most)
    const uint32_t nl = (uint32_t)a.n_list;
#pragma unroll
    for (int it = 0; it < 3; ++it) {
        pend.slot[it] = -1;
        const int u0 = 32 * it;
        if (u0 >= units) continue;
        const int unit = u0 + lane;
        const int mv = first + unit / nblk, blk = unit % nblk;
        const uint4 x = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)mv, (uint32_t)blk, kStreamSat), key);
        const bool live = unit < units && mv < a.moves;
        const int slot = (RING & (RING - 1)) == 0 ? (mv & (RING - 1)) : mv % RING;
        // Stored ready for the move: word 0 raw (the pixel), word 1 as
        // L = -ln N1 of Step 4, the others as the uniforms of the estimates.
        const float w0 = unit_uniform(x.x), w1 = unit_uniform(x.y);
        const float w2 = unit_uniform(x.z), w3 = unit_uniform(x.w);
        const uint4 y = make_uint4(blk == 0 ? x.x : __float_as_uint(w0),
                                   __float_as_uint(blk == 0 ? -__logf(w1) : w1), __float_as_uint(w2),
                                   __float_as_uint(w3));
        if (live) *reinterpret_cast<uint4*>(G.draws + slot * kWords + 4 * blk) = y;
        if (live && blk == 0) {
            const uint32_t idx = pick_index(x.x, nl);
            const int p = a.list ? __ldg(a.list + idx) : (int)idx;
            if (late) {
                pend.slot[it] = slot;
                pend.value[it] = p;
            } else {
                G.pix[slot] = p;
            }
        }
    }
}

__device__ __forceinline__ void settle_pixels(const GroupShared& G, PendingPixel& pend) {
#pragma unroll
    for (int it = 0; it < 3; ++it) {
        if (pend.slot[it] >= 0) G.pix[pend.slot[it]] = pend.value[it];
        pend.slot[it] = -1;
    }
}

// Residual values at a move's two entry cells per record.  Every cell index
// is valid: an empty entry names a cell of its own row (its length 0 keeps
// it out of every sum), a record past U names a lane-private dummy cell
// after the residual.  So loads and stores need no predicate.
template <int JMAX>
__device__ __forceinline__ void gather(const float* R, const int (&rowbase)[JMAX], const Recs<JMAX>& r,
                                       float (&v0)[JMAX], float (&v1)[JMAX], int il) {
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        v0[j] = R[resid_cell(rowbase[j], r.k[j], il)];
        v1[j] = R[resid_cell(rowbase[j], r.k[j] + 1, il)];
    }
}

struct StageCtx {
    int s, M, D, W, wig, lane, gid, gl;
    int il;   // the residual R is in global memory with interleaved row pairs (their stride), or 0
    float T;
    float* R;
    float* img;
    uint2 key;
    bool tracing;
};

// Registers of one move, prepared one move ahead.
template <int JMAX>
struct Ahead {
    Recs<JMAX> r;               // its records
    float v0[JMAX], v1[JMAX];   // residual at its cells, gathered before the previous move's update
    float s0[JMAX], s1[JMAX];   // length of the previous move's entry on the same cell (0 if none)
    float Gs, OV, h;            // sum v*l and sum s*l over the group; sum l^2 of the pixel
    int p;                      // its pixel
    float f;                    // its value as loaded (before the previous move's write)
};

struct ChainRegs {
    float S_hi, S_lo;  // Kahan-compensated sum of squared residuals
    float C;           // current cost
    unsigned long long n_acc;
    float df_prev;     // value change applied by the previous move (0 if rejected)
    int p_prev;        // pixel of the previous move
    float f_prev;      // its value after the previous move
};

// Loads of move mn's registers (records, stale residual, pixel value and
// sum of squares); the sums follow in finish_prepare.
template <bool F16, int JMAX>
__device__ __forceinline__ void start_prepare(const SatArgs& a, const GroupShared& G, const StageCtx& x,
                                              const int (&rowbase)[JMAX], const unsigned char* stage, int mn,
                                              Ahead<JMAX>& n) {
    n.p = G.pix[mn % kDrawRing];
    n.f = __ldcg(x.img + n.p);  // L2: never a line another store of this chain left stale in L1
    n.h = __ldg(a.hsum + n.p);
    decode_stage<F16, JMAX>(stage, x.gl, x.W, n.r);
    gather<JMAX>(x.R, rowbase, n.r, n.v0, n.v1, x.il);
}

// Partial sums of move n relative to the previous move's records `prev`,
// reduced over the warp (the group's warps combine them afterwards).
template <int JMAX>
__device__ __forceinline__ void finish_prepare(const Recs<JMAX>* prev, Ahead<JMAX>& n) {
    float gs0 = 0.0f, gs1 = 0.0f, ov = 0.0f;
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        if (prev) {
            const int d = n.r.k[j] - prev->k[j];
            n.s0[j] = d == 0 ? prev->l0[j] : (d == 1 ? prev->l1[j] : 0.0f);
            n.s1[j] = d == 0 ? prev->l1[j] : (d == -1 ? prev->l0[j] : 0.0f);
        } else {
            n.s0[j] = n.s1[j] = 0.0f;
        }
        gs0 = fmaf(n.v0[j], n.r.l0[j], gs0);
        gs1 = fmaf(n.v1[j], n.r.l1[j], gs1);
        ov = fmaf(n.s0[j], n.r.l0[j], ov);
        ov = fmaf(n.s1[j], n.r.l1[j], ov);
    }
    float gs = gs0 + gs1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gs += __shfl_xor_sync(0xffffffffu, gs, o);
        ov += __shfl_xor_sync(0xffffffffu, ov, o);
    }
    n.Gs = gs;
    n.OV = ov;
}

// Combines the warps' sums of a group (fixed order: identical in every warp).
__device__ __forceinline__ void group_combine(const GroupShared& G, const StageCtx& x, int parity, float& gs,
                                              float& ov) {
    float* part = G.part + parity * (4 * kMaxGroupWarps);
    if (x.lane == 0) {
        part[4 * x.wig] = gs;
        part[4 * x.wig + 1] = ov;
    }
    group_sync(x.gid, x.W);
    gs = part[0];
    ov = part[1];
    for (int w = 1; w < x.W; ++w) {
        gs += part[4 * w];
        ov += part[4 * w + 1];
    }
}

// Decides move m (Steps 2-4 with BoME) from its prepared registers `cur`,
// prepares move m+1 into `nxt`, then applies Eq. (6) for move m.
template <bool F16, int JMAX, int KMAX, bool HAS_NEXT>
__device__ __forceinline__ void move_step(const SatArgs& a, const GroupShared& G, const StageCtx& x, int m,
                                          ChainRegs& cr, const int (&rowbase)[JMAX], PendingPixel& pend,
                                          Ahead<JMAX>& cur, Ahead<JMAX>& nxt) {
    constexpr int kWords = draw_words<KMAX>();
    const int D = x.D, M = x.M;
    __syncwarp();
    // Moves [m-kBatch, m) are done: their draw slots take moves [m+2*kBatch, m+3*kBatch).
    // Their pixels are stored half a batch later, before any of them is used
    // (the first row fetch of that batch is at least 2*kBatch - D + 1 moves away).
    if ((m & (kBatch - 1)) == 0 && m + 2 * kBatch < M)
        draw_batch<KMAX>(a, G, x.s, m + 2 * kBatch, x.key, x.lane, true, pend);
    if ((m & (kBatch - 1)) == kBatch / 2) settle_pixels(G, pend);
    if (HAS_NEXT) cp_async_wait_pending(D - 3);  // this lane's chunks of move m+1 have landed

    // ---- loads for move m+1 and the draws of move m (independent of the decision) ----
    const unsigned char* st_next = G.stages + (size_t)((m + 1) % D) * a.stage_bytes;
    if (HAS_NEXT) start_prepare<F16, JMAX>(a, G, x, rowbase, st_next, m + 1, nxt);
    const uint32_t* drw = G.draws + (m % kDrawRing) * kWords;
    uint32_t raw[KMAX + 2];
#pragma unroll
    for (int q = 0; q < KMAX + 2; q += 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(drw + q);
        raw[q] = v.x;
        if (q + 1 < KMAX + 2) raw[q + 1] = v.y;
        if (q + 2 < KMAX + 2) raw[q + 2] = v.z;
        if (q + 3 < KMAX + 2) raw[q + 3] = v.w;
    }

    // ---- decision of move m: g = Gs + df(m-1) * OV is the loop-carried step ----
    const float L = __uint_as_float(raw[1]);
    const float g = fmaf(cr.df_prev, cur.OV, cur.Gs);
    const float f = cur.p == cr.p_prev ? cr.f_prev : cur.f;
    const float TL = x.T * L;
    const float theta = TL * fmaf(2.0f, cr.C, TL);
    const float lo = fmaxf(0.0f, f - a.beta), span = fminf(a.beta, f + a.beta) - lo;
    const float g2 = 2.0f * g;
    float dS[KMAX], fc[KMAX];
    int ci[KMAX];
#pragma unroll
    for (int e = 0; e < KMAX; ++e) {
        fc[e] = fmaf(__uint_as_float(raw[2 + e]), span, lo);
        const float df = fc[e] - f;
        dS[e] = e < a.K ? df * fmaf(df, cur.h, g2) : __int_as_float(0x7f800000);
        ci[e] = e;
    }
#pragma unroll
    for (int width = 1; width < KMAX; width *= 2) {
#pragma unroll
        for (int e = 0; e + width < KMAX; e += 2 * width) {
            const bool take = dS[e + width] < dS[e];
            dS[e] = take ? dS[e + width] : dS[e];
            fc[e] = take ? fc[e + width] : fc[e];
            ci[e] = take ? ci[e + width] : ci[e];
        }
    }
    const float best_dS = dS[0], best_f = fc[0];
    const float xs = best_dS * a.inv_BU;
    const bool accept = xs <= 0.0f || xs < theta;
    const float df = accept ? best_f - f : 0.0f;

    // ---- sums of move m+1 (shuffles overlap the decision above) ----
    if (HAS_NEXT) {
        finish_prepare<JMAX>(&cur.r, nxt);
        if (x.W > 1) group_combine(G, x, m & 1, nxt.Gs, nxt.OV);
    }

    // ---- Eq. (6) for move m on the lane's own cells ----
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        const float v0 = fmaf(cr.df_prev, cur.s0[j], cur.v0[j]);  // the previous move's update
        const float v1 = fmaf(cr.df_prev, cur.s1[j], cur.v1[j]);
        x.R[resid_cell(rowbase[j], cur.r.k[j], x.il)] = fmaf(df, cur.r.l0[j], v0);  // unchanged when rejected or empty
        x.R[resid_cell(rowbase[j], cur.r.k[j] + 1, x.il)] = fmaf(df, cur.r.l1[j], v1);
    }
    const float fnew = accept ? best_f : f;
    __stcg(x.img + cur.p, fnew);  // every warp of the group writes the same value
    // Kahan-compensated running sum of squared residuals, and the cost.
    const float y = (accept ? best_dS : 0.0f) - cr.S_lo;
    const float t = cr.S_hi + y;
    cr.S_lo = (t - cr.S_hi) - y;
    cr.S_hi = t;
    const float C2 = fmaxf(0.0f, cr.S_hi * a.inv_BU);
    const float C_before = cr.C;
    cr.C = accept ? (C2 > 0.0f ? C2 * rsqrtf(C2) : 0.0f) : cr.C;
    cr.n_acc += accept ? 1ull : 0ull;
    cr.df_prev = df;
    cr.p_prev = cur.p;
    cr.f_prev = fnew;

    // Row of move m+D-1 into the stage that move m-1 used (empty group past the end).
    const int mi = m + D - 1;
    const int pi = mi < M ? G.pix[mi % kDrawRing] : 0;
    if (mi < M) {
        fetch_row<F16, JMAX>(a, G.stages + (size_t)(mi % D) * a.stage_bytes, pi, x.gl, x.W);
    } else {
        cp_async_commit();
    }
    if (mi < M && x.lane == 31) prefetch_l1(a.hsum + pi);

    if (x.tracing && x.wig == 0 && x.lane == 0) {
        const float Cp = sqrtf(fmaxf(0.0f, fmaf(C_before, C_before, xs)));
        const float den = Cp + C_before;
        const long long idx = (long long)x.s * M + m;
        if (idx < a.trace_cap) {
            sat_trace_rec r;
            r.pixel = cur.p;
            r.cstar = ci[0];
            r.accepted = accept ? 1 : 0;
            r.pad = 0;
            r.dS = best_dS;
            r.dC = den > 0.0f ? xs / den : 0.0f;
            r.fnew = fnew;
            r.pad2 = 0.0f;
            a.trace[idx] = r;
        }
    }
}

// One temperature stage of one chain.
template <bool F16, int JMAX, int KMAX>
__device__ __forceinline__ void run_stage(const SatArgs& a, const GroupShared& G, const StageCtx& x, float& S_hi,
                                          float& S_lo, unsigned long long& n_acc, const int (&rowbase)[JMAX]) {
    const int M = x.M, D = x.D;
    if (M <= 0 || a.n_list <= 0) return;

    // Prologue: draws of the first two batches, rows of moves 0..D-2 in flight.
    PendingPixel pend;
    draw_batch<KMAX>(a, G, x.s, 0, x.key, x.lane, false, pend);
    draw_batch<KMAX>(a, G, x.s, kBatch, x.key, x.lane, false, pend);  // leaves pend empty
    __syncwarp();
    for (int j = 0; j < D - 1; ++j) {
        if (j < M) fetch_row<F16, JMAX>(a, G.stages + (size_t)j * a.stage_bytes, G.pix[j % kDrawRing], x.gl, x.W);
        else cp_async_commit();
    }
    cp_async_wait_pending(D - 2);  // move 0 has landed

    Ahead<JMAX> A, B;
    start_prepare<F16, JMAX>(a, G, x, rowbase, G.stages, 0, A);
    finish_prepare<JMAX>(nullptr, A);
    if (x.W > 1) {
        group_combine(G, x, 1, A.Gs, A.OV);
        group_sync(x.gid, x.W);  // the parity-1 slots are reused by move 1
    }
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        B.r.k[j] = 0;
        B.r.l0[j] = B.r.l1[j] = B.v0[j] = B.v1[j] = B.s0[j] = B.s1[j] = 0.0f;
    }
    B.Gs = B.OV = B.h = B.f = 0.0f;
    B.p = 0;
    ChainRegs cr;
    cr.S_hi = S_hi;
    cr.S_lo = S_lo;
    cr.C = sqrtf(fmaxf(0.0f, S_hi * a.inv_BU));
    cr.n_acc = n_acc;
    cr.df_prev = 0.0f;
    cr.p_prev = -1;
    cr.f_prev = 0.0f;
    int m = 0;
    // Two moves per trip: the register sets alternate roles, no copies.
    for (; m + 2 < M; m += 2) {
        move_step<F16, JMAX, KMAX, true>(a, G, x, m, cr, rowbase, pend, A, B);
        move_step<F16, JMAX, KMAX, true>(a, G, x, m + 1, cr, rowbase, pend, B, A);
    }
    if (m + 1 < M) {
        move_step<F16, JMAX, KMAX, true>(a, G, x, m, cr, rowbase, pend, A, B);
        move_step<F16, JMAX, KMAX, false>(a, G, x, m + 1, cr, rowbase, pend, B, A);
    } else if (m < M) {
        move_step<F16, JMAX, KMAX, false>(a, G, x, m, cr, rowbase, pend, A, B);
    }
    cp_async_wait_pending(0);  // nothing left in flight
    S_hi = cr.S_hi;
    S_lo = cr.S_lo;
    n_acc = cr.n_acc;
}

// Waits until another group has finished the chain's earlier stages (at
// most limit_ns of wall time).
static __device__ __forceinline__ bool wait_progress(const int* flag, int target, unsigned long long limit_ns) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (ld_acquire(flag) >= target) return true;
        if (global_ns() - t0 > limit_ns) return false;
        __nanosleep(256);
    }
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Task loop of one chain group (W warps; grp numbers the group in its CTA,
// gb is its shared memory).
template <bool F16, bool SMEM, int JMAX, int KMAX>
__device__ __forceinline__ void pipeline_group(const SatArgs& a, unsigned char* gb, int grp, int W, int wig,
                                               int lane) {
    GroupShared G;
    G.bar = reinterpret_cast<uint64_t*>(gb);
    G.part = reinterpret_cast<float*>(gb + kPartOffset);  // the pipelined kernel uses 2 * 4 * 4 of its floats
    G.flags = reinterpret_cast<volatile int*>(gb + kFlagsOffset);
    G.pix = reinterpret_cast<int*>(gb + kGroupHeader + wig * draw_ring_bytes(KMAX));
    G.draws = reinterpret_cast<uint32_t*>(gb + kGroupHeader + wig * draw_ring_bytes(KMAX) + kDrawRing * 4);
    G.stages = gb + group_ring_bytes(W, KMAX);
    float* rs = reinterpret_cast<float*>(G.stages + (size_t)a.D * a.stage_bytes);
    const int gid = 1 + grp;
    const int gl = lane + 32 * wig;  // lane index within the group

    // Stage chunks past a row stay zero (length 0 = no contribution).
    for (int e = gl; e < a.D * a.stage_bytes / 16; e += 32 * W)
        reinterpret_cast<uint4*>(G.stages)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (gl == 0) {
        mbar_init(G.bar, 1);
        for (int i = 0; i < 8; ++i) G.flags[i] = 0;
    }
    fence_proxy_async_smem();
    if (gl == 0) fence_barrier_init();
    group_sync(gid, W);

    // Residual row offsets of the lane's angles; records past U use the
    // lane's two dummy cells after the residual rows.
    const int il = SMEM ? 0 : a.resid_il;
    int rowbase[JMAX];
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        const int u = record_of<F16>(gl, W, j);
        rowbase[j] = u < a.U ? resid_row_base(u, a.pitch, il) : resid_rows_end(a.U, a.pitch, il) + 2 * gl;
    }

    uint32_t phase = 0;
    for (;;) {
        if (gl == 0) G.flags[0] = atomicAdd(a.task_counter, 1);
        group_sync(gid, W);
        const int t = G.flags[0];
        group_sync(gid, W);
        if (t >= a.n_tasks) break;
        const int c = t % a.n_chains;
        const int blk = t / a.n_chains;
        const int s0 = a.sweep_begin + blk * a.sweeps_per_task;
        const int s1 = min(s0 + a.sweeps_per_task, a.sweep_end);
        if (blk > 0) {
            if (gl == 0) G.flags[2] = wait_progress(&a.progress[c], s0, a.wait_ns) ? 1 : 0;
            group_sync(gid, W);
            const int ok = G.flags[2];
            group_sync(gid, W);
            if (!ok) {
                if (gl == 0) raise_error(a.error, SATPILA_ERR_TIMEOUT);
                break;
            }
        }
        float* gres = a.resid + (long long)c * a.resid_floats;
        float* R = SMEM ? rs : gres;
        if (SMEM) {
            // Residual into shared memory with one bulk copy (TMA).
            int ok = 1;
            if (gl == 0) {
                fence_proxy_async_global();  // written by generic stores of an earlier task
                mbar_arrive_expect_tx(G.bar, (uint32_t)(a.resid_floats * 4));
                bulk_copy_g2s(rs, gres, (uint32_t)(a.resid_floats * 4), G.bar);
                ok = mbar_wait_bounded(G.bar, phase) ? 1 : 0;
                G.flags[2] = ok;
            }
            group_sync(gid, W);
            ok = G.flags[2];
            group_sync(gid, W);
            if (!ok) {
                if (gl == 0) raise_error(a.error, SATPILA_ERR_TIMEOUT);
                break;
            }
            // every group lane observes the completed phase before reading
            mbar_wait_bounded(G.bar, phase);
            phase ^= 1u;
        }
        const double S = a.S[c];
        float S_hi = (float)S;
        float S_lo = -(float)(S - (double)S_hi);  // Kahan carries the negated remainder
        unsigned long long n_acc = 0;
        StageCtx x;
        x.M = a.moves;
        x.D = a.D;
        x.W = W;
        x.wig = wig;
        x.lane = lane;
        x.gid = gid;
        x.gl = gl;
        x.il = il;
        x.R = R;
        x.img = a.img + (long long)c * a.img_stride;
        const ChainCtl* cc = a.ctl ? a.ctl + c : nullptr;
        const int s_base = cc ? cc->stage0 : 0, s_total = cc ? cc->n_sweeps : a.n_sweeps_total;
        const int sched = cc ? cc->schedule : a.schedule;
        x.key = chain_key(cc ? cc->seed : a.seed + (unsigned long long)c);
        x.tracing = a.trace != nullptr && c == a.trace_chain;
        const double T0 = a.T0[c], TN = a.TN[c];
        for (int s = s0; s < s1 && s_base + s < s_total; ++s) {
            x.s = s_base + s;
            x.T = (float)stage_temperature(sched, T0, TN, x.s, s_total);
            run_stage<F16, JMAX, KMAX>(a, G, x, S_hi, S_lo, n_acc, rowbase);
            if (a.sweep_cost && gl == 0)
                a.sweep_cost[(long long)c * a.n_sweeps_total + s] = sqrt(((double)S_hi - (double)S_lo) * a.inv_BU_d);
        }
        group_sync(gid, W);
        if (SMEM) {
            const float4* src = reinterpret_cast<const float4*>(rs);
            float4* dst = reinterpret_cast<float4*>(gres);
            for (long long e = gl; e < a.resid_floats / 4; e += 32 * W) dst[e] = src[e];
        }
        if (gl == 0) {
            a.S[c] = (double)S_hi - (double)S_lo;
            a.accepted[c] += n_acc;
        }
        __threadfence();
        group_sync(gid, W);
        if (gl == 0 && report_progress(a, c, s0)) st_release(&a.progress[c], s1);
    }
}

template <bool F16, bool SMEM, int JMAX, int KMAX>
__global__ void __launch_bounds__(kSatMaxWarps * 32) sat_sweep_kernel(const SatArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = a.W;
    const int grp = warp / W;
    pipeline_group<F16, SMEM, JMAX, KMAX>(a, smem + (size_t)grp * a.group_smem_bytes, grp, W, warp % W, lane);
}

// ---- Eq. (8): initial temperature ------------------------------------------

struct T0Args {
    const unsigned char* table;
    long long row_stride;
    int f16;  // table precision (PILA_F32, PILA_F16, PILA_U8)
    int n, U, B;
    int pitch;
    int resid_il;  // residual rows in interleaved pairs (their stride; resid_row_base), or 0
    const int32_t* list;
    int n_list;
    float beta;
    float inv_BU;
    double inv_BU_d;
    const float* resid;
    long long resid_floats;
    const float* img;
    long long img_stride;
    const double* S;
    unsigned long long seed;
    int Q;
    double tn;     // < 0: T0 / 1000
    double t0_fixed;  // > 0: use it instead of Eq. (8)
    double* T0;
    double* TN;
    int* found;
    const ChainCtl* ctl;  // [chains] or NULL
};

}  // namespace satpila
