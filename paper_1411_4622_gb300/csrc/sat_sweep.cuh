// The annealing move of Secs. II-A/II-B/III-B on sm_103a.
//
// One warp runs one chain; a chain is strictly sequential (move m+1 sees
// move m's update).  Within a move the 32 lanes split the projection angles:
// lane l owns a fixed set of angles for the whole run, so every residual cell
// is only ever read and written by one thread and no atomics or barriers are
// needed inside a chain.
//
// Per move m (Step 2 -> Step 4):
//   * pixel and estimates come from Philox4x32-10, key = seed + chain,
//     counter (stage, move, block, 1): draw 0 picks the pixel, draw 1 is the
//     acceptance number N1, draw 2+e the value of estimate e (Eq. (3) read as
//     the uniform law on [max(0, f-beta), min(beta, f+beta)]);
//   * the pixel's PILA row (Eq. (5)) is fetched by a 1-D bulk copy
//     (cp.async.bulk + mbarrier) into a per-warp ring of D stages, issued
//     D-1 moves ahead (pixel choice does not depend on the chain's state);
//   * lanes gather the residual r = P_c - P_m at their entries' bins and form
//     g = sum r*l and h = sum l^2 (warp-shuffle butterfly); every estimate's
//     Eq. (7) sum is then dS = df * (2g + df*h), and the best one (BoME)
//     is the smallest dS, lowest index on ties;
//   * dC = (dS/(B*U)) / (C' + C) (Eq. (7) rearranged to avoid cancelling
//     square roots); Metropolis test of Step 4 at the stage temperature;
//   * on acceptance each lane applies Eq. (6) to its own residual cells.
// The residual of move m+1 is gathered while move m is being decided and is
// patched in registers where move m's update touched the same cell.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace satpila {

struct SatArgs {
    const unsigned char* table;  // PILA records [P][row_records]
    long long row_stride;        // bytes between pixel rows
    int copy_bytes;              // bytes fetched per move (multiple of 16)
    int n, U, B;
    int pitch;                   // residual row pitch (B + 1: a private pad cell per row)
    const int32_t* list;         // reconstruction-space pixels (NULL: identity)
    int n_list;
    int moves;                   // M moves per stage
    int K;                       // estimates per move
    float beta;
    float inv_BU;
    double inv_BU_d;
    int J;                       // records per lane in use (<= JMAX)
    int D;                       // prefetch stages (2..kMaxStages)
    int stage_bytes;             // bytes of one stage buffer
    int warp_smem_bytes;         // shared memory per warp
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
};

constexpr int kSatMaxWarps = 8;
// Per-warp shared memory header: barriers, stage pixels, the draw ring.
constexpr int kRingHeader = 128 + 2 * 8 * (32 + 4) * 4;

__device__ __forceinline__ double stage_temperature(int schedule, double t0, double tn, int s, int n_sweeps) {
    const double N = (double)n_sweeps, n = (double)s;
    if (schedule == SAT_SCHED_GEOMETRIC) return t0 <= 0.0 ? 0.0 : t0 * pow(tn / t0, n / N);
    if (schedule == SAT_SCHED_CUBIC) return t0 - n * n * n * (t0 - tn) / (N * N * N);
    return t0 - n * (t0 - tn) / N;
}

constexpr int kBatch = 8;       // moves per block of random draws
constexpr int kDrawRing = 2 * kBatch;

// Lane-owned decoded records of one move.  Entry 1 always sits on bin k + 1
// (the builder stores consecutive bins), so only bin 0 is kept.
template <int JMAX>
struct Recs {
    int k[JMAX];
    float l0[JMAX], l1[JMAX];
};

template <bool F16, int JMAX>
__device__ __forceinline__ void decode_stage(const unsigned char* stage, int lane, int J, Recs<JMAX>& r) {
    const uint4* q4 = reinterpret_cast<const uint4*>(stage);
    if constexpr (F16) {
#pragma unroll
        for (int i = 0; i < JMAX / 2; ++i) {
            if (2 * i < J) {
                const uint4 v = q4[lane + 32 * i];
                const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
                const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.w));
                r.k[2 * i] = (int)(v.x & 0xffffu);
                r.l0[2 * i] = a.x;
                r.l1[2 * i] = a.y;
                r.k[2 * i + 1] = (int)(v.z & 0xffffu);
                r.l0[2 * i + 1] = b.x;
                r.l1[2 * i + 1] = b.y;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < JMAX; ++i) {
            if (i < J) {
                const uint4 v = q4[lane + 32 * i];
                r.k[i] = (int)v.x;
                r.l0[i] = __uint_as_float(v.z);
                r.l1[i] = __uint_as_float(v.w);
            }
        }
    }
}

struct WarpRing {
    uint64_t* bar;       // [kMaxStages]
    int* pix;            // [kMaxStages] pixel of the move held by each stage
    float* draws;        // [kDrawRing][draw_stride]: pixel, L = -ln N1, pad, pad, u_0..u_{K-1}
    unsigned char* stages;
};

// Waits (bounded) for the copies still in flight after a failure.
static __device__ __noinline__ void drain_stages(const WarpRing& w, int D, int first_move, int last_move,
                                                 uint32_t& phase) {
    for (int mv = first_move; mv <= last_move; ++mv) {
        const int st = mv % D;
        mbar_wait_bounded(&w.bar[st], (phase >> st) & 1u);
        phase ^= 1u << st;
    }
}

__device__ __forceinline__ void cp_async_4(void* smem_dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem_dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Random draws of moves [first, first + kBatch) of stage s: one warp-wide
// Philox pass per 32 (move, block) units.  Draw d = 4*block + word: d = 0 the
// pixel, d = 1 the acceptance number N1 (stored as L = -ln N1), d = 2 + e the
// uniform of estimate e.  Pixels of a masked reconstruction space are copied
// from the pixel list asynchronously.
template <int KMAX>
__device__ __forceinline__ void draw_batch(const SatArgs& a, const WarpRing& w, int s, int first, uint2 key,
                                           int lane) {
    constexpr int kStride = KMAX + 4;
    const int nblk = (a.K + 2 + 3) / 4;
    const int units = kBatch * nblk;
    const uint32_t nl = (uint32_t)a.n_list;
    for (int u0 = 0; u0 < units; u0 += 32) {
        const int unit = u0 + lane;
        const int mv = first + unit / nblk, blk = unit % nblk;
        const uint4 x = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)mv, (uint32_t)blk, kStreamSat), key);
        if (unit < units && mv < a.moves) {
            float* rec = w.draws + (mv % kDrawRing) * kStride;
            const uint32_t wd[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int d = 4 * blk + i;
                if (d == 0) {
                    const uint32_t idx = pick_index(wd[0], nl);
                    if (a.list) cp_async_4(rec, a.list + idx);
                    else reinterpret_cast<int*>(rec)[0] = (int)idx;
                } else if (d == 1) {
                    rec[1] = -logf(unit_uniform(wd[1]));
                } else if (d - 2 < a.K) {
                    rec[4 + d - 2] = unit_uniform(wd[i]);
                }
            }
        }
    }
}

// Issue of a pixel row into a stage by one lane of the warp (the predicate),
// without a branch: barrier arrival with the expected bytes, then the copy.
__device__ __forceinline__ void issue_row_pred(bool pred, uint64_t* bar, void* dst, const void* src,
                                               uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %0, 0;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%1], %4;\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%2], [%3], %4, [%1];\n\t}" ::"r"(
            (uint32_t)pred),
        "r"(smem_u32(bar)), "r"(smem_u32(dst)), "l"(src), "r"(bytes)
        : "memory");
}

// Residual values at a move's two entry cells per record.  Every cell index
// is valid: an empty entry names a real cell of its row (and its length 0
// keeps it out of every sum), a record past U names a lane-private dummy
// cell after the residual.  So loads and stores need no predicate.
template <int JMAX>
__device__ __forceinline__ void gather(const float* R, const int (&rowbase)[JMAX], const Recs<JMAX>& r,
                                       float (&v0)[JMAX], float (&v1)[JMAX]) {
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        const float* q = R + rowbase[j] + r.k[j];
        v0[j] = q[0];
        v1[j] = q[1];
    }
}

struct MoveState {
    int p;       // pixel of the move
    float f;     // its value as loaded
    bool fwd;    // the previous move wrote this pixel: use fwd_f instead
    float fwd_f;
};

// One move (Steps 2-4 with BoME) whose records/values are (cur, rv), while
// the next move's (nxt, nv) are gathered.  has_next = false for the last move.
template <bool F16, int JMAX, int KMAX, bool HAS_NEXT>
__device__ __forceinline__ bool move_step(const SatArgs& a, const WarpRing& w, int s, int m, int M, float T, float* R,
                                          float* img, uint2 key, uint32_t& phase, float& S_hi, float& S_lo,
                                          float& C, unsigned long long& n_acc, int lane, const int (&rowbase)[JMAX],
                                          int& st_cur, int& issued, bool tracing, const Recs<JMAX>& cur,
                                          const float (&rv0)[JMAX], const float (&rv1)[JMAX], Recs<JMAX>& nxt,
                                          float (&nv0)[JMAX], float (&nv1)[JMAX], MoveState& ms) {
    constexpr int kStride = KMAX + 4;
    const int D = a.D;
    const int st_next = st_cur + 1 == D ? 0 : st_cur + 1;
    const int st_issue = st_cur == 0 ? D - 1 : st_cur - 1;
    __syncwarp();
    // Moves [m-kBatch, m) are done: their draw slots take moves [m+kBatch, m+2*kBatch).
    if ((m & (kBatch - 1)) == 0 && m > 0 && m + kBatch < M) draw_batch<KMAX>(a, w, s, m + kBatch, key, lane);
    const int mi = m + D - 1;
    if (mi < M) {
        if (a.list && (mi & (kBatch - 1)) == 0) {
            cp_async_wait_all();  // pixels of the batch that starts at mi
            __syncwarp();
        }
        const int pi = reinterpret_cast<const int*>(w.draws + (mi % kDrawRing) * kStride)[0];
        if (lane == 31) w.pix[st_issue] = pi;
        issue_row_pred(lane == 31, &w.bar[st_issue], w.stages + (size_t)st_issue * a.stage_bytes,
                       a.table + (long long)pi * a.row_stride, (uint32_t)a.copy_bytes);
        if (lane == 31) prefetch_l1(img + pi);
        issued = mi;
    }
    // Draws of this move (independent of the chain state).
    const float* drec = w.draws + (m % kDrawRing) * kStride;
    const float L = drec[1];
    float uc[KMAX];
#pragma unroll
    for (int q = 0; q < KMAX; q += 4) {
        const float4 v = *reinterpret_cast<const float4*>(drec + 4 + q);
        uc[q] = v.x;
        if (q + 1 < KMAX) uc[q + 1] = v.y;
        if (q + 2 < KMAX) uc[q + 2] = v.z;
        if (q + 3 < KMAX) uc[q + 3] = v.w;
    }
    // Partial sums of this move.
    float g0 = 0.0f, g1 = 0.0f, h0 = 0.0f, h1 = 0.0f;
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        g0 = fmaf(rv0[j], cur.l0[j], g0);
        g1 = fmaf(rv1[j], cur.l1[j], g1);
        h0 = fmaf(cur.l0[j], cur.l0[j], h0);
        h1 = fmaf(cur.l1[j], cur.l1[j], h1);
    }
    float g = g0 + g1, h = h0 + h1;
    // Gather of the next move while this one is reduced and decided.
    int p1 = 0;
    float f1 = 0.0f;
    if (HAS_NEXT) {
        if (!mbar_wait_bounded(&w.bar[st_next], (phase >> st_next) & 1u)) {
            raise_error(a.error, SATPILA_ERR_TIMEOUT);
            drain_stages(w, D, m + 1, issued, phase);
            return false;
        }
        phase ^= 1u << st_next;
        p1 = w.pix[st_next];
        f1 = img[p1];
        decode_stage<F16, JMAX>(w.stages + (size_t)st_next * a.stage_bytes, lane, JMAX, nxt);
        gather<JMAX>(R, rowbase, nxt, nv0, nv1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        g += __shfl_xor_sync(0xffffffffu, g, o);
        h += __shfl_xor_sync(0xffffffffu, h, o);
    }
    // Step 4 threshold: with L = -ln N1, N1 < exp(-dC/T) <=> dC < T L
    // <=> x < T L (2C + T L) for x = dS / (B U) (dC = sqrt(C^2 + x) - C).
    const float TL = T * L;
    const float theta = TL * fmaf(2.0f, C, TL);
    // BoME: every lane evaluates every estimate; smallest dS, lowest index on ties.
    const float f = ms.fwd ? ms.fwd_f : ms.f;
    const float lo = fmaxf(0.0f, f - a.beta), span = fminf(a.beta, f + a.beta) - lo;
    const float g2 = 2.0f * g;
    float dS[KMAX], fc[KMAX];
    int ci[KMAX];
#pragma unroll
    for (int e = 0; e < KMAX; ++e) {
        fc[e] = fmaf(uc[e], span, lo);
        const float df = fc[e] - f;
        dS[e] = e < a.K ? df * fmaf(df, h, g2) : __int_as_float(0x7f800000);
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
    const float x = best_dS * a.inv_BU;
    const bool accept = x <= 0.0f || x < theta;
    const float df = accept ? best_f - f : 0.0f;
    if (tracing && lane == 0) {
        const float Cp = sqrtf(fmaxf(0.0f, fmaf(C, C, x)));
        const float den = Cp + C;
        const long long idx = (long long)s * M + m;
        if (idx < a.trace_cap) {
            sat_trace_rec r;
            r.pixel = ms.p;
            r.cstar = ci[0];
            r.accepted = accept ? 1 : 0;
            r.pad = 0;
            r.dS = best_dS;
            r.dC = den > 0.0f ? x / den : 0.0f;
            r.fnew = accept ? best_f : f;
            r.pad2 = 0.0f;
            a.trace[idx] = r;
        }
    }
    // Eq. (6) on the lane's own residual cells, and the same update on the
    // already gathered values of the next move where the cells coincide.
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        float* q = R + rowbase[j] + cur.k[j];
        q[0] = fmaf(df, cur.l0[j], rv0[j]);  // unchanged value when rejected or empty
        q[1] = fmaf(df, cur.l1[j], rv1[j]);
        if (HAS_NEXT) {
            const int d = nxt.k[j] - cur.k[j];
            const float s0 = d == 0 ? cur.l0[j] : (d == 1 ? cur.l1[j] : 0.0f);
            const float s1 = d == 0 ? cur.l1[j] : (d == -1 ? cur.l0[j] : 0.0f);
            nv0[j] = fmaf(df, s0, nv0[j]);
            nv1[j] = fmaf(df, s1, nv1[j]);
        }
    }
    img[ms.p] = accept ? best_f : f;
    if (HAS_NEXT) {
        ms.fwd = p1 == ms.p;  // the value written just above
        ms.fwd_f = accept ? best_f : f;
        ms.f = f1;
        ms.p = p1;
    }
    // Kahan-compensated running sum of squared residuals.
    const float y = (accept ? best_dS : 0.0f) - S_lo;
    const float t = S_hi + y;
    S_lo = (t - S_hi) - y;
    S_hi = t;
    const float C2 = fmaxf(0.0f, S_hi * a.inv_BU);
    C = accept ? (C2 > 0.0f ? C2 * rsqrtf(C2) : 0.0f) : C;
    n_acc += accept ? 1ull : 0ull;
    st_cur = st_next;
    return true;
}

// One temperature stage of one chain.  Returns false if a bounded wait gave up.
template <bool F16, bool SMEM, int JMAX, int KMAX>
__device__ __forceinline__ bool run_stage(const SatArgs& a, const WarpRing& w, int c, int s, float T, float* R,
                                          float* img, uint2 key, uint32_t& phase, float& S_hi, float& S_lo,
                                          unsigned long long& n_acc, int lane, const int (&rowbase)[JMAX]) {
    constexpr int kStride = KMAX + 4;
    const int M = a.moves, D = a.D;
    if (M <= 0 || a.n_list <= 0) return true;

    // Prologue: draws of the first two batches, rows of moves 0..D-2 in flight.
    draw_batch<KMAX>(a, w, s, 0, key, lane);
    draw_batch<KMAX>(a, w, s, kBatch, key, lane);
    cp_async_wait_all();
    __syncwarp();
    const int pre = min(D - 1, M);
    for (int j = 0; j < pre; ++j) {
        const int pj = reinterpret_cast<const int*>(w.draws + (j % kDrawRing) * kStride)[0];
        if (lane == 31) w.pix[j] = pj;
        issue_row_pred(lane == 31, &w.bar[j], w.stages + (size_t)j * a.stage_bytes,
                       a.table + (long long)pj * a.row_stride, (uint32_t)a.copy_bytes);
    }
    int issued = pre - 1;
    if (!mbar_wait_bounded(&w.bar[0], phase & 1u)) {
        raise_error(a.error, SATPILA_ERR_TIMEOUT);
        drain_stages(w, D, 0, issued, phase);
        return false;
    }
    phase ^= 1u;

    Recs<JMAX> ra, rb;
    float a0[JMAX], a1[JMAX], b0[JMAX], b1[JMAX];
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        rb.k[j] = 0;
        rb.l0[j] = rb.l1[j] = 0.0f;
        b0[j] = b1[j] = 0.0f;
    }
    decode_stage<F16, JMAX>(w.stages, lane, JMAX, ra);
    gather<JMAX>(R, rowbase, ra, a0, a1);
    MoveState ms;
    ms.p = w.pix[0];
    ms.f = img[ms.p];
    ms.fwd = false;
    ms.fwd_f = 0.0f;
    float C = sqrtf(fmaxf(0.0f, S_hi * a.inv_BU));
    const bool tracing = a.trace && s >= 0 && a.trace_chain >= 0 && c == a.trace_chain;
    int st_cur = 0;
    int m = 0;
    // Two moves per trip: the register sets alternate roles, no copies.
    for (; m + 2 < M; m += 2) {
        if (!move_step<F16, JMAX, KMAX, true>(a, w, s, m, M, T, R, img, key, phase, S_hi, S_lo, C, n_acc, lane,
                                              rowbase, st_cur, issued, tracing, ra, a0, a1, rb, b0, b1, ms))
            return false;
        if (!move_step<F16, JMAX, KMAX, true>(a, w, s, m + 1, M, T, R, img, key, phase, S_hi, S_lo, C, n_acc,
                                              lane, rowbase, st_cur, issued, tracing, rb, b0, b1, ra, a0, a1, ms))
            return false;
    }
    if (m + 1 < M) {
        if (!move_step<F16, JMAX, KMAX, true>(a, w, s, m, M, T, R, img, key, phase, S_hi, S_lo, C, n_acc, lane,
                                              rowbase, st_cur, issued, tracing, ra, a0, a1, rb, b0, b1, ms))
            return false;
        return move_step<F16, JMAX, KMAX, false>(a, w, s, m + 1, M, T, R, img, key, phase, S_hi, S_lo, C, n_acc,
                                                 lane, rowbase, st_cur, issued, tracing, rb, b0, b1, ra, a0, a1, ms);
    }
    return move_step<F16, JMAX, KMAX, false>(a, w, s, m, M, T, R, img, key, phase, S_hi, S_lo, C, n_acc, lane,
                                             rowbase, st_cur, issued, tracing, ra, a0, a1, rb, b0, b1, ms);
}

// Waits until another warp has finished the chain's earlier stages (at most
// 20 s of wall time).
static __device__ __forceinline__ bool wait_progress(const int* flag, int target) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (ld_acquire(flag) >= target) return true;
        if (global_ns() - t0 > 20000000000ull) return false;
        __nanosleep(256);
    }
}

template <bool F16, bool SMEM, int JMAX, int KMAX>
__global__ void __launch_bounds__(kSatMaxWarps * 32) sat_sweep_kernel(const SatArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wb = smem + (size_t)warp * a.warp_smem_bytes;
    WarpRing w;
    w.bar = reinterpret_cast<uint64_t*>(wb);
    w.pix = reinterpret_cast<int*>(wb + 64);
    w.draws = reinterpret_cast<float*>(wb + 128);
    w.stages = wb + kRingHeader;
    float* rs = reinterpret_cast<float*>(w.stages + (size_t)a.D * a.stage_bytes);

    // Stage tails beyond a row stay zero (length 0 = no contribution).
    for (int e = lane; e < a.D * a.stage_bytes / 16; e += 32)
        reinterpret_cast<uint4*>(w.stages)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (lane == 0)
        for (int d = 0; d < a.D; ++d) mbar_init(&w.bar[d], 1);
    fence_proxy_async_smem();
    if (lane == 0) fence_barrier_init();
    __syncwarp();

    // Residual row offsets of the lane's angles.
    int rowbase[JMAX];
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        const int u = F16 ? 2 * (lane + 32 * (j / 2)) + (j & 1) : lane + 32 * j;
        rowbase[j] = u < a.U ? u * a.pitch : a.U * a.pitch + 2 * lane;  // past U: this lane's dummy cells
    }

    uint32_t phase = 0;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.task_counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.n_tasks) break;
        const int c = t % a.n_chains;
        const int blk = t / a.n_chains;
        const int s0 = a.sweep_begin + blk * a.sweeps_per_task;
        const int s1 = min(s0 + a.sweeps_per_task, a.sweep_end);
        if (blk > 0) {
            int ok = 1;
            if (lane == 0) ok = wait_progress(&a.progress[c], s0) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                raise_error(a.error, SATPILA_ERR_TIMEOUT);
                break;
            }
        }
        float* gres = a.resid + (long long)c * a.resid_floats;
        float* R = SMEM ? rs : gres;
        if (SMEM) {
            const float4* src = reinterpret_cast<const float4*>(gres);
            float4* dst = reinterpret_cast<float4*>(rs);
            for (long long e = lane; e < a.resid_floats / 4; e += 32) dst[e] = src[e];
            __syncwarp();
        }
        const double S = a.S[c];
        float S_hi = (float)S;
        float S_lo = -(float)(S - (double)S_hi);  // Kahan carries the negated remainder
        unsigned long long n_acc = 0;
        const uint2 key = chain_key(a.seed + (unsigned long long)c);
        float* img = a.img + (long long)c * a.img_stride;
        const double T0 = a.T0[c], TN = a.TN[c];
        bool ok = true;
        for (int s = s0; s < s1 && ok; ++s) {
            const float T = (float)stage_temperature(a.schedule, T0, TN, s, a.n_sweeps_total);
            ok = run_stage<F16, SMEM, JMAX, KMAX>(a, w, c, s, T, R, img, key, phase, S_hi, S_lo, n_acc, lane,
                                                  rowbase);
            if (a.sweep_cost && lane == 0)
                a.sweep_cost[(long long)c * a.n_sweeps_total + s] =
                    sqrt(((double)S_hi - (double)S_lo) * a.inv_BU_d);
        }
        __syncwarp();
        if (SMEM) {
            const float4* src = reinterpret_cast<const float4*>(rs);
            float4* dst = reinterpret_cast<float4*>(gres);
            for (long long e = lane; e < a.resid_floats / 4; e += 32) dst[e] = src[e];
        }
        if (lane == 0) {
            a.S[c] = (double)S_hi - (double)S_lo;
            a.accepted[c] += n_acc;
        }
        __syncwarp();
        __threadfence();
        if (lane == 0) st_release(&a.progress[c], s1);
        if (!ok) break;
    }
}

// ---- Eq. (8): initial temperature ------------------------------------------

struct T0Args {
    const unsigned char* table;
    long long row_stride;
    int f16;
    int n, U, B;
    int pitch;
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
};

}  // namespace satpila
