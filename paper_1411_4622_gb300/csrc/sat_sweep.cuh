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
constexpr int kURing = 40;  // floats per uniform slot (>= 4 * ceil((kMaxK + 2) / 4))

__device__ __forceinline__ double stage_temperature(int schedule, double t0, double tn, int s, int n_sweeps) {
    const double N = (double)n_sweeps, n = (double)s;
    if (schedule == SAT_SCHED_GEOMETRIC) return t0 <= 0.0 ? 0.0 : t0 * pow(tn / t0, n / N);
    if (schedule == SAT_SCHED_CUBIC) return t0 - n * n * n * (t0 - tn) / (N * N * N);
    return t0 - n * (t0 - tn) / N;
}

// Calls fn(j, u, entry) for the lane's records j < J of a stage buffer.
template <bool F16, int JMAX, typename Fn>
__device__ __forceinline__ void for_each_record(const unsigned char* stage, int lane, int J, Fn&& fn) {
    const uint4* q4 = reinterpret_cast<const uint4*>(stage);
    if constexpr (F16) {
#pragma unroll
        for (int i = 0; i < JMAX / 2; ++i) {
            if (2 * i < J) {
                const int q = lane + 32 * i;
                const uint4 v = q4[q];
                fn(2 * i, 2 * q, decode_f16(v.x, v.y));
                fn(2 * i + 1, 2 * q + 1, decode_f16(v.z, v.w));
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < JMAX; ++i) {
            if (i < J) {
                const int q = lane + 32 * i;
                fn(i, q, decode_f32(q4[q]));
            }
        }
    }
}

// Same, over two stage buffers at once (same lane, same angle u).
template <bool F16, int JMAX, typename Fn>
__device__ __forceinline__ void for_each_record_pair(const unsigned char* s0, const unsigned char* s1, int lane,
                                                     int J, Fn&& fn) {
    const uint4* a4 = reinterpret_cast<const uint4*>(s0);
    const uint4* b4 = reinterpret_cast<const uint4*>(s1);
    if constexpr (F16) {
#pragma unroll
        for (int i = 0; i < JMAX / 2; ++i) {
            if (2 * i < J) {
                const int q = lane + 32 * i;
                const uint4 va = a4[q], vb = b4[q];
                fn(2 * i, decode_f16(va.x, va.y), decode_f16(vb.x, vb.y));
                fn(2 * i + 1, decode_f16(va.z, va.w), decode_f16(vb.z, vb.w));
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < JMAX; ++i) {
            if (i < J) {
                const int q = lane + 32 * i;
                fn(i, decode_f32(a4[q]), decode_f32(b4[q]));
            }
        }
    }
}

struct WarpRing {
    uint64_t* bar;       // [kMaxStages]
    int* pix;            // [kMaxStages] pixel of the move held by each stage
    float* uring;        // [2][kURing] uniforms of the current / next move
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

// One temperature stage of one chain.  Returns false if a bounded wait gave up.
template <bool F16, bool SMEM, int JMAX>
__device__ __forceinline__ bool run_stage(const SatArgs& a, const WarpRing& w, int c, int s, float T, float* R,
                                          float* img, uint2 key, uint32_t& phase, double& S, float& C2,
                                          unsigned long long& n_acc, int lane) {
    const int M = a.moves, D = a.D, K = a.K, B = a.B, J = a.J;
    if (M <= 0 || a.n_list <= 0) return true;
    const int nblk = (K + 2 + 3) / 4;
    const uint32_t nl = (uint32_t)a.n_list;
    const int32_t* list = a.list;
    auto pixel_of = [&](uint32_t x) -> int {
        const uint32_t i = pick_index(x, nl);
        return list ? list[i] : (int)i;
    };
    auto issue = [&](int st, int p) {  // lane 31 only
        w.pix[st] = p;
        mbar_arrive_expect_tx(&w.bar[st], (uint32_t)a.copy_bytes);
        bulk_copy_g2s(w.stages + (size_t)st * a.stage_bytes, a.table + (long long)p * a.row_stride,
                      (uint32_t)a.copy_bytes, &w.bar[st]);
        prefetch_l1(img + p);
    };

    // Prologue: rows of moves 0..D-2 in flight, uniforms of move 0, pixel of move D-1.
    const int pre = min(D - 1, M);
    if (lane == 31) {
        for (int j = 0; j < pre; ++j) {
            const uint4 x = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)j, 0u, kStreamSat), key);
            issue(j, pixel_of(x.x));
        }
    }
    int pending = 0;
    {
        const uint4 ctr = lane == 31 ? make_uint4((uint32_t)s, (uint32_t)(D - 1), 0u, kStreamSat)
                                     : make_uint4((uint32_t)s, 0u, (uint32_t)lane, kStreamSat);
        const uint4 x = philox4x32_10(ctr, key);
        if (lane < nblk) {
            float* u = w.uring + 4 * lane;
            u[0] = unit_uniform(x.x);
            u[1] = unit_uniform(x.y);
            u[2] = unit_uniform(x.z);
            u[3] = unit_uniform(x.w);
        }
        if (lane == 31 && D - 1 < M) pending = pixel_of(x.x);
    }
    __syncwarp();
    int issued = pre - 1;  // last move whose row has been requested
    if (!mbar_wait_bounded(&w.bar[0], phase & 1u)) {
        raise_error(a.error, SATPILA_ERR_TIMEOUT);
        drain_stages(w, D, 0, issued, phase);
        return false;
    }
    phase ^= 1u;

    float rv0[JMAX], rv1[JMAX], nv0[JMAX], nv1[JMAX];
#pragma unroll
    for (int j = 0; j < JMAX; ++j) rv0[j] = rv1[j] = nv0[j] = nv1[j] = 0.0f;
    int p = w.pix[0];
    float f = img[p];
    for_each_record<F16, JMAX>(w.stages, lane, J, [&](int j, int u, const Entry2& e) {
        rv0[j] = e.l0 != 0.0f ? R[u * B + e.k0] : 0.0f;
        rv1[j] = e.l1 != 0.0f ? R[u * B + e.k1] : 0.0f;
    });

    int st_cur = 0;
    for (int m = 0; m < M; ++m) {
        const int st_next = st_cur + 1 == D ? 0 : st_cur + 1;
        const int st_issue = st_cur == 0 ? D - 1 : st_cur - 1;
        __syncwarp();
        // Row of move m+D-1 into the stage freed by move m-1.
        if (lane == 31 && m + D - 1 < M) issue(st_issue, pending);
        if (m + D - 1 < M) issued = m + D - 1;
        {
            // One Philox evaluation serves two purposes: lanes < nblk draw the
            // uniforms of move m+1, lane 31 the pixel of move m+D.
            const uint4 ctr = lane == 31 ? make_uint4((uint32_t)s, (uint32_t)(m + D), 0u, kStreamSat)
                                         : make_uint4((uint32_t)s, (uint32_t)(m + 1), (uint32_t)lane, kStreamSat);
            const uint4 x = philox4x32_10(ctr, key);
            if (lane < nblk && m + 1 < M) {
                float* u = w.uring + ((m + 1) & 1) * kURing + 4 * lane;
                u[0] = unit_uniform(x.x);
                u[1] = unit_uniform(x.y);
                u[2] = unit_uniform(x.z);
                u[3] = unit_uniform(x.w);
            }
            if (lane == 31 && m + D < M) pending = pixel_of(x.x);
        }
        __syncwarp();

        const unsigned char* cur = w.stages + (size_t)st_cur * a.stage_bytes;
        const unsigned char* nxt = w.stages + (size_t)st_next * a.stage_bytes;
        // Partial sums of the current move.
        float g = 0.0f, h = 0.0f;
        for_each_record<F16, JMAX>(cur, lane, J, [&](int j, int, const Entry2& e) {
            g = fmaf(rv0[j], e.l0, g);
            g = fmaf(rv1[j], e.l1, g);
            h = fmaf(e.l0, e.l0, h);
            h = fmaf(e.l1, e.l1, h);
        });
        // Gather of the next move while this one is reduced and decided.
        int p1 = -1;
        float f1 = 0.0f;
        if (m + 1 < M) {
            if (!mbar_wait_bounded(&w.bar[st_next], (phase >> st_next) & 1u)) {
                raise_error(a.error, SATPILA_ERR_TIMEOUT);
                drain_stages(w, D, m + 1, issued, phase);
                return false;
            }
            phase ^= 1u << st_next;
            p1 = w.pix[st_next];
            f1 = img[p1];
            for_each_record<F16, JMAX>(nxt, lane, J, [&](int j, int u, const Entry2& e) {
                nv0[j] = e.l0 != 0.0f ? R[u * B + e.k0] : 0.0f;
                nv1[j] = e.l1 != 0.0f ? R[u * B + e.k1] : 0.0f;
            });
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            g += __shfl_xor_sync(0xffffffffu, g, o);
            h += __shfl_xor_sync(0xffffffffu, h, o);
        }
        // BoME over the K estimates (every lane evaluates all of them).
        const float* ur = w.uring + (m & 1) * kURing;
        const float lo = fmaxf(0.0f, f - a.beta), hi = fminf(a.beta, f + a.beta), span = hi - lo;
        const float g2 = 2.0f * g;
        float best_dS = __int_as_float(0x7f800000), best_df = 0.0f, best_f = f;
        int best_c = 0;
        for (int e = 0; e < K; ++e) {
            const float fc = fmaf(ur[2 + e], span, lo);
            const float df = fc - f;
            const float dS = df * fmaf(df, h, g2);
            if (dS < best_dS) {
                best_dS = dS;
                best_df = df;
                best_f = fc;
                best_c = e;
            }
        }
        // Eq. (7) and Step 4.
        const float x = best_dS * a.inv_BU;
        const float C = sqrtf(C2);
        const float Cp = sqrtf(fmaxf(0.0f, C2 + x));
        const float den = Cp + C;
        const float dC = den > 0.0f ? x / den : 0.0f;
        const bool accept = dC <= 0.0f || (T > 0.0f && ur[1] < expf(-dC / T));
        if (accept) {
            for_each_record<F16, JMAX>(cur, lane, J, [&](int j, int u, const Entry2& e) {
                if (e.l0 != 0.0f) R[u * B + e.k0] = fmaf(best_df, e.l0, rv0[j]);
                if (e.l1 != 0.0f) R[u * B + e.k1] = fmaf(best_df, e.l1, rv1[j]);
            });
            if (m + 1 < M) {
                for_each_record_pair<F16, JMAX>(cur, nxt, lane, J, [&](int j, const Entry2& ec, const Entry2& en) {
                    if (en.l0 != 0.0f) {
                        if (ec.l0 != 0.0f && ec.k0 == en.k0) nv0[j] = fmaf(best_df, ec.l0, nv0[j]);
                        if (ec.l1 != 0.0f && ec.k1 == en.k0) nv0[j] = fmaf(best_df, ec.l1, nv0[j]);
                    }
                    if (en.l1 != 0.0f) {
                        if (ec.l0 != 0.0f && ec.k0 == en.k1) nv1[j] = fmaf(best_df, ec.l0, nv1[j]);
                        if (ec.l1 != 0.0f && ec.k1 == en.k1) nv1[j] = fmaf(best_df, ec.l1, nv1[j]);
                    }
                });
            }
            img[p] = best_f;
            if (p1 == p) f1 = best_f;
            S += (double)best_dS;
            C2 = (float)(S * a.inv_BU_d);
            ++n_acc;
        }
        if (a.trace && c == a.trace_chain && lane == 0) {
            const long long idx = (long long)s * M + m;
            if (idx < a.trace_cap) {
                sat_trace_rec r;
                r.pixel = p;
                r.cstar = best_c;
                r.accepted = accept ? 1 : 0;
                r.pad = 0;
                r.dS = best_dS;
                r.dC = dC;
                r.fnew = accept ? best_f : f;
                r.pad2 = 0.0f;
                a.trace[idx] = r;
            }
        }
#pragma unroll
        for (int j = 0; j < JMAX; ++j) {
            rv0[j] = nv0[j];
            rv1[j] = nv1[j];
        }
        f = f1;
        p = p1;
        st_cur = st_next;
    }
    return true;
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

template <bool F16, bool SMEM, int JMAX>
__global__ void __launch_bounds__(kSatMaxWarps * 32) sat_sweep_kernel(const SatArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wb = smem + (size_t)warp * a.warp_smem_bytes;
    WarpRing w;
    w.bar = reinterpret_cast<uint64_t*>(wb);
    w.pix = reinterpret_cast<int*>(wb + 64);
    w.uring = reinterpret_cast<float*>(wb + 128);
    w.stages = wb + 512;
    float* rs = reinterpret_cast<float*>(w.stages + (size_t)a.D * a.stage_bytes);

    // Stage tails beyond a row stay zero (length 0 = no contribution).
    for (int e = lane; e < a.D * a.stage_bytes / 16; e += 32)
        reinterpret_cast<uint4*>(w.stages)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (lane == 0)
        for (int d = 0; d < a.D; ++d) mbar_init(&w.bar[d], 1);
    fence_proxy_async_smem();
    if (lane == 0) fence_barrier_init();
    __syncwarp();

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
        double S = a.S[c];
        float C2 = (float)(S * a.inv_BU_d);
        unsigned long long n_acc = 0;
        const uint2 key = chain_key(a.seed + (unsigned long long)c);
        float* img = a.img + (long long)c * a.img_stride;
        const double T0 = a.T0[c], TN = a.TN[c];
        bool ok = true;
        for (int s = s0; s < s1 && ok; ++s) {
            const float T = (float)stage_temperature(a.schedule, T0, TN, s, a.n_sweeps_total);
            ok = run_stage<F16, SMEM, JMAX>(a, w, c, s, T, R, img, key, phase, S, C2, n_acc, lane);
            if (a.sweep_cost && lane == 0) a.sweep_cost[(long long)c * a.n_sweeps_total + s] = sqrt(S * a.inv_BU_d);
        }
        __syncwarp();
        if (SMEM) {
            const float4* src = reinterpret_cast<const float4*>(rs);
            float4* dst = reinterpret_cast<float4*>(gres);
            for (long long e = lane; e < a.resid_floats / 4; e += 32) dst[e] = src[e];
        }
        if (lane == 0) {
            a.S[c] = S;
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
