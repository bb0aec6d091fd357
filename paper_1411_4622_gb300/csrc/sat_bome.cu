// Best of multiple estimates as Sec. III-B words it: each of the N_e
// estimates of a move is its own random pixel with its own random value
// (Eq. (3)); all are evaluated by Eq. (7) on the same current state, the one
// with the smallest cost is kept, and Step 4 decides on it.  One warp per
// chain, residual in global memory (L2).
//
// Random words of move m (Philox key = chain seed, counter (stage, m, block,
// 1)): word 0 picks estimate 0's pixel, word 1 is N1, word 2 + e is estimate
// e's value, word 2 + N_e + (e - 1) picks estimate e's pixel (e >= 1).  With
// N_e = 1 this is the one-pixel move.
//
// Per move the warp holds the N_e PILA rows in shared memory (fetched by
// cp.async one move ahead, since pixels do not depend on the state), each
// lane accumulates its angles' part of g_e = sum r l for every estimate, a
// reduce-scatter over the lanes leaves g_e in lane e, lane e forms
// dS_e = df_e (2 g_e + df_e h_e), a shuffle argmin (lowest index on ties)
// picks the estimate, and on acceptance each lane updates its own cells of
// the chosen row (no other lane owns them).
#include "sat_sweep.cuh"

namespace satpila {
namespace {

constexpr int kBomeWarps = 4;

// Sum over the 32 lanes of v[0..31] with the total of v[e] left in lane e.
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            // keep the half this lane is responsible for, send the other
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    return v[0];
}

template <bool F16, int JMAX, int KMAX>
__device__ __forceinline__ void bome_stage(const SatArgs& a, const StageCtx& x, unsigned char* const (&buf)[2],
                                           const int (&rowbase)[JMAX], float& S_hi, float& S_lo,
                                           unsigned long long& n_acc) {
    const int M = x.M, K = a.K, lane = x.lane;
    if (M <= 0 || a.n_list <= 0) return;
    const uint32_t nl = (uint32_t)a.n_list;
    const int nblk = (2 * K + 1 + 3) / 4;
    // Philox block `lane` of move m (lanes < nblk), and word i of it by shuffle.
    auto words = [&](int m) {
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (lane < nblk) w = philox4x32_10(make_uint4((uint32_t)x.s, (uint32_t)m, (uint32_t)lane, kStreamSat), x.key);
        return w;
    };
    // word i (the same i on every lane)
    auto word = [&](const uint4& w, int i) {
        const int q = i & 3;
        const uint32_t v = q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w;
        return __shfl_sync(0xffffffffu, v, i >> 2);
    };
    // word i (i may differ between lanes)
    auto word_any = [&](const uint4& w, int i) {
        const int src = i >> 2, q = i & 3;
        const uint32_t x0 = __shfl_sync(0xffffffffu, w.x, src), x1 = __shfl_sync(0xffffffffu, w.y, src);
        const uint32_t x2 = __shfl_sync(0xffffffffu, w.z, src), x3 = __shfl_sync(0xffffffffu, w.w, src);
        return q == 0 ? x0 : q == 1 ? x1 : q == 2 ? x2 : x3;
    };
    // lane e < K: estimate e's pixel
    auto pixel_of = [&](const uint4& w) {
        int p = 0;
#pragma unroll
        for (int e = 0; e < KMAX; ++e) {
            if (e >= K) break;
            const uint32_t wx = word(w, e == 0 ? 0 : 2 + K + e - 1);
            if (lane == e) {
                const uint32_t idx = pick_index(wx, nl);
                p = a.list ? __ldg(a.list + idx) : (int)idx;
            }
        }
        return p;
    };
    auto fetch = [&](int pe_lane, unsigned char* dst) {
#pragma unroll
        for (int e = 0; e < KMAX; ++e) {
            if (e >= K) break;
            const int p = __shfl_sync(0xffffffffu, pe_lane, e);
            const unsigned char* row = a.table + (long long)p * a.row_stride;
            unsigned char* st = dst + (size_t)e * a.stage_bytes;
#pragma unroll
            for (int i = 0; i < chunks_per_lane<F16, JMAX>(); ++i) {
                const int q = lane + 32 * i;
                cp_async_16_pred(q < a.row_chunks, st + 16 * q, row + 16 * (q < a.row_chunks ? q : 0));
            }
        }
        cp_async_commit();
    };

    uint4 w_cur = words(0);
    int p_cur = pixel_of(w_cur);
    fetch(p_cur, buf[0]);
    float C = sqrtf(fmaxf(0.0f, S_hi * a.inv_BU));
    for (int m = 0; m < M; ++m) {
        // next move's words, pixels and rows while this one is evaluated
        uint4 w_nxt = w_cur;
        int p_nxt = p_cur;
        if (m + 1 < M) {
            w_nxt = words(m + 1);
            p_nxt = pixel_of(w_nxt);
            fetch(p_nxt, buf[(m + 1) & 1]);
        } else {
            cp_async_commit();
        }
        // lane e: its estimate's current value and candidate (Eq. (3))
        const float u_e = unit_uniform(word_any(w_cur, 2 + (lane < K ? lane : 0)));
        float f_e = 0.0f, fc_e = 0.0f, df_e = 0.0f, h_e = 0.0f;
        if (lane < K) {
            f_e = __ldcg(x.img + p_cur);
            h_e = __ldg(a.hsum + p_cur);
            const float lo = fmaxf(0.0f, f_e - a.beta), span = fminf(a.beta, f_e + a.beta) - lo;
            fc_e = fmaf(u_e, span, lo);
            df_e = fc_e - f_e;
        }
        const float L = -__logf(unit_uniform(word(w_cur, 1)));
        cp_async_wait_pending(1);  // this move's rows have landed
        __syncwarp();
        const unsigned char* rows = buf[m & 1];
        // each lane's part of g_e for every estimate
        float gp[KMAX > 8 ? 32 : KMAX];
#pragma unroll
        for (int e = 0; e < (KMAX > 8 ? 32 : KMAX); ++e) gp[e] = 0.0f;
#pragma unroll
        for (int e = 0; e < KMAX; ++e) {
            if (e >= K) break;
            Recs<JMAX> r;
            decode_stage<F16, JMAX>(rows + (size_t)e * a.stage_bytes, lane, 1, r);
            float g = 0.0f;
#pragma unroll
            for (int j = 0; j < JMAX; ++j) {
                const float* q = x.R + rowbase[j] + r.k[j];
                g = fmaf(__ldcg(q), r.l0[j], g);
                g = fmaf(__ldcg(q + 1), r.l1[j], g);
            }
            gp[e] = g;
        }
        float g_e;
        if constexpr (KMAX > 8) {
            g_e = reduce_scatter32(gp, lane);
        } else {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int e = 0; e < KMAX; ++e) gp[e] += __shfl_xor_sync(0xffffffffu, gp[e], o);
            g_e = 0.0f;
#pragma unroll
            for (int e = 0; e < KMAX; ++e) g_e = lane == e ? gp[e] : g_e;
        }
        // lane e: Eq. (7) sum of estimate e; argmin over the lanes
        float dS = lane < K ? df_e * fmaf(df_e, h_e, 2.0f * g_e) : __int_as_float(0x7f800000);
        int ci = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float od = __shfl_xor_sync(0xffffffffu, dS, o);
            const int oi = __shfl_xor_sync(0xffffffffu, ci, o);
            const bool take = od < dS || (od == dS && oi < ci);
            dS = take ? od : dS;
            ci = take ? oi : ci;
        }
        const int p = __shfl_sync(0xffffffffu, p_cur, ci);
        const float df = __shfl_sync(0xffffffffu, df_e, ci);
        const float f = __shfl_sync(0xffffffffu, f_e, ci);
        const float fc = __shfl_sync(0xffffffffu, fc_e, ci);
        // Step 4, threshold form: accept iff x <= 0 or x < T L (2 C + T L)
        const float TL = x.T * L;
        const float theta = TL * fmaf(2.0f, C, TL);
        const float xs = dS * a.inv_BU;
        const bool accept = xs <= 0.0f || xs < theta;
        if (x.tracing && lane == 0) {
            const long long idx = (long long)x.s * M + m;
            if (idx < a.trace_cap) {
                const float Cp = sqrtf(fmaxf(0.0f, fmaf(C, C, xs)));
                const float den = Cp + C;
                sat_trace_rec rr;
                rr.pixel = p;
                rr.cstar = ci;
                rr.accepted = accept ? 1 : 0;
                rr.pad = 0;
                rr.dS = dS;
                rr.dC = den > 0.0f ? xs / den : 0.0f;
                rr.fnew = accept ? fc : f;
                rr.pad2 = 0.0f;
                a.trace[idx] = rr;
            }
        }
        if (accept) {
            // Eq. (6) on the chosen row, each lane its own cells
            Recs<JMAX> r;
            decode_stage<F16, JMAX>(rows + (size_t)ci * a.stage_bytes, lane, 1, r);
#pragma unroll
            for (int j = 0; j < JMAX; ++j) {
                float* q = x.R + rowbase[j] + r.k[j];
                __stcg(q, fmaf(df, r.l0[j], __ldcg(q)));
                __stcg(q + 1, fmaf(df, r.l1[j], __ldcg(q + 1)));
            }
            if (lane == 0) __stcg(x.img + p, fc);
            const float y = dS - S_lo;
            const float t = S_hi + y;
            S_lo = (t - S_hi) - y;
            S_hi = t;
            const float C2 = fmaxf(0.0f, S_hi * a.inv_BU);
            C = C2 > 0.0f ? C2 * rsqrtf(C2) : 0.0f;
            ++n_acc;
        }
        __syncwarp();
        w_cur = w_nxt;
        p_cur = p_nxt;
    }
    cp_async_wait_pending(0);
}

template <bool F16, int JMAX, int KMAX>
__global__ void __launch_bounds__(kBomeWarps * 32) sat_bome_kernel(const SatArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wsm = smem + (size_t)warp * a.group_smem_bytes;
    unsigned char* const buf[2] = {wsm, wsm + (size_t)a.K * a.stage_bytes};
    // chunks past a row stay zero (length 0: no contribution)
    for (int e = lane; e < 2 * a.K * a.stage_bytes / 16; e += 32)
        reinterpret_cast<uint4*>(wsm)[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    int rowbase[JMAX];
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        const int u = record_of<F16>(lane, 1, j);
        rowbase[j] = u < a.U ? u * a.pitch : a.U * a.pitch + 2 * lane;
    }
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
            if (lane == 0) ok = wait_progress(&a.progress[c], s0, a.wait_ns) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) raise_error(a.error, SATPILA_ERR_TIMEOUT);
                break;
            }
        }
        const double S = a.S[c];
        float S_hi = (float)S;
        float S_lo = -(float)(S - (double)S_hi);
        unsigned long long n_acc = 0;
        StageCtx x;
        x.M = a.moves;
        x.D = 2;
        x.W = 1;
        x.wig = 0;
        x.lane = lane;
        x.gid = 1 + warp;
        x.gl = lane;
        x.il = 0;  // plain rows (this kernel's plans never interleave them)
        x.R = a.resid + (long long)c * a.resid_floats;
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
            bome_stage<F16, JMAX, KMAX>(a, x, buf, rowbase, S_hi, S_lo, n_acc);
            if (a.sweep_cost && lane == 0)
                a.sweep_cost[(long long)c * a.n_sweeps_total + s] = sqrt(((double)S_hi - (double)S_lo) * a.inv_BU_d);
        }
        __syncwarp();
        if (lane == 0) {
            a.S[c] = (double)S_hi - (double)S_lo;
            a.accepted[c] += n_acc;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0 && report_progress(a, c, s0)) st_release(&a.progress[c], s1);
    }
}

}  // namespace

using SweepFn = void (*)(const SatArgs);

template <bool F16, int JMAX>
SweepFn bome_by_k(int kmax) {
    switch (kmax) {
        case 4: return sat_bome_kernel<F16, JMAX, 4>;
        case 8: return sat_bome_kernel<F16, JMAX, 8>;
        case 32: return sat_bome_kernel<F16, JMAX, 32>;
        default: return nullptr;
    }
}

SweepFn bome_kernel(bool f16, int jmax, int kmax) {
    switch (jmax) {
        case 2: return f16 ? bome_by_k<true, 2>(kmax) : bome_by_k<false, 2>(kmax);
        case 4: return f16 ? bome_by_k<true, 4>(kmax) : bome_by_k<false, 4>(kmax);
        case 8: return f16 ? bome_by_k<true, 8>(kmax) : bome_by_k<false, 8>(kmax);
        case 16: return f16 ? bome_by_k<true, 16>(kmax) : bome_by_k<false, 16>(kmax);
        default: return nullptr;
    }
}

int bome_warps_per_cta() { return kBomeWarps; }

}  // namespace satpila
