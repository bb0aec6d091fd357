// Windowed form of the annealing move for one warp per chain, with the
// residual in shared memory or in global memory (identical arithmetic), or
// for a group of WG = 2 or 4 warps per chain that split its angles, with the
// residual in global memory.  Windows of kWin = 2 moves; the notes below hold
// for any kWin dividing 4.
//
// Moves are still decided one after the other, each on the exact state left
// by all earlier moves; what changes is how that state is read.  For a window
// of kWin consecutive moves j (their pixels do not depend on the chain state)
// the warp gathers every move's residual cells at the start of the window and
// reduces, in one batch of independent shuffles,
//   Gs_j = sum over j's entries of r * l_j          (residual at window start)
//   OV_ij = sum over cells shared by i and j of l_i * l_j        (i < j).
// Because Eq. (6) adds df_i * l_i on move i's cells, the sum that move j's
// Eq. (7) needs is exactly  g_j = Gs_j + sum_{i<j} df_i * OV_ij.  Each
// decision then costs a few FMAs plus the BoME selection.  Afterwards each
// cell of move j is written with its gathered value plus the updates of the
// moves i <= j that touched it (each lane owns its cells, so no
// synchronisation; a cell several moves touch is rewritten in move order).
#pragma once
#include "sat_sweep.cuh"

namespace satpila {

constexpr int kWin = 2;  // measured best: 2 beat 4 (fewer pair terms, less live state) and 1 (no batching)
constexpr int kPairs = kWin * (kWin - 1) / 2;

// For slot s, the lengths that move i (records ki, a0, a1) puts on the two
// cells of move j (bins kj, kj + 1); entry 1 of a record sits on bin k + 1.
__device__ __forceinline__ void cell_share(int ki, float a0, float a1, int kj, float& s0, float& s1) {
    const int d = kj - ki;
    s0 = d == 0 ? a0 : (d == 1 ? a1 : 0.0f);
    s1 = d == 0 ? a1 : (d == -1 ? a0 : 0.0f);
}

// Near-ties (with SAT_FLAG_NEAR_TIES): a decision whose margin is within the
// FP32 rounding of its own terms - the BoME gap between the best two
// estimates, or Step 4's ΔC against T(-ln N1) or against 0, below 2e-5 of the
// term scale 2|df| sum|r l| + df^2 sum l^2 (the FP64 comparison's tolerance) -
// where an FP64 evaluation could decide otherwise.
constexpr float kTieTol = 2e-5f;

// TRACE: the chain records its moves (x.tracing); a separate build so that
// the untraced move carries no per-move test for it.
template <int RT, bool SMEM, int JMAX, int KMAX, int WG = 1, bool NT = false, bool TRACE = false>
__device__ __forceinline__ void run_stage_window(const SatArgs& a, const GroupShared& G, const StageCtx& x,
                                                 float& S_hi, float& S_lo, unsigned long long& n_acc,
                                                 unsigned& n_ties, const int (&rowbase)[JMAX]) {
    constexpr int kWords = draw_words<KMAX>();
    constexpr int kB = batch_moves(KMAX), kR = ring_slots(KMAX);  // moves per draw block, ring slots (2^k)
    static_assert((kR & (kR - 1)) == 0, "the draw ring is a power of two");
    const int M = x.M;
    if (M <= 0 || a.n_list <= 0) return;
    const int nwin = (M + kWin - 1) / kWin;
    auto stage_of = [&](int w, int j) { return G.stages + (size_t)((w & 1) * kWin + j) * a.stage_bytes; };
    // Rows of window w's moves into its stages, one commit group (empty past
    // the stage's last move: the copies are predicated, not branched around;
    // a slot past the last move may hold any value, and its row is not read).
    auto fetch_window = [&](int w) {
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
            const int mv = w * kWin + j;
            const bool live = mv < M;
            const unsigned char* row = a.table + (long long)(live ? G.pix[mv & (kR - 1)] : 0) * a.row_stride;
            unsigned char* st = stage_of(w, j);
#pragma unroll
            for (int i = 0; i < rt_chunks_per_lane<RT, JMAX>(); ++i) {
                const int q = x.gl + 32 * WG * i;
                const bool in = live && q < a.row_chunks;
                cp_async_16_pred(in, st + 16 * q, row + 16 * (in ? q : 0));
            }
        }
        cp_async_commit();
    };

    PendingPixel pend;
    draw_batch<KMAX, kB, kR>(a, G, x.s, 0, x.key, x.lane, false, pend);
    draw_batch<KMAX, kB, kR>(a, G, x.s, kB, x.key, x.lane, false, pend);
    __syncwarp();
    fetch_window(0);
    // Pixel values of the next window are loaded before this window's
    // writes and forwarded from them where a pixel repeats.
    int pn[kWin];
    float fn[kWin], hn[kWin];  // (and the pixels' sums of squared lengths)
#pragma unroll
    for (int j = 0; j < kWin; ++j) {
        pn[j] = j < M ? G.pix[j & (kR - 1)] : -1;
        fn[j] = pn[j] >= 0 ? __ldcg(x.img + pn[j]) : 0.0f;
        hn[j] = pn[j] >= 0 ? __ldg(a.hsum + pn[j]) : 0.0f;
    }
    int pw_prev[kWin];
    float fw_prev[kWin];
#pragma unroll
    for (int j = 0; j < kWin; ++j) {
        pw_prev[j] = -1;
        fw_prev[j] = 0.0f;
    }
    // Records of the window being decided, decoded while the previous window
    // was decided (its rows land a window ahead).
    Recs<JMAX> rc[kWin];
    cp_async_wait_pending(0);
#pragma unroll
    for (int j = 0; j < kWin; ++j) rt_decode_stage<RT, JMAX>(stage_of(0, j), x.gl, WG, rc[j]);
    for (int w = 0; w < nwin; ++w) {
        const int m0 = w * kWin;
        // the draws and pixels written here are read a block later or more,
        // by every lane: each write is followed by a warp barrier
        if ((m0 & (kB - 1)) == 0 && m0 + 2 * kB < M) {
            draw_batch<KMAX, kB, kR>(a, G, x.s, m0 + 2 * kB, x.key, x.lane, true, pend);
            __syncwarp();
        }
        if ((m0 & (kB - 1)) == kB / 2) {
            settle_pixels(G, pend);
            __syncwarp();
        }
        fetch_window(w + 1);  // an empty group after the last window
        // this window's pixels and loaded values; the next window's loads
        int pc[kWin];
        float fc0[kWin], hc[kWin];
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
            pc[j] = pn[j];
            fc0[j] = fn[j];
            hc[j] = hn[j];
            const int mv = m0 + kWin + j;
            pn[j] = mv < M ? G.pix[mv & (kR - 1)] : -1;
            fn[j] = pn[j] >= 0 ? __ldcg(x.img + pn[j]) : 0.0f;
            hn[j] = pn[j] >= 0 ? __ldg(a.hsum + pn[j]) : 0.0f;
        }
        // ---- records, residual sums and pairwise overlaps of the window ----
        int k[kWin][JMAX];
        float l0[kWin][JMAX], l1[kWin][JMAX], v0[kWin][JMAX], v1[kWin][JMAX];
        float sh0[kPairs][JMAX], sh1[kPairs][JMAX];  // cell_share of each pair (i < j)
        constexpr int kRed = NT ? kWin + kPairs + kWin : kWin + kPairs;
        float red[kRed];                             // Gs_j, OV_ij, and (near-ties) sum |r l_j|
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
            const Recs<JMAX>& r = rc[j];
#pragma unroll
            for (int s = 0; s < JMAX; ++s) {
                k[j][s] = r.k[s];
                l0[j][s] = r.l0[s];
                l1[j][s] = r.l1[s];
                if (SMEM) {
                    const float* q = x.R + rowbase[s] + r.k[s];
                    v0[j][s] = q[0];
                    v1[j][s] = q[1];
                } else {
                    v0[j][s] = __ldcg(x.R + resid_cell(rowbase[s], r.k[s], x.il));
                    v1[j][s] = __ldcg(x.R + resid_cell(rowbase[s], r.k[s] + 1, x.il));
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
            float g0 = 0.0f, g1 = 0.0f;
#pragma unroll
            for (int s = 0; s < JMAX; ++s) {
                g0 = fmaf(v0[j][s], l0[j][s], g0);
                g1 = fmaf(v1[j][s], l1[j][s], g1);
            }
            red[j] = g0 + g1;
        }
        {
            int e = 0;
#pragma unroll
            for (int i = 0; i < kWin; ++i)
#pragma unroll
                for (int j = i + 1; j < kWin; ++j) {
                    float ov = 0.0f;
#pragma unroll
                    for (int s = 0; s < JMAX; ++s) {
                        cell_share(k[i][s], l0[i][s], l1[i][s], k[j][s], sh0[e][s], sh1[e][s]);
                        ov = fmaf(sh0[e][s], l0[j][s], ov);
                        ov = fmaf(sh1[e][s], l1[j][s], ov);
                    }
                    red[kWin + e] = ov;
                    ++e;
                }
        }
        if constexpr (NT) {
#pragma unroll
            for (int j = 0; j < kWin; ++j) {
                float s = 0.0f;
#pragma unroll
                for (int q = 0; q < JMAX; ++q) s = fmaf(fabsf(v0[j][q]), l0[j][q], fmaf(fabsf(v1[j][q]), l1[j][q], s));
                red[kWin + kPairs + j] = s;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int e = 0; e < kRed; ++e) red[e] += __shfl_xor_sync(0xffffffffu, red[e], o);
        if constexpr (WG > 1) {
            // each warp holds the sums over its own angles: add the warps'
            // sums in warp order (the same order in every warp).  Slots
            // alternate with the window parity; a warp can be at most one
            // window ahead of the others, so a slot is never overwritten
            // while another warp still reads it.
            float* xr = G.part + (w & 1) * (kPartSlots * kMaxGroupWarps);
            float mine = 0.0f;
#pragma unroll
            for (int e = 0; e < kRed; ++e) mine = x.lane == e ? red[e] : mine;
            if (x.lane < kRed) xr[kPartSlots * x.wig + x.lane] = mine;
            group_sync(x.gid, WG);
#pragma unroll
            for (int e = 0; e < kRed; ++e) {
                float t = xr[e];
#pragma unroll
                for (int q = 1; q < WG; ++q) t += xr[kPartSlots * q + e];
                red[e] = t;
            }
        }

        // the next window's records (past the last window: stale rows, unused)
        cp_async_wait_pending(0);
#pragma unroll
        for (int j = 0; j < kWin; ++j) rt_decode_stage<RT, JMAX>(stage_of(w + 1, j), x.gl, WG, rc[j]);

        // ---- decisions, in move order ----
        float df[kWin], fnew[kWin];
        // Candidates from the values before this window's decisions; a move
        // whose pixel an earlier move of the window also drew recomputes them
        // after that move (a warp-uniform, rare branch).
        bool rep[kWin];
        float fpre[kWin], fcp[kWin][KMAX], dpre[kWin][KMAX];
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
            float f = fc0[j];
#pragma unroll
            for (int i = 0; i < kWin; ++i) f = pw_prev[i] == pc[j] ? fw_prev[i] : f;
            fpre[j] = f;
            rep[j] = false;
#pragma unroll
            for (int i = 0; i < kWin; ++i)
                if (i < j) rep[j] = rep[j] || pc[i] == pc[j];
            const uint32_t* drw = G.draws + ((m0 + j) & (kR - 1)) * kWords;
            const float lo = fmaxf(0.0f, f - a.beta), span = fminf(a.beta, f + a.beta) - lo;
#pragma unroll
            for (int e = 0; e < KMAX; ++e) {
                fcp[j][e] = fmaf(__uint_as_float(drw[2 + e]), span, lo);
                dpre[j][e] = fcp[j][e] - f;
            }
        }
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
            const int m = m0 + j;
            const bool live = m < M;
            float g = red[j];
            {
                int e = kWin;
#pragma unroll
                for (int i = 0; i < kWin; ++i)
#pragma unroll
                    for (int jj = i + 1; jj < kWin; ++jj) {
                        if (jj == j) g = fmaf(df[i], red[e], g);
                        ++e;
                    }
            }
            const uint32_t* drw = G.draws + (m & (kR - 1)) * kWords;
            float f = fpre[j];
            float fcand[KMAX], dd[KMAX];
#pragma unroll
            for (int e = 0; e < KMAX; ++e) {
                fcand[e] = fcp[j][e];
                dd[e] = dpre[j][e];
            }
            if (rep[j]) {
#pragma unroll
                for (int i = 0; i < kWin; ++i)
                    if (i < j) f = pc[i] == pc[j] ? fnew[i] : f;
                const float lo = fmaxf(0.0f, f - a.beta), span = fminf(a.beta, f + a.beta) - lo;
#pragma unroll
                for (int e = 0; e < KMAX; ++e) {
                    fcand[e] = fmaf(__uint_as_float(drw[2 + e]), span, lo);
                    dd[e] = fcand[e] - f;
                }
            }
            const float L = __uint_as_float(drw[1]);
            // Step 4 as x < T L (2 C + T L) with x = dS / (B U), C = sqrt(S / (B U)),
            // squared so that no square root sits on the chain:
            // x <= 0, or x - (T L)^2 < 0, or (x - (T L)^2)^2 < 4 (T L)^2 S / (B U).
            const float TL = x.T * L;
            const float TL2 = TL * TL;
            const float rhs = 4.0f * TL2 * fmaxf(0.0f, S_hi * a.inv_BU);
            const float g2 = 2.0f * g;
            float dS[KMAX];
            int ci[KMAX];
#pragma unroll
            for (int e = 0; e < KMAX; ++e) {
                const float d = dd[e];
                dS[e] = e < a.K ? d * fmaf(d, hc[j], g2) : __int_as_float(0x7f800000);
                ci[e] = e;
            }
#pragma unroll
            for (int width = 1; width < KMAX; width *= 2) {
#pragma unroll
                for (int e = 0; e + width < KMAX; e += 2 * width) {
                    const bool take = dS[e + width] < dS[e];
                    dS[e] = take ? dS[e + width] : dS[e];
                    fcand[e] = take ? fcand[e + width] : fcand[e];
                    ci[e] = take ? ci[e + width] : ci[e];
                }
            }
            const float xs = dS[0] * a.inv_BU;
            const float xm = xs - TL2;
            const bool accept = live && (xs <= 0.0f || xm < 0.0f || xm * xm < rhs);
            if constexpr (NT) if (live) {
                // margins of this decision against the scale of its terms
                const float dfc = fcand[0] - f;
                const float scale = fmaf(2.0f * fabsf(dfc), red[NT ? kWin + kPairs + j : 0], dfc * dfc * hc[j]);
                float second = __int_as_float(0x7f800000);
#pragma unroll
                for (int e = 0; e < KMAX; ++e)
                    if (e < a.K && e != ci[0]) {
                        const float d = dd[e];
                        second = fminf(second, d * fmaf(d, hc[j], g2));
                    }
                const bool bome_tie = second - dS[0] <= kTieTol * scale;
                const float C = sqrtf(fmaxf(0.0f, S_hi * a.inv_BU));
                const float den = sqrtf(fmaxf(0.0f, fmaf(C, C, xs))) + C;
                const float dC = den > 0.0f ? xs / den : 0.0f;
                const float tol_C = den > 0.0f ? kTieTol * scale * a.inv_BU / den : 0.0f;
                const bool step4_tie = fabsf(dC) <= tol_C || (x.T > 0.0f && fabsf(dC - TL) <= tol_C);
                n_ties += (bome_tie || step4_tie) ? 1u : 0u;
            }
            df[j] = accept ? fcand[0] - f : 0.0f;
            fnew[j] = accept ? fcand[0] : f;
            if (TRACE && live && x.gl == 0) {
                const float C = sqrtf(fmaxf(0.0f, S_hi * a.inv_BU));
                const float Cp = sqrtf(fmaxf(0.0f, fmaf(C, C, xs)));
                const float den = Cp + C;
                const long long idx = (long long)x.s * M + m;
                if (idx < a.trace_cap) {
                    sat_trace_rec rr;
                    rr.pixel = pc[j];
                    rr.cstar = ci[0];
                    rr.accepted = accept ? 1 : 0;
                    rr.pad = 0;
                    rr.dS = dS[0];
                    rr.dC = den > 0.0f ? xs / den : 0.0f;
                    rr.fnew = fnew[j];
                    rr.pad2 = 0.0f;
                    a.trace[idx] = rr;
                }
            }
            const float y = (accept ? dS[0] : 0.0f) - S_lo;
            const float t = S_hi + y;
            S_lo = (t - S_hi) - y;
            S_hi = t;
            n_acc += accept ? 1ull : 0ull;
        }

        // ---- Eq. (6) for the window's moves, in order, on the lane's own cells:
        // gathered value + updates of the earlier moves of the window on the
        // same cell + this move's update (unchanged value where nothing moved) ----
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
#pragma unroll
            for (int s = 0; s < JMAX; ++s) {
                float c0 = v0[j][s], c1 = v1[j][s];
                int e = 0;
#pragma unroll
                for (int i = 0; i < kWin; ++i)
#pragma unroll
                    for (int jj = i + 1; jj < kWin; ++jj) {
                        if (jj == j) {
                            c0 = fmaf(df[i], sh0[e][s], c0);
                            c1 = fmaf(df[i], sh1[e][s], c1);
                        }
                        ++e;
                    }
                if (SMEM) {
                    float* q = x.R + rowbase[s] + k[j][s];
                    q[0] = fmaf(df[j], l0[j][s], c0);
                    q[1] = fmaf(df[j], l1[j][s], c1);
                } else {
                    __stcg(x.R + resid_cell(rowbase[s], k[j][s], x.il), fmaf(df[j], l0[j][s], c0));
                    __stcg(x.R + resid_cell(rowbase[s], k[j][s] + 1, x.il), fmaf(df[j], l1[j][s], c1));
                }
            }
            stcg_if(pc[j] >= 0, x.img + (pc[j] >= 0 ? pc[j] : 0), fnew[j]);  // no store past the last move
        }
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
            pw_prev[j] = pc[j];
            fw_prev[j] = fnew[j];
        }
    }
    cp_async_wait_pending(0);
}

// Task loop of one warp with its residual in shared memory (gb, window_bytes
// of shared memory; barrier id 1 + warp).
template <int RT, bool SMEM, int JMAX, int KMAX, bool NT>
__device__ __forceinline__ void window_warp(const SatArgs& a, unsigned char* gb, int warp, int lane) {
    GroupShared G;
    G.bar = reinterpret_cast<uint64_t*>(gb);
    G.part = reinterpret_cast<float*>(gb + kPartOffset);
    G.flags = reinterpret_cast<volatile int*>(gb + kFlagsOffset);
    G.pix = reinterpret_cast<int*>(gb + kGroupHeader);
    G.draws = reinterpret_cast<uint32_t*>(gb + kGroupHeader + ring_slots(KMAX) * 4);
    G.stages = gb + group_ring_bytes(1, KMAX);
    float* rs = reinterpret_cast<float*>(G.stages + (size_t)2 * kWin * a.stage_bytes);

    for (int e = lane; e < 2 * kWin * a.stage_bytes / 16; e += 32)
        reinterpret_cast<uint4*>(G.stages)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (lane == 0) {
        mbar_init(G.bar, 1);
        for (int i = 0; i < 8; ++i) G.flags[i] = 0;
    }
    fence_proxy_async_smem();
    if (lane == 0) fence_barrier_init();
    __syncwarp();

    // Cell (u, k) of the residual: R[rowbase + k].  In shared memory only the
    // band of bins [band_lo, band_lo + band_pitch) is kept, so a row starts
    // band_lo cells before its first kept cell; every record of a
    // reconstruction-space pixel addresses cells inside the band.  Lanes past
    // the last angle address two dummy cells of their own.
    const int rpitch = SMEM ? a.band_pitch : a.pitch;
    const int rshift = SMEM ? a.band_lo : 0;
    const int il = SMEM ? 0 : a.resid_il;  // global residual with interleaved row pairs (their stride)
    int rowbase[JMAX];
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        const int u = rt_record_of<RT>(lane, 1, j);
        rowbase[j] = u < a.U ? resid_row_base(u, rpitch, il) - rshift : resid_rows_end(a.U, rpitch, il) + 2 * lane;
    }
    if (SMEM) {
        rs[a.U * rpitch + 2 * lane] = 0.0f;
        rs[a.U * rpitch + 2 * lane + 1] = 0.0f;
    }

    uint32_t phase = 0;
    // Ready-first scheduling (a.claim set): a warp takes the next stages of
    // any chain that is neither running nor finished, so no warp waits on a
    // chain another warp is still running (warps of different speed share
    // the chains).  Otherwise tasks come in (stage block, chain) order from a
    // counter and a task waits for its chain's earlier stages.
    int scan = (int)(((unsigned)blockIdx.x * 8u + (unsigned)warp) * 37u % (unsigned)max(1, a.n_chains));
    for (;;) {
        int c = -1, s0 = 0;
        if (a.claim) {
            const unsigned long long t_start = global_ns();
            for (;;) {
                int got = -1;
                for (int base = 0; base < a.n_chains && got < 0; base += 32) {
                    const int q = scan + base + lane;
                    const int cq = q % a.n_chains;
                    const bool ready = base + lane < a.n_chains && ld_acquire(&a.claim[cq]) == 0 &&
                                       ld_acquire(&a.progress[cq]) < a.sweep_end;
                    unsigned m = __ballot_sync(0xffffffffu, ready);
                    while (m && got < 0) {
                        const int l = __ffs(m) - 1;
                        m &= m - 1;
                        int won = 0;
                        if (lane == l) won = atomicCAS(&a.claim[cq], 0, 1) == 0 ? 1 : 0;
                        won = __shfl_sync(0xffffffffu, won, l);
                        if (won) got = __shfl_sync(0xffffffffu, cq, l);
                    }
                }
                if (got >= 0) {
                    c = got;
                    scan = (got + 1) % a.n_chains;
                    break;
                }
                int all_done = 0;
                if (lane == 0) all_done = ld_acquire(a.task_counter) >= a.n_chains ? 1 : 0;
                if (__shfl_sync(0xffffffffu, all_done, 0)) break;
                if (global_ns() - t_start > a.wait_ns) {
                    if (lane == 0) raise_error(a.error, SATPILA_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(512);
            }
            if (c < 0) break;
            if (lane == 0) s0 = ld_acquire(&a.progress[c]);
            s0 = __shfl_sync(0xffffffffu, s0, 0);
            if (s0 >= a.sweep_end) {  // finished meanwhile: hand it back
                if (lane == 0) st_release(&a.claim[c], 0);
                continue;
            }
        } else {
            int t = 0;
            if (lane == 0) t = atomicAdd(a.task_counter, 1);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= a.n_tasks) break;
            c = t % a.n_chains;
            const int blk = t / a.n_chains;
            s0 = a.sweep_begin + blk * a.sweeps_per_task;
            if (blk > 0) {
                int ok = 1;
                if (lane == 0) ok = wait_progress(&a.progress[c], s0, a.wait_ns) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) raise_error(a.error, SATPILA_ERR_TIMEOUT);
                    break;
                }
            }
        }
        const int s1 = min(s0 + a.sweeps_per_task, a.sweep_end);
        float* gres = a.resid + (long long)c * a.resid_floats;
        if (SMEM) {
            // The band of every residual row into shared memory, one bulk copy
            // (TMA) per row, all completing on one barrier phase.
            int ok = 1;
            const uint32_t row_bytes = (uint32_t)a.band_pitch * 4u;
            fence_proxy_async_smem();  // earlier generic accesses to the band before the async-proxy writes
            fence_proxy_async_global();  // the chain's residual as the previous task left it
            if (lane == 0) {
                mbar_arrive_expect_tx(G.bar, row_bytes * (uint32_t)a.U);
            }
            __syncwarp();
            for (int u = lane; u < a.U; u += 32)
                bulk_copy_g2s(rs + (long long)u * a.band_pitch, gres + (long long)u * a.pitch + a.band_lo, row_bytes,
                              G.bar);
            ok = mbar_wait_bounded(G.bar, phase) ? 1 : 0;
            ok = __all_sync(0xffffffffu, ok);
            phase ^= 1u;
            if (!ok) {
                if (lane == 0) raise_error(a.error, SATPILA_ERR_TIMEOUT);
                break;
            }
        }
        const double S = a.S[c];
        float S_hi = (float)S;
        float S_lo = -(float)(S - (double)S_hi);
        unsigned long long n_acc = 0;
        unsigned n_ties = 0;
        StageCtx x;
        x.M = a.moves;
        x.D = a.D;
        x.W = 1;
        x.wig = 0;
        x.lane = lane;
        x.gid = 1 + warp;
        x.gl = lane;
        x.il = il;
        x.R = SMEM ? rs : gres;
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
            if (x.tracing) run_stage_window<RT, SMEM, JMAX, KMAX, 1, NT, true>(a, G, x, S_hi, S_lo, n_acc, n_ties, rowbase);
            else run_stage_window<RT, SMEM, JMAX, KMAX, 1, NT, false>(a, G, x, S_hi, S_lo, n_acc, n_ties, rowbase);
            if (a.sweep_cost && lane == 0)
                a.sweep_cost[(long long)c * a.n_sweeps_total + s] = sqrt(((double)S_hi - (double)S_lo) * a.inv_BU_d);
        }
        __syncwarp();
        if (SMEM) {
            const int q4 = a.band_pitch / 4;
            for (int e = lane; e < a.U * q4; e += 32) {
                const int u = e / q4, q = e - u * q4;
                *reinterpret_cast<float4*>(gres + (long long)u * a.pitch + a.band_lo + 4 * q) =
                    *reinterpret_cast<const float4*>(rs + (long long)u * a.band_pitch + 4 * q);
            }
        }
        if (lane == 0) {
            a.S[c] = (double)S_hi - (double)S_lo;
            a.accepted[c] += n_acc;
            if (NT) a.ties[c] += n_ties;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0 && report_progress(a, c, s0)) {  // a stalled chain also stays claimed
            st_release(&a.progress[c], s1);
            if (a.claim) {
                if (s1 >= a.sweep_end) atomicAdd(a.task_counter, 1);  // chains finished in this launch
                st_release(&a.claim[c], 0);
            }
        }
    }
}

template <int RT, bool SMEM, int JMAX, int KMAX, bool NT>
__global__ void __launch_bounds__(kSatMaxWarps * 32) sat_window_kernel(const SatArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    window_warp<RT, SMEM, JMAX, KMAX, NT>(a, smem + (size_t)warp * a.group_smem_bytes, warp, lane);
}

// Both kinds of warp in one CTA, pulling from the same task queue: the first
// a.hybrid_smem_warps warps keep the residual in shared memory, the others
// work on it in global memory.  Both run the same windowed arithmetic, so a
// chain's result does not depend on which warps ran its stages; faster warps
// simply take more tasks.
template <int RT, int JMAX, int KMAX, bool NT>
__global__ void __launch_bounds__(kSatMaxWarps * 32) sat_hybrid_kernel(const SatArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ns = a.hybrid_smem_warps;
    if (warp < ns) {
        window_warp<RT, true, JMAX, KMAX, NT>(a, smem + (size_t)warp * a.group_smem_bytes, warp, lane);
    } else {
        const int g = warp - ns;
        window_warp<RT, false, JMAX, KMAX, NT>(
            a, smem + (size_t)ns * a.group_smem_bytes + (size_t)g * a.hybrid_glob_bytes, warp, lane);
    }
}

// Task loop of a chain group: WG warps that split the chain's angles (group
// lane gl = lane + 32 * wig, named barrier 1 + grp), residual in global
// memory.  Every warp takes every decision itself (the same sums, draws and
// pixel values) and writes the same pixel values, so the warps exchange
// only the window sums; the residual cells of an angle belong to one lane.
// MULTI: the launch carries chains of several tables (a.classes); a task's
// table, geometry and chain arrays come from its chain's class.
template <int RT, int JMAX, int KMAX, int WG, bool NT, bool SMEM, bool MULTI>
__device__ __forceinline__ void window_group(const SatArgs& a, unsigned char* gb, int grp, int wig, int lane) {
    static_assert(!(MULTI && SMEM), "launches over several tables keep the residual in global memory");
    GroupShared G;
    G.bar = reinterpret_cast<uint64_t*>(gb);
    G.part = reinterpret_cast<float*>(gb + kPartOffset);
    G.flags = reinterpret_cast<volatile int*>(gb + kFlagsOffset);
    G.pix = reinterpret_cast<int*>(gb + kGroupHeader + wig * draw_ring_bytes(KMAX));
    G.draws = reinterpret_cast<uint32_t*>(gb + kGroupHeader + wig * draw_ring_bytes(KMAX) + ring_slots(KMAX) * 4);
    G.stages = gb + group_ring_bytes(WG, KMAX);
    float* rs = reinterpret_cast<float*>(G.stages + (size_t)2 * kWin * a.stage_bytes);  // SMEM: the band
    const int gl = lane + 32 * wig, gid = 1 + grp;

    for (int e = gl; e < 2 * kWin * a.stage_bytes / 16; e += 32 * WG)
        reinterpret_cast<uint4*>(G.stages)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (gl == 0) {
        for (int i = 0; i < 8; ++i) G.flags[i] = 0;
        if (SMEM) mbar_init(G.bar, 1);
    }
    if (SMEM) {
        fence_proxy_async_smem();
        if (gl == 0) fence_barrier_init();
    }
    group_sync(gid, WG);

    // Cell (u, k) of the residual: R[rowbase + k]; group lanes past the last
    // angle address two dummy cells of their own after the rows.  In shared
    // memory only the band of bins [band_lo, band_lo + band_pitch) is kept
    // (every record of a reconstruction-space pixel addresses cells inside it),
    // each warp of the group reading and writing the rows of its own angles.
    auto row_bases = [&](const SatArgs& g, int (&rb)[JMAX]) {
        const int rpitch = SMEM ? g.band_pitch : g.pitch;
        const int rshift = SMEM ? g.band_lo : 0;
        const int il = SMEM ? 0 : g.resid_il;  // global residual with interleaved row pairs (their stride)
#pragma unroll
        for (int j = 0; j < JMAX; ++j) {
            const int u = rt_record_of<RT>(gl, WG, j);
            rb[j] = u < g.U ? resid_row_base(u, rpitch, il) - rshift : resid_rows_end(g.U, rpitch, il) + 2 * gl;
        }
    };
    int rowbase[JMAX];
    if (!MULTI) row_bases(a, rowbase);
    if (SMEM) {
        rs[a.U * a.band_pitch + 2 * gl] = 0.0f;
        rs[a.U * a.band_pitch + 2 * gl + 1] = 0.0f;
    }

    uint32_t phase = 0;
    // Stages [s0, s1) of chain ci of the arguments ca (launch chain c);
    // false when a wait ran out (the group leaves together).
    auto run_task = [&](const SatArgs& ca, int ci, int c, int s0, int s1, const int (&rb)[JMAX]) -> bool {
        float* gres = ca.resid + (long long)ci * ca.resid_floats;
        if (SMEM) {
            // The band of every residual row into shared memory, one bulk copy
            // per row spread over the group's lanes, all completing on one
            // barrier phase; the group leaves together if the wait runs out.
            const uint32_t row_bytes = (uint32_t)ca.band_pitch * 4u;
            fence_proxy_async_smem();    // earlier generic accesses to the band before the async-proxy writes
            fence_proxy_async_global();  // the chain's residual as the previous task left it
            if (gl == 0) {
                G.flags[3] = 1;
                mbar_arrive_expect_tx(G.bar, row_bytes * (uint32_t)ca.U);
            }
            group_sync(gid, WG);
            for (int u = gl; u < ca.U; u += 32 * WG)
                bulk_copy_g2s(rs + (long long)u * ca.band_pitch, gres + (long long)u * ca.pitch + ca.band_lo, row_bytes,
                              G.bar);
            const bool landed = __all_sync(0xffffffffu, mbar_wait_bounded(G.bar, phase));
            phase ^= 1u;
            if (!landed && lane == 0) G.flags[3] = 0;
            group_sync(gid, WG);
            const int ok = G.flags[3];
            group_sync(gid, WG);
            if (!ok) {
                if (gl == 0) raise_error(a.error, SATPILA_ERR_TIMEOUT);
                return false;
            }
        }
        const double S = ca.S[ci];
        float S_hi = (float)S;
        float S_lo = -(float)(S - (double)S_hi);
        unsigned long long n_acc = 0;
        unsigned n_ties = 0;
        StageCtx x;
        x.M = ca.moves;
        x.D = a.D;
        x.W = WG;
        x.wig = wig;
        x.lane = lane;
        x.gid = gid;
        x.gl = gl;
        x.il = SMEM ? 0 : ca.resid_il;
        x.R = SMEM ? rs : gres;
        x.img = ca.img + (long long)ci * ca.img_stride;
        const ChainCtl* cc = ca.ctl ? ca.ctl + ci : nullptr;
        const int s_base = cc ? cc->stage0 : 0, s_total = cc ? cc->n_sweeps : ca.n_sweeps_total;
        const int sched = cc ? cc->schedule : ca.schedule;
        x.key = chain_key(cc ? cc->seed : ca.seed + (unsigned long long)ci);
        x.tracing = ca.trace != nullptr && ci == ca.trace_chain;
        const double T0 = ca.T0[ci], TN = ca.TN[ci];
        for (int s = s0; s < s1 && s_base + s < s_total; ++s) {
            x.s = s_base + s;
            x.T = (float)stage_temperature(sched, T0, TN, x.s, s_total);
            if (x.tracing) run_stage_window<RT, SMEM, JMAX, KMAX, WG, NT, true>(ca, G, x, S_hi, S_lo, n_acc, n_ties, rb);
            else run_stage_window<RT, SMEM, JMAX, KMAX, WG, NT, false>(ca, G, x, S_hi, S_lo, n_acc, n_ties, rb);
            if (ca.sweep_cost && gl == 0)
                ca.sweep_cost[(long long)ci * ca.n_sweeps_total + s] = sqrt(((double)S_hi - (double)S_lo) * ca.inv_BU_d);
        }
        if (SMEM) {
            group_sync(gid, WG);  // every warp's cells of the band are written
            const int q4 = ca.band_pitch / 4;
            for (int e = gl; e < ca.U * q4; e += 32 * WG) {
                const int u = e / q4, q = e - u * q4;
                *reinterpret_cast<float4*>(gres + (long long)u * ca.pitch + ca.band_lo + 4 * q) =
                    *reinterpret_cast<const float4*>(rs + (long long)u * ca.band_pitch + 4 * q);
            }
        }
        if (gl == 0) {
            ca.S[ci] = (double)S_hi - (double)S_lo;
            ca.accepted[ci] += n_acc;
            if (NT) ca.ties[ci] += n_ties;
        }
        __threadfence();
        group_sync(gid, WG);
        if (gl == 0 && report_progress(a, c, s0)) st_release(&a.progress[c], s1);
        return true;
    };

    for (;;) {
        if (gl == 0) G.flags[0] = atomicAdd(a.task_counter, 1);
        group_sync(gid, WG);
        const int t = G.flags[0];
        group_sync(gid, WG);
        if (t >= a.n_tasks) break;
        const int c = t % a.n_chains;
        const int blk = t / a.n_chains;
        const int s0 = a.sweep_begin + blk * a.sweeps_per_task;
        const int s1 = min(s0 + a.sweeps_per_task, a.sweep_end);
        if (blk > 0) {
            if (gl == 0) G.flags[2] = wait_progress(&a.progress[c], s0, a.wait_ns) ? 1 : 0;
            group_sync(gid, WG);
            const int ok = G.flags[2];
            group_sync(gid, WG);
            if (!ok) {
                if (gl == 0) raise_error(a.error, SATPILA_ERR_TIMEOUT);
                break;
            }
        }
        if constexpr (MULTI) {
            const int2 m = a.chain_map[c];
            const SatArgs ca = a.classes[m.x];
            int rb[JMAX];
            row_bases(ca, rb);
            if (!run_task(ca, m.y, c, s0, s1, rb)) break;
        } else {
            if (!run_task(a, c, c, s0, s1, rowbase)) break;
        }
    }
}

template <int RT, int JMAX, int KMAX, int WG, bool NT, bool SMEM = false, bool MULTI = false>
__global__ void __launch_bounds__(kSatMaxWarps * 32) sat_window_group_kernel(const SatArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = warp / WG;
    window_group<RT, JMAX, KMAX, WG, NT, SMEM, MULTI>(a, smem + (size_t)grp * a.group_smem_bytes, grp, warp % WG,
                                                      lane);
}

}  // namespace satpila
