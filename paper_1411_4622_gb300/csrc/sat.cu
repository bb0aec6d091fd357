// sat_run: orchestration of the annealer on the device.
//
// Order of work for a batch of chains (Steps 1-4 of Sec. II-A):
//   1. FP64-grade resync: residual r = P(f0) - P_m and S = sum r^2 (Eq. (4));
//   2. initial temperature per chain, given or by Eq. (8);
//   3. windows of `resync_every` stages: the persistent sweep kernel, then a
//      fresh resync that records the incremental drift;
//   4. final resync and Eq. (4) cost.
// All launches of a call are recorded once into a CUDA graph and replayed
// (unless SAT_FLAG_NO_GRAPH), so a repeated call costs one graph launch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <list>
#include <memory>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "sat_host.h"
#include "sat_sweep.cuh"
#include "sat_window.cuh"

namespace satpila {

using SweepFn = void (*)(const SatArgs);
SweepFn sweep_kernel_f32_smem(int jmax, int kmax);
SweepFn sweep_kernel_f32_glob(int jmax, int kmax);
SweepFn sweep_kernel_f16_smem(int jmax, int kmax);
SweepFn sweep_kernel_f16_glob(int jmax, int kmax);
SweepFn window_kernel(int rt, bool smem, int jmax, int kmax);
SweepFn hybrid_kernel(int rt, int jmax, int kmax);
SweepFn bome_kernel(bool f16, int jmax, int kmax);
SweepFn window_group_kernel(int rt, int jmax, int kmax, int warps_per_chain);
SweepFn window_kernel_nt(int rt, bool smem, int jmax, int kmax);
SweepFn hybrid_kernel_nt(int rt, int jmax, int kmax);
SweepFn window_group_kernel_nt(int rt, int jmax, int kmax, int warps_per_chain);
SweepFn window_group_smem_kernel(int rt, int jmax, int kmax, int warps_per_chain);
SweepFn window_group_smem_kernel_nt(int rt, int jmax, int kmax, int warps_per_chain);
SweepFn window_multi_kernel(int rt);
int bome_warps_per_cta();

namespace {

// kind: 0 pipelined, 1 windowed, 2 hybrid, 3 independent-pixel BoME, 4 and 5
// windowed on groups of 2 and 4 warps per chain; rt: the table precision
// (one-byte tables are read by the one-warp windowed kernel only)
SweepFn sweep_kernel(int rt, bool smem, int jmax, int kmax, int kind = 0, bool nt = false) {
    if (kind == 1) return nt ? window_kernel_nt(rt, smem, jmax, kmax) : window_kernel(rt, smem, jmax, kmax);
    if (kind == 4 || kind == 5) {
        const int wpc = kind == 4 ? 2 : 4;
        if (smem)
            return nt ? window_group_smem_kernel_nt(rt, jmax, kmax, wpc) : window_group_smem_kernel(rt, jmax, kmax, wpc);
        return nt ? window_group_kernel_nt(rt, jmax, kmax, wpc) : window_group_kernel(rt, jmax, kmax, wpc);
    }
    if (rt == PILA_U8) return nullptr;
    const bool f16 = rt == PILA_F16;
    if (kind == 2) return nt ? hybrid_kernel_nt(rt, jmax, kmax) : hybrid_kernel(rt, jmax, kmax);
    if (kind == 3) return bome_kernel(f16, jmax, kmax);
    if (f16) return smem ? sweep_kernel_f16_smem(jmax, kmax) : sweep_kernel_f16_glob(jmax, kmax);
    return smem ? sweep_kernel_f32_smem(jmax, kmax) : sweep_kernel_f32_glob(jmax, kmax);
}

int kmax_for(int K) { return K <= 4 ? 4 : K <= 8 ? 8 : 32; }

// The kernel's shared-memory limit must have been set (prepare_launches).
cudaError_t launch_sweep(int rt, bool smem, int kind, bool nt, int jmax, int kmax, const SatArgs& a, int grid,
                         int warps, size_t smem_bytes, cudaStream_t s) {
    SweepFn k = sweep_kernel(rt, smem, jmax, kmax, kind, nt);
    if (!k) return cudaErrorInvalidValue;
    k<<<grid, warps * 32, smem_bytes, s>>>(a);
    return cudaGetLastError();
}

// The shared-memory limit of a sweep kernel is set to the device maximum
// once: the attribute belongs to the function, so a per-launch value would
// be lowered under other callers (other sat_run calls, serving classes)
// launching the same function with more.
cudaError_t allow_max_smem(SweepFn k) {
    int dev = 0, maxopt = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, maxopt);
    return e;
}

int sweep_blocks_per_sm(int rt, bool smem, int kind, int jmax, int kmax, int warps, size_t smem_bytes) {
    SweepFn k = sweep_kernel(rt, smem, jmax, kmax, kind);
    if (!k) return 0;
    if (allow_max_smem(k) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem_bytes) != cudaSuccess) return 0;
    return nb;
}

}  // namespace

namespace {

template <int RT>
__global__ void __launch_bounds__(256) t0_kernel(const T0Args a) {
    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ float dcs[32];
    __shared__ double total_s;
    __shared__ int found_s, done_s;
    const ChainCtl* cc = a.ctl ? a.ctl + c : nullptr;
    const double t0_fixed = cc ? cc->t0 : a.t0_fixed, tn = cc ? cc->tn : a.tn;
    const int Q = cc ? (cc->t0_samples > 0 ? cc->t0_samples : 200) : a.Q;
    if (t0_fixed > 0.0) {
        if (tid == 0) {
            a.T0[c] = t0_fixed;
            a.TN[c] = tn < 0.0 ? t0_fixed / 1000.0 : tn;
            a.found[c] = 0;
        }
        return;
    }
    const uint2 key = chain_key(cc ? cc->seed : a.seed + (unsigned long long)c);
    const float* R = a.resid + (long long)c * a.resid_floats;
    const float* img = a.img + (long long)c * a.img_stride;
    const float C2 = (float)(a.S[c] * a.inv_BU_d);
    const float C = sqrtf(C2);
    const long long max_tries = 100LL * Q;
    const uint32_t nl = (uint32_t)a.n_list;
    if (tid == 0) {
        total_s = 0.0;
        found_s = 0;
        done_s = 0;
    }
    __syncthreads();
    for (long long base = 0; base < max_tries && a.n_list > 0; base += 32) {
        for (int i = 0; i < 4; ++i) {
            const long long t = base + warp * 4 + i;
            float dC = -1.0f;
            if (t < max_tries) {
                const uint4 x = philox4x32_10(make_uint4((uint32_t)t, 0u, 0u, kStreamT0), key);
                const uint32_t idx = pick_index(x.x, nl);
                const int p = a.list ? a.list[idx] : (int)idx;
                const float f = img[p];
                const float lo = fmaxf(0.0f, f - a.beta), hi = fminf(a.beta, f + a.beta);
                const float df = fmaf(unit_uniform(x.z), hi - lo, lo) - f;
                float g = 0.0f, h = 0.0f;
                const unsigned char* row = a.table + (long long)p * a.row_stride;
                for (int u = lane; u < a.U; u += 32) {
                    const Entry2 e = decode_rec(row, u, RT);
                    if (e.l0 != 0.0f) {
                        g = fmaf(R[resid_cell(resid_row_base(u, a.pitch, a.resid_il), e.k0, a.resid_il)], e.l0, g);
                        h = fmaf(e.l0, e.l0, h);
                    }
                    if (e.l1 != 0.0f) {
                        g = fmaf(R[resid_cell(resid_row_base(u, a.pitch, a.resid_il), e.k1, a.resid_il)], e.l1, g);
                        h = fmaf(e.l1, e.l1, h);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    g += __shfl_xor_sync(0xffffffffu, g, o);
                    h += __shfl_xor_sync(0xffffffffu, h, o);
                }
                const float dS = df * fmaf(df, h, 2.0f * g);
                const float xx = dS * a.inv_BU;
                const float Cp = sqrtf(fmaxf(0.0f, C2 + xx));
                const float den = Cp + C;
                dC = den > 0.0f ? xx / den : 0.0f;
            }
            if (lane == 0) dcs[warp * 4 + i] = dC;
        }
        __syncthreads();
        if (tid == 0) {
            for (int q = 0; q < 32 && found_s < Q; ++q) {
                if (base + q >= max_tries) break;
                if (dcs[q] > 0.0f) {
                    total_s += (double)dcs[q];
                    ++found_s;
                }
            }
            if (found_s >= Q) done_s = 1;
        }
        __syncthreads();
        if (done_s) break;
    }
    if (tid == 0) {
        // Eq. (8): T0 = -sum(C' - C) / (Q ln 0.9)
        const double t0 = found_s > 0 ? -total_s / ((double)found_s * log(0.9)) : 0.0;
        a.T0[c] = t0;
        a.TN[c] = tn < 0.0 ? t0 / 1000.0 : tn;
        a.found[c] = found_s;
    }
}

// Device global-timer stamp (ns), for timing launches inside a CUDA graph.
__global__ void stamp_kernel(unsigned long long* out) { *out = global_ns(); }

__global__ void copy_f64_kernel(double* dst, const double* src, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i];
}

}  // namespace

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int plan_code(const Plan& pl) {
    switch (pl.kind) {
        case 1: return pl.smem ? PLAN_WINDOW_SMEM : PLAN_WINDOW_GLOBAL;
        case 2: return PLAN_WINDOW_HYBRID;
        case 0: return pl.W == 1 ? PLAN_PIPE_1 : pl.W == 2 ? PLAN_PIPE_2 : PLAN_PIPE_4;
        case 4: return pl.smem ? PLAN_WINDOW_SMEM_G2 : PLAN_WINDOW_G2;
        case 5: return pl.smem ? PLAN_WINDOW_SMEM_G4 : PLAN_WINDOW_G4;
        default: return PLAN_RULES;  // the independent-pixel BoME kernel
    }
}

size_t Plan::sweep_smem_bytes() const {
    return kind == 2 ? (size_t)hybrid_smem_warps * group_smem + (size_t)(warps - hybrid_smem_warps) * hybrid_glob_bytes
                     : (size_t)groups * group_smem;
}

namespace {
int choose_plan_layout(const satpila_pila* p, int n_chains, int window, const sat_params* prm, int variant, Plan* pl);
}

// The launch layout, then the residual's storage: layouts that gather their
// cells from global memory keep its rows in interleaved pairs (one DRAM
// access serves neighbouring angles), the others plain rows.
int choose_plan(const satpila_pila* p, int n_chains, int window, const sat_params* prm, int variant, Plan* pl) {
    const int rc = choose_plan_layout(p, n_chains, window, prm, variant, pl);
    if (rc != SATPILA_OK) return rc;
    const bool gathers = !pl->smem && (pl->kind == 0 || pl->kind == 1 || pl->kind == 4 || pl->kind == 5);
    // pair stride: the records per 16-byte chunk of the table
    pl->resid_il = gathers ? (p->precision == PILA_U8 ? 4 : p->precision == PILA_F16 ? 2 : 1) : 0;
    if (pl->resid_il) {
        pl->pitch = (int)align_up((size_t)p->B + 1, 8);
        pl->resid_floats =
            (long long)align_up((size_t)resid_rows_end(p->U, pl->pitch, pl->resid_il) + 64 * kMaxGroupWarps, 4);
    }
    return SATPILA_OK;
}

namespace {
int choose_plan_layout(const satpila_pila* p, int n_chains, int window, const sat_params* prm, int variant, Plan* pl) {
    if (variant == PLAN_RULES && (prm->flags & SAT_FLAG_WINDOW_GROUPS)) {
        if (prm->group_warps != 2 && prm->group_warps != 4)
            return fail(SATPILA_ERR_INVALID_ARG, "sat_run: SAT_FLAG_WINDOW_GROUPS needs group_warps 2 or 4");
        variant = prm->group_warps == 2 ? PLAN_WINDOW_G2 : PLAN_WINDOW_G4;
    }
    const int rt = p->precision;
    const bool f16 = rt == PILA_F16;
    const int rpc = rt == PILA_U8 ? 4 : f16 ? 2 : 1;  // records per 16-byte chunk
    int dev = 0, maxopt = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Warps per chain: the fewest that leave each lane at most two records
    // (four for very many angles).
    auto records_per_lane = [&](int W) {
        return rpc * ((p->row_records + 32 * rpc * W - 1) / (32 * rpc * W));
    };
    // Rows of B + 1 cells (the last one private to the row's lane; rows padded
    // to 16 bytes), then 2 dummy cells per lane of a group.
    pl->pitch = (int)align_up((size_t)p->B + 1, 4);
    pl->resid_floats = (long long)align_up((size_t)p->U * pl->pitch + 64 * kMaxGroupWarps, 4);
    // A windowed warp keeps in shared memory only the band of bins that moves
    // can touch (for a disk-shaped reconstruction space about n + 2 of the B
    // bins), rows 16-byte aligned so that each row is one bulk copy, then 2
    // dummy cells per lane.
    pl->band_lo = p->band_lo & ~3;
    pl->band_pitch = (int)align_up((size_t)(p->band_hi + 1 - pl->band_lo), 4);
    pl->band_floats = (long long)p->U * pl->band_pitch + 64;
    if (p->B > projector_max_bins()) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: too many bins");
    pl->proj_G = p->U;  // per-angle partial sums of the resync, per chain
    pl->geo_n = p->n;
    pl->geo_U = p->U;
    pl->geo_B = p->B;
    pl->rays = p->d_ray_off != nullptr;
    pl->variant = variant;
    // Sec. III-B as written (an independent pixel per estimate): its own
    // kernel, one warp per chain, residual in global memory.
    if (prm->flags & SAT_FLAG_BOME_INDEPENDENT) {
        if (rt == PILA_U8) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: one-byte tables are read by the windowed kernel only");
        if (prm->residency == SAT_RESIDENT_SMEM)
            return fail(SATPILA_ERR_INVALID_ARG, "sat_run: independent-pixel BoME keeps the residual in global memory");
        const int J = records_per_lane(1);
        int jmax = 0;
        for (int c : {2, 4, 8, 16})
            if (J <= c) {
                jmax = c;
                break;
            }
        if (!jmax) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: too many angles for independent-pixel BoME");
        pl->kind = 3;
        pl->smem = false;
        pl->W = 1;
        pl->J = pl->jmax = jmax;
        pl->D = 2;
        pl->stage_bytes = 512 * (jmax / rpc);
        pl->group_smem = (int)align_up((size_t)2 * prm->bome_k * pl->stage_bytes, 128);
        const int warps = std::max(1, std::min(bome_warps_per_cta(), maxopt / pl->group_smem));
        pl->groups = pl->warps = std::min(warps, std::max(1, n_chains));
        int per_sm = sweep_blocks_per_sm(rt, false, 3, jmax, kmax_for(prm->bome_k), pl->warps,
                                         (size_t)pl->warps * pl->group_smem);
        if (per_sm < 1) per_sm = 1;
        const long long slots = (long long)sms * per_sm * pl->warps;
        pl->spt = n_chains <= slots ? window : 1;
        const long long tasks = (long long)n_chains * ((window + pl->spt - 1) / pl->spt);
        const long long want = (std::min<long long>(tasks, slots) + pl->warps - 1) / pl->warps;
        pl->grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * per_sm));
        return SATPILA_OK;
    }
    // The windowed kernel on groups of 2 or 4 warps per chain (their lanes
    // split the angles) with the residual band in shared memory: the chain's
    // per-move record work split over warps on different schedulers.
    if (variant == PLAN_WINDOW_SMEM_G2 || variant == PLAN_WINDOW_SMEM_G4) {
        const int Wg = variant == PLAN_WINDOW_SMEM_G2 ? 2 : 4;
        if (rt == PILA_U8 || prm->residency == SAT_RESIDENT_GLOBAL || records_per_lane(Wg) > 4)
            return fail(SATPILA_ERR_INVALID_ARG, "sat_run: no windowed shared-memory group launch for this table");
        const int jw = records_per_lane(Wg) <= 2 ? 2 : 4;
        const int stage = 512 * Wg * (jw / rpc);
        const long long band_floats = (long long)p->U * pl->band_pitch + 64LL * Wg;  // then 2 dummy cells per lane
        const size_t gsm =
            align_up(group_ring_bytes(Wg, kmax_for(prm->bome_k)) + (size_t)2 * kWin * stage + (size_t)band_floats * 4, 128);
        const int kmax = kmax_for(prm->bome_k);
        const int groups = std::min(kSatMaxWarps / Wg, std::min(std::max(1, n_chains), (int)(maxopt / gsm)));
        if (groups < 1) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: residual band does not fit in shared memory");
        pl->band_floats = band_floats;
        pl->kind = Wg == 2 ? 4 : 5;
        pl->smem = true;
        pl->W = Wg;
        pl->J = pl->jmax = jw;
        pl->D = 4;
        pl->stage_bytes = stage;
        pl->group_smem = (int)gsm;
        pl->groups = groups;
        pl->warps = groups * Wg;
        int per_sm = sweep_blocks_per_sm(rt, true, pl->kind, jw, kmax, pl->warps, (size_t)groups * gsm);
        if (per_sm < 1) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: windowed shared-memory group launch does not fit");
        const long long slots = (long long)sms * per_sm * groups;
        pl->spt = n_chains <= slots ? window : 1;
        const long long tasks = (long long)n_chains * ((window + pl->spt - 1) / pl->spt);
        const long long want = (std::min<long long>(tasks, slots) + groups - 1) / groups;
        pl->grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * per_sm));
        return SATPILA_OK;
    }
    // The windowed kernel on groups of 2 or 4 warps per chain (their lanes
    // split the angles), residual in global memory: one gather round trip and
    // one exchange of sums between the warps per window of moves.  (The size
    // rules keep the pipelined kernel for wide tables: with it the serving
    // engine's mixed launches gave lower request latency.)
    if (variant == PLAN_WINDOW_G2 || variant == PLAN_WINDOW_G4) {
        const int Wg = variant == PLAN_WINDOW_G2 ? 2 : 4;
        if (prm->residency == SAT_RESIDENT_SMEM || records_per_lane(Wg) > 4)
            return fail(SATPILA_ERR_INVALID_ARG, "sat_run: no windowed group launch for this table");
        const int jw = records_per_lane(Wg) <= 2 ? 2 : 4;
        const int stage = 512 * Wg * (jw / rpc);
        const size_t glob = align_up(group_ring_bytes(Wg, kmax_for(prm->bome_k)) + (size_t)2 * kWin * stage, 128);
        const int kmax = kmax_for(prm->bome_k);
        // one chain per CTA while the chains fit one per SM, else as many as fit
        const int groups =
            n_chains <= sms ? 1 : std::max(1, std::min(kSatMaxWarps / Wg, std::min(n_chains, (int)(maxopt / glob))));
        pl->kind = Wg == 2 ? 4 : 5;
        pl->smem = false;
        pl->W = Wg;
        pl->J = pl->jmax = jw;
        pl->D = 4;
        pl->stage_bytes = stage;
        pl->group_smem = (int)glob;
        pl->groups = groups;
        pl->warps = groups * Wg;
        int per_sm = sweep_blocks_per_sm(rt, false, pl->kind, jw, kmax, pl->warps, (size_t)groups * glob);
        if (per_sm < 1) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: windowed group launch does not fit");
        const long long slots = (long long)sms * per_sm * groups;
        pl->spt = n_chains <= slots ? window : 1;
        const long long tasks = (long long)n_chains * ((window + pl->spt - 1) / pl->spt);
        const long long want = (std::min<long long>(tasks, slots) + groups - 1) / groups;
        pl->grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * per_sm));
        return SATPILA_OK;
    }
    // The windowed kernel: one warp per chain; residual in shared memory, in
    // global memory, or both kinds of warp side by side (hybrid).
    const bool window_ok = records_per_lane(1) <= 4;
    const bool use_window = variant == PLAN_RULES
                                ? prm->group_warps <= 1 && window_ok && prm->pipeline_depth == 0
                                : variant == PLAN_WINDOW_SMEM || variant == PLAN_WINDOW_GLOBAL ||
                                      variant == PLAN_WINDOW_HYBRID;
    if (use_window && !window_ok)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_run: too many angles for the windowed kernel");
    if (rt == PILA_U8 && !use_window) {
        // one-byte tables past 128 angles: the windowed move on 2 or 4 warps
        // per chain (unless the caller asked for a pipelined layout)
        const bool by_size = variant == PLAN_RULES && prm->group_warps <= 1 && prm->pipeline_depth == 0;
        if (by_size && records_per_lane(2) <= 4) return choose_plan(p, n_chains, window, prm, PLAN_WINDOW_G2, pl);
        if (by_size && records_per_lane(4) <= 4) return choose_plan(p, n_chains, window, prm, PLAN_WINDOW_G4, pl);
        return fail(SATPILA_ERR_INVALID_ARG,
                    "sat_run: one-byte tables are read by the windowed kernels only (at most 512 angles)");
    }
    if (use_window) {
        const int residency = variant == PLAN_WINDOW_SMEM     ? SAT_RESIDENT_SMEM
                              : variant == PLAN_WINDOW_GLOBAL ? SAT_RESIDENT_GLOBAL
                                                              : prm->residency;
        const bool want_hybrid = rt != PILA_U8 && (variant == PLAN_WINDOW_HYBRID ||
                                                   (variant == PLAN_RULES && (prm->flags & SAT_FLAG_HYBRID)));
        const int jw = records_per_lane(1) <= 2 ? 2 : 4;
        const int stage = 512 * (jw / rpc);
        const size_t ring1 = group_ring_bytes(1, kmax_for(prm->bome_k)) + (size_t)2 * kWin * stage;
        const size_t gsm = align_up(ring1 + (size_t)pl->band_floats * 4, 128);  // shared-memory warp
        const size_t glob = align_up(ring1, 128);                                   // global-memory warp
        const int kmax = kmax_for(prm->bome_k);
        pl->W = 1;
        pl->J = pl->jmax = jw;
        pl->D = 4;
        pl->stage_bytes = stage;
        auto finish = [&](int kind, bool smem, int warps, size_t smem_bytes, bool dynamic_tasks) {
            pl->kind = kind;
            pl->smem = smem;
            pl->groups = warps;
            pl->warps = warps;
            int per_sm = sweep_blocks_per_sm(rt, smem, kind, jw, kmax, warps, smem_bytes);
            if (per_sm < 1) per_sm = 1;
            const long long slots = (long long)sms * per_sm * warps;
            pl->spt = (!dynamic_tasks && n_chains <= slots) ? window : 1;
            const long long tasks = (long long)n_chains * ((window + pl->spt - 1) / pl->spt);
            const long long want = (std::min<long long>(tasks, slots) + warps - 1) / warps;
            pl->grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * per_sm));
            return SATPILA_OK;
        };
        const int win_per_cta = (int)std::min<size_t>(kSatMaxWarps, maxopt / gsm);
        if (residency == SAT_RESIDENT_GLOBAL || (residency == SAT_RESIDENT_AUTO && win_per_cta == 0)) {
            pl->group_smem = (int)glob;
            const int warps = std::min(4, std::max(1, n_chains));
            return finish(1, false, warps, (size_t)warps * glob, false);
        }
        if (win_per_cta == 0) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: residual does not fit in shared memory");
        const int ns = std::min(win_per_cta, 3), ng = 4 - ns;
        if (want_hybrid && ng > 0 && n_chains > sms * win_per_cta &&
            (size_t)ns * gsm + (size_t)ng * glob <= (size_t)maxopt) {
            pl->group_smem = (int)gsm;
            pl->hybrid_smem_warps = ns;
            pl->hybrid_glob_bytes = (int)glob;
            // stage-sized tasks, so that chains move between the two kinds of warp
            return finish(2, true, ns + ng, (size_t)ns * gsm + (size_t)ng * glob, true);
        }
        if (variant == PLAN_WINDOW_HYBRID)
            return fail(SATPILA_ERR_INVALID_ARG, "sat_run: no hybrid launch for this size");
        pl->group_smem = (int)gsm;
        const int warps = std::min(win_per_cta, std::max(1, n_chains));
        return finish(1, true, warps, (size_t)warps * gsm, false);
    }
    int W = variant == PLAN_PIPE_1   ? 1
            : variant == PLAN_PIPE_2 ? 2
            : variant == PLAN_PIPE_4 ? 4
                                     : (prm->group_warps > 0 ? prm->group_warps : 1);
    if (variant == PLAN_RULES && prm->group_warps <= 0)
        while (W < kMaxGroupWarps && records_per_lane(W) > 2) W *= 2;
    if (W != 1 && W != 2 && W != 4) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: group_warps must be 1, 2 or 4");
    const int J = records_per_lane(W);
    int jmax = 0;
    for (int c : {2, 4, 8, 16})
        if (J <= c) {
            jmax = c;
            break;
        }
    if (!jmax) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: too many angles for this many warps per chain");
    pl->W = W;
    pl->J = jmax;  // lanes always walk jmax records; the ones past U are zero
    pl->jmax = jmax;
    pl->D = prm->pipeline_depth > 0 ? prm->pipeline_depth : 4;
    if (pl->D < 3 || pl->D > kMaxStages) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: pipeline_depth must be in [3, 8]");
    pl->stage_bytes = 512 * W * (jmax / rpc);  // 16-byte chunks of all lanes
    const size_t ring = group_ring_bytes(W, kmax_for(prm->bome_k)) + (size_t)pl->D * pl->stage_bytes;
    const size_t smem_group = align_up(ring + (size_t)pl->resid_floats * 4, 128);
    const size_t glob_group = align_up(ring, 128);
    bool smem = false;
    if (prm->residency == SAT_RESIDENT_SMEM) {
        if (smem_group > (size_t)maxopt)
            return fail(SATPILA_ERR_INVALID_ARG, "sat_run: residual does not fit in shared memory");
        smem = true;
    } else if (prm->residency == SAT_RESIDENT_AUTO) {
        smem = smem_group <= (size_t)maxopt;
    }
    pl->smem = smem;
    pl->group_smem = (int)(smem ? smem_group : glob_group);
    // Shared-memory residuals: as many groups as fit one SM.  Global residuals:
    // four warps per CTA so that chains spread over all SMs.
    int groups = smem ? std::max<int>(1, std::min<int>(kSatMaxWarps / W, maxopt / pl->group_smem))
                      : std::max(1, 4 / W);
    groups = std::min(groups, std::max(1, n_chains));
    pl->groups = groups;
    pl->warps = groups * W;
    const size_t smem_bytes = (size_t)groups * pl->group_smem;
    int per_sm = sweep_blocks_per_sm(rt, smem, 0, jmax, kmax_for(prm->bome_k), pl->warps, smem_bytes);
    if (per_sm < 1) per_sm = 1;
    const long long slots = (long long)sms * per_sm * groups;
    pl->spt = n_chains <= slots ? window : 1;
    const long long tasks = (long long)n_chains * ((window + pl->spt - 1) / pl->spt);
    const long long want = (std::min<long long>(tasks, slots) + groups - 1) / groups;
    pl->grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * per_sm));
    return SATPILA_OK;
}
}  // namespace


namespace {

struct BatchLayout {
    size_t resid, S, T0, TN, found, acc, ties, prog, claim, err, psq, pdr, dmax, c0, cF, Sinc, rayws, bytes;
};

BatchLayout batch_layout(const Plan& pl, long long cap) {
    BatchLayout L{};
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + std::max<size_t>(bytes, 1), 256);
        return o;
    };
    const size_t n = (size_t)cap, G = (size_t)pl.proj_G;
    L.resid = carve(n * (size_t)pl.resid_floats * sizeof(float));
    L.S = carve(n * 8);
    L.T0 = carve(n * 8);
    L.TN = carve(n * 8);
    L.found = carve(n * 4);
    L.acc = carve(n * 8);
    L.ties = carve(n * 4);
    L.prog = carve(n * 4);
    L.claim = carve(n * 4);
    L.err = carve(4);
    L.psq = carve(n * G * 8);
    L.pdr = carve(n * G * 4);
    L.dmax = carve(n * 8);
    L.c0 = carve(n * 8);
    L.cF = carve(n * 8);
    L.Sinc = carve(n * 8);
    L.rayws = carve(pl.rays ? ray_ws_bytes(cap, pl.geo_U, pl.geo_B, pl.geo_n) : 0);
    L.bytes = off;
    return L;
}

}  // namespace

size_t batch_bytes(const Plan& pl, long long cap) { return batch_layout(pl, cap).bytes; }

void batch_carve(void* base, const Plan& pl, long long cap, BatchDev* b) {
    const BatchLayout L = batch_layout(pl, cap);
    char* c = (char*)base;
    b->resid = (float*)(c + L.resid);
    b->S = (double*)(c + L.S);
    b->T0 = (double*)(c + L.T0);
    b->TN = (double*)(c + L.TN);
    b->found = (int*)(c + L.found);
    b->accepted = (unsigned long long*)(c + L.acc);
    b->ties = (unsigned*)(c + L.ties);
    b->progress = (int*)(c + L.prog);
    b->claim = (int*)(c + L.claim);
    b->error = (int*)(c + L.err);
    b->part_sq = (double*)(c + L.psq);
    b->part_drift = (float*)(c + L.pdr);
    b->drift_max = (double*)(c + L.dmax);
    b->cost0 = (double*)(c + L.c0);
    b->costF = (double*)(c + L.cF);
    b->S_inc = (double*)(c + L.Sinc);
    b->proj_ws = pl.rays ? (void*)(c + L.rayws) : nullptr;
}

cudaError_t prepare_launches(const satpila_pila* p, const Plan& pl, int bome_k) {
    cudaError_t e = prepare_projector();
    if (e != cudaSuccess) return e;
    for (bool nt : {false, true}) {  // both builds of the windowed kernels: either may be launched
        SweepFn k = sweep_kernel(p->precision, pl.smem, pl.jmax, kmax_for(bome_k), pl.kind, nt);
        if (!k) {
            if (nt) break;
            return cudaErrorInvalidValue;
        }
        const cudaError_t e = allow_max_smem(k);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_resync(const satpila_pila* p, const Plan& pl, const BatchDev& b, int c0, int nc, bool drift,
                           double* cost_out, cudaStream_t q) {
    if (nc <= 0) return cudaSuccess;
    const long long P = (long long)p->n * p->n, cells = (long long)p->U * p->B;
    const int G = pl.proj_G;  // = U
    ProjArgs pa{};
    pa.table = p->d_table;
    pa.f16 = p->precision;
    pa.row_records = p->row_records;
    pa.n = p->n;
    pa.U = p->U;
    pa.B = p->B;
    pa.mode = PROJ_RESYNC;
    pa.drift = drift ? 1 : 0;
    pa.img = b.img + (long long)c0 * P;
    pa.img_stride = P;
    pa.pm = b.sino + (long long)c0 * cells;
    pa.pm_stride = cells;
    pa.resid = b.resid + (long long)c0 * pl.resid_floats;
    pa.resid_stride = pl.resid_floats;
    pa.resid_pitch = pl.pitch;
    pa.resid_il = pl.resid_il;
    pa.part_sq = b.part_sq + (long long)c0 * G;
    pa.part_drift = b.part_drift + (long long)c0 * G;
    if (b.proj_ws) use_ray_projector(pa, p, b.proj_ws);
    cudaError_t e = launch_projector(pa, nc, q);
    if (e != cudaSuccess) return e;
    ReduceArgs ra{};
    ra.n_items = nc;
    ra.n_rows = G;
    ra.part_sq = pa.part_sq;
    ra.part_drift = pa.part_drift;
    ra.inv_cells = 1.0 / (double)cells;
    ra.S_out = b.S + c0;
    ra.cost_out = cost_out ? cost_out + c0 : nullptr;
    ra.cost_stride = 1;
    ra.drift_max = drift ? b.drift_max + c0 : nullptr;
    return launch_reduce(ra, q);
}

cudaError_t enqueue_t0(const satpila_pila* p, const Plan& pl, const BatchDev& b, const sat_params* prm, int c0,
                       int nc, cudaStream_t q) {
    if (nc <= 0) return cudaSuccess;
    const long long P = (long long)p->n * p->n, cells = (long long)p->U * p->B;
    T0Args ta{};
    ta.table = p->d_table;
    ta.row_stride = p->row_bytes;
    ta.f16 = p->precision;
    ta.n = p->n;
    ta.U = p->U;
    ta.B = p->B;
    ta.pitch = pl.pitch;
    ta.resid_il = pl.resid_il;
    ta.list = p->d_list;
    ta.n_list = p->n_mask;
    ta.beta = prm->beta;
    ta.inv_BU = (float)(1.0 / (double)cells);
    ta.inv_BU_d = 1.0 / (double)cells;
    ta.resid = b.resid + (long long)c0 * pl.resid_floats;
    ta.resid_floats = pl.resid_floats;
    ta.img = b.img + (long long)c0 * P;
    ta.img_stride = P;
    ta.S = b.S + c0;
    ta.seed = prm->seed + (unsigned long long)c0;
    ta.Q = prm->t0_samples > 0 ? prm->t0_samples : 200;
    ta.tn = prm->tn;
    ta.t0_fixed = prm->t0;
    ta.T0 = b.T0 + c0;
    ta.TN = b.TN + c0;
    ta.found = b.found + c0;
    ta.ctl = b.ctl ? b.ctl + c0 : nullptr;
    if (ta.f16 == PILA_U8) t0_kernel<PILA_U8><<<nc, 256, 0, q>>>(ta);
    else if (ta.f16 == PILA_F16) t0_kernel<PILA_F16><<<nc, 256, 0, q>>>(ta);
    else t0_kernel<PILA_F32><<<nc, 256, 0, q>>>(ta);
    return cudaGetLastError();
}

SatArgs sweep_args(const satpila_pila* p, const Plan& pl, const BatchDev& b, const sat_params* prm, int n_chains,
                   int M, int s_total, int s_begin, int s_end, int* task_counter) {
    const long long P = (long long)p->n * p->n, cells = (long long)p->U * p->B;
    SatArgs sa{};
    sa.table = p->d_table;
    sa.row_stride = p->row_bytes;
    sa.row_chunks = (int)(p->row_bytes / 16);
    sa.hsum = p->d_hsum;
    sa.n = p->n;
    sa.U = p->U;
    sa.B = p->B;
    sa.pitch = pl.pitch;
    sa.resid_il = pl.resid_il;
    sa.band_lo = pl.band_lo;
    sa.band_pitch = pl.band_pitch;
    sa.band_floats = pl.band_floats;
    sa.list = p->d_list;
    sa.n_list = p->n_mask;
    sa.moves = M;
    sa.K = prm->bome_k;
    sa.beta = prm->beta;
    sa.inv_BU = (float)(1.0 / (double)cells);
    sa.inv_BU_d = 1.0 / (double)cells;
    sa.D = pl.D;
    sa.stage_bytes = pl.stage_bytes;
    sa.W = pl.W;
    sa.group_smem_bytes = pl.group_smem;
    sa.hybrid_smem_warps = pl.hybrid_smem_warps;
    sa.hybrid_glob_bytes = pl.hybrid_glob_bytes;
    sa.resid_floats = pl.resid_floats;
    sa.n_chains = n_chains;
    sa.resid = b.resid;
    sa.img = b.img;
    sa.img_stride = P;
    sa.S = b.S;
    sa.T0 = b.T0;
    sa.TN = b.TN;
    sa.seed = prm->seed;
    sa.accepted = b.accepted;
    sa.progress = b.progress;
    sa.schedule = prm->schedule;
    sa.n_sweeps_total = s_total;
    sa.error = b.error;
    sa.sweep_cost = b.sweep_cost;
    sa.trace = b.trace;
    sa.trace_chain = b.trace_chain;
    sa.trace_cap = b.trace_cap;
    sa.ctl = b.ctl;
    // ready-first scheduling where warps of different speed share the chains
    sa.claim = pl.kind == 2 ? b.claim : nullptr;
    sa.sweep_begin = s_begin;
    sa.sweep_end = s_end;
    sa.wait_ns = (unsigned long long)(prm->wait_ms > 0 ? prm->wait_ms : 20000) * 1000000ull;
    sa.stall_chain = (prm->flags & SAT_FLAG_TEST_STALL) ? 0 : -1;
    sa.ties = b.ties;
    const int spt = sa.stall_chain >= 0 ? 1 : pl.spt;  // the stall needs a second task of chain 0
    sa.sweeps_per_task = spt;
    sa.n_tasks = n_chains * ((s_end - s_begin + spt - 1) / spt);
    sa.task_counter = task_counter;
    return sa;
}

cudaError_t enqueue_sweep(const satpila_pila* p, const Plan& pl, const BatchDev& b, const sat_params* prm,
                          int n_chains, int M, int s_total, int s_begin, int s_end, int* task_counter,
                          cudaStream_t q) {
    if (n_chains <= 0 || s_end <= s_begin) return cudaSuccess;
    const SatArgs sa = sweep_args(p, pl, b, prm, n_chains, M, s_total, s_begin, s_end, task_counter);
    return launch_sweep(p->precision, pl.smem, pl.kind, sweep_counts_ties(pl, prm), pl.jmax, kmax_for(prm->bome_k), sa,
                        pl.grid, pl.warps, pl.sweep_smem_bytes(), q);
}

// ---- one launch over chains of several tables ------------------------------

bool multi_table_ok(const satpila_pila* p, const sat_params* prm) {
    const int rpc = p->precision == PILA_U8 ? 4 : p->precision == PILA_F16 ? 2 : 1;
    const int per_lane = rpc * ((p->row_records + 32 * rpc * 4 - 1) / (32 * rpc * 4));
    return per_lane <= 4 && prm->bome_k >= 1 && prm->bome_k <= 8 && prm->residency != SAT_RESIDENT_SMEM &&
           prm->group_warps <= 1 && prm->pipeline_depth == 0 && !(prm->flags & SAT_FLAG_BOME_INDEPENDENT);
}

int plan_multi(int rt, int n_chains, int window, Plan* pl) {
    SweepFn k = window_multi_kernel(rt);
    if (!k) return fail(SATPILA_ERR_INVALID_ARG, "sat_server: no launch over several tables for this precision");
    int dev = 0, maxopt = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int rpc = rt == PILA_U8 ? 4 : rt == PILA_F16 ? 2 : 1;
    constexpr int Wg = 4, jw = 4, kmax = 8;
    const int stage = 512 * Wg * (jw / rpc);
    const size_t glob = align_up(group_ring_bytes(Wg, kmax) + (size_t)2 * kWin * stage, 128);
    // one chain per CTA while the chains fit one per SM (so two chains do not
    // share an SM's schedulers while others stand idle), else two
    const int groups = n_chains <= sms ? 1 : std::max(1, std::min(kSatMaxWarps / Wg, (int)(maxopt / glob)));
    *pl = Plan{};
    pl->kind = 5;
    pl->smem = false;
    pl->W = Wg;
    pl->J = pl->jmax = jw;
    pl->D = 4;
    pl->stage_bytes = stage;
    pl->group_smem = (int)glob;
    pl->groups = groups;
    pl->warps = groups * Wg;
    cudaError_t e = allow_max_smem(k);
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, pl->warps * 32, (size_t)groups * glob);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return fail(SATPILA_ERR_INVALID_ARG, "sat_server: launch over several tables does not fit");
    }
    const long long slots = (long long)sms * per_sm * groups;
    pl->spt = n_chains <= slots ? window : 1;
    const long long tasks = (long long)n_chains * ((window + pl->spt - 1) / pl->spt);
    const long long want = (std::min<long long>(tasks, slots) + groups - 1) / groups;
    pl->grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * per_sm));
    return SATPILA_OK;
}

cudaError_t prepare_multi(int rt) {
    cudaError_t e = prepare_projector();
    SweepFn k = window_multi_kernel(rt);
    if (e == cudaSuccess) e = k ? allow_max_smem(k) : cudaErrorInvalidValue;
    return e;
}

cudaError_t enqueue_sweep_multi(int rt, const Plan& pl, const SatArgs& la, cudaStream_t q) {
    if (la.n_chains <= 0 || la.sweep_end <= la.sweep_begin) return cudaSuccess;
    SweepFn k = window_multi_kernel(rt);
    if (!k) return cudaErrorInvalidValue;
    k<<<pl.grid, pl.warps * 32, pl.sweep_smem_bytes(), q>>>(la);
    return cudaGetLastError();
}

bool sweep_counts_ties(const Plan& pl, const sat_params* prm) {
    const bool windowed = pl.kind == 1 || pl.kind == 2 || pl.kind == 4 || pl.kind == 5;
    return windowed && (prm->flags & SAT_FLAG_NEAR_TIES);
}

cudaError_t enqueue_copy_f64(double* dst, const double* src, int n, cudaStream_t q) {
    if (n <= 0) return cudaSuccess;
    copy_f64_kernel<<<(n + 127) / 128, 128, 0, q>>>(dst, src, n);
    return cudaGetLastError();
}

namespace {

// ---- the whole of one sat_run call, enqueued on a stream --------------------

struct RunShape {
    int n_chains, M, S_total, window, n_windows;
};

// Sweep launches are bracketed by events (direct launches) or, inside a
// graph, by global-timer stamps written to `stamps` (2 per window).
cudaError_t enqueue_run(const satpila_pila* p, const Plan& pl, const BatchDev& b, const sat_params* prm,
                        const RunShape& r, void* ws_base, size_t ws_bytes, int* counters,
                        const std::vector<cudaEvent_t>& evs, unsigned long long* stamps, cudaStream_t q) {
    cudaError_t err = cudaMemsetAsync(ws_base, 0, ws_bytes, q);
    if (err != cudaSuccess) return err;
    // 1. initial resync, 2. temperatures
    if ((err = enqueue_resync(p, pl, b, 0, r.n_chains, false, b.cost0, q)) != cudaSuccess) return err;
    if ((err = enqueue_t0(p, pl, b, prm, 0, r.n_chains, q)) != cudaSuccess) return err;
    // 3. windows of stages, each followed by a resync that records the drift
    for (int w = 0; w < r.n_windows; ++w) {
        const int s0 = w * r.window, s1 = std::min(r.S_total, s0 + r.window);
        auto mark = [&](int i) -> cudaError_t {
            if (!stamps) return cudaEventRecord(evs[i], q);
            stamp_kernel<<<1, 1, 0, q>>>(stamps + i);
            return cudaGetLastError();
        };
        if ((err = mark(2 * w)) != cudaSuccess) return err;
        err = enqueue_sweep(p, pl, b, prm, r.n_chains, r.M, r.S_total, s0, s1, counters + w, q);
        if (err != cudaSuccess) return err;
        if ((err = mark(2 * w + 1)) != cudaSuccess) return err;
        const bool last = w + 1 == r.n_windows;
        if (last && (err = enqueue_copy_f64(b.S_inc, b.S, r.n_chains, q)) != cudaSuccess) return err;
        if ((err = enqueue_resync(p, pl, b, 0, r.n_chains, true, last ? b.costF : nullptr, q)) != cudaSuccess)
            return err;
    }
    if (r.n_windows == 0) {
        if ((err = enqueue_copy_f64(b.S_inc, b.S, r.n_chains, q)) != cudaSuccess) return err;
        err = cudaMemcpyAsync(b.costF, b.cost0, (size_t)r.n_chains * 8, cudaMemcpyDeviceToDevice, q);
    }
    return err;
}

// ---- graph cache: repeated identical calls replay one CUDA graph ------------

struct CachedRun {
    int device = 0;
    const satpila_pila* p = nullptr;
    int n_chains = 0;
    const void* sino = nullptr;
    void* images = nullptr;
    sat_params prm{};
    int variant = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    BatchDev b;
    Plan pl;
    RunShape shape{};
    std::vector<cudaEvent_t> evs;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;  // recorded after each launch: a reuse on any stream waits for it
    bool in_use = false;
    unsigned long long last_use = 0;
};

constexpr size_t kGraphCacheEntries = 4;
std::mutex g_cache_mu;
std::list<CachedRun*> g_cache;
unsigned long long g_cache_clock = 0;

void destroy_cached(CachedRun* c) {
    if (c->done) {  // an asynchronous launch may still be running on the workspace
        cudaEventSynchronize(c->done);
        cudaEventDestroy(c->done);
    }
    if (c->exec) cudaGraphExecDestroy(c->exec);
    for (auto& ev : c->evs) cudaEventDestroy(ev);
    if (c->ws) cudaFree(c->ws);
    delete c;
}

// A private stream per device for recording graphs (the caller's stream may
// be the legacy default stream, which cannot be captured).
cudaStream_t capture_stream(int dev) {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!streams[dev]) cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    return streams[dev];
}

// ---- autotuner: the fastest plan variant for a problem shape ---------------

struct TuneKey {
    int device, n, U, B, precision, n_mask, K, chains_log2, M;
    bool operator==(const TuneKey& o) const { return std::memcmp(this, &o, sizeof(TuneKey)) == 0; }
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, int>> g_tuned;

// The autotuner's picks kept across processes: with SATPILA_TUNE_CACHE set,
// one line per pick, "<device name>|n U B precision n_mask K log2(chains) M plan".
std::string tune_line_key(const TuneKey& k) {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, k.device) != cudaSuccess) {
        cudaGetLastError();
        prop.name[0] = 0;
    }
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s|%d %d %d %d %d %d %d %d", prop.name, k.n, k.U, k.B, k.precision, k.n_mask, k.K,
                  k.chains_log2, k.M);
    return buf;
}

int tune_cache_lookup(const TuneKey& k) {
    const char* path = std::getenv("SATPILA_TUNE_CACHE");
    if (!path || !*path) return -1;
    std::FILE* f = std::fopen(path, "r");
    if (!f) return -1;
    const std::string want = tune_line_key(k);
    char line[640];
    int plan = -1;
    while (std::fgets(line, sizeof(line), f)) {
        std::string ln(line);
        const size_t sp = ln.find_last_of(' ');
        if (sp == std::string::npos || ln.compare(0, sp, want) != 0 || sp != want.size()) continue;
        const int v = std::atoi(ln.c_str() + sp + 1);
        if (v > PLAN_RULES && v < PLAN_COUNT) plan = v;  // the last line for a key wins
    }
    std::fclose(f);
    return plan;
}

void tune_cache_store(const TuneKey& k, int plan) {
    const char* path = std::getenv("SATPILA_TUNE_CACHE");
    if (!path || !*path || plan <= PLAN_RULES) return;
    std::FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d\n", tune_line_key(k).c_str(), plan);
    std::fclose(f);
}

// Times one short sweep launch of each feasible variant on a scratch copy of
// the caller's images (the caller's data are not touched) and returns the
// variant with the highest moves/s.  Variants differ only in how the work is
// laid out on the GPU (warps per chain, residency, tasks), not in the moves.
int autotune(const satpila_pila* p, int n_chains, const float* sino, const float* images, const sat_params* prm,
             int M, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    int lg = 0;
    while ((1 << (lg + 1)) <= n_chains) ++lg;
    const int Mp = std::min(M, 2048);
    const TuneKey key{dev, p->n, p->U, p->B, p->precision, p->n_mask, prm->bome_k, lg, Mp};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (auto& kv : g_tuned)
            if (kv.first == key) return kv.second;
        const int cached = tune_cache_lookup(key);
        if (cached > PLAN_RULES) {
            g_tuned.push_back({key, cached});
            return cached;
        }
    }
    const long long P = (long long)p->n * p->n;
    int best = PLAN_RULES;
    double best_rate = -1.0;
    float* img = nullptr;
    if (cudaMalloc(&img, (size_t)n_chains * P * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return PLAN_RULES;
    }
    sat_params tp = *prm;
    tp.trace = nullptr;
    tp.sweep_cost = nullptr;
    tp.flags &= ~SAT_FLAG_TEST_STALL;
    tp.t0 = prm->t0 > 0.0 ? prm->t0 : 1e-3;  // a fixed temperature: the probe only times moves
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int v = PLAN_WINDOW_SMEM; v < PLAN_COUNT; ++v) {
        Plan pl;
        const std::string saved = satpila_last_error();
        if (choose_plan(p, n_chains, 1, &tp, v, &pl) != SATPILA_OK) {
            set_error(saved);
            continue;
        }
        if (prepare_launches(p, pl, tp.bome_k) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        const size_t bytes = batch_bytes(pl, n_chains) + 256;
        void* ws = nullptr;
        if (cudaMalloc(&ws, bytes) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        BatchDev b;
        batch_carve(ws, pl, n_chains, &b);
        int* counter = (int*)((char*)ws + bytes - 256);
        b.img = img;
        b.sino = sino;
        cudaError_t e = cudaMemsetAsync(ws, 0, bytes, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(img, images, (size_t)n_chains * P * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = enqueue_resync(p, pl, b, 0, n_chains, false, nullptr, s);
        if (e == cudaSuccess) e = enqueue_t0(p, pl, b, &tp, 0, n_chains, s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = enqueue_sweep(p, pl, b, &tp, n_chains, Mp, 1, 0, 1, counter, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        int err_code = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&err_code, b.error, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        float ms = 0.0f;
        if (e == cudaSuccess && err_code == 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f) {
            const double rate = (double)n_chains * Mp / ms;
            if (rate > best_rate) {
                best_rate = rate;
                best = v;
            }
        }
        if (e != cudaSuccess) cudaGetLastError();
        cudaFree(ws);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(img);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned.push_back({key, best});
    tune_cache_store(key, best);
    return best;
}

// Device staging for a caller buffer that may live on the host.
struct Staged {
    void* dev = nullptr;
    bool owned = false;
};

int stage_in(const void* src, size_t bytes, bool copy, cudaStream_t s, Staged* out) {
    if (!src || bytes == 0) return SATPILA_OK;
    if (is_device_pointer(src)) {
        out->dev = const_cast<void*>(src);
        return SATPILA_OK;
    }
    SP_CUDA(cudaMalloc(&out->dev, bytes));
    out->owned = true;
    if (copy) SP_CUDA(cudaMemcpyAsync(out->dev, src, bytes, cudaMemcpyHostToDevice, s));
    return SATPILA_OK;
}


}  // namespace

void sat_cache_purge(const satpila_pila* p) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    for (auto it = g_cache.begin(); it != g_cache.end();) {
        if ((*it)->p == p && !(*it)->in_use) {
            destroy_cached(*it);
            it = g_cache.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace satpila

using namespace satpila;

extern "C" int sat_run(const satpila_pila* p, int32_t n_chains, const float* sino_meas, float* images,
                       const sat_params* prm, sat_stats* stats, void* stream) {
    if (!p || !prm || n_chains < 0) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: bad argument");
    if (n_chains == 0) return SATPILA_OK;
    if (!sino_meas || !images) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: null data pointer");
    if (prm->bome_k < 1 || prm->bome_k > kMaxK)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_run: bome_k must be in [1, 32]");
    if (!(prm->beta > 0.0f)) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: beta must be > 0");
    if (prm->n_sweeps < 0 || prm->moves_per_sweep < 0 || prm->resync_every < 0 || prm->wait_ms < 0)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_run: negative counts");
    if (prm->schedule < SAT_SCHED_LINEAR || prm->schedule > SAT_SCHED_CUBIC)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_run: unknown schedule");
    if (prm->residency < SAT_RESIDENT_AUTO || prm->residency > SAT_RESIDENT_GLOBAL)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_run: unknown residency");
    cudaStream_t s = (cudaStream_t)stream;
    const long long P = (long long)p->n * p->n;
    const long long cells = (long long)p->U * p->B;
    RunShape shape{};
    shape.n_chains = n_chains;
    shape.S_total = prm->n_sweeps;
    shape.M = prm->moves_per_sweep > 0 ? prm->moves_per_sweep : p->n_mask;
    shape.window = prm->resync_every > 0 ? std::min(prm->resync_every, std::max(1, shape.S_total))
                                         : std::max(1, shape.S_total);
    shape.n_windows = shape.S_total > 0 ? (shape.S_total + shape.window - 1) / shape.window : 0;
    const int M = shape.M, S_total = shape.S_total, n_windows = shape.n_windows;

    // Caller buffers (host buffers are staged).
    Staged d_sino, d_img, d_trace, d_cost;
    const size_t trace_recs = prm->trace ? (size_t)S_total * M : 0;
    auto free_staged = [&]() {
        for (Staged* st : {&d_sino, &d_img, &d_trace, &d_cost})
            if (st->owned) cudaFree(st->dev);
    };
    int rc;
    if ((rc = stage_in(sino_meas, (size_t)n_chains * cells * sizeof(float), true, s, &d_sino)) ||
        (rc = stage_in(images, (size_t)n_chains * P * sizeof(float), true, s, &d_img)) ||
        (rc = stage_in(prm->trace, trace_recs * sizeof(sat_trace_rec), false, s, &d_trace)) ||
        (rc = stage_in(prm->sweep_cost, (size_t)n_chains * S_total * sizeof(double), false, s, &d_cost))) {
        free_staged();
        return rc;
    }
    const bool staged = d_sino.owned || d_img.owned || d_trace.owned || d_cost.owned;

    // Launch plan: given, chosen by rules, or by the autotuner.
    int variant = PLAN_RULES;
    if (prm->plan != PLAN_RULES) {
        if (prm->plan < PLAN_RULES || prm->plan >= PLAN_COUNT) {
            free_staged();
            return fail(SATPILA_ERR_INVALID_ARG, "sat_run: unknown plan");
        }
        variant = prm->plan;
    } else if ((prm->flags & SAT_FLAG_AUTOTUNE) && !(prm->flags & SAT_FLAG_BOME_INDEPENDENT) && S_total > 0 &&
               p->n_mask > 0) {
        variant = autotune(p, n_chains, (const float*)d_sino.dev, (const float*)d_img.dev, prm, M, s);
    }
    Plan pl;
    if ((rc = choose_plan(p, n_chains, shape.window, prm, variant, &pl)) != SATPILA_OK) {
        free_staged();
        return rc;
    }
    cudaError_t e = prepare_launches(p, pl, prm->bome_k);
    if (e != cudaSuccess) {
        free_staged();
        return cuda_fail(e, "sat_run: launch attributes");
    }
    int dev = 0;
    cudaGetDevice(&dev);

    // A cached graph for this exact call (device buffers only), else a new
    // workspace; with SAT_FLAG_NO_GRAPH the launches are issued one by one.
    const bool use_graph = !(prm->flags & SAT_FLAG_NO_GRAPH) && !staged;
    CachedRun* run = nullptr;
    bool cached = false;
    if (use_graph) {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        for (CachedRun* c : g_cache)
            if (!c->in_use && c->device == dev && c->p == p && c->n_chains == n_chains && c->sino == d_sino.dev &&
                c->images == d_img.dev && c->variant == variant &&
                std::memcmp(&c->prm, prm, sizeof(sat_params)) == 0) {
                run = c;
                run->in_use = true;
                run->last_use = ++g_cache_clock;
                cached = true;
                break;
            }
    }
    if (!run) {
        run = new CachedRun();
        run->device = dev;
        run->p = p;
        run->n_chains = n_chains;
        run->sino = d_sino.dev;
        run->images = d_img.dev;
        run->prm = *prm;
        run->variant = variant;
        run->pl = pl;
        run->shape = shape;
        run->ws_bytes = batch_bytes(pl, n_chains) + align_up((size_t)(n_windows + 1) * 4, 256) +
                        align_up((size_t)(2 * n_windows + 1) * 8, 256);
        e = cudaMalloc(&run->ws, run->ws_bytes);
        if (e != cudaSuccess) {
            delete run;
            free_staged();
            return cuda_fail(e, "sat_run: workspace");
        }
        batch_carve(run->ws, pl, n_chains, &run->b);
        run->b.img = (float*)d_img.dev;
        run->b.sino = (const float*)d_sino.dev;
        run->b.sweep_cost = (double*)d_cost.dev;
        run->b.trace = (sat_trace_rec*)d_trace.dev;
        run->b.trace_cap = (long long)trace_recs;
        run->b.trace_chain = prm->trace_chain;
        run->evs.resize(2 * (size_t)n_windows);
        for (auto& ev : run->evs) cudaEventCreate(&ev);
        run->in_use = true;
    }
    int* counters = (int*)((char*)run->ws + batch_bytes(pl, n_chains));
    unsigned long long* stamps =
        (unsigned long long*)((char*)counters + align_up((size_t)(n_windows + 1) * 4, 256));

    if (use_graph && !run->exec) {
        // Record every launch of the call once into a graph.
        cudaStream_t cs = capture_stream(dev);
        cudaGraph_t graph = nullptr;
        e = cs ? cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) : cudaErrorInvalidResourceHandle;
        if (e == cudaSuccess) {
            const cudaError_t e1 =
                enqueue_run(p, pl, run->b, prm, shape, run->ws, run->ws_bytes, counters, run->evs, stamps, cs);
            e = cudaStreamEndCapture(cs, &graph);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&run->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            run->exec = nullptr;  // fall back to direct launches
        }
    }
    if (run->exec) {
        if (!run->done && cudaEventCreateWithFlags(&run->done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            run->done = nullptr;
        }
        if (run->done) e = cudaStreamWaitEvent(s, run->done, 0);  // an earlier launch of it, on any stream
        if (e == cudaSuccess) e = cudaGraphLaunch(run->exec, s);
        if (e == cudaSuccess && run->done) e = cudaEventRecord(run->done, s);
    } else {
        e = enqueue_run(p, pl, run->b, prm, shape, run->ws, run->ws_bytes, counters, run->evs, nullptr, s);
    }
    // Without stats, and with every buffer in device memory, the call returns
    // once its graph is enqueued: the graph and its workspace stay cached, and
    // a later launch of them waits for this one.
    if (!stats && use_graph && run->exec && run->done && e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        run->in_use = false;
        run->last_use = ++g_cache_clock;
        if (!cached) g_cache.push_back(run);
        while (g_cache.size() > kGraphCacheEntries) {
            auto victim = g_cache.end();
            for (auto it = g_cache.begin(); it != g_cache.end(); ++it)
                if (!(*it)->in_use && *it != run && (victim == g_cache.end() || (*it)->last_use < (*victim)->last_use))
                    victim = it;
            if (victim == g_cache.end()) break;
            destroy_cached(*victim);
            g_cache.erase(victim);
        }
        return SATPILA_OK;
    }

    // Results.
    const BatchDev& b = run->b;
    const size_t nc = (size_t)n_chains;
    std::vector<double> T0(nc), TN(nc), c0(nc), cF(nc), Sinc(nc), dmax(nc);
    std::vector<int> found(nc);
    std::vector<unsigned> ties(nc, 0u);
    std::vector<unsigned long long> acc(nc);
    int err_code = 0;
    if (e == cudaSuccess && stats) {
        struct {
            void* dst;
            const void* src;
            size_t bytes;
        } cps[] = {{T0.data(), b.T0, nc * 8},       {TN.data(), b.TN, nc * 8},       {c0.data(), b.cost0, nc * 8},
                   {cF.data(), b.costF, nc * 8},    {Sinc.data(), b.S_inc, nc * 8},  {dmax.data(), b.drift_max, nc * 8},
                   {found.data(), b.found, nc * 4}, {acc.data(), b.accepted, nc * 8},
                   {ties.data(), b.ties, nc * 4}};
        for (auto& c : cps)
            if (e == cudaSuccess) e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err_code, b.error, 4, cudaMemcpyDeviceToHost, s);
    std::vector<unsigned long long> ts(2 * (size_t)n_windows);
    if (e == cudaSuccess && run->exec && n_windows > 0)
        e = cudaMemcpyAsync(ts.data(), stamps, ts.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && d_img.owned)
        e = cudaMemcpyAsync(images, d_img.dev, nc * P * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && d_trace.owned)
        e = cudaMemcpyAsync(prm->trace, d_trace.dev, trace_recs * sizeof(sat_trace_rec), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && d_cost.owned)
        e = cudaMemcpyAsync(prm->sweep_cost, d_cost.dev, nc * S_total * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    double sweep_ms = 0.0;
    for (int w = 0; e == cudaSuccess && w < n_windows; ++w) {
        float ms = 0.0f;
        if (run->exec) sweep_ms += 1e-6 * (double)(ts[2 * w + 1] - ts[2 * w]);
        else if (cudaEventElapsedTime(&ms, run->evs[2 * w], run->evs[2 * w + 1]) == cudaSuccess) sweep_ms += ms;
        else cudaGetLastError();
    }
    // Keep the graph and its workspace for a repeat of this call.
    if (use_graph && run->exec && e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        run->in_use = false;
        run->last_use = ++g_cache_clock;
        if (!cached) g_cache.push_back(run);
        while (g_cache.size() > kGraphCacheEntries) {
            auto victim = g_cache.end();
            for (auto it = g_cache.begin(); it != g_cache.end(); ++it)
                if (!(*it)->in_use && (victim == g_cache.end() || (*it)->last_use < (*victim)->last_use)) victim = it;
            if (victim == g_cache.end()) break;
            destroy_cached(*victim);
            g_cache.erase(victim);
        }
    } else {
        if (cached) {
            std::lock_guard<std::mutex> lock(g_cache_mu);
            g_cache.remove(run);
        }
        destroy_cached(run);
    }
    free_staged();
    if (e != cudaSuccess) return cuda_fail(e, "sat_run");
    if (stats) {
        const double inv_cells = 1.0 / (double)cells;
        for (size_t c = 0; c < nc; ++c) {
            sat_stats& st = stats[c];
            std::memset(&st, 0, sizeof(st));
            st.t0 = T0[c];
            st.tn = TN[c];
            st.initial_cost = c0[c];
            st.final_cost = cF[c];
            st.final_cost_incremental = std::sqrt(std::max(0.0, Sinc[c] * inv_cells));
            st.max_resync_drift = dmax[c];
            st.accepted = (int64_t)acc[c];
            st.proposed = (int64_t)S_total * (p->n_mask > 0 ? M : 0);
            st.t0_found = found[c];
            st.status = err_code;
            st.sweep_ms = sweep_ms;
            st.plan = variant != PLAN_RULES ? variant : plan_code(pl);
            st.near_ties = sweep_counts_ties(pl, prm) ? (int32_t)std::min<unsigned>(ties[c], 0x7fffffffu) : -1;
        }
    }
    if (err_code != 0) return fail(err_code, "sat_run: a device-side check failed");
    return SATPILA_OK;
}

// sat_run over chains given one buffer each: the chains are gathered into
// one contiguous device batch (stream-ordered copies), annealed by sat_run,
// and the images scattered back, all on `stream`.
extern "C" int sat_run_ptrs(const satpila_pila* p, int32_t n_chains, const float* const* sino_meas,
                            float* const* images, const sat_params* prm, sat_stats* stats, void* stream) {
    if (!p || !prm || n_chains < 0) return fail(SATPILA_ERR_INVALID_ARG, "sat_run_ptrs: bad argument");
    if (n_chains == 0) return SATPILA_OK;
    if (!sino_meas || !images) return fail(SATPILA_ERR_INVALID_ARG, "sat_run_ptrs: null pointer array");
    for (int32_t c = 0; c < n_chains; ++c)
        if (!sino_meas[c] || !images[c]) return fail(SATPILA_ERR_INVALID_ARG, "sat_run_ptrs: null chain buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t P = (size_t)p->n * p->n, cells = (size_t)p->U * p->B;
    float* d_sino = nullptr;
    float* d_img = nullptr;
    cudaError_t e = cudaMallocAsync(&d_sino, (size_t)n_chains * cells * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_img, (size_t)n_chains * P * sizeof(float), s);
    for (int32_t c = 0; c < n_chains && e == cudaSuccess; ++c) {
        e = cudaMemcpyAsync(d_sino + (size_t)c * cells, sino_meas[c], cells * sizeof(float), cudaMemcpyDefault, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_img + (size_t)c * P, images[c], P * sizeof(float), cudaMemcpyDefault, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (d_sino) cudaFreeAsync(d_sino, s);
        if (d_img) cudaFreeAsync(d_img, s);
        return e == cudaErrorMemoryAllocation ? fail(SATPILA_ERR_OOM, "sat_run_ptrs: batch buffers")
                                              : cuda_fail(e, "sat_run_ptrs: gathering the chains");
    }
    const int rc = sat_run(p, n_chains, d_sino, d_img, prm, stats, stream);
    // the images go back whatever sat_run reported (a device-side timeout
    // still leaves every chain's image at a stage boundary)
    for (int32_t c = 0; c < n_chains && e == cudaSuccess; ++c)
        e = cudaMemcpyAsync(images[c], d_img + (size_t)c * P, P * sizeof(float), cudaMemcpyDefault, s);
    cudaFreeAsync(d_sino, s);
    cudaFreeAsync(d_img, s);
    if (e == cudaSuccess && stats) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sat_run_ptrs: returning the images");
    return rc;
}
