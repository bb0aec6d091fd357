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
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "sat_sweep.cuh"
#include "sat_window.cuh"

namespace satpila {

using SweepFn = void (*)(const SatArgs);
SweepFn sweep_kernel_f32_smem(int jmax, int kmax);
SweepFn sweep_kernel_f32_glob(int jmax, int kmax);
SweepFn sweep_kernel_f16_smem(int jmax, int kmax);
SweepFn sweep_kernel_f16_glob(int jmax, int kmax);
SweepFn window_kernel(bool f16, bool smem, int jmax, int kmax);
SweepFn hybrid_kernel(bool f16, int jmax, int kmax);

namespace {

// kind: 0 pipelined, 1 windowed, 2 hybrid
SweepFn sweep_kernel(bool f16, bool smem, int jmax, int kmax, int kind = 0) {
    if (kind == 1) return window_kernel(f16, smem, jmax, kmax);
    if (kind == 2) return hybrid_kernel(f16, jmax, kmax);
    if (f16) return smem ? sweep_kernel_f16_smem(jmax, kmax) : sweep_kernel_f16_glob(jmax, kmax);
    return smem ? sweep_kernel_f32_smem(jmax, kmax) : sweep_kernel_f32_glob(jmax, kmax);
}

int kmax_for(int K) { return K <= 4 ? 4 : K <= 8 ? 8 : 32; }

cudaError_t launch_sweep(bool f16, bool smem, int kind, int jmax, int kmax, const SatArgs& a, int grid,
                         int warps, size_t smem_bytes, cudaStream_t s) {
    SweepFn k = sweep_kernel(f16, smem, jmax, kmax, kind);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    k<<<grid, warps * 32, smem_bytes, s>>>(a);
    return cudaGetLastError();
}

int sweep_blocks_per_sm(bool f16, bool smem, int kind, int jmax, int kmax, int warps, size_t smem_bytes) {
    SweepFn k = sweep_kernel(f16, smem, jmax, kmax, kind);
    if (!k) return 0;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem_bytes) != cudaSuccess) return 0;
    return nb;
}

}  // namespace

namespace {

template <bool F16>
__global__ void __launch_bounds__(256) t0_kernel(const T0Args a) {
    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ float dcs[32];
    __shared__ double total_s;
    __shared__ int found_s, done_s;
    if (a.t0_fixed > 0.0) {
        if (tid == 0) {
            a.T0[c] = a.t0_fixed;
            a.TN[c] = a.tn < 0.0 ? a.t0_fixed / 1000.0 : a.tn;
            a.found[c] = 0;
        }
        return;
    }
    const uint2 key = chain_key(a.seed + (unsigned long long)c);
    const float* R = a.resid + (long long)c * a.resid_floats;
    const float* img = a.img + (long long)c * a.img_stride;
    const float C2 = (float)(a.S[c] * a.inv_BU_d);
    const float C = sqrtf(C2);
    const long long max_tries = 100LL * a.Q;
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
                    Entry2 e;
                    if (F16) {
                        const uint2 v = reinterpret_cast<const uint2*>(row)[u];
                        e = decode_f16(v.x, v.y);
                    } else {
                        e = decode_f32(reinterpret_cast<const uint4*>(row)[u]);
                    }
                    if (e.l0 != 0.0f) {
                        g = fmaf(R[u * a.pitch + e.k0], e.l0, g);
                        h = fmaf(e.l0, e.l0, h);
                    }
                    if (e.l1 != 0.0f) {
                        g = fmaf(R[u * a.pitch + e.k1], e.l1, g);
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
            for (int q = 0; q < 32 && found_s < a.Q; ++q) {
                if (base + q >= max_tries) break;
                if (dcs[q] > 0.0f) {
                    total_s += (double)dcs[q];
                    ++found_s;
                }
            }
            if (found_s >= a.Q) done_s = 1;
        }
        __syncthreads();
        if (done_s) break;
    }
    if (tid == 0) {
        // Eq. (8): T0 = -sum(C' - C) / (Q ln 0.9)
        const double t0 = found_s > 0 ? -total_s / ((double)found_s * log(0.9)) : 0.0;
        a.T0[c] = t0;
        a.TN[c] = a.tn < 0.0 ? t0 / 1000.0 : a.tn;
        a.found[c] = found_s;
    }
}

__global__ void copy_f64_kernel(double* dst, const double* src, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i];
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
    float* resid = nullptr;
    double* S = nullptr;
    double* T0 = nullptr;
    double* TN = nullptr;
    int* found = nullptr;
    unsigned long long* accepted = nullptr;
    int* progress = nullptr;
    int* counters = nullptr;   // one task counter per sweep launch
    int* error = nullptr;
    double* part_sq = nullptr;
    float* part_drift = nullptr;
    double* drift_max = nullptr;
    double* cost0 = nullptr;
    double* costF = nullptr;
    double* S_inc = nullptr;
};

struct Plan {
    bool smem = false;
    int kind = 0;         // 0 pipelined, 1 windowed (shared-memory residual), 2 hybrid
    int hybrid_smem_warps = 0, hybrid_glob_bytes = 0;
    int jmax = 4, J = 4, D = 4;
    int W = 1, groups = 1, warps = 1, grid = 1;
    int stage_bytes = 0, group_smem = 0;
    long long resid_floats = 0;
    int pitch = 0;               // residual row pitch in global memory (floats, multiple of 4)
    int band_lo = 0;             // first bin of the shared-memory band (multiple of 4)
    int band_pitch = 0;          // band row length in shared memory (floats, multiple of 4)
    long long band_floats = 0;   // shared-memory residual of a windowed warp
    int spt = 1;  // stages per task
};

int choose_plan(const satpila_pila* p, int n_chains, int window, const sat_params* prm, Plan* pl) {
    const bool f16 = p->precision == PILA_F16;
    int dev = 0, maxopt = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Warps per chain: the fewest that leave each lane at most two records
    // (four for very many angles).
    auto records_per_lane = [&](int W) {
        return f16 ? 2 * ((p->row_records + 64 * W - 1) / (64 * W)) : (p->U + 32 * W - 1) / (32 * W);
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
    // The windowed kernel: one warp per chain; residual in shared memory, in
    // global memory, or both kinds of warp side by side (hybrid).
    if (prm->group_warps <= 1 && records_per_lane(1) <= 4 && prm->pipeline_depth == 0) {
        const int jw = records_per_lane(1) <= 2 ? 2 : 4;
        const int stage = 512 * (f16 ? jw / 2 : jw);
        const size_t ring1 = group_ring_bytes(1) + (size_t)2 * kWin * stage;
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
            int per_sm = sweep_blocks_per_sm(f16, smem, kind, jw, kmax, warps, smem_bytes);
            if (per_sm < 1) per_sm = 1;
            const long long slots = (long long)sms * per_sm * warps;
            pl->spt = (!dynamic_tasks && n_chains <= slots) ? window : 1;
            const long long tasks = (long long)n_chains * ((window + pl->spt - 1) / pl->spt);
            const long long want = (std::min<long long>(tasks, slots) + warps - 1) / warps;
            pl->grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * per_sm));
            return SATPILA_OK;
        };
        const int win_per_cta = (int)std::min<size_t>(kSatMaxWarps, maxopt / gsm);
        if (prm->residency == SAT_RESIDENT_GLOBAL || (prm->residency == SAT_RESIDENT_AUTO && win_per_cta == 0)) {
            pl->group_smem = (int)glob;
            const int warps = std::min(4, std::max(1, n_chains));
            return finish(1, false, warps, (size_t)warps * glob, false);
        }
        if (win_per_cta == 0) return fail(SATPILA_ERR_INVALID_ARG, "sat_run: residual does not fit in shared memory");
        const int ns = std::min(win_per_cta, 3), ng = 4 - ns;
        if ((prm->flags & SAT_FLAG_HYBRID) && ng > 0 && n_chains > sms * win_per_cta &&
            (size_t)ns * gsm + (size_t)ng * glob <= (size_t)maxopt) {
            pl->group_smem = (int)gsm;
            pl->hybrid_smem_warps = ns;
            pl->hybrid_glob_bytes = (int)glob;
            // stage-sized tasks, so that chains move between the two kinds of warp
            return finish(2, true, ns + ng, (size_t)ns * gsm + (size_t)ng * glob, true);
        }
        pl->group_smem = (int)gsm;
        const int warps = std::min(win_per_cta, std::max(1, n_chains));
        return finish(1, true, warps, (size_t)warps * gsm, false);
    }
    int W = prm->group_warps > 0 ? prm->group_warps : 1;
    if (prm->group_warps <= 0)
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
    pl->stage_bytes = 512 * W * (f16 ? jmax / 2 : jmax);  // 16-byte chunks of all lanes
    const size_t ring = group_ring_bytes(W) + (size_t)pl->D * pl->stage_bytes;
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
    int per_sm = sweep_blocks_per_sm(f16, smem, 0, jmax, kmax_for(prm->bome_k), pl->warps, smem_bytes);
    if (per_sm < 1) per_sm = 1;
    const long long slots = (long long)sms * per_sm * groups;
    pl->spt = n_chains <= slots ? window : 1;
    const long long tasks = (long long)n_chains * ((window + pl->spt - 1) / pl->spt);
    const long long want = (std::min<long long>(tasks, slots) + groups - 1) / groups;
    pl->grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * per_sm));
    return SATPILA_OK;
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
    if (prm->n_sweeps < 0 || prm->moves_per_sweep < 0 || prm->resync_every < 0)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_run: negative counts");
    if (prm->schedule < SAT_SCHED_LINEAR || prm->schedule > SAT_SCHED_CUBIC)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_run: unknown schedule");
    if (prm->residency < SAT_RESIDENT_AUTO || prm->residency > SAT_RESIDENT_GLOBAL)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_run: unknown residency");
    cudaStream_t s = (cudaStream_t)stream;
    const long long P = (long long)p->n * p->n;
    const long long cells = (long long)p->U * p->B;
    const int S_total = prm->n_sweeps;
    const int M = prm->moves_per_sweep > 0 ? prm->moves_per_sweep : p->n_mask;
    const int window = prm->resync_every > 0 ? std::min(prm->resync_every, std::max(1, S_total)) : std::max(1, S_total);
    const int n_windows = S_total > 0 ? (S_total + window - 1) / window : 0;

    Plan pl;
    int rc = choose_plan(p, n_chains, window, prm, &pl);
    if (rc != SATPILA_OK) return rc;
    int A = 0, G = 0;
    if (projector_plan(p->U, p->B, &A, &G) != SATPILA_OK)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_run: too many bins");

    // Caller buffers (host buffers are staged).
    Staged d_sino, d_img, d_trace, d_cost;
    const size_t trace_recs = prm->trace ? (size_t)S_total * M : 0;
    if ((rc = stage_in(sino_meas, (size_t)n_chains * cells * sizeof(float), true, s, &d_sino)) ||
        (rc = stage_in(images, (size_t)n_chains * P * sizeof(float), true, s, &d_img)) ||
        (rc = stage_in(prm->trace, trace_recs * sizeof(sat_trace_rec), false, s, &d_trace)) ||
        (rc = stage_in(prm->sweep_cost, (size_t)n_chains * S_total * sizeof(double), false, s, &d_cost))) {
        for (Staged* st : {&d_sino, &d_img, &d_trace, &d_cost})
            if (st->owned) cudaFree(st->dev);
        return rc;
    }

    // Workspace.
    Workspace ws;
    const size_t nc = (size_t)n_chains;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_resid = carve(nc * pl.resid_floats * sizeof(float));
    const size_t o_S = carve(nc * 8), o_T0 = carve(nc * 8), o_TN = carve(nc * 8), o_found = carve(nc * 4);
    const size_t o_acc = carve(nc * 8), o_prog = carve(nc * 4), o_cnt = carve((size_t)(n_windows + 1) * 4);
    const size_t o_err = carve(4), o_psq = carve(nc * G * 8), o_pdr = carve(nc * G * 4);
    const size_t o_dmax = carve(nc * 8), o_c0 = carve(nc * 8), o_cF = carve(nc * 8), o_Sinc = carve(nc * 8);
    ws.bytes = off;
    cudaError_t e = cudaMalloc(&ws.base, ws.bytes);
    if (e != cudaSuccess) {
        for (Staged* st : {&d_sino, &d_img, &d_trace, &d_cost})
            if (st->owned) cudaFree(st->dev);
        return cuda_fail(e, "sat_run: workspace");
    }
    char* b = (char*)ws.base;
    ws.resid = (float*)(b + o_resid);
    ws.S = (double*)(b + o_S);
    ws.T0 = (double*)(b + o_T0);
    ws.TN = (double*)(b + o_TN);
    ws.found = (int*)(b + o_found);
    ws.accepted = (unsigned long long*)(b + o_acc);
    ws.progress = (int*)(b + o_prog);
    ws.counters = (int*)(b + o_cnt);
    ws.error = (int*)(b + o_err);
    ws.part_sq = (double*)(b + o_psq);
    ws.part_drift = (float*)(b + o_pdr);
    ws.drift_max = (double*)(b + o_dmax);
    ws.cost0 = (double*)(b + o_c0);
    ws.costF = (double*)(b + o_cF);
    ws.S_inc = (double*)(b + o_Sinc);

    std::vector<cudaEvent_t> evs(2 * (size_t)n_windows);
    for (auto& ev : evs) cudaEventCreate(&ev);
    const float* sino_d = (const float*)d_sino.dev;
    float* img_d = (float*)d_img.dev;

    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t err = cudaMemsetAsync(ws.base, 0, ws.bytes, q);
        if (err != cudaSuccess) return err;
        ProjArgs pa{};
        pa.table = p->d_table;
        pa.f16 = p->precision == PILA_F16;
        pa.row_records = p->row_records;
        pa.n = p->n;
        pa.U = p->U;
        pa.B = p->B;
        pa.angles_per_group = A;
        pa.n_groups = G;
        pa.mode = PROJ_RESYNC;
        pa.img = img_d;
        pa.img_stride = P;
        pa.pm = sino_d;
        pa.pm_stride = cells;
        pa.resid = ws.resid;
        pa.resid_stride = pl.resid_floats;
        pa.resid_pitch = pl.pitch;
        pa.part_sq = ws.part_sq;
        pa.part_drift = ws.part_drift;
        ReduceArgs ra{};
        ra.n_items = n_chains;
        ra.n_groups = G;
        ra.part_sq = ws.part_sq;
        ra.part_drift = ws.part_drift;
        ra.inv_cells = 1.0 / (double)cells;
        ra.S_out = ws.S;
        ra.cost_stride = 1;
        // 1. initial resync
        pa.drift = 0;
        if ((err = launch_projector(pa, n_chains, q)) != cudaSuccess) return err;
        ra.cost_out = ws.cost0;
        ra.drift_max = nullptr;
        if ((err = launch_reduce(ra, q)) != cudaSuccess) return err;
        // 2. temperatures
        T0Args ta{};
        ta.table = p->d_table;
        ta.row_stride = p->row_bytes;
        ta.f16 = p->precision == PILA_F16;
        ta.n = p->n;
        ta.U = p->U;
        ta.B = p->B;
        ta.pitch = pl.pitch;
        ta.list = p->d_list;
        ta.n_list = p->n_mask;
        ta.beta = prm->beta;
        ta.inv_BU = (float)(1.0 / (double)cells);
        ta.inv_BU_d = 1.0 / (double)cells;
        ta.resid = ws.resid;
        ta.resid_floats = pl.resid_floats;
        ta.img = img_d;
        ta.img_stride = P;
        ta.S = ws.S;
        ta.seed = prm->seed;
        ta.Q = prm->t0_samples > 0 ? prm->t0_samples : 200;
        ta.tn = prm->tn;
        ta.t0_fixed = prm->t0;
        ta.T0 = ws.T0;
        ta.TN = ws.TN;
        ta.found = ws.found;
        if (ta.f16) t0_kernel<true><<<n_chains, 256, 0, q>>>(ta);
        else t0_kernel<false><<<n_chains, 256, 0, q>>>(ta);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        // 3. windows of stages
        SatArgs sa{};
        sa.table = p->d_table;
        sa.row_stride = p->row_bytes;
        sa.row_chunks = (int)(p->row_bytes / 16);
        sa.hsum = p->d_hsum;
        sa.n = p->n;
        sa.U = p->U;
        sa.B = p->B;
        sa.pitch = pl.pitch;
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
        sa.resid = ws.resid;
        sa.img = img_d;
        sa.img_stride = P;
        sa.S = ws.S;
        sa.T0 = ws.T0;
        sa.TN = ws.TN;
        sa.seed = prm->seed;
        sa.accepted = ws.accepted;
        sa.progress = ws.progress;
        sa.schedule = prm->schedule;
        sa.n_sweeps_total = S_total;
        sa.error = ws.error;
        sa.sweep_cost = (double*)d_cost.dev;
        sa.trace = (sat_trace_rec*)d_trace.dev;
        sa.trace_chain = prm->trace_chain;
        sa.trace_cap = (long long)trace_recs;
        for (int wdx = 0; wdx < n_windows; ++wdx) {
            sa.sweep_begin = wdx * window;
            sa.sweep_end = std::min(S_total, sa.sweep_begin + window);
            sa.sweeps_per_task = pl.spt;
            sa.n_tasks = n_chains * ((sa.sweep_end - sa.sweep_begin + pl.spt - 1) / pl.spt);
            sa.task_counter = ws.counters + wdx;
            const size_t smem_bytes = pl.kind == 2 ? (size_t)pl.hybrid_smem_warps * pl.group_smem +
                                                         (size_t)(pl.warps - pl.hybrid_smem_warps) * pl.hybrid_glob_bytes
                                                   : (size_t)pl.groups * pl.group_smem;
            cudaEventRecord(evs[2 * wdx], q);
            err = launch_sweep(pa.f16, pl.smem, pl.kind, pl.jmax, kmax_for(prm->bome_k), sa, pl.grid, pl.warps,
                               smem_bytes, q);
            if (err != cudaSuccess) return err;
            cudaEventRecord(evs[2 * wdx + 1], q);
            const bool last = wdx + 1 == n_windows;
            if (last) {
                copy_f64_kernel<<<(n_chains + 127) / 128, 128, 0, q>>>(ws.S_inc, ws.S, n_chains);
                if ((err = cudaGetLastError()) != cudaSuccess) return err;
            }
            pa.drift = 1;
            if ((err = launch_projector(pa, n_chains, q)) != cudaSuccess) return err;
            ra.cost_out = last ? ws.costF : nullptr;
            ra.drift_max = ws.drift_max;
            if ((err = launch_reduce(ra, q)) != cudaSuccess) return err;
        }
        if (n_windows == 0) {
            copy_f64_kernel<<<(n_chains + 127) / 128, 128, 0, q>>>(ws.S_inc, ws.S, n_chains);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            err = cudaMemcpyAsync(ws.costF, ws.cost0, nc * 8, cudaMemcpyDeviceToDevice, q);
        }
        return err;
    };

    e = enqueue(s);
    // Results.
    std::vector<double> T0(nc), TN(nc), c0(nc), cF(nc), Sinc(nc), dmax(nc);
    std::vector<int> found(nc);
    std::vector<unsigned long long> acc(nc);
    int err_code = 0;
    if (e == cudaSuccess && stats) {
        struct {
            void* dst;
            const void* src;
            size_t bytes;
        } cps[] = {{T0.data(), ws.T0, nc * 8},       {TN.data(), ws.TN, nc * 8},     {c0.data(), ws.cost0, nc * 8},
                   {cF.data(), ws.costF, nc * 8},    {Sinc.data(), ws.S_inc, nc * 8}, {dmax.data(), ws.drift_max, nc * 8},
                   {found.data(), ws.found, nc * 4}, {acc.data(), ws.accepted, nc * 8}};
        for (auto& c : cps)
            if (e == cudaSuccess) e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err_code, ws.error, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && d_img.owned)
        e = cudaMemcpyAsync(images, d_img.dev, nc * P * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && d_trace.owned)
        e = cudaMemcpyAsync(prm->trace, d_trace.dev, trace_recs * sizeof(sat_trace_rec), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && d_cost.owned)
        e = cudaMemcpyAsync(prm->sweep_cost, d_cost.dev, nc * S_total * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    double sweep_ms = 0.0;
    for (int wdx = 0; e == cudaSuccess && wdx < n_windows; ++wdx) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, evs[2 * wdx], evs[2 * wdx + 1]) == cudaSuccess) sweep_ms += ms;
    }
    for (auto& ev : evs) cudaEventDestroy(ev);
    cudaFree(ws.base);
    for (Staged* st : {&d_sino, &d_img, &d_trace, &d_cost})
        if (st->owned) cudaFree(st->dev);
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
        }
    }
    if (err_code != 0) return fail(err_code, "sat_run: a device-side check failed");
    return SATPILA_OK;
}
