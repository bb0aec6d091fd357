// Host-side building blocks of the annealer shared by sat_run and the
// serving engine: the launch plan, the device state of a batch of chains,
// and the enqueue steps of Sec. II-A (resync, Eq. (8), sweeps).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"
#include "sat_sweep.cuh"

namespace satpila {

size_t align_up(size_t v, size_t a);

// Plan variants (the autotuner's candidates); PLAN_RULES picks by size.
enum PlanVariant {
    PLAN_RULES = 0,
    PLAN_WINDOW_SMEM,
    PLAN_WINDOW_GLOBAL,
    PLAN_WINDOW_HYBRID,
    PLAN_PIPE_1,  // pipelined kernel, 1, 2 or 4 warps per chain, residual where it fits
    PLAN_PIPE_2,
    PLAN_PIPE_4,
    PLAN_WINDOW_G2,  // windowed, 2 or 4 warps per chain, residual in global memory
    PLAN_WINDOW_G4,
    PLAN_WINDOW_SMEM_G2,  // windowed, 2 or 4 warps per chain, residual band in shared memory
    PLAN_WINDOW_SMEM_G4,
    PLAN_COUNT
};

struct Plan {
    bool smem = false;
    int kind = 0;         // 0 pipelined, 1 windowed, 2 hybrid, 3 independent BoME, 4/5 windowed groups of 2/4 warps
                          // (residual band in shared memory when smem)
    int hybrid_smem_warps = 0, hybrid_glob_bytes = 0;
    int jmax = 4, J = 4, D = 4;
    int W = 1, groups = 1, warps = 1, grid = 1;
    int stage_bytes = 0, group_smem = 0;
    long long resid_floats = 0;
    int pitch = 0;               // residual row pitch in global memory (floats, multiple of 4; of 8 when resid_il)
    int resid_il = 0;            // global residual rows stored in pairs (u, u + resid_il) interleaved (resid_row_base)
    int band_lo = 0;             // first bin of the shared-memory band (multiple of 4)
    int band_pitch = 0;          // band row length in shared memory (floats, multiple of 4)
    long long band_floats = 0;   // shared-memory residual of a windowed warp
    int spt = 1;                 // stages per task
    int proj_G = 0;              // resync partial sums per chain (one per angle: U)
    int geo_n = 0, geo_U = 0, geo_B = 0;  // the table's geometry
    bool rays = false;           // the table has a ray-major index: resyncs run the ray-driven projector
    int variant = PLAN_RULES;
    size_t sweep_smem_bytes() const;
};

// The SAT_PLAN_* code of a plan's launch layout (PLAN_RULES for the
// independent-pixel BoME kernel, which has no other layout).
int plan_code(const Plan& pl);

// Launch plan for n_chains chains running `window` stages per sweep launch.
int choose_plan(const satpila_pila* p, int n_chains, int window, const sat_params* prm, int variant, Plan* pl);

// Device state of a batch of chains; chain c's entries at index c.
struct BatchDev {
    float* resid = nullptr;        // [n][resid_floats]
    float* img = nullptr;          // [n][n * n]
    const float* sino = nullptr;   // [n][U * B] measured sinograms
    double* S = nullptr;           // running sum of squared residuals
    double* T0 = nullptr;
    double* TN = nullptr;
    int* found = nullptr;          // uphill samples found by Eq. (8)
    unsigned long long* accepted = nullptr;
    unsigned* ties = nullptr;      // near-tie decisions (windowed layouts with SAT_FLAG_NEAR_TIES)
    int* progress = nullptr;       // per chain: stages done in the current sweep launch
    int* claim = nullptr;          // per chain: 1 while a warp runs it (ready-first scheduling)
    int* error = nullptr;          // [1]
    double* part_sq = nullptr;     // [n][U] per-angle partials of the resync
    float* part_drift = nullptr;   // [n][U]
    double* drift_max = nullptr;
    double* cost0 = nullptr;       // Eq. (4) cost at the start
    double* costF = nullptr;       // Eq. (4) cost after the latest resync
    double* S_inc = nullptr;       // incremental S before the latest resync
    void* proj_ws = nullptr;       // ray-driven projector's workspace (ray_ws_bytes for the capacity), or NULL
    const ChainCtl* ctl = nullptr; // per-chain control or NULL
    double* sweep_cost = nullptr;
    sat_trace_rec* trace = nullptr;
    long long trace_cap = 0;
    int trace_chain = -1;
};

// Bytes of the per-chain arrays (resid ... S_inc, plus the error word) for
// `cap` chains, and their placement in a buffer of that size.
size_t batch_bytes(const Plan& pl, long long cap);
void batch_carve(void* base, const Plan& pl, long long cap, BatchDev* b);

// Launch attributes that must be set before any launch is captured.
cudaError_t prepare_launches(const satpila_pila* p, const Plan& pl, int bome_k);

// FP64-grade resync of chains [c0, c0 + nc): r = P(f) - P_m, S, and the
// cost (cost_out, may be NULL); drift: record the largest |change| of r.
cudaError_t enqueue_resync(const satpila_pila* p, const Plan& pl, const BatchDev& b, int c0, int nc, bool drift,
                           double* cost_out, cudaStream_t q);
// Initial temperatures of chains [c0, c0 + nc) (Eq. (8) or given).
cudaError_t enqueue_t0(const satpila_pila* p, const Plan& pl, const BatchDev& b, const sat_params* prm, int c0,
                       int nc, cudaStream_t q);
// One persistent sweep launch: stages [s_begin, s_end) of every chain
// (offset by each chain's ChainCtl::stage0 when b.ctl is set).
cudaError_t enqueue_sweep(const satpila_pila* p, const Plan& pl, const BatchDev& b, const sat_params* prm,
                          int n_chains, int M, int s_total, int s_begin, int s_end, int* task_counter,
                          cudaStream_t q);
// The sweep launch's arguments for these chains (what enqueue_sweep launches).
SatArgs sweep_args(const satpila_pila* p, const Plan& pl, const BatchDev& b, const sat_params* prm, int n_chains,
                   int M, int s_total, int s_begin, int s_end, int* task_counter);
// One launch over chains of several tables (the serving engine's classes of
// one image size and table precision): the windowed kernel on groups of 4
// warps, four records per lane, up to 8 estimates, residual in global memory.
// multi_table_ok: a table and parameters that launch can take (at most 512
// angles, K <= 8, no layout requested).  plan_multi: its launch shape for
// n_chains chains and `window` stages per launch.  The per-class arguments
// la.classes[q] are sweep_args of class q with the class plan of
// PLAN_WINDOW_G4 (residual layout), stage_bytes from the multi plan.
bool multi_table_ok(const satpila_pila* p, const sat_params* prm);
int plan_multi(int rt, int n_chains, int window, Plan* pl);
cudaError_t prepare_multi(int rt);
cudaError_t enqueue_sweep_multi(int rt, const Plan& pl, const SatArgs& la, cudaStream_t q);
cudaError_t enqueue_copy_f64(double* dst, const double* src, int n, cudaStream_t q);
// True when the sweep launches of this plan count near-tie decisions.
bool sweep_counts_ties(const Plan& pl, const sat_params* prm);

// Drops cached graphs and plans that refer to p (called by pila_free).
void sat_cache_purge(const satpila_pila* p);

}  // namespace satpila
