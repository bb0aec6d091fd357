// Serving engine: continuous batching of annealing requests on one GPU.
//
// A request is one slice (a chain): geometry, measured sinogram, start image
// and sat_params.  Requests that share a geometry, K, beta and moves per stage
// form a class; all chains of a class live in device arrays of the class and
// advance together, `stages_per_tick` stages per persistent sweep launch
// (each chain at its own point of its own schedule, through ChainCtl),
// followed by the FP64-grade resync of Sec. II-A's incremental scheme.
// Between launches the engine retires finished chains (copying their images
// and statistics out), compacts the arrays, and admits waiting requests as
// slots and device memory allow: a new chain is set up (sinogram and image
// copied in, resync, Eq. (8)) while the other chains of its class are between
// ticks, on the stream its class runs on, and the work of different streams
// overlaps.  PILA tables are cached per geometry and dropped when unused and
// memory is needed.
//
// Classes whose tables the windowed group kernel takes (at most 512 angles,
// K <= 8) are gathered into buckets, one per image size and table precision:
// a bucket's tick is one sweep launch over the chains of all its classes
// (each chain reading its own class's table, geometry and arrays), then each
// class's resync.  So the many one-chain classes of a stream of mixed
// geometries share launches and a few streams, instead of each holding a
// stream whose long launches delay the others behind it in the device's
// hardware queues.  Other classes (and all with SAT_SERVER_PER_CLASS) tick
// on their own streams.
//
// A chain's result does not depend on what else is running: its random
// stream is keyed by its own seed, its stages are numbered from its own
// start, and its resyncs fall every stages_per_tick of its own stages.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "sat_host.h"

namespace satpila {
namespace {

__global__ void tick_stamp_kernel(unsigned long long* out) { *out = global_ns(); }

// S before the resync that follows a window, for the chains that ran stages
// in it (so a chain's incremental cost is the one at its last stage).
__global__ void s_inc_kernel(double* S_inc, const double* S, const ChainCtl* ctl, int n, int s_begin) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n && ctl[c].stage0 + s_begin < ctl[c].n_sweeps) S_inc[c] = S[c];
}

constexpr int kMaxWindowsPerTick = 32;
constexpr double kTickTargetMs = 40.0;

double now_ms(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

struct Request {
    uint64_t ticket = 0;
    int n = 0, U = 0, B = 0, precision = PILA_F32;
    std::vector<double> angles;  // empty: u * pi / U
    std::vector<uint8_t> mask;   // empty: every pixel
    std::vector<float> sino, image;
    sat_params prm{};
    double t_submit = 0.0;
};

struct Done {
    sat_result res{};
    std::vector<float> image;
};

struct GeomKey {
    int n, U, B, precision;
    std::vector<double> angles;
    std::vector<uint8_t> mask;
    bool operator==(const GeomKey& o) const {
        return n == o.n && U == o.U && B == o.B && precision == o.precision && angles == o.angles && mask == o.mask;
    }
};

struct Geometry {
    GeomKey key;
    satpila_pila* p = nullptr;
    size_t bytes = 0;
    int users = 0;  // classes holding it
    double last_use = 0.0;
    std::vector<cudaEvent_t> released;  // end of the work of classes that used it
};

// Page-locked host blocks, reused by size class and released only when the
// server stops (so no host allocation call stalls the device's work).
struct PinnedPool {
    std::map<size_t, std::vector<void*>> free_blocks;
    std::vector<void*> all;
    static size_t bucket(size_t b) {
        size_t s = 256;
        while (s < b) s <<= 1;
        return s;
    }
    void* get(size_t bytes) {
        auto& v = free_blocks[bucket(bytes)];
        if (!v.empty()) {
            void* q = v.back();
            v.pop_back();
            return q;
        }
        void* q = nullptr;
        if (cudaMallocHost(&q, bucket(bytes)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        all.push_back(q);
        return q;
    }
    void put(void* q, size_t bytes) {
        if (q) free_blocks[bucket(bytes)].push_back(q);
    }
    void release() {
        for (void* q : all) cudaFreeHost(q);
        all.clear();
        free_blocks.clear();
    }
};

// One chain of a class (host mirror of slot state).
struct Slot {
    uint64_t ticket = 0;
    ChainCtl ctl{};
    double t_submit = 0.0, t_admit = 0.0;
};

struct Bucket;

struct Class {
    Geometry* g = nullptr;
    Bucket* bk = nullptr;  // the bucket whose launches run this class, or NULL (own stream and launches)
    int K = 1, M = 0;
    float beta = 1.0f;
    sat_params prm{};  // class-wide fields (K, beta, M, residency, group warps)
    Plan pl;
    int plan_n = -1;   // n the plan was made for
    int cap = 0;       // chain capacity of the arrays
    void* dev = nullptr;
    size_t dev_bytes = 0;
    BatchDev b;
    ChainCtl* d_ctl = nullptr;
    int* d_counter = nullptr;
    unsigned long long* d_stamps = nullptr;
    // pinned host mirrors
    ChainCtl* h_ctl = nullptr;
    double* h_scal = nullptr;  // [8][cap]: T0, TN, cost0, costF, S_inc, drift_max, accepted, found
    int* h_err = nullptr;
    unsigned long long* h_stamps = nullptr;
    float* h_img = nullptr;    // [cap][P] images of finishing chains
    size_t hb_ctl = 0, hb_scal = 0, hb_img = 0;  // their sizes (pinned-pool blocks)
    std::vector<std::pair<void*, size_t>> staging;  // request inputs being copied in
    std::vector<Slot> slots;   // [n] active chains
    int n_ready = 0;           // chains whose setup has been enqueued
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool in_flight = false;
    std::vector<int> finishing;  // slots that complete with the tick in flight
    cudaGraphExec_t exec = nullptr;
    int exec_n = -1, exec_windows = 0;
    int windows = 1;       // resync windows per tick (grows until a tick is ~kTickTargetMs)
    int tick_windows = 1;  // windows of the tick in flight
    double tick_ms = 0.0;
};

// Classes of one image size and table precision, run by one sweep launch
// per window over all their chains (the windowed kernel on groups of 4 warps
// reading each chain's class arguments).
struct Bucket {
    int n = 0, precision = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool in_flight = false;
    std::vector<Class*> members;  // classes of the tick in flight
    Plan pl;
    int plan_chains = -1;
    int cap_chains = 0, cap_classes = 0;
    void* dev = nullptr;
    size_t dev_bytes = 0;
    int2* d_map = nullptr;         // [cap_chains] (class, chain in class)
    int* d_progress = nullptr;     // [cap_chains]
    SatArgs* d_classes = nullptr;  // [cap_classes]
    int* d_counter = nullptr;      // [kMaxWindowsPerTick]
    int* d_error = nullptr;
    unsigned long long* d_stamps = nullptr;
    int2* h_map = nullptr;
    SatArgs* h_classes = nullptr;
    size_t hb_map = 0, hb_classes = 0;
    int windows = 1;
};

}  // namespace
}  // namespace satpila

using namespace satpila;

struct satpila_server {
    sat_server_cfg cfg{};
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::unique_ptr<Request>> queue;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_map<uint64_t, int> state;  // 0 queued, 1 active
    uint64_t next_ticket = 1;
    bool stop = false;
    int fatal = 0;
    std::string fatal_msg;
    sat_server_stats st{};
    // engine-thread state
    std::list<std::unique_ptr<Geometry>> geoms;
    std::list<std::unique_ptr<Class>> classes;
    std::list<std::unique_ptr<Bucket>> buckets;
    size_t bytes_in_use = 0;
    cudaStream_t build_stream = nullptr;
    cudaMemPool_t pool = nullptr;  // stream-ordered device memory of tables and classes
    std::string where;             // the step a failed CUDA call belonged to
    PinnedPool pinned;
    std::thread worker;

    void run();
    Geometry* geometry_for(const Request& r, size_t budget_left);
    Class* class_for(Geometry* g, const Request& r);
    int grow(Class* c, int need);
    cudaError_t setup_chains(Class* c, int first, int count, std::vector<std::unique_ptr<Request>>& reqs);
    cudaError_t launch_tick(Class* c);
    cudaError_t enqueue_results(Class* c, const int* d_error, const unsigned long long* d_stamps);
    cudaError_t finish_tick(Class* c);
    Bucket* bucket_for(int n, int precision);
    int bucket_reserve(Bucket* bk, int chains, int n_classes);
    cudaError_t launch_bucket_tick(Bucket* bk);
    void release_bucket(Bucket* bk);
    void release_class(Class* c);
    void fail_all(int code, const std::string& msg);
    size_t budget() const { return (size_t)cfg.mem_budget; }
};

// ---- memory ----------------------------------------------------------------

Geometry* satpila_server::geometry_for(const Request& r, size_t budget_left) {
    GeomKey key{r.n, r.U, r.B, r.precision, r.angles, r.mask};
    for (auto& g : geoms)
        if (g->key == key) return g.get();
    // a table of this size: records + list + mask + per-pixel sums
    const size_t P = (size_t)r.n * r.n;
    const size_t rec = r.precision == PILA_U8 ? 4 : r.precision == PILA_F16 ? 8 : 16;
    const size_t rows = ((size_t)r.U + 16 / rec - 1) / (16 / rec) * (16 / rec);
    const size_t need = P * rows * rec + P * 9 + (size_t)r.U * 16 + 4096;
    // evict unused tables, least recently used first
    while (need > budget_left) {
        Geometry* victim = nullptr;
        for (auto& g : geoms)
            if (g->users == 0 && (!victim || g->last_use < victim->last_use)) victim = g.get();
        if (!victim) return nullptr;
        bytes_in_use -= victim->bytes;
        budget_left += victim->bytes;
        for (cudaEvent_t ev : victim->released) {
            cudaStreamWaitEvent(build_stream, ev, 0);  // its classes' last kernels come first
            cudaEventDestroy(ev);
        }
        pila_free(victim->p);  // stream-ordered release on build_stream
        geoms.remove_if([&](const std::unique_ptr<Geometry>& g) { return g.get() == victim; });
    }
    pila_geom pg{};
    pg.n = r.n;
    pg.n_angles = r.U;
    pg.n_bins = r.B;
    pg.angles_rad = r.angles.empty() ? nullptr : r.angles.data();
    pg.mask = r.mask.empty() ? nullptr : r.mask.data();
    satpila_pila* p = nullptr;
    // no ray index: tables are what bounds the engine's memory (its resyncs
    // take the pixel-driven projector)
    if (pila_build_in(&pg, r.precision, build_stream, pool, &p, false) != SATPILA_OK) return nullptr;
    auto g = std::make_unique<Geometry>();
    g->key = std::move(key);
    g->p = p;
    g->bytes = (size_t)p->table_bytes + P * 9 + (size_t)p->U * 16;
    bytes_in_use += g->bytes;
    geoms.push_back(std::move(g));
    return geoms.back().get();
}

Class* satpila_server::class_for(Geometry* g, const Request& r) {
    const int M = r.prm.moves_per_sweep > 0 ? r.prm.moves_per_sweep : g->p->n_mask;
    const bool merged = !(cfg.flags & SAT_SERVER_PER_CLASS) && multi_table_ok(g->p, &r.prm);
    for (auto& c : classes)
        if (c->g == g && c->K == r.prm.bome_k && c->beta == r.prm.beta && c->M == M &&
            c->prm.residency == r.prm.residency && c->prm.group_warps == r.prm.group_warps &&
            c->prm.pipeline_depth == r.prm.pipeline_depth && (c->bk != nullptr) == merged &&
            !(merged && c->in_flight))  // a bucket class in flight: a sibling class takes the request
            return c.get();
    auto c = std::make_unique<Class>();
    c->g = g;
    c->K = r.prm.bome_k;
    c->beta = r.prm.beta;
    c->M = M;
    c->prm = r.prm;
    c->prm.flags = 0;
    c->prm.trace = nullptr;
    c->prm.sweep_cost = nullptr;
    c->prm.trace_chain = -1;
    if (merged) {
        // the residual layout of the windowed group kernel (interleaved rows)
        if (choose_plan(g->p, 1, cfg.stages_per_tick, &c->prm, PLAN_WINDOW_G4, &c->pl) != SATPILA_OK) return nullptr;
        c->bk = bucket_for(g->p->n, g->p->precision);
        if (!c->bk) return nullptr;
        c->stream = c->bk->stream;
    } else {
        if (choose_plan(g->p, 1, cfg.stages_per_tick, &c->prm, PLAN_RULES, &c->pl) != SATPILA_OK) return nullptr;
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (c->stream) cudaStreamDestroy(c->stream);
            return nullptr;
        }
    }
    g->users++;
    classes.push_back(std::move(c));
    return classes.back().get();
}

// Capacity for `need` chains: new arrays, the active chains copied over.
int satpila_server::grow(Class* c, int need) {
    if (need <= c->cap) return SATPILA_OK;
    const satpila_pila* p = c->g->p;
    const int cap = std::max(need, std::max(4, c->cap * 2));
    const size_t P = (size_t)p->n * p->n, cells = (size_t)p->U * p->B;
    const size_t bb = batch_bytes(c->pl, cap);
    const size_t off_img = align_up(bb, 256);
    const size_t off_sino = align_up(off_img + (size_t)cap * P * 4, 256);
    const size_t off_ctl = align_up(off_sino + (size_t)cap * cells * 4, 256);
    const size_t off_cnt = align_up(off_ctl + (size_t)cap * sizeof(ChainCtl), 256);
    const size_t off_st = off_cnt + 256;
    const size_t bytes = off_st + 256;
    if (bytes_in_use - c->dev_bytes + bytes > budget()) return SATPILA_ERR_OOM;
    void* dev = nullptr;
    if (cudaMallocFromPoolAsync(&dev, bytes, pool, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return SATPILA_ERR_OOM;
    }
    const size_t hb_ctl = (size_t)cap * sizeof(ChainCtl), hb_scal = (size_t)8 * cap * sizeof(double) + 64;
    const size_t hb_img = (size_t)cap * P * sizeof(float);
    auto* h_ctl = (ChainCtl*)pinned.get(hb_ctl);
    auto* h_scal = (double*)pinned.get(hb_scal);
    auto* h_img = (float*)pinned.get(hb_img);
    if (!h_ctl || !h_scal || !h_img) {
        pinned.put(h_ctl, hb_ctl);
        pinned.put(h_scal, hb_scal);
        pinned.put(h_img, hb_img);
        cudaFreeAsync(dev, c->stream);
        return SATPILA_ERR_OOM;
    }
    BatchDev nb;
    batch_carve(dev, c->pl, cap, &nb);
    char* base = (char*)dev;
    nb.img = (float*)(base + off_img);
    nb.sino = (const float*)(base + off_sino);
    ChainCtl* d_ctl = (ChainCtl*)(base + off_ctl);
    nb.ctl = d_ctl;
    cudaError_t e = cudaMemsetAsync(dev, 0, bytes, c->stream);
    const int n = c->n_ready;
    if (n > 0 && e == cudaSuccess) {
        // move the live chains' state into the new arrays (stream-ordered)
        const BatchDev& ob = c->b;
        const int G = c->pl.proj_G;
        struct {
            void* d;
            const void* s;
            size_t bytes;
        } cps[] = {{nb.resid, ob.resid, (size_t)n * c->pl.resid_floats * 4},
                   {nb.img, ob.img, (size_t)n * P * 4},
                   {(void*)nb.sino, ob.sino, (size_t)n * cells * 4},
                   {nb.S, ob.S, (size_t)n * 8},
                   {nb.T0, ob.T0, (size_t)n * 8},
                   {nb.TN, ob.TN, (size_t)n * 8},
                   {nb.found, ob.found, (size_t)n * 4},
                   {nb.accepted, ob.accepted, (size_t)n * 8},
                   {nb.part_sq, ob.part_sq, (size_t)n * G * 8},
                   {nb.part_drift, ob.part_drift, (size_t)n * G * 4},
                   {nb.drift_max, ob.drift_max, (size_t)n * 8},
                   {nb.cost0, ob.cost0, (size_t)n * 8},
                   {nb.costF, ob.costF, (size_t)n * 8},
                   {nb.S_inc, ob.S_inc, (size_t)n * 8},
                   {d_ctl, c->d_ctl, (size_t)n * sizeof(ChainCtl)}};
        for (auto& cp : cps)
            if (e == cudaSuccess) e = cudaMemcpyAsync(cp.d, cp.s, cp.bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) std::memcpy(h_ctl, c->h_ctl, (size_t)n * sizeof(ChainCtl));
    }
    if (e != cudaSuccess) {
        pinned.put(h_ctl, hb_ctl);
        pinned.put(h_scal, hb_scal);
        pinned.put(h_img, hb_img);
        cudaFreeAsync(dev, c->stream);
        return cuda_fail(e, "sat_server: growing a class");
    }
    // the old arrays go back to the pool after the copies (stream order);
    // no copy into the old host blocks is pending between ticks
    if (c->dev) cudaFreeAsync(c->dev, c->stream);
    pinned.put(c->h_ctl, c->hb_ctl);
    pinned.put(c->h_scal, c->hb_scal);
    pinned.put(c->h_img, c->hb_img);
    bytes_in_use = bytes_in_use - c->dev_bytes + bytes;
    c->dev = dev;
    c->dev_bytes = bytes;
    c->cap = cap;
    c->b = nb;
    c->d_ctl = d_ctl;
    c->d_counter = (int*)(base + off_cnt);
    c->d_stamps = (unsigned long long*)(base + off_st);
    c->h_ctl = h_ctl;
    c->h_scal = h_scal;
    c->h_img = h_img;
    c->h_err = reinterpret_cast<int*>(h_scal + 8 * (size_t)cap);
    c->h_stamps = reinterpret_cast<unsigned long long*>(h_scal + 8 * (size_t)cap) + 2;
    c->hb_ctl = hb_ctl;
    c->hb_scal = hb_scal;
    c->hb_img = hb_img;
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
        c->exec_n = -1;
    }
    return SATPILA_OK;
}

void satpila_server::release_class(Class* c) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->dev) cudaFreeAsync(c->dev, c->stream);
    cudaEvent_t done_ev = nullptr;
    if (cudaEventCreateWithFlags(&done_ev, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventRecord(done_ev, c->stream) == cudaSuccess)
        c->g->released.push_back(done_ev);
    else if (done_ev)
        cudaEventDestroy(done_ev);
    cudaGetLastError();
    // between ticks no copy into these host blocks is pending
    pinned.put(c->h_ctl, c->hb_ctl);
    pinned.put(c->h_scal, c->hb_scal);
    pinned.put(c->h_img, c->hb_img);
    for (auto& b : c->staging) pinned.put(b.first, b.second);
    c->staging.clear();
    if (!c->bk) {
        if (c->ev) cudaEventDestroy(c->ev);
        if (c->stream) cudaStreamDestroy(c->stream);  // returns at once; queued work still completes
    }
    bytes_in_use -= c->dev_bytes;
    c->g->users--;
    c->g->last_use = now_ms(t0);
}

// ---- chain setup, ticks, retirement ----------------------------------------

// Chains [first, first + count) of c: inputs in, residual and S by a fresh
// resync, Eq. (4) cost, temperatures.
cudaError_t satpila_server::setup_chains(Class* c, int first, int count,
                                         std::vector<std::unique_ptr<Request>>& reqs) {
    const satpila_pila* p = c->g->p;
    const size_t P = (size_t)p->n * p->n, cells = (size_t)p->U * p->B;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        const Request& r = *reqs[i];
        const int s = first + i;
        // inputs through a page-locked block, released after the next tick
        const size_t bytes = (cells + P) * 4;
        auto* st = (float*)pinned.get(bytes);
        if (!st) return cudaErrorMemoryAllocation;
        c->staging.push_back({st, bytes});
        std::memcpy(st, r.sino.data(), cells * 4);
        std::memcpy(st + cells, r.image.data(), P * 4);
        e = cudaMemcpyAsync((void*)(c->b.sino + (size_t)s * cells), st, cells * 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->b.img + (size_t)s * P, st + cells, P * 4, cudaMemcpyHostToDevice, c->stream);
    }
    const int G = c->pl.proj_G;
    auto zero = [&](void* ptr, size_t each) {
        if (e == cudaSuccess) e = cudaMemsetAsync((char*)ptr + (size_t)first * each, 0, (size_t)count * each, c->stream);
    };
    zero(c->b.accepted, 8);
    zero(c->b.drift_max, 8);
    zero(c->b.found, 4);
    zero(c->b.part_drift, (size_t)G * 4);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_ctl + first, c->h_ctl + first, (size_t)count * sizeof(ChainCtl),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = enqueue_resync(p, c->pl, c->b, first, count, false, c->b.cost0, c->stream);
    if (e == cudaSuccess) e = enqueue_t0(p, c->pl, c->b, &c->prm, first, count, c->stream);
    // until a window runs, the final and the incremental cost are the initial ones
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->b.costF + first, c->b.cost0 + first, (size_t)count * 8, cudaMemcpyDeviceToDevice,
                            c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->b.S_inc + first, c->b.S + first, (size_t)count * 8, cudaMemcpyDeviceToDevice,
                            c->stream);
    return e;
}

cudaError_t satpila_server::launch_tick(Class* c) {
    const satpila_pila* p = c->g->p;
    const int n = (int)c->slots.size();
    const int w = cfg.stages_per_tick;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        where = "an earlier call";
        return e;
    }
    if (c->plan_n != n) {
        Plan pl;
        if (choose_plan(p, n, w, &c->prm, PLAN_RULES, &pl) != SATPILA_OK) {
            where = std::string("plan: ") + satpila_last_error();
            return cudaErrorInvalidValue;
        }
        if ((e = prepare_launches(p, pl, c->K)) != cudaSuccess) {
            where = "launch attributes";
            return e;
        }
        c->pl = pl;  // array layout (resid_floats, proj_G) does not depend on n
        c->plan_n = n;
    }
    // A tick is `T` windows of w stages, each followed by the resync (so the
    // resync cadence, and with it every result, does not depend on T).
    const int T = c->windows;
    c->tick_windows = T;
    int max_total = 0;
    c->finishing.clear();
    for (int i = 0; i < n; ++i) {
        c->h_ctl[i] = c->slots[i].ctl;
        max_total = std::max(max_total, c->slots[i].ctl.n_sweeps);
        if (c->slots[i].ctl.stage0 + w * T >= c->slots[i].ctl.n_sweeps) c->finishing.push_back(i);
    }
    // The compute of a tick as one graph, rebuilt when the batch size or T changes.
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t err = cudaMemcpyAsync(c->d_ctl, c->h_ctl, (size_t)n * sizeof(ChainCtl), cudaMemcpyHostToDevice, q);
        if (err == cudaSuccess) err = cudaMemsetAsync(c->b.progress, 0, (size_t)n * 4, q);
        if (err == cudaSuccess) err = cudaMemsetAsync(c->d_counter, 0, (size_t)T * 4, q);
        if (err == cudaSuccess) {
            tick_stamp_kernel<<<1, 1, 0, q>>>(c->d_stamps);
            err = cudaGetLastError();
        }
        for (int t = 0; t < T && err == cudaSuccess; ++t) {
            err = enqueue_sweep(p, c->pl, c->b, &c->prm, n, c->M, max_total, t * w, (t + 1) * w, c->d_counter + t, q);
            if (err == cudaSuccess) {
                s_inc_kernel<<<(n + 127) / 128, 128, 0, q>>>(c->b.S_inc, c->b.S, c->d_ctl, n, t * w);
                err = cudaGetLastError();
            }
            if (err == cudaSuccess) err = enqueue_resync(p, c->pl, c->b, 0, n, true, c->b.costF, q);
        }
        if (err == cudaSuccess) {
            tick_stamp_kernel<<<1, 1, 0, q>>>(c->d_stamps + 1);
            err = cudaGetLastError();
        }
        return err;
    };
    if (c->exec_n != n || c->exec_windows != T) {
        if (c->exec) cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
        cudaGraph_t graph = nullptr;
        cudaStream_t cs = nullptr;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e1 = enqueue(cs);
            e = cudaStreamEndCapture(cs, &graph);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->exec = nullptr;
        }
        c->exec_n = c->exec ? n : -1;
        c->exec_windows = T;
    }
    e = c->exec ? cudaGraphLaunch(c->exec, c->stream) : enqueue(c->stream);
    if (e != cudaSuccess) {
        where = c->exec ? "graph launch" : "direct launches";
        return e;
    }
    e = enqueue_results(c, c->b.error, c->d_stamps);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev, c->stream);
    if (e == cudaSuccess) c->in_flight = true;
    else where = "result copies";
    return e;
}

// Statistics of every chain of c, the images of its finishing ones, the
// tick's error word and time stamps, copied out behind the tick.
cudaError_t satpila_server::enqueue_results(Class* c, const int* d_error, const unsigned long long* d_stamps) {
    const int n = (int)c->slots.size();
    const double* src[7] = {c->b.T0, c->b.TN, c->b.cost0, c->b.costF, c->b.S_inc, c->b.drift_max,
                            (const double*)c->b.accepted};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 7 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(c->h_scal + (size_t)k * c->cap, src[k], (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->h_scal + (size_t)7 * c->cap, c->b.found, (size_t)n * 4, cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_err, d_error, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_stamps, d_stamps, 16, cudaMemcpyDeviceToHost, c->stream);
    const size_t P = (size_t)c->g->p->n * c->g->p->n;
    for (int i : c->finishing)
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->h_img + (size_t)i * P, c->b.img + (size_t)i * P, P * 4, cudaMemcpyDeviceToHost,
                                c->stream);
    return e;
}

// ---- buckets: one sweep launch over the classes of an image size -----------

Bucket* satpila_server::bucket_for(int n, int precision) {
    for (auto& b : buckets)
        if (b->n == n && b->precision == precision) return b.get();
    auto b = std::make_unique<Bucket>();
    b->n = n;
    b->precision = precision;
    if (prepare_multi(precision) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (b->stream) cudaStreamDestroy(b->stream);
        return nullptr;
    }
    buckets.push_back(std::move(b));
    return buckets.back().get();
}

// Room for `chains` chains of `n_classes` classes in the bucket's arrays (the
// bucket is between ticks, so nothing in flight reads the old ones).  These
// few kilobytes of launch bookkeeping sit outside the memory budget, which
// bounds tables and chain state: a tick never waits for them.
int satpila_server::bucket_reserve(Bucket* bk, int chains, int n_classes) {
    if (chains <= bk->cap_chains && n_classes <= bk->cap_classes) return SATPILA_OK;
    const int cc = std::max(chains, std::max(16, bk->cap_chains * 2));
    const int nc = std::max(n_classes, std::max(8, bk->cap_classes * 2));
    const size_t off_prog = align_up((size_t)cc * sizeof(int2), 256);
    const size_t off_cls = align_up(off_prog + (size_t)cc * 4, 256);
    const size_t off_cnt = align_up(off_cls + (size_t)nc * sizeof(SatArgs), 256);
    const size_t off_err = align_up(off_cnt + (size_t)kMaxWindowsPerTick * 4, 256);
    const size_t off_st = off_err + 256;
    const size_t bytes = off_st + 256;
    void* dev = nullptr;
    if (cudaMallocFromPoolAsync(&dev, bytes, pool, bk->stream) != cudaSuccess) {
        cudaGetLastError();
        return SATPILA_ERR_OOM;
    }
    const size_t hb_map = (size_t)cc * sizeof(int2), hb_classes = (size_t)nc * sizeof(SatArgs);
    auto* h_map = (int2*)pinned.get(hb_map);
    auto* h_classes = (SatArgs*)pinned.get(hb_classes);
    if (!h_map || !h_classes) {
        pinned.put(h_map, hb_map);
        pinned.put(h_classes, hb_classes);
        cudaFreeAsync(dev, bk->stream);
        return SATPILA_ERR_OOM;
    }
    if (bk->dev) cudaFreeAsync(bk->dev, bk->stream);
    pinned.put(bk->h_map, bk->hb_map);
    pinned.put(bk->h_classes, bk->hb_classes);
    char* base = (char*)dev;
    bk->dev = dev;
    bk->dev_bytes = bytes;
    bk->cap_chains = cc;
    bk->cap_classes = nc;
    bk->d_map = (int2*)base;
    bk->d_progress = (int*)(base + off_prog);
    bk->d_classes = (SatArgs*)(base + off_cls);
    bk->d_counter = (int*)(base + off_cnt);
    bk->d_error = (int*)(base + off_err);
    bk->d_stamps = (unsigned long long*)(base + off_st);
    bk->h_map = h_map;
    bk->h_classes = h_classes;
    bk->hb_map = hb_map;
    bk->hb_classes = hb_classes;
    if (cudaMemsetAsync(dev, 0, bytes, bk->stream) != cudaSuccess) {
        cudaGetLastError();
        return SATPILA_ERR_CUDA;
    }
    return SATPILA_OK;
}

// A tick of every class of the bucket with chains: `windows` windows of
// stages_per_tick stages, each one sweep launch over all their chains
// followed by every class's resync, then each class's results.
cudaError_t satpila_server::launch_bucket_tick(Bucket* bk) {
    bk->members.clear();
    int total = 0;
    for (auto& c : classes)
        if (c->bk == bk && !c->slots.empty()) {
            bk->members.push_back(c.get());
            total += (int)c->slots.size();
        }
    if (bk->members.empty()) return cudaSuccess;
    const int w = cfg.stages_per_tick;
    const int T = bk->windows;
    const int nq = (int)bk->members.size();
    if (bucket_reserve(bk, total, nq) != SATPILA_OK) {
        where = std::string("bucket arrays: ") + satpila_last_error();
        return cudaErrorMemoryAllocation;
    }
    if (bk->plan_chains != total) {
        if (plan_multi(bk->precision, total, w, &bk->pl) != SATPILA_OK) {
            where = std::string("plan: ") + satpila_last_error();
            return cudaErrorInvalidValue;
        }
        bk->plan_chains = total;
    }
    int off = 0;
    for (int q = 0; q < nq; ++q) {
        Class* c = bk->members[q];
        const int n = (int)c->slots.size();
        int max_total = 0;
        c->finishing.clear();
        c->tick_windows = T;
        for (int i = 0; i < n; ++i) {
            c->h_ctl[i] = c->slots[i].ctl;
            max_total = std::max(max_total, c->slots[i].ctl.n_sweeps);
            if (c->slots[i].ctl.stage0 + w * T >= c->slots[i].ctl.n_sweeps) c->finishing.push_back(i);
            bk->h_map[off + i] = make_int2(q, i);
        }
        SatArgs ca = sweep_args(c->g->p, c->pl, c->b, &c->prm, n, c->M, max_total, 0, w, nullptr);
        ca.stage_bytes = bk->pl.stage_bytes;
        ca.D = bk->pl.D;
        ca.W = bk->pl.W;
        ca.group_smem_bytes = bk->pl.group_smem;
        ca.classes = nullptr;
        ca.chain_map = nullptr;
        bk->h_classes[q] = ca;
        off += n;
    }
    cudaStream_t q = bk->stream;
    cudaError_t e = cudaSuccess;
    for (Class* c : bk->members)
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->d_ctl, c->h_ctl, c->slots.size() * sizeof(ChainCtl), cudaMemcpyHostToDevice, q);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bk->d_classes, bk->h_classes, (size_t)nq * sizeof(SatArgs), cudaMemcpyHostToDevice, q);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bk->d_map, bk->h_map, (size_t)total * sizeof(int2), cudaMemcpyHostToDevice, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(bk->d_progress, 0, (size_t)total * 4, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(bk->d_counter, 0, (size_t)T * 4, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(bk->d_error, 0, 4, q);
    if (e == cudaSuccess) {
        tick_stamp_kernel<<<1, 1, 0, q>>>(bk->d_stamps);
        e = cudaGetLastError();
    }
    const int spt = bk->pl.spt;
    for (int t = 0; t < T && e == cudaSuccess; ++t) {
        SatArgs la = bk->h_classes[0];
        la.classes = bk->d_classes;
        la.chain_map = bk->d_map;
        la.n_chains = total;
        la.progress = bk->d_progress;
        la.error = bk->d_error;
        la.claim = nullptr;
        la.ctl = nullptr;
        la.trace = nullptr;
        la.sweep_cost = nullptr;
        la.stall_chain = -1;
        la.sweep_begin = t * w;
        la.sweep_end = (t + 1) * w;
        la.sweeps_per_task = spt;
        la.n_tasks = total * ((w + spt - 1) / spt);
        la.task_counter = bk->d_counter + t;
        e = enqueue_sweep_multi(bk->precision, bk->pl, la, q);
        for (Class* c : bk->members) {
            const int n = (int)c->slots.size();
            if (e == cudaSuccess) {
                s_inc_kernel<<<(n + 127) / 128, 128, 0, q>>>(c->b.S_inc, c->b.S, c->d_ctl, n, t * w);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = enqueue_resync(c->g->p, c->pl, c->b, 0, n, true, c->b.costF, q);
        }
    }
    if (e == cudaSuccess) {
        tick_stamp_kernel<<<1, 1, 0, q>>>(bk->d_stamps + 1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        where = "bucket launches";
        return e;
    }
    for (Class* c : bk->members)
        if (e == cudaSuccess) e = enqueue_results(c, bk->d_error, bk->d_stamps);
    if (e == cudaSuccess) e = cudaEventRecord(bk->ev, q);
    if (e != cudaSuccess) {
        where = "result copies";
        return e;
    }
    bk->in_flight = true;
    for (Class* c : bk->members) c->in_flight = true;
    return cudaSuccess;
}

void satpila_server::release_bucket(Bucket* bk) {
    if (bk->in_flight) cudaEventSynchronize(bk->ev);
    if (bk->dev) cudaFreeAsync(bk->dev, bk->stream);
    cudaStreamSynchronize(bk->stream);
    pinned.put(bk->h_map, bk->hb_map);
    pinned.put(bk->h_classes, bk->hb_classes);
    if (bk->ev) cudaEventDestroy(bk->ev);
    if (bk->stream) cudaStreamDestroy(bk->stream);
    cudaGetLastError();
}

cudaError_t satpila_server::finish_tick(Class* c) {
    c->in_flight = false;
    for (auto& b : c->staging) pinned.put(b.first, b.second);  // copied in before the tick
    c->staging.clear();
    const satpila_pila* p = c->g->p;
    const int w = cfg.stages_per_tick;
    const int n = (int)c->slots.size();
    const size_t P = (size_t)p->n * p->n, cells = (size_t)p->U * p->B;
    const double t = now_ms(t0);
    const int err_code = *c->h_err;
    c->tick_ms = 1e-6 * (double)(c->h_stamps[1] - c->h_stamps[0]);
    long long moves = 0;
    const int ws = w * c->tick_windows;
    if (c->tick_ms < 0.5 * kTickTargetMs && c->windows < kMaxWindowsPerTick) c->windows *= 2;
    else if (c->tick_ms > 4.0 * kTickTargetMs && c->windows > 1) c->windows /= 2;
    for (int i = 0; i < n; ++i) {
        Slot& sl = c->slots[i];
        const int run = std::max(0, std::min(ws, sl.ctl.n_sweeps - sl.ctl.stage0));
        moves += (long long)run * (p->n_mask > 0 ? c->M : 0);
        sl.ctl.stage0 += run;
    }
    const double* sc = c->h_scal;
    const int cap = c->cap;
    {
        std::lock_guard<std::mutex> lock(mu);
        st.ticks++;
        st.moves += moves;
        for (int i : c->finishing) {
            Slot& sl = c->slots[i];
            Done d;
            sat_stats& s = d.res.stats;
            s.t0 = sc[0 * cap + i];
            s.tn = sc[1 * cap + i];
            s.initial_cost = sc[2 * cap + i];
            s.final_cost = sc[3 * cap + i];
            s.final_cost_incremental = std::sqrt(std::max(0.0, sc[4 * cap + i] / (double)cells));
            s.max_resync_drift = sc[5 * cap + i];
            unsigned long long acc;
            std::memcpy(&acc, &sc[6 * cap + i], 8);
            s.accepted = (int64_t)acc;
            s.proposed = (int64_t)sl.ctl.n_sweeps * (p->n_mask > 0 ? c->M : 0);
            s.t0_found = reinterpret_cast<const int*>(sc + (size_t)7 * cap)[i];
            s.status = err_code;
            s.sweep_ms = c->tick_ms;
            s.plan = plan_code(c->pl);
            s.near_ties = -1;
            d.res.submit_ms = sl.t_submit;
            d.res.admit_ms = sl.t_admit;
            d.res.done_ms = t;
            d.image.assign(c->h_img + (size_t)i * P, c->h_img + (size_t)(i + 1) * P);
            done[sl.ticket] = std::move(d);
            state.erase(sl.ticket);
            if (err_code) st.failed++;
            else st.completed++;
        }
    }
    cv_done.notify_all();
    // compaction: the last live chains move into the finished slots
    std::vector<int> fin = c->finishing;
    std::sort(fin.rbegin(), fin.rend());
    cudaError_t e = cudaSuccess;
    const int G = c->pl.proj_G;
    for (int f : fin) {
        const int last = (int)c->slots.size() - 1;
        if (f != last) {
            const BatchDev& b = c->b;
            struct {
                void* base;
                size_t each;
            } arrs[] = {{b.resid, (size_t)c->pl.resid_floats * 4},
                        {b.img, P * 4},
                        {(void*)b.sino, cells * 4},
                        {b.S, 8},
                        {b.T0, 8},
                        {b.TN, 8},
                        {b.found, 4},
                        {b.accepted, 8},
                        {b.part_sq, (size_t)G * 8},
                        {b.part_drift, (size_t)G * 4},
                        {b.drift_max, 8},
                        {b.cost0, 8},
                        {b.costF, 8},
                        {b.S_inc, 8}};
            for (auto& a : arrs)
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync((char*)a.base + (size_t)f * a.each, (char*)a.base + (size_t)last * a.each,
                                        a.each, cudaMemcpyDeviceToDevice, c->stream);
            c->slots[f] = c->slots[last];
        }
        c->slots.pop_back();
    }
    c->n_ready = (int)c->slots.size();
    if (err_code) {
        // a device-side check failed: the class's remaining chains fail too
        std::lock_guard<std::mutex> lock(mu);
        for (Slot& sl : c->slots) {
            Done d;
            d.res.stats.status = err_code;
            d.res.submit_ms = sl.t_submit;
            d.res.admit_ms = sl.t_admit;
            d.res.done_ms = t;
            done[sl.ticket] = std::move(d);
            state.erase(sl.ticket);
            st.failed++;
        }
        c->slots.clear();
        c->n_ready = 0;
        cudaMemsetAsync(c->b.error, 0, 4, c->stream);
        cv_done.notify_all();
    }
    return e;
}

void satpila_server::fail_all(int code, const std::string& msg) {
    std::lock_guard<std::mutex> lock(mu);
    fatal = code;
    fatal_msg = msg;
    const double t = now_ms(t0);
    auto fail_ticket = [&](uint64_t tk, double ts) {
        Done d;
        d.res.stats.status = code;
        d.res.submit_ms = ts;
        d.res.done_ms = t;
        done[tk] = std::move(d);
        st.failed++;
    };
    for (auto& c : classes)
        for (Slot& sl : c->slots) fail_ticket(sl.ticket, sl.t_submit);
    for (auto& r : queue) fail_ticket(r->ticket, r->t_submit);
    queue.clear();
    state.clear();
    cv_done.notify_all();
}

void satpila_server::run() {
    cudaSetDevice(cfg.device);
    cudaStreamCreateWithFlags(&build_stream, cudaStreamNonBlocking);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = cfg.device;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pool = nullptr;
        fail_all(SATPILA_ERR_CUDA, "sat_server: no device memory pool");
        return;
    }
    uint64_t keep = UINT64_MAX;  // freed blocks stay in the pool for reuse
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    bool failed = false;
    while (!failed) {
        bool worked = false;
        // 1. admission, in arrival order, while slots and memory allow
        {
            std::unique_lock<std::mutex> lock(mu);
            if (stop) break;
        }
        std::map<Class*, std::vector<std::unique_ptr<Request>>> admitted;
        for (;;) {
            std::unique_ptr<Request> r;
            {
                std::lock_guard<std::mutex> lock(mu);
                if (queue.empty()) break;
                int active = 0;
                for (auto& c : classes) active += (int)c->slots.size();
                for (auto& kv : admitted) active += (int)kv.second.size();
                if (active >= cfg.max_active) break;
                r = std::move(queue.front());
                queue.pop_front();
            }
            // table (possibly evicting unused ones), class, capacity
            const size_t left = budget() > bytes_in_use ? budget() - bytes_in_use : 0;
            Geometry* g = geometry_for(*r, left);
            Class* c = g ? class_for(g, *r) : nullptr;
            int rc = c ? SATPILA_OK : SATPILA_ERR_OOM;
            if (c && !c->in_flight) {
                const int need = (int)c->slots.size() + (int)admitted[c].size() + 1;
                rc = grow(c, need);
            } else if (c) {
                rc = SATPILA_ERR_BUSY;  // its class is between launches only after the tick
            }
            if (rc != SATPILA_OK) {
                // does not fit now: back to the head of the queue
                std::lock_guard<std::mutex> lock(mu);
                queue.push_front(std::move(r));
                break;
            }
            g->last_use = now_ms(t0);
            admitted[c].push_back(std::move(r));
        }
        for (auto& kv : admitted) {
            Class* c = kv.first;
            auto& reqs = kv.second;
            if (reqs.empty()) continue;
            const int first = (int)c->slots.size();
            const double t = now_ms(t0);
            for (auto& r : reqs) {
                Slot sl;
                sl.ticket = r->ticket;
                sl.t_submit = r->t_submit;
                sl.t_admit = t;
                sl.ctl.seed = r->prm.seed;
                sl.ctl.t0 = r->prm.t0;
                sl.ctl.tn = r->prm.tn;
                sl.ctl.stage0 = 0;
                sl.ctl.n_sweeps = r->prm.n_sweeps;
                sl.ctl.schedule = r->prm.schedule;
                sl.ctl.t0_samples = r->prm.t0_samples;
                c->h_ctl[c->slots.size()] = sl.ctl;
                c->slots.push_back(sl);
            }
            cudaError_t e = setup_chains(c, first, (int)reqs.size(), reqs);
            if (e != cudaSuccess) {
                fail_all(SATPILA_ERR_CUDA, std::string("sat_server: chain setup: ") + cudaGetErrorString(e));
                failed = true;
                break;
            }
            c->n_ready = (int)c->slots.size();
            std::lock_guard<std::mutex> lock(mu);
            st.admitted += (int64_t)reqs.size();
            for (auto& r : reqs) state[r->ticket] = 1;
            worked = true;
        }
        if (failed) break;
        // 2. every class with chains and no tick in flight launches one (a
        //    chain with no stages left finishes with it)
        for (auto& c : classes) {
            if (c->bk || c->in_flight || c->slots.empty()) continue;
            cudaError_t e = launch_tick(c.get());
            if (e != cudaSuccess) {
                fail_all(SATPILA_ERR_CUDA, std::string("sat_server: tick launch (") + where + "): " + cudaGetErrorString(e));
                failed = true;
                break;
            }
            worked = true;
        }
        if (failed) break;
        for (auto& b : buckets) {
            if (b->in_flight) continue;
            cudaError_t e = launch_bucket_tick(b.get());
            if (e != cudaSuccess) {
                fail_all(SATPILA_ERR_CUDA, std::string("sat_server: tick launch (") + where + "): " + cudaGetErrorString(e));
                failed = true;
                break;
            }
            if (b->in_flight) worked = true;
        }
        if (failed) break;
        // 3. retire finished ticks
        for (auto& b : buckets) {
            if (!b->in_flight) continue;
            const cudaError_t q = cudaEventQuery(b->ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                fail_all(SATPILA_ERR_CUDA, std::string("sat_server: tick: ") + cudaGetErrorString(q));
                failed = true;
                break;
            }
            b->in_flight = false;
            double tick_ms = 0.0;
            for (Class* c : b->members) {
                cudaError_t e = finish_tick(c);
                tick_ms = std::max(tick_ms, c->tick_ms);
                if (e != cudaSuccess) {
                    fail_all(SATPILA_ERR_CUDA, std::string("sat_server: retiring: ") + cudaGetErrorString(e));
                    failed = true;
                    break;
                }
            }
            if (failed) break;
            if (tick_ms < 0.5 * kTickTargetMs && b->windows < kMaxWindowsPerTick) b->windows *= 2;
            else if (tick_ms > 4.0 * kTickTargetMs && b->windows > 1) b->windows /= 2;
            b->members.clear();
            worked = true;
        }
        if (failed) break;
        for (auto& c : classes) {
            if (c->bk || !c->in_flight) continue;
            const cudaError_t q = cudaEventQuery(c->ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                fail_all(SATPILA_ERR_CUDA, std::string("sat_server: tick: ") + cudaGetErrorString(q));
                failed = true;
                break;
            }
            cudaError_t e = finish_tick(c.get());
            if (e != cudaSuccess) {
                fail_all(SATPILA_ERR_CUDA, std::string("sat_server: retiring: ") + cudaGetErrorString(e));
                failed = true;
                break;
            }
            worked = true;
        }
        if (failed) break;
        // 4. empty classes give their memory back
        for (auto it = classes.begin(); it != classes.end();) {
            Class* c = it->get();
            if (!c->in_flight && c->slots.empty()) {
                release_class(c);
                it = classes.erase(it);
            } else {
                ++it;
            }
        }
        {
            std::lock_guard<std::mutex> lock(mu);
            int active = 0;
            for (auto& c : classes) active += (int)c->slots.size();
            st.active = active;
            st.queued = (int32_t)queue.size();
            st.geometries = (int32_t)geoms.size();
            st.classes = (int32_t)classes.size();
            st.bytes_in_use = bytes_in_use;
            st.bytes_peak = std::max<uint64_t>(st.bytes_peak, bytes_in_use);
        }
        if (!worked) {
            std::unique_lock<std::mutex> lock(mu);
            cv_work.wait_for(lock, std::chrono::microseconds(200));
        }
    }
    // shutdown: every class and table back, then wait for this server's
    // device work before its host blocks go
    for (auto& b : buckets)
        if (b->in_flight) cudaEventSynchronize(b->ev);
    for (auto& c : classes) {
        if (!c->bk && c->in_flight) cudaEventSynchronize(c->ev);
        release_class(c.get());
    }
    classes.clear();
    for (auto& b : buckets) release_bucket(b.get());
    buckets.clear();
    for (auto& g : geoms) {
        for (cudaEvent_t ev : g->released) {
            cudaStreamWaitEvent(build_stream, ev, 0);
            cudaEventDestroy(ev);
        }
        g->released.clear();
        pila_free(g->p);
    }
    geoms.clear();
    if (build_stream) {
        cudaStreamSynchronize(build_stream);
        cudaStreamDestroy(build_stream);
    }
    pinned.release();
    if (pool) cudaMemPoolDestroy(pool);
}

// ---- C ABI -------------------------------------------------------------------

namespace {

size_t request_bytes_estimate(int n, int U, int B, int precision) {
    const size_t P = (size_t)n * n;
    const size_t rec = precision == PILA_U8 ? 4 : precision == PILA_F16 ? 8 : 16;
    const size_t rows = ((size_t)U + 16 / rec - 1) / (16 / rec) * (16 / rec);
    const size_t table = P * rows * rec + P * 9 + (size_t)U * 16 + 4096;
    const size_t chain = ((size_t)U * (((size_t)B + 4) & ~(size_t)3) + 256 + P + (size_t)U * B) * 4 + 1024;
    return table + 4 * chain + 8192;  // the class arrays hold at least four chains
}

int copy_in(void* dst, const void* src, size_t bytes) {
    if (is_device_pointer(src)) {
        const cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "sat_server_submit: copying a device buffer");
    } else {
        std::memcpy(dst, src, bytes);
    }
    return SATPILA_OK;
}

}  // namespace

extern "C" int sat_server_create(const sat_server_cfg* cfg, satpila_server** out) {
    if (!out) return fail(SATPILA_ERR_INVALID_ARG, "sat_server_create: null output");
    *out = nullptr;
    sat_server_cfg c{};
    if (cfg) c = *cfg;
    if (c.max_active < 0 || c.stages_per_tick < 0 || c.queue_limit < 0)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_server_create: negative limit");
    if (c.max_active == 0) c.max_active = 4096;
    if (c.stages_per_tick == 0) c.stages_per_tick = 5;
    if (c.queue_limit == 0) c.queue_limit = 1 << 16;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return fail(SATPILA_ERR_INVALID_ARG, "sat_server_create: no such CUDA device");
    }
    int prev = 0;
    cudaGetDevice(&prev);
    size_t free_b = 0, total_b = 0;
    cudaSetDevice(c.device);
    const cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "sat_server_create");
    const uint64_t headroom = 2ull << 30;
    const uint64_t avail = free_b > headroom ? free_b - headroom : free_b / 2;
    if (c.mem_budget == 0) c.mem_budget = 120000000000ull;  // 120 GB (10^9 bytes each)
    c.mem_budget = std::min<uint64_t>(c.mem_budget, avail);
    auto* s = new satpila_server();
    s->cfg = c;
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return SATPILA_OK;
}

extern "C" int sat_server_submit(satpila_server* s, const sat_request* r, uint64_t* ticket) {
    if (!s || !r || !ticket) return fail(SATPILA_ERR_INVALID_ARG, "sat_server_submit: null argument");
    const sat_params& prm = r->prm;
    if (r->n < 1 || r->n_angles < 1 || r->n_bins < 1 || !r->sino)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_server_submit: bad geometry or no sinogram");
    if (r->precision != PILA_F32 && r->precision != PILA_F16 && r->precision != PILA_U8)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_server_submit: unknown precision");
    if (r->precision != PILA_F32 && r->n_bins > 32767)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_server_submit: too many bins for 16-bit indices");
    if (r->precision == PILA_U8 && r->n_angles > 512)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_server_submit: one-byte tables take at most 512 angles");
    if (prm.bome_k < 1 || prm.bome_k > kMaxK || !(prm.beta > 0.0f) || prm.n_sweeps < 0 || prm.moves_per_sweep < 0 ||
        prm.schedule < SAT_SCHED_LINEAR || prm.schedule > SAT_SCHED_CUBIC || prm.residency < SAT_RESIDENT_AUTO ||
        prm.residency > SAT_RESIDENT_GLOBAL)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_server_submit: bad sat_params");
    if (request_bytes_estimate(r->n, r->n_angles, r->n_bins, r->precision) > s->cfg.mem_budget)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_server_submit: request needs more device memory than the budget");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->fatal) return fail(s->fatal, "sat_server_submit: server failed: " + s->fatal_msg);
        if ((int)s->queue.size() >= s->cfg.queue_limit)
            return fail(SATPILA_ERR_BUSY, "sat_server_submit: queue full");
    }
    auto q = std::make_unique<Request>();
    q->n = r->n;
    q->U = r->n_angles;
    q->B = r->n_bins;
    q->precision = r->precision;
    q->prm = prm;
    const size_t P = (size_t)r->n * r->n, cells = (size_t)r->n_angles * r->n_bins;
    int rc = SATPILA_OK;
    if (r->angles_rad) {
        q->angles.resize(r->n_angles);
        rc = copy_in(q->angles.data(), r->angles_rad, (size_t)r->n_angles * 8);
    }
    if (rc == SATPILA_OK && r->mask) {
        q->mask.resize(P);
        rc = copy_in(q->mask.data(), r->mask, P);
        for (auto& m : q->mask) m = m ? 1 : 0;
    }
    q->sino.resize(cells);
    if (rc == SATPILA_OK) rc = copy_in(q->sino.data(), r->sino, cells * 4);
    q->image.resize(P);
    if (rc == SATPILA_OK && r->image) {
        rc = copy_in(q->image.data(), r->image, P * 4);
    } else if (rc == SATPILA_OK) {
        for (size_t i = 0; i < P; ++i) q->image[i] = (q->mask.empty() || q->mask[i]) ? 0.5f : 0.0f;
    }
    if (rc != SATPILA_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if ((int)s->queue.size() >= s->cfg.queue_limit)
            return fail(SATPILA_ERR_BUSY, "sat_server_submit: queue full");
        q->ticket = s->next_ticket++;
        q->t_submit = now_ms(s->t0);
        *ticket = q->ticket;
        s->state[q->ticket] = 0;
        s->queue.push_back(std::move(q));
        s->st.submitted++;
    }
    s->cv_work.notify_one();
    return SATPILA_OK;
}

namespace {

int take_result(satpila_server* s, uint64_t ticket, float* image_out, sat_result* res) {
    // caller holds s->mu
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        if (s->state.count(ticket)) return SATPILA_ERR_PENDING;
        return fail(SATPILA_ERR_NOT_FOUND, "sat_server: unknown or already collected ticket");
    }
    if (res) *res = it->second.res;
    if (image_out && !it->second.image.empty()) {
        const size_t bytes = it->second.image.size() * sizeof(float);
        if (is_device_pointer(image_out)) {
            const cudaError_t e = cudaMemcpy(image_out, it->second.image.data(), bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "sat_server: copying the image");
        } else {
            std::memcpy(image_out, it->second.image.data(), bytes);
        }
    }
    const int status = it->second.res.stats.status;
    s->done.erase(it);
    if (!status) return SATPILA_OK;
    return fail(status, s->fatal ? "sat_server: the server stopped: " + s->fatal_msg
                                 : std::string("sat_server: a device-side check failed for the request"));
}

}  // namespace

extern "C" int sat_server_poll(satpila_server* s, uint64_t ticket, float* image_out, sat_result* res) {
    if (!s) return fail(SATPILA_ERR_INVALID_ARG, "sat_server_poll: null server");
    std::lock_guard<std::mutex> lock(s->mu);
    return take_result(s, ticket, image_out, res);
}

extern "C" int sat_server_wait(satpila_server* s, uint64_t ticket, int32_t timeout_ms, float* image_out,
                               sat_result* res) {
    if (!s) return fail(SATPILA_ERR_INVALID_ARG, "sat_server_wait: null server");
    std::unique_lock<std::mutex> lock(s->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    for (;;) {
        const int rc = take_result(s, ticket, image_out, res);
        if (rc != SATPILA_ERR_PENDING) return rc;
        if (timeout_ms >= 0 && std::chrono::steady_clock::now() >= until) return SATPILA_ERR_PENDING;
        if (timeout_ms < 0) s->cv_done.wait(lock);
        else s->cv_done.wait_until(lock, until);
    }
}

extern "C" int sat_server_info(satpila_server* s, sat_server_stats* out) {
    if (!s || !out) return fail(SATPILA_ERR_INVALID_ARG, "sat_server_info: null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->st;
    out->queued = (int32_t)s->queue.size();
    out->mem_budget = s->cfg.mem_budget;
    return SATPILA_OK;
}

extern "C" int sat_server_destroy(satpila_server* s) {
    if (!s) return SATPILA_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return SATPILA_OK;
}
