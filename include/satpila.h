/*
 * satpila — simulated annealing tomography with a pre-calculated intersection
 * lengths array (PILA), for NVIDIA GB300 (sm_103a).
 *
 * Method: Vo, Breese & Moser, "Feasibility of Simulated Annealing Tomography".
 * Section and equation numbers below refer to that paper.
 *
 * Conventions for every call
 *  - Return value: SATPILA_OK (0) or a negative SATPILA_ERR_* code;
 *    satpila_last_error() then returns a message for the calling thread.
 *  - Geometry (parallel beam, unit pixels, Sec. II-B): pixel (i, j) of an
 *    n x n image (row i from the top) has its centre at
 *    x = j - (n-1)/2, y = (n-1)/2 - i.  Angle u is theta_u (default pi*u/U).
 *    Ray (u, k) is the line x cos(theta_u) + y sin(theta_u) = s_k,
 *    s_k = k - (B-1)/2, i.e. B unit-width bins centred on the axis.  A ray
 *    exactly on a pixel edge (0 and 90 degrees only) belongs to the pixel on
 *    its +s side.
 *  - Layouts: images are row-major float32 [n][n]; sinograms are angle-major
 *    [U][B]; batches are contiguous ([n_chains][U][B], [n_chains][n][n]).
 *  - Buffers are owned by the caller.  Data pointers may be device pointers
 *    (e.g. from torch) or host pointers; host buffers are staged through
 *    device memory inside the call, which then returns only after the
 *    results are back on the host.  With device buffers the call is
 *    asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream)
 *    except where stated.
 *  - Handles (satpila_pila, satpila_server) are owned by the library and are
 *    released with their *_free / *_destroy call.
 */
#ifndef SATPILA_H
#define SATPILA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SATPILA_OK 0
#define SATPILA_ERR_INVALID_ARG (-1)
#define SATPILA_ERR_OOM (-2)
#define SATPILA_ERR_CUDA (-3)
#define SATPILA_ERR_TIMEOUT (-4)   /* a bounded device-side wait gave up */
/* -5 is not used */
#define SATPILA_ERR_BUSY (-6)      /* serving: no slot or memory free right now */
#define SATPILA_ERR_NOT_FOUND (-7) /* serving: unknown ticket */
#define SATPILA_ERR_PENDING (-8)   /* serving: result not ready yet */

/* Thread-local message for the last failing call (never NULL). */
const char* satpila_last_error(void);
/* Library version, major*10000 + minor*100 + patch. */
int satpila_version(void);

/* ------------------------------------------------------------------------ */
/* PILA: Eq. (5) and the surrounding text of Sec. II-B.                       */
/* ------------------------------------------------------------------------ */

#define PILA_F32 0 /* record: int32 bin0, int32 bin1, float len0, float len1 (16 B) */
#define PILA_F16 1 /* record: int16 bin0, int16 bin1, half len0, half len1 (8 B)    */
#define PILA_U8 2  /* record: uint16 bin0, uint8 180*len0, uint8 180*len1 (4 B): the
                      one-byte lengths of Sec. II-B (length = q * fl(1/180)); entry 1
                      sits on bin0 + 1.  Read by the windowed kernels (one warp per chain
                      up to 128 angles, groups of 2 or 4 warps up to 256 and 512) */

typedef struct satpila_pila satpila_pila;

typedef struct {
    int32_t n;                /* image side, >= 1 */
    int32_t n_angles;         /* U, >= 1 */
    int32_t n_bins;           /* B, >= 1 (<= 32767 for PILA_F16 and PILA_U8) */
    const double* angles_rad; /* host, U angles; NULL: theta_u = pi*u/U */
    const uint8_t* mask;      /* host, n*n reconstruction space (Sec. III, Fig. 2(c));
                                 NULL: every pixel.  Moves pick pixels from it and
                                 the SIRT factor matrix sums over it. */
} pila_geom;

typedef struct {
    int32_t n, n_angles, n_bins, precision;
    int32_t n_mask;        /* pixels in the reconstruction space */
    int32_t record_bytes;  /* 16, 8 or 4 */
    int32_t row_records;   /* records stored per pixel (U, or U rounded up to even for F16) */
    int32_t pad;
    int64_t table_bytes;   /* device bytes of the record table */
    int64_t entries;       /* non-empty (bin, length) pairs */
} pila_info_t;

/*
 * Build the PILA (Eq. (5), Sec. II-B): for every pixel and angle, the detector
 * bins whose rays cross the pixel and the exact intersection lengths.  Eq. (5)
 * stores one {k_u, l_u} per angle; a unit pixel can meet two unit-spaced rays
 * of one angle, so each record holds up to two entries on consecutive bins
 * (bin1 = bin0 + 1), sorted by bin.  An empty entry has length 0 and a bin
 * that is safe to index.  Lengths come from the closed-form chord of a unit
 * square (computed in FP64, then rounded to the record's precision); entries
 * shorter than 1e-12 or on bins outside [0, B) are dropped.
 * Layout in device memory: pixel-major, angle-contiguous [n*n][row_records].
 * Also builds the reconstruction-space pixel list and (lazily) the SIRT
 * factor matrix.  Synchronous: returns when the table is built.
 * Errors: INVALID_ARG (sizes, precision, B > 32767 with F16), OOM, CUDA.
 */
int pila_build(const pila_geom* g, int32_t precision, void* stream, satpila_pila** out);
/* Release a PILA built by pila_build (NULL is a no-op). */
int pila_free(satpila_pila* p);
/* Sizes of a built PILA. */
int pila_info(const satpila_pila* p, pila_info_t* info);
/*
 * Copy the table out in a precision-independent form: bins [n*n][U][2]
 * (int32; -1 for an empty entry) and lens [n*n][U][2] (float32, the stored
 * value dequantised).  Host or device outputs.  Synchronous.
 */
int pila_export(const satpila_pila* p, int32_t* bins, float* lens, void* stream);
/*
 * Forward projection through the PILA, i.e. the DRT of Eq. (1) with the
 * stored lengths: sino[i][u][k] = sum over pixels p of images[i][p] * l.
 * Accumulated exactly in 64-bit fixed point (order-independent, hence
 * deterministic) and returned as float64 [n_images][U][B].  images and sino
 * are host or device memory (host buffers make the call synchronous).  For
 * few images the call takes a stream-ordered device workspace (n_images *
 * chunks * U * B * 8 bytes, chunks <= 64) to split their pixels over more
 * CTAs, released on `stream` when the work is done.
 * Errors: INVALID_ARG (null pointers, B above the projector's limit), CUDA.
 */
int pila_forward(const satpila_pila* p, int32_t n_images, const float* images, double* sino, void* stream);
/*
 * SIRT factor matrix of Sec. III-D: w[u][k] = sum over reconstruction-space
 * pixels of l^2 along ray (u, k), as float64 [U][B].
 */
int pila_sirt_factor(const satpila_pila* p, double* w, void* stream);

/* ------------------------------------------------------------------------ */
/* Simulated annealing: Steps 1-4 of Sec. II-A, Eqs. (2)-(4), (6)-(9), BoME.  */
/* ------------------------------------------------------------------------ */

#define SAT_SCHED_LINEAR 0    /* Eq. (2) */
#define SAT_SCHED_GEOMETRIC 1 /* T0 (TN/T0)^(n/N), the second Eq. (8) */
#define SAT_SCHED_CUBIC 2     /* Eq. (9) */

#define SAT_RESIDENT_AUTO 0   /* pick by size (and the autotuner when enabled) */
#define SAT_RESIDENT_SMEM 1   /* residual sinogram in shared memory */
#define SAT_RESIDENT_GLOBAL 2 /* residual sinogram in global memory (L2) */

#define SAT_FLAG_NO_GRAPH 1u  /* launch kernels directly instead of a cached CUDA graph */
#define SAT_FLAG_AUTOTUNE 2u  /* time the launch candidates once per shape and keep the best:
                                 warps per chain (angle tiling), chains per CTA and residency.
                                 With SATPILA_TUNE_CACHE=<file> in the environment the picks are
                                 also read from and appended to that file, so that later processes
                                 use the same layout (sat_stats.plan reports it; pass it back as
                                 sat_params.plan to pin it) */
#define SAT_FLAG_HYBRID 4u    /* with more chains than shared-memory slots, also run chains on
                                 global-memory warps beside them (same arithmetic) */
#define SAT_FLAG_BOME_INDEPENDENT 8u /* BoME as Sec. III-B words it: each estimate is its own random
                                 pixel with its own value (default: bome_k values at one pixel).
                                 Draw 2 + e is estimate e's value, draw 0 (e = 0) or
                                 2 + bome_k + e - 1 (e >= 1) picks its pixel; the trace records
                                 the chosen estimate's pixel.  Residual in global memory. */
#define SAT_FLAG_WINDOW_GROUPS 16u /* with group_warps 2 or 4 (and no autotuning): the windowed
                                 move on that many warps per chain, residual in global memory */
#define SAT_FLAG_NEAR_TIES 64u /* count near-tie decisions per chain (sat_stats.near_ties): one more
                                 reduction per window of moves; windowed layouts only */
#define SAT_FLAG_TEST_STALL 32u /* test hook for the timeout path: the sweep kernel never reports
                                 chain 0's first stage as done, so the task of its next stage waits
                                 until wait_ms runs out, gives up, and the call returns
                                 SATPILA_ERR_TIMEOUT (stats.status too) with the device usable.
                                 Stages are then one task each.  Not for production runs. */

typedef struct {
    int32_t pixel;     /* pixel index i*n + j */
    int32_t cstar;     /* chosen estimate (BoME) */
    int32_t accepted;  /* Step 4 outcome */
    int32_t pad;
    float dS;          /* the Eq. (7) sum (before 1/(B*U)) of the chosen estimate */
    float dC;          /* C' - C of the chosen estimate */
    float fnew;        /* pixel value after the move */
    float pad2;
} sat_trace_rec;

typedef struct {
    float beta;              /* pixel values live in [0, beta] (Eq. (3)); > 0 */
    int32_t bome_k;          /* estimates per move N_e (Sec. III-B), 1..32 */
    int32_t n_sweeps;        /* temperature stages N (each of M moves) */
    int32_t moves_per_sweep; /* M; 0: the number of reconstruction-space pixels */
    double t0;               /* T0; <= 0: estimated per chain by Eq. (8) */
    double tn;               /* T_N; < 0: T0 / 1000 */
    int32_t schedule;        /* SAT_SCHED_* */
    int32_t t0_samples;      /* Q of Eq. (8); 0: 200 */
    uint64_t seed;           /* chain c uses Philox key seed + c */
    int32_t resync_every;    /* FP64 resync of the residual every this many sweeps; 0: only at the end */
    int32_t residency;       /* SAT_RESIDENT_* */
    uint32_t flags;          /* SAT_FLAG_* */
    int32_t trace_chain;     /* chain whose moves are recorded, or -1 */
    int32_t group_warps;     /* warps that share one chain's angles (1, 2, 4); 0: chosen by size */
    int32_t pipeline_depth;  /* PILA rows in flight per chain, 3..8; 0: default (4) */
    sat_trace_rec* trace;    /* n_sweeps*M records for trace_chain (host or device), or NULL */
    double* sweep_cost;      /* [n_chains][n_sweeps] cost after each sweep (host or device), or NULL */
    int32_t plan;            /* SAT_PLAN_* launch layout to use (1..10; INVALID_ARG if it does not fit);
                                0: size rules, or the autotuner with SAT_FLAG_AUTOTUNE */
    int32_t wait_ms;         /* bound on every device-side wait of a chain for its earlier stages
                                (ms); 0: 20000 */
} sat_params;

typedef struct {
    double t0, tn;            /* temperatures used */
    double initial_cost;      /* Eq. (4) of the initial image, FP64 */
    double final_cost;        /* Eq. (4) of the final image, from a fresh FP64 projection */
    double final_cost_incremental; /* the cost carried by Eq. (7) just before the final resync */
    double max_resync_drift;  /* max |incremental residual - fresh residual| over all resyncs */
    int64_t accepted, proposed;
    int32_t t0_found;         /* uphill samples found for Eq. (8) (0 if T0 was given) */
    int32_t status;           /* 0, or a SATPILA_ERR_* raised on the device */
    double sweep_ms;          /* device time of the sweep kernels of this call (same for every chain):
                                 CUDA events on `stream` around each sweep launch (direct launches), or
                                 the device's global timer read just before and after it (graphs) */
    int32_t plan;             /* SAT_PLAN_* layout the launches used (SAT_PLAN_RULES: the
                                 independent-pixel BoME kernel) */
    int32_t near_ties;        /* with SAT_FLAG_NEAR_TIES and a windowed layout: decisions whose
                                 margin (BoME gap, or Step 4's C' - C against T(-ln N1) or 0) was
                                 within 2e-5 of the scale of their FP32 terms; else -1 */
} sat_stats;

/* Launch layouts (sat_stats.plan).  They differ in how chains map onto the
 * GPU, not in the moves: the windowed layouts use the windowed form of the
 * move (exact in-window corrections), the pipelined layouts the per-move
 * form; both follow Eq. (7) to FP32 rounding. */
#define SAT_PLAN_RULES 0         /* input: chosen by size rules (no autotuning) */
#define SAT_PLAN_WINDOW_SMEM 1   /* one warp per chain, residual band in shared memory */
#define SAT_PLAN_WINDOW_GLOBAL 2 /* one warp per chain, residual in global memory */
#define SAT_PLAN_WINDOW_HYBRID 3 /* both kinds of warp in one launch */
#define SAT_PLAN_PIPE_1 4        /* pipelined, 1 warp per chain */
#define SAT_PLAN_PIPE_2 5        /* pipelined, 2 warps per chain */
#define SAT_PLAN_PIPE_4 6        /* pipelined, 4 warps per chain */
#define SAT_PLAN_WINDOW_G2 7     /* windowed, 2 warps per chain, residual in global memory */
#define SAT_PLAN_WINDOW_G4 8     /* windowed, 4 warps per chain, residual in global memory */
#define SAT_PLAN_WINDOW_SMEM_G2 9  /* windowed, 2 warps per chain, residual band in shared memory */
#define SAT_PLAN_WINDOW_SMEM_G4 10 /* windowed, 4 warps per chain, residual band in shared memory */

/*
 * Anneal n_chains independent slices that share one PILA.  Chain c reads its
 * measured sinogram sino_meas[c] ([U][B]) and anneals images[c] ([n][n]) in
 * place from the given initial estimate.  Every move: pick a pixel of the
 * reconstruction space, draw bome_k candidate values (Eq. (3)), evaluate each
 * by Eq. (7) on the residual P_c - P_m, keep the best (BoME), accept by the
 * Metropolis rule of Step 4 at the stage temperature, and on acceptance apply
 * Eq. (6) to the residual.  Each chain is strictly sequential; parallelism is
 * over angles (within a warp), estimates, and chains.
 * Random numbers: Philox4x32-10, key = seed + c, counter (stage, move, block,
 * 1); draw 0 picks the pixel, draw 1 is N1, draw 2 + e is estimate e.
 * stats (host, n_chains entries, may be NULL) are filled before return; the
 * call then synchronizes `stream` at its end.  With stats == NULL, every
 * buffer in device memory and SAT_FLAG_NO_GRAPH clear, the call is
 * asynchronous: it returns once its CUDA graph is enqueued on `stream` (the
 * images are final when the stream reaches that point; a device-side timeout
 * is then not reported - pass stats to see it).
 * Launches: unless SAT_FLAG_NO_GRAPH, a call whose buffers are all device
 * memory is recorded into a CUDA graph (on a private stream) and launched on
 * `stream`; the graph and its workspace are kept (a few entries, least
 * recently used first out, dropped by pila_free) so that repeating the call
 * with the same table, buffers and parameters replays it.  Calls with host
 * buffers launch directly.
 * Errors: INVALID_ARG, OOM, CUDA; TIMEOUT if a bounded device-side wait gave
 * up (also reported per chain in stats.status).
 */
int sat_run(const satpila_pila* p, int32_t n_chains, const float* sino_meas, float* images,
            const sat_params* prm, sat_stats* stats, void* stream);

/*
 * sat_run over chains given one buffer each: sino_meas[c] ([U][B]) and
 * images[c] ([n][n], annealed in place) for c < n_chains, each host or device
 * memory independently (the arrays of pointers are host memory).  The chains
 * are copied into one contiguous device batch on `stream`, annealed exactly as
 * sat_run anneals that batch (same results, bit for bit), and the images copied
 * back on `stream`.  The batch is allocated stream-ordered and freed after the
 * copies back.  With stats (host, n_chains entries) the call synchronizes
 * `stream` before it returns; without, and with device buffers only, it returns
 * once the work is enqueued.  The caller owns every buffer.
 * Errors: INVALID_ARG (a null pointer), OOM, CUDA; otherwise sat_run's.
 */
int sat_run_ptrs(const satpila_pila* p, int32_t n_chains, const float* const* sino_meas, float* const* images,
                 const sat_params* prm, sat_stats* stats, void* stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of annealing requests (no counterpart in the  */
/* paper, which reconstructs one slice at a time; each request runs Steps 1-4 */
/* of Sec. II-A exactly as sat_run does for one chain).                       */
/* ------------------------------------------------------------------------ */

typedef struct satpila_server satpila_server;

typedef struct {
    int32_t device;          /* CUDA device the server runs on */
    int32_t max_active;      /* chains on the device at once; 0: 4096 */
    int32_t stages_per_tick; /* stages every active chain advances per batched launch; each tick ends
                                with the FP64-grade resync, so a request behaves as sat_run with
                                resync_every = stages_per_tick; 0: 5 */
    int32_t queue_limit;     /* waiting requests beyond which submit returns SATPILA_ERR_BUSY; 0: 65536 */
    uint64_t mem_budget;     /* device bytes for tables and chain state; 0: 120 GB (1.2e11 bytes); capped at the
                                device's free memory less 2 GiB */
    uint32_t flags;          /* SAT_SERVER_* */
} sat_server_cfg;

/* sat_server_cfg.flags: every class ticks on its own stream with its own
 * launches (the layout sat_run's size rules pick), instead of sharing its
 * image size's launches. */
#define SAT_SERVER_PER_CLASS 1u

typedef struct {
    int32_t n, n_angles, n_bins; /* geometry, as pila_geom */
    int32_t precision;           /* PILA_F32, PILA_F16 or PILA_U8 */
    const double* angles_rad;    /* [n_angles] or NULL (u * pi / U) */
    const uint8_t* mask;         /* [n][n] reconstruction space or NULL (all pixels) */
    const float* sino;           /* [n_angles][n_bins] measured sinogram P_m */
    const float* image;          /* [n][n] start image, or NULL: 0.5 on the reconstruction space, 0 elsewhere */
    sat_params prm;              /* as for sat_run; prm.seed is this chain's Philox key; trace,
                                    sweep_cost, resync_every and flags are not used */
} sat_request;

typedef struct {
    sat_stats stats;             /* as sat_run's (sweep_ms: the chain's last tick) */
    double submit_ms, admit_ms, done_ms; /* server clock, ms since sat_server_create */
} sat_result;

typedef struct {
    int64_t submitted, admitted, completed, failed;
    int32_t active, queued, geometries, classes;
    uint64_t bytes_in_use, bytes_peak, mem_budget;
    int64_t ticks, moves;
} sat_server_stats;

/*
 * Start a server: one engine thread that owns the device work.  Requests
 * sharing geometry, bome_k, beta and moves per stage form a class, whose
 * chains live in the class's arrays, each at its own stage of its own
 * schedule.  The classes of one image size and table precision share one
 * persistent sweep launch per window of stages_per_tick stages (the windowed
 * kernel on groups of 4 warps, every chain reading its own class's table and
 * geometry; for tables of at most 512 angles and bome_k <= 8 without a
 * requested layout), followed by each class's resync; other classes, and all
 * of them with SAT_SERVER_PER_CLASS, run their own launches on their own
 * streams.  Between ticks finished chains are copied out and waiting
 * requests are admitted, in arrival order, while chain slots and the memory
 * budget allow (PILA tables are cached per geometry and unused ones dropped
 * when memory is needed).  A chain's result is the same alone and in any mix:
 * sat_run on that chain with resync_every = stages_per_tick and
 * plan = SAT_PLAN_WINDOW_G4 for a request of a shared launch (the size rules'
 * layout with SAT_SERVER_PER_CLASS or for other requests).
 * Errors: INVALID_ARG (no such device), OOM.
 */
int sat_server_create(const sat_server_cfg* cfg, satpila_server** out);

/* Queue one request; its buffers (host or device) are copied before return.
 * Errors: BUSY (queue full), INVALID_ARG (bad request, or one that can never
 * fit the budget), or the error that stopped the server. */
int sat_server_submit(satpila_server* s, const sat_request* r, uint64_t* ticket);

/* Collect a finished request: image_out ([n][n], host or device, may be NULL)
 * and res (may be NULL).  PENDING while it is queued or running; NOT_FOUND for
 * an unknown or already collected ticket; a device-side error code if the
 * request failed. */
int sat_server_poll(satpila_server* s, uint64_t ticket, float* image_out, sat_result* res);

/* As sat_server_poll, waiting up to timeout_ms (< 0: no limit); PENDING on
 * timeout. */
int sat_server_wait(satpila_server* s, uint64_t ticket, int32_t timeout_ms, float* image_out, sat_result* res);

/* Counters of the server. */
int sat_server_info(satpila_server* s, sat_server_stats* out);

/* Stop after the current tick, free every device buffer and table; results
 * not collected are lost. */
int sat_server_destroy(satpila_server* s);

/* ------------------------------------------------------------------------ */
/* The conventional SAT that the PILA replaces (Sec. III-A, Fig. 3): a full   */
/* DRT by bilinear interpolation for every estimate.  A speed baseline.       */
/* ------------------------------------------------------------------------ */

/*
 * Bilinear-interpolation DRT of n_items images ([n][n] each, device memory)
 * into sino ([n_items][n_angles][n_bins], device memory).  Ray (u, k) is the
 * line x cos + y sin = s_k, sampled at n_bins unit steps
 * t_m = m - (n_bins - 1)/2 along (-sin, cos); each sample interpolates
 * bilinearly between pixel centres (zero outside); angles_rad (host, may be
 * NULL: u pi / n_angles).  Synchronizes `stream`.  Errors: INVALID_ARG, CUDA.
 */
int drt_bilinear(int32_t n, int32_t n_angles, int32_t n_bins, const double* angles_rad, int32_t n_items,
                 const float* images, float* sino, void* stream);

/*
 * SAT without the PILA: Steps 1-4 with the random stream of sat_run (key
 * seed + c, draw 0 the pixel of the mask list (host mask, NULL: all pixels),
 * draw 1 N1, draw 2 + e estimate e), each estimate evaluated by a full
 * bilinear DRT of the candidate image and Eq. (4), the best kept, Step 4 with
 * the exponential.  One CTA per chain.  sino_meas [n_chains][U][B] and images
 * [n_chains][n][n] are device memory (images annealed in place); prm->t0 must
 * be > 0 (no Eq. (8)); resync, residency, flags, group_warps and
 * pipeline_depth are ignored; trace (device) records trace_chain's moves
 * with dS = S' - S.  stats: final_cost, accepted, proposed, sweep_ms (the
 * kernel's time).  Synchronizes `stream`.
 */
int sat_drt_run(int32_t n, int32_t n_angles, int32_t n_bins, const uint8_t* mask, int32_t n_chains,
                const float* sino_meas, float* images, const sat_params* prm, sat_stats* stats, void* stream);

/* ------------------------------------------------------------------------ */
/* FBP prior (Step 1, Step 2, Fig. 9): start image, beta and spatial          */
/* constraint from a filtered back-projection.                                */
/* ------------------------------------------------------------------------ */

/*
 * Parallel-beam FBP of n_items sinograms ([n_items][n_angles][n_bins], device)
 * into images ([n_items][n][n], device).  The paper gives no filter; this uses
 * the discrete Ram-Lak filter for unit bins (h(0) = 1/4, h(k) = -1/(pi^2 k^2)
 * for odd k, 0 otherwise) and linear interpolation between bin centres in the
 * back-projection f(x, y) = (pi / U) sum_u q_u(x cos + y sin).  angles_rad
 * (host) may be NULL (u pi / U).  Synchronizes `stream`.
 */
int fbp(int32_t n, int32_t n_angles, int32_t n_bins, const double* angles_rad, int32_t n_items,
        const float* sino, float* images, void* stream);

/*
 * From FBP images ([n_items][n][n], device): beta[i] = max(0, max image i)
 * (the pixel range of Eq. (3), Step 2), mask = pixels above mask_frac * beta
 * (the spatial constraint, by a threshold filter), init = the image clipped to
 * [0, beta] on the mask and 0 elsewhere (the start image of Step 1).  Each
 * output (device) may be NULL.  Synchronizes `stream`.
 */
int fbp_prior(int32_t n, int32_t n_items, const float* images, float mask_frac, float* init, uint8_t* mask,
              float* beta, void* stream);

/* ------------------------------------------------------------------------ */
/* SIRT with PILA: Eqs. (10)-(11), Sec. III-D.                                */
/* ------------------------------------------------------------------------ */

#define SIRT_SIMULTANEOUS 0 /* all pixels from the same P_c (classic SIRT) */
#define SIRT_SEQUENTIAL 1   /* pixel by pixel in raster order over the reconstruction
                               space, each update written into P_c through the PILA */

typedef struct {
    int32_t n_iter; /* passes N over the reconstruction space */
    int32_t mode;   /* SIRT_* */
    float relax;    /* multiplies the Eq. (10) increment; 1 reproduces the paper */
    int32_t pad;
} sirt_params;

/*
 * n_slices independent SIRT reconstructions sharing the PILA.  costs (host or
 * device, [n_slices][n_iter], may be NULL) receives Eq. (4) after each pass.
 * Allocates its device scratch (corrections, partial sums, and for few slices
 * the projector's pixel-chunk slices) for the call.  Synchronizes `stream` at
 * its end.
 */
int sirt_run(const satpila_pila* p, int32_t n_slices, const float* sino_meas, float* images,
             const sirt_params* prm, double* costs, void* stream);

/* Size of the static device scratch that sirt_run_noalloc works in. */
#define SATPILA_NOALLOC_SCRATCH_BYTES (8u << 20)

/*
 * sirt_run without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * during the call, for instance processes confined to a memory budget fixed
 * at start-up, hosts whose own allocator has reserved the device's memory,
 * or real-time loops that cannot afford the device-wide synchronisation a
 * cudaMalloc/cudaFree pair may cause.  Instead of allocating scratch,
 * it works in one statically sized array of this library
 * (SATPILA_NOALLOC_SCRATCH_BYTES; every GPU that loads the library keeps it
 * until the process exits).  Same arguments and results as sirt_run, except:
 *  - sino_meas, images and costs must be device pointers (nothing is staged);
 *  - the call is asynchronous on `stream` and does not synchronize it;
 *  - a problem whose scratch (n_slices * U * B floats, partial sums, and the
 *    factor matrix when the PILA has not cached one) exceeds the array is
 *    rejected with SATPILA_ERR_INVALID_ARG; the projector's pixel-chunk
 *    slices are used only when they fit beside it (results are the same
 *    either way);
 *  - the first call on a device looks up the array's device address once,
 *    so make that first call before any stream capture begins;
 *  - all calls share the array: calls whose work overlaps on the GPU (other
 *    streams, other host threads) race and must be serialised by the caller.
 */
int sirt_run_noalloc(const satpila_pila* p, int32_t n_slices, const float* sino_meas, float* images,
                     const sirt_params* prm, double* costs, void* stream);

/* ------------------------------------------------------------------------ */
/* Memory-level probes.  No counterpart in the paper: they measure, on the    */
/* running GPU, the read rates that bound the move's gathers (its roofline):  */
/* the PILA row is read as consecutive 16-byte chunks, the residual cells as  */
/* one 32-byte sector per record at scattered places.                         */
/* ------------------------------------------------------------------------ */

#define SATPILA_PROBE_STREAM 0 /* consecutive 16-byte loads, whole lines per warp */
#define SATPILA_PROBE_SECTOR 1 /* one 32-byte sector at a pseudo-random place per load */

/*
 * Read rate over buf (device memory, 16-byte aligned, bytes >= 4096): about
 * `loads` loads of the given kind from every SM, bypassing L1, timed with
 * CUDA events on `stream` after one untimed pass.  A buffer that fits in L2
 * measures L2; one many times larger than L2 measures HBM.  For
 * SATPILA_PROBE_SECTOR each warp gathers inside one region of region_bytes
 * (warp w in region w mod (bytes / region_bytes); 0: the whole buffer, at
 * most 2^32 sectors), as a chain's warps gather inside its own residual.
 * *gbs = bytes / s / 1e9, counting 32 bytes per sector load (the unit the
 * memory moves) and 16 per stream load.  buf is only read.  Synchronizes
 * `stream`.  Errors: INVALID_ARG (host pointer, sizes, kind), CUDA.
 */
int satpila_probe_read(const void* buf, uint64_t bytes, int32_t kind, uint64_t region_bytes, uint64_t loads,
                       double* gbs, void* stream);
/*
 * Shared-memory 4-byte load rate summed over all SMs (about `loads` loads):
 * kind 0 conflict-free (lane i reads bank i), kind 1 pseudo-random words of a
 * 32 KB array per CTA (the pattern of residual cells at scattered bins).
 * *gbs = 4 * loads / s / 1e9.  Synchronizes `stream`.
 */
int satpila_probe_smem(int32_t kind, uint64_t loads, double* gbs, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SATPILA_H */
