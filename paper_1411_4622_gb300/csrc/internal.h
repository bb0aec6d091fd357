// Host-side internals of libsatpila shared between translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "satpila.h"

struct satpila_pila {
    int device = 0;
    int n = 0, U = 0, B = 0, precision = PILA_F32;
    int record_bytes = 16;
    int row_records = 0;      // records per pixel row
    int64_t row_bytes = 0;    // row_records * record_bytes (multiple of 16)
    int64_t table_bytes = 0;
    int64_t entries = 0;
    int n_mask = 0;
    unsigned char* d_table = nullptr;  // [P][row_records] records
    int32_t* d_list = nullptr;         // reconstruction-space pixels, raster order
    uint8_t* d_mask = nullptr;         // [P]
    double* d_cos = nullptr;           // [U]
    double* d_sin = nullptr;           // [U]
    double* d_w64 = nullptr;           // SIRT factor matrix [U][B], built on first use
    float* d_w32 = nullptr;
    float* d_hsum = nullptr;           // [P] sum of squared stored lengths of each pixel
    // Residual band: every cell an annealing move can touch (bins k and k + 1
    // of each record of a reconstruction-space pixel) has band_lo <= bin <= band_hi.
    int band_lo = 0, band_hi = 0;
    // Ray-major index of the table, read by the ray-driven projector: the
    // entries of ray (u, k) are d_ray_ent[d_ray_off[u*B + k] .. d_ray_off[u*B + k + 1]),
    // each {pixel, the stored length l as (significand of l with its hidden
    // bit) << 7 | biased exponent of l}, ascending pixel (rays longer than the
    // sort's capacity keep their build order).  NULL when not built (the
    // pixel-driven projector is used instead).
    uint32_t* d_ray_off = nullptr;  // [U*B + 1]
    uint2* d_ray_ent = nullptr;     // [entries]
    int64_t ray_bytes = 0;
    // Tables built for the serving engine come from a stream-ordered memory
    // pool (no device-wide synchronisation on allocation or release).
    cudaMemPool_t pool = nullptr;
    cudaStream_t alloc_stream = nullptr;
};

namespace satpila {

// pila_build with its allocations taken from `pool` in the order of stream s
// (pool == NULL: ordinary allocations, as pila_build); ray_index: also build
// the ray-major index of the ray-driven projector.
int pila_build_in(const pila_geom* g, int32_t precision, cudaStream_t s, cudaMemPool_t pool, satpila_pila** out,
                  bool ray_index = true);

// Thread-local last-error message.
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define SP_CUDA(call)                                         \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ::satpila::cuda_fail(e_, #call); \
    } while (0)

// True if p is a device (or managed) pointer usable by kernels.
bool is_device_pointer(const void* p);

// ---- projector (fixed-point forward projection through the PILA) ----------

enum ProjMode { PROJ_FORWARD = 0, PROJ_RESYNC = 1, PROJ_FACTOR = 2, PROJ_SIRT = 3 };

struct ProjArgs {
    const unsigned char* table;
    int f16;                    // table precision (PILA_F32, PILA_F16, PILA_U8)
    int row_records;
    int n, U, B;
    int angles_per_group, n_groups;  // set by launch_projector from the plan
    int lanes_log2;             // log2 of the angles per group (set with the plan)
    int mode;
    int drift;                  // RESYNC: compare with the residual being replaced
    const float* img;           // FORWARD/RESYNC/SIRT images
    long long img_stride;
    const uint8_t* mask;        // FACTOR pixel weights
    double* out64;              // FORWARD [item][U][B]; FACTOR [U][B]
    long long out_stride;
    float* out32;               // FACTOR: float copy [U][B]
    const float* pm;            // RESYNC/SIRT measured sinograms
    long long pm_stride;
    float* resid;               // RESYNC: residual P_c - P_m; SIRT: correction
    long long resid_stride;
    int resid_pitch;            // row pitch of resid (B when 0)
    int resid_il;               // RESYNC: 0, or resid rows (u, u + resid_il) stored in interleaved pairs (resid_row_base)
    const float* w;             // SIRT: factor matrix (float)
    double* part_sq;            // [item][U] per-angle sums of (P_c - P_m)^2
    float* part_drift;          // [item][U]
    void* ws;                   // optional, projector_ws_bytes(items, U, B, n) bytes: lets few
                                // images split their pixels over more CTAs
    const uint32_t* ray_off;    // ray-major index of the table (satpila_pila::d_ray_off), or NULL
    const uint2* ray_ent;
    void* ray_ws;               // ray_ws_bytes(items, U, B, n) bytes: with the index, selects the
                                // ray-driven projector (else the pixel-driven one runs)
    float* timg;                // carved from ray_ws: images transposed to [group][P][32]
    int* neg_group;             // carved from ray_ws: 1 for a group of 32 images holding a negative value
    int chunks;                 // set with the plan
    long long* partial;         // carved from ws when chunks > 1: [item][chunk][U][B] sums
    float* max_parts;           // [item][32] partial max|f|
};

int projector_smem_bytes(int angles_per_group, int B);
// Angle groups of 2^l <= 16 angles for n_items n x n images; when they give
// too few CTAs, pixel chunks (can_chunk: a workspace is given) or else
// narrower groups.
int projector_plan(int U, int B, int n, long long n_items, bool can_chunk, int* angles_per_group, int* n_groups,
                   int* lanes_log2, int* chunks);
// Workspace that lets launch_projector split the pixels of n_items n x n
// images into chunks (0 when it would not).
size_t projector_ws_bytes(long long n_items, int U, int B, int n);
// Workspace of the ray-driven projector for n_items n x n images.
size_t ray_ws_bytes(long long n_items, int U, int B, int n);
// True when SATPILA_PROJECTOR=pixel asks for the pixel-driven projector.
bool projector_forced_pixel();
// Fills the ray-driven projector's fields of a from p (index) and ws.
void use_ray_projector(ProjArgs& a, const satpila_pila* p, void* ws);
// Builds p's ray-major index on stream s (allocations from pool when given).
int build_ray_index(satpila_pila* p, cudaStream_t s, cudaMemPool_t pool);
// Chooses the plan for n_items (filling a's group fields) and launches.
cudaError_t launch_projector(ProjArgs& a, int n_items, cudaStream_t s);
// The largest B the projector takes (one angle per group in shared memory).
int projector_max_bins();

// Sums the per-group partials of a RESYNC/SIRT projection in a fixed order.
struct ReduceArgs {
    int n_items, n_rows;        // n_rows = U: the per-angle partials of each item
    const double* part_sq;
    const float* part_drift;    // may be NULL
    double inv_cells;           // 1 / (B*U)
    double* S_out;              // per item sum of squares (may be NULL)
    double* cost_out;           // per item Eq. (4) cost (may be NULL)
    long long cost_stride;
    double* drift_max;          // per item running max (may be NULL)
};
cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t s);
// Sets the projector's launch attributes on the current device; call before
// capturing launches of it into a graph.
cudaError_t prepare_projector();

// Builds the SIRT factor matrix of a PILA on first use.
int ensure_factor(satpila_pila* p, cudaStream_t s);

}  // namespace satpila
