/*
 * Reference oracle for simulated annealing tomography with a pre-calculated
 * intersection-lengths array (Vo, Breese & Moser, "Feasibility of Simulated
 * Annealing Tomography").
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64 CPU
 * restatement of the method, written so that it can be checked against the
 * paper by eye.  Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or helper with
 * the CUDA library, and the CUDA library never calls it.
 *
 * Geometry (parallel beam, unit pixels as in Sec. II-B):
 *   pixel (i, j) of an n x n image (row i from the top, column j) has its
 *   centre at x = j - (n-1)/2, y = (n-1)/2 - i; the image covers the square
 *   [-n/2, n/2]^2.  Angle u is theta_u (default pi*u/U).  Ray (u, k) is the
 *   line x*cos(theta_u) + y*sin(theta_u) = s_k with s_k = k - (B-1)/2.
 *   A ray lying exactly on a pixel edge (only possible at 0 and 90 degrees)
 *   is counted for the pixel on its +s side.
 */
#ifndef SATPILA_ORACLE_H
#define SATPILA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n;              /* image side */
    int32_t n_angles;       /* U */
    int32_t n_bins;         /* B */
    const double* angles;   /* U angles in radians, or NULL for pi*u/U */
} or_geom;

/* Philox4x32 with 10 rounds (Salmon et al., SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Siddon traversal of ray (theta, s) through the n x n grid: pixel indices
 * (i*n + j) and chord lengths in traversal order; returns the count (<= cap)
 * or -1 if cap is too small.  Chords shorter than 1e-12 are dropped. */
int or_siddon_ray(int32_t n, double theta, double s, int32_t* pix, double* len, int32_t cap);

/* Discrete Radon transform, Eq. (1): sino[u*B + k] = sum over pixels crossed
 * by ray (u, k) of image[p] * l.  Ray-driven, by Siddon traversal. */
int or_drt(const or_geom* g, const double* image, double* sino);

/* The conventional forward model of Sec. III-A: a DRT by bilinear
 * interpolation, each ray sampled at B unit steps t_m = m - (B-1)/2 along its
 * direction (see drt_bilinear.cpp). */
int or_drt_bilinear(const or_geom* g, const double* image, double* sino);

/* PILA, Eq. (5), built by transposing the Siddon traversals of every ray.
 * Up to two entries per (pixel, angle), sorted by bin:
 *   bins[(p*U + u)*2 + s], lens[(p*U + u)*2 + s]; an empty slot has len 0
 *   and bin -1.  Returns 0, or -1 if a (pixel, angle) met more than 2 rays. */
int or_pila(const or_geom* g, int32_t* bins, double* lens);

/* Eq. (4): C = sqrt(1/(B*U) * sum (pc - pm)^2). */
double or_cost(int32_t n_angles, int32_t n_bins, const double* pc, const double* pm);

/* SIRT factor matrix of Sec. III-D: w[u*B + k] = sum over mask pixels of l^2
 * along ray (u, k), by Siddon traversal.  mask may be NULL (all pixels). */
int or_sirt_factor(const or_geom* g, const uint8_t* mask, double* w);

enum { OR_SCHED_LINEAR = 0, OR_SCHED_GEOMETRIC = 1, OR_SCHED_CUBIC = 2 };

typedef struct {
    double beta;            /* pixel values live in [0, beta], Eq. (3) */
    int32_t bome_k;         /* number of estimates N_e (Sec. III-B) */
    int32_t n_sweeps;       /* temperature stages */
    int32_t moves_per_sweep;/* M; 0 means the number of mask pixels */
    double t0;              /* initial temperature; <= 0: estimate by Eq. (8) */
    double tn;              /* final temperature; < 0: t0 / 1000 */
    int32_t schedule;       /* OR_SCHED_* */
    int32_t t0_samples;     /* Q of Eq. (8); 0 means 200 */
    uint64_t seed;          /* this chain's Philox key */
    int32_t bome_mode;      /* OR_BOME_SAME_PIXEL or OR_BOME_INDEPENDENT */
    int32_t grid_levels;    /* 0: Eq. (3); L >= 2: an estimate is level floor(u L) of the grid
                               {0, beta/(L-1), ..., beta} (for the exhaustive-search check) */
    int32_t length_format;  /* OR_LEN_*: how the PILA stores its lengths (Sec. II-B); with a
                               rounded format the initial and final projections are sums over
                               the rounded table, so the whole run sees one set of lengths */
} or_sat_params;

/* Stored PILA lengths (Sec. II-B keeps them in reduced precision): exact FP64;
 * IEEE binary16 (round to nearest, ties to even; 11 significant bits,
 * subnormal quantum 2^-24); one byte, round(180 l) / 180 (ties to even). */
enum { OR_LEN_EXACT = 0, OR_LEN_BINARY16 = 1, OR_LEN_BYTE180 = 2 };

/* A length l >= 0 as the given format stores it. */
double or_round_length(int32_t format, double l);

/* Exhaustive search over every image whose pixels take the L grid values
 * {0, beta/(L-1), ..., beta} (n*n <= 16, L^(n*n) <= 2^26 images): the least
 * Eq. (4) cost against pm, how many images attain it (within 1e-9 of the
 * least sum of squares, relative to max(1, sum P_m^2)), and the first such
 * image.  The sinogram is updated along a reflected Gray order (one pixel,
 * one level per step) through the PILA. */
int or_exhaustive_grid(const or_geom* g, const double* pm, int32_t levels, double beta, double* min_cost,
                       int64_t* n_min, double* argmin_image);

/* Sec. III-B: every estimate at the move's one pixel, or (the paper's own
 * wording) each estimate at its own randomly chosen pixel. */
enum { OR_BOME_SAME_PIXEL = 0, OR_BOME_INDEPENDENT = 1 };

typedef struct {
    double t0, tn;
    double initial_cost, final_cost;   /* Eq. (4) values carried by Eq. (7) */
    double final_cost_fresh;           /* Eq. (4) recomputed from scratch */
    int64_t accepted, proposed;
    int32_t t0_found;                  /* uphill samples found for Eq. (8) */
} or_sat_stats;

typedef struct {
    int32_t pixel, cstar, accepted, pad;
    double dS;        /* sum in Eq. (7) of the chosen estimate, before 1/(B*U) */
    double dC;        /* C' - C of the chosen estimate */
    double fnew;      /* pixel value after the move */
    double u_acc;     /* acceptance uniform N1 */
    double temp;      /* T_n */
    double scale_S;   /* 2*|df|*sum|r*l| + df^2*sum l^2 : magnitude of dS terms */
    double gap_S;     /* dS gap between best and second-best estimate */
} or_trace_rec;

/* Sample-average temperature rule Eq. (8) from the given image. */
int or_sat_t0(const or_geom* g, const uint8_t* mask, const double* pm, const double* image,
              const or_sat_params* prm, double* t0_out, int32_t* found_out);

/* Temperature of stage s out of n_sweeps: Eq. (2), (8) (second form), (9). */
double or_schedule_temp(int32_t schedule, double t0, double tn, int32_t s, int32_t n_sweeps);

/* Steps 1-4 of Sec. II-A with PILA updates, Eqs. (6)-(7), and BoME.
 * image is n*n, updated in place.  trace (may be NULL) receives
 * n_sweeps*moves records.  Returns 0 or a negative error. */
int or_sat_run(const or_geom* g, const uint8_t* mask, const double* pm, double* image,
               const or_sat_params* prm, or_sat_stats* stats, or_trace_rec* trace);

/* SAT without the PILA (Sec. III-A's baseline): every estimate evaluated by a
 * full bilinear DRT of the candidate image; same random stream as or_sat_run;
 * prm->t0 must be given (> 0). */
int or_sat_drt_run(const or_geom* g, const uint8_t* mask, const double* pm, double* image,
                   const or_sat_params* prm, or_sat_stats* stats, or_trace_rec* trace);

typedef struct {
    int32_t pixel, cstar, accepted, pad;
    float dS, dC, fnew, pad2;
} or_gpu_trace;

typedef struct {
    int64_t moves;
    int64_t near_ties;          /* decisions that differed at a recorded near-tie */
    int64_t pixel_mismatch;     /* first move where the pixel differed, or -1 */
    int64_t hard_mismatch;      /* first decision mismatch outside a near-tie, or -1 */
    double max_err_dS;          /* max |dS_gpu - dS_oracle| / scale_S */
    double max_err_dC;          /* max |dC_gpu - dC_oracle| / scale_C */
    double max_err_f;           /* max |fnew_gpu - fnew_oracle| */
} or_lockstep_report;

/* Follow another implementation's move trace: recompute every move in FP64,
 * compare, and where decisions differ at a near-tie, take the other side's
 * decision.  tol is the relative tolerance used for near-tie detection. */
int or_sat_lockstep(const or_geom* g, const uint8_t* mask, const double* pm, double* image,
                    const or_sat_params* prm, double t0, double tn,
                    const or_gpu_trace* trace, int64_t n_moves, double tol,
                    or_lockstep_report* rep);

enum { OR_SIRT_SIMULTANEOUS = 0, OR_SIRT_SEQUENTIAL = 1 };

/* SIRT with PILA, Eqs. (10)-(11); costs[it] receives Eq. (4) after each
 * iteration (may be NULL). */
int or_sirt_run(const or_geom* g, const uint8_t* mask, const double* pm, double* image,
                int32_t n_iter, int32_t mode, double relax, double* costs);

#ifdef __cplusplus
}
#endif
#endif
