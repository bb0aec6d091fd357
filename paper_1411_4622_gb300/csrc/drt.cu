// The conventional SAT of Sec. III-A, which the PILA replaces: every
// estimate is evaluated by a full DRT of the candidate image computed by
// bilinear interpolation.  Kept as the baseline for the paper's speed
// comparison (Fig. 3), not as a reconstruction path.
//
// DRT: ray (u, k) is the line x cos(theta_u) + y sin(theta_u) = s_k, sampled
// at B unit steps t_m = m - (B - 1)/2 along (-sin, cos); a sample is the
// bilinear interpolation between pixel centres (zero outside the grid); the
// projection is the sum of the samples.
//
// sat_drt_run: one CTA per chain.  Per move thread 0 draws the pixel, N1 and
// the estimates (the same Philox stream as sat_run); for each estimate the
// CTA writes the candidate value into the chain's image, every thread sums
// (P - P_m)^2 over its rays, a block reduction gives C', the value is
// restored; thread 0 keeps the best estimate and decides by Step 4.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace satpila {
namespace {

constexpr int kDrtThreads = 512;

__device__ __forceinline__ float px(const float* img, int n, int i, int j) {
    return (i >= 0 && j >= 0 && i < n && j < n) ? img[i * n + j] : 0.0f;
}

// One ray of the bilinear DRT of img.
__device__ __forceinline__ float ray_sum(const float* img, int n, int B, float c, float s, float sk) {
    const float half_n = 0.5f * (float)(n - 1), half_b = 0.5f * (float)(B - 1);
    float acc = 0.0f;
    for (int m = 0; m < B; ++m) {
        const float t = (float)m - half_b;
        const float x = sk * c - t * s, y = sk * s + t * c;
        const float cj = x + half_n, ri = half_n - y;
        const float j0 = floorf(cj), i0 = floorf(ri);
        const float a = cj - j0, b = ri - i0;
        const int j = (int)j0, i = (int)i0;
        const float top = fmaf(a, px(img, n, i, j + 1) - px(img, n, i, j), px(img, n, i, j));
        const float bot = fmaf(a, px(img, n, i + 1, j + 1) - px(img, n, i + 1, j), px(img, n, i + 1, j));
        acc += fmaf(b, bot - top, top);
    }
    return acc;
}

__global__ void drt_bilinear_kernel(const float* img, long long n_items, int n, int U, int B, const double* cs,
                                    const double* sn, float* out) {
    const long long rays = (long long)U * B;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_items * rays) return;
    const long long item = idx / rays;
    const int r = (int)(idx % rays), u = r / B, k = r % B;
    out[idx] = ray_sum(img + item * (long long)n * n, n, B, (float)cs[u], (float)sn[u], (float)k - 0.5f * (float)(B - 1));
}

struct DrtArgs {
    int n, U, B;
    const double* cs;
    const double* sn;
    const int32_t* list;
    int n_list;
    int moves, n_sweeps, K, schedule;
    float beta;
    double t0, tn;
    unsigned long long seed;
    const float* sino;  // [chains][U][B]
    float* img;         // [chains][n][n]
    double* S;          // [chains] sum of squared residuals
    unsigned long long* accepted;
    sat_trace_rec* trace;
    int trace_chain;
    long long trace_cap;
};

// Sum over the CTA of v (FP64), returned to every thread.
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];  // fixed order
    return t;
}

__device__ double chain_S(const DrtArgs& a, const float* img, const float* pm, double* red) {
    const int rays = a.U * a.B;
    float acc = 0.0f;
    for (int r = threadIdx.x; r < rays; r += blockDim.x) {
        const int u = r / a.B, k = r % a.B;
        const float d = ray_sum(img, a.n, a.B, (float)a.cs[u], (float)a.sn[u], (float)k - 0.5f * (float)(a.B - 1)) - pm[r];
        acc = fmaf(d, d, acc);
    }
    return block_sum((double)acc, red);
}

__global__ void __launch_bounds__(kDrtThreads) sat_drt_kernel(const DrtArgs a) {
    __shared__ double red[kDrtThreads / 32];
    __shared__ int s_p;
    __shared__ float s_f, s_vals[kMaxK], s_n1;
    __shared__ float s_best_f;
    __shared__ int s_accept;
    const int c = blockIdx.x;
    float* img = a.img + (long long)c * a.n * a.n;
    const float* pm = a.sino + (long long)c * a.U * a.B;
    const uint2 key = chain_key(a.seed + (unsigned long long)c);
    const double cells = (double)a.U * a.B;
    double S = chain_S(a, img, pm, red);
    unsigned long long n_acc = 0;
    const double TN = a.tn < 0.0 ? a.t0 / 1000.0 : a.tn;
    const int nblk = (a.K + 2 + 3) / 4;
    for (int st = 0; st < a.n_sweeps && a.n_list > 0; ++st) {
        const double N = (double)a.n_sweeps, sd = (double)st;
        const double T = a.schedule == SAT_SCHED_GEOMETRIC ? a.t0 * pow(TN / a.t0, sd / N)
                         : a.schedule == SAT_SCHED_CUBIC   ? a.t0 - sd * sd * sd * (a.t0 - TN) / (N * N * N)
                                                           : a.t0 - sd * (a.t0 - TN) / N;
        for (int m = 0; m < a.moves; ++m) {
            if (threadIdx.x == 0) {
                for (int b = 0; b < nblk; ++b) {
                    const uint4 x = philox4x32_10(make_uint4((uint32_t)st, (uint32_t)m, (uint32_t)b, kStreamSat), key);
                    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
                    for (int q = 0; q < 4; ++q) {
                        const int d = 4 * b + q;
                        if (d == 0) s_p = a.list ? a.list[pick_index(w[q], (uint32_t)a.n_list)] : (int)pick_index(w[q], (uint32_t)a.n_list);
                        else if (d == 1) s_n1 = unit_uniform(w[q]);
                        else if (d - 2 < a.K) s_vals[d - 2] = unit_uniform(w[q]);
                    }
                }
                s_f = img[s_p];
            }
            __syncthreads();
            const int p = s_p;
            const float f = s_f;
            const float lo = fmaxf(0.0f, f - a.beta), span = fminf(a.beta, f + a.beta) - lo;
            double best_S = INFINITY;
            int best = 0;
            for (int e = 0; e < a.K; ++e) {
                const float fc = fmaf(s_vals[e], span, lo);
                if (threadIdx.x == 0) img[p] = fc;
                __syncthreads();
                const double Sc = chain_S(a, img, pm, red);  // the full DRT of the candidate image
                if (Sc < best_S) {
                    best_S = Sc;
                    best = e;
                }
                __syncthreads();
                if (threadIdx.x == 0) img[p] = f;
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                const double C = sqrt(S / cells), Cp = sqrt(best_S / cells);
                const double dC = Cp - C;
                const bool accept = dC <= 0.0 || (T > 0.0 && (double)s_n1 < exp(-dC / T));
                const float fb = fmaf(s_vals[best], span, lo);
                s_accept = accept ? 1 : 0;
                s_best_f = fb;
                if (a.trace && c == a.trace_chain) {
                    const long long idx = (long long)st * a.moves + m;
                    if (idx < a.trace_cap) {
                        sat_trace_rec rr;
                        rr.pixel = p;
                        rr.cstar = best;
                        rr.accepted = accept ? 1 : 0;
                        rr.pad = 0;
                        rr.dS = (float)(best_S - S);
                        rr.dC = (float)dC;
                        rr.fnew = accept ? fb : f;
                        rr.pad2 = 0.0f;
                        a.trace[idx] = rr;
                    }
                }
                if (accept) img[p] = fb;
            }
            __syncthreads();
            if (s_accept) {
                S = best_S;
                ++n_acc;
            }
        }
    }
    if (threadIdx.x == 0) {
        a.S[c] = S;
        a.accepted[c] = n_acc;
    }
}

void angle_tables(int U, const double* angles, std::vector<double>& cs, std::vector<double>& sn) {
    cs.resize(U);
    sn.resize(U);
    for (int u = 0; u < U; ++u) {
        const double th = angles ? angles[u] : M_PI * (double)u / (double)U;
        cs[u] = std::cos(th);
        sn[u] = std::sin(th);
        if (std::fabs(cs[u]) < 1e-12) cs[u] = 0.0;
        if (std::fabs(sn[u]) < 1e-12) sn[u] = 0.0;
    }
}

}  // namespace
}  // namespace satpila

using namespace satpila;

extern "C" int drt_bilinear(int32_t n, int32_t n_angles, int32_t n_bins, const double* angles_rad, int32_t n_items,
                            const float* images, float* sino, void* stream) {
    if (n < 1 || n_angles < 1 || n_bins < 1 || n_items < 0 || !images || !sino)
        return fail(SATPILA_ERR_INVALID_ARG, "drt_bilinear: bad argument");
    if (!is_device_pointer(images) || !is_device_pointer(sino))
        return fail(SATPILA_ERR_INVALID_ARG, "drt_bilinear: images and sino must be device memory");
    if (n_items == 0) return SATPILA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> cs, sn;
    angle_tables(n_angles, angles_rad, cs, sn);
    double* d_tab = nullptr;
    SP_CUDA(cudaMalloc(&d_tab, 2 * (size_t)n_angles * sizeof(double)));
    cudaError_t e = cudaMemcpyAsync(d_tab, cs.data(), n_angles * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tab + n_angles, sn.data(), n_angles * sizeof(double), cudaMemcpyHostToDevice, s);
    const long long total = (long long)n_items * n_angles * n_bins;
    if (e == cudaSuccess) {
        drt_bilinear_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(images, n_items, n, n_angles, n_bins, d_tab,
                                                                           d_tab + n_angles, sino);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_tab);
    if (e != cudaSuccess) return cuda_fail(e, "drt_bilinear");
    return SATPILA_OK;
}

extern "C" int sat_drt_run(int32_t n, int32_t n_angles, int32_t n_bins, const uint8_t* mask, int32_t n_chains,
                           const float* sino_meas, float* images, const sat_params* prm, sat_stats* stats,
                           void* stream) {
    if (n < 1 || n_angles < 1 || n_bins < 1 || n_chains < 0 || !prm || !sino_meas || !images)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_drt_run: bad argument");
    if (prm->bome_k < 1 || prm->bome_k > kMaxK || !(prm->beta > 0.0f) || prm->n_sweeps < 0 ||
        prm->moves_per_sweep < 0 || !(prm->t0 > 0.0) || prm->schedule < SAT_SCHED_LINEAR ||
        prm->schedule > SAT_SCHED_CUBIC)
        return fail(SATPILA_ERR_INVALID_ARG, "sat_drt_run: bad sat_params (t0 must be given)");
    if (!is_device_pointer(sino_meas) || !is_device_pointer(images) || (prm->trace && !is_device_pointer(prm->trace)))
        return fail(SATPILA_ERR_INVALID_ARG, "sat_drt_run: buffers must be device memory");
    if (n_chains == 0) return SATPILA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const long long P = (long long)n * n;
    std::vector<int32_t> list;
    for (long long q = 0; q < P; ++q)
        if (!mask || mask[q]) list.push_back((int32_t)q);
    std::vector<double> cs, sn;
    angle_tables(n_angles, nullptr, cs, sn);
    const size_t off_tab = 0, off_list = 2 * (size_t)n_angles * 8, off_S = off_list + ((list.size() * 4 + 255) & ~(size_t)255);
    const size_t off_acc = off_S + (size_t)n_chains * 8, bytes = off_acc + (size_t)n_chains * 8;
    char* ws = nullptr;
    SP_CUDA(cudaMalloc(&ws, bytes));
    cudaError_t e = cudaMemcpyAsync(ws + off_tab, cs.data(), n_angles * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws + off_tab + n_angles * 8, sn.data(), n_angles * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !list.empty())
        e = cudaMemcpyAsync(ws + off_list, list.data(), list.size() * 4, cudaMemcpyHostToDevice, s);
    DrtArgs a{};
    a.n = n;
    a.U = n_angles;
    a.B = n_bins;
    a.cs = (const double*)(ws + off_tab);
    a.sn = a.cs + n_angles;
    a.list = (const int32_t*)(ws + off_list);
    a.n_list = (int)list.size();
    a.moves = prm->moves_per_sweep > 0 ? prm->moves_per_sweep : (int)list.size();
    a.n_sweeps = prm->n_sweeps;
    a.K = prm->bome_k;
    a.schedule = prm->schedule;
    a.beta = prm->beta;
    a.t0 = prm->t0;
    a.tn = prm->tn;
    a.seed = prm->seed;
    a.sino = sino_meas;
    a.img = images;
    a.S = (double*)(ws + off_S);
    a.accepted = (unsigned long long*)(ws + off_acc);
    a.trace = prm->trace;
    a.trace_chain = prm->trace_chain;
    a.trace_cap = prm->trace ? (long long)prm->n_sweeps * a.moves : 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        sat_drt_kernel<<<n_chains, kDrtThreads, 0, s>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    std::vector<double> S(n_chains);
    std::vector<unsigned long long> acc(n_chains);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.data(), a.S, n_chains * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(acc.data(), a.accepted, n_chains * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.0f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ws);
    if (e != cudaSuccess) return cuda_fail(e, "sat_drt_run");
    if (stats) {
        const double cells = (double)n_angles * n_bins;
        for (int c = 0; c < n_chains; ++c) {
            sat_stats& st = stats[c];
            std::memset(&st, 0, sizeof(st));
            st.t0 = prm->t0;
            st.tn = prm->tn < 0.0 ? prm->t0 / 1000.0 : prm->tn;
            st.final_cost = std::sqrt(std::max(0.0, S[c] / cells));
            st.final_cost_incremental = st.final_cost;
            st.accepted = (int64_t)acc[c];
            st.proposed = (int64_t)prm->n_sweeps * (list.empty() ? 0 : a.moves);
            st.near_ties = -1;
            st.sweep_ms = ms;
        }
    }
    return SATPILA_OK;
}
