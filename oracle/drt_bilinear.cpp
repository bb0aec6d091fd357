// Reference oracle: the conventional SAT of Sec. III-A that the PILA
// replaces.  TEST INFRASTRUCTURE ONLY (see oracle.h).  FP64.
//
//  * DRT by bilinear interpolation (the standard scheme the paper compares
//    against): ray (u, k) is the line x cos(theta_u) + y sin(theta_u) = s_k;
//    it is sampled at unit steps t_m = m - (B - 1)/2, m = 0..B-1, along its
//    direction (-sin, cos), i.e. at (s_k cos - t_m sin, s_k sin + t_m cos);
//    each sample is the bilinear interpolation of the image between pixel
//    centres (pixel (i, j) at (j - (n-1)/2, (n-1)/2 - i); zero outside the
//    grid), and the projection is the sum of the samples (step 1).
//    B = 2 floor(n / sqrt 2) + 1 samples cover the image diagonal.
//  * SAT with a full DRT per move: Steps 1-4 with the same random stream as
//    the PILA form (draw 0 pixel, 1 = N1, 2 + e = estimate e at that pixel),
//    every estimate evaluated by a fresh bilinear DRT of the candidate image
//    and Eq. (4); Step 4 with the exponential.
#include "oracle.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace {

void dir_of(const or_geom* g, int u, double* c, double* s) {
    const double th = g->angles ? g->angles[u] : M_PI * (double)u / (double)g->n_angles;
    *c = std::cos(th);
    *s = std::sin(th);
    if (std::fabs(*c) < 1e-12) *c = 0.0;
    if (std::fabs(*s) < 1e-12) *s = 0.0;
}

double pixel(const double* img, int n, int i, int j) {
    if (i < 0 || j < 0 || i >= n || j >= n) return 0.0;
    return img[(size_t)i * n + j];
}

// Bilinear interpolation at (x, y) between pixel centres.
double bilinear(const double* img, int n, double x, double y) {
    const double cj = x + 0.5 * (n - 1), ri = 0.5 * (n - 1) - y;
    const double j0 = std::floor(cj), i0 = std::floor(ri);
    const double a = cj - j0, b = ri - i0;
    const int j = (int)j0, i = (int)i0;
    return (1.0 - a) * (1.0 - b) * pixel(img, n, i, j) + a * (1.0 - b) * pixel(img, n, i, j + 1) +
           (1.0 - a) * b * pixel(img, n, i + 1, j) + a * b * pixel(img, n, i + 1, j + 1);
}

void drt_bilinear(const or_geom* g, const double* img, double* out) {
    const int n = g->n, U = g->n_angles, B = g->n_bins;
    for (int u = 0; u < U; ++u) {
        double c, s;
        dir_of(g, u, &c, &s);
        for (int k = 0; k < B; ++k) {
            const double sk = (double)k - 0.5 * (B - 1);
            double acc = 0.0;
            for (int m = 0; m < B; ++m) {
                const double t = (double)m - 0.5 * (B - 1);
                acc += bilinear(img, n, sk * c - t * s, sk * s + t * c);
            }
            out[(size_t)u * B + k] = acc;
        }
    }
}

double cost_of(const double* p, const double* pm, size_t cells) {
    double acc = 0.0;
    for (size_t e = 0; e < cells; ++e) {
        const double d = p[e] - pm[e];
        acc += d * d;
    }
    return std::sqrt(acc / (double)cells);
}

double uniform01(uint32_t x) { return (double)((x >> 9) * 2u + 1u) * 0x1p-24; }

}  // namespace

extern "C" int or_drt_bilinear(const or_geom* g, const double* image, double* sino) {
    if (!g || !image || !sino || g->n < 1 || g->n_angles < 1 || g->n_bins < 1) return -1;
    drt_bilinear(g, image, sino);
    return 0;
}

extern "C" int or_sat_drt_run(const or_geom* g, const uint8_t* mask, const double* pm, double* image,
                              const or_sat_params* prm, or_sat_stats* stats, or_trace_rec* trace) {
    if (prm->bome_k < 1 || prm->bome_k > 32 || prm->n_sweeps < 0 || !(prm->t0 > 0.0)) return -2;
    const int n = g->n;
    const size_t P = (size_t)n * n, cells = (size_t)g->n_angles * g->n_bins;
    std::vector<int32_t> list;
    for (size_t q = 0; q < P; ++q)
        if (!mask || mask[q]) list.push_back((int32_t)q);
    std::vector<double> pc(cells), trial(cells);
    drt_bilinear(g, image, pc.data());
    double C = cost_of(pc.data(), pm, cells);
    or_sat_stats st;
    std::memset(&st, 0, sizeof(st));
    st.initial_cost = C;
    st.t0 = prm->t0;
    st.tn = prm->tn < 0.0 ? prm->t0 / 1000.0 : prm->tn;
    const int64_t M = prm->moves_per_sweep > 0 ? prm->moves_per_sweep : (int64_t)list.size();
    const int K = prm->bome_k, nblk = (K + 2 + 3) / 4;
    std::vector<uint32_t> w(4 * nblk);
    const uint32_t key[2] = {(uint32_t)prm->seed, (uint32_t)(prm->seed >> 32)};
    int64_t rec = 0;
    for (int sg = 0; sg < prm->n_sweeps && !list.empty(); ++sg) {
        const double T = or_schedule_temp(prm->schedule, st.t0, st.tn, sg, prm->n_sweeps);
        for (int64_t m = 0; m < M; ++m) {
            for (int b = 0; b < nblk; ++b) {
                const uint32_t ctr[4] = {(uint32_t)sg, (uint32_t)m, (uint32_t)b, 1u};
                or_philox4x32_10(ctr, key, &w[4 * b]);
            }
            const int p = list[(uint32_t)(((uint64_t)w[0] * (uint64_t)list.size()) >> 32)];
            const double f = image[p];
            const double lo = std::fmax(0.0, f - prm->beta), hi = std::fmin(prm->beta, f + prm->beta);
            int best = 0;
            double best_C = INFINITY, best_f = f;
            for (int e = 0; e < K; ++e) {
                const double fc = lo + uniform01(w[2 + e]) * (hi - lo);
                image[p] = fc;
                drt_bilinear(g, image, trial.data());  // the full DRT of the candidate image
                const double Cp = cost_of(trial.data(), pm, cells);
                if (Cp < best_C) {
                    best_C = Cp;
                    best = e;
                    best_f = fc;
                }
            }
            image[p] = f;
            const double dC = best_C - C;
            const double n1 = uniform01(w[1]);
            const bool accept = dC <= 0.0 || (T > 0.0 && n1 < std::exp(-dC / T));
            ++st.proposed;
            if (accept) {
                ++st.accepted;
                image[p] = best_f;
                C = best_C;
            }
            if (trace) {
                or_trace_rec& tr = trace[rec++];
                tr.pixel = p;
                tr.cstar = best;
                tr.accepted = accept ? 1 : 0;
                tr.pad = 0;
                tr.dS = 0.0;
                tr.dC = dC;
                tr.fnew = image[p];
                tr.u_acc = n1;
                tr.temp = T;
                tr.scale_S = 0.0;
                tr.gap_S = 0.0;
            }
        }
    }
    drt_bilinear(g, image, pc.data());
    st.final_cost = C;
    st.final_cost_fresh = cost_of(pc.data(), pm, cells);
    if (stats) *stats = st;
    return 0;
}
