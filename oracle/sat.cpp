// Reference oracle: simulated annealing tomography.  TEST INFRASTRUCTURE ONLY
// (see oracle.h).  FP64 throughout; follows Steps 1-4 of Sec. II-A in the
// paper's order, with the PILA update of Eq. (6), the cost update of Eq. (7)
// and the best-of-multiple-estimates rule of Sec. III-B.
//
// Readings where the paper is silent (each also listed in the design notes):
//  * Random stream: Philox4x32-10 keyed by the chain seed, counter
//    (stage, move, block, stream id 1).  Draw d = 4*block + word; d = 0 picks
//    the pixel (floor(x * M / 2^32) over the mask list in raster order),
//    d = 1 is the acceptance number N1, d = 2 + c is estimate c's uniform.
//    A uniform is ((x >> 9) * 2 + 1) * 2^-24, exact in FP32 and FP64.
//  * Eq. (3) with its redraw rule is the uniform law on
//    [max(0, f - beta), min(beta, f + beta)]: one draw, same distribution.
//  * BoME, OR_BOME_SAME_PIXEL: all N_e estimates are values at the pixel
//    drawn for the move.  OR_BOME_INDEPENDENT (the paper's wording, Sec.
//    III-B): estimate c is a value at its own pixel; draw 2 + c is its value,
//    draw 2 + N_e + (c - 1) picks its pixel for c >= 1 (estimate 0 uses draw
//    0), so with N_e = 1 both modes draw the same move.
//  * Step 4 with dC == 0 accepts; with T == 0 only dC <= 0 is accepted.
//  * Stage s = 0..S-1 runs at T_s of the chosen schedule (T_N itself is the
//    limit that is never run).
//  * Eq. (8): proposals from the initial image (stream id 2, counter
//    (try, 0, block, 2)), single estimate, first Q with C' > C.
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

const uint32_t kStreamSat = 1u;
const uint32_t kStreamT0 = 2u;

double uniform01(uint32_t x) { return (double)((x >> 9) * 2u + 1u) * 0x1p-24; }

uint32_t pick(uint32_t x, uint32_t m) { return (uint32_t)(((uint64_t)x * (uint64_t)m) >> 32); }

void draw_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t stream, int nblk, uint32_t* w) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int b = 0; b < nblk; ++b) {
        const uint32_t ctr[4] = {c0, c1, (uint32_t)b, stream};
        or_philox4x32_10(ctr, key, w + 4 * b);
    }
}

struct Problem {
    int n = 0, U = 0, B = 0;
    std::vector<int32_t> bins;   // PILA, Eq. (5)
    std::vector<double> lens;
    std::vector<double> pc;      // calculated projections P_c
    const double* pm = nullptr;  // measured projections P_m
    std::vector<int32_t> list;   // pixels that may be chosen
    double inv_BU = 0.0;
    double C = 0.0;              // current cost, Eq. (4)
    int32_t format = OR_LEN_EXACT;
};

// Projections of image through the table: sum_p f_p l(p, u, k).
void table_projection(const Problem& pb, const double* image, double* out) {
    std::fill(out, out + (size_t)pb.U * pb.B, 0.0);
    const size_t P = (size_t)pb.n * pb.n;
    for (size_t p = 0; p < P; ++p)
        for (int u = 0; u < pb.U; ++u)
            for (int slot = 0; slot < 2; ++slot) {
                const size_t e = (p * pb.U + u) * 2 + slot;
                if (pb.lens[e] != 0.0) out[(size_t)u * pb.B + pb.bins[e]] += image[p] * pb.lens[e];
            }
}

int setup(Problem& pb, const or_geom* g, const uint8_t* mask, const double* pm, const double* image,
          int32_t length_format) {
    pb.n = g->n;
    pb.U = g->n_angles;
    pb.B = g->n_bins;
    const size_t P = (size_t)pb.n * pb.n;
    pb.bins.assign(P * pb.U * 2, -1);
    pb.lens.assign(P * pb.U * 2, 0.0);
    if (or_pila(g, pb.bins.data(), pb.lens.data()) != 0) return -1;
    pb.format = length_format;
    pb.pc.assign((size_t)pb.U * pb.B, 0.0);
    if (length_format == OR_LEN_EXACT) {
        if (or_drt(g, image, pb.pc.data()) != 0) return -1;  // initial projections by the DRT
    } else {
        if (length_format != OR_LEN_BINARY16 && length_format != OR_LEN_BYTE180) return -1;
        for (size_t e = 0; e < pb.lens.size(); ++e) pb.lens[e] = or_round_length(length_format, pb.lens[e]);
        table_projection(pb, image, pb.pc.data());  // the same projections through the stored table
    }
    pb.pm = pm;
    pb.list.clear();
    for (size_t p = 0; p < P; ++p)
        if (!mask || mask[p]) pb.list.push_back((int32_t)p);
    pb.inv_BU = 1.0 / ((double)pb.U * pb.B);
    pb.C = or_cost(pb.U, pb.B, pb.pc.data(), pm);
    return 0;
}

// Eq. (7) summand total for a change df at pixel p:
//   sum_u { 2 [P_c - P_m](alpha_u, k_u) * df * l_u + (df * l_u)^2 }.
// Also returns the magnitude of its terms for tolerance bookkeeping.
double eq7_sum(const Problem& pb, int p, double df, double* scale) {
    double sum = 0.0, mag_rl = 0.0, l2 = 0.0;
    const size_t base = (size_t)p * pb.U * 2;
    for (int u = 0; u < pb.U; ++u) {
        for (int slot = 0; slot < 2; ++slot) {
            const size_t e = base + (size_t)u * 2 + slot;
            const double l = pb.lens[e];
            if (l == 0.0) continue;
            const size_t cell = (size_t)u * pb.B + pb.bins[e];
            const double r = pb.pc[cell] - pb.pm[cell];
            sum += 2.0 * r * df * l + (df * l) * (df * l);
            mag_rl += std::fabs(r * l);
            l2 += l * l;
        }
    }
    if (scale) *scale = 2.0 * std::fabs(df) * mag_rl + df * df * l2;
    return sum;
}

// Eq. (6): P'_c(alpha_u, k_u) = P_c(alpha_u, k_u) + df * l_u.
void eq6_apply(Problem& pb, int p, double df) {
    const size_t base = (size_t)p * pb.U * 2;
    for (int u = 0; u < pb.U; ++u)
        for (int slot = 0; slot < 2; ++slot) {
            const size_t e = base + (size_t)u * 2 + slot;
            if (pb.lens[e] == 0.0) continue;
            pb.pc[(size_t)u * pb.B + pb.bins[e]] += df * pb.lens[e];
        }
}

double cost_after(const Problem& pb, double sum) {
    return std::sqrt(std::fmax(0.0, pb.C * pb.C + sum * pb.inv_BU));  // Eq. (7)
}

int t0_estimate(const Problem& pb, const double* image, const or_sat_params* prm, double* t0, int32_t* found) {
    const int Q = prm->t0_samples > 0 ? prm->t0_samples : 200;
    const int64_t max_tries = 100LL * Q;
    double total = 0.0;
    int got = 0;
    if (!pb.list.empty()) {
        for (int64_t t = 0; t < max_tries && got < Q; ++t) {
            uint32_t w[4];
            draw_words(prm->seed, (uint32_t)t, 0u, kStreamT0, 1, w);
            const int p = pb.list[pick(w[0], (uint32_t)pb.list.size())];
            const double f = image[p];
            const double lo = std::fmax(0.0, f - prm->beta), hi = std::fmin(prm->beta, f + prm->beta);
            const double fc = lo + uniform01(w[2]) * (hi - lo);
            const double Cp = cost_after(pb, eq7_sum(pb, p, fc - f, nullptr));
            const double dC = Cp - pb.C;
            if (dC > 0.0) {
                total += dC;
                ++got;
            }
        }
    }
    *found = got;
    // Eq. (8): T0 = -sum(C' - C) / (Q ln 0.9), Q = samples actually found.
    *t0 = got > 0 ? -total / ((double)got * std::log(0.9)) : 0.0;
    return 0;
}

// Eq. (3): uniform on [lo, hi]; or, for the exhaustive-search check, a
// uniformly drawn level of the grid {0, beta/(L-1), ..., beta}.
double estimate_value(const or_sat_params* prm, double f, double lo, double hi, uint32_t word) {
    (void)f;
    if (prm->grid_levels >= 2) {
        const int L = prm->grid_levels;
        const int lev = std::min(L - 1, (int)(uniform01(word) * L));
        return prm->beta * (double)lev / (double)(L - 1);
    }
    return lo + uniform01(word) * (hi - lo);
}

struct Choice {
    int cstar;
    double fbest, dfbest, sum_best, Cp_best, scale_best, gap;
};

// Sec. III-B: evaluate the N_e estimates and keep the one with the smallest
// cost C' (the lowest index wins a tie).  gap is how far the runner-up's
// Eq. (7) sum lies above the winner's.
Choice best_estimate(const Problem& pb, int p, double f, const uint32_t* w, const or_sat_params* prm,
                     std::vector<double>* sums_out) {
    const int K = prm->bome_k;
    const double lo = std::fmax(0.0, f - prm->beta), hi = std::fmin(prm->beta, f + prm->beta);
    std::vector<double> local;
    std::vector<double>& sums = sums_out ? *sums_out : local;
    sums.assign(K, 0.0);
    std::vector<double> fcs(K), scales(K), cps(K);
    for (int c = 0; c < K; ++c) {
        fcs[c] = estimate_value(prm, f, lo, hi, w[2 + c]);
        sums[c] = eq7_sum(pb, p, fcs[c] - f, &scales[c]);
        cps[c] = cost_after(pb, sums[c]);
    }
    int best = 0;
    for (int c = 1; c < K; ++c)
        if (cps[c] < cps[best]) best = c;
    double second = INFINITY;
    for (int c = 0; c < K; ++c)
        if (c != best && sums[c] < second) second = sums[c];
    return Choice{best, fcs[best], fcs[best] - f, sums[best], cps[best], scales[best], second - sums[best]};
}

// Words per move: 2 + N_e, plus N_e - 1 pixel draws in the independent mode.
int move_blocks(const or_sat_params* prm) {
    const int words = prm->bome_mode == OR_BOME_INDEPENDENT ? 2 * prm->bome_k + 1 : prm->bome_k + 2;
    return (words + 3) / 4;
}

int estimate_pixel(const Problem& pb, const uint32_t* w, int K, int c) {
    const uint32_t x = c == 0 ? w[0] : w[2 + K + (c - 1)];
    return pb.list[pick(x, (uint32_t)pb.list.size())];
}

struct IndChoice {
    Choice ch;
    int pixel;  // the chosen estimate's pixel
    double f;   // its value before the move
};

// Sec. III-B as written: N_e estimates, each a random pixel of the
// reconstruction space with a random value by Eq. (3); all are evaluated on
// the same current state and the one with the smallest cost is kept.
IndChoice best_independent(const Problem& pb, const double* image, const uint32_t* w, const or_sat_params* prm,
                           std::vector<double>* sums_out, std::vector<int>* pix_out) {
    const int K = prm->bome_k;
    std::vector<double> local;
    std::vector<double>& sums = sums_out ? *sums_out : local;
    std::vector<int> lpix;
    std::vector<int>& pix = pix_out ? *pix_out : lpix;
    sums.assign(K, 0.0);
    pix.assign(K, 0);
    std::vector<double> fcs(K), fs(K), scales(K), cps(K);
    for (int c = 0; c < K; ++c) {
        pix[c] = estimate_pixel(pb, w, K, c);
        fs[c] = image[pix[c]];
        const double lo = std::fmax(0.0, fs[c] - prm->beta), hi = std::fmin(prm->beta, fs[c] + prm->beta);
        fcs[c] = estimate_value(prm, fs[c], lo, hi, w[2 + c]);
        sums[c] = eq7_sum(pb, pix[c], fcs[c] - fs[c], &scales[c]);
        cps[c] = cost_after(pb, sums[c]);
    }
    int best = 0;
    for (int c = 1; c < K; ++c)
        if (cps[c] < cps[best]) best = c;
    double second = INFINITY;
    for (int c = 0; c < K; ++c)
        if (c != best && sums[c] < second) second = sums[c];
    IndChoice r;
    r.ch = Choice{best, fcs[best], fcs[best] - fs[best], sums[best], cps[best], scales[best], second - sums[best]};
    r.pixel = pix[best];
    r.f = fs[best];
    return r;
}

}  // namespace

extern "C" double or_round_length(int32_t format, double l) {
    if (format == OR_LEN_BYTE180) return std::nearbyint(l * 180.0) / 180.0;
    if (format != OR_LEN_BINARY16 || l == 0.0) return l;
    int e;
    std::frexp(l, &e);                                  // 2^(e-1) <= l < 2^e
    const double q = std::ldexp(1.0, std::max(e - 11, -24));  // 11 significant bits; subnormal quantum 2^-24
    return std::nearbyint(l / q) * q;
}

extern "C" double or_schedule_temp(int32_t schedule, double t0, double tn, int32_t s, int32_t n_sweeps) {
    const double N = (double)n_sweeps, n = (double)s;
    switch (schedule) {
        case OR_SCHED_GEOMETRIC:  // T_n = T0 (T_N / T0)^(n/N)
            if (t0 <= 0.0) return 0.0;
            return t0 * std::pow(tn / t0, n / N);
        case OR_SCHED_CUBIC:  // T_n = T0 - n^3 (T0 - T_N) / N^3, Eq. (9)
            return t0 - n * n * n * (t0 - tn) / (N * N * N);
        default:  // T_n = T0 - n (T0 - T_N) / N, Eq. (2)
            return t0 - n * (t0 - tn) / N;
    }
}

extern "C" int or_sat_t0(const or_geom* g, const uint8_t* mask, const double* pm, const double* image,
                         const or_sat_params* prm, double* t0_out, int32_t* found_out) {
    Problem pb;
    if (setup(pb, g, mask, pm, image, prm->length_format) != 0) return -1;
    return t0_estimate(pb, image, prm, t0_out, found_out);
}

extern "C" int or_sat_run(const or_geom* g, const uint8_t* mask, const double* pm, double* image,
                          const or_sat_params* prm, or_sat_stats* stats, or_trace_rec* trace) {
    if (prm->bome_k < 1 || prm->bome_k > 32 || prm->n_sweeps < 0) return -2;
    Problem pb;
    if (setup(pb, g, mask, pm, image, prm->length_format) != 0) return -1;
    or_sat_stats st;
    std::memset(&st, 0, sizeof(st));
    st.initial_cost = pb.C;
    // Step 1: the cooling schedule.
    double t0 = prm->t0;
    if (t0 <= 0.0) {
        if (t0_estimate(pb, image, prm, &t0, &st.t0_found) != 0) return -1;
    }
    const double tn = prm->tn < 0.0 ? t0 / 1000.0 : prm->tn;
    st.t0 = t0;
    st.tn = tn;
    const int64_t M = prm->moves_per_sweep > 0 ? prm->moves_per_sweep : (int64_t)pb.list.size();
    const int nblk = move_blocks(prm);
    std::vector<uint32_t> w(4 * nblk);
    int64_t rec = 0;
    for (int s = 0; s < prm->n_sweeps && !pb.list.empty(); ++s) {
        const double T = or_schedule_temp(prm->schedule, t0, tn, s, prm->n_sweeps);
        for (int64_t m = 0; m < M; ++m) {
            // Step 2: a random pixel and N_e candidate values for it.
            draw_words(prm->seed, (uint32_t)s, (uint32_t)m, kStreamSat, nblk, w.data());
            int p;
            Choice ch;
            if (prm->bome_mode == OR_BOME_INDEPENDENT) {
                // Step 2 + 3 + BoME: N_e (pixel, value) estimates, the cheapest kept.
                const IndChoice ic = best_independent(pb, image, w.data(), prm, nullptr, nullptr);
                p = ic.pixel;
                ch = ic.ch;
            } else {
                p = pb.list[pick(w[0], (uint32_t)pb.list.size())];
                // Step 3 + BoME: the estimate with the smallest cost, by Eq. (7).
                ch = best_estimate(pb, p, image[p], w.data(), prm, nullptr);
            }
            const double dC = ch.Cp_best - pb.C;
            // Step 4: Metropolis acceptance.
            const double n1 = uniform01(w[1]);
            const bool accept = (dC <= 0.0) || (T > 0.0 && n1 < std::exp(-dC / T));
            ++st.proposed;
            if (accept) {
                ++st.accepted;
                image[p] = ch.fbest;
                eq6_apply(pb, p, ch.dfbest);
                pb.C = ch.Cp_best;
            }
            if (trace) {
                or_trace_rec& tr = trace[rec++];
                tr.pixel = p;
                tr.cstar = ch.cstar;
                tr.accepted = accept ? 1 : 0;
                tr.pad = 0;
                tr.dS = ch.sum_best;
                tr.dC = dC;
                tr.fnew = image[p];
                tr.u_acc = n1;
                tr.temp = T;
                tr.scale_S = ch.scale_best;
                tr.gap_S = ch.gap;
            }
        }
    }
    st.final_cost = pb.C;
    std::vector<double> fresh((size_t)pb.U * pb.B);
    if (pb.format == OR_LEN_EXACT) {
        if (or_drt(g, image, fresh.data()) != 0) return -1;
    } else {
        table_projection(pb, image, fresh.data());
    }
    st.final_cost_fresh = or_cost(pb.U, pb.B, fresh.data(), pm);
    if (stats) *stats = st;
    return 0;
}

extern "C" int or_sat_lockstep(const or_geom* g, const uint8_t* mask, const double* pm, double* image,
                               const or_sat_params* prm, double t0, double tn, const or_gpu_trace* trace,
                               int64_t n_moves, double tol, or_lockstep_report* rep) {
    if (prm->bome_k < 1 || prm->bome_k > 32) return -2;
    Problem pb;
    if (setup(pb, g, mask, pm, image, prm->length_format) != 0) return -1;
    or_lockstep_report r;
    r.moves = 0;
    r.near_ties = 0;
    r.pixel_mismatch = -1;
    r.hard_mismatch = -1;
    r.max_err_dS = 0.0;
    r.max_err_dC = 0.0;
    r.max_err_f = 0.0;
    const int64_t M = prm->moves_per_sweep > 0 ? prm->moves_per_sweep : (int64_t)pb.list.size();
    const int nblk = move_blocks(prm);
    const bool indep = prm->bome_mode == OR_BOME_INDEPENDENT;
    std::vector<uint32_t> w(4 * nblk);
    std::vector<double> sums;
    std::vector<int> pix;
    int64_t idx = 0;
    for (int s = 0; s < prm->n_sweeps && idx < n_moves && !pb.list.empty(); ++s) {
        const double T = or_schedule_temp(prm->schedule, t0, tn, s, prm->n_sweeps);
        for (int64_t m = 0; m < M && idx < n_moves; ++m, ++idx) {
            const or_gpu_trace& gt = trace[idx];
            draw_words(prm->seed, (uint32_t)s, (uint32_t)m, kStreamSat, nblk, w.data());
            const int p0 = pb.list[pick(w[0], (uint32_t)pb.list.size())];
            if (!indep && p0 != gt.pixel) {
                r.pixel_mismatch = idx;
                goto done;
            }
            {
                Choice ch;
                if (indep) ch = best_independent(pb, image, w.data(), prm, &sums, &pix).ch;
                else ch = best_estimate(pb, p0, image[p0], w.data(), prm, &sums);
                int c = ch.cstar;
                if (gt.cstar != c) {
                    // BoME near-tie: the other side's pick is within tolerance of ours.
                    if (gt.cstar < 0 || gt.cstar >= prm->bome_k) {
                        r.hard_mismatch = idx;
                        goto done;
                    }
                    const double gap = sums[gt.cstar] - sums[c];
                    if (gap > 2.0 * tol * ch.scale_best) {
                        r.hard_mismatch = idx;
                        goto done;
                    }
                    ++r.near_ties;
                    c = gt.cstar;
                }
                // the move the other side made: estimate c at its pixel
                const int p = indep ? pix[c] : p0;
                if (p != gt.pixel) {
                    r.pixel_mismatch = idx;
                    goto done;
                }
                const double f = image[p];
                const double lo = std::fmax(0.0, f - prm->beta), hi = std::fmin(prm->beta, f + prm->beta);
                const double fc = estimate_value(prm, f, lo, hi, w[2 + c]);
                double scale = 0.0;
                const double sum = eq7_sum(pb, p, fc - f, &scale);
                const double Cp = cost_after(pb, sum);
                const double dC = Cp - pb.C;
                const double denom = Cp + pb.C;
                const double scale_C = denom > 0.0 ? scale * pb.inv_BU / denom : std::sqrt(scale * pb.inv_BU);
                if (scale > 0.0) r.max_err_dS = std::fmax(r.max_err_dS, std::fabs((double)gt.dS - sum) / scale);
                if (scale_C > 0.0) r.max_err_dC = std::fmax(r.max_err_dC, std::fabs((double)gt.dC - dC) / scale_C);
                const double n1 = uniform01(w[1]);
                bool accept = (dC <= 0.0) || (T > 0.0 && n1 < std::exp(-dC / T));
                if ((gt.accepted != 0) != accept) {
                    // Acceptance near-tie: dC within tolerance of the threshold
                    // T * (-ln N1), or of 0 when T == 0.
                    const double thr = T > 0.0 ? -T * std::log(n1) : 0.0;
                    if (std::fabs(dC - thr) > 2.0 * tol * scale_C && std::fabs(dC) > 2.0 * tol * scale_C) {
                        r.hard_mismatch = idx;
                        goto done;
                    }
                    ++r.near_ties;
                    accept = gt.accepted != 0;
                }
                if (accept) {
                    image[p] = fc;
                    eq6_apply(pb, p, fc - f);
                    pb.C = Cp;
                }
                r.max_err_f = std::fmax(r.max_err_f, std::fabs((double)gt.fnew - image[p]));
            }
        }
    }
done:
    r.moves = idx;
    if (rep) *rep = r;
    return 0;
}

// ---- exhaustive search over grid-valued images -----------------------------

namespace {

struct Exhaustive {
    int P = 0, L = 0, cells = 0;
    double beta = 0.0, tol = 0.0;
    std::vector<int32_t> bins;   // PILA [P][U][2]
    std::vector<double> lens;
    int U = 0, B = 0;
    const double* pm = nullptr;
    std::vector<double> pc;      // current projections
    std::vector<int> lev, dir;   // current level and direction per pixel
    double best = INFINITY;
    int64_t count = 0;
    std::vector<double> arg;

    void change(int p, int d) {  // pixel p moves by d levels
        const double df = beta * (double)d / (double)(L - 1);
        for (int u = 0; u < U; ++u)
            for (int e = 0; e < 2; ++e) {
                const size_t q = ((size_t)p * U + u) * 2 + e;
                if (bins[q] >= 0) pc[(size_t)u * B + bins[q]] += df * lens[q];
            }
        lev[p] += d;
    }
    void leaf() {
        double S = 0.0;
        for (int c = 0; c < cells; ++c) {
            const double r = pc[c] - pm[c];
            S += r * r;
        }
        if (S < best - tol) {
            best = S;
            count = 1;
            for (int p = 0; p < P; ++p) arg[p] = beta * (double)lev[p] / (double)(L - 1);
        } else if (S <= best + tol) {
            ++count;
        }
    }
    void visit(int d) {
        if (d == P) {
            leaf();
            return;
        }
        for (int t = 0; t < L; ++t) {
            if (t > 0) change(d, dir[d]);
            visit(d + 1);
        }
        dir[d] = -dir[d];
    }
};

}  // namespace

extern "C" int or_exhaustive_grid(const or_geom* g, const double* pm, int32_t levels, double beta, double* min_cost,
                                  int64_t* n_min, double* argmin_image) {
    const int P = g->n * g->n;
    if (levels < 2 || P > 16 || std::pow((double)levels, (double)P) > 67108864.0) return -2;
    Exhaustive ex;
    ex.P = P;
    ex.L = levels;
    ex.beta = beta;
    ex.U = g->n_angles;
    ex.B = g->n_bins;
    ex.cells = ex.U * ex.B;
    ex.pm = pm;
    ex.bins.resize((size_t)P * ex.U * 2);
    ex.lens.resize((size_t)P * ex.U * 2);
    if (or_pila(g, ex.bins.data(), ex.lens.data()) != 0) return -1;
    ex.pc.assign(ex.cells, 0.0);  // every pixel starts at level 0
    ex.lev.assign(P, 0);
    ex.dir.assign(P, 1);
    ex.arg.assign(P, 0.0);
    double norm = 0.0;
    for (int c = 0; c < ex.cells; ++c) norm += pm[c] * pm[c];
    ex.tol = 1e-9 * std::max(1.0, norm);
    ex.visit(0);
    if (min_cost) *min_cost = std::sqrt(ex.best / (double)ex.cells);
    if (n_min) *n_min = ex.count;
    if (argmin_image)
        for (int p = 0; p < P; ++p) argmin_image[p] = ex.arg[p];
    return 0;
}
