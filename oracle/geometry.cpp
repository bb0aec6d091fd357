// Reference oracle: geometry part.  TEST INFRASTRUCTURE ONLY (see oracle.h).
//
//  * Philox4x32-10 counter-based generator, written from its published
//    definition (Salmon, Moraes, Dror & Shaw, SC'11): two 32x32->64
//    multiplications per round, Weyl-sequence key schedule, 10 rounds.
//  * Siddon-style ray traversal (cited by the paper in Sec. II-B): crossings
//    of the ray with every grid line, sorted; each interval between crossings
//    lies in one pixel and its length is the chord length.
//  * Eq. (1) (discrete Radon transform), Eq. (4) (cost), Eq. (5) (PILA, by
//    transposing the traversals), and the SIRT factor matrix of Sec. III-D.
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <vector>

extern "C" void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    // Round constants and key increments of Philox4x32 as published.
    const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = M0 * (uint64_t)c0;
        uint64_t p1 = M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

namespace {

const double kMinChord = 1e-12;

// cos/sin of a projection angle; values below 1e-12 in magnitude are exact
// zeros (pi/2 is not representable, so cos(pi/2) would otherwise be 6e-17).
void direction(double theta, double* c, double* s) {
    *c = std::cos(theta);
    *s = std::sin(theta);
    if (std::fabs(*c) < 1e-12) *c = 0.0;
    if (std::fabs(*s) < 1e-12) *s = 0.0;
}

double angle_of(const or_geom* g, int u) {
    if (g->angles) return g->angles[u];
    return M_PI * (double)u / (double)g->n_angles;
}

double bin_centre(const or_geom* g, int k) { return (double)k - 0.5 * (double)(g->n_bins - 1); }

}  // namespace

extern "C" int or_siddon_ray(int32_t n, double theta, double s, int32_t* pix, double* len, int32_t cap) {
    double c, sn;
    direction(theta, &c, &sn);
    const double half = 0.5 * n;
    // Ray: points q + t*d, q = s*(c, sn) on the normal, d = (-sn, c) along it.
    const double qx = s * c, qy = s * sn;
    const double dx = -sn, dy = c;
    int count = 0;
    auto emit = [&](int p, double l) -> bool {
        if (l < kMinChord) return true;
        if (count >= cap) return false;
        pix[count] = p;
        len[count] = l;
        ++count;
        return true;
    };
    if (dx == 0.0) {
        // Vertical line x = qx.  On a column edge it belongs to the column on
        // the +s side, i.e. towards +x when c > 0 and towards -x when c < 0.
        const double t = qx + half;
        const double colf = (c > 0) ? std::floor(t) : std::ceil(t) - 1.0;
        if (colf < 0 || colf >= n) return 0;
        const int col = (int)colf;
        for (int i = 0; i < n; ++i)
            if (!emit(i * n + col, 1.0)) return -1;
        return count;
    }
    if (dy == 0.0) {
        // Horizontal line y = qy; row i covers y in [n/2 - i - 1, n/2 - i].
        const double t = half - qy;
        const double rowf = (sn > 0) ? std::ceil(t) - 1.0 : std::floor(t);
        if (rowf < 0 || rowf >= n) return 0;
        const int row = (int)rowf;
        for (int j = 0; j < n; ++j)
            if (!emit(row * n + j, 1.0)) return -1;
        return count;
    }
    // General direction: parameters of the crossings with the grid lines
    // x = -n/2 + m and y = -n/2 + m, m = 0..n.
    const double tx0 = (-half - qx) / dx, tx1 = (half - qx) / dx;
    const double ty0 = (-half - qy) / dy, ty1 = (half - qy) / dy;
    const double t_in = std::max(std::min(tx0, tx1), std::min(ty0, ty1));
    const double t_out = std::min(std::max(tx0, tx1), std::max(ty0, ty1));
    if (!(t_in < t_out)) return 0;
    std::vector<double> ts;
    ts.reserve(2 * n + 4);
    ts.push_back(t_in);
    ts.push_back(t_out);
    for (int m = 0; m <= n; ++m) {
        const double t = (-half + m - qx) / dx;
        if (t > t_in && t < t_out) ts.push_back(t);
        const double t2 = (-half + m - qy) / dy;
        if (t2 > t_in && t2 < t_out) ts.push_back(t2);
    }
    std::sort(ts.begin(), ts.end());
    int cur_pix = -1;
    double cur_len = 0.0;
    for (size_t a = 0; a + 1 < ts.size(); ++a) {
        const double l = ts[a + 1] - ts[a];
        if (!(l > 0.0)) continue;
        const double tm = 0.5 * (ts[a] + ts[a + 1]);
        const double x = qx + tm * dx, y = qy + tm * dy;
        int col = (int)std::floor(x + half);
        int row = (int)std::floor(half - y);
        col = std::min(std::max(col, 0), n - 1);
        row = std::min(std::max(row, 0), n - 1);
        const int p = row * n + col;
        if (p == cur_pix) {
            cur_len += l;
        } else {
            if (cur_pix >= 0 && !emit(cur_pix, cur_len)) return -1;
            cur_pix = p;
            cur_len = l;
        }
    }
    if (cur_pix >= 0 && !emit(cur_pix, cur_len)) return -1;
    return count;
}

extern "C" int or_drt(const or_geom* g, const double* image, double* sino) {
    const int n = g->n, U = g->n_angles, B = g->n_bins;
    std::vector<int32_t> pix(4 * n + 8);
    std::vector<double> len(4 * n + 8);
    for (int u = 0; u < U; ++u) {
        const double theta = angle_of(g, u);
        for (int k = 0; k < B; ++k) {
            const int cnt = or_siddon_ray(n, theta, bin_centre(g, k), pix.data(), len.data(), (int)pix.size());
            if (cnt < 0) return -1;
            double acc = 0.0;
            for (int e = 0; e < cnt; ++e) acc += image[pix[e]] * len[e];
            sino[(size_t)u * B + k] = acc;
        }
    }
    return 0;
}

extern "C" int or_pila(const or_geom* g, int32_t* bins, double* lens) {
    const int n = g->n, U = g->n_angles, B = g->n_bins;
    const size_t P = (size_t)n * n;
    for (size_t e = 0; e < P * U * 2; ++e) {
        bins[e] = -1;
        lens[e] = 0.0;
    }
    std::vector<int32_t> pix(4 * n + 8);
    std::vector<double> len(4 * n + 8);
    for (int u = 0; u < U; ++u) {
        const double theta = angle_of(g, u);
        for (int k = 0; k < B; ++k) {  // ascending k keeps the two slots sorted
            const int cnt = or_siddon_ray(n, theta, bin_centre(g, k), pix.data(), len.data(), (int)pix.size());
            if (cnt < 0) return -1;
            for (int e = 0; e < cnt; ++e) {
                const size_t rec = ((size_t)pix[e] * U + u) * 2;
                if (bins[rec] < 0) {
                    bins[rec] = k;
                    lens[rec] = len[e];
                } else if (bins[rec + 1] < 0) {
                    bins[rec + 1] = k;
                    lens[rec + 1] = len[e];
                } else {
                    return -1;
                }
            }
        }
    }
    return 0;
}

extern "C" double or_cost(int32_t n_angles, int32_t n_bins, const double* pc, const double* pm) {
    const size_t cells = (size_t)n_angles * n_bins;
    double acc = 0.0;
    for (size_t e = 0; e < cells; ++e) {
        const double d = pc[e] - pm[e];
        acc += d * d;
    }
    return std::sqrt(acc / (double)cells);
}

extern "C" int or_sirt_factor(const or_geom* g, const uint8_t* mask, double* w) {
    const int n = g->n, U = g->n_angles, B = g->n_bins;
    std::vector<int32_t> pix(4 * n + 8);
    std::vector<double> len(4 * n + 8);
    for (int u = 0; u < U; ++u) {
        const double theta = angle_of(g, u);
        for (int k = 0; k < B; ++k) {
            const int cnt = or_siddon_ray(n, theta, bin_centre(g, k), pix.data(), len.data(), (int)pix.size());
            if (cnt < 0) return -1;
            double acc = 0.0;
            for (int e = 0; e < cnt; ++e)
                if (!mask || mask[pix[e]]) acc += len[e] * len[e];
            w[(size_t)u * B + k] = acc;
        }
    }
    return 0;
}
