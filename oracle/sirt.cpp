// Reference oracle: SIRT with PILA, Eqs. (10)-(11) of Sec. III-D.
// TEST INFRASTRUCTURE ONLY (see oracle.h).  FP64 throughout.
//
//   f(i,j) <- f(i,j) + relax * (1/U) * sum_u Delta f_u(i,j)              (10)
//   Delta f_u = (P_m - P_c)(alpha_u, k) / (sum l_uk^2) * l_u              (11)
// where sum l_uk^2 is the factor matrix over the reconstruction space.
// Readings: a pixel that two rays of one angle cross gets both rays' terms;
// rays whose factor is 0 contribute nothing; only mask pixels are updated.
//   SIMULTANEOUS: every mask pixel is updated from the same P_c, which is then
//                 recomputed by the DRT (classic SIRT).
//   SEQUENTIAL:   the paper's description: the mask pixels are visited one
//                 by one (raster order), each update immediately written into
//                 P_c through the PILA (Eq. (6)) before the next pixel.
#include "oracle.h"

#include <cmath>
#include <vector>

extern "C" int or_sirt_run(const or_geom* g, const uint8_t* mask, const double* pm, double* image,
                           int32_t n_iter, int32_t mode, double relax, double* costs) {
    const int n = g->n, U = g->n_angles, B = g->n_bins;
    const size_t P = (size_t)n * n, cells = (size_t)U * B;
    std::vector<int32_t> bins(P * U * 2);
    std::vector<double> lens(P * U * 2);
    if (or_pila(g, bins.data(), lens.data()) != 0) return -1;
    std::vector<double> w(cells);
    if (or_sirt_factor(g, mask, w.data()) != 0) return -1;
    std::vector<double> pc(cells);
    if (or_drt(g, image, pc.data()) != 0) return -1;

    auto pixel_update = [&](size_t p) {  // (1/U) sum_u Delta f_u, Eq. (10)-(11)
        double acc = 0.0;
        for (int u = 0; u < U; ++u)
            for (int slot = 0; slot < 2; ++slot) {
                const size_t e = (p * U + u) * 2 + slot;
                const double l = lens[e];
                if (l == 0.0) continue;
                const size_t cell = (size_t)u * B + bins[e];
                if (w[cell] == 0.0) continue;
                acc += (pm[cell] - pc[cell]) / w[cell] * l;
            }
        return acc / (double)U;
    };

    std::vector<double> delta(P, 0.0);
    for (int it = 0; it < n_iter; ++it) {
        if (mode == OR_SIRT_SIMULTANEOUS) {
            for (size_t p = 0; p < P; ++p) delta[p] = (!mask || mask[p]) ? pixel_update(p) : 0.0;
            for (size_t p = 0; p < P; ++p) image[p] += relax * delta[p];
            if (or_drt(g, image, pc.data()) != 0) return -1;
        } else if (mode == OR_SIRT_SEQUENTIAL) {
            for (size_t p = 0; p < P; ++p) {
                if (mask && !mask[p]) continue;
                const double d = relax * pixel_update(p);
                image[p] += d;
                for (int u = 0; u < U; ++u)
                    for (int slot = 0; slot < 2; ++slot) {
                        const size_t e = (p * U + u) * 2 + slot;
                        if (lens[e] == 0.0) continue;
                        pc[(size_t)u * B + bins[e]] += d * lens[e];
                    }
            }
        } else {
            return -2;
        }
        if (costs) costs[it] = or_cost(U, B, pc.data(), pm);
    }
    return 0;
}
