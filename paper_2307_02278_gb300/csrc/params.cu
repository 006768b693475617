// Host-side choice of the Ewald splitting, the cutoffs and the SPME mesh:
// the paper's default mesh density (1.2 points per angstrom) and an
// accuracy-driven chooser whose error estimates were calibrated against a
// converged direct Ewald sum.
#include "mbd_internal.cuh"

#include <algorithm>
#include <cmath>

namespace mbd {
namespace {

// smallest 2^a 3^b 5^c >= n
int smooth_at_least(double n) {
    if (!(n < 1e9)) return 0;
    int k = std::max(1, (int)std::ceil(n - 1e-9));
    for (;; ++k) {
        int m = k;
        for (int f : {2, 3, 5})
            while (m % f == 0) m /= f;
        if (m == 1) return k;
    }
}

// plane spacings w_a = 1 / |a*_a| of the cell; false for a degenerate cell
bool plane_spacings(const double *c, double w[3]) {
    const double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                       c[2] * (c[3] * c[7] - c[4] * c[6]);
    if (!(std::fabs(det) > 1e-12)) return false;
    // a*_a = (a_b x a_c) / det
    for (int a = 0; a < 3; ++a) {
        const double *u = c + 3 * ((a + 1) % 3), *v = c + 3 * ((a + 2) % 3);
        const double x = u[1] * v[2] - u[2] * v[1], y = u[2] * v[0] - u[0] * v[2], z = u[0] * v[1] - u[1] * v[0];
        w[a] = std::fabs(det) / std::sqrt(x * x + y * y + z * z);
    }
    return true;
}

bool order_ok(int p) { return p >= 4 && p <= kMaxOrder && p % 2 == 0; }

}  // namespace
}  // namespace mbd

using namespace mbd;

extern "C" mbd_status mbd_mesh_for_density(const double cell[9], double points_per_bohr, int32_t spline_order,
                                           int32_t mesh[3]) {
    if (!cell || !mesh || !order_ok(spline_order)) return MBD_ERR_INVALID_ARG;
    double w[3];
    if (!plane_spacings(cell, w)) return MBD_ERR_INVALID_ARG;
    const double rho = points_per_bohr > 0.0 ? points_per_bohr : MBD_DEFAULT_MESH_DENSITY;
    int out[3];
    for (int a = 0; a < 3; ++a) {
        const double len = std::sqrt(cell[3 * a] * cell[3 * a] + cell[3 * a + 1] * cell[3 * a + 1] +
                                     cell[3 * a + 2] * cell[3 * a + 2]);
        out[a] = smooth_at_least(std::max(rho * len, 2.0 * spline_order));
        if (out[a] < 1 || out[a] > 1000) return MBD_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a) mesh[a] = out[a];
    return MBD_OK;
}

extern "C" mbd_status mbd_spme_params(mbd_system_desc *desc, double tol, double *est_err) {
    if (!desc || !(tol > 0.0 && tol < 1.0) || desc->n_atoms < 1 || !desc->r_vdw) return MBD_ERR_INVALID_ARG;
    const int p = desc->spline_order;
    if (!order_ok(p) || !(desc->damp_beta > 0.0) || !(desc->damp_d > 0.0)) return MBD_ERR_INVALID_ARG;
    double w[3];
    if (!plane_spacings(desc->cell, w)) return MBD_ERR_INVALID_ARG;
    const double lim = 0.49 * std::min(w[0], std::min(w[1], w[2]));
    const double cap = desc->r_cut > 0.0 ? desc->r_cut : 12.0;
    const double rc = std::min(cap, lim);
    const double part = tol / 3.0;
    // erfc truncation: 2 exp(-(beta rc)^2) = part
    const double beta = std::sqrt(std::log(2.0 / part)) / rc;
    // damping correction: 0.1 exp(-d (dc / R - 1)) = part, R = damp_beta x the largest pair of radii
    double rmax = 0.0;
    for (int i = 0; i < desc->n_atoms; ++i) {
        if (!(desc->r_vdw[i] > 0.0)) return MBD_ERR_INVALID_ARG;
        rmax = std::max(rmax, desc->r_vdw[i]);
    }
    const double R = desc->damp_beta * 2.0 * rmax;
    const double dc_need = R * (1.0 + std::log(0.1 / part) / desc->damp_d);
    const double dc = std::min(std::max(dc_need, rc), lim);
    // mesh: c_p (beta h)^p = part
    const double cp = p <= 4 ? 0.4 : 0.1;
    const double h = std::pow(part / cp, 1.0 / p) / beta;
    int K[3];
    for (int a = 0; a < 3; ++a) {
        K[a] = smooth_at_least(std::max(w[a] / h, 2.0 * p));
        if (K[a] < 1 || K[a] > 1000) return MBD_ERR_UNSUPPORTED;
    }
    double e_mesh = 0.0;
    for (int a = 0; a < 3; ++a) e_mesh = std::max(e_mesh, cp * std::pow(beta * w[a] / K[a], (double)p));
    const double e_real = 2.0 * std::exp(-(beta * rc) * (beta * rc));
    const double e_damp = 0.1 * std::exp(-desc->damp_d * (dc / R - 1.0));
    desc->ewald_beta = beta;
    desc->r_cut = rc;
    desc->damp_cut = dc;
    for (int a = 0; a < 3; ++a) desc->mesh[a] = K[a];
    const double est = e_real + e_damp + e_mesh;
    if (est_err) *est_err = est;
    return dc_need <= lim ? MBD_OK : MBD_ERR_UNSUPPORTED;
}
