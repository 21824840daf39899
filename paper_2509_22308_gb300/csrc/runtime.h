// Host-side helpers shared by the single-domain and the batched runtimes.
#pragma once

#include <string>
#include <vector>

#include "../../include/lbm_em.h"
#include "common.cuh"

namespace lbmem {

extern thread_local std::string g_last_error;
lbm_em_status set_error(lbm_em_status st, const std::string &msg);
lbm_em_status cuda_status(cudaError_t e, const char *what);

// Constants of the exact discrete incident plane wave for period T (see common.cuh).
void incident_constants(int period, double E0, double *pr, double *pi, double *qr, double *qi);
// Wavenumber of the lattice's right-going vacuum plane wave of period T (arg w).
double lattice_wavenumber(int period);
// (cos w t, sin w t) for t = 0..T-1, w = 2 pi / T.
std::vector<double2> phase_table(int period);

// Constants of one material in the kernel's type.  3 eps_r is rounded once and
// c_d = 2 (3 eps_r) - 4 is derived from the rounded value (exact in FP32 and FP64 for
// eps_r < 2^20), so that (c_d + 4) / c3 = 2 holds in the table: the collision conserves D
// up to the one rounding of D / c3 instead of scaling it by a fixed rounded constant.
template <typename T>
inline MatT<T> material_entry(double eps, bool pec) {
    if (pec) return MatT<T>{(T)0, (T)0, (T)0, (T)1};
    const T c3 = (T)(3.0 * eps);
    return MatT<T>{(T)(1.0 / (3.0 * eps)), (T)2 * c3 - (T)4, (T)(1.0 / eps), c3};
}

// Double-float table: every constant is the nearest double-float of its FP64 value (the
// residual bias, ~2^-48 per step, stays below 1e-10 over 10^5 steps).
template <>
inline MatT<df> material_entry<df>(double eps, bool pec) {
    if (pec) return MatT<df>{df(0.0), df(0.0), df(0.0), df(1.0)};
    return MatT<df>{df(1.0 / (3.0 * eps)), df(6.0 * eps - 4.0), df(1.0 / eps), df(3.0 * eps)};
}

lbm_em_status check_source(const lbm_em_source *s);
lbm_em_status check_janus(const lbm_em_janus *j);
void janus_center(const lbm_em_janus *j, int nx, int ny, double *cx, double *cy);
int round_up(int v, int m);

// Circle contour in lattice coordinates with its unique stencil sites.
struct ContourHost {
    double E0 = 1.0, R = 0.0, dl = 0.0, F0 = 1.0, M0 = 1.0;
    std::vector<ContourPt> pts;
    std::vector<int> site_xy;  // 2 per slot
    int n_slots = 0, y0 = 0, y1 = -1;
};
lbm_em_status build_contour(int nx, int ny, const lbm_em_contour *c, ContourHost *out);

}  // namespace lbmem
