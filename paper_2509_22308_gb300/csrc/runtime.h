// Host-side helpers shared by the single-domain and the batched runtimes.
#pragma once

#include <cmath>
#include <string>
#include <type_traits>
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

// Power-of-two scale of an amplitude: k with 2^k <= |E0| < 2^(k + 1), 0 for E0 = 0, clamped
// to [-100, 100].  Every field and force of the (linear) scheme scales with E0, so the
// reduced-precision forms and the runaway test use thresholds relative to 2^k.
inline int amplitude_exponent(double E0) {
    if (!(E0 != 0.0) || !std::isfinite(E0)) return 0;
    int e = 0;
    std::frexp(E0, &e);  // |E0| = m 2^e, 0.5 <= m < 1
    const int k = e - 1;
    return k < -100 ? -100 : k > 100 ? 100 : k;
}

// Threshold on the exponent field of the runaway test (field_runaway): |E/3| >= 2^(20 + k)
// for the amplitude exponent k; FP32 (and the leading word of double-float) in bits 23-30,
// FP64 in bits 20-30 of the high word.
template <typename T>
inline unsigned runaway_bits(double E0) {
    const int k = amplitude_exponent(E0);
    if constexpr (sizeof(T) == 8 && !std::is_same<T, df>::value)
        return (unsigned)(1023 + 20 + k) << 20;
    else
        return (unsigned)(127 + 20 + k) << 23;
}

// Scale of the FP16 deviations, 2^(10 - k): with E0 = 1 deviations up to ~64 stay below the FP16
// maximum after scaling and down to ~6e-8 stay normal, and the same holds relative to any E0.
inline float f16_scale(double E0) { return std::ldexp(1.0f, 10 - amplitude_exponent(E0)); }

// Allocation of device memory (cudaMalloc / stream-ordered cudaMallocAsync) and its release,
// through the library's fault-injection hook and count (alloc.cu, lbm_em_test_alloc_hook).
cudaError_t dmalloc(void **p, size_t bytes);
cudaError_t dmalloc_async(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p);                     // NULL is ignored
void dfree_async(void *p, cudaStream_t s);
template <typename P>
inline cudaError_t dmalloc(P **p, size_t bytes) { return dmalloc(reinterpret_cast<void **>(p), bytes); }
// cudaMemcpyAsync / cudaMemcpy2DAsync (same arguments) that also count the bytes moved per
// direction (lbm_em_transfer_bytes).
cudaError_t copy_async(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s);
cudaError_t copy2d_async(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t height,
                         cudaMemcpyKind kind, cudaStream_t s);
// One allocation attempt of any kind: true if the armed hook fails it.  alloc_held counts a
// buffer or pinned block taken (+1) or given back (-1) by a handle or batch.
bool alloc_should_fail();
void alloc_held(long long delta);

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
