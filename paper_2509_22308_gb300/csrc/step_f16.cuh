// Arguments of the FP16-deviation storage form (see step_f16.cu).
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"

namespace lbmem {

// Deviation scale 2^10: |g| up to ~64 E0 stays below the FP16 maximum, and
// deviations down to ~6e-8 / 2^10 stay normal.
constexpr float kF16Scale = 1024.0f;

struct F16Args {
    int nx, ny, pitch, pad;
    size_t pstride;
    const uint8_t *mat;
    const MatT<float> *mtab;
    SourceParams src;
    AccParams accp;
    unsigned *err;
    float scale, inv_scale;
    const __half *g;            // 16 deviation planes (input, time t)
    const float *fe, *fhx, *fhy;  // field planes (input)
    __half *g_out;
    float *fe_out, *fhx_out, *fhy_out;
};

// Byte layout of one FP16-deviation buffer: 16 half planes, then 3 float planes,
// each plane pstride elements (offsets rounded to 256 bytes).
inline size_t f16_half_bytes(size_t pstride) { return ((size_t)NPLANES * pstride * 2 + 255) / 256 * 256; }
inline size_t f16_plane_bytes(size_t pstride) { return (pstride * 4 + 255) / 256 * 256; }
inline size_t f16_buffer_bytes(size_t pstride) { return f16_half_bytes(pstride) + 3 * f16_plane_bytes(pstride); }

// Equilibria (Eq. equilibrium distribution functions, TM^z components), each /6:
//   e_z: +x (E-Hy), -x (E+Hy), +y (E+Hx), -y (E-Hx), z E;     e_0 = (eps - 1) E
//   h_x: +-x Hx, +y (Hx+E), -y (Hx-E), z Hx;   h_y: +x (Hy-E), -x (Hy+E), +-y Hy, z Hy
struct Fld {
    float e, hx, hy;
};

__device__ __forceinline__ Fld load_fld(const F16Args &a, size_t i) {
    return Fld{a.fe[i], a.fhx[i], a.fhy[i]};
}

__device__ __forceinline__ float ldg_dev(const __half *p, float inv_scale) {
    return __half2float(*p) * inv_scale;
}

// f_i(r, t+1) for all 16 populations of site (x, y); F of time t at the neighbours.
__device__ __forceinline__ void pull_f16(const F16Args &a, int x, int y, long long t1, Pop<float> &p,
                                         float em1) {
    const size_t ps = a.pstride;
    const int xm = x > 0 ? x - 1 : 0;
    const int xp = x < a.nx - 1 ? x + 1 : x;
    const size_t r = (size_t)y * a.pitch;
    const size_t rm = (size_t)(y > 0 ? y - 1 : 0) * a.pitch;
    const size_t rp = (size_t)(y < a.ny - 1 ? y + 1 : y) * a.pitch;
    const float is = a.inv_scale, s6 = 1.0f / 6.0f;
    const Fld c = load_fld(a, r + x), w = load_fld(a, r + xm), e = load_fld(a, r + xp);
    const Fld so = load_fld(a, rm + x), no = load_fld(a, rp + x);
    const __half *g = a.g;
    p.e0 = em1 * c.e - ldg_dev(g + P_E0 * ps + r + x, is);
    p.ez = c.e * s6 - ldg_dev(g + P_EZ * ps + r + x, is);
    p.epx = (w.e - w.hy) * s6 - ldg_dev(g + P_EPX * ps + r + xm, is);
    p.emx = (e.e + e.hy) * s6 - ldg_dev(g + P_EMX * ps + r + xp, is);
    p.epy = (so.e + so.hx) * s6 - ldg_dev(g + P_EPY * ps + rm + x, is);
    p.emy = (no.e - no.hx) * s6 - ldg_dev(g + P_EMY * ps + rp + x, is);
    p.hxpx = w.hx * s6 - ldg_dev(g + P_HXPX * ps + r + xm, is);
    p.hxmx = e.hx * s6 - ldg_dev(g + P_HXMX * ps + r + xp, is);
    p.hxpy = (so.hx + so.e) * s6 - ldg_dev(g + P_HXPY * ps + rm + x, is);
    p.hxmy = (no.hx - no.e) * s6 - ldg_dev(g + P_HXMY * ps + rp + x, is);
    p.hxz = c.hx * s6 - ldg_dev(g + P_HXZ * ps + r + x, is);
    p.hypx = (w.hy - w.e) * s6 - ldg_dev(g + P_HYPX * ps + r + xm, is);
    p.hymx = (e.hy + e.e) * s6 - ldg_dev(g + P_HYMX * ps + r + xp, is);
    p.hypy = so.hy * s6 - ldg_dev(g + P_HYPY * ps + rm + x, is);
    p.hymy = no.hy * s6 - ldg_dev(g + P_HYMY * ps + rp + x, is);
    p.hyz = c.hy * s6 - ldg_dev(g + P_HYZ * ps + r + x, is);
    if (x == 0 && t1 >= 1 && a.src.kind != SRC_NONE) {
        double gs, inc;
        source_values(a.src, t1, &gs, &inc);
        if (a.src.kind == SRC_OPEN) {
            p.epx += (float)gs;
            p.hypx -= (float)gs;
        } else {
            p.epx = (float)inc;
            p.hxpx = 0.0f;
            p.hypx = (float)(-inc);
        }
    }
}

// Deviations from the new equilibrium, g_i = f_i - f_i^eq(F(t)), scaled.
__device__ __forceinline__ void deviations(const Pop<float> &p, float Ez, float Hx, float Hy, float em1,
                                           float g[NPLANES]) {
    const float s6 = 1.0f / 6.0f;
    g[P_E0] = p.e0 - em1 * Ez;
    g[P_EZ] = p.ez - Ez * s6;
    g[P_EPX] = p.epx - (Ez - Hy) * s6;
    g[P_EMX] = p.emx - (Ez + Hy) * s6;
    g[P_EPY] = p.epy - (Ez + Hx) * s6;
    g[P_EMY] = p.emy - (Ez - Hx) * s6;
    g[P_HXPX] = p.hxpx - Hx * s6;
    g[P_HXMX] = p.hxmx - Hx * s6;
    g[P_HXPY] = p.hxpy - (Hx + Ez) * s6;
    g[P_HXMY] = p.hxmy - (Hx - Ez) * s6;
    g[P_HXZ] = p.hxz - Hx * s6;
    g[P_HYPX] = p.hypx - (Hy - Ez) * s6;
    g[P_HYMX] = p.hymx - (Hy + Ez) * s6;
    g[P_HYPY] = p.hypy - Hy * s6;
    g[P_HYMY] = p.hymy - Hy * s6;
    g[P_HYZ] = p.hyz - Hy * s6;
}

cudaError_t launch_step_f16(const F16Args &a, const long long *t_in, long long *t_out, bool accumulate,
                            cudaStream_t s);
cudaError_t launch_fields_f16(const F16Args &a, const long long *t_dev, double *ez, double *hx, double *hy,
                              cudaStream_t s);

}  // namespace lbmem
