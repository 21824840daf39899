// FP16-deviation storage form of the fused stream-collide step (arXiv 2509.22308,
// Sec. III, Eq. LBGK equation), FP32 arithmetic.
//
// Stored per site for time t: the fields F = (E_z, H_x, H_y)(t) in FP32 and the 16
// deviations g_i(t) = f_i(t) - f_i^eq(F(t)) in FP16, multiplied by 2^10.  Because
// the scheme's post-collision value is f*_i = 2 f_i^eq - f_i = f_i^eq - g_i, the pull
// for time t + 1 rebuilds f_i(r, t + 1) = f_i^eq(F(s, t)) - g_i(s, t) from the
// upstream site s = r - c_i; the deviations are small (of the order of the field
// change over one cell), so FP16 keeps about 11 bits of them.
// Bytes per lattice update: 16 x 2 + 3 x 4 (+1 material) read, 16 x 2 + 3 x 4 written.
#include <cuda_fp16.h>

#include "common.cuh"
#include "step_f16.cuh"

namespace lbmem {

constexpr int BX = 32, BY = 8;

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

__device__ __forceinline__ void st_dev(__half *p, float v, float scale) { *p = __float2half_rn(v * scale); }

template <bool ACC>
__global__ void __launch_bounds__(BX *BY) k_step_f16(const F16Args a, const long long *__restrict__ t_in,
                                                     long long *__restrict__ t_out) {
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    const long long t = *t_in;
    if (x == 0 && y == 0) *t_out = t + 1;
    if (x >= a.nx || y >= a.ny) return;
    const size_t idx = (size_t)y * a.pitch + x;
    const MatT<float> m = a.mtab[a.mat[idx]];
    const float em1 = m.six_em1 * (1.0f / 6.0f);
    Pop<float> p;
    pull_f16(a, x, y, t, p, em1);
    float E3, Hx, Hy, D;
    moments(p, m.inv_eps3, &E3, &Hx, &Hy, &D);
    if (field_runaway(E3)) atomicOr(a.err, 1u);
    const float Ez = 3.0f * E3;
    if (ACC) {
        if (y >= a.accp.y0 && y <= a.accp.y1) {
            const int s = a.accp.slot[idx];
            if (s >= 0) {
                const double2 c = a.src.cs[(int)(t % (long long)a.src.period)];
                double *q = a.accp.acc + 6 * (size_t)s;
                q[0] += (double)Ez * c.x;
                q[1] += (double)Ez * c.y;
                q[2] += (double)Hx * c.x;
                q[3] += (double)Hx * c.y;
                q[4] += (double)Hy * c.x;
                q[5] += (double)Hy * c.y;
            }
        }
    }
    // deviations from the new equilibrium, g_i = f_i - f_i^eq(F(t))
    const float s6 = 1.0f / 6.0f, sc = a.scale;
    const size_t ps = a.pstride;
    __half *go = a.g_out;
    st_dev(go + P_E0 * ps + idx, p.e0 - em1 * Ez, sc);
    st_dev(go + P_EZ * ps + idx, p.ez - Ez * s6, sc);
    st_dev(go + P_EPX * ps + idx, p.epx - (Ez - Hy) * s6, sc);
    st_dev(go + P_EMX * ps + idx, p.emx - (Ez + Hy) * s6, sc);
    st_dev(go + P_EPY * ps + idx, p.epy - (Ez + Hx) * s6, sc);
    st_dev(go + P_EMY * ps + idx, p.emy - (Ez - Hx) * s6, sc);
    st_dev(go + P_HXPX * ps + idx, p.hxpx - Hx * s6, sc);
    st_dev(go + P_HXMX * ps + idx, p.hxmx - Hx * s6, sc);
    st_dev(go + P_HXPY * ps + idx, p.hxpy - (Hx + Ez) * s6, sc);
    st_dev(go + P_HXMY * ps + idx, p.hxmy - (Hx - Ez) * s6, sc);
    st_dev(go + P_HXZ * ps + idx, p.hxz - Hx * s6, sc);
    st_dev(go + P_HYPX * ps + idx, p.hypx - (Hy - Ez) * s6, sc);
    st_dev(go + P_HYMX * ps + idx, p.hymx - (Hy + Ez) * s6, sc);
    st_dev(go + P_HYPY * ps + idx, p.hypy - Hy * s6, sc);
    st_dev(go + P_HYMY * ps + idx, p.hymy - Hy * s6, sc);
    st_dev(go + P_HYZ * ps + idx, p.hyz - Hy * s6, sc);
    a.fe_out[idx] = Ez;
    a.fhx_out[idx] = Hx;
    a.fhy_out[idx] = Hy;
}

__global__ void __launch_bounds__(BX *BY) k_fields_f16(const F16Args a, const long long *__restrict__ t_dev,
                                                       double *ez, double *hx, double *hy) {
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const size_t idx = (size_t)y * a.pitch + x;
    const MatT<float> m = a.mtab[a.mat[idx]];
    Pop<float> p;
    pull_f16(a, x, y, *t_dev, p, m.six_em1 * (1.0f / 6.0f));
    float E3, Hx, Hy, D;
    moments(p, m.inv_eps3, &E3, &Hx, &Hy, &D);
    const size_t o = (size_t)y * a.nx + x;
    ez[o] = (double)(3.0f * E3);
    hx[o] = (double)Hx;
    hy[o] = (double)Hy;
}

cudaError_t launch_step_f16(const F16Args &a, const long long *t_in, long long *t_out, bool accumulate,
                            cudaStream_t s) {
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY), block(BX, BY);
    if (accumulate)
        k_step_f16<true><<<grid, block, 0, s>>>(a, t_in, t_out);
    else
        k_step_f16<false><<<grid, block, 0, s>>>(a, t_in, t_out);
    return cudaGetLastError();
}

cudaError_t launch_fields_f16(const F16Args &a, const long long *t_dev, double *ez, double *hx, double *hy,
                              cudaStream_t s) {
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY), block(BX, BY);
    k_fields_f16<<<grid, block, 0, s>>>(a, t_dev, ez, hx, hy);
    return cudaGetLastError();
}

}  // namespace lbmem
