// FP16-deviation storage form of the fused stream-collide step (arXiv 2509.22308,
// Sec. III, Eq. LBGK equation), FP32 arithmetic.
//
// Stored per site for time t: the fields F = (E_z/3, H_x/3, H_y/3)(t) in FP32 and the
// 11 deviations g_i(t) = f_i(t) - f_i^eq(F(t)) in FP16, multiplied by 2^10.  Because
// the scheme's post-collision value is f*_i = 2 f_i^eq - f_i = f_i^eq - g_i, the pull
// for time t + 1 rebuilds f_i(r, t + 1) = f_i^eq(F(s, t)) - g_i(s, t) from the
// upstream site s = r - c_i; the deviations are small (of the order of the field
// change over one cell), so FP16 keeps about 11 bits of them.
// Bytes per lattice update: 11 x 2 + 3 x 4 (+1 material) read, 11 x 2 + 3 x 4 written.
#include <cuda_fp16.h>

#include "common.cuh"
#include "step_f16.cuh"

namespace lbmem {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ void accumulate_site(const F16Args &a, size_t idx, int y, long long t, double Ez,
                                                double Hx, double Hy) {
    if (y < a.accp.y0 || y > a.accp.y1) return;
    const int s = a.accp.slot[idx];
    if (s < 0) return;
    const double2 c = a.src.cs[(int)(t % (long long)a.src.period)];
    double *q = a.accp.acc + 6 * (size_t)s;
    q[0] += Ez * c.x;
    q[1] += Ez * c.y;
    q[2] += Hx * c.x;
    q[3] += Hx * c.y;
    q[4] += Hy * c.x;
    q[5] += Hy * c.y;
}

// Two sites (x0, x0 + 1), x0 even, per thread: the x-aligned planes, the fields of the
// pair and of its rows y -+ 1, the material ids and every store move as 2-element
// vectors; the +-x planes and the fields one site beyond the pair are single loads at
// the clamped upstream index.  A warp covers 64 sites of one row.
template <bool ACC>
__global__ void __launch_bounds__(BX *BY) k_step_f16(const F16Args a, const long long *__restrict__ t_in,
                                                     long long *__restrict__ t_out) {
    const int x0 = 2 * (blockIdx.x * BX + threadIdx.x);
    const int y = blockIdx.y * BY + threadIdx.y;
    const long long t = *t_in;
    if (x0 == 0 && y == 0) *t_out = t + 1;
    if (x0 >= a.nx || y >= a.ny) return;
    const bool has1 = x0 + 1 < a.nx;
    const size_t ps = a.pstride;
    const size_t r = (size_t)y * a.pitch;
    const size_t rm = (size_t)(y > 0 ? y - 1 : 0) * a.pitch;
    const size_t rp = (size_t)(y < a.ny - 1 ? y + 1 : y) * a.pitch;
    const int xw = x0 > 0 ? x0 - 1 : 0;                   // +x upstream of site 0
    const int xe = x0 + 2 < a.nx ? x0 + 2 : a.nx - 1;      // -x upstream of site 1
    const float is = a.inv_scale;
    const __half *g = a.g;

    // fields at time t - 1 of the pair, of its rows y -+ 1 and of the sites x0 - 1, x0 + 2
    const float2 Ec = *(const float2 *)(a.fe + r + x0), Xc = *(const float2 *)(a.fhx + r + x0),
                 Yc = *(const float2 *)(a.fhy + r + x0);
    const float2 Es = *(const float2 *)(a.fe + rm + x0), Xs = *(const float2 *)(a.fhx + rm + x0),
                 Ys = *(const float2 *)(a.fhy + rm + x0);
    const float2 En = *(const float2 *)(a.fe + rp + x0), Xn = *(const float2 *)(a.fhx + rp + x0),
                 Yn = *(const float2 *)(a.fhy + rp + x0);
    const float Ew = a.fe[r + xw], Xw = a.fhx[r + xw], Yw = a.fhy[r + xw];
    const float Ee = a.fe[r + xe], Xe = a.fhx[r + xe], Ye = a.fhy[r + xe];
    // -x upstream of site 0 is x0 + 1 (clamped to x0 at the last column)
    const float E0e = has1 ? Ec.y : Ec.x, X0e = has1 ? Xc.y : Xc.x, Y0e = has1 ? Yc.y : Yc.x;

    auto h2 = [&](int plane, size_t row) { return *(const __half2 *)(g + plane * ps + row + x0); };
    auto h1 = [&](int plane, size_t row, int x) { return g[plane * ps + row + x]; };

    const uchar2 id = *(const uchar2 *)(a.mat + r + x0);
    const MatT<float> m0 = a.mtab[id.x], m1 = a.mtab[id.y];

    Pop<float> p0, p1;
    __half2 v;
    v = h2(P_EZ, r);
    p0.ez = rebuild(Ec.x, __low2half(v), is);
    p1.ez = rebuild(Ec.y, __high2half(v), is);
    v = h2(P_EPX, r);
    p0.epx = rebuild(eq2_epx(Ew, Xw, Yw), h1(P_EPX, r, xw), is);
    p1.epx = rebuild(eq2_epx(Ec.x, Xc.x, Yc.x), __low2half(v), is);
    v = h2(P_EMX, r);
    p0.emx = rebuild(eq2_emx(E0e, X0e, Y0e), has1 ? __high2half(v) : __low2half(v), is);
    p1.emx = rebuild(eq2_emx(Ee, Xe, Ye), h1(P_EMX, r, xe), is);
    v = h2(P_EPY, rm);
    p0.epy = rebuild(eq2_epy(Es.x, Xs.x, Ys.x), __low2half(v), is);
    p1.epy = rebuild(eq2_epy(Es.y, Xs.y, Ys.y), __high2half(v), is);
    v = h2(P_EMY, rp);
    p0.emy = rebuild(eq2_emy(En.x, Xn.x, Yn.x), __low2half(v), is);
    p1.emy = rebuild(eq2_emy(En.y, Xn.y, Yn.y), __high2half(v), is);
    v = h2(P_HXPX, r);
    p0.hxpx = rebuild(Xw, h1(P_HXPX, r, xw), is);
    p1.hxpx = rebuild(Xc.x, __low2half(v), is);
    v = h2(P_HXMX, r);
    p0.hxmx = rebuild(X0e, has1 ? __high2half(v) : __low2half(v), is);
    p1.hxmx = rebuild(Xe, h1(P_HXMX, r, xe), is);
    v = h2(P_HXZ, r);
    p0.hxz = rebuild(Xc.x, __low2half(v), is);
    p1.hxz = rebuild(Xc.y, __high2half(v), is);
    v = h2(P_HYPY, rm);
    p0.hypy = rebuild(Ys.x, __low2half(v), is);
    p1.hypy = rebuild(Ys.y, __high2half(v), is);
    v = h2(P_HYMY, rp);
    p0.hymy = rebuild(Yn.x, __low2half(v), is);
    p1.hymy = rebuild(Yn.y, __high2half(v), is);
    v = h2(P_HYZ, r);
    p0.hyz = rebuild(Yc.x, __low2half(v), is);
    p1.hyz = rebuild(Yc.y, __high2half(v), is);
    f16_source(a.src, x0, t, p0);

    float E30, Hx0, Hy0, D0, E31, Hx1, Hy1, D1;
    moments(p0, m0, &E30, &Hx0, &Hy0, &D0);
    moments(p1, m1, &E31, &Hx1, &Hy1, &D1);
    if (field_runaway(E30, a.runaway) || (has1 && field_runaway(E31, a.runaway))) atomicOr(a.err, 1u);
    const size_t idx = r + x0;
    if (ACC) {
        accumulate_site(a, idx, y, t, 3.0 * (double)E30, Hx0, Hy0);
        if (has1) accumulate_site(a, idx + 1, y, t, 3.0 * (double)E31, Hx1, Hy1);
    }
    const Fld F0 = stored_fields(E30, Hx0, Hy0), F1 = stored_fields(E31, Hx1, Hy1);
    __half g0[NPLANES], g1[NPLANES];
    encode_all(p0, F0, a.scale, g0);
    encode_all(p1, F1, a.scale, g1);
#pragma unroll
    for (int q = 0; q < NPLANES; ++q) *(__half2 *)(a.g_out + q * ps + idx) = __halves2half2(g0[q], g1[q]);
    *(float2 *)(a.fe_out + idx) = make_float2(F0.e, F1.e);
    *(float2 *)(a.fhx_out + idx) = make_float2(F0.hx, F1.hx);
    *(float2 *)(a.fhy_out + idx) = make_float2(F0.hy, F1.hy);
}

__global__ void __launch_bounds__(BX *BY) k_fields_f16(const F16Args a, const long long *__restrict__ t_dev,
                                                       double *ez, double *hx, double *hy) {
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const size_t idx = (size_t)y * a.pitch + x;
    const MatT<float> m = a.mtab[a.mat[idx]];
    Pop<float> p;
    pull_f16(a, x, y, *t_dev, p);
    float E3, Hx, Hy, D;
    moments(p, m, &E3, &Hx, &Hy, &D);
    const size_t o = (size_t)y * a.nx + x;
    ez[o] = 3.0 * (double)E3;
    hx[o] = (double)Hx;
    hy[o] = (double)Hy;
}

// Total electromagnetic energy (eps E_z^2 + H_x^2 + H_y^2) / 2 summed over sites.
__global__ void __launch_bounds__(BX *BY) k_energy_f16(const F16Args a, const long long *__restrict__ t_dev,
                                                       double *energy) {
    __shared__ double sh[32];
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    double w = 0.0;
    if (x < a.nx && y < a.ny) {
        const MatT<float> m = a.mtab[a.mat[(size_t)y * a.pitch + x]];
        Pop<float> p;
        pull_f16(a, x, y, *t_dev, p);
        float E3, Hx, Hy, D;
        moments(p, m, &E3, &Hx, &Hy, &D);
        w = 0.5 * ((double)D * (3.0 * (double)E3) + (double)Hx * (double)Hx + (double)Hy * (double)Hy);
    }
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    const int tid = threadIdx.y * BX + threadIdx.x;
    if ((tid & 31) == 0) sh[tid >> 5] = w;
    __syncthreads();
    if (tid < 32) {
        w = tid < (BX * BY) / 32 ? sh[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if (tid == 0) atomicAdd(energy, w);
    }
}

cudaError_t launch_energy_f16(const F16Args &a, const long long *t_dev, double *energy, cudaStream_t s) {
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY), block(BX, BY);
    k_energy_f16<<<grid, block, 0, s>>>(a, t_dev, energy);
    return cudaGetLastError();
}

cudaError_t launch_step_f16(const F16Args &a, const long long *t_in, long long *t_out, bool accumulate,
                            cudaStream_t s) {
    dim3 grid((a.nx + 2 * BX - 1) / (2 * BX), (a.ny + BY - 1) / BY), block(BX, BY);
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
