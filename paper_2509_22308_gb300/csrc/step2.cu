// Two time steps per launch for the HBM-bound storage forms (FP32, FP16-deviation):
// temporal blocking of the fused stream-collide step (arXiv 2509.22308, Sec. III).
//
// A CTA owns a TW x TH tile.  Phase 1 computes the post-collision f*(t) of the tile and
// a one-site halo (pulled from global memory exactly as the one-step kernel does) into
// shared memory; phase 2 pulls f(t + 1) of the tile from shared memory, collides and
// writes f*(t + 1) (FP32) or the fields and deviations of t + 1 (FP16-deviation) to
// global memory.  Each state element crosses HBM once per two steps (plus the halo,
// which neighbouring CTAs read at about the same time and L2 serves); the per-site
// arithmetic is the one-step kernel's, so the FP32 result is bit-identical to two
// one-step launches.  The FP16-deviation form keeps the intermediate f*(t) in FP32,
// so only every second state is rounded to FP16.
#include <cuda_fp16.h>

#include "common.cuh"
#include "step2.cuh"
#include "step_f16.cuh"

namespace lbmem {

constexpr int TW = 64, TH = 14, SW = TW + 2, SH = TH + 2, NT = 256;
constexpr size_t kStep2Smem = (size_t)NPLANES * SH * SW * sizeof(float);

__device__ __forceinline__ float &smv(float *sm, int plane, int ly, int lx) {
    return sm[(plane * SH + ly) * SW + lx];
}

__device__ __forceinline__ void put_smem(float *sm, int ly, int lx, const Pop<float> &p) {
    smv(sm, P_E0, ly, lx) = p.e0;
    smv(sm, P_EZ, ly, lx) = p.ez;
    smv(sm, P_EPX, ly, lx) = p.epx;
    smv(sm, P_EMX, ly, lx) = p.emx;
    smv(sm, P_EPY, ly, lx) = p.epy;
    smv(sm, P_EMY, ly, lx) = p.emy;
    smv(sm, P_HXPX, ly, lx) = p.hxpx;
    smv(sm, P_HXMX, ly, lx) = p.hxmx;
    smv(sm, P_HXPY, ly, lx) = p.hxpy;
    smv(sm, P_HXMY, ly, lx) = p.hxmy;
    smv(sm, P_HXZ, ly, lx) = p.hxz;
    smv(sm, P_HYPX, ly, lx) = p.hypx;
    smv(sm, P_HYMX, ly, lx) = p.hymx;
    smv(sm, P_HYPY, ly, lx) = p.hypy;
    smv(sm, P_HYMY, ly, lx) = p.hymy;
    smv(sm, P_HYZ, ly, lx) = p.hyz;
}

// f_i(r, t + 1) from the shared-memory f*(t); (cx, cy) is the site's cell in the tile
// with halo, the upstream cell is clamped at the lattice edge exactly as pull_site does.
__device__ __forceinline__ void pull_smem(float *sm, const SourceParams &src, int nx, int ny, int x, int y,
                                          int cx, int cy, long long t1, Pop<float> &p) {
    const int xm = x > 0 ? cx - 1 : cx, xp = x < nx - 1 ? cx + 1 : cx;
    const int ym = y > 0 ? cy - 1 : cy, yp = y < ny - 1 ? cy + 1 : cy;
    p.e0 = smv(sm, P_E0, cy, cx);
    p.ez = smv(sm, P_EZ, cy, cx);
    p.epx = smv(sm, P_EPX, cy, xm);
    p.emx = smv(sm, P_EMX, cy, xp);
    p.epy = smv(sm, P_EPY, ym, cx);
    p.emy = smv(sm, P_EMY, yp, cx);
    p.hxpx = smv(sm, P_HXPX, cy, xm);
    p.hxmx = smv(sm, P_HXMX, cy, xp);
    p.hxpy = smv(sm, P_HXPY, ym, cx);
    p.hxmy = smv(sm, P_HXMY, yp, cx);
    p.hxz = smv(sm, P_HXZ, cy, cx);
    p.hypx = smv(sm, P_HYPX, cy, xm);
    p.hymx = smv(sm, P_HYMX, cy, xp);
    p.hypy = smv(sm, P_HYPY, ym, cx);
    p.hymy = smv(sm, P_HYMY, yp, cx);
    p.hyz = smv(sm, P_HYZ, cy, cx);
    if (x == 0 && t1 >= 1 && src.kind != SRC_NONE) {
        double g, inc;
        source_values(src, t1, &g, &inc);
        if (src.kind == SRC_OPEN) {
            p.epx += (float)g;
            p.hypx -= (float)g;
        } else {
            p.epx = (float)inc;
            p.hxpx = 0.0f;
            p.hypx = (float)(-inc);
        }
    }
}

__device__ __forceinline__ void acc_site(const AccParams &ap, const SourceParams &src, size_t idx, int y,
                                         long long t, double ez, double hx, double hy) {
    if (y < ap.y0 || y > ap.y1) return;
    const int s = ap.slot[idx];
    if (s < 0) return;
    const double2 c = src.cs[(int)(t % (long long)src.period)];
    double *q = ap.acc + 6 * (size_t)s;
    q[0] += ez * c.x;
    q[1] += ez * c.y;
    q[2] += hx * c.x;
    q[3] += hx * c.y;
    q[4] += hy * c.x;
    q[5] += hy * c.y;
}

template <bool ACC>
__global__ void __launch_bounds__(NT) k_step2_f32(const StepArgs<float> a, const float *__restrict__ fin,
                                                  float *__restrict__ fout, const long long *__restrict__ t_in,
                                                  long long *__restrict__ t_out) {
    extern __shared__ float sm[];
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const long long t = *t_in;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *t_out = t + 2;
    for (int k = threadIdx.x; k < SW * SH; k += NT) {
        const int lx = k % SW, ly = k / SW, x = x0 - 1 + lx, y = y0 - 1 + ly;
        if (x < 0 || x >= a.nx || y < 0 || y >= a.ny) continue;
        Pop<float> p;
        pull_site(a, fin, x, y, t, p);
        const size_t idx = (size_t)y * a.pitch + x;
        const MatT<float> m = a.mtab[a.mat[idx]];
        float E3, Hx, Hy, D;
        moments(p, m.inv_eps3, &E3, &Hx, &Hy, &D);
        if (field_runaway(E3)) atomicOr(a.err, 1u);
        if (ACC && lx >= 1 && lx <= TW && ly >= 1 && ly <= TH)
            acc_site(a.accp, a.src, idx, y, t, (double)(D * m.inv_eps), (double)Hx, (double)Hy);
        collide(p, E3, Hx, Hy, m.six_em1);
        put_smem(sm, ly, lx, p);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < TW * TH; k += NT) {
        const int lx = k % TW, ly = k / TW, x = x0 + lx, y = y0 + ly;
        if (x >= a.nx || y >= a.ny) continue;
        Pop<float> p;
        pull_smem(sm, a.src, a.nx, a.ny, x, y, lx + 1, ly + 1, t + 1, p);
        const size_t idx = (size_t)y * a.pitch + x;
        const MatT<float> m = a.mtab[a.mat[idx]];
        float E3, Hx, Hy, D;
        moments(p, m.inv_eps3, &E3, &Hx, &Hy, &D);
        if (field_runaway(E3)) atomicOr(a.err, 1u);
        if (ACC) acc_site(a.accp, a.src, idx, y, t + 1, (double)(D * m.inv_eps), (double)Hx, (double)Hy);
        collide(p, E3, Hx, Hy, m.six_em1);
        store_site(fout, a.pstride, idx, p);
    }
}

template <bool ACC>
__global__ void __launch_bounds__(NT) k_step2_f16(const F16Args a, const long long *__restrict__ t_in,
                                                  long long *__restrict__ t_out) {
    extern __shared__ float sm[];
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const long long t = *t_in;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *t_out = t + 2;
    for (int k = threadIdx.x; k < SW * SH; k += NT) {
        const int lx = k % SW, ly = k / SW, x = x0 - 1 + lx, y = y0 - 1 + ly;
        if (x < 0 || x >= a.nx || y < 0 || y >= a.ny) continue;
        const size_t idx = (size_t)y * a.pitch + x;
        const MatT<float> m = a.mtab[a.mat[idx]];
        Pop<float> p;
        pull_f16(a, x, y, t, p, m.six_em1 * (1.0f / 6.0f));
        float E3, Hx, Hy, D;
        moments(p, m.inv_eps3, &E3, &Hx, &Hy, &D);
        if (field_runaway(E3)) atomicOr(a.err, 1u);
        if (ACC && lx >= 1 && lx <= TW && ly >= 1 && ly <= TH)
            acc_site(a.accp, a.src, idx, y, t, (double)(3.0f * E3), (double)Hx, (double)Hy);
        collide(p, E3, Hx, Hy, m.six_em1);
        put_smem(sm, ly, lx, p);
    }
    __syncthreads();
    const float sc = a.scale, s6 = 1.0f / 6.0f;
    const size_t ps = a.pstride;
    for (int k = threadIdx.x; k < TW * TH; k += NT) {
        const int lx = k % TW, ly = k / TW, x = x0 + lx, y = y0 + ly;
        if (x >= a.nx || y >= a.ny) continue;
        Pop<float> p;
        pull_smem(sm, a.src, a.nx, a.ny, x, y, lx + 1, ly + 1, t + 1, p);
        const size_t idx = (size_t)y * a.pitch + x;
        const MatT<float> m = a.mtab[a.mat[idx]];
        float E3, Hx, Hy, D;
        moments(p, m.inv_eps3, &E3, &Hx, &Hy, &D);
        if (field_runaway(E3)) atomicOr(a.err, 1u);
        const float Ez = 3.0f * E3, em1 = m.six_em1 * s6;
        if (ACC) acc_site(a.accp, a.src, idx, y, t + 1, (double)Ez, (double)Hx, (double)Hy);
        float g[NPLANES];
        deviations(p, Ez, Hx, Hy, em1, g);
#pragma unroll
        for (int q = 0; q < NPLANES; ++q) a.g_out[q * ps + idx] = __float2half_rn(g[q] * sc);
        a.fe_out[idx] = Ez;
        a.fhx_out[idx] = Hx;
        a.fhy_out[idx] = Hy;
    }
}

cudaError_t step2_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_step2_f32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStep2Smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step2_f32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStep2Smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step2_f16<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStep2Smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step2_f16<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStep2Smem);
    return e;
}

cudaError_t launch_step2_f32(const StepArgs<float> &a, const float *fin, float *fout, const long long *t_in,
                             long long *t_out, bool accumulate, cudaStream_t s) {
    dim3 grid((a.nx + TW - 1) / TW, (a.ny + TH - 1) / TH), block(NT);
    if (accumulate)
        k_step2_f32<true><<<grid, block, kStep2Smem, s>>>(a, fin, fout, t_in, t_out);
    else
        k_step2_f32<false><<<grid, block, kStep2Smem, s>>>(a, fin, fout, t_in, t_out);
    return cudaGetLastError();
}

cudaError_t launch_step2_f16(const F16Args &a, const long long *t_in, long long *t_out, bool accumulate,
                             cudaStream_t s) {
    dim3 grid((a.nx + TW - 1) / TW, (a.ny + TH - 1) / TH), block(NT);
    if (accumulate)
        k_step2_f16<true><<<grid, block, kStep2Smem, s>>>(a, t_in, t_out);
    else
        k_step2_f16<false><<<grid, block, kStep2Smem, s>>>(a, t_in, t_out);
    return cudaGetLastError();
}

}  // namespace lbmem
