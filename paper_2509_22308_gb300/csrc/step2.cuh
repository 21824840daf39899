// The double-float two-steps-per-launch kernel's tile and launcher (step2.cu), and the
// helpers every temporally blocked kernel shares: the source values of a launch and the
// Fourier accumulation of one site.
#pragma once

#include "common.cuh"
#include "step_f16.cuh"

namespace lbmem {

// Tile of the double-float two-step kernel: TW x TH sites with a one-site halo in shared
// memory (11 planes of SW x SH double-float values: 93 KB, 2 CTAs per SM).
constexpr int TW = 64, TH = 14, SW = TW + 2, SH = TH + 2, NT = 256;
template <typename T>
constexpr size_t step2_smem() { return (size_t)NPLANES * SH * SW * sizeof(T); }

template <typename T>
__device__ __forceinline__ T &smv(T *sm, int plane, int ly, int lx) {
    return sm[(plane * SH + ly) * SW + lx];
}

template <typename T>
__device__ __forceinline__ void put_smem(T *sm, int ly, int lx, const Pop<T> &p) {
    smv(sm, P_EZ, ly, lx) = p.ez;
    smv(sm, P_EPX, ly, lx) = p.epx;
    smv(sm, P_EMX, ly, lx) = p.emx;
    smv(sm, P_EPY, ly, lx) = p.epy;
    smv(sm, P_EMY, ly, lx) = p.emy;
    smv(sm, P_HXPX, ly, lx) = p.hxpx;
    smv(sm, P_HXMX, ly, lx) = p.hxmx;
    smv(sm, P_HXZ, ly, lx) = p.hxz;
    smv(sm, P_HYPY, ly, lx) = p.hypy;
    smv(sm, P_HYMY, ly, lx) = p.hymy;
    smv(sm, P_HYZ, ly, lx) = p.hyz;
}

// f_i(r, t + 1) from the shared-memory f*(t); (cx, cy) is the site's cell in the tile
// with halo, the upstream cell is clamped at the lattice edge exactly as pull_site does.
template <typename T>
__device__ __forceinline__ void pull_smem(T *sm, int nx, int ny, int x, int y, int cx, int cy, Pop<T> &p) {
    const int xm = x > 0 ? cx - 1 : cx, xp = x < nx - 1 ? cx + 1 : cx;
    const int ym = y > 0 ? cy - 1 : cy, yp = y < ny - 1 ? cy + 1 : cy;
    p.ez = smv(sm, P_EZ, cy, cx);
    p.epx = smv(sm, P_EPX, cy, xm);
    p.emx = smv(sm, P_EMX, cy, xp);
    p.epy = smv(sm, P_EPY, ym, cx);
    p.emy = smv(sm, P_EMY, yp, cx);
    p.hxpx = smv(sm, P_HXPX, cy, xm);
    p.hxmx = smv(sm, P_HXMX, cy, xp);
    p.hxz = smv(sm, P_HXZ, cy, cx);
    p.hypy = smv(sm, P_HYPY, ym, cx);
    p.hymy = smv(sm, P_HYMY, yp, cx);
    p.hyz = smv(sm, P_HYZ, cy, cx);
}

// Source values of the two times of a launch (t, t + 1), evaluated once per block by one
// thread of the blocks that own column 0 (see pull_site for why not per site).
struct SrcPair {
    double g0, inc0, g1, inc1;
};
__device__ __forceinline__ void source_pair(const SourceParams &src, int x0, long long t, SrcPair *sp) {
    if (threadIdx.x == 0) {
        SrcPair v{0.0, 0.0, 0.0, 0.0};
        if (x0 == 0 && src.kind != SRC_NONE) {
            if (t >= 1) source_values(src, t, &v.g0, &v.inc0);
            source_values(src, t + 1, &v.g1, &v.inc1);
        }
        *sp = v;
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

// Allow the kernels' dynamic shared memory (call once per device, outside stream capture).
cudaError_t step2_prepare();
template <typename T>
cudaError_t launch_step2(const StepArgs<T> &a, const T *fin, T *fout, const long long *t_in, long long *t_out,
                         bool accumulate, cudaStream_t s);

}  // namespace lbmem
