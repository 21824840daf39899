// Fused stream-collide step of the D3Q7 Maxwell lattice Boltzmann scheme
// (arXiv 2509.22308, Sec. III) for the FP64 and FP32 storage forms and both
// polarizations, plus the kernel that reconstructs the fields at the current time.
#include "common.cuh"
#include "launchers.h"

namespace lbmem {

constexpr int BX = 32, BY = 8;

// One thread per site; a warp covers 32 consecutive x of one row, so each of the 11
// plane reads and writes is a contiguous 128-byte (FP32) / 256-byte (FP64) segment,
// shifted by one element for the +-x planes.  No population is read twice.
// POL selects TM^z (the paper's case) or TE^z; both keep 11 planes (common.cuh).
template <typename T, bool ACC, int POL>
__global__ void __launch_bounds__(BX *BY) k_step(const StepArgs<T> a, const T *__restrict__ fin,
                                                 T *__restrict__ fout, const long long *__restrict__ t_in,
                                                 long long *__restrict__ t_out) {
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    const long long t = *t_in;
    if (x == 0 && y == 0) *t_out = t + 1;
    if (x >= a.nx || y >= a.ny) return;

    Pop<T> p;
    pull_site(a, fin, x, y, t, p);
    const size_t idx = (size_t)y * a.pitch + x;
    const MatT<T> m = a.mtab[a.mat[idx]];
    const bool acc = ACC && y >= a.accp.y0 && y <= a.accp.y1 && a.accp.slot[idx] >= 0;
    double f3[3];
    if (update_site<POL, true>(p, m, a.runaway, acc ? f3 : nullptr, nullptr)) atomicOr(a.err, 1u);
    if (acc) {
        const double2 c = a.src.cs[(int)(t % (long long)a.src.period)];
        double *q = a.accp.acc + 6 * (size_t)a.accp.slot[idx];
        q[0] += f3[0] * c.x;
        q[1] += f3[0] * c.y;
        q[2] += f3[1] * c.x;
        q[3] += f3[1] * c.y;
        q[4] += f3[2] * c.x;
        q[5] += f3[2] * c.y;
    }
    store_site(fout, a.pstride, idx, p);
}

// The field triple at time *t_dev (pull + moments, no collision), packed [ny][nx]:
// TM E_z, H_x, H_y; TE H_z, E_x, E_y.
template <typename T, int POL>
__global__ void __launch_bounds__(BX *BY) k_fields(const StepArgs<T> a, const T *__restrict__ f,
                                                   const long long *__restrict__ t_dev, double *o0,
                                                   double *o1, double *o2) {
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    Pop<T> p;
    pull_site(a, f, x, y, *t_dev, p);
    const size_t idx = (size_t)y * a.pitch + x;
    double f3[3];
    update_site<POL, false>(p, a.mtab[a.mat[idx]], a.runaway, f3, nullptr);
    const size_t o = (size_t)y * a.nx + x;
    o0[o] = f3[0];
    o1[o] = f3[1];
    o2[o] = f3[2];
}

template <typename T>
cudaError_t launch_step(const StepArgs<T> &a, const T *fin, T *fout, const long long *t_in,
                        long long *t_out, bool accumulate, cudaStream_t s) {
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY), block(BX, BY);
    if (a.pol == POL_TE) {
        if (accumulate)
            k_step<T, true, POL_TE><<<grid, block, 0, s>>>(a, fin, fout, t_in, t_out);
        else
            k_step<T, false, POL_TE><<<grid, block, 0, s>>>(a, fin, fout, t_in, t_out);
    } else {
        if (accumulate)
            k_step<T, true, POL_TM><<<grid, block, 0, s>>>(a, fin, fout, t_in, t_out);
        else
            k_step<T, false, POL_TM><<<grid, block, 0, s>>>(a, fin, fout, t_in, t_out);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fields(const StepArgs<T> &a, const T *f, const long long *t_dev, double *ez,
                          double *hx, double *hy, cudaStream_t s) {
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY), block(BX, BY);
    if (a.pol == POL_TE)
        k_fields<T, POL_TE><<<grid, block, 0, s>>>(a, f, t_dev, ez, hx, hy);
    else
        k_fields<T, POL_TM><<<grid, block, 0, s>>>(a, f, t_dev, ez, hx, hy);
    return cudaGetLastError();
}

template cudaError_t launch_step<double>(const StepArgs<double> &, const double *, double *,
                                         const long long *, long long *, bool, cudaStream_t);
template cudaError_t launch_step<float>(const StepArgs<float> &, const float *, float *,
                                        const long long *, long long *, bool, cudaStream_t);
template cudaError_t launch_fields<double>(const StepArgs<double> &, const double *, const long long *,
                                           double *, double *, double *, cudaStream_t);
template cudaError_t launch_fields<float>(const StepArgs<float> &, const float *, const long long *,
                                          double *, double *, double *, cudaStream_t);

template cudaError_t launch_step<df>(const StepArgs<df> &, const df *, df *, const long long *, long long *, bool,
                                     cudaStream_t);
template cudaError_t launch_fields<df>(const StepArgs<df> &, const df *, const long long *, double *, double *,
                                       double *, cudaStream_t);

}  // namespace lbmem
