// Fused stream-collide step of the D3Q7 Maxwell lattice Boltzmann scheme
// (arXiv 2509.22308, Sec. III) for the FP64 and FP32 storage forms, plus the
// kernel that reconstructs the fields at the current time.
#include "common.cuh"
#include "launchers.h"

namespace lbmem {

constexpr int BX = 32, BY = 8;

// One thread per site; a warp covers 32 consecutive x of one row, so each of the 16
// plane reads and writes is a contiguous 128-byte (FP32) / 256-byte (FP64) segment,
// shifted by one element for the +-x planes.  No population is read twice.
template <typename T, bool ACC>
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
    T E3, Hx, Hy, D;
    moments(p, m, &E3, &Hx, &Hy, &D);
    if (field_runaway(E3)) atomicOr(a.err, 1u);
    if (ACC) {
        if (y >= a.accp.y0 && y <= a.accp.y1) {
            const int s = a.accp.slot[idx];
            if (s >= 0) {
                const double2 c = a.src.cs[(int)(t % (long long)a.src.period)];
                const double ez = (double)(D * m.inv_eps), hx = (double)Hx, hy = (double)Hy;
                double *q = a.accp.acc + 6 * (size_t)s;
                q[0] += ez * c.x;
                q[1] += ez * c.y;
                q[2] += hx * c.x;
                q[3] += hx * c.y;
                q[4] += hy * c.x;
                q[5] += hy * c.y;
            }
        }
    }
    collide(p, E3, Hx, Hy);
    store_site(fout, a.pstride, idx, p);
}

// Fields E_z, H_x, H_y at time *t_dev (pull + moments, no collision), packed [ny][nx].
template <typename T>
__global__ void __launch_bounds__(BX *BY) k_fields(const StepArgs<T> a, const T *__restrict__ f,
                                                   const long long *__restrict__ t_dev, double *ez,
                                                   double *hx, double *hy) {
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    Pop<T> p;
    pull_site(a, f, x, y, *t_dev, p);
    const size_t idx = (size_t)y * a.pitch + x;
    const MatT<T> m = a.mtab[a.mat[idx]];
    T E3, Hx, Hy, D;
    moments(p, m, &E3, &Hx, &Hy, &D);
    const size_t o = (size_t)y * a.nx + x;
    ez[o] = (double)(D * m.inv_eps);
    hx[o] = (double)Hx;
    hy[o] = (double)Hy;
}

template <typename T>
cudaError_t launch_step(const StepArgs<T> &a, const T *fin, T *fout, const long long *t_in,
                        long long *t_out, bool accumulate, cudaStream_t s) {
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY), block(BX, BY);
    if (accumulate)
        k_step<T, true><<<grid, block, 0, s>>>(a, fin, fout, t_in, t_out);
    else
        k_step<T, false><<<grid, block, 0, s>>>(a, fin, fout, t_in, t_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fields(const StepArgs<T> &a, const T *f, const long long *t_dev, double *ez,
                          double *hx, double *hy, cudaStream_t s) {
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY), block(BX, BY);
    k_fields<T><<<grid, block, 0, s>>>(a, f, t_dev, ez, hx, hy);
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

}  // namespace lbmem
