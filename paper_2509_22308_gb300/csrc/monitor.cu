// Convergence monitor: total electromagnetic energy of the lattice (arXiv 2509.22308,
// Sec. III: the energy in the domain approaches a constant at steady state).
#include "common.cuh"
#include "launchers.h"

namespace lbmem {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31, wid = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    v = (wid == 0 && lane < nw) ? sh[lane] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Total electromagnetic energy sum over sites of (D . E + H . H) / 2 at time *t_dev (the
// convergence monitor of Sec. III), accumulated into *energy (FP64); TM D.E = eps E_z^2,
// TE D.E = eps (E_x^2 + E_y^2).
template <typename T, int POL>
__global__ void __launch_bounds__(BX *BY) k_energy(const StepArgs<T> a, const T *__restrict__ f,
                                                   const long long *__restrict__ t_dev, double *energy) {
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    double w = 0.0;
    if (x < a.nx && y < a.ny) {
        Pop<T> p;
        pull_site(a, f, x, y, *t_dev, p);
        update_site<POL, false>(p, a.mtab[a.mat[(size_t)y * a.pitch + x]], a.runaway, nullptr, &w);
    }
    w = block_sum(w);
    if (threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(energy, w);
}

template <typename T>
cudaError_t launch_energy(const StepArgs<T> &a, const T *f, const long long *t_dev, double *energy, cudaStream_t s) {
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY), block(BX, BY);
    if (a.pol == POL_TE)
        k_energy<T, POL_TE><<<grid, block, 0, s>>>(a, f, t_dev, energy);
    else
        k_energy<T, POL_TM><<<grid, block, 0, s>>>(a, f, t_dev, energy);
    return cudaGetLastError();
}
template cudaError_t launch_energy<double>(const StepArgs<double> &, const double *, const long long *, double *,
                                           cudaStream_t);
template cudaError_t launch_energy<float>(const StepArgs<float> &, const float *, const long long *, double *,
                                          cudaStream_t);

template cudaError_t launch_energy<df>(const StepArgs<df> &, const df *, const long long *, double *,
                                       cudaStream_t);

}  // namespace lbmem
