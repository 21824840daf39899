// Host-side launchers of the single-domain kernels (defined in the .cu files).
#pragma once

#include "common.cuh"

namespace lbmem {

template <typename T>
cudaError_t launch_step(const StepArgs<T> &a, const T *fin, T *fout, const long long *t_in,
                        long long *t_out, bool accumulate, cudaStream_t s);
template <typename T>
cudaError_t launch_fields(const StepArgs<T> &a, const T *f, const long long *t_dev, double *ez,
                          double *hx, double *hy, cudaStream_t s);
template <typename T>
cudaError_t launch_energy(const StepArgs<T> &a, const T *f, const long long *t_dev, double *energy, cudaStream_t s);
cudaError_t launch_rasterize(int nx, int ny, int pitch, double cx, double cy, double a,
                             double ndx, double ndy, uint8_t *ids, cudaStream_t s);
cudaError_t launch_contour(const double *acc, double scale, const ContourPt *pts, int npts,
                           double R, double dl, double F0, double M0, double *out, cudaStream_t s);
cudaError_t launch_farfield(const double *acc, double scale, const ContourPt *pts, int npts, const double2 *inc,
                            double R, double dl, double k, double E0, int pol, const double *angles, int n_angles,
                            double *out, cudaStream_t s);

}  // namespace lbmem
