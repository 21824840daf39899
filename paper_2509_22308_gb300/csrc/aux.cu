// Set-up and reduction kernels: staircase rasterisation of a Janus disc and the
// period-averaged Maxwell-stress-tensor contour integral.
#include "common.cuh"
#include "launchers.h"

namespace lbmem {

// Region id per site (Sec. II; staircase of Sec. IV.A): 0 outside |d| <= a,
// 1 (region II) where d . n_d > 1e-9, 2 (region III) otherwise.  Explicit
// round-to-nearest operations keep the decisions identical to a plain
// evaluation of the same expressions in double precision.  Rows are walked with a
// grid stride, so a lattice of any height (grid.y is limited to 65535) is covered.
__global__ void k_rasterize(int nx, int ny, int pitch, double cx, double cy, double a2, double ndx,
                            double ndy, uint8_t *ids) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    const double dx = __dsub_rn((double)x, cx);
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        const double dy = __dsub_rn((double)y, cy);
        const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        uint8_t id = 0;
        if (r2 <= a2) {
            const double side = __dadd_rn(__dmul_rn(dx, ndx), __dmul_rn(dy, ndy));
            id = side > 1e-9 ? 1 : 2;
        }
        ids[(size_t)y * pitch + x] = id;
    }
}

cudaError_t launch_rasterize(int nx, int ny, int pitch, double cx, double cy, double a, double ndx,
                             double ndy, uint8_t *ids, cudaStream_t s) {
    dim3 block(256), grid((nx + 255) / 256, ny < 65535 ? ny : 65535);
    k_rasterize<<<grid, block, 0, s>>>(nx, ny, pitch, cx, cy, a * a, ndx, ndy, ids);
    return cudaGetLastError();
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// <T> . n at each contour point from bilinearly interpolated phasors
// (Eq. stress tensor average with eps0 = mu0 = 1; E = E_z z, H = (H_x, H_y)):
//   T_xx = (|H_x|^2 - (|E|^2 + |H|^2)/2)/2, T_yy = (|H_y|^2 - (|E|^2 + |H|^2)/2)/2,
//   T_xy = Re(H_x H_y*)/2;  F = sum (T . n) dl (Eq. force),
//   M_z = sum (r x (T . n))_z dl (Eq. torque); out = (F_x/F0, F_y/F0, M_z/M0).
// One block; per-thread partial sums, warp shuffles, then one warp over the warps.
__global__ void __launch_bounds__(256) k_contour(const double *__restrict__ acc, double scale,
                                                 const ContourPt *__restrict__ pts, int npts, double R,
                                                 double dl, double F0, double M0, double *out) {
    double fx = 0.0, fy = 0.0, mz = 0.0;
    for (int k = threadIdx.x; k < npts; k += blockDim.x) {
        const ContourPt p = pts[k];
        double v[6] = {0, 0, 0, 0, 0, 0};
        for (int c = 0; c < 4; ++c) {
            const double *q = acc + 6 * (size_t)p.s[c];
            for (int j = 0; j < 6; ++j) v[j] += p.w[c] * q[j];
        }
        for (int j = 0; j < 6; ++j) v[j] *= scale;
        const double e2 = v[0] * v[0] + v[1] * v[1];
        const double hx2 = v[2] * v[2] + v[3] * v[3];
        const double hy2 = v[4] * v[4] + v[5] * v[5];
        const double tr = 0.5 * (e2 + hx2 + hy2);
        const double txx = 0.5 * (hx2 - tr);
        const double tyy = 0.5 * (hy2 - tr);
        const double txy = 0.5 * (v[2] * v[4] + v[3] * v[5]);
        const double tnx = txx * p.nx + txy * p.ny;
        const double tny = txy * p.nx + tyy * p.ny;
        fx += tnx;
        fy += tny;
        mz += R * (p.nx * tny - p.ny * tnx);
    }
    __shared__ double sh[3][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    mz = warp_sum(mz);
    if (lane == 0) {
        sh[0][wid] = fx;
        sh[1][wid] = fy;
        sh[2][wid] = mz;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        fx = lane < nw ? sh[0][lane] : 0.0;
        fy = lane < nw ? sh[1][lane] : 0.0;
        mz = lane < nw ? sh[2][lane] : 0.0;
        fx = warp_sum(fx);
        fy = warp_sum(fy);
        mz = warp_sum(mz);
        if (lane == 0) {
            out[0] = fx * dl / F0;
            out[1] = fy * dl / F0;
            out[2] = mz * dl / M0;
        }
    }
}

// Near-to-far-field transform (far-field scattering intensity, Sec. II.A): block j sums
// over the contour points for observation angle angles[j] (lattice frame, 0 = +x):
//   A = (k/4) sum [ (u . n) E^s + (-n_x H_y^s + n_y H_x^s) ] e^{-i k R (u . n)} dl,
// with scattered phasors = total - incident (incident E_z phasor per stencil site given,
// H_y^I = -E^I, H_x^I = 0), interpolated bilinearly; out[3 j] = (2/pi)|A|^2 / E0^2,
// out[3 j + 1 .. 2] = Re, Im A.
// TE^z (triple H_z, E_x, E_y): the same transform of H_z with dH_z/dn = -i k (-n_x E_y + n_y E_x)
// (curl H = -i k E) and the incident wave E_y^I = +H_z^I, so sgn = -1 flips both.
__global__ void __launch_bounds__(256) k_farfield(const double *__restrict__ acc, double scale,
                                                  const ContourPt *__restrict__ pts, int npts,
                                                  const double2 *__restrict__ inc, double R, double dl, double k,
                                                  double E0, double sgn, const double *__restrict__ angles,
                                                  double *out) {
    const double phi = angles[blockIdx.x];
    double su, cu;
    sincos(phi, &su, &cu);
    double sr = 0.0, si = 0.0;
    for (int q = threadIdx.x; q < npts; q += blockDim.x) {
        const ContourPt p = pts[q];
        double v[6] = {0, 0, 0, 0, 0, 0};
        for (int c = 0; c < 4; ++c) {
            const double *a = acc + 6 * (size_t)p.s[c];
            const double2 ei = inc[p.s[c]];
            v[0] += p.w[c] * (a[0] * scale - ei.x);
            v[1] += p.w[c] * (a[1] * scale - ei.y);
            v[2] += p.w[c] * (a[2] * scale);
            v[3] += p.w[c] * (a[3] * scale);
            v[4] += p.w[c] * (a[4] * scale + sgn * ei.x);
            v[5] += p.w[c] * (a[5] * scale + sgn * ei.y);
        }
        const double un = cu * p.nx + su * p.ny;
        const double fr = un * v[0] + sgn * (-p.nx * v[4] + p.ny * v[2]);
        const double fi = un * v[1] + sgn * (-p.nx * v[5] + p.ny * v[3]);
        double sp, cp;
        sincos(-k * R * un, &sp, &cp);
        sr += fr * cp - fi * sp;
        si += fr * sp + fi * cp;
    }
    __shared__ double sh[2][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) {
        sh[0][wid] = sr;
        sh[1][wid] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        const double Ar = 0.25 * k * a * dl, Ai = 0.25 * k * b * dl;
        out[3 * blockIdx.x] = (2.0 / 3.14159265358979323846) * (Ar * Ar + Ai * Ai) / (E0 * E0);
        out[3 * blockIdx.x + 1] = Ar;
        out[3 * blockIdx.x + 2] = Ai;
    }
}

cudaError_t launch_farfield(const double *acc, double scale, const ContourPt *pts, int npts, const double2 *inc,
                            double R, double dl, double k, double E0, int pol, const double *angles, int n_angles,
                            double *out, cudaStream_t s) {
    k_farfield<<<n_angles, 256, 0, s>>>(acc, scale, pts, npts, inc, R, dl, k, E0, pol == POL_TE ? -1.0 : 1.0,
                                        angles, out);
    return cudaGetLastError();
}

cudaError_t launch_contour(const double *acc, double scale, const ContourPt *pts, int npts, double R,
                           double dl, double F0, double M0, double *out, cudaStream_t s) {
    k_contour<<<1, 256, 0, s>>>(acc, scale, pts, npts, R, dl, F0, M0, out);
    return cudaGetLastError();
}

}  // namespace lbmem
