// Device-side definitions shared by the lattice Boltzmann Maxwell kernels.
//
// TM^z reduction of the D3Q7 vector scheme (arXiv 2509.22308, Sec. III).  With
// E = (0, 0, E_z) and H = (H_x, H_y, 0) the equilibria of
// Eq. (equilibrium distribution functions) only reach 16 of the 42 vector components:
// the e_z component of e_0, e_+-x, e_+-y, e_+-z and the h_x, h_y components of h_+-x,
// h_+-y, h_+-z (h_0 = 0 because mu_r = 1; the x/y parts of e_+-z cancel in every moment).
// Starting from zero, five more relations hold exactly at every step, because the two
// populations involved move together and have equal or opposite equilibria, so their
// difference only changes sign in the collision (the source, the open edges and PEC
// cells preserve them too):
//   e_+z,z = e_-z,z,  h_+z = h_-z,
//   h_+x,y = -e_+x,z,  h_-x,y = e_-x,z,  h_+y,x = e_+y,z,  h_-y,x = -e_-y,z,
//   e_0,z = 6 (eps_r - 1) e_z,z  (0 in PEC cells).
// The state is therefore 11 scalars per site, stored as structure-of-arrays planes:
//   e_z of the z pair and of +x, -x, +y, -y;  h_x of +x, -x, z;  h_y of +y, -y, z.
//
// Storage: plane p of site (x, y) at p * pstride + y * pitch + x.  A buffer holds the
// post-collision values f*(t-1); the step kernel at time t pulls
// f_i(r, t) = f*_i(r - c_i, t - 1) ("pull" streaming), so every plane is read once and
// written once per step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "df32.cuh"

namespace lbmem {

enum Plane {
    P_EZ = 0, P_EPX, P_EMX, P_EPY, P_EMY,
    P_HXPX, P_HXMX, P_HXZ,
    P_HYPY, P_HYMY, P_HYZ,
    NPLANES
};

// Bits of the sticky error word that the host reads back: a field became non-finite or
// ran away, or a bounded device-side wait gave up.
constexpr unsigned kErrUnstable = 1u, kErrTimeout = 2u;

enum SourceKind { SRC_HARD = 0, SRC_OPEN = 1, SRC_NONE = 2 };  // values of lbm_em_source_kind
enum Polarization { POL_TM = 0, POL_TE = 1 };

// Per-material constants in the kernel's arithmetic type:
// inv_eps3 = 1/(3 eps_r) (0 for PEC: E := 0), c_d = 6 eps_r - 4 (the weight of the z pair
// in D once e_0 = 6 (eps_r - 1) e_z is substituted), inv_eps = 1/eps_r, c3 = 3 eps_r
// (1 for PEC).  The host builds the table so that c_d + 4 = 2 c3 holds exactly in T.
template <typename T>
struct MatT {
    T inv_eps3, c_d, inv_eps, c3;
};

// Left-edge source: the exact discrete plane wave of the lattice.  With
// z = e^{-i w}, w = 2 pi / T, the +x population of e_z carries Re[P z^t] at x = 0 and
// Re[P w z^t] at x = 1 (P, w from the dispersion relation, computed on the host).
struct SourceParams {
    int kind, period, ramp, pad;
    double pr, pi;        // P
    double qr, qi;        // P * w
    const double2 *cs;    // cs[t mod T] = (cos w t, sin w t)
};

// Accumulation at the contour's stencil sites (Sec. III: Fourier analysis over one period).
struct AccParams {
    const int *slot;      // per-site slot (pitch layout), -1: not a stencil site
    double *acc;          // 6 doubles per slot: Re/Im of E_z, H_x, H_y
    int y0, y1;           // rows holding stencil sites
};

template <typename T>
struct StepArgs {
    int nx, ny, pitch, pol;  // pol: POL_TM or POL_TE
    size_t pstride;
    const uint8_t *mat;   // material id per site (pitch layout)
    const MatT<T> *mtab;  // 256 entries
    SourceParams src;
    AccParams accp;
    unsigned *err;        // sticky error word
    unsigned runaway;     // exponent-field threshold of the runaway test (runaway_bits)
    int pad2;
};

template <typename T>
struct Pop {
    T ez, epx, emx, epy, emy;
    T hxpx, hxmx, hxz;
    T hypy, hymy, hyz;
};

// Source values at time t: *g_open = ramp (Re[P z^t] - Re[P w z^t]) (added to the
// extrapolated incoming population), *inc = ramp Re[P z^t] (the incident one).
__device__ __forceinline__ void source_values(const SourceParams &s, long long t, double *g_open,
                                              double *inc) {
    const int tm = (int)(t % (long long)s.period);
    const double2 c = s.cs[tm];
    const double p0 = s.pr * c.x + s.pi * c.y;
    const double p1 = s.qr * c.x + s.qi * c.y;
    double ramp = 1.0;
    if (t < (long long)s.ramp) {
        const double v = sin(0.5 * 3.14159265358979323846 * (double)t / (double)s.ramp);
        ramp = v * v;
    }
    *g_open = ramp * (p0 - p1);
    *inc = ramp * p0;
}

// Adds the left-edge source of time t to the pulled populations of a site at x = 0, from
// the values source_values() gives for t: OPEN adds g_open to e_+x,z (and so, through
// h_+x,y = -e_+x,z, subtracts it from h_+x,y); HARD replaces the incoming pair by the
// incident one.
template <typename T>
__device__ __forceinline__ void inject_source_t(int kind, T g_open, T inc, Pop<T> &p) {
    if (kind == SRC_OPEN) {
        p.epx += g_open;
    } else {
        p.epx = inc;
        p.hxpx = (T)0;
    }
}
template <typename T>
__device__ __forceinline__ void inject_source(int kind, double g_open, double inc, Pop<T> &p) {
    inject_source_t<T>(kind, (T)g_open, (T)inc, p);
}

// f_i(r, t) = f*_i(r - c_i, t - 1) without the source; an upstream site outside the
// lattice is replaced by the site itself (open edge: zero-gradient copy along the
// population's own direction).
template <typename T>
__device__ __forceinline__ void pull_planes(const StepArgs<T> &a, const T *__restrict__ f, int x, int y,
                                            Pop<T> &p) {
    const size_t ps = a.pstride;
    const int xm = x > 0 ? x - 1 : 0;
    const int xp = x < a.nx - 1 ? x + 1 : x;
    const size_t r = (size_t)y * a.pitch;
    const size_t rm = (size_t)(y > 0 ? y - 1 : 0) * a.pitch;
    const size_t rp = (size_t)(y < a.ny - 1 ? y + 1 : y) * a.pitch;
    p.ez = f[P_EZ * ps + r + x];
    p.epx = f[P_EPX * ps + r + xm];
    p.emx = f[P_EMX * ps + r + xp];
    p.epy = f[P_EPY * ps + rm + x];
    p.emy = f[P_EMY * ps + rp + x];
    p.hxpx = f[P_HXPX * ps + r + xm];
    p.hxmx = f[P_HXMX * ps + r + xp];
    p.hxz = f[P_HXZ * ps + r + x];
    p.hypy = f[P_HYPY * ps + rm + x];
    p.hymy = f[P_HYMY * ps + rp + x];
    p.hyz = f[P_HYZ * ps + r + x];
}

// pull_planes plus the source at x = 0 (t >= 1), evaluated by the thread that needs it.
// Kernels that pull many sites per thread in a loop evaluate source_values() once per
// block instead and call inject_source(): the evaluation (a double-precision sine and
// the phase) does not depend on the site, and a compiler may hoist it out of the loop,
// running it in every thread on the low-throughput FP64 pipe.
template <typename T>
__device__ __forceinline__ void pull_site(const StepArgs<T> &a, const T *__restrict__ f, int x,
                                          int y, long long t, Pop<T> &p) {
    pull_planes(a, f, x, y, p);
    if (x == 0 && t >= 1 && a.src.kind != SRC_NONE) {
        double g, inc;
        source_values(a.src, t, &g, &inc);
        inject_source(a.src.kind, g, inc, p);
    }
}

template <typename T>
__device__ __forceinline__ T fmat(T a, T b, T c) { return fma(a, b, c); }

// num / den in FP32 without a fixed bias: q = num * inv carries the rounding of the
// constant inv ~ 1/den, the same relative error at every site and step; the residual
// num - q den is exact in one FMA, and adding residual * inv corrects q to within about
// one unit in the last place of the true quotient, with a sign that varies from site to
// site (one Newton-Raphson residual correction, as in Markstein's division scheme).
// Why it matters: the scheme at tau = 1/2 has no damping, so a relative bias b in the
// equilibria (1/3 rounded to FP32 is 1/3 (1 + 3.0e-8)) multiplies the wave by (1 + 2b)
// every step: +7e-4 in amplitude after 12 000 steps, twice that in the forces.
__device__ __forceinline__ float quot(float num, float den, float inv) {
    const float q = __fmul_rn(num, inv);
    return __fmaf_rn(__fmaf_rn(-q, den, num), inv, q);
}

// Moments (Sec. III): D = sum e_i = (6 eps_r - 4) e_z + e_+x + e_-x + e_+y + e_-y (the rest
// population and the z pair folded in), E_z = D / eps_r, H = sum h_i with the tied
// populations substituted.  Returns D, E_z/3 (the scale every equilibrium uses), H_x, H_y.
// FP32 takes E_z/3 = D / c3 through quot(); with c_d + 4 = 2 c3 exact in the table the
// collision then conserves D up to that one unbiased rounding.
template <typename T>
__device__ __forceinline__ void moments(const Pop<T> &p, const MatT<T> &m, T *E3, T *Hx, T *Hy, T *D) {
    const T d = fmat(m.c_d, p.ez, p.epx) + p.emx + p.epy + p.emy;
    *D = d;
    if constexpr (sizeof(T) == 4)
        *E3 = quot(d, m.c3, m.inv_eps3);
    else
        *E3 = d * m.inv_eps3;
    *Hx = fmat((T)2, p.hxz, p.hxpx + p.hxmx) + (p.epy - p.emy);
    *Hy = fmat((T)2, p.hyz, p.hypy + p.hymy) + (p.emx - p.epx);
}

// Post-collision f* = 2 f^eq - f (Eq. LBGK equation), with 2 f^eq written out from
// Eq. (equilibrium distribution functions) for the stored components:
//   e_z:  z E/3, +x (E-H_y)/3, -x (E+H_y)/3, +y (E+H_x)/3, -y (E-H_x)/3
//   h_x:  +-x and z H_x/3;   h_y: +-y and z H_y/3
// FP64: 28 arithmetic operations per site with the moments (FP64 is bound by its pipe
// on GB300): every 2 f^eq that is E/3 +- H/3 is one fused multiply-add; the bias of 1/3
// rounded to FP64 (2^-54 relative) stays below 1e-11 over 10^5 steps.  FP32 forms H/3
// once per component through quot() (see there) and adds or subtracts it.
template <typename T>
__device__ __forceinline__ void collide(Pop<T> &p, T E3, T Hx, T Hy) {
    if constexpr (sizeof(T) == 4) {
        const float third = 1.0f / 3.0f;
        const float hx3 = quot(Hx, 3.0f, third), hy3 = quot(Hy, 3.0f, third);
        p.ez = E3 - p.ez;
        p.epx = (E3 - hy3) - p.epx;
        p.emx = (E3 + hy3) - p.emx;
        p.epy = (E3 + hx3) - p.epy;
        p.emy = (E3 - hx3) - p.emy;
        p.hxpx = hx3 - p.hxpx;
        p.hxmx = hx3 - p.hxmx;
        p.hxz = hx3 - p.hxz;
        p.hypy = hy3 - p.hypy;
        p.hymy = hy3 - p.hymy;
        p.hyz = hy3 - p.hyz;
    } else {
        const T third = (T)(1.0 / 3.0), mthird = (T)(-1.0 / 3.0);
        const T A = fmat(Hy, mthird, E3), B = fmat(Hy, third, E3);
        const T C = fmat(Hx, third, E3), D = fmat(Hx, mthird, E3);
        p.ez = E3 - p.ez;
        p.epx = A - p.epx;
        p.emx = B - p.emx;
        p.epy = C - p.epy;
        p.emy = D - p.emy;
        p.hxpx = fmat(Hx, third, -p.hxpx);
        p.hxmx = fmat(Hx, third, -p.hxmx);
        p.hxz = fmat(Hx, third, -p.hxz);
        p.hypy = fmat(Hy, third, -p.hypy);
        p.hymy = fmat(Hy, third, -p.hymy);
        p.hyz = fmat(Hy, third, -p.hyz);
    }
}

// ---- TE^z (H_z, E_x, E_y), the polarization the paper leaves for future work ----------
// The same scheme with E = (E_x, E_y, 0), H = (0, 0, H_z).  By the argument given for TM
// at the top of this file the state reduces exactly to 11 scalars per site, and they
// stream like the TM planes, so TE keeps them in the same planes (same pull, source and
// edge handling):
//   P_EZ   e_y of the z pair   P_HXZ  e_x of the z pair   P_HYZ  h_z of the z pair
//   P_EPX  e_+x,y   P_EMX  e_-x,y   P_EPY  e_+y,y   P_EMY  e_-y,y
//   P_HXPX e_+x,x   P_HXMX e_-x,x   P_HYPY e_+y,x   P_HYMY e_-y,x
// with h_+x,z = e_+x,y, h_-x,z = -e_-x,y, h_+y,z = -e_+y,x, h_-y,z = e_-y,x, e_+z = e_-z,
// h_+z,z = h_-z,z and e_0 = 6 (eps_r - 1) e_z (0 in PEC cells); h_+-z in x and y cancel
// pairwise and never reach a field.  The incident wave E_y = H_z enters through e_+x,y as
// the TM wave enters through e_+x,z, and its e_+x,x is zero (the HARD source's h_+x,x slot).

// TE moments: D_y and D_x formed like D of TM, E/3 = D / (3 eps_r),
// H_z = 2 h_z,z + e_+x,y - e_-x,y - e_+y,x + e_-y,x.
template <typename T>
__device__ __forceinline__ void moments_te(const Pop<T> &p, const MatT<T> &m, T *Ey3, T *Ex3, T *Hz, T *Dy,
                                           T *Dx) {
    const T dy = fmat(m.c_d, p.ez, p.epx) + p.emx + p.epy + p.emy;
    const T dx = fmat(m.c_d, p.hxz, p.hxpx) + p.hxmx + p.hypy + p.hymy;
    *Dy = dy;
    *Dx = dx;
    if constexpr (sizeof(T) == 4) {
        *Ey3 = quot(dy, m.c3, m.inv_eps3);
        *Ex3 = quot(dx, m.c3, m.inv_eps3);
    } else {
        *Ey3 = dy * m.inv_eps3;
        *Ex3 = dx * m.inv_eps3;
    }
    *Hz = fmat((T)2, p.hyz, p.epx - p.emx) + (p.hymy - p.hypy);
}

// TE collision f* = 2 f^eq - f: e_x of z, +-x: E_x/3; of +y: E_x/3 - H_z/3; of -y:
// E_x/3 + H_z/3; e_y of z, +-y: E_y/3; of +x: E_y/3 + H_z/3; of -x: E_y/3 - H_z/3;
// h_z of the z pair: H_z/3.
template <typename T>
__device__ __forceinline__ void collide_te(Pop<T> &p, T Ey3, T Ex3, T Hz) {
    if constexpr (sizeof(T) == 4) {
        const float hz3 = quot(Hz, 3.0f, 1.0f / 3.0f);
        p.epx = (Ey3 + hz3) - p.epx;
        p.emx = (Ey3 - hz3) - p.emx;
        p.hypy = (Ex3 - hz3) - p.hypy;
        p.hymy = (Ex3 + hz3) - p.hymy;
        p.hyz = hz3 - p.hyz;
    } else {
        const T third = (T)(1.0 / 3.0), mthird = (T)(-1.0 / 3.0);
        p.epx = fmat(Hz, third, Ey3) - p.epx;
        p.emx = fmat(Hz, mthird, Ey3) - p.emx;
        p.hypy = fmat(Hz, mthird, Ex3) - p.hypy;
        p.hymy = fmat(Hz, third, Ex3) - p.hymy;
        p.hyz = fmat(Hz, third, -p.hyz);
    }
    p.ez = Ey3 - p.ez;
    p.epy = Ey3 - p.epy;
    p.emy = Ey3 - p.emy;
    p.hxpx = Ex3 - p.hxpx;
    p.hxmx = Ex3 - p.hxmx;
    p.hxz = Ex3 - p.hxz;
}

// Runaway test on the exponent bits (integer ALU only): |E/3| >= 2^(20 + k) or non-finite,
// where 2^k <= |E0| < 2^(k + 1) for the incident amplitude E0 (k = 0 for E0 = 0), so the test
// fires when a field has grown by about 2^20 over its drive whatever the amplitude (the
// scheme is linear: every field and force scales with E0).  thr is the threshold on the
// exponent field of the type: runaway_bits<T>(E0) on the host.
__device__ __forceinline__ bool field_runaway(double e3, unsigned thr) {
    return (unsigned)(__double2hiint(e3) & 0x7ff00000) >= thr;
}
__device__ __forceinline__ bool field_runaway(float e3, unsigned thr) {
    return (__float_as_uint(e3) & 0x7f800000u) >= thr;
}

template <typename T>
__device__ __forceinline__ void store_site(T *__restrict__ f, size_t ps, size_t idx, const Pop<T> &p) {
    f[P_EZ * ps + idx] = p.ez;
    f[P_EPX * ps + idx] = p.epx;
    f[P_EMX * ps + idx] = p.emx;
    f[P_EPY * ps + idx] = p.epy;
    f[P_EMY * ps + idx] = p.emy;
    f[P_HXPX * ps + idx] = p.hxpx;
    f[P_HXMX * ps + idx] = p.hxmx;
    f[P_HXZ * ps + idx] = p.hxz;
    f[P_HYPY * ps + idx] = p.hypy;
    f[P_HYMY * ps + idx] = p.hymy;
    f[P_HYZ * ps + idx] = p.hyz;
}

// One site of either polarization: the field triple (TM: E_z, H_x, H_y; TE: H_z, E_x, E_y)
// from the moments, into f3 when wanted; the energy density (D.E + H^2)/2 when wanted;
// then, if COLLIDE, the post-collision populations.  Returns whether the field ran away
// (field_runaway with threshold rthr).
template <int POL, bool COLLIDE, typename T>
__device__ __forceinline__ bool update_site(Pop<T> &p, const MatT<T> &m, unsigned rthr, double *f3, double *w) {
    bool bad;
    if constexpr (POL == POL_TM) {
        T E3, Hx, Hy, D;
        moments(p, m, &E3, &Hx, &Hy, &D);
        bad = field_runaway(E3, rthr);
        if (f3) {
            f3[0] = (double)(D * m.inv_eps);
            f3[1] = (double)Hx;
            f3[2] = (double)Hy;
        }
        if (w) *w = 0.5 * ((double)D * (double)(D * m.inv_eps) + (double)Hx * (double)Hx + (double)Hy * (double)Hy);
        if (COLLIDE) collide(p, E3, Hx, Hy);
    } else {
        T Ey3, Ex3, Hz, Dy, Dx;
        moments_te(p, m, &Ey3, &Ex3, &Hz, &Dy, &Dx);
        bad = field_runaway(Ey3, rthr) || field_runaway(Ex3, rthr);
        if (f3) {
            f3[0] = (double)Hz;
            f3[1] = (double)(Dx * m.inv_eps);
            f3[2] = (double)(Dy * m.inv_eps);
        }
        if (w)
            *w = 0.5 * ((double)Dx * (double)(Dx * m.inv_eps) + (double)Dy * (double)(Dy * m.inv_eps) +
                        (double)Hz * (double)Hz);
        if (COLLIDE) collide_te(p, Ey3, Ex3, Hz);
    }
    return bad;
}

// Contour sample: four stencil slots with bilinear weights, outward normal.
struct ContourPt {
    int s[4];
    double w[4];
    double nx, ny;
};

}  // namespace lbmem
