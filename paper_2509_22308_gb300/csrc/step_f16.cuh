// FP16-deviation storage form: arguments, layout and the per-population arithmetic
// shared by every kernel of this form (see step_f16.cu).
//
// A population is stored as its deviation from the equilibrium of its own site,
// g_i = f_i - f_i^eq(F), in FP16 scaled by 2^10, next to the site's fields in FP32,
// kept as F = (E_z/3, H_x/3, H_y/3): every 2 f^eq is then a sum or difference of two
// stored values and f^eq itself an exact halving, so no rounded constant (1/3, 1/6)
// enters the state (see quot() in common.cuh for why a fixed bias must not).  Every
// kernel rebuilds and re-encodes a population with the explicitly rounded helpers
// below, so the one-step, two-step and field kernels of this form agree bit for bit.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace lbmem {

struct F16Args {
    int nx, ny, pitch, pad;
    size_t pstride;
    const uint8_t *mat;
    const MatT<float> *mtab;
    SourceParams src;
    AccParams accp;
    unsigned *err;
    unsigned runaway;             // FP32 runaway threshold (runaway_bits<float>)
    float scale, inv_scale;       // deviation scale 2^(10 - k) (f16_scale) and its inverse
    const __half *g;              // 11 deviation planes (input)
    const float *fe, *fhx, *fhy;  // field planes (input)
    __half *g_out;
    float *fe_out, *fhx_out, *fhy_out;
};

// Byte layout of one FP16-deviation buffer: 11 half planes, then 3 float planes,
// each plane pstride elements (offsets rounded to 256 bytes).
inline size_t f16_half_bytes(size_t pstride) { return ((size_t)NPLANES * pstride * 2 + 255) / 256 * 256; }
inline size_t f16_plane_bytes(size_t pstride) { return (pstride * 4 + 255) / 256 * 256; }
inline size_t f16_buffer_bytes(size_t pstride) { return f16_half_bytes(pstride) + 3 * f16_plane_bytes(pstride); }

// 2 f_i^eq of each stored population from the stored fields of its site
// (Eq. equilibrium distribution functions): e_z: z E/3, +x E/3 - H_y/3, -x E/3 + H_y/3,
// +y E/3 + H_x/3, -y E/3 - H_x/3;  h_x: +-x, z H_x/3;  h_y: +-y, z H_y/3.
__device__ __forceinline__ float eq2_epx(float e, float hx, float hy) { return __fsub_rn(e, hy); }
__device__ __forceinline__ float eq2_emx(float e, float hx, float hy) { return __fadd_rn(e, hy); }
__device__ __forceinline__ float eq2_epy(float e, float hx, float hy) { return __fadd_rn(e, hx); }
__device__ __forceinline__ float eq2_emy(float e, float hx, float hy) { return __fsub_rn(e, hx); }

// f = eq2 / 2 - g * inv_scale (inv_scale = 2^(k - 10), the inverse of the deviation scale)
__device__ __forceinline__ float rebuild(float eq2, __half g, float inv_scale) {
    return __fmaf_rn(-__half2float(g), inv_scale, __fmul_rn(eq2, 0.5f));
}

// f = eq2 / 2 + g * nis, nis = -2^(k - 10): the value of rebuild() with the FP16
// deviation g taken straight into the FMA, one of the pair g2 (HI: the high half).  The
// mixed-precision fma (PTX fma.rn.f32.f16, sm_100 and later) multiplies two FP16 operands and
// adds an FP32 one with a single rounding to FP32; FP16 values and -2^(k - 10) are exact in FP32,
// so this is the FP32 FMA of rebuild() without the separate conversion of g.  nis must be
// exactly representable in FP16 (k >= -14).
// The FP16 bit pattern of -2^m, -24 <= m <= 15 (normal from 2^-14, subnormal below): the
// nis operand of rebuild_h.
inline unsigned short f16_neg_pow2_bits(int m) {
    return (unsigned short)(0x8000u | (m >= -14 ? (unsigned)(m + 15) << 10 : 1u << (m + 24)));
}

template <bool HI>
__device__ __forceinline__ float rebuild_h(float eq2, unsigned g2, unsigned short nis) {
    float r;
    if constexpr (HI)
        asm("{\n\t.reg .f16 l, h;\n\tmov.b32 {l, h}, %1;\n\tfma.rn.f32.f16 %0, h, %2, %3;\n\t}"
            : "=f"(r) : "r"(g2), "h"(nis), "f"(__fmul_rn(eq2, 0.5f)));
    else
        asm("{\n\t.reg .f16 l, h;\n\tmov.b32 {l, h}, %1;\n\tfma.rn.f32.f16 %0, l, %2, %3;\n\t}"
            : "=f"(r) : "r"(g2), "h"(nis), "f"(__fmul_rn(eq2, 0.5f)));
    return r;
}

// Encoding g = (f - eq2 / 2) * s, rounded to FP16, as one FMA: f * s - (eq2 / 2) * s.  The
// scale s is a power of two, and scaling by one commutes with rounding, so the FMA's single
// rounding gives the value of "subtract, round, scale"; a result that underflows FP32's normal
// range in one form and not the other converts to the same FP16 zero or subnormal.  The
// scaled halves of every 2 f^eq come from the scaled fields of the site (eq2 * s / 2 is a
// sum or difference of two of them, by the same argument).
struct EqS {
    float z, px, mx, py, my, hx, hy;
};
__device__ __forceinline__ EqS eq_scaled(float e3, float hx3, float hy3, float scale) {
    const float h = 0.5f * scale;
    const float e = __fmul_rn(e3, h), hx = __fmul_rn(hx3, h), hy = __fmul_rn(hy3, h);
    return EqS{e, __fsub_rn(e, hy), __fadd_rn(e, hy), __fadd_rn(e, hx), __fsub_rn(e, hx), hx, hy};
}
__device__ __forceinline__ float encode_f(float f, float eqs, float scale) { return __fmaf_rn(f, scale, -eqs); }

// Stored fields of a site: E_z/3, H_x/3, H_y/3.
struct Fld {
    float e, hx, hy;
};

__device__ __forceinline__ Fld load_fld(const F16Args &a, size_t i) { return Fld{a.fe[i], a.fhx[i], a.fhy[i]}; }

// The stored fields from the moments (E3 = E_z/3 already; H/3 through quot()).
__device__ __forceinline__ Fld stored_fields(float E3, float Hx, float Hy) {
    return Fld{E3, quot(Hx, 3.0f, 1.0f / 3.0f), quot(Hy, 3.0f, 1.0f / 3.0f)};
}

// Source at x = 0 (t >= 1): adds to e_+x (and so, through the tie h_+x,y = -e_+x,z, to h_+x,y).
__device__ __forceinline__ void f16_source(const SourceParams &src, int x, long long t, Pop<float> &p) {
    if (x == 0 && t >= 1 && src.kind != SRC_NONE) {
        double gs, inc;
        source_values(src, t, &gs, &inc);
        inject_source(src.kind, gs, inc, p);
    }
}

// f_i(r, t) for the 11 populations of site (x, y), rebuilt from the upstream sites'
// fields and deviations of time t - 1 (one site per call), without the source.
__device__ __forceinline__ void pull_f16_planes(const F16Args &a, int x, int y, Pop<float> &p) {
    const size_t ps = a.pstride;
    const int xm = x > 0 ? x - 1 : 0;
    const int xp = x < a.nx - 1 ? x + 1 : x;
    const size_t r = (size_t)y * a.pitch;
    const size_t rm = (size_t)(y > 0 ? y - 1 : 0) * a.pitch;
    const size_t rp = (size_t)(y < a.ny - 1 ? y + 1 : y) * a.pitch;
    const float is = a.inv_scale;
    const Fld c = load_fld(a, r + x), w = load_fld(a, r + xm), e = load_fld(a, r + xp);
    const Fld so = load_fld(a, rm + x), no = load_fld(a, rp + x);
    const __half *g = a.g;
    p.ez = rebuild(c.e, g[P_EZ * ps + r + x], is);
    p.epx = rebuild(eq2_epx(w.e, w.hx, w.hy), g[P_EPX * ps + r + xm], is);
    p.emx = rebuild(eq2_emx(e.e, e.hx, e.hy), g[P_EMX * ps + r + xp], is);
    p.epy = rebuild(eq2_epy(so.e, so.hx, so.hy), g[P_EPY * ps + rm + x], is);
    p.emy = rebuild(eq2_emy(no.e, no.hx, no.hy), g[P_EMY * ps + rp + x], is);
    p.hxpx = rebuild(w.hx, g[P_HXPX * ps + r + xm], is);
    p.hxmx = rebuild(e.hx, g[P_HXMX * ps + r + xp], is);
    p.hxz = rebuild(c.hx, g[P_HXZ * ps + r + x], is);
    p.hypy = rebuild(so.hy, g[P_HYPY * ps + rm + x], is);
    p.hymy = rebuild(no.hy, g[P_HYMY * ps + rp + x], is);
    p.hyz = rebuild(c.hy, g[P_HYZ * ps + r + x], is);
}

// pull_f16_planes plus the source (see pull_site for when to use inject_source instead).
__device__ __forceinline__ void pull_f16(const F16Args &a, int x, int y, long long t, Pop<float> &p) {
    pull_f16_planes(a, x, y, p);
    f16_source(a.src, x, t, p);
}

// The 11 encoded deviations of a site whose pulled populations are p and stored fields F.
__device__ __forceinline__ void encode_all(const Pop<float> &p, const Fld &F, float sc, __half g[NPLANES]) {
    const EqS q = eq_scaled(F.e, F.hx, F.hy, sc);
    g[P_EZ] = __float2half_rn(encode_f(p.ez, q.z, sc));
    g[P_EPX] = __float2half_rn(encode_f(p.epx, q.px, sc));
    g[P_EMX] = __float2half_rn(encode_f(p.emx, q.mx, sc));
    g[P_EPY] = __float2half_rn(encode_f(p.epy, q.py, sc));
    g[P_EMY] = __float2half_rn(encode_f(p.emy, q.my, sc));
    g[P_HXPX] = __float2half_rn(encode_f(p.hxpx, q.hx, sc));
    g[P_HXMX] = __float2half_rn(encode_f(p.hxmx, q.hx, sc));
    g[P_HXZ] = __float2half_rn(encode_f(p.hxz, q.hx, sc));
    g[P_HYPY] = __float2half_rn(encode_f(p.hypy, q.hy, sc));
    g[P_HYMY] = __float2half_rn(encode_f(p.hymy, q.hy, sc));
    g[P_HYZ] = __float2half_rn(encode_f(p.hyz, q.hy, sc));
}

// encode_all of two sites at once, site a in the low and site b in the high half of each
// pair (one paired conversion per population).
__device__ __forceinline__ void encode_pair(const Pop<float> &a, const Pop<float> &b, const Fld &Fa, const Fld &Fb,
                                            float sc, __half2 g[NPLANES]) {
    const EqS qa = eq_scaled(Fa.e, Fa.hx, Fa.hy, sc), qb = eq_scaled(Fb.e, Fb.hx, Fb.hy, sc);
#define LBMEM_ENC2(P, m, eq) g[P] = __floats2half2_rn(encode_f(a.m, qa.eq, sc), encode_f(b.m, qb.eq, sc))
    LBMEM_ENC2(P_EZ, ez, z);
    LBMEM_ENC2(P_EPX, epx, px);
    LBMEM_ENC2(P_EMX, emx, mx);
    LBMEM_ENC2(P_EPY, epy, py);
    LBMEM_ENC2(P_EMY, emy, my);
    LBMEM_ENC2(P_HXPX, hxpx, hx);
    LBMEM_ENC2(P_HXMX, hxmx, hx);
    LBMEM_ENC2(P_HXZ, hxz, hx);
    LBMEM_ENC2(P_HYPY, hypy, hy);
    LBMEM_ENC2(P_HYMY, hymy, hy);
    LBMEM_ENC2(P_HYZ, hyz, hy);
#undef LBMEM_ENC2
}

// What the next step's pull rebuilds from this site (its stored fields and encoded
// deviations): the post-collision populations exactly as storage followed by a pull
// would give them.
__device__ __forceinline__ void rebuild_all(const __half g[NPLANES], const Fld &F, float is, Pop<float> &q) {
    q.ez = rebuild(F.e, g[P_EZ], is);
    q.epx = rebuild(eq2_epx(F.e, F.hx, F.hy), g[P_EPX], is);
    q.emx = rebuild(eq2_emx(F.e, F.hx, F.hy), g[P_EMX], is);
    q.epy = rebuild(eq2_epy(F.e, F.hx, F.hy), g[P_EPY], is);
    q.emy = rebuild(eq2_emy(F.e, F.hx, F.hy), g[P_EMY], is);
    q.hxpx = rebuild(F.hx, g[P_HXPX], is);
    q.hxmx = rebuild(F.hx, g[P_HXMX], is);
    q.hxz = rebuild(F.hx, g[P_HXZ], is);
    q.hypy = rebuild(F.hy, g[P_HYPY], is);
    q.hymy = rebuild(F.hy, g[P_HYMY], is);
    q.hyz = rebuild(F.hy, g[P_HYZ], is);
}

cudaError_t launch_step_f16(const F16Args &a, const long long *t_in, long long *t_out, bool accumulate,
                            cudaStream_t s);

// Two steps per launch on TMA-staged 64 x 8 tiles (step2_f16_tma.cu), bit-identical to two
// launch_step_f16 calls.  encode_f16_maps builds the tensor maps of one buffer's deviation
// planes (*gmap) and field planes (*fmap): buf 16-byte aligned, pitch and pstride multiples
// of 8 (cudaErrorInvalidValue otherwise, or if the driver rejects a map).  The prepare call
// (once per device, outside stream capture) allows the kernel's shared memory and returns
// the persistent grid in *max_ctas; ids is the id map of encode_id_map for 64 x 8 tiles.
cudaError_t encode_f16_maps(CUtensorMap *gmap, CUtensorMap *fmap, const void *buf, int nx, int ny, int pitch,
                            size_t pstride);
cudaError_t step2_f16_tma_prepare(int *max_ctas);
cudaError_t launch_step2_f16_tma(const F16Args &a, const CUtensorMap *gmap, const CUtensorMap *fmap,
                                 const CUtensorMap *ids, const long long *t_in, long long *t_out, bool accumulate,
                                 int max_ctas, cudaStream_t s);
cudaError_t launch_energy_f16(const F16Args &a, const long long *t_dev, double *energy, cudaStream_t s);
cudaError_t launch_fields_f16(const F16Args &a, const long long *t_dev, double *ez, double *hx, double *hy,
                              cudaStream_t s);

}  // namespace lbmem
