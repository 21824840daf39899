// Arguments of the FP16-deviation storage form (see step_f16.cu).
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"

namespace lbmem {

// Deviation scale 2^10: |g| up to ~64 E0 stays below the FP16 maximum, and
// deviations down to ~6e-8 / 2^10 stay normal.
constexpr float kF16Scale = 1024.0f;

struct F16Args {
    int nx, ny, pitch, pad;
    size_t pstride;
    const uint8_t *mat;
    const MatT<float> *mtab;
    SourceParams src;
    AccParams accp;
    unsigned *err;
    float scale, inv_scale;
    const __half *g;            // 16 deviation planes (input, time t)
    const float *fe, *fhx, *fhy;  // field planes (input)
    __half *g_out;
    float *fe_out, *fhx_out, *fhy_out;
};

// Byte layout of one FP16-deviation buffer: 16 half planes, then 3 float planes,
// each plane pstride elements (offsets rounded to 256 bytes).
inline size_t f16_half_bytes(size_t pstride) { return ((size_t)NPLANES * pstride * 2 + 255) / 256 * 256; }
inline size_t f16_plane_bytes(size_t pstride) { return (pstride * 4 + 255) / 256 * 256; }
inline size_t f16_buffer_bytes(size_t pstride) { return f16_half_bytes(pstride) + 3 * f16_plane_bytes(pstride); }

cudaError_t launch_step_f16(const F16Args &a, const long long *t_in, long long *t_out, bool accumulate,
                            cudaStream_t s);
cudaError_t launch_fields_f16(const F16Args &a, const long long *t_dev, double *ez, double *hx, double *hy,
                              cudaStream_t s);

}  // namespace lbmem
