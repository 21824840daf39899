// Host-side interface of the four-steps-per-launch streaming kernels (step_stream.cu).
#pragma once

#include <cuda.h>

#include "common.cuh"
#include "step_f16.cuh"

namespace lbmem {

// A warp stages kStreamLoadW columns of every row (two sites per lane) and outputs the
// kStreamOutW inner ones; kStreamHalo columns on each side feed the four steps.  Thread
// blocks of kStreamWarps warps, three per SM.
constexpr int kStreamLoadW = 64, kStreamHalo = 4, kStreamOutW = 56, kStreamWarps = 4, kStreamSteps = 4;

// How a lattice is cut into work units (a strip of kStreamOutW columns and a segment of
// seg_rows rows each, one per warp): strips first, then as many segments as fit in one wave
// of resident warps.
struct StreamPlan {
    int n_strips, seg_rows, n_units, grid;
};
StreamPlan stream_plan(int nx, int ny, int resident_warps);

// Once per device, outside stream capture: allows the kernels' shared memory and returns
// the warps resident on the whole GPU (blocks per SM x SMs x kStreamWarps).
cudaError_t stream_prepare(bool f16, int *resident_warps);

// Tensor maps of one state buffer: FP32 (smap: 11 planes, box 64 x 1 x 11 floats) or
// FP16-deviation (smap: the 11 deviation planes, box 64 x 1 x 11 halves; fmap: the 3 field
// planes, box 64 x 1 x 3 floats), and the id map (box 80 x 1 bytes).  buf and ids 16-byte
// aligned, pitch a multiple of 16, pstride of 8; cudaErrorInvalidValue otherwise or if the
// driver rejects a map.
cudaError_t encode_stream_maps(CUtensorMap *smap, CUtensorMap *fmap, CUtensorMap *imap, const void *buf, bool f16,
                               const uint8_t *ids, int nx, int ny, int pitch, size_t pstride);

// Four steps: the state described by the maps (time word t_in) -> fout / the FP16-deviation
// output planes of fa (t_out = t + 4).  FP32 of either polarization (a.pol), or the
// FP16-deviation form (TM) when fa is not NULL.  No Fourier accumulation.
cudaError_t launch_step4_stream(const StepArgs<float> &a, const F16Args *fa, const CUtensorMap *smap,
                                const CUtensorMap *fmap, const CUtensorMap *imap, float *fout, const StreamPlan &plan,
                                const long long *t_in, long long *t_out, cudaStream_t s);

}  // namespace lbmem
