// Host-side interface of the TMA-staged two-steps-per-launch FP32 kernel (step2_tma.cu).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace lbmem {

// Tile of the single-domain TMA-staged kernel: kTmaTileW x kTmaTileH sites, kTmaThreads
// threads per CTA.  Shared memory per CTA: one stage (the 11 planes over the tile and a
// two-site halo, 72 x 12 x 11 floats, and the ids over the same rows, 96 x 12 bytes: 39 KB),
// the intermediate state with a one-site halo and its ids (29 KB) and the 256-entry
// material table (4 KB): 72 KB, three CTAs per SM.  The batch also runs 32 x 16 tiles
// (tile_tma.cuh).
constexpr int kTmaTileW = 64, kTmaTileH = 8, kTmaThreads = 256;

// cuTensorMapEncodeTiled (through the driver entry point, no link against libcuda): no
// interleave, no swizzle, 256-byte L2 promotion, zero fill outside the tensor.
cudaError_t encode_tiled(CUtensorMap *map, CUtensorMapDataType type, cuuint32_t rank, const void *base,
                         const cuuint64_t *dims, const cuuint64_t *strides, const cuuint32_t *box);

// Tensor map of an FP32 state buffer (11 planes of ny rows of `pitch` floats, plane stride
// `pstride` floats) with the stage box of kw x kh tiles (64 x 8 or 32 x 16).  base 16-byte
// aligned, pitch and pstride multiples of 4; cudaErrorInvalidValue otherwise or if the
// driver rejects the map.
cudaError_t encode_plane_map(CUtensorMap *map, const float *base, int nx, int ny, int pitch, size_t pstride, int kw,
                             int kh);

// Tensor map of the material ids (ny rows of `pitch` bytes, pitch a multiple of 16) with
// the id box of kw x kh tiles.
cudaError_t encode_id_map(CUtensorMap *map, const uint8_t *ids, int nx, int ny, int pitch, int kw, int kh);

// Once per device, outside stream capture: allows the kernels' shared memory and returns
// the persistent grid (resident CTAs per SM x SMs) in *max_ctas.
cudaError_t step2_tma_prepare(int *max_ctas);

// Two steps: the state described by *fin (time word t_in) -> fout (t_out = t + 2).
cudaError_t launch_step2_tma(const StepArgs<float> &a, const CUtensorMap *fin, const CUtensorMap *ids, float *fout,
                             const long long *t_in, long long *t_out, bool accumulate, int max_ctas, cudaStream_t s);

// Three steps per launch (step3_tma.cu): kTma3TileW x kTma3TileH tiles with a three-site
// halo (stage box 36 x 18 x 11 floats, id box 48 x 18 bytes), 74 KB of shared memory per
// CTA, three CTAs per SM.  encode_step3_maps builds the stage map of one FP32 state buffer
// and, if imap is not NULL, the id map (base and ids 16-byte aligned, pitch a multiple of
// 16, pstride of 4; cudaErrorInvalidValue otherwise or if the driver rejects a map).
constexpr int kTma3TileW = 28, kTma3TileH = 12;
cudaError_t encode_step3_maps(CUtensorMap *fmap, const float *base, CUtensorMap *imap, const uint8_t *ids, int nx,
                              int ny, int pitch, size_t pstride);
cudaError_t step3_tma_prepare(int *max_ctas);
// Three steps: the state described by *fin (time word t_in) -> fout (t_out = t + 3).
cudaError_t launch_step3_tma(const StepArgs<float> &a, const CUtensorMap *fin, const CUtensorMap *ids, float *fout,
                             const long long *t_in, long long *t_out, bool accumulate, int max_ctas, cudaStream_t s);

}  // namespace lbmem
