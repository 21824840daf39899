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
// seg_rows rows each, one per warp): strips first, then row segments for a few full waves of
// the resident warps (see stream_plan).  f16: the FP16-deviation kernel.
struct StreamPlan {
    int n_strips, seg_rows, n_units, grid;
};
StreamPlan stream_plan(int nx, int ny, int resident_warps, bool f16);

// Once per device, outside stream capture: allows the kernels' shared memory and returns
// the warps resident on the whole GPU (blocks per SM x SMs x kStreamWarps), of the plain kernel
// and of the accumulating one.
cudaError_t stream_prepare(bool f16, int *resident_warps, int *resident_warps_acc);

// Tensor maps of one state buffer: FP32 (smap: 11 planes, box 64 x 1 x 11 floats) or
// FP16-deviation (smap: the 11 deviation planes, box 64 x 1 x 11 halves; fmap: the 3 field
// planes, box 64 x 1 x 3 floats), and the id map (box 80 x 1 bytes).  buf and ids 16-byte
// aligned, pitch a multiple of 16, pstride of 8; cudaErrorInvalidValue otherwise or if the
// driver rejects a map.
cudaError_t encode_stream_maps(CUtensorMap *smap, CUtensorMap *fmap, CUtensorMap *imap, const void *buf, bool f16,
                               const uint8_t *ids, int nx, int ny, int pitch, size_t pstride);

// The source values of a launch's four times (FP32, for the lanes at x = 0).
struct SrcLevels {
    float g[kStreamSteps], inc[kStreamSteps];
};

// One instance of a batched design map as the four-step batch kernel reads it: lattice, run
// length and accumulated period, the rows holding contour stencil sites, the element offsets of
// its state, slot map and accumulators in the packed buffers, its phase table and its region
// table (vacuum, region II, region III) in FP32.
struct alignas(16) StreamInst {
    int nx, ny, pitch, kind;
    int seg_rows, n_strips, ay0, ay1;
    long long steps, acc_from;
    long long base, pstride;
    long long slot_base;
    int acc_base, period;
    const double2 *cs;
    unsigned runaway;
    int pad;
    MatT<float> m[3];
};

// Once per device, outside stream capture: shared memory of the batch kernel, resident warps.
cudaError_t batch_stream_prepare(int *resident_warps);
// The three tensor maps of one instance (state in buffer 0, in buffer 1, ids) in maps[0..2].
cudaError_t encode_batch_stream_maps(CUtensorMap *maps, const float *buf0, const float *buf1, const uint8_t *ids,
                                     int nx, int ny, int pitch, size_t pstride);
// Four steps of every unfinished instance: the source values of each instance at the launch's
// four times into srcs (from srcp[n_inst]), then the kernel over units[n_units] (int4:
// instance, strip, segment; walked with a stride of grid x kStreamWarps warps), input state
// buffer p (maps[3 i + p]), output buf_out; the stencil sites of instances in their accumulated
// period staged in stage (12 floats per slot of the packed accumulators acc[6 n_slots]) and
// added to acc by a flush over the slots (slot_inst[n_slots]: each slot's instance).
cudaError_t launch_batch_step4(const StreamInst *insts, const SourceParams *srcp, int n_inst, const int4 *units,
                               int n_units, SrcLevels *srcs, const CUtensorMap *maps, int p, float *buf_out,
                               const int *slot, double *acc, float *stage, const int *slot_inst, int n_slots,
                               unsigned *err, const long long *t_in, long long *t_out, int grid, int pol,
                               cudaStream_t s);

// Four steps: the state described by the maps (time word t_in) -> fout / the FP16-deviation
// output planes of fa (t_out = t + 4).  FP32 of either polarization (a.pol), or the
// FP16-deviation form (TM) when fa is not NULL.  accumulate: the Fourier sums of the four times
// at the n_slots stencil sites of a.accp, with the phases a.src.cs, through the staging buffer
// stage (12 floats per slot) and a second launch that adds it to a.accp.acc.
cudaError_t launch_step4_stream(const StepArgs<float> &a, const F16Args *fa, const CUtensorMap *smap,
                                const CUtensorMap *fmap, const CUtensorMap *imap, float *fout, const StreamPlan &plan,
                                const long long *t_in, long long *t_out, bool accumulate, float *stage, int n_slots,
                                cudaStream_t s);

}  // namespace lbmem
