// Diagnostics (the paper has no counterpart): the bounded device-side waits, and the FP64
// pipe's throughput that bounds the FP64 step.
//
// Bounded waits.
// The TMA-staged kernels wait on an mbarrier for their own tile copies, and every such wait
// gives up after a limit and reports through the error word instead of spinning forever.
// This probe runs that same wait (mbar_wait) in one block on an mbarrier that nothing ever
// arrives on, with a short limit, and reports the outcome exactly as a kernel's timeout is
// reported: LBM_EM_ETIMEOUT.  No copy is in flight, so the device stays usable.
#include <algorithm>
#include <cmath>

#include "../../include/lbm_em.h"
#include "common.cuh"
#include "runtime.h"
#include "step_f16.cuh"
#include "tma.cuh"

namespace lbmem {
namespace {

__device__ unsigned g_probe_err;

__global__ void k_wait_probe(long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected, none ever made
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0u, limit);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(&g_probe_err, kErrTimeout);
}

// FP64 pipe throughput: kFmaChains independent fused multiply-add chains per thread, so
// the pipe, not the latency of one chain, limits the rate.  The multiplier and addend come
// from the arguments and the sums are written under a condition the host never meets, so
// the compiler can neither fold nor drop the chains.
constexpr int kFmaChains = 8, kFmaThreads = 256;
__device__ double g_fp64_sink;

__global__ void __launch_bounds__(kFmaThreads) k_fp64_fma(long long iters, double m, double c) {
    double v[kFmaChains];
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) v[j] = (double)(threadIdx.x + j) * 1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kFmaChains; ++j) v[j] = fma(v[j], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) s += v[j];
    if (s == -1.0) g_fp64_sink = s;  // never true for the host's arguments (every chain stays > 0)
}

// The FP16-deviation rebuild with the mixed-precision FMA (rebuild_h) against the converting one
// (rebuild), both halves of every pair: counts the results whose bits differ.
__global__ void k_f16_rebuild_probe(const unsigned *__restrict__ g2, const float *__restrict__ eq2, long long n,
                                    unsigned short nis, float inv, unsigned long long *bad) {
    unsigned long long d = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned g = g2[i];
        const float e = eq2[i];
        const __half lo = __ushort_as_half((unsigned short)(g & 0xffffu));
        const __half hi = __ushort_as_half((unsigned short)(g >> 16));
        const float m[2] = {rebuild_h<false>(e, g, nis), rebuild_h<true>(e, g, nis)};
        const float r[2] = {rebuild(e, lo, inv), rebuild(e, hi, inv)};
        for (int j = 0; j < 2; ++j)
            d += !(__float_as_uint(m[j]) == __float_as_uint(r[j]) || (isnan(m[j]) && isnan(r[j])));
    }
    if (d) atomicAdd(bad, d);
}

}  // namespace
}  // namespace lbmem

using namespace lbmem;

extern "C" lbm_em_status lbm_em_probe_f16_rebuild(const uint32_t *g2, const float *eq2, int64_t n, int32_t m,
                                                   int64_t *mismatches) {
    if (!g2 || !eq2 || !mismatches || n < 1 || m < -24 || m > 15)
        return set_error(LBM_EM_EINVAL, "need arrays of n >= 1 values, an output and -24 <= m <= 15");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_error(LBM_EM_ECUDA, "no CUDA device available (the solver has no CPU path)");
    }
    const unsigned short nis = f16_neg_pow2_bits(m);
    void *dg = nullptr, *de = nullptr, *db = nullptr;
    lbm_em_status st = cuda_status(dmalloc(&dg, (size_t)n * 4), "cudaMalloc(probe)");
    if (!st) st = cuda_status(dmalloc(&de, (size_t)n * 4), "cudaMalloc(probe)");
    if (!st) st = cuda_status(dmalloc(&db, 8), "cudaMalloc(probe)");
    if (!st) st = cuda_status(copy_async(dg, g2, (size_t)n * 4, cudaMemcpyHostToDevice, 0), "upload");
    if (!st) st = cuda_status(copy_async(de, eq2, (size_t)n * 4, cudaMemcpyHostToDevice, 0), "upload");
    if (!st) st = cuda_status(cudaMemsetAsync(db, 0, 8, 0), "clear");
    if (!st) {
        const long long blocks = std::min<long long>((n + 255) / 256, 4096);
        k_f16_rebuild_probe<<<(unsigned)blocks, 256>>>((const unsigned *)dg, (const float *)de, (long long)n, nis,
                                                       std::ldexp(1.0f, m), (unsigned long long *)db);
        st = cuda_status(cudaGetLastError(), "probe launch");
    }
    unsigned long long bad = 0;
    if (!st) st = cuda_status(copy_async(&bad, db, 8, cudaMemcpyDeviceToHost, 0), "read");
    if (!st) st = cuda_status(cudaStreamSynchronize(0), "cudaStreamSynchronize");
    dfree(dg);
    dfree(de);
    dfree(db);
    if (!st) *mismatches = (int64_t)bad;
    return st;
}

extern "C" lbm_em_status lbm_em_probe_fp64_fma(void *stream, int64_t iters, double *fma_per_launch) {
    if (iters < 1 || !fma_per_launch) return set_error(LBM_EM_EINVAL, "need iters >= 1 and an output");
    int ndev = 0, dev = 0, sms = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_error(LBM_EM_ECUDA, "no CUDA device available (the solver has no CPU path)");
    }
    lbm_em_status st = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (!st) st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (st) return st;
    const int blocks = 8 * sms;  // 8 resident blocks of 256 threads per SM: every scheduler busy
    k_fp64_fma<<<blocks, kFmaThreads, 0, (cudaStream_t)stream>>>((long long)iters, 1.0 - 1e-12, 1e-9);
    st = cuda_status(cudaGetLastError(), "FP64 probe launch");
    if (!st) *fma_per_launch = (double)blocks * kFmaThreads * kFmaChains * (double)iters;
    return st;
}

extern "C" lbm_em_status lbm_em_probe_bounded_wait(int64_t limit_cycles) {
    if (limit_cycles <= 0 || limit_cycles > kWaitCycles)
        return set_error(LBM_EM_EINVAL, "limit_cycles must be in 1 .. 2e9");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_error(LBM_EM_ECUDA, "no CUDA device available (the solver has no CPU path)");
    }
    const unsigned zero = 0;
    lbm_em_status st = cuda_status(cudaMemcpyToSymbol(g_probe_err, &zero, sizeof(zero)), "clearing the probe word");
    if (st) return st;
    k_wait_probe<<<1, 32>>>((long long)limit_cycles);
    st = cuda_status(cudaGetLastError(), "probe launch");
    if (st) return st;
    unsigned err = 0;
    st = cuda_status(cudaMemcpyFromSymbol(&err, g_probe_err, sizeof(err)), "reading the probe word");
    if (st) return st;
    if (err & kErrTimeout) return set_error(LBM_EM_ETIMEOUT, "the bounded wait gave up and reported, as designed");
    return set_error(LBM_EM_ECUDA, "a wait on an mbarrier that nothing arrives on did not give up");
}
