// Diagnostics (the paper has no counterpart): the bounded device-side waits, and the FP64
// pipe's throughput that bounds the FP64 step.
//
// Bounded waits.
// The TMA-staged kernels wait on an mbarrier for their own tile copies, and every such wait
// gives up after a limit and reports through the error word instead of spinning forever.
// This probe runs that same wait (mbar_wait) in one block on an mbarrier that nothing ever
// arrives on, with a short limit, and reports the outcome exactly as a kernel's timeout is
// reported: LBM_EM_ETIMEOUT.  No copy is in flight, so the device stays usable.
#include "../../include/lbm_em.h"
#include "common.cuh"
#include "runtime.h"
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

}  // namespace
}  // namespace lbmem

using namespace lbmem;

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
