// Diagnostic of the bounded device-side waits (the paper has no counterpart).
//
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

}  // namespace
}  // namespace lbmem

using namespace lbmem;

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
