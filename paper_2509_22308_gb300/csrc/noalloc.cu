// Rasterisation of a Janus disc for callers that must not allocate device memory.
//
// Some hosts of this library cannot call cudaMalloc: an application whose own memory
// pool has already reserved the device's free memory, or a latency-critical loop in
// which cudaMalloc / cudaFree would synchronise the whole device.  This entry point
// writes the region ids into one fixed scratch array that lives in this library's
// device image instead of a per-call allocation.
//
// The array is a file-scope __device__ variable: every GPU that loads the library
// holds its 4 MiB until the process exits.  Host code cannot use the variable's name
// as a device address (on the host it is only a stand-in symbol), so each call looks
// the device address up with cudaGetSymbolAddress while the caller's device is current
// and passes it to the kernel.  The lookup is a host-side table query (no allocation,
// no device work); doing it on every call instead of caching it per device keeps the
// address right when the caller has reset the device (cudaDeviceReset) or otherwise
// recreated its primary context, after which the module, and the array with it, can
// sit at a different address.
#include <cmath>

#include "../../include/lbm_em.h"
#include "common.cuh"
#include "launchers.h"
#include "runtime.h"

using namespace lbmem;

namespace {

static __device__ __align__(256) uint8_t g_raster_scratch[LBM_EM_NOALLOC_RASTER_BYTES];

// Device address of g_raster_scratch in the current context.
lbm_em_status scratch_address(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_raster_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(no-allocation scratch)");
    *out = p;
    return LBM_EM_OK;
}

}  // namespace

extern "C" lbm_em_status lbm_em_rasterize_janus_noalloc(const lbm_em_janus *j, int32_t nx, int32_t ny,
                                                        uint8_t *regions) {
    lbm_em_status st = check_janus(j);
    if (st) return st;
    if (nx < 1 || ny < 1 || !regions) return set_error(LBM_EM_EINVAL, "bad size or NULL output");
    const int pitch = round_up(nx, 32);
    if ((size_t)pitch * (size_t)ny > (size_t)LBM_EM_NOALLOC_RASTER_BYTES)
        return set_error(LBM_EM_EINVAL, "lattice too large for the no-allocation scratch: ny * (nx rounded up to "
                                        "a multiple of 32) must be <= LBM_EM_NOALLOC_RASTER_BYTES (4 MiB)");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_error(LBM_EM_ECUDA, "no CUDA device available (the solver has no CPU path)");
    }
    void *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st) return st;
    double cx, cy;
    janus_center(j, nx, ny, &cx, &cy);
    // every site of the nx x ny window is written, so nothing needs clearing first
    st = cuda_status(launch_rasterize(nx, ny, pitch, cx, cy, j->a, -std::sin(j->phi0), -std::cos(j->phi0),
                                      (uint8_t *)scratch, 0),
                     "rasterise kernel");
    if (!st)
        st = cuda_status(cudaMemcpy2D(regions, nx, scratch, pitch, nx, ny, cudaMemcpyDeviceToHost),
                         "reading regions from the no-allocation scratch");
    return st;
}
