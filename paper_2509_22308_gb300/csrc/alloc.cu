// Every device and pinned-host allocation of the library, in one place, with a hook that
// makes a chosen one fail (host-side fault injection for tests of the clean-up paths) and
// a count of what the library currently holds; and the host <-> device copies of the
// solver and batch calls, counted in bytes per direction.
//
// Counting: each call of dmalloc, dmalloc_async or of the pinned-block allocator of the
// solver's runtime (api.cu) is one allocation attempt; while the hook is armed with fail_at = k the k-th attempt after arming returns
// cudaErrorMemoryAllocation without calling CUDA, exactly what an exhausted device or host
// would return, and the caller's ordinary error path runs.  `held` is the number of device
// buffers and pinned blocks the library's handles and batches hold (pinned blocks parked in
// the process-wide reuse list are not held by anyone and are not counted).
#include <atomic>

#include "../../include/lbm_em.h"
#include "runtime.h"

namespace lbmem {

namespace {
std::atomic<long long> g_fail_at{0};   // 0: the hook is off
std::atomic<long long> g_attempts{0};  // allocation attempts since the hook was armed
std::atomic<long long> g_held{0};
std::atomic<unsigned long long> g_h2d{0}, g_d2h{0};

void count_copy(size_t bytes, cudaMemcpyKind kind) {
    if (kind == cudaMemcpyHostToDevice) g_h2d.fetch_add(bytes);
    if (kind == cudaMemcpyDeviceToHost) g_d2h.fetch_add(bytes);
}
}  // namespace

cudaError_t copy_async(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) {
    const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, s);
    if (e == cudaSuccess) count_copy(bytes, kind);
    return e;
}

cudaError_t copy2d_async(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t height,
                         cudaMemcpyKind kind, cudaStream_t s) {
    const cudaError_t e = cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, kind, s);
    if (e == cudaSuccess) count_copy(width * height, kind);
    return e;
}

bool alloc_should_fail() {
    const long long k = g_fail_at.load();
    if (k <= 0) return false;
    return g_attempts.fetch_add(1) + 1 == k;
}

void alloc_held(long long delta) { g_held.fetch_add(delta); }

cudaError_t dmalloc(void **p, size_t bytes) {
    *p = nullptr;
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) alloc_held(1);
    return e;
}

cudaError_t dmalloc_async(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaSuccess) alloc_held(1);
    return e;
}

void dfree(void *p) {
    if (!p) return;
    cudaFree(p);
    alloc_held(-1);
}

void dfree_async(void *p, cudaStream_t s) {
    if (!p) return;
    cudaFreeAsync(p, s);
    alloc_held(-1);
}

}  // namespace lbmem

extern "C" lbm_em_status lbm_em_transfer_bytes(uint64_t *h2d, uint64_t *d2h) {
    if (h2d) *h2d = lbmem::g_h2d.load();
    if (d2h) *d2h = lbmem::g_d2h.load();
    return LBM_EM_OK;
}

extern "C" lbm_em_status lbm_em_test_alloc_hook(int64_t fail_at, int64_t *live) {
    using namespace lbmem;
    if (fail_at < 0) return set_error(LBM_EM_EINVAL, "fail_at must be >= 0");
    g_attempts.store(0);
    g_fail_at.store(fail_at);
    if (live) *live = g_held.load();
    return LBM_EM_OK;
}
