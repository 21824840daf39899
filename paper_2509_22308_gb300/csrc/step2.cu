// Two time steps per launch for the double-float form: temporal blocking of the fused
// stream-collide step (arXiv 2509.22308, Sec. III).  (The FP32 and FP16-deviation forms
// stage their tiles with the copy engine: step2_tma.cu, step2_f16_tma.cu.)
//
// A CTA owns a TW x TH tile.  Phase 1 computes the post-collision f*(t) of the tile and
// a one-site halo (pulled from global memory exactly as the one-step kernel does) into
// shared memory; phase 2 pulls f(t + 1) of the tile from shared memory, collides and
// writes f*(t + 1) to global memory.  Each state element crosses HBM once per two steps
// (plus the halo, which neighbouring CTAs read at about the same time and L2 serves); the
// per-site arithmetic is the one-step kernel's, so the result is bit-identical to two
// one-step launches.
#include "common.cuh"
#include "step2.cuh"
#include "step_f16.cuh"

namespace lbmem {

// T = df (double-float form).
template <typename T, bool ACC, int POL>
__global__ void __launch_bounds__(NT) k_step2(const StepArgs<T> a, const T *__restrict__ fin, T *__restrict__ fout,
                                              const long long *__restrict__ t_in, long long *__restrict__ t_out) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *sm = reinterpret_cast<T *>(sm_raw);
    __shared__ SrcPair sp;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const long long t = *t_in;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *t_out = t + 2;
    source_pair(a.src, x0, t, &sp);
    __syncthreads();
    const bool src0 = t >= 1 && a.src.kind != SRC_NONE, src1 = a.src.kind != SRC_NONE;
    for (int k = threadIdx.x; k < SW * SH; k += NT) {
        const int lx = k % SW, ly = k / SW, x = x0 - 1 + lx, y = y0 - 1 + ly;
        if (x < 0 || x >= a.nx || y < 0 || y >= a.ny) continue;
        Pop<T> p;
        pull_planes(a, fin, x, y, p);
        if (x == 0 && src0) inject_source(a.src.kind, sp.g0, sp.inc0, p);
        const size_t idx = (size_t)y * a.pitch + x;
        const bool acc = ACC && lx >= 1 && lx <= TW && ly >= 1 && ly <= TH;
        double f3[3];
        if (update_site<POL, true>(p, a.mtab[a.mat[idx]], a.runaway, acc ? f3 : nullptr, nullptr)) atomicOr(a.err, 1u);
        if (acc) acc_site(a.accp, a.src, idx, y, t, f3[0], f3[1], f3[2]);
        put_smem(sm, ly, lx, p);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < TW * TH; k += NT) {
        const int lx = k % TW, ly = k / TW, x = x0 + lx, y = y0 + ly;
        if (x >= a.nx || y >= a.ny) continue;
        Pop<T> p;
        pull_smem(sm, a.nx, a.ny, x, y, lx + 1, ly + 1, p);
        if (x == 0 && src1) inject_source(a.src.kind, sp.g1, sp.inc1, p);
        const size_t idx = (size_t)y * a.pitch + x;
        double f3[3];
        if (update_site<POL, true>(p, a.mtab[a.mat[idx]], a.runaway, ACC ? f3 : nullptr, nullptr)) atomicOr(a.err, 1u);
        if (ACC) acc_site(a.accp, a.src, idx, y, t + 1, f3[0], f3[1], f3[2]);
        store_site(fout, a.pstride, idx, p);
    }
}

template <typename T>
static cudaError_t allow_smem() {
    const int b = (int)step2_smem<T>();
    cudaError_t e = cudaFuncSetAttribute(k_step2<T, false, POL_TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step2<T, true, POL_TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step2<T, false, POL_TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step2<T, true, POL_TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
}

cudaError_t step2_prepare() { return allow_smem<df>(); }

template <typename T>
cudaError_t launch_step2(const StepArgs<T> &a, const T *fin, T *fout, const long long *t_in, long long *t_out,
                         bool accumulate, cudaStream_t s) {
    dim3 grid((a.nx + TW - 1) / TW, (a.ny + TH - 1) / TH), block(NT);
    const size_t sb = step2_smem<T>();
    if (a.pol == POL_TE) {
        if (accumulate)
            k_step2<T, true, POL_TE><<<grid, block, sb, s>>>(a, fin, fout, t_in, t_out);
        else
            k_step2<T, false, POL_TE><<<grid, block, sb, s>>>(a, fin, fout, t_in, t_out);
    } else {
        if (accumulate)
            k_step2<T, true, POL_TM><<<grid, block, sb, s>>>(a, fin, fout, t_in, t_out);
        else
            k_step2<T, false, POL_TM><<<grid, block, sb, s>>>(a, fin, fout, t_in, t_out);
    }
    return cudaGetLastError();
}
template cudaError_t launch_step2<df>(const StepArgs<df> &, const df *, df *, const long long *, long long *, bool,
                                      cudaStream_t);

}  // namespace lbmem
