// Two time steps per launch for the FP32 form with TMA-staged tiles: the temporally
// blocked fused stream-collide step of arXiv 2509.22308, Sec. III (Eq. LBGK equation with
// the equilibria of Eq. equilibrium distribution functions), as in step2.cu, with the
// global-memory side rebuilt around the copy engine.
//
// A persistent CTA walks tiles of KW x KH sites: tile blockIdx.x, then + gridDim.x, ...,
// numbered row-major over the lattice, so the tiles in flight at any time form a band a
// few tile rows high whose halos meet in L2.  For each tile one thread issues two
// cp.async.bulk.tensor copies on one mbarrier: the 11 planes over the tile and a two-site
// halo (x from x0 - 4, so that the box starts on a 16-byte boundary: RW x RH x 11 floats)
// and the material ids over the same rows (x from x0 - 16: MW x RH bytes).
//   phase 1: f*(t) of the tile and a one-site halo, pulled from the stage (source at
//            x = 0, collision), into the intermediate buffer, with each site's id;
//   then the stage is free and the next tile's copies go out, so they run during
//   phase 2 (and during the other resident CTAs' work);
//   phase 2: f(t + 1) of the tile pulled from the intermediate buffer, collision,
//            f*(t + 1) stored to global memory.
// The material table sits in shared memory for the whole launch, so the per-site loop
// makes no dependent global loads.  Sites outside the lattice are skipped and pulls at the
// lattice edge clamp to the site itself (the zero-gradient open edge), so the zeros the
// copy engine reads outside the tensor are never used.  The per-site arithmetic is the
// one-step kernel's, so the result is bit-identical to two one-step launches.
//
// Measured on GB300 (8192^2, FP32): one stage per CTA with three CTAs per SM beat two
// stages per CTA with two CTAs per SM (128 vs 90 GLUPS): the resident CTAs cover each
// other's waits, and more warps per SM matter more than a deeper pipeline per CTA.
#include <mutex>

#include "common.cuh"
#include "step2.cuh"
#include "step2_tma.h"
#include "tma.cuh"

namespace lbmem {

namespace {

constexpr int KW = kTmaTileW, KH = kTmaTileH, NTH = kTmaThreads;
constexpr int RW = KW + 8, RH = KH + 4;  // stage: x0 - 4 .. x0 + KW + 3, y0 - 2 .. y0 + KH + 1
constexpr int IW = KW + 2, IH = KH + 2;  // intermediate: x0 - 1 .. x0 + KW, y0 - 1 .. y0 + KH
constexpr int MW = 96, MOFF = 16;        // ids: x0 - 16 .. x0 + 79, the stage's rows
static_assert(RW * sizeof(float) % 16 == 0 && MW % 16 == 0, "TMA box rows must be multiples of 16 bytes");
static_assert(KW % 16 == 0, "x0 - 4 floats and x0 - 16 bytes must start on 16-byte boundaries");
static_assert(MW >= MOFF + KW + 2, "the id box must cover x0 - 2 .. x0 + KW + 1");

constexpr int STATE_FLOATS = NPLANES * RH * RW;
constexpr unsigned STATE_BYTES = STATE_FLOATS * sizeof(float), ID_BYTES = MW * RH;
constexpr size_t OFF_IDS = (STATE_BYTES + 127) / 128 * 128;          // ids box, 128-byte aligned
constexpr size_t OFF_INTER = OFF_IDS + (ID_BYTES + 127) / 128 * 128;  // intermediate state
constexpr size_t OFF_TABLE = OFF_INTER + (size_t)NPLANES * IH * IW * sizeof(float);
constexpr size_t OFF_INTER_IDS = OFF_TABLE + 256 * sizeof(MatT<float>);
constexpr size_t kSmemBytes = OFF_INTER_IDS + (IW * IH + 15) / 16 * 16 + 128;  // + alignment slack
static_assert(STATE_BYTES % 16 == 0 && OFF_TABLE % 16 == 0, "shared-memory layout");
static_assert(3 * (kSmemBytes + 1024 + 64) <= 233472, "three CTAs per SM");

// f_i(r, t + 1) from post-collision values in a W x H x 11 shared-memory buffer; (cx, cy)
// is the site's cell in the buffer; the upstream cell clamps at the lattice edge.
template <int W, int H>
__device__ __forceinline__ void pull_buf(const float *sm, int nx, int ny, int x, int y, int cx, int cy,
                                         Pop<float> &p) {
    const int xm = x > 0 ? cx - 1 : cx, xp = x < nx - 1 ? cx + 1 : cx;
    const int ym = y > 0 ? cy - 1 : cy, yp = y < ny - 1 ? cy + 1 : cy;
    auto v = [&](int plane, int yy, int xx) { return sm[(plane * H + yy) * W + xx]; };
    p.ez = v(P_EZ, cy, cx);
    p.epx = v(P_EPX, cy, xm);
    p.emx = v(P_EMX, cy, xp);
    p.epy = v(P_EPY, ym, cx);
    p.emy = v(P_EMY, yp, cx);
    p.hxpx = v(P_HXPX, cy, xm);
    p.hxmx = v(P_HXMX, cy, xp);
    p.hxz = v(P_HXZ, cy, cx);
    p.hypy = v(P_HYPY, ym, cx);
    p.hymy = v(P_HYMY, yp, cx);
    p.hyz = v(P_HYZ, cy, cx);
}

__device__ __forceinline__ void put_inter(float *sm, int ly, int lx, const Pop<float> &p) {
    auto r = [&](int plane) -> float & { return sm[(plane * IH + ly) * IW + lx]; };
    r(P_EZ) = p.ez;
    r(P_EPX) = p.epx;
    r(P_EMX) = p.emx;
    r(P_EPY) = p.epy;
    r(P_EMY) = p.emy;
    r(P_HXPX) = p.hxpx;
    r(P_HXMX) = p.hxmx;
    r(P_HXZ) = p.hxz;
    r(P_HYPY) = p.hypy;
    r(P_HYMY) = p.hymy;
    r(P_HYZ) = p.hyz;
}

__device__ __forceinline__ void issue_tile(const CUtensorMap *fmap, const CUtensorMap *imap, int tile, int ntx,
                                           unsigned char *stage, uint64_t *bar) {
    const int x0 = (tile % ntx) * KW, y0 = (tile / ntx) * KH;
    mbar_arrive_expect_tx(bar, STATE_BYTES + ID_BYTES);
    tma_load_3d(stage, fmap, x0 - 4, y0 - 2, 0, bar);
    tma_load_2d(stage + OFF_IDS, imap, x0 - MOFF, y0 - 2, bar);
}

// Source values of the launch's two times in FP32, set by one thread per tile at x0 = 0
// (the double-precision evaluation runs once, not in every thread).
struct SrcPairF {
    float g0, inc0, g1, inc1;
};

template <bool ACC, int POL>
__global__ void __launch_bounds__(NTH, 3)
    k_step2_tma(const StepArgs<float> a, const __grid_constant__ CUtensorMap fin,
                const __grid_constant__ CUtensorMap ids_map, float *__restrict__ fout,
                const long long *__restrict__ t_in, long long *__restrict__ t_out, int ntx, int n_tiles) {
    extern __shared__ unsigned char sm_dyn[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ SrcPairF sp;
    unsigned char *stage = sm_dyn + ((128u - (smem_u32(sm_dyn) & 127u)) & 127u);
    const float *raw = reinterpret_cast<const float *>(stage);
    const uint8_t *ids = stage + OFF_IDS;
    float *inter = reinterpret_cast<float *>(stage + OFF_INTER);
    MatT<float> *smt = reinterpret_cast<MatT<float> *>(stage + OFF_TABLE);
    uint8_t *inter_ids = stage + OFF_INTER_IDS;

    const long long t = *t_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *t_out = t + 2;
    const int n_mine = (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // >= 1
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    for (int k = threadIdx.x; k < 256; k += NTH) smt[k] = a.mtab[k];
    __syncthreads();
    if (threadIdx.x == 0) issue_tile(&fin, &ids_map, blockIdx.x, ntx, stage, &bar);
    const bool src0 = t >= 1 && a.src.kind != SRC_NONE, src1 = a.src.kind != SRC_NONE;
    const int nx = a.nx, ny = a.ny;

    for (int i = 0; i < n_mine; ++i) {
        const int tile = blockIdx.x + i * gridDim.x;
        const int x0 = (tile % ntx) * KW, y0 = (tile / ntx) * KH;
        if (threadIdx.x == 0) {
            SrcPair v;
            source_pair(a.src, x0, t, &v);
            sp = SrcPairF{(float)v.g0, (float)v.inc0, (float)v.g1, (float)v.inc1};
        }
        const bool ok = mbar_wait(&bar, (unsigned)i & 1u);
        if (__syncthreads_or(!ok)) {  // the tile's copies never completed: report, leave
            if (threadIdx.x == 0) atomicOr(a.err, kErrTimeout);
            return;
        }
        for (int k = threadIdx.x; k < IW * IH; k += NTH) {
            const int lx = k % IW, ly = k / IW, x = x0 - 1 + lx, y = y0 - 1 + ly;
            if (x < 0 || x >= nx || y < 0 || y >= ny) continue;
            Pop<float> p;
            pull_buf<RW, RH>(raw, nx, ny, x, y, lx + 3, ly + 1, p);
            if (x == 0 && src0) inject_source_t(a.src.kind, sp.g0, sp.inc0, p);
            const uint8_t id = ids[(ly + 1) * MW + lx + MOFF - 1];
            const bool acc = ACC && lx >= 1 && lx <= KW && ly >= 1 && ly <= KH;
            double f3[3];
            if (update_site<POL, true>(p, smt[id], acc ? f3 : nullptr, nullptr)) atomicOr(a.err, kErrUnstable);
            if (acc) acc_site(a.accp, a.src, (size_t)y * a.pitch + x, y, t, f3[0], f3[1], f3[2]);
            put_inter(inter, ly, lx, p);
            inter_ids[ly * IW + lx] = id;
        }
        __syncthreads();  // the stage is read, the intermediate state written
        if (threadIdx.x == 0 && i + 1 < n_mine) {
            fence_proxy_async_smem();
            issue_tile(&fin, &ids_map, tile + gridDim.x, ntx, stage, &bar);
        }
        for (int k = threadIdx.x; k < KW * KH; k += NTH) {
            const int lx = k % KW, ly = k / KW, x = x0 + lx, y = y0 + ly;
            if (x >= nx || y >= ny) continue;
            Pop<float> p;
            pull_buf<IW, IH>(inter, nx, ny, x, y, lx + 1, ly + 1, p);
            if (x == 0 && src1) inject_source_t(a.src.kind, sp.g1, sp.inc1, p);
            const size_t idx = (size_t)y * a.pitch + x;
            double f3[3];
            if (update_site<POL, true>(p, smt[inter_ids[(ly + 1) * IW + lx + 1]], ACC ? f3 : nullptr, nullptr))
                atomicOr(a.err, kErrUnstable);
            if (ACC) acc_site(a.accp, a.src, idx, y, t + 1, f3[0], f3[1], f3[2]);
            store_site(fout, a.pstride, idx, p);
        }
        __syncthreads();  // the intermediate buffer and sp are free for the next tile
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver through the runtime (no link against libcuda).
EncodeTiled encoder() {
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

template <bool ACC, int POL>
cudaError_t allow_smem() {
    return cudaFuncSetAttribute(k_step2_tma<ACC, POL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

cudaError_t encode(CUtensorMap *map, CUtensorMapDataType type, cuuint32_t rank, const void *base,
                   const cuuint64_t *dims, const cuuint64_t *strides, const cuuint32_t *box) {
    EncodeTiled fn = encoder();
    if (!fn) return cudaErrorNotSupported;
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, type, rank, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t encode_plane_map(CUtensorMap *map, const float *base, int nx, int ny, int pitch, size_t pstride) {
    if (((uintptr_t)base & 15u) || (pitch % 4) || (pstride % 4)) return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)NPLANES};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(float), (cuuint64_t)pstride * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)RW, (cuuint32_t)RH, (cuuint32_t)NPLANES};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box);
}

cudaError_t encode_id_map(CUtensorMap *map, const uint8_t *ids, int nx, int ny, int pitch) {
    if (((uintptr_t)ids & 15u) || (pitch % 16)) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {(cuuint32_t)MW, (cuuint32_t)RH};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ids, dims, strides, box);
}

cudaError_t step2_tma_prepare(int *max_ctas) {
    cudaError_t e = allow_smem<false, POL_TM>();
    if (e == cudaSuccess) e = allow_smem<true, POL_TM>();
    if (e == cudaSuccess) e = allow_smem<false, POL_TE>();
    if (e == cudaSuccess) e = allow_smem<true, POL_TE>();
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step2_tma<false, POL_TM>, NTH, kSmemBytes);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) *max_ctas = per_sm * sms;
    return e;
}

cudaError_t launch_step2_tma(const StepArgs<float> &a, const CUtensorMap *fin, const CUtensorMap *ids, float *fout,
                             const long long *t_in, long long *t_out, bool accumulate, int max_ctas, cudaStream_t s) {
    const int ntx = (a.nx + KW - 1) / KW, nty = (a.ny + KH - 1) / KH, n_tiles = ntx * nty;
    const int grid = n_tiles < max_ctas ? n_tiles : max_ctas;
    if (a.pol == POL_TE) {
        if (accumulate)
            k_step2_tma<true, POL_TE><<<grid, NTH, kSmemBytes, s>>>(a, *fin, *ids, fout, t_in, t_out, ntx, n_tiles);
        else
            k_step2_tma<false, POL_TE><<<grid, NTH, kSmemBytes, s>>>(a, *fin, *ids, fout, t_in, t_out, ntx, n_tiles);
    } else {
        if (accumulate)
            k_step2_tma<true, POL_TM><<<grid, NTH, kSmemBytes, s>>>(a, *fin, *ids, fout, t_in, t_out, ntx, n_tiles);
        else
            k_step2_tma<false, POL_TM><<<grid, NTH, kSmemBytes, s>>>(a, *fin, *ids, fout, t_in, t_out, ntx, n_tiles);
    }
    return cudaGetLastError();
}

}  // namespace lbmem
