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
// and the material ids over the same rows (MW x RH bytes from x0 - 2 rounded down to 16).
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
#include "tile_tma.cuh"

namespace lbmem {

namespace {

using namespace tma_tile;
using G = GeoWide;
constexpr int KW = G::KW, KH = G::KH, RW = G::RW, RH = G::RH, IW = G::IW, IH = G::IH, MW = G::MW;
constexpr size_t kSmemBytes = G::kSmemBytes;

template <bool ACC, int POL>
__global__ void __launch_bounds__(NTH, 3)
    k_step2_tma(const StepArgs<float> a, const __grid_constant__ CUtensorMap fin,
                const __grid_constant__ CUtensorMap ids_map, float *__restrict__ fout,
                const long long *__restrict__ t_in, long long *__restrict__ t_out, int ntx, int n_tiles) {
    extern __shared__ unsigned char sm_dyn[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ SrcPairF sp;
    const TileSmem S = carve<G>(sm_dyn);

    const long long t = *t_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *t_out = t + 2;
    const int n_mine = (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // >= 1
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        sp = source_pair_f(a.src, t);  // the same for every tile of the launch
    }
    for (int k = threadIdx.x; k < 256; k += NTH) S.table[k] = a.mtab[k];
    __syncthreads();
    // tile coordinates step by the grid stride without a division per tile (a 32-bit
    // division by a run-time divisor executes on the FP64 pipe here, which GB300 keeps narrow)
    int tx = (int)blockIdx.x % ntx, ty = (int)blockIdx.x / ntx;
    const int sx = (int)gridDim.x % ntx, sy = (int)gridDim.x / ntx;
    auto advance = [&](int &x, int &y) {
        x += sx;
        y += sy;
        if (x >= ntx) {
            x -= ntx;
            ++y;
        }
    };
    if (threadIdx.x == 0) issue_tile<G>(&fin, &ids_map, tx * KW, ty * KH, S.stage, &bar);
    const bool src0 = t >= 1 && a.src.kind != SRC_NONE, src1 = a.src.kind != SRC_NONE;
    const int nx = a.nx, ny = a.ny;

    for (int i = 0; i < n_mine; ++i) {
        const int x0 = tx * KW, y0 = ty * KH;
        const int ioff = x0 - 1 - id_box_x(x0);  // column of site x0 - 1 in the id box
        const bool ok = mbar_wait(&bar, (unsigned)i & 1u);
        if (__syncthreads_or(!ok)) {  // the tile's copies never completed: report, leave
            if (threadIdx.x == 0) atomicOr(a.err, kErrTimeout);
            return;
        }
        for (int k = threadIdx.x; k < IW * IH; k += NTH) {
            const int lx = k % IW, ly = k / IW, x = x0 - 1 + lx, y = y0 - 1 + ly;
            if (x < 0 || x >= nx || y < 0 || y >= ny) continue;
            Pop<float> p;
            pull_buf<RW, RH>(S.raw, nx, ny, x, y, lx + 3, ly + 1, p);
            if (x == 0 && src0) inject_source_t(a.src.kind, sp.g0, sp.inc0, p);
            const uint8_t id = S.ids[(ly + 1) * MW + lx + ioff];
            const bool acc = ACC && lx >= 1 && lx <= KW && ly >= 1 && ly <= KH;
            double f3[3];
            if (update_site<POL, true>(p, S.table[id], a.runaway, acc ? f3 : nullptr, nullptr)) atomicOr(a.err, kErrUnstable);
            if (acc) acc_site(a.accp, a.src, (size_t)y * a.pitch + x, y, t, f3[0], f3[1], f3[2]);
            put_inter<G>(S.inter, ly, lx, p);
            S.inter_ids[ly * IW + lx] = id;
        }
        __syncthreads();  // the stage is read, the intermediate state written
        advance(tx, ty);  // the next tile of this CTA
        if (threadIdx.x == 0 && i + 1 < n_mine) {
            fence_proxy_async_smem();
            issue_tile<G>(&fin, &ids_map, tx * KW, ty * KH, S.stage, &bar);
        }
        for (int k = threadIdx.x; k < KW * KH; k += NTH) {
            const int lx = k % KW, ly = k / KW, x = x0 + lx, y = y0 + ly;
            if (x >= nx || y >= ny) continue;
            Pop<float> p;
            pull_buf<IW, IH>(S.inter, nx, ny, x, y, lx + 1, ly + 1, p);
            if (x == 0 && src1) inject_source_t(a.src.kind, sp.g1, sp.inc1, p);
            const size_t idx = (size_t)y * a.pitch + x;
            double f3[3];
            if (update_site<POL, true>(p, S.table[S.inter_ids[(ly + 1) * IW + lx + 1]], a.runaway, ACC ? f3 : nullptr, nullptr))
                atomicOr(a.err, kErrUnstable);
            if (ACC) acc_site(a.accp, a.src, idx, y, t + 1, f3[0], f3[1], f3[2]);
            store_site(fout, a.pstride, idx, p);
        }
        __syncthreads();  // the intermediate buffer is free for the next tile
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

}  // namespace

cudaError_t encode_tiled(CUtensorMap *map, CUtensorMapDataType type, cuuint32_t rank, const void *base,
                         const cuuint64_t *dims, const cuuint64_t *strides, const cuuint32_t *box) {
    EncodeTiled fn = encoder();
    if (!fn) return cudaErrorNotSupported;
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, type, rank, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The boxes of a tile shape: the stage (RW x RH x 11) and the ids (MW x RH).
static bool tile_boxes(int kw, int kh, int *rw, int *rh, int *mw) {
    if (kw == GeoWide::KW && kh == GeoWide::KH) {
        *rw = GeoWide::RW, *rh = GeoWide::RH, *mw = GeoWide::MW;
    } else if (kw == GeoTall::KW && kh == GeoTall::KH) {
        *rw = GeoTall::RW, *rh = GeoTall::RH, *mw = GeoTall::MW;
    } else if (kw == GeoMid::KW && kh == GeoMid::KH) {
        *rw = GeoMid::RW, *rh = GeoMid::RH, *mw = GeoMid::MW;
    } else {
        return false;
    }
    return true;
}

cudaError_t encode_plane_map(CUtensorMap *map, const float *base, int nx, int ny, int pitch, size_t pstride, int kw,
                             int kh) {
    int rw, rh, mw;
    if (((uintptr_t)base & 15u) || (pitch % 4) || (pstride % 4) || !tile_boxes(kw, kh, &rw, &rh, &mw))
        return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)NPLANES};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(float), (cuuint64_t)pstride * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)rw, (cuuint32_t)rh, (cuuint32_t)NPLANES};
    return encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box);
}

cudaError_t encode_id_map(CUtensorMap *map, const uint8_t *ids, int nx, int ny, int pitch, int kw, int kh) {
    int rw, rh, mw;
    if (((uintptr_t)ids & 15u) || (pitch % 16) || !tile_boxes(kw, kh, &rw, &rh, &mw)) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {(cuuint32_t)mw, (cuuint32_t)rh};
    return encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ids, dims, strides, box);
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
