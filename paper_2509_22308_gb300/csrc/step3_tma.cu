// Three time steps per launch for the FP32 form with TMA-staged tiles: the temporally
// blocked fused stream-collide step of arXiv 2509.22308, Sec. III (Eq. LBGK equation with
// the equilibria of Eq. equilibrium distribution functions), one step deeper than
// step2_tma.cu.
//
// A persistent CTA walks 28 x 12 tiles (row-major, grid stride).  For each tile one thread
// issues two cp.async.bulk.tensor copies on one mbarrier: the 11 planes over the tile and a
// three-site halo (x from x0 - 4, the 16-byte boundary: 36 x 18 x 11 floats from y0 - 3)
// and the material ids over the same rows (48 bytes a row from x0 - 3 rounded down to 16).
//   phase 1: f*(t) of the tile and a two-site halo (32 x 16) from the stage into buffer 1;
//   then the stage is free and the next tile's copies go out;
//   phase 2: f*(t + 1) of the tile and a one-site halo (30 x 14) from buffer 1 into buffer 2;
//   phase 3: f*(t + 2) of the tile from buffer 2, stored to global memory.
// The tile shape keeps the halo work low (3.77 site updates per tile site per launch) and
// phase 1 at exactly two passes of the 256 threads.
// Each state element crosses HBM once per three steps (plus the halo rows, which
// neighbouring CTAs read at about the same time and L2 serves).  The per-site arithmetic is
// the one-step kernel's and every intermediate value stays FP32, so the result is
// bit-identical to three one-step launches.  Sites outside the lattice are skipped and
// pulls at the lattice edge clamp to the site itself, so the zeros the copy engine reads
// outside the tensor, and whatever a buffer holds outside the lattice, are never used.
#include <mutex>

#include "common.cuh"
#include "step2.cuh"
#include "step2_tma.h"
#include "tile_tma.cuh"

namespace lbmem {

namespace {

using namespace tma_tile;
constexpr int KW = kTma3TileW, KH = kTma3TileH;
constexpr int RW = KW + 8, RH = KH + 6;    // stage: x0 - 4 .. x0 + KW + 3, y0 - 3 .. y0 + KH + 2
constexpr int AW = KW + 4, AH = KH + 4;    // buffer 1: x0 - 2 .. x0 + KW + 1, y0 - 2 .. y0 + KH + 1
constexpr int BW = KW + 2, BH = KH + 2;    // buffer 2: x0 - 1 .. x0 + KW, y0 - 1 .. y0 + KH
constexpr int MW = (16 + KW + 4 + 15) / 16 * 16;  // id row: from x0 - 3 rounded down to 16 (offset <= 15)
static_assert(RW * sizeof(float) % 16 == 0 && MW % 16 == 0 && KW % 4 == 0, "TMA box rules");
constexpr unsigned STATE_BYTES = NPLANES * RH * RW * sizeof(float), ID_BYTES = MW * RH;
constexpr size_t r128(size_t b) { return (b + 127) / 128 * 128; }
constexpr size_t OFF_IDS = r128(STATE_BYTES);
constexpr size_t OFF_A = OFF_IDS + r128(ID_BYTES);
constexpr size_t OFF_B = OFF_A + (size_t)NPLANES * AH * AW * sizeof(float);
constexpr size_t OFF_TABLE = OFF_B + (size_t)NPLANES * BH * BW * sizeof(float);
constexpr size_t OFF_A_IDS = OFF_TABLE + 256 * sizeof(MatT<float>);
constexpr size_t OFF_B_IDS = OFF_A_IDS + (AW * AH + 15) / 16 * 16;
constexpr size_t kSmemBytes = OFF_B_IDS + (BW * BH + 15) / 16 * 16 + 128;  // + alignment slack
static_assert(OFF_B % 16 == 0 && OFF_TABLE % 16 == 0, "shared-memory layout");
static_assert(3 * (kSmemBytes + 1024 + 64) <= 233472, "three CTAs per SM");

// First column of a tile's id box: x0 - 3 rounded down to a multiple of 16.
__host__ __device__ __forceinline__ int id_box_x3(int x0) { return ((x0 - 3) >> 4) * 16; }

template <int W, int H>
__device__ __forceinline__ void put_buf(float *sm, int ly, int lx, const Pop<float> &p) {
    auto r = [&](int plane) -> float & { return sm[(plane * H + ly) * W + lx]; };
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

__device__ __forceinline__ void issue_tile3(const CUtensorMap *fmap, const CUtensorMap *imap, int x0, int y0,
                                            unsigned char *stage, uint64_t *bar) {
    mbar_arrive_expect_tx(bar, STATE_BYTES + ID_BYTES);
    tma_load_3d(stage, fmap, x0 - 4, y0 - 3, 0, bar);
    tma_load_2d(stage + OFF_IDS, imap, id_box_x3(x0), y0 - 3, bar);
}

// Source values of a launch's times t, t + 1, t + 2 in FP32 (g[0], inc[0] only for t >= 1).
struct SrcTripleF {
    float g[3], inc[3];
};
// Not inlined, called by one thread: see source_pair_f.
static __device__ __noinline__ SrcTripleF source_triple_f(const SourceParams src, long long t) {
    SrcTripleF v{{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    if (src.kind != SRC_NONE) {
        for (int k = 0; k < 3; ++k) {
            if (t + k < 1) continue;
            double g, inc;
            source_values(src, t + k, &g, &inc);
            v.g[k] = (float)g;
            v.inc[k] = (float)inc;
        }
    }
    return v;
}

template <bool ACC, int POL>
__global__ void __launch_bounds__(NTH, 3)
    k_step3_tma(const StepArgs<float> a, const __grid_constant__ CUtensorMap fin,
                const __grid_constant__ CUtensorMap ids_map, float *__restrict__ fout,
                const long long *__restrict__ t_in, long long *__restrict__ t_out, int ntx, int n_tiles) {
    extern __shared__ unsigned char sm_dyn[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ SrcTripleF sp;
    unsigned char *s = sm_dyn + ((128u - (smem_u32(sm_dyn) & 127u)) & 127u);
    const float *stage = reinterpret_cast<const float *>(s);
    const uint8_t *ids = s + OFF_IDS;
    float *bufa = reinterpret_cast<float *>(s + OFF_A);
    float *bufb = reinterpret_cast<float *>(s + OFF_B);
    MatT<float> *table = reinterpret_cast<MatT<float> *>(s + OFF_TABLE);
    uint8_t *ids_a = s + OFF_A_IDS;
    uint8_t *ids_b = s + OFF_B_IDS;

    const long long t = *t_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *t_out = t + 3;
    const int n_mine = (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // >= 1
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        sp = source_triple_f(a.src, t);
    }
    for (int k = threadIdx.x; k < 256; k += NTH) table[k] = a.mtab[k];
    __syncthreads();
    int tx = (int)blockIdx.x % ntx, ty = (int)blockIdx.x / ntx;
    const int sx = (int)gridDim.x % ntx, sy = (int)gridDim.x / ntx;
    if (threadIdx.x == 0) issue_tile3(&fin, &ids_map, tx * KW, ty * KH, s, &bar);
    const bool src0 = t >= 1 && a.src.kind != SRC_NONE, src12 = a.src.kind != SRC_NONE;
    const int nx = a.nx, ny = a.ny;

    for (int i = 0; i < n_mine; ++i) {
        const int x0 = tx * KW, y0 = ty * KH;
        const int ioff = x0 - 2 - id_box_x3(x0);  // column of site x0 - 2 in the id box
        const bool ok = mbar_wait(&bar, (unsigned)i & 1u);
        if (__syncthreads_or(!ok)) {  // the tile's copies never completed: report, leave
            if (threadIdx.x == 0) atomicOr(a.err, kErrTimeout);
            return;
        }
        // phase 1: time t at x0 - 2 + lx, y0 - 2 + ly
        for (int k = threadIdx.x; k < AW * AH; k += NTH) {
            const int lx = k % AW, ly = k / AW, x = x0 - 2 + lx, y = y0 - 2 + ly;
            if (x < 0 || x >= nx || y < 0 || y >= ny) continue;
            Pop<float> p;
            pull_buf<RW, RH>(stage, nx, ny, x, y, lx + 2, ly + 1, p);
            if (x == 0 && src0) inject_source_t(a.src.kind, sp.g[0], sp.inc[0], p);
            const uint8_t id = ids[(ly + 1) * MW + lx + ioff];
            const bool acc = ACC && lx >= 2 && lx < KW + 2 && ly >= 2 && ly < KH + 2;
            double f3[3];
            if (update_site<POL, true>(p, table[id], a.runaway, acc ? f3 : nullptr, nullptr)) atomicOr(a.err, kErrUnstable);
            if (acc) acc_site(a.accp, a.src, (size_t)y * a.pitch + x, y, t, f3[0], f3[1], f3[2]);
            put_buf<AW, AH>(bufa, ly, lx, p);
            ids_a[ly * AW + lx] = id;
        }
        __syncthreads();  // the stage is read, buffer 1 written
        tx += sx;         // the next tile of this CTA (grid stride, no division)
        ty += sy;
        if (tx >= ntx) {
            tx -= ntx;
            ++ty;
        }
        if (threadIdx.x == 0 && i + 1 < n_mine) {
            fence_proxy_async_smem();
            issue_tile3(&fin, &ids_map, tx * KW, ty * KH, s, &bar);
        }
        // phase 2: time t + 1 at x0 - 1 + lx, y0 - 1 + ly
        for (int k = threadIdx.x; k < BW * BH; k += NTH) {
            const int lx = k % BW, ly = k / BW, x = x0 - 1 + lx, y = y0 - 1 + ly;
            if (x < 0 || x >= nx || y < 0 || y >= ny) continue;
            Pop<float> p;
            pull_buf<AW, AH>(bufa, nx, ny, x, y, lx + 1, ly + 1, p);
            if (x == 0 && src12) inject_source_t(a.src.kind, sp.g[1], sp.inc[1], p);
            const uint8_t id = ids_a[(ly + 1) * AW + lx + 1];
            const bool acc = ACC && lx >= 1 && lx <= KW && ly >= 1 && ly <= KH;
            double f3[3];
            if (update_site<POL, true>(p, table[id], a.runaway, acc ? f3 : nullptr, nullptr)) atomicOr(a.err, kErrUnstable);
            if (acc) acc_site(a.accp, a.src, (size_t)y * a.pitch + x, y, t + 1, f3[0], f3[1], f3[2]);
            put_buf<BW, BH>(bufb, ly, lx, p);
            ids_b[ly * BW + lx] = id;
        }
        __syncthreads();  // buffer 1 is read, buffer 2 written
        // phase 3: time t + 2 on the tile
        for (int k = threadIdx.x; k < KW * KH; k += NTH) {
            const int lx = k % KW, ly = k / KW, x = x0 + lx, y = y0 + ly;
            if (x >= nx || y >= ny) continue;
            Pop<float> p;
            pull_buf<BW, BH>(bufb, nx, ny, x, y, lx + 1, ly + 1, p);
            if (x == 0 && src12) inject_source_t(a.src.kind, sp.g[2], sp.inc[2], p);
            const size_t idx = (size_t)y * a.pitch + x;
            double f3[3];
            if (update_site<POL, true>(p, table[ids_b[(ly + 1) * BW + lx + 1]], a.runaway, ACC ? f3 : nullptr, nullptr))
                atomicOr(a.err, kErrUnstable);
            if (ACC) acc_site(a.accp, a.src, idx, y, t + 2, f3[0], f3[1], f3[2]);
            store_site(fout, a.pstride, idx, p);
        }
        __syncthreads();  // buffers 1 and 2 are free for the next tile
    }
}

template <bool ACC, int POL>
cudaError_t allow_smem3() {
    return cudaFuncSetAttribute(k_step3_tma<ACC, POL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

}  // namespace

cudaError_t encode_step3_maps(CUtensorMap *fmap, const float *base, CUtensorMap *imap, const uint8_t *ids, int nx,
                              int ny, int pitch, size_t pstride) {
    if (((uintptr_t)base & 15u) || ((uintptr_t)ids & 15u) || (pitch % 16) || (pstride % 4))
        return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)NPLANES};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(float), (cuuint64_t)pstride * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)RW, (cuuint32_t)RH, (cuuint32_t)NPLANES};
    cudaError_t e = encode_tiled(fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box);
    if (e != cudaSuccess || !imap) return e;
    const cuuint64_t idims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t istrides[1] = {(cuuint64_t)pitch};
    const cuuint32_t ibox[2] = {(cuuint32_t)MW, (cuuint32_t)RH};
    return encode_tiled(imap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ids, idims, istrides, ibox);
}

cudaError_t step3_tma_prepare(int *max_ctas) {
    cudaError_t e = allow_smem3<false, POL_TM>();
    if (e == cudaSuccess) e = allow_smem3<true, POL_TM>();
    if (e == cudaSuccess) e = allow_smem3<false, POL_TE>();
    if (e == cudaSuccess) e = allow_smem3<true, POL_TE>();
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step3_tma<false, POL_TM>, NTH, kSmemBytes);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) *max_ctas = per_sm * sms;
    return e;
}

cudaError_t launch_step3_tma(const StepArgs<float> &a, const CUtensorMap *fin, const CUtensorMap *ids, float *fout,
                             const long long *t_in, long long *t_out, bool accumulate, int max_ctas, cudaStream_t s) {
    const int ntx = (a.nx + KW - 1) / KW, nty = (a.ny + KH - 1) / KH, n_tiles = ntx * nty;
    const int grid = n_tiles < max_ctas ? n_tiles : max_ctas;
    if (a.pol == POL_TE) {
        if (accumulate)
            k_step3_tma<true, POL_TE><<<grid, NTH, kSmemBytes, s>>>(a, *fin, *ids, fout, t_in, t_out, ntx, n_tiles);
        else
            k_step3_tma<false, POL_TE><<<grid, NTH, kSmemBytes, s>>>(a, *fin, *ids, fout, t_in, t_out, ntx, n_tiles);
    } else {
        if (accumulate)
            k_step3_tma<true, POL_TM><<<grid, NTH, kSmemBytes, s>>>(a, *fin, *ids, fout, t_in, t_out, ntx, n_tiles);
        else
            k_step3_tma<false, POL_TM><<<grid, NTH, kSmemBytes, s>>>(a, *fin, *ids, fout, t_in, t_out, ntx, n_tiles);
    }
    return cudaGetLastError();
}

}  // namespace lbmem
