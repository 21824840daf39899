// Two time steps per launch for the FP16-deviation storage form with TMA-staged tiles:
// the temporally blocked fused stream-collide step of arXiv 2509.22308, Sec. III (Eq. LBGK
// equation, Eq. equilibrium distribution functions), on this form's layout (step_f16.cuh:
// 11 FP16 deviation planes and 3 FP32 field planes per buffer).
//
// The CTA walks 64 x 8 tiles as the FP32 kernel of step2_tma.cu does.  For each tile one
// thread issues three cp.async.bulk.tensor copies on one mbarrier: the deviations over the
// tile and a two-site halo (x from x0 - 8, so that the box starts on a 16-byte boundary:
// 80 x 12 x 11 halves), the fields over the same rows (x from x0 - 4: 72 x 12 x 3 floats)
// and the material ids (the FP32 kernel's id box).
//   phase 1: f(t) of the tile and a one-site halo rebuilt from the staged deviations and
//            the upstream sites' fields, source at x = 0, moments; the intermediate buffer
//            receives what a pull would rebuild from the state this site stores for t (its
//            fields, its deviations rounded to FP16), so the launch equals two one-step
//            launches bit for bit;
//   then the stage is free and the next tile's copies go out;
//   phase 2: f(t + 1) of the tile pulled from the intermediate buffer, moments, and the
//            fields and FP16 deviations of t + 1 stored to global memory.
// Each state byte crosses HBM once per two steps (34 B read and 34 B written per site,
// plus the halo that L2 serves), against once per step for k_step_f16.
#include <cuda_fp16.h>

#include "common.cuh"
#include "step2.cuh"
#include "step2_tma.h"
#include "step_f16.cuh"
#include "tile_tma.cuh"

namespace lbmem {

namespace {

using namespace tma_tile;
using G = GeoWide;  // the tile, its intermediate buffer and its id box
constexpr int KW = G::KW, KH = G::KH, RH = G::RH, IW = G::IW, IH = G::IH, MW = G::MW;
constexpr int HW = KW + 16;  // halves per staged row: x0 - 8 .. x0 + KW + 7
constexpr int FW = KW + 8;   // floats per staged row: x0 - 4 .. x0 + KW + 3
constexpr int kFields = 3;
constexpr unsigned HALF_BYTES = NPLANES * RH * HW * 2, FLD_BYTES = kFields * RH * FW * 4;
constexpr size_t round128(size_t b) { return (b + 127) / 128 * 128; }
constexpr size_t OFF_FLD = round128(HALF_BYTES);
constexpr size_t OFF_IDS = OFF_FLD + round128(FLD_BYTES);
constexpr size_t OFF_INTER = OFF_IDS + round128(G::ID_BYTES);
constexpr size_t OFF_TABLE = OFF_INTER + (size_t)NPLANES * IH * IW * sizeof(float);
constexpr size_t OFF_INTER_IDS = OFF_TABLE + 256 * sizeof(MatT<float>);
constexpr size_t kSmemBytes = OFF_INTER_IDS + (IW * IH + 15) / 16 * 16 + 128;  // + alignment slack
static_assert(HW * 2 % 16 == 0 && FW * 4 % 16 == 0, "TMA box rows must be multiples of 16 bytes");
static_assert(KW % 8 == 0, "x0 - 8 halves must start on a 16-byte boundary");
static_assert(OFF_TABLE % 16 == 0, "shared-memory layout");
static_assert(3 * (kSmemBytes + 1024 + 64) <= 233472, "three CTAs per SM");

// The copies of the tile at (x0, y0): deviations, fields and ids, completing on bar.
__device__ __forceinline__ void issue_f16_tile(const CUtensorMap *gmap, const CUtensorMap *fmap,
                                               const CUtensorMap *imap, int x0, int y0, unsigned char *s,
                                               uint64_t *bar) {
    mbar_arrive_expect_tx(bar, HALF_BYTES + FLD_BYTES + G::ID_BYTES);
    tma_load_3d(s, gmap, x0 - 8, y0 - 2, 0, bar);
    tma_load_3d(s + OFF_FLD, fmap, x0 - 4, y0 - 2, 0, bar);
    tma_load_2d(s + OFF_IDS, imap, id_box_x(x0), y0 - 2, bar);
}

// f_i(r, t) of the site at staged row ry, staged half column hx and staged float column fx
// (the same site), rebuilt from the upstream sites' stored fields and deviations exactly as
// pull_f16_planes does from global memory; the upstream site clamps at the lattice edge.
__device__ __forceinline__ void pull_staged(const __half *sg, const float *sf, int nx, int ny, int x, int y,
                                            int ry, int hx, int fx, float is, Pop<float> &p) {
    const int dxm = x > 0 ? -1 : 0, dxp = x < nx - 1 ? 1 : 0;
    const int rym = y > 0 ? ry - 1 : ry, ryp = y < ny - 1 ? ry + 1 : ry;
    auto fld = [&](int row, int col) {
        return Fld{sf[row * FW + col], sf[(RH + row) * FW + col], sf[(2 * RH + row) * FW + col]};
    };
    auto dev = [&](int plane, int row, int col) { return sg[(plane * RH + row) * HW + col]; };
    const Fld c = fld(ry, fx), w = fld(ry, fx + dxm), e = fld(ry, fx + dxp);
    const Fld so = fld(rym, fx), no = fld(ryp, fx);
    p.ez = rebuild(c.e, dev(P_EZ, ry, hx), is);
    p.epx = rebuild(eq2_epx(w.e, w.hx, w.hy), dev(P_EPX, ry, hx + dxm), is);
    p.emx = rebuild(eq2_emx(e.e, e.hx, e.hy), dev(P_EMX, ry, hx + dxp), is);
    p.epy = rebuild(eq2_epy(so.e, so.hx, so.hy), dev(P_EPY, rym, hx), is);
    p.emy = rebuild(eq2_emy(no.e, no.hx, no.hy), dev(P_EMY, ryp, hx), is);
    p.hxpx = rebuild(w.hx, dev(P_HXPX, ry, hx + dxm), is);
    p.hxmx = rebuild(e.hx, dev(P_HXMX, ry, hx + dxp), is);
    p.hxz = rebuild(c.hx, dev(P_HXZ, ry, hx), is);
    p.hypy = rebuild(so.hy, dev(P_HYPY, rym, hx), is);
    p.hymy = rebuild(no.hy, dev(P_HYMY, ryp, hx), is);
    p.hyz = rebuild(c.hy, dev(P_HYZ, ry, hx), is);
}

template <bool ACC>
__global__ void __launch_bounds__(NTH, 3)
    k_step2_f16_tma(const F16Args a, const __grid_constant__ CUtensorMap gmap, const __grid_constant__ CUtensorMap fmap,
                    const __grid_constant__ CUtensorMap ids_map, const long long *__restrict__ t_in,
                    long long *__restrict__ t_out, int ntx, int n_tiles) {
    extern __shared__ unsigned char sm_dyn[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ SrcPairF sp;
    unsigned char *s = sm_dyn + ((128u - (smem_u32(sm_dyn) & 127u)) & 127u);
    const __half *sg = reinterpret_cast<const __half *>(s);
    const float *sf = reinterpret_cast<const float *>(s + OFF_FLD);
    const uint8_t *sids = s + OFF_IDS;
    float *inter = reinterpret_cast<float *>(s + OFF_INTER);
    MatT<float> *table = reinterpret_cast<MatT<float> *>(s + OFF_TABLE);
    uint8_t *inter_ids = s + OFF_INTER_IDS;

    const long long t = *t_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *t_out = t + 2;
    const int n_mine = (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // >= 1
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        sp = source_pair_f(a.src, t);
    }
    for (int k = threadIdx.x; k < 256; k += NTH) table[k] = a.mtab[k];
    __syncthreads();
    int tx = (int)blockIdx.x % ntx, ty = (int)blockIdx.x / ntx;
    const int sx = (int)gridDim.x % ntx, sy = (int)gridDim.x / ntx;
    if (threadIdx.x == 0) issue_f16_tile(&gmap, &fmap, &ids_map, tx * KW, ty * KH, s, &bar);
    const bool src0 = t >= 1 && a.src.kind != SRC_NONE, src1 = a.src.kind != SRC_NONE;
    const int nx = a.nx, ny = a.ny;
    const float is = a.inv_scale, sc = a.scale;
    const size_t ps = a.pstride;

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
            pull_staged(sg, sf, nx, ny, x, y, ly + 1, lx + 7, lx + 3, is, p);
            if (x == 0 && src0) inject_source_t(a.src.kind, sp.g0, sp.inc0, p);
            const uint8_t id = sids[(ly + 1) * MW + lx + ioff];
            float E3, Hx, Hy, D;
            moments(p, table[id], &E3, &Hx, &Hy, &D);
            if (field_runaway(E3, a.runaway)) atomicOr(a.err, kErrUnstable);
            if (ACC && lx >= 1 && lx <= KW && ly >= 1 && ly <= KH)
                acc_site(a.accp, a.src, (size_t)y * a.pitch + x, y, t, 3.0 * (double)E3, (double)Hx, (double)Hy);
            const Fld F = stored_fields(E3, Hx, Hy);
            __half g[NPLANES];
            encode_all(p, F, sc, g);
            Pop<float> q;
            rebuild_all(g, F, is, q);
            put_inter<G>(inter, ly, lx, q);
            inter_ids[ly * IW + lx] = id;
        }
        __syncthreads();  // the stage is read, the intermediate state written
        tx += sx;         // the next tile of this CTA (grid stride, no division)
        ty += sy;
        if (tx >= ntx) {
            tx -= ntx;
            ++ty;
        }
        if (threadIdx.x == 0 && i + 1 < n_mine) {
            fence_proxy_async_smem();
            issue_f16_tile(&gmap, &fmap, &ids_map, tx * KW, ty * KH, s, &bar);
        }
        for (int k = threadIdx.x; k < KW * KH; k += NTH) {
            const int lx = k % KW, ly = k / KW, x = x0 + lx, y = y0 + ly;
            if (x >= nx || y >= ny) continue;
            Pop<float> p;
            pull_buf<IW, IH>(inter, nx, ny, x, y, lx + 1, ly + 1, p);
            if (x == 0 && src1) inject_source_t(a.src.kind, sp.g1, sp.inc1, p);
            const size_t idx = (size_t)y * a.pitch + x;
            float E3, Hx, Hy, D;
            moments(p, table[inter_ids[(ly + 1) * IW + lx + 1]], &E3, &Hx, &Hy, &D);
            if (field_runaway(E3, a.runaway)) atomicOr(a.err, kErrUnstable);
            if (ACC) acc_site(a.accp, a.src, idx, y, t + 1, 3.0 * (double)E3, (double)Hx, (double)Hy);
            const Fld F = stored_fields(E3, Hx, Hy);
            __half g[NPLANES];
            encode_all(p, F, sc, g);
#pragma unroll
            for (int q = 0; q < NPLANES; ++q) a.g_out[q * ps + idx] = g[q];
            a.fe_out[idx] = F.e;
            a.fhx_out[idx] = F.hx;
            a.fhy_out[idx] = F.hy;
        }
        __syncthreads();  // the intermediate buffer is free for the next tile
    }
}

template <bool ACC>
cudaError_t allow_smem() {
    return cudaFuncSetAttribute(k_step2_f16_tma<ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

}  // namespace

cudaError_t encode_f16_maps(CUtensorMap *gmap, CUtensorMap *fmap, const void *buf, int nx, int ny, int pitch,
                            size_t pstride) {
    const size_t hb = f16_half_bytes(pstride), fb = f16_plane_bytes(pstride);
    if (((uintptr_t)buf & 15u) || (pitch % 8) || (pstride % 8) || (fb % 16)) return cudaErrorInvalidValue;
    const cuuint64_t gdims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)NPLANES};
    const cuuint64_t gstrides[2] = {(cuuint64_t)pitch * 2, (cuuint64_t)pstride * 2};
    const cuuint32_t gbox[3] = {(cuuint32_t)HW, (cuuint32_t)RH, (cuuint32_t)NPLANES};
    cudaError_t e = encode_tiled(gmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, buf, gdims, gstrides, gbox);
    if (e != cudaSuccess) return e;
    const cuuint64_t fdims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)kFields};
    const cuuint64_t fstrides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)fb};
    const cuuint32_t fbox[3] = {(cuuint32_t)FW, (cuuint32_t)RH, (cuuint32_t)kFields};
    return encode_tiled(fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (const char *)buf + hb, fdims, fstrides, fbox);
}

cudaError_t step2_f16_tma_prepare(int *max_ctas) {
    cudaError_t e = allow_smem<false>();
    if (e == cudaSuccess) e = allow_smem<true>();
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step2_f16_tma<false>, NTH, kSmemBytes);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) *max_ctas = per_sm * sms;
    return e;
}

cudaError_t launch_step2_f16_tma(const F16Args &a, const CUtensorMap *gmap, const CUtensorMap *fmap,
                                 const CUtensorMap *ids, const long long *t_in, long long *t_out, bool accumulate,
                                 int max_ctas, cudaStream_t s) {
    const int ntx = (a.nx + KW - 1) / KW, nty = (a.ny + KH - 1) / KH, n_tiles = ntx * nty;
    const int grid = n_tiles < max_ctas ? n_tiles : max_ctas;
    if (accumulate)
        k_step2_f16_tma<true><<<grid, NTH, kSmemBytes, s>>>(a, *gmap, *fmap, *ids, t_in, t_out, ntx, n_tiles);
    else
        k_step2_f16_tma<false><<<grid, NTH, kSmemBytes, s>>>(a, *gmap, *fmap, *ids, t_in, t_out, ntx, n_tiles);
    return cudaGetLastError();
}

}  // namespace lbmem
