// The tile of the TMA-staged two-steps-per-launch FP32 kernels (single-domain in
// step2_tma.cu, batched in batch.cu): geometry, shared-memory layout and the per-site
// helpers both use.
//
// A tile is KW x KH sites at (x0, y0) (two shapes, Geo below).  Its stage holds the 11 planes over the tile and a
// two-site halo, x0 - 4 .. x0 + KW + 3 and y0 - 2 .. y0 + KH + 1 (RW x RH floats per
// plane; the box starts at x0 - 4 so that it begins on a 16-byte boundary), and the
// material ids over the same rows from x0 - 2 rounded down to 16 bytes (MW bytes per row).  Phase 1 writes the
// post-collision state of the tile and a one-site halo, x0 - 1 .. x0 + KW and y0 - 1 ..
// y0 + KH (IW x IH), with each site's id, to the intermediate buffer.
#pragma once

#include "common.cuh"
#include "step2_tma.h"
#include "tma.cuh"

namespace lbmem {
namespace tma_tile {

constexpr int NTH = kTmaThreads;

// First column of a tile's id box: x0 - 2 rounded down to a multiple of 16 (a TMA box starts
// on a 16-byte boundary), so the box reaches x0 - 2 .. x0 + KW + 1 from an offset of 2 .. 17.
__host__ __device__ __forceinline__ int id_box_x(int x0) { return ((x0 - 2) >> 4) * 16; }

// Geometry of a KW_ x KH_ tile (KW_ a multiple of 4, so that x0 - 4 floats starts on 16
// bytes): the stage holds x0 - 4 .. x0 + KW + 3 and y0 - 2 .. y0 + KH + 1 (RW x RH), the id box
// MW bytes from id_box_x(x0) on the stage's rows, the intermediate buffer x0 - 1 .. x0 + KW
// and y0 - 1 .. y0 + KH (IW x IH).
template <int KW_, int KH_>
struct Geo {
    static constexpr int KW = KW_, KH = KH_;
    static constexpr int RW = KW + 8, RH = KH + 4, IW = KW + 2, IH = KH + 2;
    static constexpr int MW = (17 + KW + 2 + 15) / 16 * 16;
    static_assert(RW * sizeof(float) % 16 == 0 && MW % 16 == 0, "TMA box rows must be multiples of 16 bytes");
    static_assert(KW % 4 == 0, "x0 - 4 floats must start on a 16-byte boundary");
    static constexpr int STATE_FLOATS = NPLANES * RH * RW;
    static constexpr unsigned STATE_BYTES = STATE_FLOATS * sizeof(float), ID_BYTES = MW * RH;
    static constexpr size_t OFF_IDS = (STATE_BYTES + 127) / 128 * 128;          // 128-byte aligned
    static constexpr size_t OFF_INTER = OFF_IDS + (ID_BYTES + 127) / 128 * 128;  // intermediate state
    static constexpr size_t OFF_TABLE = OFF_INTER + (size_t)NPLANES * IH * IW * sizeof(float);
    static constexpr size_t OFF_INTER_IDS = OFF_TABLE + 256 * sizeof(MatT<float>);
    static constexpr size_t kSmemBytes = OFF_INTER_IDS + (IW * IH + 15) / 16 * 16 + 128;  // + slack
    static_assert(STATE_BYTES % 16 == 0 && OFF_TABLE % 16 == 0, "shared-memory layout");
    static_assert(3 * (kSmemBytes + 1024 + 64) <= 233472, "three CTAs per SM");
};
// The single-domain kernel's tile, and the other shapes the batch autotuner also times
// (instance sizes that are multiples of 32, or of 40, but not of 64 fill them without idle
// columns: the paper's 160^2 and 200^2 maps).
using GeoWide = Geo<kTmaTileW, kTmaTileH>;
using GeoTall = Geo<32, 16>;
using GeoMid = Geo<40, 12>;

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

template <class G>
__device__ __forceinline__ void put_inter(float *sm, int ly, int lx, const Pop<float> &p) {
    auto r = [&](int plane) -> float & { return sm[(plane * G::IH + ly) * G::IW + lx]; };
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

// The copies of the tile at (x0, y0): state box and id box, completing on bar.
template <class G>
__device__ __forceinline__ void issue_tile(const CUtensorMap *fmap, const CUtensorMap *imap, int x0, int y0,
                                           unsigned char *stage, uint64_t *bar) {
    mbar_arrive_expect_tx(bar, G::STATE_BYTES + G::ID_BYTES);
    tma_load_3d(stage, fmap, x0 - 4, y0 - 2, 0, bar);
    tma_load_2d(stage + G::OFF_IDS, imap, id_box_x(x0), y0 - 2, bar);
}

// Source values of a launch's two times t and t + 1 in FP32 (g0, inc0 only for t >= 1).
struct SrcPairF {
    float g0, inc0, g1, inc1;
};
// Not inlined on purpose: inlined under a one-thread test, the compiler predicated the
// double-precision evaluation into every thread of the block, and on GB300's narrow FP64
// pipe that cost 15 % of the FP32 kernel's time.  Called by one thread.
static __device__ __noinline__ SrcPairF source_pair_f(const SourceParams src, long long t) {
    SrcPairF v{0.f, 0.f, 0.f, 0.f};
    if (src.kind != SRC_NONE) {
        double g, inc;
        if (t >= 1) {
            source_values(src, t, &g, &inc);
            v.g0 = (float)g;
            v.inc0 = (float)inc;
        }
        source_values(src, t + 1, &g, &inc);
        v.g1 = (float)g;
        v.inc1 = (float)inc;
    }
    return v;
}

// The regions of the dynamic shared memory (aligned to 128 bytes here).
struct TileSmem {
    unsigned char *stage;  // state box, then id box
    const float *raw;
    const uint8_t *ids;
    float *inter;
    MatT<float> *table;
    uint8_t *inter_ids;
};
template <class G>
__device__ __forceinline__ TileSmem carve(unsigned char *sm_dyn) {
    unsigned char *s = sm_dyn + ((128u - (smem_u32(sm_dyn) & 127u)) & 127u);
    return TileSmem{s,
                    reinterpret_cast<const float *>(s),
                    s + G::OFF_IDS,
                    reinterpret_cast<float *>(s + G::OFF_INTER),
                    reinterpret_cast<MatT<float> *>(s + G::OFF_TABLE),
                    s + G::OFF_INTER_IDS};
}

}  // namespace tma_tile
}  // namespace lbmem
