// Four time steps per launch for the FP32 and FP16-deviation forms: the fused stream-collide
// step of arXiv 2509.22308, Sec. III (Eq. LBGK equation, Eq. equilibrium distribution
// functions), temporally blocked in registers along a streaming row sweep.
//
// Work unit: one warp, a strip of 64 columns (two sites per lane) and a segment of rows.  The
// strip's 56 inner columns are its output; the 4 columns on each side are the halo that four
// steps consume (a site's value after k steps needs its neighbours after k - 1, so the valid
// width shrinks by one column per side and step).  The warp walks down its rows: each row of
// the stored state (time t - 1) arrives in shared memory through one cp.async.bulk.tensor copy
// into a per-warp ring of row slots and goes straight into registers.  Time level k + 1 of row
// q needs level k of rows q - 1, q and q + 1, so after row i has arrived the warp computes
// level 1 of row i - 1, level 2 of row i - 2, level 3 of row i - 3 and level 4 of row i - 4,
// and stores that one: a wavefront over (row, time).  Per level the registers keep the newest
// row the next level still needs (9 of its populations) and the +y pair of the row before.
// Neighbours along x come from the adjacent lane by warp shuffles, neighbours along y from
// these registers.  No thread-block barrier is taken after the start: each warp waits only
// for its own row copies (bounded waits, as in the tile kernels).
//
// The per-site arithmetic is the one-step kernel's (update_site), so the FP32 form gives the
// bits of four one-step launches.  The FP16-deviation form rebuilds the stored state (fields
// and FP16 deviations) into FP32 post-collision populations as level 0 reads it, runs levels
// 1-3 in FP32 and stores the fields and deviations of level 4: its state is rounded to FP16
// once per launch instead of once per step, so it differs from one step per launch by FP16
// rounding noise.
//
// Each state element crosses HBM once per four steps: 89 B per four FP32 updates, 69 B per
// four FP16-deviation updates, plus the 8 halo columns of every 56 that the neighbouring
// strips also read (served by L2 when they run at about the same time).
//
// Accumulating launches (the Fourier sums of the last period, Sec. III) store the FP32 fields
// of the contour's stencil sites at each level into a staging buffer; a one-thread-per-slot
// flush adds them to the FP64 sums after the launch (k_stage_flush; k_batch_flush4 for the
// batch, whose kernel k_batch_step4 runs the same work unit over the packed instances of a
// design map).
#include <cuda_fp16.h>

#include <climits>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "step2_tma.h"
#include "step_f16.cuh"
#include "step_stream.h"
#include "tma.cuh"

namespace lbmem {

namespace {

constexpr int LW = kStreamLoadW, HALO = kStreamHalo, OUTW = kStreamOutW, NW = kStreamWarps, BT = kStreamSteps;
constexpr int IDBOX = 80;                      // id bytes per row copy (from a 16-byte boundary)
constexpr unsigned ROW32 = NPLANES * LW * 4;   // FP32 state row: 11 planes x 64 floats
// FP16 deviations row: 11 planes x 72 halves from 4 columns before the strip, because a
// copy of 2-byte elements must start on a multiple of 8 elements (16 bytes)
constexpr int DEVW = LW + 8, DEVOFF = 4;
constexpr unsigned ROWDEV = NPLANES * DEVW * 2;
constexpr unsigned ROWFLD = 3 * LW * 4;        // FP32 fields row: 3 planes x 64 floats
constexpr size_t r128(size_t b) { return (b + 127) / 128 * 128; }
static_assert(LW == 64 && OUTW + 2 * HALO == LW && HALO % 4 == 0 && HALO >= BT,
              "two sites per lane, a 16-byte aligned halo as wide as the steps");
static_assert(IDBOX >= LW + 12 && IDBOX % 16 == 0, "the id box covers the strip from any 16-byte boundary");

// Shared memory: the material table, then per warp RING row slots (state row, id row) and the
// -y pairs of the last lattice row per level (the bottom edge, see below).  Level 0 (the stored
// state) is read straight from the slots, so a row's slot stays in use until the row two further
// on has arrived: 5 slots, 3 rows in use and 2 in flight.  The FP16-deviation form's copies
// (deviations, then fields) fill the first 2432 bytes of the slot.  With the mixed-precision
// rebuild (|E0| >= 2^-14) level 0 reads them as they are and rebuilds each population where it
// reads it; otherwise, on arrival, each lane rebuilds its two sites into FP32 populations and
// writes them over the slot in the FP32 row layout, which level 0 then reads as in FP32.
template <bool F16>
struct Layout {
    static constexpr int RING = 5;
    static constexpr size_t FLD = r128(ROWDEV);  // FP16 form: the field row, 128-byte aligned
    static_assert(FLD + ROWFLD <= ROW32, "the FP16 copies fit under the FP32 row they are rebuilt into");
    static constexpr size_t IDS = r128(ROW32);
    static constexpr size_t SLOT = IDS + 128;
    static constexpr size_t EDGE = BT * 32 * sizeof(float4);
    static constexpr size_t WARP = RING * SLOT + EDGE;
    static constexpr size_t TABLE = 256 * sizeof(MatT<float>);
    static constexpr size_t SMEM = TABLE + NW * WARP + 128;  // + alignment slack
};
static_assert(3 * (Layout<false>::SMEM + 1024 + 256) <= 233472 && 3 * (Layout<true>::SMEM + 1024 + 256) <= 233472,
              "three blocks per SM");

// Not inlined, called by one thread: see source_pair_f.
static __device__ __noinline__ SrcLevels source_levels_f(const SourceParams src, long long t) {
    SrcLevels v;
    for (int k = 0; k < BT; ++k) v.g[k] = v.inc[k] = 0.f;
    if (src.kind != SRC_NONE) {
        for (int k = 0; k < BT; ++k) {
            if (t + k < 1) continue;
            double g, inc;
            source_values(src, t + k, &g, &inc);
            v.g[k] = (float)g;
            v.inc[k] = (float)inc;
        }
    }
    return v;
}

// The nine populations of a row that the next level reads at the row itself or from its x
// neighbours, for this lane's sites A (even column, [0]) and B (odd column, [1]).  The +y
// pair is read one row further down, the -y pair one row further up (not kept).
struct Row9 {
    float ez[2], epx[2], emx[2], epy[2], hxpx[2], hxmx[2], hxz[2], hypy[2], hyz[2];
};

__device__ __forceinline__ void keep_row(Row9 &r, const Pop<float> &a, const Pop<float> &b) {
    r.ez[0] = a.ez, r.ez[1] = b.ez;
    r.epx[0] = a.epx, r.epx[1] = b.epx;
    r.emx[0] = a.emx, r.emx[1] = b.emx;
    r.epy[0] = a.epy, r.epy[1] = b.epy;
    r.hxpx[0] = a.hxpx, r.hxpx[1] = b.hxpx;
    r.hxmx[0] = a.hxmx, r.hxmx[1] = b.hxmx;
    r.hxz[0] = a.hxz, r.hxz[1] = b.hxz;
    r.hypy[0] = a.hypy, r.hypy[1] = b.hypy;
    r.hyz[0] = a.hyz, r.hyz[1] = b.hyz;
}

// f_i(q, next time) of sites A and B of this lane from the post-collision values of row q
// (cur), the +y pair of row q - 1 (ey, hy) and the -y pair of row q + 1 (my, mh).  Along x
// the upstream site is the adjacent one (across lanes by shuffles), or the site itself at
// the lattice edge (the zero-gradient open edge).
__device__ __forceinline__ void pull_row(const Row9 &cur, const float ey[2], const float hy[2], const float my[2],
                                         const float mh[2], bool xa0, bool xa_last, bool xb_last, Pop<float> &a,
                                         Pop<float> &b) {
    const unsigned full = 0xffffffffu;
    const float l_epx = __shfl_up_sync(full, cur.epx[1], 1);    // site B of the lane to the left
    const float l_hxpx = __shfl_up_sync(full, cur.hxpx[1], 1);
    const float r_emx = __shfl_down_sync(full, cur.emx[0], 1);  // site A of the lane to the right
    const float r_hxmx = __shfl_down_sync(full, cur.hxmx[0], 1);
    a.ez = cur.ez[0];
    a.hxz = cur.hxz[0];
    a.hyz = cur.hyz[0];
    a.epx = xa0 ? cur.epx[0] : l_epx;
    a.hxpx = xa0 ? cur.hxpx[0] : l_hxpx;
    a.emx = xa_last ? cur.emx[0] : cur.emx[1];
    a.hxmx = xa_last ? cur.hxmx[0] : cur.hxmx[1];
    a.epy = ey[0];
    a.hypy = hy[0];
    a.emy = my[0];
    a.hymy = mh[0];
    b.ez = cur.ez[1];
    b.hxz = cur.hxz[1];
    b.hyz = cur.hyz[1];
    b.epx = cur.epx[0];
    b.hxpx = cur.hxpx[0];
    b.emx = xb_last ? cur.emx[1] : r_emx;
    b.hxmx = xb_last ? cur.hxmx[1] : r_hxmx;
    b.epy = ey[1];
    b.hypy = hy[1];
    b.emy = my[1];
    b.hymy = mh[1];
}

// One plane of a staged FP32 row: the lane's two sites.
__device__ __forceinline__ float2 lds2(const float *row, int plane, int lane) {
    return reinterpret_cast<const float2 *>(row + plane * LW)[lane];
}

template <bool F16>
__device__ __forceinline__ void issue_row(const CUtensorMap *smap, const CUtensorMap *fmap, const CUtensorMap *imap,
                                          int xs, int xid, int r, unsigned char *slot, uint64_t *bar) {
    if constexpr (F16) {
        mbar_arrive_expect_tx(bar, ROWDEV + ROWFLD + IDBOX);
        tma_load_3d(slot, smap, xs - DEVOFF, r, 0, bar);  // xs - 4: a multiple of 8 halves
        tma_load_3d(slot + Layout<F16>::FLD, fmap, xs, r, 0, bar);
    } else {
        mbar_arrive_expect_tx(bar, ROW32 + IDBOX);
        tma_load_3d(slot, smap, xs, r, 0, bar);
    }
    tma_load_2d(slot + Layout<F16>::IDS, imap, xid, r, bar);
}

struct StreamArgs {
    int nx, ny, pitch, n_strips, seg_rows, n_units;
    size_t pstride;
    const MatT<float> *mtab;
    SourceParams src;
    unsigned *err;
    unsigned runaway;
    float scale, inv_scale;       // FP16-deviation form
    float *fout;                  // FP32 form: 11 planes
    __half *g_out;                // FP16-deviation form: 11 deviation planes, 3 field planes
    float *fe_out, *fhx_out, *fhy_out;
};

__device__ __forceinline__ void store2(float *p, bool two, float a, float b) {
    if (two)
        *reinterpret_cast<float2 *>(p) = make_float2(a, b);
    else
        *p = a;
}

// Time levels 1..3 of the wavefront: per level the kept row (row i - 1 - k when row i arrives,
// 9 populations), the +y pair of the row before it, and the ids of row i - 1 - k.  Level 0 lives
// in the ring; index 0 of these arrays is unused.
struct Wave {
    Row9 cur[BT];
    float oe[BT][2], oh[BT][2];
    unsigned ids[BT];
};

// The stored fields of a lane's two sites in an FP16-deviation row slot, one of its deviation
// pairs, and a plane's two rebuilt populations f* = eq2 / 2 + g nis (rebuild_h, step_f16.cuh).
struct Fld2 {
    float2 e, hx, hy;
};
__device__ __forceinline__ Fld2 slot_fields(const unsigned char *sl, int lane) {
    const float2 *fl = reinterpret_cast<const float2 *>(sl + Layout<true>::FLD);
    return Fld2{fl[lane], fl[LW / 2 + lane], fl[LW + lane]};
}
__device__ __forceinline__ unsigned slot_dev(const unsigned char *sl, int plane, int lane) {
    return reinterpret_cast<const unsigned *>(reinterpret_cast<const __half *>(sl) + DEVOFF + plane * DEVW)[lane];
}
__device__ __forceinline__ void rebuild2(float eq2a, float eq2b, unsigned g2, unsigned short nis, float o[2]) {
    o[0] = rebuild_h<false>(eq2a, g2, nis);
    o[1] = rebuild_h<true>(eq2b, g2, nis);
}

// One row of level 0 from a slot: FP32 as staged; FP16-deviation rebuilt in place first (see
// Layout) by converting each deviation (inv_scale = 2^(k - 10)), unless MIX: then the level-0
// reads rebuild each population with the mixed-precision FMA (slot_fields, slot_dev below).
template <bool F16, bool MIX>
__device__ __forceinline__ void take_row(unsigned char *sl, int lane, float inv_scale) {
    if constexpr (F16 && !MIX) {
        const __half *dv = reinterpret_cast<const __half *>(sl) + DEVOFF;
        const float *fl = reinterpret_cast<const float *>(sl + Layout<F16>::FLD);
        const float2 fe = reinterpret_cast<const float2 *>(fl)[lane];
        const float2 fhx = reinterpret_cast<const float2 *>(fl + LW)[lane];
        const float2 fhy = reinterpret_cast<const float2 *>(fl + 2 * LW)[lane];
        // the post-collision populations of the stored state: f* = f^eq - g
        Pop<float> na, nb;
        __half ga[NPLANES], gb[NPLANES];
#pragma unroll
        for (int p = 0; p < NPLANES; ++p) {
            const __half2 g2 = reinterpret_cast<const __half2 *>(dv + p * DEVW)[lane];
            ga[p] = __low2half(g2);
            gb[p] = __high2half(g2);
        }
        rebuild_all(ga, Fld{fe.x, fhx.x, fhy.x}, inv_scale, na);
        rebuild_all(gb, Fld{fe.y, fhx.y, fhy.y}, inv_scale, nb);
        __syncwarp();  // every lane has read the copies before any lane overwrites them
        float2 *row = reinterpret_cast<float2 *>(sl);
        row[P_EZ * 32 + lane] = make_float2(na.ez, nb.ez);
        row[P_EPX * 32 + lane] = make_float2(na.epx, nb.epx);
        row[P_EMX * 32 + lane] = make_float2(na.emx, nb.emx);
        row[P_EPY * 32 + lane] = make_float2(na.epy, nb.epy);
        row[P_EMY * 32 + lane] = make_float2(na.emy, nb.emy);
        row[P_HXPX * 32 + lane] = make_float2(na.hxpx, nb.hxpx);
        row[P_HXMX * 32 + lane] = make_float2(na.hxmx, nb.hxmx);
        row[P_HXZ * 32 + lane] = make_float2(na.hxz, nb.hxz);
        row[P_HYPY * 32 + lane] = make_float2(na.hypy, nb.hypy);
        row[P_HYMY * 32 + lane] = make_float2(na.hymy, nb.hymy);
        row[P_HYZ * 32 + lane] = make_float2(na.hyz, nb.hyz);
        // each lane reads back only its own two sites (neighbours come by shuffles)
    }
}

// What a warp needs of the lattice it works on: sizes, outputs and (ACC) the Fourier
// accumulation of times acc_from <= t' < steps at the rows ay0 .. ay1.  The single-domain
// kernel receives it as a grid-constant parameter, so its fields are read from the constant
// bank instead of taking registers; the batch kernel keeps the current instance's in shared
// memory.
struct UnitCtx {
    int nx, ny, pitch, kind;
    unsigned runaway;
    int ay0, ay1, period;
    size_t pstride;
    float scale, inv_scale;                       // FP16-deviation form
    unsigned short nis;                           // -inv_scale in FP16 (the MIX kernel)
    float *fout;                                  // FP32: the output state (11 planes)
    __half *g_out;                                // FP16-deviation: output planes
    float *fe_out, *fhx_out, *fhy_out;
    long long acc_from, steps;
    const int *slot;                              // the lattice's slot map (pitch layout)
    double *acc;                                  // its accumulators (6 per slot)
    const double2 *cs;                            // (cos w t, sin w t) for t mod period
    float *stage;                                 // ACC: 12 staged FP32 fields per slot (see stream_unit)
};

// One work unit: a strip of the lattice (columns xs .. xs + 63, 16-byte aligned) and a segment
// of rows (output rows y0 .. y1 - 1), from the stored state of time t - 1 to time t + 3; the
// tensor maps of the input state and ids, the material constants by id (shared memory) and the
// source values of the launch's four times.
struct UnitRun {
    int xs, y0, y1;
    long long t;
    const CUtensorMap *smap, *fmap, *imap;
    const MatT<float> *table;
    const float *src_g, *src_inc;
};

// A warp's row ring: the slot of the next row to arrive and the parity its barrier completes
// with.  Slots are used strictly in turn, unit after unit.
struct RingState {
    unsigned char *ring;
    uint64_t *bars;
    float4 *edge;
    int s0;
    unsigned ph;
};

// update_site<POL, true> (common.cuh) with the fields that enter the Fourier sums returned in
// FP32: f3 holds the values update_site converts to FP64 (the flush kernels convert them).
template <int POL>
__device__ __forceinline__ bool update_site_f3(Pop<float> &p, const MatT<float> &m, unsigned rthr, float f3[3]) {
    bool bad;
    if constexpr (POL == POL_TM) {
        float E3, Hx, Hy, D;
        moments(p, m, &E3, &Hx, &Hy, &D);
        bad = field_runaway(E3, rthr);
        f3[0] = D * m.inv_eps;
        f3[1] = Hx;
        f3[2] = Hy;
        collide(p, E3, Hx, Hy);
    } else {
        float Ey3, Ex3, Hz, Dy, Dx;
        moments_te(p, m, &Ey3, &Ex3, &Hz, &Dy, &Dx);
        bad = field_runaway(Ey3, rthr) || field_runaway(Ex3, rthr);
        f3[0] = Hz;
        f3[1] = Dx * m.inv_eps;
        f3[2] = Dy * m.inv_eps;
        collide_te(p, Ey3, Ex3, Hz);
    }
    return bad;
}

// ACC: the FP32 fields of one owned stencil site (slot sl >= 0) at level k of the launch, into
// the staging buffer that a flush kernel adds to the site's Fourier sums (Sec. III: Fourier
// analysis over one period) after the launch.
__device__ __forceinline__ void stage_owned(float *stage, int sl, int k, const float f3f[3]) {
    if (sl < 0) return;
    float *s = stage + 12 * (size_t)sl + 3 * k;
    s[0] = f3f[0];
    s[1] = f3f[1];
    s[2] = f3f[2];
}

// Four steps of one work unit (see the top of this file).  Returns false after a bounded wait
// for a row copy gave up.  bad: set when a stored site's field ran away.  SPLIT: the
// steady-state rows take the copies of the row loop without the general loop's tests.  ACC:
// instead of adding each stencil site's Fourier terms to its FP64 sums, store its FP32 fields at
// level k to stage[12 slot + 3 k ..] (u.stage); a flush kernel adds them after the launch in the
// same order and arithmetic as one step per launch.  Adding them here cost a few FP64
// instructions per stencil site, which on GB300's FP64 pipe made the units along the contour's
// vertical tangents (a stencil site in every row) the launch's long tail.
template <bool F16, int POL, bool ACC, bool SPLIT, bool MIX = false>
__device__ __forceinline__ bool stream_unit(const UnitCtx &u, const UnitRun &r, RingState &R, bool &bad) {
    // the steady-state copies treat every computed row as owned, which holds for the stored level
    // only: the Fourier sums of the levels before it would count halo rows twice
    static_assert(!(ACC && SPLIT), "accumulating units take the general row loop");
    using LY = Layout<F16>;
    constexpr int RING = LY::RING;
    const int lane = (int)threadIdx.x & 31;
    unsigned char *const ring = R.ring;
    uint64_t *const bars = R.bars;
    float4 *const edge = R.edge;
    const int nx = u.nx, ny = u.ny, xs = r.xs;
    const int xid = xs & ~15, idoff = xs - xid;   // first column of the id box, xs in it
    const int xa = xs + 2 * lane, xb = xa + 1;    // this lane's sites
    const int y0 = r.y0, y1 = r.y1;
    const int ylo = max(y0 - BT, 0), yhi = min(y1 + BT, ny);
    const bool xa0 = xa == 0, xa_last = xa == nx - 1, xb_last = xb == nx - 1;
    // the strip's staged columns include a lattice edge: edge clamps (any lane) and the source
    const bool xedge = xs <= 0 || xs + LW - 1 >= nx - 1;
    const bool out_lane = lane >= HALO / 2 && lane < 32 - HALO / 2 && xa >= 0 && xa < nx;
    const bool two = xb < nx;
    const int kind = u.kind;
    const bool src_lane = xa0 && kind != SRC_NONE;
    const size_t ps = u.pstride;
    const long long t = r.t;

    // ring slots of rows i, i - 1, i - 2 and the barrier phase of row i
    int s0 = R.s0, s1 = s0 == 0 ? RING - 1 : s0 - 1, s2 = s1 == 0 ? RING - 1 : s1 - 1;
    unsigned ph = R.ph;
    // prologue: the first RING rows in flight
    if (lane == 0)
        for (int j = 0; j < RING && ylo + j < yhi; ++j) {
            const int sj = (s0 + j) % RING;
            issue_row<F16>(r.smap, r.fmap, r.imap, xs, xid, ylo + j, ring + (size_t)sj * LY::SLOT, &bars[sj]);
        }

    Wave wa;
#pragma unroll
    for (int k = 0; k < BT; ++k) {
        keep_row(wa.cur[k], Pop<float>{}, Pop<float>{});
        wa.oe[k][0] = wa.oe[k][1] = wa.oh[k][0] = wa.oh[k][1] = 0.f;
        wa.ids[k] = 0u;
    }

    // One wavefront row: row i arrives as level 0; level k + 1 of row q = i - 1 - k is computed
    // from level k of rows q - 1, q and q + 1 (k = 0 from the ring, k >= 1 from `in`); `out`
    // receives the kept rows for the next row.  MODE 0: the general row; 1 and 2: a row in the
    // steady state (every level computes, every level-4 row is stored, no lattice top or bottom)
    // without those tests, 1 in an interior strip (no left or right edge either), 2 in a strip
    // at the lattice's left or right edge.  Returns false after a bounded wait gave up.
    auto row = [&](auto fast_tag, int i, const Wave &in, Wave &out) -> bool {
        constexpr int MODE = decltype(fast_tag)::value;
        constexpr bool FAST = MODE != 0;  // no test at the lattice's top and bottom or the segment's ends
        constexpr bool NOX = MODE == 1;   // and none at its left and right edges
        // level 0 of row i
        if (FAST || i < yhi) {
            const bool ok = mbar_wait(&bars[s0], ph);
            if (__any_sync(0xffffffffu, !ok)) return false;
            take_row<F16, MIX>(ring + (size_t)s0 * LY::SLOT, lane, u.inv_scale);
        }
        // ACC: the slots of this lane's two sites in the rows whose Fourier sums the levels take,
        // loaded before the levels' arithmetic so that the loads' latency overlaps it
        int2 slots[BT];
        if constexpr (ACC) {
#pragma unroll
            for (int k = 0; k < BT; ++k) {
                const int q = i - 1 - k;
                slots[k] = make_int2(-1, -1);
                if (out_lane && t + k >= u.acc_from && t + k < u.steps && q >= u.ay0 && q <= u.ay1 &&
                    (FAST || (q >= y0 && q < y1)))  // xa even, pitch a multiple of 32: 8-byte aligned
                    slots[k] = *reinterpret_cast<const int2 *>(u.slot + (size_t)q * u.pitch + xa);
            }
        }
        Pop<float> na{}, nb{};  // level k of row i - k, the -y pair for level k + 1
        bool have = FAST || i < yhi;
        unsigned id_k0 = 0;
#pragma unroll
        for (int k = 0; k < BT; ++k) {
            const int q = i - 1 - k;
            const bool compute = FAST || (q >= ylo && q < ny);  // uniform over the warp
            Pop<float> ca{}, cb{};
            if (compute) {
                unsigned idq;
                if (k == 0) {
                    // level 0 from the ring: rows q - 1, q, q + 1, clamped to q at the lattice's first
                    // and last rows and at the segment's first row (whose row above was never
                    // loaded: its level-1 value is a halo value no output depends on)
                    const unsigned char *sq = ring + (size_t)s1 * LY::SLOT;
                    const unsigned char *su = ring + (size_t)(FAST || q > ylo ? s2 : s1) * LY::SLOT;
                    const unsigned char *sd = ring + (size_t)(FAST || q < ny - 1 ? s0 : s1) * LY::SLOT;
                    Row9 c0;
                    float ey[2], hy[2], my[2], mh[2];
                    if constexpr (F16 && MIX) {
                        // the stored deviations rebuilt where they are read, each with its own row's
                        // fields: row q's seven in-row populations, row q - 1's +y pair, row q + 1's
                        // -y pair (every population of every row is read, and rebuilt, once)
                        const unsigned short nis = u.nis;
                        const Fld2 Q = slot_fields(sq, lane), U = slot_fields(su, lane), D = slot_fields(sd, lane);
                        rebuild2(Q.e.x, Q.e.y, slot_dev(sq, P_EZ, lane), nis, c0.ez);
                        rebuild2(eq2_epx(Q.e.x, Q.hx.x, Q.hy.x), eq2_epx(Q.e.y, Q.hx.y, Q.hy.y),
                                 slot_dev(sq, P_EPX, lane), nis, c0.epx);
                        rebuild2(eq2_emx(Q.e.x, Q.hx.x, Q.hy.x), eq2_emx(Q.e.y, Q.hx.y, Q.hy.y),
                                 slot_dev(sq, P_EMX, lane), nis, c0.emx);
                        rebuild2(Q.hx.x, Q.hx.y, slot_dev(sq, P_HXPX, lane), nis, c0.hxpx);
                        rebuild2(Q.hx.x, Q.hx.y, slot_dev(sq, P_HXMX, lane), nis, c0.hxmx);
                        rebuild2(Q.hx.x, Q.hx.y, slot_dev(sq, P_HXZ, lane), nis, c0.hxz);
                        rebuild2(Q.hy.x, Q.hy.y, slot_dev(sq, P_HYZ, lane), nis, c0.hyz);
                        rebuild2(eq2_epy(U.e.x, U.hx.x, U.hy.x), eq2_epy(U.e.y, U.hx.y, U.hy.y),
                                 slot_dev(su, P_EPY, lane), nis, ey);
                        rebuild2(U.hy.x, U.hy.y, slot_dev(su, P_HYPY, lane), nis, hy);
                        rebuild2(eq2_emy(D.e.x, D.hx.x, D.hy.x), eq2_emy(D.e.y, D.hx.y, D.hy.y),
                                 slot_dev(sd, P_EMY, lane), nis, my);
                        rebuild2(D.hy.x, D.hy.y, slot_dev(sd, P_HYMY, lane), nis, mh);
                    } else {
                        const float *rq = reinterpret_cast<const float *>(sq);
                        const float *ru = reinterpret_cast<const float *>(su);
                        const float *rd = reinterpret_cast<const float *>(sd);
                        float2 v;
                        v = lds2(rq, P_EZ, lane), c0.ez[0] = v.x, c0.ez[1] = v.y;
                        v = lds2(rq, P_EPX, lane), c0.epx[0] = v.x, c0.epx[1] = v.y;
                        v = lds2(rq, P_EMX, lane), c0.emx[0] = v.x, c0.emx[1] = v.y;
                        v = lds2(rq, P_HXPX, lane), c0.hxpx[0] = v.x, c0.hxpx[1] = v.y;
                        v = lds2(rq, P_HXMX, lane), c0.hxmx[0] = v.x, c0.hxmx[1] = v.y;
                        v = lds2(rq, P_HXZ, lane), c0.hxz[0] = v.x, c0.hxz[1] = v.y;
                        v = lds2(rq, P_HYZ, lane), c0.hyz[0] = v.x, c0.hyz[1] = v.y;
                        v = lds2(ru, P_EPY, lane), ey[0] = v.x, ey[1] = v.y;
                        v = lds2(ru, P_HYPY, lane), hy[0] = v.x, hy[1] = v.y;
                        v = lds2(rd, P_EMY, lane), my[0] = v.x, my[1] = v.y;
                        v = lds2(rd, P_HYMY, lane), mh[0] = v.x, mh[1] = v.y;
                    }
                    if (NOX)
                        pull_row(c0, ey, hy, my, mh, false, false, false, ca, cb);
                    else
                        pull_row(c0, ey, hy, my, mh, xa0, xa_last, xb_last, ca, cb);
                    idq = *reinterpret_cast<const unsigned short *>(sq + LY::IDS + idoff + 2 * lane);
                    id_k0 = idq;
                } else {
                    float ey[2], hy[2], my[2], mh[2];
                    if (!FAST && q == 0) {  // top edge: the +y pair of row 0 itself
                        ey[0] = in.cur[k].epy[0], ey[1] = in.cur[k].epy[1];
                        hy[0] = in.cur[k].hypy[0], hy[1] = in.cur[k].hypy[1];
                    } else {
                        ey[0] = in.oe[k][0], ey[1] = in.oe[k][1], hy[0] = in.oh[k][0], hy[1] = in.oh[k][1];
                    }
                    if (!FAST && q == ny - 1) {  // bottom edge: the -y pair of the last row itself
                        const float4 e = edge[k * 32 + lane];
                        my[0] = e.x, my[1] = e.y, mh[0] = e.z, mh[1] = e.w;
                    } else {
                        my[0] = na.emy, my[1] = nb.emy, mh[0] = na.hymy, mh[1] = nb.hymy;
                    }
                    if (NOX)
                        pull_row(in.cur[k], ey, hy, my, mh, false, false, false, ca, cb);
                    else
                        pull_row(in.cur[k], ey, hy, my, mh, xa0, xa_last, xb_last, ca, cb);
                    idq = in.ids[k];
                }
                if (!NOX && src_lane && t + k >= 1) inject_source_t(kind, r.src_g[k], r.src_inc[k], ca);
                const MatT<float> ma = r.table[idq & 0xffu], mb = r.table[(idq >> 8) & 0xffu];
                const bool owned = out_lane && (FAST || (q >= y0 && q < y1));
                const bool store = k == BT - 1 && owned;
                if (F16 && k == BT - 1) {
                    // the stored state of the last level: fields and FP16 deviations g = f - f^eq
                    float E3a, Hxa, Hya, Da, E3b, Hxb, Hyb, Db;
                    moments(ca, ma, &E3a, &Hxa, &Hya, &Da);
                    moments(cb, mb, &E3b, &Hxb, &Hyb, &Db);
                    if constexpr (ACC) {  // the fields of the stored level, staged as at the others
                        if (owned && t + k >= u.acc_from && t + k < u.steps && q >= u.ay0 && q <= u.ay1) {
                            const float f3a[3] = {Da * ma.inv_eps, Hxa, Hya}, f3b[3] = {Db * mb.inv_eps, Hxb, Hyb};
                            stage_owned(u.stage, slots[k].x, k, f3a);
                            if (two) stage_owned(u.stage, slots[k].y, k, f3b);
                        }
                    }
                    if (store) {
                        bad |= field_runaway(E3a, u.runaway) || (two && field_runaway(E3b, u.runaway));
                        const Fld Fa = stored_fields(E3a, Hxa, Hya), Fb = stored_fields(E3b, Hxb, Hyb);
                        __half2 g2[NPLANES];
                        encode_pair(ca, cb, Fa, Fb, u.scale, g2);
                        const size_t idx = (size_t)q * u.pitch + xa;
                        if (two) {
#pragma unroll
                            for (int p = 0; p < NPLANES; ++p)
                                *reinterpret_cast<__half2 *>(u.g_out + p * ps + idx) = g2[p];
                            *reinterpret_cast<float2 *>(u.fe_out + idx) = make_float2(Fa.e, Fb.e);
                            *reinterpret_cast<float2 *>(u.fhx_out + idx) = make_float2(Fa.hx, Fb.hx);
                            *reinterpret_cast<float2 *>(u.fhy_out + idx) = make_float2(Fa.hy, Fb.hy);
                        } else {
#pragma unroll
                            for (int p = 0; p < NPLANES; ++p) u.g_out[p * ps + idx] = __low2half(g2[p]);
                            u.fe_out[idx] = Fa.e;
                            u.fhx_out[idx] = Fa.hx;
                            u.fhy_out[idx] = Fa.hy;
                        }
                    }
                } else {
                    bool ra, rb;
                    if (ACC && t + k >= u.acc_from && t + k < u.steps && q >= u.ay0 && q <= u.ay1 &&
                        (FAST || (q >= y0 && q < y1))) {
                        // a row of contour stencil sites in the accumulated period (uniform over the
                        // warp): the fields of the owned sites enter their Fourier sums
                        float f3a[3], f3b[3];
                        ra = update_site_f3<POL>(ca, ma, u.runaway, f3a);
                        rb = update_site_f3<POL>(cb, mb, u.runaway, f3b);
                        if (out_lane) {
                            stage_owned(u.stage, slots[k].x, k, f3a);
                            if (two) stage_owned(u.stage, slots[k].y, k, f3b);
                        }
                    } else {
                        ra = update_site<POL, true>(ca, ma, u.runaway, nullptr, nullptr);
                        rb = update_site<POL, true>(cb, mb, u.runaway, nullptr, nullptr);
                    }
                    if (store) {
                        bad |= ra || (two && rb);
                        float *f = u.fout + (size_t)q * u.pitch + xa;
                        store2(f + P_EZ * ps, two, ca.ez, cb.ez);
                        store2(f + P_EPX * ps, two, ca.epx, cb.epx);
                        store2(f + P_EMX * ps, two, ca.emx, cb.emx);
                        store2(f + P_EPY * ps, two, ca.epy, cb.epy);
                        store2(f + P_EMY * ps, two, ca.emy, cb.emy);
                        store2(f + P_HXPX * ps, two, ca.hxpx, cb.hxpx);
                        store2(f + P_HXMX * ps, two, ca.hxmx, cb.hxmx);
                        store2(f + P_HXZ * ps, two, ca.hxz, cb.hxz);
                        store2(f + P_HYPY * ps, two, ca.hypy, cb.hypy);
                        store2(f + P_HYMY * ps, two, ca.hymy, cb.hymy);
                        store2(f + P_HYZ * ps, two, ca.hyz, cb.hyz);
                    }
                }
            }
            if (k == 0) {
                // the slot of row i - 2 is no longer read: it receives row i + 3
                __syncwarp();
                if (lane == 0 && (FAST || i - 2 >= ylo) && i + RING - 2 < yhi) {
                    fence_proxy_async_smem();
                    issue_row<F16>(r.smap, r.fmap, r.imap, xs, xid, i + RING - 2, ring + (size_t)s2 * LY::SLOT,
                                   &bars[s2]);
                }
            } else {
                // level k moves on by one row: row i - k becomes the kept row
                if (FAST || have) {
                    if (!FAST && i - k == ny - 1) edge[k * 32 + lane] = make_float4(na.emy, nb.emy, na.hymy, nb.hymy);
                    out.oe[k][0] = in.cur[k].epy[0], out.oe[k][1] = in.cur[k].epy[1];
                    out.oh[k][0] = in.cur[k].hypy[0], out.oh[k][1] = in.cur[k].hypy[1];
                    keep_row(out.cur[k], na, nb);
                }
            }
            na = ca;
            nb = cb;
            have = compute;
        }
        // ids: row i - 1 - k for level k + 1 at the next row
#pragma unroll
        for (int k = BT - 1; k > 1; --k) out.ids[k] = in.ids[k - 1];
        out.ids[1] = id_k0;
        // the ring moves on by one row when one arrived (the rows past the lattice's last row,
        // at the bottom of its last segment, take none: the slot and barrier phase of the next
        // row to arrive stay where they are, for the warp's next unit)
        if (FAST || i < yhi) {
            s2 = s1;
            s1 = s0;
            if (++s0 == RING) {
                s0 = 0;
                ph ^= 1u;
            }
        }
        return true;
    };

    // With SPLIT, the steady-state rows (every level computes and stores, no lattice top or
    // bottom, no segment end) run copies of the row without those tests: one for interior strips,
    // without the left and right edge tests too, one for the two strips at the lattice's edges.
    // Measured on GB300 (GLUPS on 8192^2 / 2048^2): FP32 with the general loop for every row
    // 240.1 / 180.3, with both copies 257.2 / 195.0; FP16-deviation with the interior copy only
    // (the edge strips, on the general loop, then finish last) 253.5 / 166.8, with both copies
    // 263.4 / 187.2.  Every kernel takes the copies except the accumulating ones (see the check at
    // the top of this function); the batch's gain: 256-instance design map 116.6 -> 129.6 cells/s.
    // An L2
    // prefetch of the rows beyond the ring (cp.async.bulk.prefetch.tensor) lost in both forms
    // (FP32 212.8 against 220.4, FP16 173.7 against 199.5, with one wave of units) and is not used.
    using General = std::integral_constant<int, 0>;
    using Interior = std::integral_constant<int, 1>;
    using EdgeStrip = std::integral_constant<int, 2>;
    const int f0 = max(y0 + BT, BT + 1), f1 = !SPLIT ? f0 : min(min(y1 + BT, yhi), ny);
    bool ok = true;
    int i = ylo;
    for (; i < f0 && i < y1 + BT; ++i)
        if (!row(General{}, i, wa, wa)) {
            ok = false;
            break;
        }
    if (SPLIT && xedge) {  // (without SPLIT these loops never run: f1 = f0)
        for (; ok && i < f1; ++i)
            if (!row(EdgeStrip{}, i, wa, wa)) {
                ok = false;
                break;
            }
    } else {
        for (; ok && i < f1; ++i)
            if (!row(Interior{}, i, wa, wa)) {
                ok = false;
                break;
            }
    }
    for (; ok && i < y1 + BT; ++i)
        if (!row(General{}, i, wa, wa)) {
            ok = false;
            break;
        }
    R.s0 = s0;
    R.ph = ph;
    return ok;
}


// F16: the FP16-deviation form (TM; MIX: rebuilt with the mixed-precision FMA); otherwise FP32
// of either polarization, with ACC the FP32 fields of every level at the contour's stencil sites
// into the staging buffer (the general row loop; k_stage_flush adds them to the Fourier sums).  One work unit per
// warp: strip unit % n_strips, row segment unit / n_strips.
template <bool F16, int POL, bool MIX, bool ACC>
__global__ void __launch_bounds__(NW * 32, 3)
    k_step4_stream(const __grid_constant__ UnitCtx u, const StreamArgs a, const __grid_constant__ CUtensorMap smap,
                   const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap imap,
                   const long long *__restrict__ t_in, long long *__restrict__ t_out) {
    using LY = Layout<F16>;
    constexpr int RING = LY::RING;
    extern __shared__ unsigned char sm_dyn[];
    __shared__ __align__(8) uint64_t bars[NW][RING];
    __shared__ SrcLevels sp;
    unsigned char *s = sm_dyn + ((128u - (smem_u32(sm_dyn) & 127u)) & 127u);
    MatT<float> *table = reinterpret_cast<MatT<float> *>(s);
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    unsigned char *ring = s + LY::TABLE + (size_t)warp * LY::WARP;

    const long long t = *t_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *t_out = t + BT;
    if (threadIdx.x == 0) sp = source_levels_f(a.src, t);
    for (int k = threadIdx.x; k < 256; k += NW * 32) table[k] = a.mtab[k];
    if (lane == 0) {
        for (int j = 0; j < RING; ++j) mbar_init(&bars[warp][j], 1);
        fence_mbar_init();
    }
    __syncthreads();  // the only block-wide barrier: from here on each warp runs alone
    const int unit = (int)blockIdx.x * NW + warp;
    if (unit >= a.n_units) return;
    const int strip = unit % a.n_strips, seg = unit / a.n_strips;
    UnitRun r;
    r.xs = strip * OUTW - HALO;
    r.y0 = seg * a.seg_rows;
    r.y1 = min(r.y0 + a.seg_rows, u.ny);
    r.t = t;
    r.smap = &smap;
    r.fmap = &fmap;
    r.imap = &imap;
    r.table = table;
    r.src_g = sp.g;
    r.src_inc = sp.inc;
    RingState R{ring, bars[warp], reinterpret_cast<float4 *>(ring + RING * LY::SLOT), 0, 0u};
    bool bad = false;
    const bool ok = stream_unit<F16, POL, ACC, !ACC, MIX>(u, r, R, bad);
    if (lane == 0 && !ok) atomicOr(a.err, kErrTimeout);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, kErrUnstable);
}

// Batched design maps: the warps walk the work units of every instance (instance, strip, row
// segment; ordered by decreasing run length, then segment, then strip) with a grid stride,
// skipping instances that have finished, four steps per launch; the batch launches one warp per
// unit, so each warp normally takes one.  Two instantiations run one after the other in
// every launch and split the unfinished instances between them: ACC = false takes those with
// no time of their accumulated (last) period among the launch's four, ACC = true the others,
// whose stencil sites' fields it stages for the levels whose time falls in that period
// (k_batch_flush4 adds them to the Fourier sums after it; ACC = true takes the general row
// loop).  An instance that ends inside a launch runs on past its end without accumulating; its
// state is not needed afterwards.  FP32.
template <int POL, bool ACC>
__global__ void __launch_bounds__(NW * 32, 3)
    k_batch_step4(const StreamInst *__restrict__ insts, const int4 *__restrict__ units, int n_units,
                  const SrcLevels *__restrict__ srcs, const CUtensorMap *__restrict__ maps, int p,
                  float *__restrict__ buf_out, const int *__restrict__ slot, float *__restrict__ stage,
                  unsigned *__restrict__ err, const long long *__restrict__ t_in, long long *__restrict__ t_out) {
    using LY = Layout<false>;
    constexpr int RING = LY::RING;
    extern __shared__ unsigned char sm_dyn[];
    __shared__ __align__(8) uint64_t bars[NW][RING];
    __shared__ MatT<float> wtab[NW][4];  // the current unit's region table, per warp
    __shared__ UnitCtx uctx[NW];         // the current instance, per warp (read from here, not kept in registers)
    __shared__ UnitRun urun[NW];         // the current unit, per warp
    unsigned char *s = sm_dyn + ((128u - (smem_u32(sm_dyn) & 127u)) & 127u);
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    unsigned char *ring = s + LY::TABLE + (size_t)warp * LY::WARP;
    const long long t = *t_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *t_out = t + BT;
    if (lane == 0) {
        for (int j = 0; j < RING; ++j) mbar_init(&bars[warp][j], 1);
        fence_mbar_init();
    }
    __syncthreads();  // the only block-wide barrier
    RingState R{ring, bars[warp], reinterpret_cast<float4 *>(ring + RING * LY::SLOT), 0, 0u};
    const int stride = (int)gridDim.x * NW;
    for (int w = (int)blockIdx.x * NW + warp; w < n_units; w += stride) {
        const int4 un = units[w];
        const StreamInst &I = insts[un.x];
        const long long steps = I.steps;
        if (t >= steps || (t + BT - 1 >= I.acc_from) != ACC) continue;  // uniform over the warp
        __syncwarp();              // the previous unit's reads of the table and context are done
        if (lane < 3) wtab[warp][lane] = I.m[lane];
        UnitCtx &u = uctx[warp];
        if (lane == 0) {
            u.nx = I.nx;
            u.ny = I.ny;
            u.pitch = I.pitch;
            u.kind = I.kind;
            u.runaway = I.runaway;
            u.ay0 = I.ay0;
            u.ay1 = I.ay1;
            u.period = I.period;
            u.pstride = (size_t)I.pstride;
            u.fout = buf_out + I.base;
            u.acc_from = I.acc_from;
            u.steps = steps;
            u.slot = slot + I.slot_base;
            u.stage = stage + 12 * (size_t)I.acc_base;
            u.cs = I.cs;
        }
        UnitRun &r = urun[warp];
        if (lane == 0) {
            r.xs = un.y * OUTW - HALO;
            r.y0 = un.z * I.seg_rows;
            r.y1 = min(r.y0 + I.seg_rows, I.ny);
            r.t = t;
            r.smap = maps + 3 * un.x + p;
            r.fmap = r.smap;
            r.imap = maps + 3 * un.x + 2;
            tmap_acquire(r.smap);  // lane 0 issues every row copy of the unit
            tmap_acquire(r.imap);
            r.table = wtab[warp];
            r.src_g = srcs[un.x].g;
            r.src_inc = srcs[un.x].inc;
        }
        __syncwarp();
        bool bad = false;
        const bool ok = stream_unit<false, POL, ACC, !ACC>(u, r, R, bad);
        if (!ok) {  // a row copy never completed: report, leave
            if (lane == 0) atomicOr(err + un.x, kErrTimeout);
            return;
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err + un.x, kErrUnstable);
    }
}

// The source values of every instance at the launch's four times, one thread per instance.
__global__ void k_batch_source4(const SourceParams *__restrict__ src, int n, const long long *__restrict__ t_in,
                                SrcLevels *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = source_levels_f(src[i], *t_in);
}

// After an accumulating launch from time *t_in: adds every stencil slot's staged FP32 fields of
// the launch's four levels to its Fourier sums (Sec. III), in time order, exactly as the
// one-step kernel adds them step by step.
__global__ void k_stage_flush(const float *__restrict__ stage, double *__restrict__ acc, int n_slots,
                              const double2 *__restrict__ cs, int period, const long long *__restrict__ t_in) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slots) return;
    const long long t = *t_in;
    const float *s = stage + 12 * (size_t)i;
    double *a = acc + 6 * (size_t)i;
    double a0 = a[0], a1 = a[1], a2 = a[2], a3 = a[3], a4 = a[4], a5 = a[5];
#pragma unroll
    for (int k = 0; k < BT; ++k) {
        const double2 c = cs[(int)((t + k) % (long long)period)];
        const double f0 = (double)s[3 * k], f1 = (double)s[3 * k + 1], f2 = (double)s[3 * k + 2];
        a0 += f0 * c.x;
        a1 += f0 * c.y;
        a2 += f1 * c.x;
        a3 += f1 * c.y;
        a4 += f2 * c.x;
        a5 += f2 * c.y;
    }
    a[0] = a0, a[1] = a1, a[2] = a2, a[3] = a3, a[4] = a4, a[5] = a5;
}

// The batch's flush after each four-step launch from time *t_in: every stencil slot of the packed
// accumulators (slot_inst: its instance) adds the staged fields of the levels whose time lies
// in its instance's accumulated period, in time order; the same test selects the levels the
// accumulating kernel staged.
__global__ void k_batch_flush4(const float *__restrict__ stage, double *__restrict__ acc,
                               const int *__restrict__ slot_inst, const StreamInst *__restrict__ insts, int n_slots,
                               const long long *__restrict__ t_in) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slots) return;
    const long long t = *t_in;
    const StreamInst &I = insts[slot_inst[i]];
    if (t + BT - 1 < I.acc_from || t >= I.steps) return;
    const float *s = stage + 12 * (size_t)i;
    double *a = acc + 6 * (size_t)i;
    double a0 = a[0], a1 = a[1], a2 = a[2], a3 = a[3], a4 = a[4], a5 = a[5];
#pragma unroll
    for (int k = 0; k < BT; ++k) {
        const long long tk = t + k;
        if (tk < I.acc_from || tk >= I.steps) continue;
        const double2 c = I.cs[(int)(tk % (long long)I.period)];
        const double f0 = (double)s[3 * k], f1 = (double)s[3 * k + 1], f2 = (double)s[3 * k + 2];
        a0 += f0 * c.x;
        a1 += f0 * c.y;
        a2 += f1 * c.x;
        a3 += f1 * c.y;
        a4 += f2 * c.x;
        a5 += f2 * c.y;
    }
    a[0] = a0, a[1] = a1, a[2] = a2, a[3] = a3, a[4] = a4, a[5] = a5;
}

template <bool F16, int POL, bool MIX, bool ACC>
cudaError_t allow_smem_stream() {
    return cudaFuncSetAttribute(k_step4_stream<F16, POL, MIX, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Layout<F16>::SMEM);
}

}  // namespace

StreamPlan stream_plan(int nx, int ny, int resident_warps, bool f16) {
    // Units in k full waves of the resident warps (k x resident / strips row segments per
    // strip): the warps of a wave start together and stream their rows in step, and later waves
    // start as blocks of the earlier ones finish, which spreads the GPU's row copies and
    // arithmetic over time; a wave only partly filled leaves SMs idle at the end.  Every segment
    // pays a 4-row halo at each end, so k is the largest that keeps segments of at least
    // min_rows rows, at most max_waves: FP32 5 waves of at least 45 rows, FP16-deviation 3 of
    // at least 80 (measured on GB300 from 2048^2 to 8192^2, each within 1.5 % of the best number
    // of waves at every size; 8192^2: one wave 227.9 (FP32) and 254.9 (FP16) GLUPS, the plan
    // 266.3 and 277.5).
    StreamPlan p;
    p.n_strips = (nx + OUTW - 1) / OUTW;
    const int max_waves = f16 ? 3 : 5, min_rows = f16 ? 80 : 45;
    int segs = 1;
    for (int k = 1; k <= max_waves; ++k) {
        int sk = (int)((long long)k * resident_warps / p.n_strips);
        if (sk < 1) sk = 1;
        if (k > 1 && (ny + sk - 1) / sk < min_rows) break;
        segs = sk;
    }
    // but at least 16 rows each (shorter ones spend most of their time on the halo)
    if (segs > (ny + 15) / 16) segs = (ny + 15) / 16;
    p.seg_rows = (ny + segs - 1) / segs;
    segs = (ny + p.seg_rows - 1) / p.seg_rows;
    p.n_units = p.n_strips * segs;
    p.grid = (p.n_units + NW - 1) / NW;
    return p;
}

cudaError_t stream_prepare(bool f16, int *resident_warps, int *resident_warps_acc) {
    cudaError_t e = f16 ? allow_smem_stream<true, POL_TM, false, false>() : allow_smem_stream<false, POL_TM, false, false>();
    if (e == cudaSuccess && f16) e = allow_smem_stream<true, POL_TM, true, false>();
    if (e == cudaSuccess && f16) e = allow_smem_stream<true, POL_TM, true, true>();
    if (e == cudaSuccess && f16) e = allow_smem_stream<true, POL_TM, false, true>();
    if (e == cudaSuccess && !f16) e = allow_smem_stream<false, POL_TE, false, false>();
    if (e == cudaSuccess && !f16) e = allow_smem_stream<false, POL_TM, false, true>();
    if (e == cudaSuccess && !f16) e = allow_smem_stream<false, POL_TE, false, true>();
    int dev = 0, sms = 0, per_sm = 0, per_sm_acc = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = f16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step4_stream<true, POL_TM, true, false>,
                                                                NW * 32, Layout<true>::SMEM)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step4_stream<false, POL_TM, false, false>,
                                                                NW * 32, Layout<false>::SMEM);
    if (e == cudaSuccess)
        e = f16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_acc, k_step4_stream<true, POL_TM, true, true>,
                                                                NW * 32, Layout<true>::SMEM)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_acc, k_step4_stream<false, POL_TM, false, true>,
                                                                NW * 32, Layout<false>::SMEM);
    if (e == cudaSuccess && (per_sm < 1 || per_sm_acc < 1)) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) {
        *resident_warps = per_sm * sms * NW;
        *resident_warps_acc = per_sm_acc * sms * NW;
    }
    return e;
}

cudaError_t encode_stream_maps(CUtensorMap *smap, CUtensorMap *fmap, CUtensorMap *imap, const void *buf, bool f16,
                               const uint8_t *ids, int nx, int ny, int pitch, size_t pstride) {
    if (((uintptr_t)buf & 15u) || ((uintptr_t)ids & 15u) || (pitch % 16) || (pstride % 8))
        return cudaErrorInvalidValue;
    cudaError_t e;
    if (f16) {
        const size_t hb = f16_half_bytes(pstride), fb = f16_plane_bytes(pstride);
        const cuuint64_t gdims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)NPLANES};
        const cuuint64_t gstrides[2] = {(cuuint64_t)pitch * 2, (cuuint64_t)pstride * 2};
        const cuuint32_t gbox[3] = {(cuuint32_t)DEVW, 1u, (cuuint32_t)NPLANES};
        e = encode_tiled(smap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, buf, gdims, gstrides, gbox);
        if (e != cudaSuccess) return e;
        const cuuint64_t fdims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 3};
        const cuuint64_t fstrides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)fb};
        const cuuint32_t fbox[3] = {(cuuint32_t)LW, 1u, 3u};
        e = encode_tiled(fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (const char *)buf + hb, fdims, fstrides, fbox);
    } else {
        const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)NPLANES};
        const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pstride * 4};
        const cuuint32_t box[3] = {(cuuint32_t)LW, 1u, (cuuint32_t)NPLANES};
        e = encode_tiled(smap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, buf, dims, strides, box);
        if (e == cudaSuccess && fmap) *fmap = *smap;  // unused by the FP32 kernel (may be NULL)
    }
    if (e != cudaSuccess || !imap) return e;
    const cuuint64_t idims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t istrides[1] = {(cuuint64_t)pitch};
    const cuuint32_t ibox[2] = {(cuuint32_t)IDBOX, 1u};
    return encode_tiled(imap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ids, idims, istrides, ibox);
}

template <int POL, bool ACC>
cudaError_t allow_smem_batch4() {
    return cudaFuncSetAttribute(k_batch_step4<POL, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Layout<false>::SMEM);
}

cudaError_t batch_stream_prepare(int *resident_warps) {
    cudaError_t e = allow_smem_batch4<POL_TM, false>();
    if (e == cudaSuccess) e = allow_smem_batch4<POL_TM, true>();
    if (e == cudaSuccess) e = allow_smem_batch4<POL_TE, false>();
    if (e == cudaSuccess) e = allow_smem_batch4<POL_TE, true>();
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step4<POL_TM, false>, NW * 32,
                                                          Layout<false>::SMEM);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) *resident_warps = per_sm * sms * NW;
    return e;
}

cudaError_t encode_batch_stream_maps(CUtensorMap *maps, const float *buf0, const float *buf1, const uint8_t *ids,
                                     int nx, int ny, int pitch, size_t pstride) {
    cudaError_t e = encode_stream_maps(&maps[0], nullptr, &maps[2], buf0, false, ids, nx, ny, pitch, pstride);
    if (e == cudaSuccess) e = encode_stream_maps(&maps[1], nullptr, nullptr, buf1, false, ids, nx, ny, pitch, pstride);
    return e;
}

cudaError_t launch_batch_step4(const StreamInst *insts, const SourceParams *srcp, int n_inst, const int4 *units,
                               int n_units, SrcLevels *srcs, const CUtensorMap *maps, int p, float *buf_out,
                               const int *slot, double *acc, float *stage, const int *slot_inst, int n_slots,
                               unsigned *err, const long long *t_in, long long *t_out, int grid, int pol,
                               cudaStream_t s) {
    k_batch_source4<<<(n_inst + 127) / 128, 128, 0, s>>>(srcp, n_inst, t_in, srcs);
    const size_t sm = Layout<false>::SMEM;
    // both write t + 4 to t_out; neither reads it
    if (pol == POL_TE) {
        k_batch_step4<POL_TE, false><<<grid, NW * 32, sm, s>>>(insts, units, n_units, srcs, maps, p, buf_out, slot,
                                                              stage, err, t_in, t_out);
        k_batch_step4<POL_TE, true><<<grid, NW * 32, sm, s>>>(insts, units, n_units, srcs, maps, p, buf_out, slot,
                                                             stage, err, t_in, t_out);
    } else {
        k_batch_step4<POL_TM, false><<<grid, NW * 32, sm, s>>>(insts, units, n_units, srcs, maps, p, buf_out, slot,
                                                              stage, err, t_in, t_out);
        k_batch_step4<POL_TM, true><<<grid, NW * 32, sm, s>>>(insts, units, n_units, srcs, maps, p, buf_out, slot,
                                                             stage, err, t_in, t_out);
    }
    if (n_slots > 0)
        k_batch_flush4<<<(n_slots + 255) / 256, 256, 0, s>>>(stage, acc, slot_inst, insts, n_slots, t_in);
    return cudaGetLastError();
}

cudaError_t launch_step4_stream(const StepArgs<float> &sa, const F16Args *fa, const CUtensorMap *smap,
                                const CUtensorMap *fmap, const CUtensorMap *imap, float *fout, const StreamPlan &plan,
                                const long long *t_in, long long *t_out, bool accumulate, float *stage, int n_slots,
                                cudaStream_t s) {
    if (accumulate && !stage && n_slots > 0) return cudaErrorInvalidValue;  // needs the staging buffer
    StreamArgs a{};
    a.nx = sa.nx;
    a.ny = sa.ny;
    a.pitch = sa.pitch;
    a.n_strips = plan.n_strips;
    a.seg_rows = plan.seg_rows;
    a.n_units = plan.n_units;
    a.pstride = sa.pstride;
    a.mtab = sa.mtab;
    a.src = sa.src;
    a.err = sa.err;
    a.runaway = sa.runaway;
    a.fout = fout;
    UnitCtx u{};
    u.nx = sa.nx;
    u.ny = sa.ny;
    u.pitch = sa.pitch;
    u.kind = sa.src.kind;
    u.runaway = sa.runaway;
    u.pstride = sa.pstride;
    u.fout = fout;
    if (accumulate) {  // every level of the launch, at the contour's stencil rows
        u.acc_from = 0;
        u.steps = LLONG_MAX;
        u.ay0 = sa.accp.y0;
        u.ay1 = sa.accp.y1;
        u.slot = sa.accp.slot;
        u.acc = sa.accp.acc;
        u.cs = sa.src.cs;
        u.period = sa.src.period;
        u.stage = stage;
    }
    if (fa) {
        a.scale = u.scale = fa->scale;
        a.inv_scale = u.inv_scale = fa->inv_scale;
        a.g_out = u.g_out = fa->g_out;
        a.fe_out = u.fe_out = fa->fe_out;
        a.fhx_out = u.fhx_out = fa->fhx_out;
        a.fhy_out = u.fhy_out = fa->fhy_out;
        // -inv_scale = -2^m in FP16: exact from 2^-24 (subnormal below 2^-14) to 2^15
        const int m = std::ilogb(fa->inv_scale);
        const bool mix = m >= -24 && m <= 15;
        if (mix) u.nis = f16_neg_pow2_bits(m);
        if (mix && accumulate)
            k_step4_stream<true, POL_TM, true, true>
                <<<plan.grid, NW * 32, Layout<true>::SMEM, s>>>(u, a, *smap, *fmap, *imap, t_in, t_out);
        else if (mix)
            k_step4_stream<true, POL_TM, true, false>
                <<<plan.grid, NW * 32, Layout<true>::SMEM, s>>>(u, a, *smap, *fmap, *imap, t_in, t_out);
        else if (accumulate)
            k_step4_stream<true, POL_TM, false, true>
                <<<plan.grid, NW * 32, Layout<true>::SMEM, s>>>(u, a, *smap, *fmap, *imap, t_in, t_out);
        else
            k_step4_stream<true, POL_TM, false, false>
                <<<plan.grid, NW * 32, Layout<true>::SMEM, s>>>(u, a, *smap, *fmap, *imap, t_in, t_out);
    } else if (sa.pol == POL_TE) {
        if (accumulate)
            k_step4_stream<false, POL_TE, false, true>
                <<<plan.grid, NW * 32, Layout<false>::SMEM, s>>>(u, a, *smap, *smap, *imap, t_in, t_out);
        else
            k_step4_stream<false, POL_TE, false, false>
                <<<plan.grid, NW * 32, Layout<false>::SMEM, s>>>(u, a, *smap, *smap, *imap, t_in, t_out);
    } else {
        if (accumulate)
            k_step4_stream<false, POL_TM, false, true>
                <<<plan.grid, NW * 32, Layout<false>::SMEM, s>>>(u, a, *smap, *smap, *imap, t_in, t_out);
        else
            k_step4_stream<false, POL_TM, false, false>
                <<<plan.grid, NW * 32, Layout<false>::SMEM, s>>>(u, a, *smap, *smap, *imap, t_in, t_out);
    }
    if (accumulate && n_slots > 0)
        k_stage_flush<<<(n_slots + 127) / 128, 128, 0, s>>>(stage, sa.accp.acc, n_slots, sa.src.cs, sa.src.period,
                                                            t_in);
    return cudaGetLastError();
}

}  // namespace lbmem
