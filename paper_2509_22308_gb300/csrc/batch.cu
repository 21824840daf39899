// Batched design diagrams (the force/torque maps of arXiv 2509.22308, Sec. IV.A-B):
// many Janus instances of uneven size and run length advance together.
//
// Layout: every instance keeps its own 16 structure-of-arrays planes (pitch rounded
// to 32 sites), packed one after another in two ping-pong buffers; material ids,
// contour slot maps and Fourier accumulators are packed the same way.  A tile list
// covers every instance with tile_w x tile_h tiles, ordered by decreasing run length,
// so at any time the tiles still running form a prefix of the list.
//
// Kernel: a persistent grid (ctas_per_sm x SMs) walks the tile list with a grid
// stride once per time step, running the same per-site pull / moments / collide as
// the single-domain step; a tile whose instance has finished is skipped, a tile in
// its instance's last period also accumulates the Fourier sums.  Two steps are
// captured in a CUDA graph and replayed; time comes from the device words as in the
// single-domain path.  Tile shape and CTAs per SM are chosen by timing a few steps of
// each candidate on the actual packed data (then the state is cleared).
#include <algorithm>
#include <array>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <numeric>
#include <vector>

#include "../../include/lbm_em.h"
#include "common.cuh"
#include "launchers.h"
#include "runtime.h"
#include "step2.cuh"
#include "step2_tma.h"
#include "step_stream.h"
#include "tile_tma.cuh"

using namespace lbmem;

namespace lbmem {

struct InstDesc {
    int nx, ny, pitch, period;
    size_t pstride, base, mat_base, slot_base;
    long long steps, acc_from;
    int acc_base, y0, y1;
    unsigned runaway;   // exponent-field threshold of the runaway test in the batch's type (runaway_bits)
    SourceParams src;
    double mtab[3][4];  // per region id: MatT in the batch's type, widened (exactly) to double
    MatT<float> mtabf[3];  // the same in FP32 (FP32 batches), so no tile converts on the FP64 pipe
};

struct Tile {
    int inst, x0, y0, pad;
};

// Everything the two-step kernel needs of a tile and its instance: one 128-byte record per
// tile, built with the tile list, so that a CTA reads it with one vector load per lane of
// one warp instead of walking tile -> instance -> fields in every warp.
struct alignas(16) TileCtx {
    int inst, x0, y0, nx;
    int ny, pitch, kind, ay0;  // ay0, ay1: rows holding contour stencil sites
    int ay1;
    unsigned runaway;          // FP32 runaway threshold of the instance (runaway_bits<float>)
    int pad1, pad2;
    long long base, pstride, steps, acc_from;
    MatT<float> m[3];  // region table in FP32
};
static_assert(sizeof(TileCtx) == 128, "TileCtx is eight 16-byte words");

template <typename T>
struct BatchArgs {
    const InstDesc *inst;
    const Tile *tiles;
    int n_tiles, tile_w, tile_h, log2_tile_w;  // log2_tile_w < 0: tile_w is not a power of two
    const T *fin;
    T *fout;
    const uint8_t *mat;
    const int *slot;
    double *acc;
    unsigned *err;     // one word per instance
    double *energy;    // per-instance energy sum of the current period-boundary step
    int conv;          // 1: sample the energy at period boundaries (convergence exits)
};

// Material constants of region r of an instance in the kernel's type.
template <typename T>
__device__ __forceinline__ MatT<T> mat_entry(const InstDesc &d, int r) {
    if constexpr (sizeof(T) == 4) {
        return d.mtabf[r];
    } else {
        return MatT<T>{(T)d.mtab[r][0], (T)d.mtab[r][1], (T)d.mtab[r][2], (T)d.mtab[r][3]};
    }
}

// The sites of one tile at time t.  BOOK: the tile accumulates Fourier sums or samples the
// energy this step (both uniform over the tile); without it no FP64 operation is compiled
// in, so none can be predicated into the plain steps (see batch2_tile).  Returns the
// thread's share of the tile's energy when sampling.
template <typename T, int POL, bool BOOK, bool POW2>
__device__ __forceinline__ double batch_tile(const BatchArgs<T> &b, const Tile &tl, const InstDesc &d, long long t,
                                             bool acc, bool sample, bool src, const MatT<T> *smat,
                                             const double *ssrc) {
    StepArgs<T> a;
    a.nx = d.nx;
    a.ny = d.ny;
    a.pitch = d.pitch;
    a.pstride = d.pstride;
    a.src = d.src;
    const T *fin = b.fin + d.base;
    T *fout = b.fout + d.base;
    const uint8_t *mat = b.mat + d.mat_base;
    const int tsz = b.tile_w * b.tile_h;
    double wsum_t = 0.0;
    for (int k = threadIdx.x; k < tsz; k += blockDim.x) {
        // POW2: power-of-two widths (every one-step shape) by mask and shift; otherwise (the
        // 40-wide tiles of the two-step kernel, whose odd-length runs end with one one-step
        // launch) by division
        const int lx = POW2 ? (k & (b.tile_w - 1)) : k % b.tile_w;
        const int ly = POW2 ? (k >> b.log2_tile_w) : k / b.tile_w;
        const int x = tl.x0 + lx, y = tl.y0 + ly;
        if (x >= d.nx || y >= d.ny) continue;
        Pop<T> p;
        pull_planes(a, fin, x, y, p);
        if (x == 0 && src) inject_source(d.src.kind, ssrc[0], ssrc[1], p);
        const size_t idx = (size_t)y * d.pitch + x;
        const MatT<T> m = smat[mat[idx]];
        // moments, runaway test, field triple (TM: E_z, H_x, H_y; TE: H_z, E_x, E_y) and energy
        // density when wanted, collision: update_site, the single-domain kernels' site update
        bool bad;
        if (BOOK) {
            const bool acc_row = acc && y >= d.y0 && y <= d.y1;
            double f3[3], w;
            bad = update_site<POL, true>(p, m, d.runaway, acc_row ? f3 : nullptr, sample ? &w : nullptr);
            if (acc_row) {
                const int s = b.slot[d.slot_base + idx];
                if (s >= 0) {
                    const double2 c = d.src.cs[(int)(t % (long long)d.period)];
                    double *q = b.acc + 6 * ((size_t)d.acc_base + s);
                    q[0] += f3[0] * c.x;
                    q[1] += f3[0] * c.y;
                    q[2] += f3[1] * c.x;
                    q[3] += f3[1] * c.y;
                    q[4] += f3[2] * c.x;
                    q[5] += f3[2] * c.y;
                }
            }
            if (sample) wsum_t += w;
        } else {
            bad = update_site<POL, true>(p, m, d.runaway, nullptr, nullptr);
        }
        if (bad) atomicOr(b.err + tl.inst, kErrUnstable);
        store_site(fout, d.pstride, idx, p);
    }
    return wsum_t;
}

// FP32 and FP64: at most 85 registers so that 3 CTAs of 256 threads stay resident per SM (FP64,
// bound by its pipe, needs the warps: 102 registers and 2 CTAs per SM gave 9.9 design-map cells/s,
// 80 registers and 3 CTAs 10.3, 64 registers and 4 CTAs 10.4 with 150-byte spills).
template <typename T, int POL>
__global__ void __launch_bounds__(256, std::is_same<T, df>::value ? 2 : 3)
    k_batch_step(const BatchArgs<T> b, const long long *__restrict__ t_in, long long *__restrict__ t_out) {
    const long long t = *t_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *t_out = t + 1;
    __shared__ MatT<T> smat[3];
    __shared__ double ssrc[2];  // source values of the tile's instance at time t (column-0 tiles)
    for (int tile = blockIdx.x; tile < b.n_tiles; tile += gridDim.x) {
        const Tile tl = b.tiles[tile];
        const InstDesc &d = b.inst[tl.inst];
        const long long steps = d.steps;
        if (t >= steps) continue;  // uniform over the block
        const bool acc = t >= d.acc_from;
        const bool sample = b.conv && t > 0 && t < d.acc_from && (t % (long long)d.period) == 0;
        __syncthreads();
        if (threadIdx.x < 3)
            smat[threadIdx.x] = mat_entry<T>(d, threadIdx.x);
        // once per tile, not per site (see pull_site)
        const bool src = tl.x0 == 0 && t >= 1 && d.src.kind != SRC_NONE;
        if (threadIdx.x == 32 && src) source_values(d.src, t, &ssrc[0], &ssrc[1]);
        __syncthreads();
        if (!(acc || sample)) {  // uniform over the block
            if (b.log2_tile_w >= 0)
                batch_tile<T, POL, false, true>(b, tl, d, t, false, false, src, smat, ssrc);
            else
                batch_tile<T, POL, false, false>(b, tl, d, t, false, false, src, smat, ssrc);
            continue;
        }
        double wsum_t = b.log2_tile_w >= 0 ? batch_tile<T, POL, true, true>(b, tl, d, t, acc, sample, src, smat, ssrc)
                                           : batch_tile<T, POL, true, false>(b, tl, d, t, acc, sample, src, smat, ssrc);
        if (sample) {  // block sum of the tile's energy into the instance's accumulator
            __shared__ double wsh[8];
            for (int o = 16; o > 0; o >>= 1) wsum_t += __shfl_down_sync(0xffffffffu, wsum_t, o);
            if ((threadIdx.x & 31) == 0) wsh[threadIdx.x >> 5] = wsum_t;
            __syncthreads();
            if (threadIdx.x == 0) {
                double w = 0.0;
                for (int q = 0; q < (int)(blockDim.x >> 5); ++q) w += wsh[q];
                atomicAdd(b.energy + tl.inst, w);
            }
        }
    }
}

// Fourier accumulation of one site of an instance at time t (its slot map and accumulators).
__device__ __forceinline__ void batch_acc(const double *f3, const int *slot, double *acc, const InstDesc &d,
                                          size_t idx, long long t) {
    const int s = slot[d.slot_base + idx];
    if (s < 0) return;
    const double2 c = d.src.cs[(int)(t % (long long)d.period)];
    double *q = acc + 6 * ((size_t)d.acc_base + s);
    q[0] += f3[0] * c.x;
    q[1] += f3[0] * c.y;
    q[2] += f3[1] * c.x;
    q[3] += f3[1] * c.y;
    q[4] += f3[2] * c.x;
    q[5] += f3[2] * c.y;
}

// Two steps per launch for the FP32 batch with fixed run lengths, on the TMA-staged tile
// of the single-domain FP32 kernel (tile_tma.cuh, step2_tma.cu): each 64 x 8 (32 x 16, 40 x 12) tile of an
// instance arrives in shared memory with a two-site halo and its material ids through
// the instance's tensor maps, advances to t + 1 together with a one-site halo, then to
// t + 2, so the packed state crosses HBM once per two steps.  A persistent CTA walks the
// tile list with a grid stride, skipping tiles of finished instances, and issues the
// copies of its next tile as soon as phase 1 has read the stage.  The per-site arithmetic
// is the one-step kernel's (same bits).  An instance whose run ends at t + 1 takes only
// the first step (its state is not needed afterwards; its forces come from the
// accumulators).  Convergence exits need a decision between any two steps, so they keep
// the one-step kernel.
// ACC: the tile's instance accumulates at t or t + 1; without it no FP64 operation is
// compiled in (a run-time accumulation test per site let the compiler predicate the FP64
// conversions of the field triple into every site's update, and GB300's FP64 pipe made
// that the kernel's bottleneck).
using namespace tma_tile;

// Tensor maps of instance i (in the kernels' `maps`): maps[3 i + p] its state in buffer p,
// maps[3 i + 2] its ids.

// Source values of every instance at the launch's two times, once per launch (one thread
// per instance), so that no step-kernel thread evaluates them in FP64.
__global__ void k_batch_source(const InstDesc *__restrict__ desc, int n, const long long *__restrict__ t_in,
                               SrcPairF *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = source_pair_f(desc[i].src, *t_in);
}

// TWO: the instance runs both steps of the launch (the common case; a run that ends at t + 1
// takes phase 1 only, on the tile's own sites, straight to global memory).  ACC: the
// instance accumulates Fourier sums at t or t + 1.  Both are template parameters so that
// the common body carries no per-site branch on them.  c: the tile's record (shared
// memory, copied to registers here).
template <class G, int POL, bool ACC, bool TWO, class OnStageFree>
__device__ __forceinline__ void batch2_tile(const BatchArgs<float> &b, const TileCtx &c, long long t,
                                            const TileSmem &S, const SrcPairF &sp, OnStageFree on_stage_free) {
    const int nx = c.nx, ny = c.ny, x0 = c.x0, y0 = c.y0, pitch = c.pitch, kind = c.kind;
    const int ay0 = c.ay0, ay1 = c.ay1;
    const unsigned rthr = c.runaway;
    const size_t ps = (size_t)c.pstride;
    const long long acc_from = c.acc_from;
    const MatT<float> *smat = c.m;
    float *fout = b.fout + c.base;
    unsigned *err = b.err + c.inst;
    const InstDesc &d = b.inst[c.inst];  // read by the accumulation only
    const bool src0 = t >= 1 && kind != SRC_NONE, src1 = kind != SRC_NONE;
    const int ioff = x0 - 1 - id_box_x(x0);  // column of site x0 - 1 in the id box
    for (int k = threadIdx.x; k < G::IW * G::IH; k += NTH) {
        const int lx = k % G::IW, ly = k / G::IW, x = x0 - 1 + lx, y = y0 - 1 + ly;
        if (x < 0 || x >= nx || y < 0 || y >= ny) continue;
        const bool interior = lx >= 1 && lx <= G::KW && ly >= 1 && ly <= G::KH;
        if (!TWO && !interior) continue;
        Pop<float> q;
        pull_buf<G::RW, G::RH>(S.raw, nx, ny, x, y, lx + 3, ly + 1, q);
        if (x == 0 && src0) inject_source_t(kind, sp.g0, sp.inc0, q);
        const uint8_t id = S.ids[(ly + 1) * G::MW + lx + ioff];
        const size_t idx = (size_t)y * pitch + x;
        bool bad;
        if (ACC && interior && t >= acc_from && y >= ay0 && y <= ay1) {
            double f3[3];
            bad = update_site<POL, true>(q, smat[id], rthr, f3, nullptr);
            batch_acc(f3, b.slot, b.acc, d, idx, t);
        } else {
            bad = update_site<POL, true>(q, smat[id], rthr, nullptr, nullptr);
        }
        if (bad) atomicOr(err, kErrUnstable);
        if (TWO) {
            put_inter<G>(S.inter, ly, lx, q);
            S.inter_ids[ly * G::IW + lx] = id;
        } else {
            store_site(fout, ps, idx, q);
        }
    }
    __syncthreads();  // the stage is read
    if (threadIdx.x == 0) on_stage_free();
    if constexpr (TWO) {
        for (int k = threadIdx.x; k < G::KW * G::KH; k += NTH) {
            const int lx = k % G::KW, ly = k / G::KW, x = x0 + lx, y = y0 + ly;
            if (x >= nx || y >= ny) continue;
            Pop<float> q;
            pull_buf<G::IW, G::IH>(S.inter, nx, ny, x, y, lx + 1, ly + 1, q);
            if (x == 0 && src1) inject_source_t(kind, sp.g1, sp.inc1, q);
            const MatT<float> m = smat[S.inter_ids[(ly + 1) * G::IW + lx + 1]];
            const size_t idx = (size_t)y * pitch + x;
            bool bad;
            if (ACC && t + 1 >= acc_from && y >= ay0 && y <= ay1) {
                double f3[3];
                bad = update_site<POL, true>(q, m, rthr, f3, nullptr);
                batch_acc(f3, b.slot, b.acc, d, idx, t + 1);
            } else {
                bad = update_site<POL, true>(q, m, rthr, nullptr, nullptr);
            }
            if (bad) atomicOr(err, kErrUnstable);
            store_site(fout, ps, idx, q);
        }
    }
}

template <class G, int POL>
__global__ void __launch_bounds__(NTH, 3)
    k_batch_step2(const BatchArgs<float> b, const TileCtx *__restrict__ ctx, const SrcPairF *__restrict__ srcs,
                  const CUtensorMap *__restrict__ maps, int p, const long long *__restrict__ t_in,
                  long long *__restrict__ t_out) {
    extern __shared__ unsigned char sm_dyn[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(128) TileCtx sc[2];  // tile records, copied with their tiles' state
    __shared__ SrcPairF sp;
    __shared__ int s_next;
    const TileSmem S = carve<G>(sm_dyn);
    const long long t = *t_in;
    const int n = b.n_tiles;
    if (blockIdx.x == 0 && threadIdx.x == 0) *t_out = t + 2;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // Tiles are ordered by decreasing run length, so once one of a CTA's tiles has finished
    // all its later ones have: the next tile is the next grid-stride index if that runs.
    // Thread 0 owns the walk: it issues each tile's copies (state, ids and its 128-byte
    // record, on one mbarrier) and prefetches in registers what the next issue needs,
    // so no global load sits on the path from a tile's arrival to its phase 1.
    int cur = (int)blockIdx.x < n && t < ctx[blockIdx.x].steps ? (int)blockIdx.x : -1;
    SrcPairF nsp{0.f, 0.f, 0.f, 0.f};  // thread 0: source values of the tile issued last
    auto issue = [&](int j, int slot) {  // thread 0: the copies of tile j, record into sc[slot]
        const int4 h = reinterpret_cast<const int4 *>(ctx + j)[0];  // inst, x0, y0
        tmap_acquire(maps + 3 * h.x + p);
        tmap_acquire(maps + 3 * h.x + 2);
        mbar_arrive_expect_tx(&bar, G::STATE_BYTES + G::ID_BYTES + (unsigned)sizeof(TileCtx));
        tma_load_3d(S.stage, maps + 3 * h.x + p, h.y - 4, h.z - 2, 0, &bar);
        tma_load_2d(S.stage + G::OFF_IDS, maps + 3 * h.x + 2, id_box_x(h.y), h.z - 2, &bar);
        bulk_load(&sc[slot], ctx + j, (unsigned)sizeof(TileCtx), &bar);
        nsp = h.y == 0 ? srcs[h.x] : SrcPairF{0.f, 0.f, 0.f, 0.f};
    };
    if (threadIdx.x == 0 && cur >= 0) issue(cur, 0);
    unsigned phase = 0;
    for (int i = 0; cur >= 0; ++i) {  // uniform over the block
        const int slot = i & 1, cand = cur + (int)gridDim.x;
        // thread 0: the candidate next tile's run length, read here and used after phase 1
        long long cand_steps = 0;
        if (threadIdx.x == 0) {
            sp = nsp;
            if (cand < n) cand_steps = ctx[cand].steps;
        }
        const bool ok = mbar_wait(&bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {  // the tile's copies never completed: report, leave
            if (threadIdx.x == 0) atomicOr(b.err + ctx[cur].inst, kErrTimeout);  // sc[slot] never arrived
            return;
        }
        const TileCtx &c = sc[slot];
        auto on_stage_free = [&]() {  // thread 0, once phase 1 has read the stage
            const bool next = cand < n && t < cand_steps;
            s_next = next ? cand : -1;
            if (next) {
                fence_proxy_async_smem();
                issue(cand, slot ^ 1);
            }
        };
        const bool acc = t + 1 >= c.acc_from, two = t + 1 < c.steps;  // uniform over the block
        if (two) {
            if (acc)
                batch2_tile<G, POL, true, true>(b, c, t, S, sp, on_stage_free);
            else
                batch2_tile<G, POL, false, true>(b, c, t, S, sp, on_stage_free);
        } else {
            if (acc)
                batch2_tile<G, POL, true, false>(b, c, t, S, sp, on_stage_free);
            else
                batch2_tile<G, POL, false, false>(b, c, t, S, sp, on_stage_free);
        }
        __syncthreads();  // shared memory is free for the next tile; s_next is written
        cur = s_next;
    }
}

// After a step of time t (*t_next = t + 1): every instance at a period boundary compares
// its energy with the previous boundary's (Sec. III convergence criterion); once two
// successive changes are <= tol * W and at least min_periods - 1 periods have run, the
// instance runs one more period, with Fourier accumulation, and stops.
__global__ void k_batch_converge(InstDesc *desc, double *energy, double *prev, int *settled,
                                 const long long *__restrict__ t_next, double tol, int min_periods, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long t = *t_next - 1;
    InstDesc &d = desc[i];
    if (t <= 0 || t >= d.acc_from || (t % (long long)d.period) != 0) return;
    const double W = energy[i];
    energy[i] = 0.0;
    const double P = prev[i];
    const int s = (P > 0.0 && fabs(W - P) <= tol * W) ? settled[i] + 1 : 0;
    settled[i] = s;
    prev[i] = W;
    const long long periods_done = t / d.period;
    if (s >= 2 && periods_done + 1 >= min_periods) {
        d.acc_from = t + 1;
        d.steps = t + 1 + d.period;
    }
}

// Per-instance stress-tensor integral: block i reduces instance i's contour.
struct ContourDesc {
    int pt_base, npts, acc_base, pad;
    double scale, R, dl, F0, M0;
};

__device__ __forceinline__ double wsum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) k_batch_contour(const ContourDesc *__restrict__ cd,
                                                       const ContourPt *__restrict__ pts,
                                                       const double *__restrict__ acc, double *out) {
    const ContourDesc c = cd[blockIdx.x];
    const double *A = acc + 6 * (size_t)c.acc_base;
    double fx = 0.0, fy = 0.0, mz = 0.0;
    for (int k = threadIdx.x; k < c.npts; k += blockDim.x) {
        const ContourPt p = pts[c.pt_base + k];
        double v[6] = {0, 0, 0, 0, 0, 0};
        for (int q = 0; q < 4; ++q)
            for (int j = 0; j < 6; ++j) v[j] += p.w[q] * A[6 * (size_t)p.s[q] + j];
        for (int j = 0; j < 6; ++j) v[j] *= c.scale;
        const double e2 = v[0] * v[0] + v[1] * v[1];
        const double hx2 = v[2] * v[2] + v[3] * v[3];
        const double hy2 = v[4] * v[4] + v[5] * v[5];
        const double tr = 0.5 * (e2 + hx2 + hy2);
        const double txx = 0.5 * (hx2 - tr), tyy = 0.5 * (hy2 - tr);
        const double txy = 0.5 * (v[2] * v[4] + v[3] * v[5]);
        const double tnx = txx * p.nx + txy * p.ny, tny = txy * p.nx + tyy * p.ny;
        fx += tnx;
        fy += tny;
        mz += c.R * (p.nx * tny - p.ny * tnx);
    }
    __shared__ double sh[3][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    fx = wsum(fx);
    fy = wsum(fy);
    mz = wsum(mz);
    if (lane == 0) {
        sh[0][wid] = fx;
        sh[1][wid] = fy;
        sh[2][wid] = mz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double F[3] = {0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int j = 0; j < 3; ++j) F[j] += sh[j][w];
        out[3 * blockIdx.x + 0] = F[0] * c.dl / c.F0;
        out[3 * blockIdx.x + 1] = F[1] * c.dl / c.F0;
        out[3 * blockIdx.x + 2] = F[2] * c.dl / c.M0;
    }
}

}  // namespace lbmem

struct lbm_em_batch {
    int dev = 0, n = 0, prec = LBM_EM_F32, sms = 0;
    int pol = POL_TM;  // polarization of every instance (lbm_em_batch_opts.polarization)
    size_t elem = 4;
    cudaStream_t stream = nullptr, cap = nullptr;
    bool own_stream = false;
    std::vector<lbm_em_instance> specs;
    std::vector<InstDesc> desc;
    std::vector<long long> order;  // instance indices by decreasing steps
    long long max_steps = 0;
    void *buf[2] = {nullptr, nullptr};
    size_t buf_elems = 0, mat_bytes = 0, slot_elems = 0, acc_slots = 0;
    uint8_t *d_mat = nullptr;
    int *d_slot = nullptr;
    double *d_acc = nullptr, *d_out = nullptr;
    double2 *d_cs = nullptr;
    InstDesc *d_desc = nullptr;
    Tile *d_tiles = nullptr;
    int n_tiles = 0;
    ContourDesc *d_cdesc = nullptr;
    ContourPt *d_pts = nullptr;
    long long *d_time = nullptr;
    unsigned *d_err = nullptr;
    int tile_w = 0, tile_h = 0, ctas = 0;
    bool two = false;  // two steps per launch (FP32, fixed run lengths; TMA-staged 64 x 8, 32 x 16 or 40 x 12 tiles)
    // FP32, per tile shape of the two-step kernel (0: GeoWide, 1: GeoTall, 2: GeoMid): per
    // instance, tensor maps of its state in buffer 0 and 1 and of its ids; resident CTAs per SM
    CUtensorMap *d_maps[3] = {nullptr, nullptr, nullptr};
    TileCtx *d_ctx = nullptr;       // FP32: one record per tile of the tile list
    SrcPairF *d_srcs = nullptr;     // FP32: per instance, the source values of the current launch
    int two_ctas[3] = {0, 0, 0};
    // four steps per launch (FP32, fixed run lengths): row-streaming kernel over work units
    // (instance, strip, row segment of four_seg rows), per-instance records, tensor maps and
    // source parameters, and the source values of the current launch
    bool four = false;
    int four_seg = 0, four_grid = 0, four_blocks = 0, four_ctas = 0, n_units = 0;
    int4 *d_units = nullptr;
    StreamInst *d_sinsts = nullptr;
    SourceParams *d_srcp = nullptr;
    SrcLevels *d_srcs4 = nullptr;
    CUtensorMap *d_smaps4 = nullptr;
    float *d_stage4 = nullptr;  // staged stencil fields of the accumulating launches (12 per slot)
    int *d_slot_inst = nullptr; // each accumulator slot's instance
    int want_spl = 0;  // lbm_em_batch_opts.steps_per_launch
    cudaGraphExec_t graph = nullptr;
    bool ran = false;
    // a bounded wait for a tile copy gave up (seen by lbm_em_batch_results): a copy may
    // still have been in flight when its CTA left, so the batch refuses further runs
    bool timed_out = false;
    // convergence exits
    double conv_tol = 0.0;
    int min_periods = 1;
    double *d_energy = nullptr, *d_prev = nullptr;
    int *d_settled = nullptr;
};

static void batch_free(lbm_em_batch *b) {
    if (!b) return;
    cudaSetDevice(b->dev);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    dfree(b->buf[0]);
    dfree(b->buf[1]);
    dfree(b->d_mat);
    dfree(b->d_slot);
    dfree(b->d_acc);
    dfree(b->d_out);
    dfree(b->d_cs);
    dfree(b->d_desc);
    dfree(b->d_tiles);
    dfree(b->d_cdesc);
    dfree(b->d_pts);
    dfree(b->d_time);
    dfree(b->d_err);
    dfree(b->d_energy);
    dfree(b->d_prev);
    dfree(b->d_settled);
    for (CUtensorMap *m : b->d_maps) dfree(m);
    dfree(b->d_ctx);
    dfree(b->d_srcs);
    dfree(b->d_units);
    dfree(b->d_sinsts);
    dfree(b->d_srcp);
    dfree(b->d_srcs4);
    dfree(b->d_smaps4);
    dfree(b->d_stage4);
    dfree(b->d_slot_inst);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

static lbm_em_status batch_tiles(lbm_em_batch *b, int tw, int th) {
    std::vector<Tile> tiles;
    for (long long ii : b->order) {
        const int i = (int)ii;
        const InstDesc &d = b->desc[i];
        for (int y0 = 0; y0 < d.ny; y0 += th)
            for (int x0 = 0; x0 < d.nx; x0 += tw) tiles.push_back(Tile{i, x0, y0, 0});
    }
    dfree(b->d_tiles);
    b->d_tiles = nullptr;
    lbm_em_status st = cuda_status(dmalloc(&b->d_tiles, tiles.size() * sizeof(Tile)), "cudaMalloc(tiles)");
    if (!st)
        st = cuda_status(copy_async(b->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice,
                                         b->stream),
                         "uploading tiles");
    b->n_tiles = (int)tiles.size();
    b->tile_w = tw;
    b->tile_h = th;
    if (!st && b->two) {  // the two-step kernel's per-tile records (set b->two first)
        std::vector<TileCtx> ctx(tiles.size());
        for (size_t k = 0; k < tiles.size(); ++k) {
            const Tile &tl = tiles[k];
            const InstDesc &d = b->desc[tl.inst];
            TileCtx &c = ctx[k];
            std::memset(&c, 0, sizeof(c));
            c.inst = tl.inst, c.x0 = tl.x0, c.y0 = tl.y0, c.nx = d.nx;
            c.ny = d.ny, c.pitch = d.pitch, c.kind = d.src.kind, c.ay0 = d.y0, c.ay1 = d.y1;
            c.runaway = runaway_bits<float>(b->specs[tl.inst].E0);
            c.base = (long long)d.base, c.pstride = (long long)d.pstride, c.steps = d.steps, c.acc_from = d.acc_from;
            for (int r = 0; r < 3; ++r) c.m[r] = d.mtabf[r];
        }
        dfree(b->d_ctx);
        b->d_ctx = nullptr;
        st = cuda_status(dmalloc(&b->d_ctx, ctx.size() * sizeof(TileCtx)), "cudaMalloc(tile records)");
        if (!st)
            st = cuda_status(copy_async(b->d_ctx, ctx.data(), ctx.size() * sizeof(TileCtx),
                                             cudaMemcpyHostToDevice, b->stream),
                             "uploading tile records");  // pageable: staged before the call returns
    }
    return st;
}

// The four-step kernel's work units for row segments of `seg` rows: instance by decreasing run
// length, then segment, then strip (neighbouring strips run side by side and share their halo
// columns in L2); and the per-instance records with that segment height.
static lbm_em_status batch_units(lbm_em_batch *b, int seg) {
    std::vector<int4> units;
    std::vector<StreamInst> si(b->n);
    for (int i = 0; i < b->n; ++i) {
        const InstDesc &d = b->desc[i];
        StreamInst &r = si[i];
        std::memset(&r, 0, sizeof(r));
        r.nx = d.nx, r.ny = d.ny, r.pitch = d.pitch, r.kind = d.src.kind;
        r.seg_rows = seg, r.n_strips = (d.nx + kStreamOutW - 1) / kStreamOutW, r.ay0 = d.y0, r.ay1 = d.y1;
        r.steps = d.steps, r.acc_from = d.acc_from, r.base = (long long)d.base, r.pstride = (long long)d.pstride;
        r.slot_base = (long long)d.slot_base, r.acc_base = d.acc_base, r.period = d.period;
        r.cs = d.src.cs;
        r.runaway = runaway_bits<float>(b->specs[i].E0);
        for (int q = 0; q < 3; ++q) r.m[q] = d.mtabf[q];
    }
    for (long long ii : b->order) {
        const int i = (int)ii;
        for (int y = 0; y < b->desc[i].ny; y += seg)
            for (int st = 0; st < si[i].n_strips; ++st) units.push_back(make_int4(i, st, y / seg, 0));
    }
    dfree(b->d_units);
    b->d_units = nullptr;
    lbm_em_status st = cuda_status(dmalloc(&b->d_units, units.size() * sizeof(int4)), "cudaMalloc(units)");
    if (!st)
        st = cuda_status(copy_async(b->d_units, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                    b->stream),
                         "uploading units");
    if (!st && !b->d_sinsts)
        st = cuda_status(dmalloc(&b->d_sinsts, si.size() * sizeof(StreamInst)), "cudaMalloc(stream records)");
    if (!st)
        st = cuda_status(copy_async(b->d_sinsts, si.data(), si.size() * sizeof(StreamInst), cudaMemcpyHostToDevice,
                                    b->stream),
                         "uploading stream records");
    if (!st) st = cuda_status(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");  // pageable sources
    b->n_units = (int)units.size();
    b->four_seg = seg;
    // one warp per unit: the hardware starts each thread block as an earlier one finishes, which
    // balanced the units better than resident warps walking them (256-instance design map on
    // GB300: 116.7 against 105.4 cells/s, same bits)
    b->four_blocks = b->four_ctas > 0 ? b->four_ctas * b->sms : (b->n_units + kStreamWarps - 1) / kStreamWarps;
    return st;
}

// log2 of a power of two, -1 for any other width.
static int ilog2(int v) {
    int l = 0;
    while ((1 << (l + 1)) <= v) ++l;
    return (1 << l) == v ? l : -1;
}

// Staircase Janus disc of every instance into the packed material ids (Sec. II).
static cudaError_t batch_rasterize(lbm_em_batch *b) {
    for (int i = 0; i < b->n; ++i) {
        const InstDesc &d = b->desc[i];
        const lbm_em_janus &j = b->specs[i].janus;
        double cx, cy;
        janus_center(&j, d.nx, d.ny, &cx, &cy);
        cudaError_t e = launch_rasterize(d.nx, d.ny, d.pitch, cx, cy, j.a, -std::sin(j.phi0), -std::cos(j.phi0),
                                         b->d_mat + d.mat_base, b->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The two-step kernel of the batch's tile shape and polarization.
template <int POL>
static void launch_batch_step2(const lbm_em_batch *b, const BatchArgs<float> &a, int grid, int p, cudaStream_t s) {
    if (b->tile_w == GeoWide::KW)
        k_batch_step2<GeoWide, POL><<<grid, NTH, GeoWide::kSmemBytes, s>>>(a, b->d_ctx, b->d_srcs, b->d_maps[0], p,
                                                                           b->d_time + p, b->d_time + (1 - p));
    else if (b->tile_w == GeoTall::KW)
        k_batch_step2<GeoTall, POL><<<grid, NTH, GeoTall::kSmemBytes, s>>>(a, b->d_ctx, b->d_srcs, b->d_maps[1], p,
                                                                           b->d_time + p, b->d_time + (1 - p));
    else
        k_batch_step2<GeoMid, POL><<<grid, NTH, GeoMid::kSmemBytes, s>>>(a, b->d_ctx, b->d_srcs, b->d_maps[2], p,
                                                                         b->d_time + p, b->d_time + (1 - p));
}

// One launch from the state in buf[p] (time word p) to buf[1 - p]: one step, or two with
// b->two.  The caller alternates p launch by launch.
static cudaError_t batch_launch(lbm_em_batch *b, cudaStream_t s, int p) {
    const int grid = b->ctas * b->sms;
    if (b->prec == LBM_EM_F32X2) {
        BatchArgs<df> a{b->d_desc, b->d_tiles, b->n_tiles, b->tile_w, b->tile_h, ilog2(b->tile_w),
                        (const df *)b->buf[p], (df *)b->buf[1 - p], b->d_mat, b->d_slot,
                        b->d_acc, b->d_err, b->d_energy, b->conv_tol > 0.0};
        if (b->pol == POL_TE)
            k_batch_step<df, POL_TE><<<grid, 256, 0, s>>>(a, b->d_time + p, b->d_time + (1 - p));
        else
            k_batch_step<df, POL_TM><<<grid, 256, 0, s>>>(a, b->d_time + p, b->d_time + (1 - p));
    } else if (b->prec == LBM_EM_F64) {
        BatchArgs<double> a{b->d_desc, b->d_tiles, b->n_tiles, b->tile_w, b->tile_h, ilog2(b->tile_w),
                            (const double *)b->buf[p], (double *)b->buf[1 - p], b->d_mat, b->d_slot,
                            b->d_acc, b->d_err, b->d_energy, b->conv_tol > 0.0};
        if (b->pol == POL_TE)
            k_batch_step<double, POL_TE><<<grid, 256, 0, s>>>(a, b->d_time + p, b->d_time + (1 - p));
        else
            k_batch_step<double, POL_TM><<<grid, 256, 0, s>>>(a, b->d_time + p, b->d_time + (1 - p));
    } else {
        BatchArgs<float> a{b->d_desc, b->d_tiles, b->n_tiles, b->tile_w, b->tile_h, ilog2(b->tile_w),
                           (const float *)b->buf[p], (float *)b->buf[1 - p], b->d_mat, b->d_slot,
                           b->d_acc, b->d_err, b->d_energy, b->conv_tol > 0.0};
        if (b->four) {
            launch_batch_step4(b->d_sinsts, b->d_srcp, b->n, b->d_units, b->n_units, b->d_srcs4, b->d_smaps4, p,
                               (float *)b->buf[1 - p], b->d_slot, b->d_acc, b->d_stage4, b->d_slot_inst,
                               (int)b->acc_slots, b->d_err, b->d_time + p, b->d_time + (1 - p), b->four_blocks,
                               b->pol, s);
        } else if (b->two) {
            k_batch_source<<<(b->n + 127) / 128, 128, 0, s>>>(b->d_desc, b->n, b->d_time + p, b->d_srcs);
            if (b->pol == POL_TE)
                launch_batch_step2<POL_TE>(b, a, grid, p, s);
            else
                launch_batch_step2<POL_TM>(b, a, grid, p, s);
        }
        else if (b->pol == POL_TE)
            k_batch_step<float, POL_TE><<<grid, 256, 0, s>>>(a, b->d_time + p, b->d_time + (1 - p));
        else
            k_batch_step<float, POL_TM><<<grid, 256, 0, s>>>(a, b->d_time + p, b->d_time + (1 - p));
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && b->conv_tol > 0.0) {
        k_batch_converge<<<(b->n + 127) / 128, 128, 0, s>>>(b->d_desc, b->d_energy, b->d_prev, b->d_settled,
                                                           b->d_time + (1 - p), b->conv_tol, b->min_periods, b->n);
        e = cudaGetLastError();
    }
    return e;
}

// A single step with the one-step kernel (the tail of a multi-step run).
static cudaError_t batch_launch_one(lbm_em_batch *b, cudaStream_t s, int p) {
    const bool two = b->two, four = b->four;
    b->two = false;
    b->four = false;
    cudaError_t e = batch_launch(b, s, p);
    b->two = two;
    b->four = four;
    return e;
}

// Steps one launch of the batch's configuration advances.
static int batch_spl(const lbm_em_batch *b) { return b->four ? 4 : b->two ? 2 : 1; }

static lbm_em_status batch_clear(lbm_em_batch *b) {
    lbm_em_status st = cuda_status(cudaMemsetAsync(b->buf[0], 0, b->buf_elems * b->elem, b->stream), "clear");
    if (!st) st = cuda_status(cudaMemsetAsync(b->d_acc, 0, b->acc_slots * 6 * sizeof(double), b->stream), "clear");
    if (!st) st = cuda_status(cudaMemsetAsync(b->d_time, 0, 2 * sizeof(long long), b->stream), "clear");
    if (!st) st = cuda_status(cudaMemsetAsync(b->d_err, 0, b->n * sizeof(unsigned), b->stream), "clear");
    if (!st) st = cuda_status(cudaMemsetAsync(b->d_energy, 0, b->n * sizeof(double), b->stream), "clear");
    if (!st) st = cuda_status(cudaMemsetAsync(b->d_prev, 0, b->n * sizeof(double), b->stream), "clear");
    if (!st) st = cuda_status(cudaMemsetAsync(b->d_settled, 0, b->n * sizeof(int), b->stream), "clear");
    // run lengths may have been shortened on the device by a convergence exit
    if (!st)
        st = cuda_status(copy_async(b->d_desc, b->desc.data(), b->n * sizeof(InstDesc), cudaMemcpyHostToDevice,
                                         b->stream),
                         "restoring descriptors");
    if (!st) st = cuda_status(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    return st;
}

// Time a few steps of each (tile shape, CTAs per SM, steps per launch) candidate from the
// cleared state.  FP32 runs of fixed length also have the two-step kernel (TMA-staged 64 x 8,
// 32 x 16 and 40 x 12 tiles, as many CTAs per SM as their shared memory allows) and the
// four-step row-streaming kernel (row segments of 64, 128 or 256 rows; its runs end with
// one-step launches on 64 x 4 tiles).  lbm_em_batch_opts.steps_per_launch restricts the
// candidates to one kind; a pinned tile shape or CTA count to the matching ones.
static lbm_em_status batch_autotune(lbm_em_batch *b, int want_w, int want_h, int want_c) {
    struct Cand {
        int w, h, c, spl, seg;
    };
    std::vector<Cand> cands;
    const bool pinned = want_w || want_h || want_c;
    const bool multi = b->prec == LBM_EM_F32 && b->conv_tol <= 0.0;
    if (multi && b->four_grid > 0 && ((b->want_spl == 0 && !pinned) || b->want_spl == 4))
        for (int seg : {64, 128, 256}) cands.push_back(Cand{64, 4, 4, 4, seg});
    const int two_shapes[3][2] = {{GeoWide::KW, GeoWide::KH}, {GeoTall::KW, GeoTall::KH}, {GeoMid::KW, GeoMid::KH}};
    for (int g = 0; g < 3; ++g) {
        const int w = two_shapes[g][0], h = two_shapes[g][1], c = b->two_ctas[g];
        if (c > 0 && multi && (b->want_spl == 0 || b->want_spl == 2) && (!want_w || want_w == w) &&
            (!want_h || want_h == h) && (!want_c || want_c == c))
            cands.push_back(Cand{w, h, c, 2, 0});
    }
    // One step per launch moves twice the bytes per update; on GB300 it lost to every two-step
    // shape on every FP32 map measured, so with nothing pinned by the caller only the multi-step
    // candidates are timed when they apply (they do not for FP64, double-float or convergence exits).
    const bool only_multi = !cands.empty() && !pinned && b->want_spl != 1;
    const int shapes[][2] = {{32, 8}, {64, 4}, {128, 2}, {256, 1}, {64, 8}, {128, 4}, {256, 2}, {128, 8}, {256, 4}};
    const int ctas[] = {2, 4, 8};
    if (b->want_spl == 0 || b->want_spl == 1)
        for (auto &sh : shapes)
            for (int c : ctas) {
                if (only_multi) break;
                if (want_w && sh[0] != want_w) continue;
                if (want_h && sh[1] != want_h) continue;
                if (want_c && c != want_c) continue;
                cands.push_back(Cand{sh[0], sh[1], c, 1, 0});
            }
    if (cands.empty()) cands.push_back(Cand{want_w ? want_w : 64, want_h ? want_h : 4, want_c ? want_c : 4, 1, 0});
    auto apply = [&](const Cand &c) {
        b->ctas = c.c;
        b->two = c.spl == 2;
        b->four = c.spl == 4;
        lbm_em_status st = batch_tiles(b, c.w, c.h);
        if (!st && b->four) st = batch_units(b, c.seg);
        return st;
    };
    if (cands.size() == 1) return apply(cands[0]);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Cand bc = cands[0];
    const int trial = 8;  // steps timed per candidate
    lbm_em_status st = LBM_EM_OK;
    for (const Cand &c : cands) {
        st = apply(c);
        if (st) break;
        st = batch_clear(b);
        if (st) break;
        const int launches = trial / c.spl;
        cudaError_t e = batch_launch(b, b->stream, 0);  // warm-up
        cudaEventRecord(e0, b->stream);
        for (int k = 1; k <= launches && e == cudaSuccess; ++k) e = batch_launch(b, b->stream, k & 1);
        cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        st = cuda_status(e, "autotune launch");
        if (st) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            bc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    st = apply(bc);
    if (!st) st = batch_clear(b);
    return st;
}

extern "C" {

lbm_em_status lbm_em_batch_create(const lbm_em_instance *specs, int32_t n, const lbm_em_batch_opts *o,
                                  lbm_em_batch_t **out) {
    if (!specs || n <= 0 || !o || !out) return set_error(LBM_EM_EINVAL, "bad batch arguments");
    *out = nullptr;
    if (o->precision != LBM_EM_F32 && o->precision != LBM_EM_F64 && o->precision != LBM_EM_F32X2)
        return set_error(LBM_EM_EINVAL, "batch precision must be LBM_EM_F32, LBM_EM_F64 or LBM_EM_F32X2");
    if (o->tile_w < 0 || o->tile_h < 0 || o->ctas_per_sm < 0 || o->ctas_per_sm > 8)
        return set_error(LBM_EM_EINVAL, "bad tile shape or CTAs per SM");
    if (o->tile_w && o->tile_w != 32 && o->tile_w != 40 && o->tile_w != 64 && o->tile_w != 128 && o->tile_w != 256)
        return set_error(LBM_EM_EINVAL, "tile_w must be 32, 40, 64, 128 or 256");
    if (o->tile_w == 40 && (o->precision != LBM_EM_F32 || o->conv_tol > 0.0 || (o->tile_h && o->tile_h != 12)))
        return set_error(LBM_EM_EINVAL, "tile_w 40 is the two-step kernel's 40 x 12 tile (FP32, conv_tol 0)");
    if (!(o->conv_tol >= 0.0) || o->min_periods < 0) return set_error(LBM_EM_EINVAL, "conv_tol >= 0, min_periods >= 0");
    if (o->polarization != 0 && o->polarization != 1)
        return set_error(LBM_EM_EINVAL, "polarization must be 0 (TM^z) or 1 (TE^z)");
    if (o->tile_h && (o->tile_h > 16)) return set_error(LBM_EM_EINVAL, "tile_h must be <= 16");
    if (o->steps_per_launch != 0 && o->steps_per_launch != 1 && o->steps_per_launch != 2 && o->steps_per_launch != 4)
        return set_error(LBM_EM_EINVAL, "steps_per_launch must be 0, 1, 2 or 4");
    if ((o->steps_per_launch == 2 || o->steps_per_launch == 4) && (o->precision != LBM_EM_F32 || o->conv_tol > 0.0))
        return set_error(LBM_EM_EINVAL, "two and four steps per launch are for LBM_EM_F32 without convergence exits");
    if (o->steps_per_launch == 4 && (o->tile_w || o->tile_h))
        return set_error(LBM_EM_EINVAL, "four steps per launch take no tile shape");
    for (int i = 0; i < n; ++i) {
        const lbm_em_instance &s = specs[i];
        if (s.nx < 4 || s.ny < 4 || s.period_steps < 4 || s.periods < 1 || s.ramp_steps < 0 || !std::isfinite(s.E0))
            return set_error(LBM_EM_EINVAL, "bad instance " + std::to_string(i));
        lbm_em_status st = check_janus(&s.janus);
        if (st) return st;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_error(LBM_EM_ECUDA, "no CUDA device available (the solver has no CPU path)");
    }
    lbm_em_batch *b = new lbm_em_batch();
    cudaGetDevice(&b->dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev);
    b->n = n;
    b->prec = o->precision;
    b->pol = o->polarization == 1 ? POL_TE : POL_TM;
    b->elem = b->prec == LBM_EM_F32 ? 4 : 8;
    b->specs.assign(specs, specs + n);
    lbm_em_status st = LBM_EM_OK;
#define BTRY(call, what)            \
    do {                            \
        st = cuda_status(call, what); \
        if (st) {                   \
            batch_free(b);          \
            return st;              \
        }                           \
    } while (0)
    if (o->stream) {
        b->stream = (cudaStream_t)o->stream;
    } else {
        BTRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        b->own_stream = true;
    }
    BTRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    // layout.  Contours, incident-wave constants and phase tables depend only on the lattice
    // size, the contour and the period; the instances of a design map mostly share them, so
    // each distinct one is built once (per instance they cost 0.5 s per 4096 instances).
    std::vector<ContourHost> uniq;  // distinct contours
    std::vector<int> cid(n);        // instance -> its contour in uniq
    std::map<std::tuple<int, int, double, double, double, int, double, double>, int> contour_ids;
    std::map<std::pair<int, double>, std::array<double, 4>> incident;  // (period, E0) -> P, P w
    std::map<int, size_t> cs_at;    // period -> offset of its phase table in cs_all
    std::vector<double2> cs_all;
    std::vector<size_t> cs_off(n);
    b->desc.resize(n);
    size_t base = 0, mat = 0, slot = 0, accs = 0;
    for (int i = 0; i < n; ++i) {
        const lbm_em_instance &s = specs[i];
        InstDesc &d = b->desc[i];
        std::memset(&d, 0, sizeof(d));
        d.nx = s.nx;
        d.ny = s.ny;
        d.pitch = round_up(s.nx, 32);
        d.period = s.period_steps;
        d.pstride = (size_t)d.pitch * s.ny;
        d.base = base;
        d.mat_base = mat;
        d.slot_base = slot;
        base += (size_t)NPLANES * d.pstride;
        mat += d.pstride;
        slot += d.pstride;
        d.steps = (long long)s.periods * s.period_steps;
        d.acc_from = d.steps - s.period_steps;
        b->max_steps = std::max(b->max_steps, d.steps);
        lbm_em_contour c{std::nan(""), std::nan(""), s.contour_radius, s.n_points, 0, s.janus.a};
        if (!std::isnan(s.janus.cx)) c.cx = s.janus.cx;
        if (!std::isnan(s.janus.cy)) c.cy = s.janus.cy;
        // NaN (the lattice centre) gets a sentinel: NaN keys would compare equal to anything
        const auto key = std::make_tuple(s.nx, s.ny, std::isnan(c.cx) ? -1e300 : c.cx, std::isnan(c.cy) ? -1e300 : c.cy,
                                         c.radius, c.n_points, c.a, s.E0);
        auto found = contour_ids.find(key);
        if (found == contour_ids.end()) {
            ContourHost C;
            C.E0 = s.E0;
            st = build_contour(s.nx, s.ny, &c, &C);
            if (st) {
                batch_free(b);
                return set_error(st, "instance " + std::to_string(i) + ": " + g_last_error);
            }
            found = contour_ids.emplace(key, (int)uniq.size()).first;
            uniq.push_back(std::move(C));
        }
        cid[i] = found->second;
        const ContourHost &C = uniq[cid[i]];
        d.acc_base = (int)accs;
        accs += C.n_slots;
        d.y0 = C.y0;
        d.y1 = C.y1;
        d.runaway = b->prec == LBM_EM_F64 ? runaway_bits<double>(s.E0) : runaway_bits<float>(s.E0);
        d.src.kind = o->source_kind;
        d.src.period = s.period_steps;
        d.src.ramp = s.ramp_steps;
        auto inc = incident.find({s.period_steps, s.E0});
        if (inc == incident.end()) {
            std::array<double, 4> v;
            incident_constants(s.period_steps, s.E0, &v[0], &v[1], &v[2], &v[3]);
            inc = incident.emplace(std::make_pair(s.period_steps, s.E0), v).first;
        }
        d.src.pr = inc->second[0], d.src.pi = inc->second[1], d.src.qr = inc->second[2], d.src.qi = inc->second[3];
        auto at = cs_at.find(s.period_steps);
        if (at == cs_at.end()) {
            at = cs_at.emplace(s.period_steps, cs_all.size()).first;
            std::vector<double2> cs = phase_table(s.period_steps);
            cs_all.insert(cs_all.end(), cs.begin(), cs.end());
        }
        cs_off[i] = at->second;
        const double eps[3] = {1.0, s.janus.eps1, s.janus.pec2 ? 0.0 : s.janus.eps2};
        for (int r = 0; r < 3; ++r) {
            const bool pec = r == 2 && s.janus.pec2;
            double *e = d.mtab[r];
            if (b->prec == LBM_EM_F32) {
                const MatT<float> m = material_entry<float>(eps[r], pec);
                e[0] = m.inv_eps3, e[1] = m.c_d, e[2] = m.inv_eps, e[3] = m.c3;
                d.mtabf[r] = m;
            } else {
                const MatT<double> m = material_entry<double>(eps[r], pec);
                e[0] = m.inv_eps3, e[1] = m.c_d, e[2] = m.inv_eps, e[3] = m.c3;
            }
        }
    }
    b->buf_elems = base;
    b->mat_bytes = mat;
    b->slot_elems = slot;
    b->acc_slots = accs;
    BTRY(dmalloc(&b->buf[0], base * b->elem), "cudaMalloc(batch distributions)");
    BTRY(dmalloc(&b->buf[1], base * b->elem), "cudaMalloc(batch distributions)");
    BTRY(dmalloc(&b->d_mat, mat), "cudaMalloc(batch materials)");
    BTRY(dmalloc(&b->d_slot, slot * sizeof(int)), "cudaMalloc(batch slots)");
    BTRY(dmalloc(&b->d_acc, std::max<size_t>(accs, 1) * 6 * sizeof(double)), "cudaMalloc(batch acc)");
    BTRY(dmalloc(&b->d_out, (size_t)n * 3 * sizeof(double)), "cudaMalloc(batch out)");
    BTRY(dmalloc(&b->d_cs, cs_all.size() * sizeof(double2)), "cudaMalloc(batch phases)");
    BTRY(dmalloc(&b->d_desc, n * sizeof(InstDesc)), "cudaMalloc(batch desc)");
    BTRY(dmalloc(&b->d_time, 2 * sizeof(long long)), "cudaMalloc(time)");
    BTRY(dmalloc(&b->d_err, n * sizeof(unsigned)), "cudaMalloc(err)");
    BTRY(dmalloc(&b->d_energy, n * sizeof(double)), "cudaMalloc(energy)");
    BTRY(dmalloc(&b->d_prev, n * sizeof(double)), "cudaMalloc(energy)");
    BTRY(dmalloc(&b->d_settled, n * sizeof(int)), "cudaMalloc(energy)");
    b->conv_tol = o->conv_tol;
    b->min_periods = o->min_periods > 0 ? o->min_periods : 1;
    b->want_spl = o->steps_per_launch;
    BTRY(copy_async(b->d_cs, cs_all.data(), cs_all.size() * sizeof(double2), cudaMemcpyHostToDevice, b->stream), "upload");
    for (int i = 0; i < n; ++i) b->desc[i].src.cs = b->d_cs + cs_off[i];
    BTRY(copy_async(b->d_desc, b->desc.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice, b->stream), "upload");
    // slot maps, contour points and per-instance contour descriptors
    {
        std::vector<int> smap(slot, -1);
        std::vector<ContourPt> pts;  // each distinct contour's points once, shared by its instances
        std::vector<int> pts_at(uniq.size(), -1);
        std::vector<ContourDesc> cd(n);
        for (int i = 0; i < n; ++i) {
            const InstDesc &d = b->desc[i];
            const ContourHost &C = uniq[cid[i]];
            for (int s = 0; s < C.n_slots; ++s)
                smap[d.slot_base + (size_t)C.site_xy[2 * s + 1] * d.pitch + C.site_xy[2 * s]] = s;
            if (pts_at[cid[i]] < 0) {
                pts_at[cid[i]] = (int)pts.size();
                pts.insert(pts.end(), C.pts.begin(), C.pts.end());
            }
            cd[i] = ContourDesc{pts_at[cid[i]], (int)C.pts.size(), d.acc_base, 0,
                                2.0 / (double)specs[i].period_steps, C.R, C.dl, C.F0, C.M0};
        }
        BTRY(copy_async(b->d_slot, smap.data(), slot * sizeof(int), cudaMemcpyHostToDevice, b->stream), "upload slots");
        BTRY(dmalloc(&b->d_pts, pts.size() * sizeof(ContourPt)), "cudaMalloc(points)");
        BTRY(copy_async(b->d_pts, pts.data(), pts.size() * sizeof(ContourPt), cudaMemcpyHostToDevice, b->stream), "upload");
        BTRY(dmalloc(&b->d_cdesc, n * sizeof(ContourDesc)), "cudaMalloc(contour desc)");
        BTRY(copy_async(b->d_cdesc, cd.data(), n * sizeof(ContourDesc), cudaMemcpyHostToDevice, b->stream), "upload");
    }
    // FP32: tensor maps of every instance for the two-step kernel, for both tile shapes
    if (b->prec == LBM_EM_F32) {
        const void *kern[3] = {(const void *)k_batch_step2<GeoWide, POL_TM>, (const void *)k_batch_step2<GeoTall, POL_TM>,
                               (const void *)k_batch_step2<GeoMid, POL_TM>};
        const void *kern_te[3] = {(const void *)k_batch_step2<GeoWide, POL_TE>,
                                  (const void *)k_batch_step2<GeoTall, POL_TE>, (const void *)k_batch_step2<GeoMid, POL_TE>};
        const size_t smem[3] = {GeoWide::kSmemBytes, GeoTall::kSmemBytes, GeoMid::kSmemBytes};
        const int shape[3][2] = {{GeoWide::KW, GeoWide::KH}, {GeoTall::KW, GeoTall::KH}, {GeoMid::KW, GeoMid::KH}};
        for (int g = 0; g < 3; ++g) {
            int per_sm = 0;
            BTRY(cudaFuncSetAttribute(kern[g], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem[g]),
                 "configuring the two-step batch kernel");
            BTRY(cudaFuncSetAttribute(kern_te[g], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem[g]),
                 "configuring the two-step batch kernel");
            BTRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[g], NTH, smem[g]),
                 "occupancy of the two-step batch kernel");
            std::vector<CUtensorMap> maps(3 * (size_t)n);
            for (int i = 0; i < n; ++i) {
                const InstDesc &d = b->desc[i];
                for (int q = 0; q < 2; ++q)
                    BTRY(encode_plane_map(&maps[3 * i + q], (const float *)b->buf[q] + d.base, d.nx, d.ny, d.pitch,
                                          d.pstride, shape[g][0], shape[g][1]),
                         "encoding an instance's tensor map");
                BTRY(encode_id_map(&maps[3 * i + 2], b->d_mat + d.mat_base, d.nx, d.ny, d.pitch, shape[g][0],
                                   shape[g][1]),
                     "encoding an instance's id map");
            }
            BTRY(dmalloc(&b->d_maps[g], maps.size() * sizeof(CUtensorMap)), "cudaMalloc(tensor maps)");
            BTRY(copy_async(b->d_maps[g], maps.data(), maps.size() * sizeof(CUtensorMap),
                                 cudaMemcpyHostToDevice, b->stream),
                 "upload");
            b->two_ctas[g] = per_sm;
        }
        BTRY(dmalloc(&b->d_srcs, (size_t)n * sizeof(SrcPairF)), "cudaMalloc(source values)");
        // the four-step kernel: per instance the three tensor maps of its rows, its source
        // parameters, room for a launch's source values
        if (o->conv_tol <= 0.0 && (o->steps_per_launch == 0 || o->steps_per_launch == 4)) {
            int warps = 0;
            BTRY(batch_stream_prepare(&warps), "configuring the four-step batch kernel");
            b->four_grid = warps / kStreamWarps;  // resident blocks (reported per SM)
            if (o->steps_per_launch == 4 && o->ctas_per_sm > b->four_grid / b->sms) {
                batch_free(b);
                return set_error(LBM_EM_EINVAL, "four steps per launch: ctas_per_sm at most " +
                                                    std::to_string(b->four_grid / b->sms));
            }
            if (o->steps_per_launch == 4) b->four_ctas = o->ctas_per_sm;
            std::vector<CUtensorMap> maps(3 * (size_t)n);
            std::vector<SourceParams> sp(n);
            for (int i = 0; i < n; ++i) {
                const InstDesc &d = b->desc[i];
                BTRY(encode_batch_stream_maps(&maps[3 * i], (const float *)b->buf[0] + d.base,
                                              (const float *)b->buf[1] + d.base, b->d_mat + d.mat_base, d.nx, d.ny,
                                              d.pitch, d.pstride),
                     "encoding an instance's row maps");
                sp[i] = d.src;
            }
            BTRY(dmalloc(&b->d_smaps4, maps.size() * sizeof(CUtensorMap)), "cudaMalloc(row maps)");
            BTRY(copy_async(b->d_smaps4, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                            b->stream),
                 "upload");
            BTRY(dmalloc(&b->d_srcp, (size_t)n * sizeof(SourceParams)), "cudaMalloc(source parameters)");
            BTRY(copy_async(b->d_srcp, sp.data(), sp.size() * sizeof(SourceParams), cudaMemcpyHostToDevice, b->stream),
                 "upload");
            BTRY(dmalloc(&b->d_srcs4, (size_t)n * sizeof(SrcLevels)), "cudaMalloc(source values)");
            // the accumulating launches' staged fields (12 floats per stencil slot) and each
            // slot's instance, for the flush that adds them to the Fourier sums
            if (accs > 0) {
                std::vector<int> owner(accs);
                for (int i = 0; i < n; ++i) {
                    const size_t end = i + 1 < n ? (size_t)b->desc[i + 1].acc_base : accs;
                    for (size_t q = (size_t)b->desc[i].acc_base; q < end; ++q) owner[q] = i;
                }
                BTRY(dmalloc(&b->d_stage4, accs * 12 * sizeof(float)), "cudaMalloc(accumulation stage)");
                BTRY(dmalloc(&b->d_slot_inst, accs * sizeof(int)), "cudaMalloc(slot instances)");
                BTRY(copy_async(b->d_slot_inst, owner.data(), accs * sizeof(int), cudaMemcpyHostToDevice, b->stream),
                     "upload");
                BTRY(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");  // pageable source
            }
        }
    }
    // rasterise every instance on the device (again at every run)
    BTRY(batch_rasterize(b), "rasterise");
    // run order: decreasing number of steps
    b->order.resize(n);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](long long x, long long y) { return b->desc[x].steps > b->desc[y].steps; });
    st = batch_autotune(b, o->tile_w, o->tile_h, o->ctas_per_sm);
    if (!st) st = cuda_status(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (st) {
        batch_free(b);
        return st;
    }
#undef BTRY
    *out = b;
    return LBM_EM_OK;
}

lbm_em_status lbm_em_batch_run(lbm_em_batch_t *b) {
    if (!b) return set_error(LBM_EM_EINVAL, "batch is NULL");
    if (b->timed_out)
        return set_error(LBM_EM_ESTATE, "a tile copy timed out in this batch: destroy it and create a new one");
    cudaSetDevice(b->dev);
    // every run starts from the cleared state, the first one too: a batch whose tuning had a
    // single candidate has never cleared its buffers, which hold what freed allocations left
    lbm_em_status st = batch_clear(b);
    if (!st) st = cuda_status(batch_rasterize(b), "rasterise");
    if (st) return st;
    if (!b->graph) {
        cudaGraph_t g = nullptr;
        st = cuda_status(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        if (st) return st;
        cudaError_t e = batch_launch(b, b->cap, 0);
        if (e == cudaSuccess) e = batch_launch(b, b->cap, 1);
        cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_status(e != cudaSuccess ? e : e2, "capturing the batch graph");
        }
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        st = cuda_status(e, "cudaGraphInstantiate");
        if (st) return st;
    }
    // the graph holds two launches (state buf[0] -> buf[1] -> buf[0]) of spl steps each; the
    // tail runs at most one more multi-step launch and then one-step launches
    const long long spl = batch_spl(b), per_graph = 2 * spl;
    long long t = 0;
    int p = 0;
    while (t + per_graph <= b->max_steps) {
        st = cuda_status(cudaGraphLaunch(b->graph, b->stream), "cudaGraphLaunch");
        if (st) return st;
        t += per_graph;
    }
    if (spl > 1 && t + spl <= b->max_steps) {
        st = cuda_status(batch_launch(b, b->stream, p), "batch step");
        if (st) return st;
        p ^= 1;
        t += spl;
    }
    while (t < b->max_steps) {
        st = cuda_status(batch_launch_one(b, b->stream, p), "batch step");
        if (st) return st;
        p ^= 1;
        ++t;
    }
    k_batch_contour<<<b->n, 256, 0, b->stream>>>(b->d_cdesc, b->d_pts, b->d_acc, b->d_out);
    st = cuda_status(cudaGetLastError(), "batch contour");
    b->ran = true;
    return st;
}

lbm_em_status lbm_em_batch_results(lbm_em_batch_t *b, double *out, int32_t *status) {
    if (!b) return set_error(LBM_EM_EINVAL, "batch is NULL");
    if (!b->ran) return set_error(LBM_EM_ESTATE, "batch has not run");
    cudaSetDevice(b->dev);
    std::vector<double> res((size_t)b->n * 3);
    std::vector<unsigned> err(b->n);
    lbm_em_status st = cuda_status(
        copy_async(res.data(), b->d_out, res.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "read");
    if (!st)
        st = cuda_status(copy_async(err.data(), b->d_err, err.size() * sizeof(unsigned), cudaMemcpyDeviceToHost,
                                         b->stream),
                         "read");
    if (!st) st = cuda_status(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (st) return st;
    if (out) std::memcpy(out, res.data(), res.size() * sizeof(double));
    bool any = false, timeout = false;
    for (int i = 0; i < b->n; ++i) {
        if (status) status[i] = (err[i] & kErrTimeout) ? LBM_EM_ETIMEOUT : err[i] ? LBM_EM_EUNSTABLE : LBM_EM_OK;
        any |= err[i] != 0;
        timeout |= (err[i] & kErrTimeout) != 0;
    }
    if (timeout) {
        b->timed_out = true;
        return set_error(LBM_EM_ETIMEOUT, "a bounded wait for a tile load gave up");
    }
    if (any) return set_error(LBM_EM_EUNSTABLE, "at least one instance became unstable");
    return LBM_EM_OK;
}

lbm_em_status lbm_em_batch_steps(lbm_em_batch_t *b, int64_t *steps) {
    if (!b || !steps) return set_error(LBM_EM_EINVAL, "NULL argument");
    if (!b->ran) return set_error(LBM_EM_ESTATE, "batch has not run");
    cudaSetDevice(b->dev);
    std::vector<InstDesc> d(b->n);
    lbm_em_status st = cuda_status(
        copy_async(d.data(), b->d_desc, b->n * sizeof(InstDesc), cudaMemcpyDeviceToHost, b->stream), "read");
    if (!st) st = cuda_status(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (st) return st;
    for (int i = 0; i < b->n; ++i) steps[i] = d[i].steps;
    return LBM_EM_OK;
}

lbm_em_status lbm_em_batch_config(lbm_em_batch_t *b, int32_t *tile_w, int32_t *tile_h, int32_t *ctas_per_sm) {
    if (!b) return set_error(LBM_EM_EINVAL, "batch is NULL");
    if (b->four) {  // the four-step kernel: strips of 56 output columns, row segments, its blocks per SM
        if (tile_w) *tile_w = kStreamOutW;
        if (tile_h) *tile_h = b->four_seg;
        if (ctas_per_sm) *ctas_per_sm = b->four_ctas > 0 ? b->four_ctas : b->four_grid / b->sms;
        return LBM_EM_OK;
    }
    if (tile_w) *tile_w = b->tile_w;
    if (tile_h) *tile_h = b->tile_h;
    if (ctas_per_sm) *ctas_per_sm = b->ctas;
    return LBM_EM_OK;
}

lbm_em_status lbm_em_batch_steps_per_launch(lbm_em_batch_t *b, int32_t *n) {
    if (!b || !n) return set_error(LBM_EM_EINVAL, "NULL argument");
    *n = batch_spl(b);
    return LBM_EM_OK;
}

lbm_em_status lbm_em_batch_destroy(lbm_em_batch_t *b) {
    batch_free(b);
    return LBM_EM_OK;
}

}  // extern "C"
